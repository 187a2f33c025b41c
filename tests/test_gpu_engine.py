"""The persistent cluster engine of the fixed-c schedule, through the C ABI.

Every block's solves and CholeskyQR2 run in one launch (one cluster of
ceil(c / 4) CTAs per dependency path).  Its bases must match the FP64 oracle's
OI (Sec. 4, Algorithm 1, warm start from the parent) at the FP32 gates, agree
with the per-wave schedule, replay bit for bit from the captured graph, and a
withheld parent flag must end in BSP_ERR_TIMEOUT without hanging.
"""
import numpy as np
import pytest

from oracle import bsp_oracle as O
from paper_1810_02719_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1810_02719_gb300 import bsp  # noqa: E402

SINE_F32, PROJ_F32 = 1e-4, 1e-5


def bases(h, om):
    return [bsp.bsp_get_basis(h, b, blk.verts.size, np.float32).astype(np.float64)
            for b, blk in enumerate(om.blocks)]


def worst(Ug, Ur, om, xyz):
    s = max(O.max_sine(u, r) for u, r in zip(Ug, Ur))
    p = max(O.projector_rel_error(u, r, xyz[blk.verts])
            for u, r, blk in zip(Ug, Ur, om.blocks))
    return s, p


def torus_chain(N, T, seed=0):
    xyz, faces = synth.torus(N, seed=seed)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(len(ptr) - 1)
    om = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    return xyz, faces, ptr, verts, parent, om


@pytest.mark.parametrize("c,t_max", [(64, 2), (48, 2), (32, 3), (12, 1), (5, 2), (1, 2)])
def test_engine_chain_matches_oracle_and_wave_schedule(c, t_max):
    """128^2 torus, 16 chained tiles of 32 x 32 (1,024 rows): widths from one CTA
    (c <= 4) to 16 CTAs, ragged c, the first-order and the full second pass."""
    xyz, faces, ptr, verts, parent, om = torus_chain(128, 32, seed=3)
    starts = synth.gaussian_starts(ptr, parent, c, seed=4)
    U_ref = O.oi_track(om, c, t_max, starts, delta=1e-2)
    out = {}
    for sched in (bsp.BSP_SCHED_AUTO, bsp.BSP_SCHED_WAVES):
        h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                                bsp.make_opts(precision=bsp.BSP_PREC_F32, schedule=sched))
        try:
            bsp.bsp_oi_track(h, c, t_max, starts.astype(np.float32))
            out[sched] = (bases(h, om), bsp.bsp_get_stats(h))
        finally:
            bsp.bsp_mesh_destroy(h)
    # c = 1 tracks the constant null vector: x ~ b / delta, so an FP32
    # residual b - A x is only known to u ||A|| ||x|| ~ u ||A|| ||b|| / delta, and
    # the error of x along u_1 is up to u ||A|| / (lambda_1 + delta) ~ 3.6e-5 on
    # these tiles (||A|| <= 12, lambda_1 ~ 0.0096): the projector gate is 5e-5.
    proj_tol = 5e-5 if c == 1 else PROJ_F32
    for sched, (Ug, st) in out.items():
        s, p = worst(Ug, U_ref, om, xyz)
        assert s <= SINE_F32 and p <= proj_tol, (sched, s, p)
        assert st["not_converged"] == 0
    # the engine is one launch for all 16 blocks (plus the batched Rayleigh-Ritz)
    assert out[bsp.BSP_SCHED_AUTO][1]["gpu_launches"] < out[bsp.BSP_SCHED_WAVES][1]["gpu_launches"]
    s, p = worst(out[bsp.BSP_SCHED_AUTO][0], out[bsp.BSP_SCHED_WAVES][0], om, xyz)
    assert s <= SINE_F32 and p <= 2 * proj_tol


@pytest.mark.parametrize("z,c", [(1, 24), (2, 16), (1, 64)])
def test_engine_forest_several_clusters_row_transfer(z, c):
    """Uneven BFS blocks (<= 1,024 rows) in a forest with 3 roots: several
    clusters, ready flags between them, row-transferred starts, z solves per step."""
    N = 72
    xyz, faces = synth.torus(N, seed=6)
    ptr, verts = synth.bfs_partition(N, target_blocks=12, min_size=150, max_size=900, seed=7)
    ptr, verts, parent = synth.block_forest(ptr, verts, N, roots=3, seed=8)
    sizes = np.diff(ptr)
    assert sizes.max() <= 1024 and len(set(sizes.tolist())) > 1
    assert np.sum(parent < 0) == 3
    om = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, c, seed=9)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F32, z=z))
    try:
        bsp.bsp_oi_track(h, c, 2, starts.astype(np.float32))
        st = bsp.bsp_get_stats(h)
        assert st["levels"] > 1 and st["not_converged"] == 0
        U_ref = O.oi_track(om, c, 2, starts, delta=1e-2, z=z)
        s, p = worst(bases(h, om), U_ref, om, xyz)
        assert s <= SINE_F32 and p <= PROJ_F32, (s, p)
    finally:
        bsp.bsp_mesh_destroy(h)


def test_engine_ranges_with_deferred_work_on_a_side_stream():
    """A chain of 256 blocks (256^2 torus, 16 x 16 tiles) takes the engine in
    consecutive ranges, each range's second CholeskyQR pass and Rayleigh-Ritz
    running beside the next range: same bases as the per-wave schedule and the
    oracle, bit-identical between the captured graph, its replay and the eager
    launches."""
    xyz, faces, ptr, verts, parent, om = torus_chain(256, 16, seed=5)
    assert len(ptr) - 1 == 256
    c, t_max = 16, 2
    starts = synth.gaussian_starts(ptr, parent, c, seed=6)
    U_ref = O.oi_track(om, c, t_max, starts, delta=1e-2)
    runs = {}
    for name, kw in [("graph", dict(schedule=bsp.BSP_SCHED_AUTO)),
                     ("eager", dict(schedule=bsp.BSP_SCHED_AUTO, use_graph=0)),
                     ("waves", dict(schedule=bsp.BSP_SCHED_WAVES))]:
        h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                                bsp.make_opts(precision=bsp.BSP_PREC_F32, **kw))
        try:
            bsp.bsp_oi_track(h, c, t_max, starts.astype(np.float32))
            runs[name] = bases(h, om)
            if name == "graph":
                bsp.bsp_oi_track(h, c, t_max, starts.astype(np.float32))
                assert all(np.array_equal(a, b) for a, b in zip(runs[name], bases(h, om)))
            assert bsp.bsp_get_stats(h)["not_converged"] == 0
        finally:
            bsp.bsp_mesh_destroy(h)
    assert all(np.array_equal(a, b) for a, b in zip(runs["graph"], runs["eager"]))
    for name in ("graph", "waves"):
        s, p = worst(runs[name], U_ref, om, xyz)
        assert s <= SINE_F32 and p <= PROJ_F32, (name, s, p)


def test_engine_graph_replay_is_deterministic_and_projects():
    xyz, faces, ptr, verts, parent, om = torus_chain(64, 32, seed=1)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F32))
    try:
        c = 64
        starts = synth.gaussian_starts(ptr, parent, c, seed=2).astype(np.float32)
        bsp.bsp_oi_track(h, c, 2, starts)
        U1 = [bsp.bsp_get_basis(h, b, 1024) for b in range(4)]
        bsp.bsp_oi_track(h, c, 2, starts)       # cached graph
        U2 = [bsp.bsp_get_basis(h, b, 1024) for b in range(4)]
        assert all(np.array_equal(a, b) for a, b in zip(U1, U2))
        # projection and reconstruction on the engine's bases equal the definition
        X = xyz.astype(np.float32)
        E = np.empty((4 * c, 3), np.float32)
        Xo = np.empty_like(X)
        bsp.bsp_project(h, X, bsp.BSP_DT_F32, 3, E)
        bsp.bsp_reconstruct(h, E, 3, Xo)
        for b, blk in enumerate(om.blocks):
            U = U2[b].astype(np.float64)
            Eb = U.T @ xyz[blk.verts]
            assert np.abs(E[b * c:(b + 1) * c] - Eb).max() <= 1e-4 * np.abs(Eb).max()
            assert np.abs(Xo[blk.verts] - U @ Eb).max() <= 1e-4
    finally:
        bsp.bsp_mesh_destroy(h)


def test_engine_withheld_flag_times_out_and_the_context_stays_usable():
    """A host-side hook makes block 3 wait for a flag that nothing sets: the
    bounded wait runs out (100 ms), the call returns BSP_ERR_TIMEOUT, and the
    next calls on the same device work."""
    xyz, faces, ptr, verts, parent, om = torus_chain(64, 16, seed=2)
    c = 16
    starts = synth.gaussian_starts(ptr, parent, c, seed=3)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F32, withhold_block=3,
                                          wait_limit_ms=100))
    try:
        for _ in range(2):
            with pytest.raises(bsp.BspError) as ei:
                bsp.bsp_oi_track(h, c, 2, starts.astype(np.float32))
            assert ei.value.code == bsp.BSP_ERR_TIMEOUT
    finally:
        bsp.bsp_mesh_destroy(h)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F32))
    try:
        bsp.bsp_oi_track(h, c, 2, starts.astype(np.float32))
        U_ref = O.oi_track(om, c, 2, starts, delta=1e-2)
        s, p = worst(bases(h, om), U_ref, om, xyz)
        assert s <= SINE_F32 and p <= PROJ_F32
    finally:
        bsp.bsp_mesh_destroy(h)
