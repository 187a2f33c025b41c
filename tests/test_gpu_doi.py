"""The paper's own dynamic OI (Sec. 5, Algorithm 2) on the GPU, through the C ABI.

One column at a time with two thresholds: every block's widths and iteration
counts must equal the oracle's (doi_paper_track), and the bases must match it
as subspaces at the FP64 and FP32 gates.  The workload (64^2 height field, 16
chained tiles of 16 x 16, c0 = 20, eps_l = 0.2, eps_h = 0.25, widths 4..24, at
most 5 iterations) makes blocks grow, shrink, stop and reach the iteration
cap; in the oracle's trace every ||e|| lies at least 0.38% (relative) from a
threshold, far beyond the FP32 error of ||e||, so the decisions are
comparable exactly.
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

C0, EPS_L, EPS_H, CMIN, CMAX, TCAP = 20, 0.2, 0.25, 4, 24, 5


def case():
    N, T = 64, 16
    xyz, faces = synth.grid_heightfield(N, seed=0)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(len(ptr) - 1)
    om = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, C0, seed=1)
    return xyz, faces, ptr, verts, parent, om, starts


@pytest.mark.parametrize("prec,real,sine_tol,proj_tol",
                         [(bsp.BSP_PREC_F64, np.float64, 1e-8, 1e-10),
                          (bsp.BSP_PREC_F32, np.float32, 1e-4, 1e-5),
                          (bsp.BSP_PREC_MIXED, np.float32, 1e-4, 1e-5)])
def test_paper_doi_matches_oracle(prec, real, sine_tol, proj_tol):
    xyz, faces, ptr, verts, parent, om, starts = case()
    U_ref, c_ref, it_ref = O.doi_paper_track(om, xyz, starts, C0, EPS_L, EPS_H, c_min=CMIN,
                                             c_max=CMAX, t_cap=TCAP)
    # the workload exercises every branch
    assert len(set(c_ref.tolist())) > 3 and (it_ref == TCAP).any() and (it_ref < TCAP).any()
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=prec,
                                          cg_rtol=1e-12 if real == np.float64 else 1e-6))
    try:
        c, its = bsp.bsp_oi_track_paper_doi(h, xyz.astype(real), C0, EPS_L, EPS_H, CMIN, CMAX,
                                            TCAP, starts.astype(real))
        assert c.tolist() == c_ref.tolist()
        assert its.tolist() == it_ref.tolist()
        worst_s = worst_p = 0.0
        for b, blk in enumerate(om.blocks):
            U = bsp.bsp_get_basis(h, b, blk.verts.size, real).astype(np.float64)
            assert U.shape[1] == c_ref[b]
            worst_s = max(worst_s, O.max_sine(U, U_ref[b]))
            worst_p = max(worst_p, O.projector_rel_error(U, U_ref[b], xyz[blk.verts]))
            assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 10 * sine_tol
        assert worst_s <= sine_tol and worst_p <= proj_tol, (worst_s, worst_p)
        # projection and reconstruction work on the variable widths
        E = np.empty((int(c.sum()), 3), real)
        Xo = np.empty((xyz.shape[0], 3), real)
        bsp.bsp_project(h, xyz.astype(real), bsp.BSP_DT_F64 if real == np.float64
                        else bsp.BSP_DT_F32, 3, E)
        bsp.bsp_reconstruct(h, E, 3, Xo)
        ref = O.reconstruct(om, U_ref, O.project(om, U_ref, xyz), 3)
        assert np.linalg.norm(Xo - ref) / np.linalg.norm(ref) <= proj_tol
    finally:
        bsp.bsp_mesh_destroy(h)


def test_paper_doi_rejects_bad_arguments():
    xyz, faces, ptr, verts, parent, om, starts = case()
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F32))
    try:
        X, V = xyz.astype(np.float32), starts.astype(np.float32)
        for args in [(C0, 0.3, 0.2, CMIN, CMAX, TCAP),     # eps_l > eps_h
                     (C0, 0.0, 0.2, CMIN, CMAX, TCAP),     # eps_l = 0
                     (2, EPS_L, EPS_H, CMIN, CMAX, TCAP),  # c0 < c_min
                     (C0, EPS_L, EPS_H, CMIN, 300, TCAP),  # c_max > 128
                     (C0, EPS_L, EPS_H, CMIN, CMAX, 0)]:   # t_cap = 0
            with pytest.raises(bsp.BspError) as ei:
                bsp.bsp_oi_track_paper_doi(h, X, *args[:6], V)
            assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
    finally:
        bsp.bsp_mesh_destroy(h)


@pytest.mark.parametrize("prec,real", [(bsp.BSP_PREC_MIXED, np.float32),
                                       (bsp.BSP_PREC_F64, np.float64)])
def test_paper_doi_graph_and_host_driven_agree(prec, real):
    """The iterations are decided on the device; the captured graph (WHILE over
    iterations, SWITCH over width classes) and the host-driven replay of the
    same launches give the same widths, iterations and bases bit for bit, and
    a second call replays the cached graph."""
    xyz, faces, ptr, verts, parent, om, starts = case()
    out = []
    for use_graph, reps in ((1, 2), (0, 1)):
        h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                                bsp.make_opts(precision=prec, use_graph=use_graph,
                                              cg_rtol=1e-12 if real == np.float64 else 1e-6))
        try:
            for _ in range(reps):
                c, its = bsp.bsp_oi_track_paper_doi(h, xyz.astype(real), C0, EPS_L, EPS_H, CMIN,
                                                    CMAX, TCAP, starts.astype(real))
                U = [bsp.bsp_get_basis(h, b, blk.verts.size) for b, blk in enumerate(om.blocks)]
                out.append((c.copy(), its.copy(), U, bsp.bsp_get_stats(h)["gpu_launches"]))
        finally:
            bsp.bsp_mesh_destroy(h)
    (c1, i1, U1, n1), (c2, i2, U2, n2), (c3, i3, U3, n3) = out
    for c, its, U, n in ((c2, i2, U2, n2), (c3, i3, U3, n3)):
        assert np.array_equal(c, c1) and np.array_equal(its, i1)
        assert all(np.array_equal(a, b) for a, b in zip(U, U1))
        assert n == n1 > 0
