"""The device-driven dynamic-c schedule (Sec. 5, Algorithm 2 over the block
forest of Sec. 4) through the C ABI.

The rounds are decided on the device.  With use_graph the whole call is one
CUDA graph with conditional nodes: a WHILE over rounds per wave and SWITCH
nodes over width classes.  Without it the host replays the same launches,
reading the control values back (the profiling path).  Both runs must give
the same widths, the same bases bit for bit, the same CG step counts and the
same number of kernel launches.  The test also checks a graph replay, a graph
rebuilt for new parameters, and the widths against the oracle.
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


def forest_case(N=96, roots=3, seed=2):
    """Uneven BFS blocks of a 96^2 torus in a 3-root forest: several waves of
    several blocks, children starting at their parents' widths."""
    xyz, faces = synth.torus(N, seed=seed)
    ptr, verts = synth.bfs_partition(N, target_blocks=30, min_size=150, max_size=900, seed=11)
    ptr, verts, parent = synth.block_forest(ptr, verts, N, roots=roots, seed=1)
    return xyz, faces, ptr, verts, parent


def run(xyz, faces, ptr, verts, parent, prec, use_graph, tol, profiling=False, reps=1,
        c_min=8, c_max=64, t_max=2, seed=5):
    real = np.float64 if prec == bsp.BSP_PREC_F64 else np.float32
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=prec, use_graph=use_graph,
                                          cg_rtol=1e-12 if real == np.float64 else 1e-6))
    try:
        if profiling:
            bsp.bsp_set_profiling(h, True)
        k = len(ptr) - 1
        starts = synth.gaussian_starts(ptr, parent, c_min, seed=3).astype(real)
        out = []
        for _ in range(reps):
            cb = np.empty(k, np.int32)
            bsp.bsp_oi_track_dynamic(h, xyz.astype(real), tol, c_min, c_max, 8, t_max, seed,
                                     starts, None, cb)
            U = [bsp.bsp_get_basis(h, b, int(ptr[b + 1] - ptr[b]), real) for b in range(k)]
            out.append((cb, U, bsp.bsp_get_stats(h)))
        return out
    finally:
        bsp.bsp_mesh_destroy(h)


@pytest.mark.parametrize("prec", [bsp.BSP_PREC_MIXED, bsp.BSP_PREC_F64])
def test_graph_and_eager_schedules_agree(prec):
    xyz, faces, ptr, verts, parent = forest_case()
    (cg, Ug, sg), = run(xyz, faces, ptr, verts, parent, prec, 1, 1e-2)
    (ce, Ue, se), = run(xyz, faces, ptr, verts, parent, prec, 0, 1e-2)
    assert len(set(cg.tolist())) > 2, cg            # widths vary: several rounds ran
    assert np.array_equal(cg, ce)
    for b in range(len(cg)):
        assert Ug[b].shape == Ue[b].shape and np.array_equal(Ug[b], Ue[b]), b
    assert sg["cg_steps_total"] == se["cg_steps_total"]
    assert sg["gpu_launches"] == se["gpu_launches"] > 0


def test_graph_replay_and_rebuild():
    """A second call replays the cached graph (same results); new parameters
    rebuild it (results equal to the host-driven replay of those parameters);
    profiling takes the host-driven path with the same results."""
    xyz, faces, ptr, verts, parent = forest_case()
    prec = bsp.BSP_PREC_MIXED
    r = run(xyz, faces, ptr, verts, parent, prec, 1, 1e-2, reps=2)
    assert np.array_equal(r[0][0], r[1][0])
    assert all(np.array_equal(a, b) for a, b in zip(r[0][1], r[1][1]))
    assert r[0][2]["gpu_launches"] == r[1][2]["gpu_launches"]
    # new tolerance and width range through the same mesh handle
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent, bsp.make_opts(precision=prec))
    try:
        k = len(ptr) - 1
        starts = synth.gaussian_starts(ptr, parent, 16, seed=3).astype(np.float32)
        starts8 = synth.gaussian_starts(ptr, parent, 8, seed=3).astype(np.float32)
        cb = np.empty(k, np.int32)
        bsp.bsp_oi_track_dynamic(h, xyz.astype(np.float32), 1e-2, 8, 64, 8, 2, 5, starts8, None, cb)
        assert np.array_equal(cb, r[0][0])
        bsp.bsp_oi_track_dynamic(h, xyz.astype(np.float32), 4e-3, 16, 96, 8, 2, 5, starts, None, cb)
        U1 = [bsp.bsp_get_basis(h, b, int(ptr[b + 1] - ptr[b]), np.float32) for b in range(k)]
        launches = bsp.bsp_get_stats(h)["gpu_launches"]
    finally:
        bsp.bsp_mesh_destroy(h)
    (ce, Ue, se), = run(xyz, faces, ptr, verts, parent, prec, 0, 4e-3, c_min=16, c_max=96)
    assert np.array_equal(cb, ce) and cb.max() > 16
    assert all(np.array_equal(a, b) for a, b in zip(U1, Ue))
    assert launches == se["gpu_launches"]
    (cp, Up, sp), = run(xyz, faces, ptr, verts, parent, prec, 1, 1e-2, profiling=True)
    assert np.array_equal(cp, r[0][0])
    assert all(np.array_equal(a, b) for a, b in zip(Up, r[0][1]))


def test_device_schedule_widths_match_oracle():
    """The graph-driven widths on a multi-wave forest equal the FP64 oracle's
    Algorithm 2 (FP64 path), and the bases match it as subspaces."""
    xyz, faces, ptr, verts, parent = forest_case()
    om = O.build_mesh(xyz.shape[0], ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, 8, seed=3)
    Ur, cr, *_ = O.oi_track_dynamic(om, xyz, starts, tol=1e-2, c_min=8, c_max=64, c_step=8,
                                    t_max=2, delta=1e-2, seed=5)
    (cg, Ug, _), = run(xyz, faces, ptr, verts, parent, bsp.BSP_PREC_F64, 1, 1e-2)
    assert np.array_equal(cg, cr), (cg, cr)
    for b in range(len(cg)):
        assert O.max_sine(Ug[b], Ur[b]) <= 1e-6, b
