"""The allocation-free orthonormalisation entry point, called through the C ABI.

Some callers may not allocate device memory while they run (a streaming
pipeline with a latency bound, or an application whose device memory belongs
to its own allocator).  bsp_onorm_noalloc serves them with a fixed static
scratch array; its result must equal the orthonormal basis that the regular
entry point bsp_oi_track produces for the same start matrix (t_max = 0 and no
Rayleigh-Ritz: U = Onorm(V0)), on consecutive calls.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

from paper_1810_02719_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1810_02719_gb300 import bsp  # noqa: E402

TOL = 1e-5   # the FP32 reconstruction/projector tolerance used by the parity tests


@pytest.mark.parametrize("N,c", [(32, 64), (16, 12)])
def test_noalloc_matches_regular_entry_point(N, c):
    xyz, faces = synth.torus(N, seed=5)
    ptr = np.array([0, N * N])
    verts = np.arange(N * N)
    parent = np.array([-1])
    start = synth.gaussian_starts(ptr, parent, c, seed=7).astype(np.float32)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F32, rayleigh_ritz=0))
    try:
        bsp.bsp_oi_track(h, c, 0, start)
        U_ref = bsp.bsp_get_basis(h, 0, N * N).astype(np.float64)
    finally:
        bsp.bsp_mesh_destroy(h)
    Y = torch.tensor(start, device="cuda")
    for call in range(2):
        Q = torch.full_like(Y, float("nan"))
        bsp.bsp_onorm_noalloc(Y, Q, N * N, c)
        torch.cuda.synchronize()
        Qh = Q.cpu().double().numpy()
        assert np.abs(Qh - U_ref).max() <= TOL, (call, np.abs(Qh - U_ref).max())
        assert np.abs(Qh.T @ Qh - np.eye(c)).max() <= TOL


def test_noalloc_rejects_oversized_blocks():
    Y = torch.zeros(4096, 8, device="cuda")
    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_onorm_noalloc(Y, Y, 4096, 8)
    assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
    Y = torch.zeros(256, 80, device="cuda")
    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_onorm_noalloc(Y, Y, 256, 80)
    assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
