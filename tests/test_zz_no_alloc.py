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


def regular_onorm(n, c, start):
    """U = Onorm(start) through bsp_oi_track (t_max = 0) on a one-block path mesh."""
    ptr = np.array([0, n])
    h = bsp.bsp_mesh_create_edges(np.zeros((n, 3)), synth.path_edges(n), ptr, np.arange(n),
                                  np.array([-1]),
                                  bsp.make_opts(precision=bsp.BSP_PREC_F32, rayleigh_ritz=0))
    try:
        bsp.bsp_oi_track(h, c, 0, start)
        return bsp.bsp_get_basis(h, 0, n).astype(np.float64)
    finally:
        bsp.bsp_mesh_destroy(h)


# 1,024 and 144 rows (torus tiles), 2,048 (the documented maximum: 256 rows per
# panel), 1,001 (not a multiple of the 8 panels), 1 column
@pytest.mark.parametrize("n,c", [(1024, 64), (144, 12), (2048, 64), (1001, 40), (300, 1)])
@pytest.mark.parametrize("in_place", [False, True])
def test_noalloc_matches_regular_entry_point(n, c, in_place):
    ptr = np.array([0, n])
    start = synth.gaussian_starts(ptr, np.array([-1]), c, seed=7).astype(np.float32)
    U_ref = regular_onorm(n, c, start)
    for call in range(2):
        Y = torch.tensor(start, device="cuda")
        Q = Y if in_place else torch.full_like(Y, float("nan"))
        bsp.bsp_onorm_noalloc(Y, Q, n, c)
        torch.cuda.synchronize()
        Qh = Q.cpu().double().numpy()
        assert np.abs(Qh - U_ref).max() <= TOL, (call, np.abs(Qh - U_ref).max())
        assert np.abs(Qh.T @ Qh - np.eye(c)).max() <= TOL


def test_noalloc_on_a_side_stream_orders_after_the_producer():
    n, c = 1024, 32
    start = synth.gaussian_starts(np.array([0, n]), np.array([-1]), c, seed=3).astype(np.float32)
    U_ref = regular_onorm(n, c, start)
    s = torch.cuda.Stream()
    host = torch.tensor(start).pin_memory()
    with torch.cuda.stream(s):
        Y = torch.empty(n, c, device="cuda")
        Y.copy_(host, non_blocking=True)       # written on s
        Q = torch.empty_like(Y)
        bsp.bsp_onorm_noalloc(Y, Q, n, c)      # stream=None: runs on s, after the copy
    s.synchronize()
    assert np.abs(Q.cpu().double().numpy() - U_ref).max() <= TOL


def test_noalloc_rejects_oversized_blocks():
    Y = torch.zeros(4096, 8, device="cuda")
    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_onorm_noalloc(Y, Y, 4096, 8)
    assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
    Y = torch.zeros(256, 80, device="cuda")
    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_onorm_noalloc(Y, Y, 256, 80)
    assert ei.value.code == bsp.BSP_ERR_INVALID_ARG


def test_noalloc_rejects_host_buffers():
    """Host memory never reaches the kernel: the library checks the pointers first."""
    Y = np.ones((256, 8), np.float32)
    Q = np.zeros((256, 8), np.float32)
    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_onorm_noalloc(Y, Q, 256, 8)
    assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
    assert np.all(Q == 0)
    with pytest.raises(ValueError):          # a CPU tensor is refused by the binding
        bsp.bsp_onorm_noalloc(torch.ones(256, 8), torch.zeros(256, 8), 256, 8)


def test_noalloc_rank_deficient_input_reports_numerical():
    n, c = 512, 16
    Y = torch.tensor(synth.gaussian_starts(np.array([0, n]), np.array([-1]), c, seed=2)
                     .astype(np.float32), device="cuda")
    Y[:, 5] = 0.0                            # a zero column: the Gram is singular
    Q = torch.empty_like(Y)
    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_onorm_noalloc(Y, Q, n, c)
    assert ei.value.code == bsp.BSP_ERR_NUMERICAL
    # the next regular call on the shared scratch is unaffected
    start = synth.gaussian_starts(np.array([0, n]), np.array([-1]), c, seed=4).astype(np.float32)
    Y2 = torch.tensor(start, device="cuda")
    bsp.bsp_onorm_noalloc(Y2, Q, n, c)
    torch.cuda.synchronize()
    assert np.abs(Q.cpu().double().numpy() - regular_onorm(n, c, start)).max() <= TOL
