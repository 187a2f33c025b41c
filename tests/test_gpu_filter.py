"""GPU adjoint of the block low-pass filter vs the FP64 oracle's autograd.

Gradients of loss = ||filter(x_noisy) - x_clean||^2 with respect to the
coordinates and to the per-edge weights, through t_max unrolled OI steps with
detached warm starts.  FP64 path: relative error <= 1e-7 (exact solves in the
oracle vs CG to 1e-13 on the GPU).  FP32 path: relative error <= 2e-3 (CG to
1e-6 and FP32 Onorm; the weight gradient sums products of differences of
neighbouring rows, which cancel to about 1e-3 of their size).
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
from paper_1810_02719_gb300.filter import block_low_pass  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_case(clean, noisy, faces, ptr, verts, parent, c, t, prec, rtol, seed=1):
    n = clean.shape[0]
    real = np.float64 if prec == bsp.BSP_PREC_F64 else np.float32
    tdt = torch.float64 if real == np.float64 else torch.float32
    om = O.build_mesh(n, ptr, verts, parent, faces=faces, weight_mode=O.WEIGHT_EDGE)
    E = sum(b.edges.shape[0] for b in om.blocks)
    rng = np.random.default_rng(seed)
    w = 1.0 + 0.25 * rng.random(E)
    starts = synth.gaussian_starts(ptr, parent, c, seed=seed + 1)
    loss_ref, gx_ref, gw_ref, xh_ref = O.filter_loss_grads(om, noisy, clean, w, c, t, starts)
    h = bsp.bsp_mesh_create(clean, faces, ptr, verts, parent,
                            bsp.make_opts(precision=prec, weight_mode=bsp.BSP_W_EDGE, cg_rtol=rtol))
    try:
        x = torch.tensor(noisy, dtype=tdt, device="cuda", requires_grad=True)
        wt = torch.tensor(w, dtype=tdt, device="cuda", requires_grad=True)
        V0 = torch.tensor(starts, dtype=tdt, device="cuda")
        y = block_low_pass(x, wt, h, c, t, V0)
        loss = ((y - torch.tensor(clean, dtype=tdt, device="cuda")) ** 2).sum()
        loss.backward()
        return (float(loss), loss_ref, y.detach().cpu().double().numpy(), xh_ref,
                x.grad.cpu().double().numpy(), gx_ref, wt.grad.cpu().double().numpy(), gw_ref)
    finally:
        bsp.bsp_mesh_destroy(h)


def test_filter_gradients_fp64_patch_2000v():
    """40 x 50 open patch of the noisy torus (2,000 v), 4 blocks of 20 x 25, c = 32, 4 steps."""
    clean, noisy, faces = synth.noisy_torus_patch(40, 50, N=512, seed=0)
    ptr, verts = synth.rect_partition(40, 50, 20, 25)
    parent = synth.raster_chain(4)
    L, Lr, y, yr, gx, gxr, gw, gwr = run_case(clean, noisy, faces, ptr, verts, parent, 32, 4,
                                              bsp.BSP_PREC_F64, 1e-13)
    assert L == pytest.approx(Lr, rel=1e-9)
    assert rel(y, yr) <= 1e-9
    assert rel(gx, gxr) <= 1e-7, rel(gx, gxr)
    assert rel(gw, gwr) <= 1e-7, rel(gw, gwr)


def test_filter_gradients_fp32_torus_tiles():
    """128 x 128 noisy torus, 16 blocks of 32 x 32, c = 32, 4 steps, FP32 path."""
    clean, noisy, faces = synth.noisy_torus(128, seed=2)
    ptr, verts = synth.tile_partition(128, 32)
    parent = synth.raster_chain(16)
    L, Lr, y, yr, gx, gxr, gw, gwr = run_case(clean, noisy, faces, ptr, verts, parent, 32, 4,
                                              bsp.BSP_PREC_F32, 1e-6)
    assert L == pytest.approx(Lr, rel=1e-4)
    assert rel(y, yr) <= 1e-5
    assert rel(gx, gxr) <= 2e-3, rel(gx, gxr)
    assert rel(gw, gwr) <= 2e-3, rel(gw, gwr)
    # element by element, against the largest entry of each gradient
    ex = float(np.abs(gx - gxr).max() / np.abs(gxr).max())
    ew = float(np.abs(gw - gwr).max() / np.abs(gwr).max())
    assert ex <= 5e-3 and ew <= 5e-3, (ex, ew)


def test_gradcheck_through_the_library():
    """torch.autograd.gradcheck of the library's forward/backward (FP64), all blocks roots."""
    clean, noisy, faces = synth.noisy_torus_patch(8, 12, N=64, seed=5)
    ptr, verts = synth.rect_partition(8, 12, 4, 6)
    parent = np.full(4, -1)
    om = O.build_mesh(96, ptr, verts, parent, faces=faces, weight_mode=O.WEIGHT_EDGE)
    E = sum(b.edges.shape[0] for b in om.blocks)
    h = bsp.bsp_mesh_create(clean, faces, ptr, verts, parent,
                            bsp.make_opts(precision=bsp.BSP_PREC_F64, weight_mode=bsp.BSP_W_EDGE,
                                          cg_rtol=1e-14))
    try:
        V0 = torch.tensor(synth.gaussian_starts(ptr, parent, 3, seed=6), dtype=torch.float64,
                          device="cuda")
        x = torch.tensor(noisy, dtype=torch.float64, device="cuda", requires_grad=True)
        w = torch.tensor(1.0 + 0.2 * np.random.default_rng(7).random(E), dtype=torch.float64,
                         device="cuda", requires_grad=True)
        f = lambda xx, ww: block_low_pass(xx, ww, h, 3, 2, V0)  # noqa: E731
        assert torch.autograd.gradcheck(f, (x, w), eps=1e-6, atol=1e-6, rtol=1e-5)
    finally:
        bsp.bsp_mesh_destroy(h)
