"""GPU codec (Sec. 7.1, Sec. 8) vs the oracle, through the C ABI.

Codes and quantiser ranges are integers and extreme values decided in the
coefficients' own precision on both sides: they must match bit for bit, and
so must the decoded coefficients (one rounding per operation on both sides).
The NMSVE is accumulated in FP64 on both sides in different orders: relative
tolerance 1e-10.
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


def tracked_mesh(N, T, c, prec, seed=0):
    xyz, faces = synth.torus(N, seed=seed)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(len(ptr) - 1)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent, bsp.make_opts(precision=prec))
    real = np.float64 if prec == bsp.BSP_PREC_F64 else np.float32
    starts = synth.gaussian_starts(ptr, parent, c, seed=seed).astype(real)
    bsp.bsp_oi_track(h, c, 2, starts)
    return h, xyz, faces, ptr, real


def split_rows(E, c_b):
    off = np.concatenate([[0], np.cumsum(c_b)])
    return [E[off[b]:off[b + 1]] for b in range(len(c_b))]


def synthetic_coefficients(c_b, cols, real, seed):
    """Coefficient-like data with the awkward cases mixed in: constant columns,
    an exactly representable grid, a column with a single non-zero, wide ranges."""
    rng = np.random.default_rng(seed)
    E = (rng.standard_normal((int(np.sum(c_b)), cols)) *
         rng.uniform(1e-3, 1e2, size=cols)).astype(real)
    E[:, 1] = real(0.75)
    E[:, 2] = (np.arange(E.shape[0]) % 7 * 0.25).astype(real)
    E[:, 3] = 0
    E[::5, 3] = real(-2.0)
    return E


@pytest.mark.parametrize("prec", [bsp.BSP_PREC_MIXED, bsp.BSP_PREC_F64])
def test_codes_ranges_and_decoding_bit_exact(prec):
    h, xyz, faces, ptr, real = tracked_mesh(64, 16, 12, prec)
    try:
        k = len(ptr) - 1
        c_b = bsp.bsp_get_block_c(h, k)
        # (a) projected coordinates, host buffers; (b) 600 wide columns on the
        # device (5 column CTAs, the last one ragged)
        E3 = np.empty((int(c_b.sum()), 3), real)
        bsp.bsp_project(h, xyz.astype(real), bsp.BSP_DT_F64 if real == np.float64 else
                        bsp.BSP_DT_F32, 3, E3)
        cases = [(E3, False), (synthetic_coefficients(c_b, 600, real, seed=1), True)]
        for E, on_device in cases:
            cols = E.shape[1]
            ref_blocks = split_rows(E, c_b)
            for bits in (1, 8, 12, 16):
                ref_codes, ref_ranges = O.quantize(ref_blocks, bits)
                ref_dec = O.dequantize(ref_codes, ref_ranges, bits, real)
                if on_device:
                    dE = torch.from_numpy(E).cuda()
                    dC = torch.empty(E.shape, dtype=torch.int16, device="cuda")
                    dR = torch.empty((k, cols, 2), dtype=dE.dtype, device="cuda")
                    bsp.bsp_quantize(h, dE, cols, bits, dC, dR)
                    dD = torch.empty_like(dE)
                    bsp.bsp_dequantize(h, dC, dR, cols, bits, dD)
                    codes = dC.cpu().numpy().view(np.uint16)
                    rng_ = dR.cpu().numpy()
                    dec = dD.cpu().numpy()
                else:
                    codes = np.empty(E.shape, np.uint16)
                    rng_ = np.empty((k, cols, 2), real)
                    bsp.bsp_quantize(h, E, cols, bits, codes, rng_)
                    dec = np.empty_like(E)
                    bsp.bsp_dequantize(h, codes, rng_, cols, bits, dec)
                assert np.array_equal(codes, np.concatenate(ref_codes)), (bits, cols)
                assert np.array_equal(rng_, np.stack(ref_ranges)), (bits, cols)
                assert np.array_equal(dec, np.concatenate(ref_dec)), (bits, cols)
            # bits per vertex: the paper's formula over the tracked c_b
            assert bsp.bsp_bits_per_vertex(h, 12) == pytest.approx(
                O.bits_per_vertex(c_b, xyz.shape[0], 12), rel=1e-15)
    finally:
        bsp.bsp_mesh_destroy(h)


def test_codec_argument_errors():
    xyz, faces = synth.torus(32)
    ptr, verts = synth.tile_partition(32, 16)
    parent = synth.raster_chain(len(ptr) - 1)
    h = bsp.bsp_mesh_create(xyz, faces, ptr, verts, parent, bsp.make_opts())
    try:
        E = np.zeros((4 * 8, 3), np.float32)
        codes = np.empty(E.shape, np.uint16)
        rng_ = np.empty((4, 3, 2), np.float32)
        with pytest.raises(bsp.BspError) as e:           # nothing tracked yet
            bsp.bsp_quantize(h, E, 3, 12, codes, rng_)
        assert e.value.code == bsp.BSP_ERR_INVALID_ARG
        starts = synth.gaussian_starts(ptr, parent, 8, seed=0).astype(np.float32)
        bsp.bsp_oi_track(h, 8, 1, starts)
        for bits in (0, 17):
            with pytest.raises(bsp.BspError) as e:
                bsp.bsp_quantize(h, E, 3, bits, codes, rng_)
            assert e.value.code == bsp.BSP_ERR_INVALID_ARG
            with pytest.raises(bsp.BspError):
                bsp.bsp_dequantize(h, codes, rng_, 3, bits, E)
        with pytest.raises(bsp.BspError):
            bsp.bsp_bits_per_vertex(h, 0)
    finally:
        bsp.bsp_mesh_destroy(h)


@pytest.mark.parametrize("real", [np.float32, np.float64])
def test_nmsve_matches_oracle(real):
    """NMSVE of the tracked reconstruction (coarse approximation) and of its 12-bit coded
    version, on a 128^2 torus (16,384 vertices, 16 blocks): GPU vs oracle."""
    prec = bsp.BSP_PREC_F64 if real == np.float64 else bsp.BSP_PREC_MIXED
    dt = bsp.BSP_DT_F64 if real == np.float64 else bsp.BSP_DT_F32
    h, xyz, faces, ptr, _ = tracked_mesh(128, 32, 16, prec, seed=2)
    try:
        n = xyz.shape[0]
        k = len(ptr) - 1
        X = xyz.astype(real)
        c_b = bsp.bsp_get_block_c(h, k)
        E = np.empty((int(c_b.sum()), 3), real)
        bsp.bsp_project(h, X, dt, 3, E)
        Xr = np.empty_like(X)
        bsp.bsp_reconstruct(h, E, 3, Xr)
        codes = np.empty(E.shape, np.uint16)
        rng_ = np.empty((k, 3, 2), real)
        bsp.bsp_quantize(h, E, 3, 12, codes, rng_)
        Eq = np.empty_like(E)
        bsp.bsp_dequantize(h, codes, rng_, 3, 12, Eq)
        Xq = np.empty_like(X)
        bsp.bsp_reconstruct(h, Eq, 3, Xq)
        # host inputs, then device inputs (faces too)
        got = [bsp.bsp_nmsve(X, Xr, dt, n, faces, len(faces)),
               bsp.bsp_nmsve(torch.from_numpy(X).cuda(), torch.from_numpy(Xq).cuda(), dt, n,
                             torch.from_numpy(faces).cuda(), len(faces))]
        refs = [O.nmsve(X, Xr, faces), O.nmsve(X, Xq, faces)]
        for g, r in zip(got, refs):
            assert np.allclose(g, r, rtol=1e-10, atol=0), (g, r)
        assert bsp.bsp_nmsve(X, X, dt, n, faces, len(faces))[0] == 0.0
    finally:
        bsp.bsp_mesh_destroy(h)


def test_nmsve_edge_cases():
    """Hand-worked triangles, an isolated vertex, repeated faces and a bad index."""
    tri = np.array([[0, 1, 2]], np.int32)
    X = np.array([[0, 0, 0], [3, 0, 0], [0, 4, 0], [7, 7, 7]], np.float64)
    Xr = np.array([[0, 0, 0], [5, 0, 0], [0, 12, 0], [7, 7, 8]], np.float64)
    got = bsp.bsp_nmsve(X, Xr, bsp.BSP_DT_F64, 4, tri, 1)
    assert np.allclose(got, O.nmsve(X, Xr, tri), rtol=1e-13)
    rep = np.concatenate([tri, tri[:, ::-1], tri]).astype(np.int32)
    assert np.allclose(bsp.bsp_nmsve(X, Xr, bsp.BSP_DT_F64, 4, rep, 3), got, rtol=1e-13)
    # no faces: only the coordinate term (every GL is the vertex itself)
    got0 = bsp.bsp_nmsve(X, Xr, bsp.BSP_DT_F64, 4, np.zeros((0, 3), np.int32), 0)
    assert np.allclose(got0, O.nmsve(X, Xr, np.zeros((0, 3), np.int64)), rtol=1e-13)
    bad = np.array([[0, 1, 4]], np.int32)
    with pytest.raises(bsp.BspError) as e:
        bsp.bsp_nmsve(X, Xr, bsp.BSP_DT_F64, 4, bad, 1)
    assert e.value.code == bsp.BSP_ERR_INVALID_ARG
    with pytest.raises(bsp.BspError):
        bsp.bsp_nmsve(X, Xr, bsp.BSP_DT_BF16, 4, tri, 1)
