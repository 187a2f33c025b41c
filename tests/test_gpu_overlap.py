"""Overlapped submeshes (Sec. 6.1, Algorithm 3) on the GPU, through the C ABI.

Parts that share vertices run as an expanded mesh (one vertex per part and
copy, each part's induced edges re-indexed); bsp_merge_overlapped then forms
every vertex's degree-weighted mean of its copies.  Checked against the
oracle's Algorithm 3 on arbitrary copy values, and end to end (tracking,
projection, reconstruction of the copies, merge) against the oracle's
overlapped reconstruction.
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


def overlapped_case(N=96, T=32, r=2, seed=3):
    xyz, faces = synth.torus(N, seed=seed)
    ptr, verts = synth.overlapped_tiles(N, T, r)
    k = len(ptr) - 1
    parent = synth.raster_chain(k)
    xptr, xverts, xedges, orig = synth.expand_overlapped(ptr, verts, faces)
    om = O.build_overlapped_mesh(N * N, ptr, verts, parent, faces=faces)
    return xyz, faces, ptr, verts, parent, xptr, xverts, xedges, orig, om


def make_expanded(xyz, xptr, xverts, xedges, orig, parent, prec):
    return bsp.bsp_mesh_create_edges(xyz[orig], xedges, xptr, xverts, parent,
                                     bsp.make_opts(precision=prec,
                                                   cg_rtol=1e-12 if prec == bsp.BSP_PREC_F64
                                                   else 1e-6))


@pytest.mark.parametrize("real,dt,tol", [(np.float64, bsp.BSP_DT_F64, 1e-13),
                                         (np.float32, bsp.BSP_DT_F32, 2e-6)])
def test_merge_equals_degree_weighted_average(real, dt, tol):
    """Arbitrary copy values (not reconstructions): the merge is exactly Algorithm 3."""
    xyz, faces, ptr, verts, parent, xptr, xverts, xedges, orig, om = overlapped_case()
    n = xyz.shape[0]
    h = make_expanded(xyz, xptr, xverts, xedges, orig, parent,
                      bsp.BSP_PREC_F64 if real == np.float64 else bsp.BSP_PREC_F32)
    try:
        rng = np.random.default_rng(0)
        Xc = rng.standard_normal((orig.size, 5)).astype(real)
        out = np.empty((n, 5), real)
        bsp.bsp_merge_overlapped(h, orig, n, Xc, dt, 5, out)
        # the oracle's Algorithm 3 on the same copies (part b's copies in part order)
        Xb = [Xc[xptr[b]:xptr[b + 1]].astype(np.float64) for b in range(len(ptr) - 1)]
        ref = O.weighted_average(om, Xb, 5)
        assert np.abs(out - ref).max() <= tol * np.abs(ref).max()
        # device buffers give the same bits
        Xd = torch.tensor(Xc, device="cuda")
        od = torch.empty((n, 5), dtype=Xd.dtype, device="cuda")
        bsp.bsp_merge_overlapped(h, torch.tensor(orig, device="cuda"), n, Xd, dt, 5, od)
        assert np.array_equal(od.cpu().numpy(), out)
    finally:
        bsp.bsp_mesh_destroy(h)


def test_vertices_without_copies_and_bad_indices():
    xyz, faces, ptr, verts, parent, xptr, xverts, xedges, orig, om = overlapped_case(N=64, T=32, r=1)
    n = xyz.shape[0]
    h = make_expanded(xyz, xptr, xverts, xedges, orig, parent, bsp.BSP_PREC_F64)
    try:
        Xc = np.ones((orig.size, 3))
        out = np.full((n + 7, 3), np.nan)
        bsp.bsp_merge_overlapped(h, orig, n + 7, Xc, bsp.BSP_DT_F64, 3, out)
        assert np.all(out[:n] == 1.0) and np.all(out[n:] == 0.0)   # 7 vertices in no part
        bad = orig.copy()
        bad[5] = n + 100
        with pytest.raises(bsp.BspError) as ei:
            bsp.bsp_merge_overlapped(h, bad, n, Xc, bsp.BSP_DT_F64, 3, out)
        assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
        with pytest.raises(bsp.BspError) as ei:
            bsp.bsp_merge_overlapped(h, orig, n, Xc, bsp.BSP_DT_BF16, 3, out)
        assert ei.value.code == bsp.BSP_ERR_INVALID_ARG
    finally:
        bsp.bsp_mesh_destroy(h)


@pytest.mark.parametrize("prec,real,tol", [(bsp.BSP_PREC_F64, np.float64, 1e-10),
                                           (bsp.BSP_PREC_F32, np.float32, 1e-5)])
def test_overlapped_reconstruction_matches_oracle(prec, real, tol):
    """Equal-size parts (36 x 36 tiles of a 96^2 torus, 2 rings of overlap) in a
    warm-start chain, c = 24, 2 steps: every part's copy U_b U_b^T X_b, merged."""
    xyz, faces, ptr, verts, parent, xptr, xverts, xedges, orig, om = overlapped_case()
    n, k, c = xyz.shape[0], len(ptr) - 1, 24
    starts = synth.gaussian_starts(xptr, parent, c, seed=5)
    h = make_expanded(xyz, xptr, xverts, xedges, orig, parent, prec)
    try:
        bsp.bsp_oi_track(h, c, 2, starts.astype(real))
        Xc = xyz[orig].astype(real)
        E = np.empty((k * c, 3), real)
        Xr = np.empty_like(Xc)
        bsp.bsp_project(h, Xc, bsp.BSP_DT_F64 if real == np.float64 else bsp.BSP_DT_F32, 3, E)
        bsp.bsp_reconstruct(h, E, 3, Xr)
        out = np.empty((n, 3), real)
        bsp.bsp_merge_overlapped(h, orig, n, Xr,
                                 bsp.BSP_DT_F64 if real == np.float64 else bsp.BSP_DT_F32, 3, out)
        U_ref = O.oi_track(om, c, 2, starts, delta=1e-2)
        ref = O.reconstruct_overlapped(om, U_ref, xyz)
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= tol, err
        # the merge differs from a plain scatter of one copy per vertex
        assert np.linalg.norm(ref - Xr[np.unique(orig, return_index=True)[1]]) > 0
    finally:
        bsp.bsp_mesh_destroy(h)
