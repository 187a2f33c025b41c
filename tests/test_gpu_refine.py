"""GPU fine denoising (Sec. 7.2) and normal-angle metric (Sec. 8) vs the oracle,
through the C ABI.

FP64: filtered normals and fitted positions within 1e-10 of the oracle (the
same operations; the kernel merges the two Gaussian factors into one exp and
sums rings in sorted face order).  FP32: positions within 2e-5 and normals
within 1e-4 (unit-length vectors from FP32 edge vectors of ~0.2 on a radius-1
torus: a few 1e-7 relative per rounding, through 3 filter passes and 5
fitting steps).  The metric accumulates in FP64: 1e-10 relative.
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


def mean_edge(X, faces):
    e = O.undirected_edges(faces=faces)
    return float(np.linalg.norm(X[e[:, 0]] - X[e[:, 1]], axis=1).mean())


def open_grid_with_oddities():
    """Open height-field grid (boundary vertices), one degenerate face with a repeated vertex,
    and one vertex that no face uses."""
    xyz, faces = synth.grid_heightfield(16, seed=3, noise_sigma=0.05)
    faces = np.concatenate([faces, [[0, 0, 1]]]).astype(np.int32)
    xyz = np.concatenate([xyz, [[3.0, 3.0, 3.0]]])
    return xyz, faces


@pytest.mark.parametrize("case", ["torus", "open"])
def test_fine_denoise_fp64_matches_oracle(case):
    if case == "torus":
        _, X, faces = synth.noisy_torus(32, seed=4)
    else:
        X, faces = open_grid_with_oddities()
    n, m = X.shape[0], faces.shape[0]
    ss, sr = mean_edge(X, faces), 0.35
    out = np.empty_like(X)
    nrm = np.empty((m, 3))
    bsp.bsp_fine_denoise(X, out, bsp.BSP_DT_F64, n, faces, m, ss, sr, 3, 5, normals_out=nrm)
    ref, ref_n = O.fine_denoise(X, faces, ss, sr, 3, 5)
    assert np.abs(nrm - ref_n).max() <= 1e-10
    assert np.abs(out - ref).max() <= 1e-10
    if case == "open":
        assert np.array_equal(out[-1], X[-1])            # the unused vertex stays
    # device buffers in and out, filter only / fitting only
    dX = torch.from_numpy(X).cuda()
    dO = torch.empty_like(dX)
    bsp.bsp_fine_denoise(dX, dO, bsp.BSP_DT_F64, n, torch.from_numpy(faces).cuda(), m, ss, sr,
                         0, 4)
    ref0, _ = O.fine_denoise(X, faces, ss, sr, 0, 4)
    assert np.abs(dO.cpu().numpy() - ref0).max() <= 1e-10
    bsp.bsp_fine_denoise(X, out, bsp.BSP_DT_F64, n, faces, m, ss, sr, 2, 0, normals_out=nrm)
    assert np.array_equal(out, X)
    assert np.abs(nrm - O.bilateral_normals(X, faces, ss, sr, 2)).max() <= 1e-10


def test_fine_denoise_fp32_matches_oracle():
    _, X64, faces = synth.noisy_torus(48, seed=5)
    X = X64.astype(np.float32)
    n, m = X.shape[0], faces.shape[0]
    ss, sr = mean_edge(X64, faces), 0.35
    out = np.empty_like(X)
    nrm = np.empty((m, 3), np.float32)
    bsp.bsp_fine_denoise(X, out, bsp.BSP_DT_F32, n, faces, m, ss, sr, 3, 5, normals_out=nrm)
    ref, ref_n = O.fine_denoise(X.astype(np.float64), faces, ss, sr, 3, 5)
    assert np.abs(nrm - ref_n).max() <= 1e-4
    assert np.abs(out - ref).max() <= 2e-5


@pytest.mark.parametrize("real", [np.float32, np.float64])
def test_normal_angle_matches_oracle(real):
    clean, noisy, faces = synth.noisy_torus(40, seed=6)
    dt = bsp.BSP_DT_F64 if real == np.float64 else bsp.BSP_DT_F32
    X, Y = clean.astype(real), noisy.astype(real)
    n, m = X.shape[0], faces.shape[0]
    got = bsp.bsp_normal_angle_error(X, Y, dt, n, faces, m)
    ref = O.normal_angle_error(X.astype(np.float64), Y.astype(np.float64), faces)
    assert got == pytest.approx(ref, rel=1e-10)
    got_d = bsp.bsp_normal_angle_error(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(),
                                       dt, n, torch.from_numpy(faces).cuda(), m)
    assert got_d == pytest.approx(ref, rel=1e-10)
    assert bsp.bsp_normal_angle_error(X, X, dt, n, faces, m) == 0.0


def test_normal_angle_closed_forms_and_errors():
    """A flat grid rotated about x by alpha: every normal turns by alpha; a mirrored copy: 180."""
    xyz, faces = synth.grid_heightfield(12, seed=1, noise_sigma=0.0)
    P = xyz.copy()
    P[:, 2] = 0.0
    n, m = P.shape[0], faces.shape[0]
    for deg in (3.0, 30.0, 100.0):
        a = np.radians(deg)
        R = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
        got = bsp.bsp_normal_angle_error(P, P @ R.T, bsp.BSP_DT_F64, n, faces, m)
        assert got == pytest.approx(deg, rel=1e-10)
    mir = P * np.array([-1.0, 1.0, 1.0])
    assert bsp.bsp_normal_angle_error(P, mir, bsp.BSP_DT_F64, n, faces, m) == pytest.approx(180.0)
    bad = faces.copy()
    bad[3, 1] = n
    with pytest.raises(bsp.BspError) as e:
        bsp.bsp_normal_angle_error(P, P, bsp.BSP_DT_F64, n, bad, m)
    assert e.value.code == bsp.BSP_ERR_INVALID_ARG
    out = np.empty_like(P)
    with pytest.raises(bsp.BspError) as e:
        bsp.bsp_fine_denoise(P, out, bsp.BSP_DT_F64, n, bad, m, 0.1, 0.3, 1, 1)
    assert e.value.code == bsp.BSP_ERR_INVALID_ARG
    for ss, sr in [(0.0, 0.3), (0.1, -1.0), (float("inf"), 0.3)]:
        with pytest.raises(bsp.BspError):
            bsp.bsp_fine_denoise(P, out, bsp.BSP_DT_F64, n, faces, m, ss, sr, 1, 1)
    # no faces: nothing moves
    bsp.bsp_fine_denoise(P, out, bsp.BSP_DT_F64, n, np.zeros((0, 3), np.int32), 0, 0.1, 0.3, 2, 2)
    assert np.array_equal(out, P)
