"""Pins for the oracle's fine denoising step (Sec. 7.2) and the normal-angle
metric theta (Sec. 8).

Each check reaches the expected value another way: face areas by Heron's
formula, normals from another vertex of the triangle, face neighbourhoods by
brute force over all face pairs, the Gaussian kernels through scipy's normal
density, limits of the kernel widths, rotation and translation behaviour, a
lifted vertex on a flat grid whose first update is worked out by hand, and
rotations whose normal angle is known.  ``test_denoise_planted_mistakes_are_caught``
plants slips on the CPU.
"""
import numpy as np
import pytest

from oracle import bsp_oracle as O


def grid(N, jitter=0.0, height=0.0, seed=0):
    """N x N planar grid in z = 0, quads split along one diagonal (counter-clockwise)."""
    rng = np.random.default_rng(seed)
    xs, ys = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64))
    X = np.stack([xs.ravel(), ys.ravel(), np.zeros(N * N)], axis=1)
    X[:, :2] += jitter * rng.uniform(-1, 1, size=(N * N, 2))
    X[:, 2] += height * rng.standard_normal(N * N)
    f = []
    for i in range(N - 1):
        for j in range(N - 1):
            a, b, c, d = i * N + j, i * N + j + 1, (i + 1) * N + j, (i + 1) * N + j + 1
            f += [[a, b, d], [a, d, c]]
    return X, np.array(f)


def heron(X, f):
    a = np.linalg.norm(X[f[:, 1]] - X[f[:, 0]], axis=1)
    b = np.linalg.norm(X[f[:, 2]] - X[f[:, 1]], axis=1)
    c = np.linalg.norm(X[f[:, 0]] - X[f[:, 2]], axis=1)
    s = (a + b + c) / 2
    return np.sqrt(np.maximum(s * (s - a) * (s - b) * (s - c), 0))


def brute_rings(f):
    sets = [set(t) for t in f.tolist()]
    return [[j for j in range(len(f)) if sets[i] & sets[j]] for i in range(len(f))]


def rot_x(a):
    return np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])


# --------------------------------------------------------------------------
# face geometry
# --------------------------------------------------------------------------

def check_face_geometry(O=O):
    X = np.array([[0.0, 0, 0], [3, 0, 0], [0, 4, 0], [1, 1, 0], [2, 2, 0]])
    f = np.array([[0, 1, 2], [0, 2, 1], [0, 3, 4]])
    nrm, cen, area = O.face_geometry(X, f)
    assert np.allclose(nrm[0], [0, 0, 1]) and np.allclose(nrm[1], [0, 0, -1])   # right hand
    assert np.allclose(nrm[2], 0) and area[2] == 0                              # collinear
    assert np.allclose(area[:2], 6.0) and np.allclose(cen[0], [1, 4 / 3, 0])
    Y, g = grid(6, jitter=0.2, height=0.3, seed=1)
    nrm, cen, area = O.face_geometry(Y, g)
    assert np.allclose(area, heron(Y, g), rtol=1e-10)
    alt = np.cross(Y[g[:, 2]] - Y[g[:, 1]], Y[g[:, 0]] - Y[g[:, 1]])   # from the second vertex
    assert np.allclose(nrm, alt / np.linalg.norm(alt, axis=1)[:, None], atol=1e-12)


def test_face_geometry():
    check_face_geometry()


# --------------------------------------------------------------------------
# bilateral normal filter
# --------------------------------------------------------------------------

def check_wide_kernels_give_area_weighted_ring_mean(O=O):
    """sigma_s, sigma_r -> infinity: the filtered normal is the area-weighted mean of the normals
    of every face sharing a vertex with the face, normalised."""
    Y, g = grid(6, jitter=0.2, height=0.3, seed=2)
    nrm, _, _ = O.face_geometry(Y, g)
    area = heron(Y, g)
    out = O.bilateral_normals(Y, g, 1e7, 1e7, 1)
    for i, J in enumerate(brute_rings(g)):
        s = (area[J, None] * nrm[J]).sum(0)
        assert np.allclose(out[i], s / np.linalg.norm(s), atol=1e-9), i


def check_kernels_are_gaussians(O=O):
    """Two faces sharing an edge: n^_0 = normalise(A_0 n_0 + A_1 w n_1) with w the product of
    two Gaussian densities (scipy) of the centroid distance and of the normal difference, each
    relative to its value at 0."""
    stats = pytest.importorskip("scipy.stats")
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.6]])
    f = np.array([[0, 1, 2], [1, 3, 2]])
    nrm, cen, area = O.face_geometry(X, f)
    d = np.linalg.norm(cen[0] - cen[1])
    dn = np.linalg.norm(nrm[0] - nrm[1])
    for ss, sr in [(0.3, 0.4), (1.0, 0.2), (0.5, 2.0)]:
        w = (stats.norm.pdf(d, scale=ss) / stats.norm.pdf(0, scale=ss) *
             stats.norm.pdf(dn, scale=sr) / stats.norm.pdf(0, scale=sr))
        exp0 = area[0] * nrm[0] + area[1] * w * nrm[1]
        out = O.bilateral_normals(X, f, ss, sr, 1)
        assert np.allclose(out[0], exp0 / np.linalg.norm(exp0), atol=1e-12)


def check_narrow_kernels_keep_normals(O=O):
    """sigma_r -> 0 (or sigma_s -> 0): every face keeps its own normal."""
    Y, g = grid(6, jitter=0.2, height=0.3, seed=3)
    nrm, _, _ = O.face_geometry(Y, g)
    assert np.allclose(O.bilateral_normals(Y, g, 1.0, 1e-6, 2), nrm, atol=1e-12)
    assert np.allclose(O.bilateral_normals(Y, g, 1e-6, 1.0, 2), nrm, atol=1e-12)


def check_filter_is_equivariant(O=O):
    Y, g = grid(6, jitter=0.2, height=0.3, seed=4)
    R = rot_x(0.7)
    t = np.array([0.5, -2.0, 1.0])
    a = O.bilateral_normals(Y, g, 0.8, 0.35, 3)
    b = O.bilateral_normals(Y @ R.T + t, g, 0.8, 0.35, 3)
    assert np.allclose(b, a @ R.T, atol=1e-12)
    # planar input is a fixed point
    P, h = grid(6, jitter=0.2)
    assert np.allclose(O.bilateral_normals(P, h, 0.8, 0.35, 3), [0, 0, 1], atol=1e-14)


def test_wide_kernels_give_area_weighted_ring_mean():
    check_wide_kernels_give_area_weighted_ring_mean()


def test_kernels_are_gaussians():
    check_kernels_are_gaussians()


def test_narrow_kernels_keep_normals():
    check_narrow_kernels_keep_normals()


def test_filter_is_equivariant():
    check_filter_is_equivariant()


def test_filter_smooths_noise():
    """More passes bring a noisy flat grid's normals closer to the plane's."""
    Y, g = grid(8, height=0.05, seed=5)
    errs = [np.arccos(np.clip(O.face_geometry(Y, g)[0][:, 2], -1, 1)).mean()]
    for it in (1, 3, 6):
        n = O.bilateral_normals(Y, g, 1.5, 1.0, it)
        errs.append(np.arccos(np.clip(n[:, 2], -1, 1)).mean())
    assert errs[0] > errs[1] > errs[2] > errs[3]


# --------------------------------------------------------------------------
# vertex fitting
# --------------------------------------------------------------------------

def check_lifted_vertex_first_update(O=O):
    """Flat 5 x 5 grid, centre lifted by h, target normals = the plane's: after one update the
    centre sits at h / 3 and a neighbour u at (k_u / |F_u|) h / 3, k_u = faces shared with the
    centre (from the previous positions: every centroid of a face with the centre is at h / 3)."""
    X, f = grid(5)
    c, h = 12, 0.3
    X[c, 2] = h
    plane = np.tile([0.0, 0.0, 1.0], (len(f), 1))
    out = O.fit_vertices(X, f, plane, 1)
    assert out[c, 2] == pytest.approx(h / 3, rel=1e-13)
    for u in range(25):
        if u == c:
            continue
        Fu = [i for i, t in enumerate(f) if u in t]
        k = sum(1 for i in Fu if c in f[i])
        assert out[u, 2] == pytest.approx(k / len(Fu) * h / 3, abs=1e-15)
    assert np.allclose(out[:, :2], X[:, :2])       # motion only along the normals


def check_fit_fixed_points(O=O):
    """In-plane jitter with the plane's normals is a fixed point; repeated updates flatten a
    noisy grid towards the plane of its normals."""
    P, f = grid(6, jitter=0.25, seed=6)
    plane = np.tile([0.0, 0.0, 1.0], (len(f), 1))
    assert np.allclose(O.fit_vertices(P, f, plane, 3), P, atol=1e-14)
    Y, g = grid(6, height=0.1, seed=7)
    z0 = np.abs(Y[:, 2] - Y[:, 2].mean()).max()
    z1 = O.fit_vertices(Y, g, plane, 40)[:, 2]
    assert np.abs(z1 - z1.mean()).max() < 0.2 * z0


def test_lifted_vertex_first_update():
    check_lifted_vertex_first_update()


def test_fit_fixed_points():
    check_fit_fixed_points()


def test_vertex_without_faces_stays():
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0.2], [5, 5, 5]])
    f = np.array([[0, 1, 2]])
    out, _ = O.fine_denoise(X, f, 1.0, 0.5, 2, 3)
    assert np.array_equal(out[3], X[3])


# --------------------------------------------------------------------------
# normal-angle metric
# --------------------------------------------------------------------------

def check_angle_metric(O=O):
    P, f = grid(5, jitter=0.2, seed=8)
    for deg in (0.5, 10.0, 45.0, 120.0):
        R = rot_x(np.radians(deg))
        assert O.normal_angle_error(P, P @ R.T, f) == pytest.approx(deg, rel=1e-10)
    assert O.normal_angle_error(P, P, f) == 0.0
    # mirroring x reverses every triangle's orientation: each normal flips, 180 degrees
    assert O.normal_angle_error(P, P * np.array([-1.0, 1.0, 1.0]), f) == pytest.approx(180.0)
    # a degenerate face in one mesh drops out of the mean
    Q = P.copy()
    Q[f[0, 1]] = Q[f[0, 0]]
    R = rot_x(np.radians(30.0))
    assert O.normal_angle_error(Q, P @ R.T, f) == pytest.approx(30.0, rel=1e-10)


def test_angle_metric():
    check_angle_metric()


# --------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------

class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
        self.__dict__.update(over)


def test_denoise_planted_mistakes_are_caught():
    def geom_flipped(X, faces):
        nrm, cen, area = O.face_geometry(X, faces)
        return -nrm, cen, area

    def geom_two_vertex_centroid(X, faces):
        nrm, _, area = O.face_geometry(X, faces)
        f = np.asarray(faces)
        return nrm, (X[f[:, 0]] + X[f[:, 1]]) / 2.0, area

    def rings_edge_only(faces, n):            # faces sharing an edge instead of a vertex
        f = np.asarray(faces)
        sets = [set(t) for t in f.tolist()]
        return [np.array([j for j in range(len(f)) if len(sets[i] & sets[j]) >= 2])
                for i in range(len(f))]

    def geom_unit_area(X, faces):
        nrm, cen, _ = O.face_geometry(X, faces)
        return nrm, cen, np.ones(len(nrm))

    def with_helpers(**over):               # the filter built on replaced helpers
        M = _Mutant(**over)
        return lambda X, f, ss, sr, it: _bilateral(M, X, f, ss, sr, it)

    def fit_no_average(X, faces, normals, iters):
        X = np.asarray(X, float).copy()
        f = np.asarray(faces)
        vf = O.vertex_faces(f, len(X))
        for _ in range(iters):
            cen = X[f].mean(axis=1)
            Xn = X.copy()
            for v, F in enumerate(vf):
                if F.size:
                    d = np.sum(normals[F] * (cen[F] - X[v]), axis=1)
                    Xn[v] = X[v] + np.sum(normals[F] * d[:, None], axis=0)   # no 1 / |F_v|
            X = Xn
        return X

    def angle_radians(X, Xr, faces):
        return np.radians(O.normal_angle_error(X, Xr, faces))

    mutants = [
        (check_face_geometry, _Mutant(face_geometry=geom_flipped)),
        (check_kernels_are_gaussians,
         _Mutant(bilateral_normals=with_helpers(face_geometry=geom_two_vertex_centroid))),
        (check_wide_kernels_give_area_weighted_ring_mean,
         _Mutant(bilateral_normals=with_helpers(face_rings=rings_edge_only))),
        (check_wide_kernels_give_area_weighted_ring_mean,
         _Mutant(bilateral_normals=with_helpers(face_geometry=geom_unit_area))),
        (check_lifted_vertex_first_update, _Mutant(fit_vertices=fit_no_average)),
        (check_angle_metric, _Mutant(normal_angle_error=angle_radians)),
    ]
    for check, mut in mutants:
        with pytest.raises(AssertionError):
            check(O=mut)


def _bilateral(M, X, faces, sigma_s, sigma_r, iters):
    """The oracle's filter written against a replaceable module (for the planted mistakes)."""
    X = np.asarray(X, dtype=np.float64)
    nrm, cen, area = M.face_geometry(X, faces)
    rings = M.face_rings(faces, X.shape[0])
    for _ in range(iters):
        new = nrm.copy()
        for i, J in enumerate(rings):
            ks = np.exp(-np.sum((cen[i] - cen[J]) ** 2, axis=1) / (2.0 * sigma_s ** 2))
            kr = np.exp(-np.sum((nrm[i] - nrm[J]) ** 2, axis=1) / (2.0 * sigma_r ** 2))
            acc = np.sum((area[J] * ks * kr)[:, None] * nrm[J], axis=0)
            ln = np.linalg.norm(acc)
            if ln > 0:
                new[i] = acc / ln
        nrm = new
    return nrm


def test_face_rings_brute_force():
    Y, g = grid(5, jitter=0.1, seed=9)
    rings = O.face_rings(g, Y.shape[0])
    for i, J in enumerate(brute_rings(g)):
        assert np.array_equal(rings[i], J), i
