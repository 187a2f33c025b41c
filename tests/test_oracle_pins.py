"""Pins for the CPU oracle: closed forms, invariants and brute force.

Each test checks the oracle against something other than itself (a closed-form
spectrum, a textbook algorithm written out differently, an invariant that the
paper's method must satisfy), chosen so that a plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand) fails at least one
of them.  ``test_planted_mistakes_are_caught`` plants such slips on the CPU.
"""
import os

import numpy as np
import pytest

from oracle import bsp_oracle as O
from paper_1810_02719_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def single_block_mesh(n, edges=None, faces=None, xyz=None, mode=O.WEIGHT_COMBINATORIAL,
                      literal=False):
    return O.build_mesh(n, [0, n], np.arange(n), [-1], faces=faces, edges=edges,
                        xyz=xyz, weight_mode=mode, literal_degree=literal)


def tile_block(T, mode=O.WEIGHT_COMBINATORIAL, seed=0):
    xyz, faces = synth.grid_heightfield(T, seed=seed)
    m = single_block_mesh(T * T, faces=faces, xyz=xyz, mode=mode)
    return m, xyz


# --------------------------------------------------------------------------
# Sec. 3: Laplacian, closed-form spectra
# --------------------------------------------------------------------------

def check_path_spectrum(O=O):
    n = 17
    m = single_block_mesh(n, edges=synth.path_edges(n))
    lam = np.linalg.eigvalsh(O.laplacian(m.blocks[0]))
    k = np.arange(n)
    ref = np.sort(2 - 2 * np.cos(np.pi * k / n))
    assert np.allclose(lam, ref, atol=1e-12)


def test_path_spectrum():
    check_path_spectrum()


def test_cycle_spectrum():
    n = 12
    m = single_block_mesh(n, edges=synth.cycle_edges(n))
    lam = np.linalg.eigvalsh(O.laplacian(m.blocks[0]))
    k = np.arange(n)
    ref = np.sort(2 - 2 * np.cos(2 * np.pi * k / n))
    assert np.allclose(lam, ref, atol=1e-12)


def test_grid_spectrum_is_sum_of_paths():
    a, b = 5, 7
    m = single_block_mesh(a * b, edges=synth.grid_edges(a, b))
    lam = np.linalg.eigvalsh(O.laplacian(m.blocks[0]))
    pa = 2 - 2 * np.cos(np.pi * np.arange(a) / a)
    pb = 2 - 2 * np.cos(np.pi * np.arange(b) / b)
    ref = np.sort((pa[:, None] + pb[None, :]).ravel())
    assert np.allclose(lam, ref, atol=1e-12)


def check_cycle_spectrum_odd(O=O):
    """Odd cycle: not bipartite, so the signless Laplacian D + C has another spectrum."""
    n = 9
    m = O.build_mesh(n, [0, n], np.arange(n), [-1], edges=synth.cycle_edges(n))
    lam = np.linalg.eigvalsh(O.laplacian(m.blocks[0]))
    ref = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))
    assert np.allclose(lam, ref, atol=1e-12)


def test_cycle_spectrum_odd():
    check_cycle_spectrum_odd()


@pytest.mark.parametrize("T", [16, 32])
def test_tile_laplacian_invariants(T):
    m, _ = tile_block(T)
    L = O.laplacian(m.blocks[0])
    # edges of a T x T grid with one diagonal per quad
    E = 2 * T * (T - 1) + (T - 1) ** 2
    assert m.blocks[0].edges.shape[0] == E
    assert np.count_nonzero(L) == T * T + 2 * E          # 1666 and 6914
    assert np.allclose(L, L.T)
    assert np.allclose(L @ np.ones(T * T), 0.0, atol=1e-12)
    assert np.linalg.eigvalsh(L)[0] > -1e-10
    deg = np.diag(L).reshape(T, T)
    assert np.all(deg[1:-1, 1:-1] == 6)                  # interior valence
    # the diagonal runs (i,j)-(i+1,j+1): those two corners get it, the others do not
    assert deg[0, 0] == 3 and deg[-1, -1] == 3 and deg[0, -1] == 2 and deg[-1, 0] == 2


def test_inverse_square_distance_weights():
    xyz = np.array([[0, 0, 0], [2, 0, 0], [0, 1, 0], [3, 3, 0]], float)
    faces = np.array([[0, 1, 2], [1, 3, 2]])
    m = single_block_mesh(4, faces=faces, xyz=xyz, mode=O.WEIGHT_INV_SQ_DIST)
    L = O.laplacian(m.blocks[0])
    assert L[0, 1] == pytest.approx(-1 / 4)
    assert L[0, 2] == pytest.approx(-1 / 1)
    assert L[1, 2] == pytest.approx(-1 / 5)
    assert L[1, 3] == pytest.approx(-1 / 10)
    assert L[0, 3] == 0.0
    assert np.allclose(L.sum(axis=1), 0.0)
    # the paper's literal degree counts neighbours instead of summing weights
    ml = single_block_mesh(4, faces=faces, xyz=xyz, mode=O.WEIGHT_INV_SQ_DIST, literal=True)
    Ll = O.laplacian(ml.blocks[0], literal_degree=True)
    assert np.allclose(np.diag(Ll), [2, 3, 3, 2])


def test_edges_from_faces():
    tet = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]])
    assert O.undirected_edges(faces=tet).shape[0] == 6
    two = np.array([[0, 1, 2], [2, 1, 3]])
    e = O.undirected_edges(faces=two)
    assert e.tolist() == [[0, 1], [0, 2], [1, 2], [1, 3], [2, 3]]


def test_block_induced_edges_and_csr():
    # 3x3 grid, blocks {0,1,3,4} and {2,5,6,7,8}; induced edges only.
    edges = synth.grid_edges(3, 3)
    ptr = [0, 4, 9]
    verts = [4, 0, 1, 3, 2, 5, 8, 7, 6]    # deliberately permuted local orders
    m = O.build_mesh(9, ptr, verts, [-1, 0], edges=edges)
    b0, b1 = m.blocks
    # block 0 local: 4->0, 0->1, 1->2, 3->3 ; edges 0-1, 0-3, 1-4, 3-4
    assert b0.edges.tolist() == [[0, 2], [0, 3], [1, 2], [1, 3]]
    # block 1 local: 2->0, 5->1, 8->2, 7->3, 6->4 ; edges 2-5, 5-8, 7-8, 6-7
    assert b1.edges.tolist() == [[0, 1], [1, 2], [2, 3], [3, 4]]
    rp, cols, vals, diag = O.csr_pattern(b0)
    assert rp.tolist() == [0, 2, 4, 6, 8]
    assert cols.tolist() == [2, 3, 2, 3, 0, 1, 0, 1]
    assert np.all(vals == 1.0) and diag.tolist() == [2, 2, 2, 2]


# --------------------------------------------------------------------------
# Sec. 4: operator, Onorm, Algorithm 1
# --------------------------------------------------------------------------

def check_operator_spectrum(O=O, z=2, delta=0.05):
    m, _ = tile_block(8)
    L = O.laplacian(m.blocks[0])
    lam, W = np.linalg.eigh(L)
    SW = O.apply_S(L, W, delta, z)
    assert np.allclose(SW, W * (lam + delta) ** (-z), atol=1e-10)


@pytest.mark.parametrize("z", [1, 2, 3])
def test_operator_spectrum(z):
    check_operator_spectrum(z=z)


def mgs(Y):
    """Textbook modified Gram-Schmidt, pure Python loops (a different algorithm)."""
    n, c = Y.shape
    Q = [list(map(float, Y[:, j])) for j in range(c)]
    R = [[0.0] * c for _ in range(c)]
    for j in range(c):
        for i in range(j):
            R[i][j] = sum(Q[i][r] * Q[j][r] for r in range(n))
            Q[j] = [Q[j][r] - R[i][j] * Q[i][r] for r in range(n)]
        R[j][j] = sum(q * q for q in Q[j]) ** 0.5
        Q[j] = [q / R[j][j] for q in Q[j]]
    return np.array(Q).T, np.array(R)


def check_onorm(O=O):
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((9, 4)) @ np.diag([1, 1e-2, 3, 0.5])
    Q, R = O.onorm(Y)
    Qm, Rm = mgs(Y)
    assert np.allclose(Q, Qm, atol=1e-10)
    assert np.allclose(R, Rm, atol=1e-10)
    assert np.allclose(Q.T @ Q, np.eye(4), atol=1e-13)
    assert np.allclose(np.triu(R), R) and np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, Y, atol=1e-13)


def test_onorm_equals_gram_schmidt():
    check_onorm()


def test_onorm_nested_spans():
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((40, 10))
    Q, _ = O.onorm(Y)
    for j in range(1, 11):
        Qj = Q[:, :j]
        assert np.linalg.norm(Y[:, :j] - Qj @ (Qj.T @ Y[:, :j])) < 1e-12


def eigen_tangent(U, W):
    """Largest principal tangent between span(U) and span(W)."""
    s = O.principal_sines(U, W)
    s = s.max()
    return s / np.sqrt(max(1e-300, 1 - s * s))


@pytest.mark.parametrize("z", [1, 2])
def test_oi_convergence_rate_bound(z):
    """tan(theta_t) <= tan(theta_0) * ((lam_c+delta)/(lam_{c+1}+delta))^(z t) (Sec. 4)."""
    m, _ = tile_block(8)
    L = O.laplacian(m.blocks[0])
    lam, W = np.linalg.eigh(L)
    c, delta = 5, 0.05
    rho = (lam[c - 1] + delta) / (lam[c] + delta)
    assert lam[c] - lam[c - 1] > 1e-3
    rng = np.random.default_rng(1)
    U, _ = O.onorm(rng.standard_normal((64, c)))
    t0 = eigen_tangent(U, W[:, :c])
    for t in range(1, 7):
        U, _ = O.onorm(O.apply_S(L, U, delta, z))
        tt = eigen_tangent(U, W[:, :c])
        assert tt <= t0 * rho ** (z * t) * (1 + 1e-8) + 1e-12


def test_oi_power_equals_repeated_steps():
    """span after t steps on R^2 equals span after 2t steps on R (Sec. 8.2 claim)."""
    m, _ = tile_block(8)
    L = O.laplacian(m.blocks[0])
    rng = np.random.default_rng(2)
    V0 = rng.standard_normal((64, 6))
    U2, _ = O.oi_block(L, V0, 0.1, 2, 2, rr=False)
    U1, _ = O.oi_block(L, V0, 0.1, 1, 4, rr=False)
    assert O.max_sine(U1, U2) < 1e-10


def test_oi_exact_eigenbasis_is_fixed_point():
    m, _ = tile_block(8)
    L = O.laplacian(m.blocks[0])
    W, lam = O.eigh_basis(L, 7)
    U, theta = O.oi_block(L, W, 1e-2, 1, 3, rr=True)
    assert O.max_sine(U, W) < 1e-10
    assert np.allclose(theta, lam[:7], atol=1e-10)


def test_oi_brute_force_converges_to_eigh():
    m, _ = tile_block(6)          # n_b = 36
    L = O.laplacian(m.blocks[0])
    W, lam = O.eigh_basis(L, 4)
    assert lam[4] - lam[3] > 1e-3
    rng = np.random.default_rng(5)
    U, theta = O.oi_block(L, rng.standard_normal((36, 4)), 1e-2, 2, 200, rr=True)
    assert O.max_sine(U, W) < 1e-9
    assert np.allclose(theta, lam[:4], atol=1e-9)


def test_chain_of_identical_blocks_is_longer_oi():
    """Warm start (Alg. 1, first line): a chain over identical blocks continues one iteration."""
    T, nt = 6, 3
    N = T * nt
    xyz, faces = synth.grid_heightfield(N, seed=1)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(nt * nt)
    # interior tile bodies are identical graphs; use the first row of tiles only
    mesh = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, 4, seed=9)
    U = O.oi_track(mesh, 4, 2, starts, delta=0.1, z=1, rr=True)
    L0 = O.laplacian(mesh.blocks[0])
    for b in range(3):
        assert np.allclose(O.laplacian(mesh.blocks[b]), L0)
        Ub, _ = O.oi_block(L0, starts[:T * T], 0.1, 1, 2 * (b + 1), rr=False)
        assert O.max_sine(U[b], Ub) < 1e-9


def test_row_transfer_small_example():
    Up = np.arange(8.0).reshape(4, 2)
    V = O.row_transfer(Up, 6)       # rows floor(r*4/6) = 0,0,1,2,2,3
    assert V[:, 0].tolist() == [0, 0, 2, 4, 4, 6]
    V = O.row_transfer(Up, 2)       # rows 0, 2
    assert V[:, 1].tolist() == [1, 5]


def test_rayleigh_ritz_keeps_span_and_orders():
    m, _ = tile_block(8)
    L = O.laplacian(m.blocks[0])
    rng = np.random.default_rng(6)
    V, _ = O.onorm(rng.standard_normal((64, 6)))
    W, theta = O.rayleigh_ritz(L, V)
    assert O.max_sine(V, W) < 1e-12
    assert np.all(np.diff(theta) >= 0)
    assert np.allclose(W.T @ W, np.eye(6), atol=1e-12)
    assert np.allclose(W.T @ L @ W, np.diag(theta), atol=1e-10)


# --------------------------------------------------------------------------
# Sec. 3, Sec. 7: projection and reconstruction
# --------------------------------------------------------------------------

def test_full_basis_reconstructs_exactly():
    m, xyz = tile_block(6)
    L = O.laplacian(m.blocks[0])
    W, _ = O.eigh_basis(L, 36)
    E = O.project(m, [W], xyz)
    Xh = O.reconstruct(m, [W], E, 3)
    assert np.allclose(Xh, xyz, atol=1e-12)


def test_single_vector_gives_centroid():
    m, xyz = tile_block(6)
    L = O.laplacian(m.blocks[0])
    rng = np.random.default_rng(7)
    U, _ = O.oi_block(L, rng.standard_normal((36, 1)), 1e-3, 1, 30, rr=True)
    Xh = O.reconstruct(m, [U], O.project(m, [U], xyz), 3)
    assert np.allclose(Xh, xyz.mean(axis=0)[None, :], atol=1e-10)


def test_parseval_and_projector():
    m, xyz = tile_block(8)
    L = O.laplacian(m.blocks[0])
    U, _ = O.eigh_basis(L, 10)
    E = O.project(m, [U], xyz)[0]
    Xh = O.reconstruct(m, [U], [E], 3)
    assert np.sum(E * E) + np.sum((xyz - Xh) ** 2) == pytest.approx(np.sum(xyz * xyz), rel=1e-12)
    P = U @ U.T
    assert np.allclose(P @ P, P, atol=1e-12) and np.allclose(P, P.T)


# --------------------------------------------------------------------------
# Sec. 5: dynamic OI
# --------------------------------------------------------------------------

def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        ref = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    s, out = 0, []
    for _ in range(4):
        s = (s + O._GOLDEN) & O._M64
        out.append(O._mix64(s))
    assert out == ref


def test_hash_uniform_range_and_mean():
    v = np.array([O.hash_uniform(11, 3, 1, r, 2) for r in range(4000)])
    assert v.min() >= -1 and v.max() < 1
    assert abs(v.mean()) < 0.05 and abs(v.var() - 1 / 3) < 0.02
    assert O.hash_uniform(11, 3, 1, 5, 2) != O.hash_uniform(11, 3, 1, 5, 3)


def test_residual_ratios_monotone_and_exact_at_full_width():
    m, xyz = tile_block(6)
    L = O.laplacian(m.blocks[0])
    W, _ = O.eigh_basis(L, 36)
    rng = np.random.default_rng(8)
    V, _ = O.rayleigh_ritz(L, O.onorm(rng.standard_normal((36, 36)))[0])
    r = O.residual_ratios(V, xyz, 4)
    assert np.all(np.diff(r) <= 1e-15)
    assert r[-1] < 1e-13
    # brute force: the ratio at width j from scratch, with the Frobenius norm as a sum of squares
    for j, rj in zip(range(4, 37, 4), r):
        P = V[:, :j] @ V[:, :j].T
        num = sum(((xyz[i] - P[i] @ xyz) ** 2).sum() for i in range(36))
        assert rj == pytest.approx(np.sqrt(num / (xyz ** 2).sum()), rel=1e-10)


def test_dynamic_choice_is_smallest_passing_width():
    N, T = 24, 12
    xyz, faces = synth.grid_heightfield(N, seed=2)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(4)
    mesh = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, 8, seed=1)
    tol = 2e-3
    U, cs, met, rho = O.oi_track_dynamic(mesh, xyz, starts, tol=tol, c_min=8, c_max=48,
                                         c_step=8, t_max=2, delta=1e-2, seed=5)
    for b in range(4):
        Xb = xyz[mesh.blocks[b].verts]
        assert np.allclose(U[b].T @ U[b], np.eye(cs[b]), atol=1e-10)
        r = O.residual_ratios(U[b], Xb, 8)
        if met[b]:
            assert r[-1] <= tol
        # growth columns are orthogonal to the basis they extend
    G = O.growth_columns(U[0], xyz[mesh.blocks[0].verts], 8, 5, 0, 0)
    assert np.abs(U[0].T @ G).max() < 1e-12


def test_dynamic_forced_width_replays():
    N, T = 24, 12
    xyz, faces = synth.grid_heightfield(N, seed=2)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(4)
    mesh = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, 8, seed=1)
    forced = np.array([16, 24, 16, 32])
    U, cs, met, _ = O.oi_track_dynamic(mesh, xyz, starts, c_max=48, forced_c=forced)
    assert cs.tolist() == forced.tolist()


# --------------------------------------------------------------------------
# Planted mistakes: a slip in the oracle must trip a pin
# --------------------------------------------------------------------------

class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
        self.__dict__.update(over)


def test_planted_mistakes_are_caught():
    orig_lap = O.laplacian

    def lap_wrong_sign(block, literal_degree=False):
        L = orig_lap(block, literal_degree)
        off = L - np.diag(np.diag(L))
        return np.diag(np.diag(L)) + off * -1.0     # C added instead of subtracted

    def lap_dropped_degree(block, literal_degree=False):
        L = orig_lap(block, literal_degree)
        return L - np.diag(np.diag(L)) + np.diag(np.diag(L) - 1)

    def apply_no_shift(L, V, delta, z):
        Y = V
        for _ in range(z):
            Y = np.linalg.solve(L + 1e-9 * np.eye(L.shape[0]) + 0 * delta, Y)
        return Y

    def apply_one_power(L, V, delta, z):
        return np.linalg.solve(L + delta * np.eye(L.shape[0]), V)

    def onorm_no_sign(Y):
        return np.linalg.qr(Y)

    def onorm_transposed(Y):
        Q, R = O.onorm(Y)
        return Q, R.T

    mutants = [
        (check_cycle_spectrum_odd, _Mutant(laplacian=lap_wrong_sign)),
        (check_path_spectrum, _Mutant(laplacian=lap_dropped_degree)),
        (check_operator_spectrum, _Mutant(apply_S=apply_no_shift)),
        (check_operator_spectrum, _Mutant(apply_S=apply_one_power)),
        (check_onorm, _Mutant(onorm=onorm_no_sign)),
        (check_onorm, _Mutant(onorm=onorm_transposed)),
    ]
    for check, mut in mutants:
        with pytest.raises(AssertionError):
            check(O=mut)


# --------------------------------------------------------------------------
# Differentiable filter: the autograd oracle against central finite differences
# --------------------------------------------------------------------------

def test_filter_gradients_match_finite_differences():
    """Sub-mesh gradients of ||filter(x) - x_clean||^2 by FP64 autograd vs central differences."""
    import torch  # noqa: F401
    N, T = 12, 6
    clean, noisy, faces = synth.noisy_torus(N, seed=3)
    # an open patch: the torus grid's interior tiles only
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(len(ptr) - 1)
    mesh = O.build_mesh(N * N, ptr, verts, parent, faces=faces, weight_mode=O.WEIGHT_EDGE)
    E = sum(b.edges.shape[0] for b in mesh.blocks)
    rng = np.random.default_rng(0)
    w = 1.0 + 0.3 * rng.random(E)
    c, t = 5, 3
    starts = synth.gaussian_starts(ptr, parent, c, seed=4)
    loss, gx, gw, _ = O.filter_loss_grads(mesh, noisy, clean, w, c, t, starts)
    # The warm start is detached (stop-gradient), so the gradient is the
    # derivative of the same computation with every block's start frozen at its
    # unperturbed value: every block a root whose start is given.
    import torch
    _, U = O.filter_forward_torch(mesh, torch.tensor(noisy), torch.tensor(w), c, t, starts)
    frozen = np.concatenate([
        starts[:T * T, :c] if mesh.parent[b] < 0 else O.row_transfer(U[mesh.parent[b]].numpy(), T * T)
        for b in range(mesh.k)])
    roots = np.full(mesh.k, -1)
    mesh_r = O.build_mesh(N * N, ptr, verts, roots, faces=faces, weight_mode=O.WEIGHT_EDGE)
    _, gx_r, gw_r, _ = O.filter_loss_grads(mesh_r, noisy, clean, w, c, t, frozen)
    assert np.allclose(gw_r, gw, rtol=1e-8, atol=1e-12)
    assert np.allclose(gx_r, gx, rtol=1e-8, atol=1e-12)

    def f(xv, wv):
        return O.filter_loss_grads(mesh_r, xv, clean, wv, c, t, frozen)[0]

    h = 1e-6
    for e in rng.choice(E, 6, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd = (f(noisy, wp) - f(noisy, wm)) / (2 * h)
        assert fd == pytest.approx(gw[e], rel=1e-5, abs=1e-9)
    for k in rng.choice(N * N * 3, 6, replace=False):
        xp, xm = noisy.copy(), noisy.copy()
        xp.flat[k] += h
        xm.flat[k] -= h
        fd = (f(xp, w) - f(xm, w)) / (2 * h)
        assert fd == pytest.approx(gx.flat[k], rel=1e-5, abs=1e-9)
    # at w = 1 the filter's Laplacian is the combinatorial one of Sec. 3
    mesh1 = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    U = O.oi_track(mesh1, c, t, starts, rr=False)
    _, _, _, xh = O.filter_loss_grads(mesh, noisy, clean, np.ones(E), c, t, starts)
    ref = O.reconstruct(mesh1, U, O.project(mesh1, U, noisy), 3)
    assert np.allclose(xh, ref, atol=1e-10)


def test_comparison_metrics_closed_forms():
    """projector_rel_error and max_sine on bases whose angles are known."""
    e = np.eye(3)
    X = np.array([[1.0], [1.0], [0.0]])
    assert O.projector_rel_error(e[:, :1], e[:, 1:2], X) == pytest.approx(np.sqrt(2.0))
    assert O.projector_rel_error(e[:, :2], e[:, :2], X) == 0.0
    a = 0.3
    U = np.array([[np.cos(a)], [np.sin(a)], [0.0]])
    assert O.max_sine(U, e[:, :1]) == pytest.approx(np.sin(a), rel=1e-12)
    assert O.principal_sines(np.c_[U, e[:, 2]], e[:, [0, 2]]) == pytest.approx([np.sin(a), 0.0],
                                                                               abs=1e-12)
