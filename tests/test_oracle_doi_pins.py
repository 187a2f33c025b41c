"""Pins for the oracle's restatement of the paper's own dynamic OI (Sec. 5,
Algorithm 2: one column at a time between two thresholds).

The checks start from exact eigenbases (a fixed point of every OI step) so
that the summed residual of Sec. 5 at each width has a closed form, use a
shift so large that R is almost a multiple of the identity (the span is then
kept by every step and one appended column absorbs the residual), and compare
the no-change case with Algorithm 1 run by ``oi_block`` / ``oi_track``.
``test_doi_planted_mistakes_are_caught`` plants slips on the CPU.
"""
import numpy as np
import pytest

from oracle import bsp_oracle as O
from paper_1810_02719_gb300 import synth


def path_block(n=30):
    m = O.build_mesh(n, [0, n], np.arange(n), [-1], edges=synth.path_edges(n))
    return m, O.laplacian(m.blocks[0])


def closed_form_input(W, eta):
    """X (n x 3) whose summed coordinate vector s = sum_j x_j has eigen-coefficients
    (1, 1, 1, eta, eta, eta, 0, ...): rows 3..5 of A sum to eta over j but have a larger
    Frobenius norm, so a stacked residual would differ from the summed one."""
    A = np.zeros((W.shape[1], 3))
    A[:3, :3] = np.eye(3)
    A[3:6] = [eta, eta, -eta]
    return W @ A


def check_shrinks_to_the_closed_form_width(O=O):
    """Start from the 8 lowest eigenvectors; ||e(c)|| = 0 for c >= 6, eta at c = 5, sqrt(2) eta
    at 4: with eps_l = eta / 2 and eps_h = 3 eta / 2 the width shrinks 8 -> 5 in 4 iterations."""
    _, L = path_block()
    lam, W = np.linalg.eigh(L)
    eta = 1e-3
    X = closed_form_input(W, eta)
    U, c, t, ne = O.doi_paper_block(L, X, W[:, :8], 1e-2, 1, 0.5 * eta, 1.5 * eta, 1, 16, 20)
    assert (c, t) == (5, 4)
    assert ne == pytest.approx(eta, rel=1e-8)
    assert O.max_sine(U, W[:, :5]) < 1e-10


def check_grows_by_one_under_a_near_identity_operator(O=O):
    """delta = 1e9: R^z is a multiple of I up to 1e-8, so a step keeps the span; the appended
    e / ||e|| then contains the summed residual and the loop stops at c0 + 1 after 2 iterations."""
    _, L = path_block()
    _, W = np.linalg.eigh(L)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((L.shape[0], 3))
    s = X.sum(axis=1)
    eps_h = 1e-6 * np.linalg.norm(s)
    U, c, t, ne = O.doi_paper_block(L, X, W[:, :2], 1e9, 1, 0.0, eps_h, 1, 16, 20)
    assert (c, t) == (3, 2)
    assert np.linalg.norm(s - U @ (U.T @ s)) <= eps_h
    assert np.allclose(U.T @ U, np.eye(3), atol=1e-12)


def check_no_change_is_algorithm_1(O=O):
    """eps_l = 0, eps_h = inf: one iteration, the span of one step of Algorithm 1; over a chain
    of blocks, the span of oi_track with one step and no Rayleigh-Ritz."""
    _, L = path_block()
    rng = np.random.default_rng(1)
    V0 = rng.standard_normal((L.shape[0], 4))
    X = rng.standard_normal((L.shape[0], 3))
    U, c, t, _ = O.doi_paper_block(L, X, V0, 1e-2, 2, 0.0, np.inf, 1, 16, 20)
    ref, _ = O.oi_block(L, V0, 1e-2, 2, 1, rr=False)
    assert (c, t) == (4, 1) and O.max_sine(U, ref) < 1e-12
    N, T = 24, 8
    xyz, faces = synth.grid_heightfield(N, seed=2)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(len(ptr) - 1)
    mesh = O.build_mesh(N * N, ptr, verts, parent, faces=faces, xyz=xyz)
    starts = synth.gaussian_starts(ptr, parent, 5, seed=3)
    Ud, cs, its = O.doi_paper_track(mesh, xyz, starts, 5, 0.0, np.inf)
    Ur = O.oi_track(mesh, 5, 1, starts, rr=False)
    assert np.all(cs == 5) and np.all(its == 1)
    assert max(O.max_sine(a, b) for a, b in zip(Ud, Ur)) < 1e-10


def test_shrinks_to_the_closed_form_width():
    check_shrinks_to_the_closed_form_width()


def test_grows_by_one_under_a_near_identity_operator():
    check_grows_by_one_under_a_near_identity_operator()


def test_no_change_is_algorithm_1():
    check_no_change_is_algorithm_1()


def test_width_bounds_and_iteration_cap():
    _, L = path_block()
    _, W = np.linalg.eigh(L)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((L.shape[0], 3))
    # always shrink: 6 -> 1 in five iterations, the sixth stops at c_min
    U, c, t, _ = O.doi_paper_block(L, X, W[:, :6], 1e-2, 1, 1e9, 2e9, 1, 16, 20)
    assert (c, t) == (1, 6) and U.shape == (L.shape[0], 1)
    # always grow with a cap of 3 iterations: 3 more columns, returned orthonormal
    U, c, t, _ = O.doi_paper_block(L, X, W[:, :2], 1e-2, 1, 0.0, 1e-12, 1, 16, 3)
    assert (c, t) == (5, 3) and np.allclose(U.T @ U, np.eye(5), atol=1e-12)
    # always grow, capped by c_max = 4: stops there
    U, c, t, _ = O.doi_paper_block(L, X, W[:, :2], 1e-2, 1, 0.0, 1e-12, 1, 4, 20)
    assert (c, t) == (4, 3)


class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
        self.__dict__.update(over)


def test_doi_planted_mistakes_are_caught():
    def branches_as_printed(L, X, V0, delta, z, eps_l, eps_h, c_min, c_max, t_cap):
        # Algorithm 2's printed branches: grow below eps_l, shrink above eps_h
        return _doi(L, X, V0, delta, z, eps_l, eps_h, c_min, c_max, t_cap, swap=True)

    def stacked_residual(L, X, V0, delta, z, eps_l, eps_h, c_min, c_max, t_cap):
        return _doi(L, X, V0, delta, z, eps_l, eps_h, c_min, c_max, t_cap, stacked=True)

    def no_shift(L, X, V0, delta, z, eps_l, eps_h, c_min, c_max, t_cap):
        return _doi(L, X, V0, 1e-12, z, eps_l, eps_h, c_min, c_max, t_cap)

    mutants = [
        (check_shrinks_to_the_closed_form_width, _Mutant(doi_paper_block=branches_as_printed)),
        (check_shrinks_to_the_closed_form_width, _Mutant(doi_paper_block=stacked_residual)),
        (check_grows_by_one_under_a_near_identity_operator, _Mutant(doi_paper_block=no_shift)),
    ]
    for check, mut in mutants:
        with pytest.raises(AssertionError):
            check(O=mut)


def _doi(L, X, V0, delta, z, eps_l, eps_h, c_min, c_max, t_cap, swap=False, stacked=False):
    """The oracle's loop with a slip switched on (for the planted mistakes)."""
    U = np.asarray(V0, dtype=np.float64)
    ne = 0.0
    for t in range(1, t_cap + 1):
        U, _ = O.onorm(O.apply_S(L, U, delta, z))
        R = X - U @ (U.T @ X)
        e = R.sum(axis=1)
        ne = float(np.linalg.norm(R if stacked else e))
        c = U.shape[1]
        grow = ne < eps_l if swap else ne > eps_h
        shrink = ne > eps_h if swap else ne < eps_l
        if grow and c < c_max:
            U = np.concatenate([U, (e / max(np.linalg.norm(e), 1e-300))[:, None]], axis=1)
        elif shrink and c > c_min:
            U = U[:, :c - 1]
        else:
            return U, c, t, ne
    U, _ = O.onorm(U)
    return U, U.shape[1], t_cap, ne


def test_higher_powers_of_r_converge_in_fewer_iterations():
    """The trend of the paper's R^z experiments (Sec. 8): with the same number of OI steps,
    a higher power z brings the basis closer to the exact eigenspace (the rate is
    ((lambda_c + delta) / (lambda_{c+1} + delta))^z per step)."""
    xyz, faces = synth.grid_heightfield(16, seed=0)
    m = O.build_mesh(256, [0, 256], np.arange(256), [-1], faces=faces)
    L = O.laplacian(m.blocks[0])
    c = 6
    W, _ = O.eigh_basis(L, c)
    V0 = np.random.default_rng(5).standard_normal((256, c))
    errs = [O.max_sine(O.oi_block(L, V0, 1e-2, z, 2, rr=False)[0], W) for z in (1, 2, 3, 4)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
