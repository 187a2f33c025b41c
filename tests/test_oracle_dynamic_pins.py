"""Pins for the oracle's dynamic-c decision and its growth direction (Sec. 5).

Two parts of ``oi_dynamic_block`` are pinned here against values worked out
independently of the oracle's own code:

* the width choice: the smallest j in {c_step, 2 c_step, ...} whose Ritz
  prefix meets the quality target.  A path graph has closed-form eigenpairs
  (lambda_k = 2 - 2 cos(pi k / n), u_k(i) = cos(pi k (i + 1/2) / n)), all
  distinct, and its exact eigenbasis is a fixed point of OI; coordinates
  built from chosen eigenvectors then give residual ratios known in closed
  form, so the right width is known before the oracle runs;
* the first growth column: e / ||e||, with e the residual X - U U^T X summed
  over the x, y and z columns (Sec. 5, Eq. residual and Eq. newU), checked on
  a four-vertex block worked by hand.

Planted slips (the largest passing prefix, widths off by one step, the x
residual alone, the norm of the stacked residual, no normalisation, no
projection) must each fail a pin.
"""
import numpy as np
import pytest

from oracle import bsp_oracle as O
from paper_1810_02719_gb300 import synth


# --------------------------------------------------------------------------
# closed-form path eigenbasis
# --------------------------------------------------------------------------

def path_eigvecs(n, cols):
    """Columns u_0 .. u_{cols-1} of the path Laplacian, unit norm (closed form)."""
    i = np.arange(n) + 0.5
    U = np.empty((n, cols))
    for k in range(cols):
        u = np.cos(np.pi * k * i / n)
        U[:, k] = u / np.linalg.norm(u)
    return U


def path_laplacian(n):
    m = O.build_mesh(n, [0, n], np.arange(n), [-1], edges=synth.path_edges(n))
    return O.laplacian(m.blocks[0])


N_PATH = 40


def path_case():
    """V0 = the exact lowest 24 eigenvectors; X built so that rho(8) ~ 0.16,
    rho(16) ~ 2.5e-5 and rho(24) = 0: with tol = 1e-3 the answer is 16."""
    U = path_eigvecs(N_PATH, 32)
    X = np.stack([3 * U[:, 0] + U[:, 1],
                  2 * U[:, 2] + 0.5 * U[:, 10],
                  U[:, 0] + 0.4 * U[:, 12] + 1e-4 * U[:, 20]], axis=1)
    nx = np.sqrt(9 + 1 + 4 + 0.25 + 1 + 0.16 + 1e-8)
    rho = {8: np.sqrt(0.25 + 0.16 + 1e-8) / nx, 16: 1e-4 / nx, 24: 0.0}
    return U, X, rho


def check_closed_form_path_basis(O=O):
    """The closed-form vectors are eigenvectors of the oracle's path Laplacian."""
    U = path_eigvecs(N_PATH, 32)
    L = O.laplacian(O.build_mesh(N_PATH, [0, N_PATH], np.arange(N_PATH), [-1],
                                 edges=synth.path_edges(N_PATH)).blocks[0])
    lam = 2 - 2 * np.cos(np.pi * np.arange(32) / N_PATH)
    assert np.abs(L @ U - U * lam).max() < 1e-12


def test_closed_form_path_basis():
    check_closed_form_path_basis()


def check_smallest_passing_width(O=O, dyn=None):
    dyn = dyn or O.oi_dynamic_block
    U, X, rho = path_case()
    L = path_laplacian(N_PATH)
    tol = 1e-3
    assert rho[8] > tol and rho[16] < tol
    Ub, cb, met, rounds, r = dyn(L, X, U[:, :24], 1e-2, 1, 2, tol, 8, 32, 8, 7, 0)
    assert cb == 16 and met and rounds == 0
    assert r == pytest.approx(rho[16], rel=1e-6)
    # the basis returned spans the lowest 16 eigenvectors
    assert O.max_sine(Ub, U[:, :16]) < 1e-10
    # brute force on the returned basis: this width passes, the next smaller fails
    P = lambda W: np.linalg.norm(X - W @ (W.T @ X)) / np.linalg.norm(X)
    assert P(Ub) <= tol < P(Ub[:, :cb - 8])


def test_dynamic_width_is_smallest_passing_prefix_closed_form():
    check_smallest_passing_width()


def test_dynamic_width_fails_one_step_smaller_on_tracked_blocks():
    """On tracked blocks (growth included), the chosen Ritz prefix passes and the
    prefix one step narrower does not (brute-force ratios on the returned basis)."""
    N, T = 24, 12
    xyz, faces = synth.grid_heightfield(N, seed=2)
    ptr, verts = synth.tile_partition(N, T)
    parent = synth.raster_chain(4)
    mesh = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    starts = synth.gaussian_starts(ptr, parent, 8, seed=1)
    tol = 1.5e-2   # reached at widths 32-56 on these tiles (growth rounds included)
    U, cs, met, rho = O.oi_track_dynamic(mesh, xyz, starts, tol=tol, c_min=8, c_max=64,
                                         c_step=8, t_max=2, delta=1e-2, seed=5)
    checked = 0
    for b in range(4):
        Xb = xyz[mesh.blocks[b].verts]
        ratio = lambda W: np.linalg.norm(Xb - W @ (W.T @ Xb)) / np.linalg.norm(Xb)
        assert met[b]
        assert ratio(U[b]) <= tol
        if cs[b] > 8:
            assert ratio(U[b][:, :cs[b] - 8]) > tol
            checked += 1
    assert checked == 4


# --------------------------------------------------------------------------
# growth direction: the summed residual of a hand-worked block
# --------------------------------------------------------------------------

def check_growth_first_column(O=O):
    """Four vertices, U = the constant unit vector, X as below.

    Residual columns (X minus its column means): x (0.5, -0.5, -0.5, 0.5),
    y (-0.75, 1.25, -0.75, 0.25), z (-1, -1, 2, 0); summed:
    e = (-1.25, -0.25, 0.75, 0.75), ||e||^2 = 2.75.
    """
    X = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.0], [1.0, 1.0, 1.0]])
    V = np.full((4, 1), 0.5)
    G = O.growth_columns(V, X, 2, 3, 0, 0)
    assert G.shape == (4, 2)
    e = np.array([-1.25, -0.25, 0.75, 0.75]) / np.sqrt(2.75)
    assert np.abs(G[:, 0] - e).max() < 1e-14
    # the hash column is projected off V as well
    assert abs(G[:, 1].sum()) < 1e-14


def test_growth_first_column_is_normalised_summed_residual():
    check_growth_first_column()


# --------------------------------------------------------------------------
# planted slips
# --------------------------------------------------------------------------

class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
        self.__dict__.update(over)


def _dyn_with(choose):
    """oi_dynamic_block with its width decision replaced by ``choose(rho, c, tol,
    c_step)`` (returns an index into rho, or None for "no width passes")."""
    def dyn(L, X, V0, delta, z, t_max, tol, c_min, c_max, c_step, seed, block, forced_c=-1):
        V, _ = O.oi_block(L, V0, delta, z, t_max, rr=True)
        rnd = 0
        while True:
            c = V.shape[1]
            rho = O.residual_ratios(V, X, c_step)
            q = choose(rho, c, tol, c_step)
            if q is not None:
                j = q
                return V[:, :j], j, True, rnd, rho[min(j // c_step, rho.size) - 1]
            if c >= c_max:
                return V, c, False, rnd, rho[-1]
            G = O.growth_columns(V, X, c_step, seed, block, rnd)
            V, _ = O.onorm(np.concatenate([V, G], axis=1))
            rnd += 1
            V, _ = O.oi_block(L, V, delta, z, t_max, rr=True)
    return dyn


def _largest(rho, c, tol, s):
    ok = np.nonzero(rho <= tol)[0]
    return int(np.arange(s, c + 1, s)[ok[-1]]) if ok.size else None


def _widths_shifted_up(rho, c, tol, s):
    ok = np.nonzero(rho <= tol)[0]
    return int((np.arange(s, c + 1, s) + s)[ok[0]]) if ok.size else None


def _widths_from_zero(rho, c, tol, s):
    ok = np.nonzero(rho <= tol)[0]
    return max(int(np.arange(0, c, s)[ok[0]]), s) if ok.size else None


def _growth_with(first):
    def growth(V, X, c_step, seed, block, rnd):
        G = O.growth_columns(V, X, c_step, seed, block, rnd)
        G[:, 0] = first(V, X)
        return G - V @ (V.T @ G)
    return growth


def _res(V, X):
    return X - V @ (V.T @ X)


def test_planted_dynamic_slips_are_caught():
    # the unmodified pieces pass (guards against a vacuous check)
    check_smallest_passing_width(O, _dyn_with(
        lambda rho, c, tol, s: (int(np.arange(s, c + 1, s)[np.nonzero(rho <= tol)[0][0]])
                                if np.any(rho <= tol) else None)))
    for choose in (_largest, _widths_shifted_up, _widths_from_zero):
        with pytest.raises(AssertionError):
            check_smallest_passing_width(O, _dyn_with(choose))
    firsts = [
        lambda V, X: _res(V, X)[:, 0] / np.linalg.norm(_res(V, X)[:, 0]),        # x only
        lambda V, X: _res(V, X).sum(1) / np.linalg.norm(_res(V, X)),             # stacked norm
        lambda V, X: _res(V, X).sum(1),                                           # unnormalised
        lambda V, X: X.sum(1) / np.linalg.norm(X.sum(1)),                         # not projected
    ]
    for f in firsts:
        with pytest.raises(AssertionError):
            check_growth_first_column(O=_Mutant(growth_columns=_growth_with(f)))
