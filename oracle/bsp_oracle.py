"""CPU oracle for block-based spectral processing with orthogonal iterations.

TEST INFRASTRUCTURE ONLY.  This module is a plain, slow, obviously correct
FP64 NumPy restatement of the method of "Block-Based Spectral Processing of
Static and Dynamic 3D Meshes using Orthogonal Iterations" (Arvanitis, Lalos,
Moustakas).  Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import it; the library never does.  It shares no code with the CUDA
path: both sides only consume the seeded inputs of
``paper_1810_02719_gb300.synth``.

Every function cites the passage of the paper it follows.  Dense matrices and
LAPACK routines (``numpy.linalg.solve``, ``qr``, ``eigh``) serve as steps; no
blocking, fusion or reordering is done beyond what the definitions state.

Readings taken where the paper is silent or inconsistent (each is a parameter
or a documented choice here):
  * degree matrix: D_ii = sum_j C_ij (a true Laplacian, L 1 = 0); the paper's
    literal D_ii = |N(i)| is available as ``literal_degree=True`` (Sec. 3).
  * unequal block sizes: a child's start matrix takes row r from row
    floor(r * n_parent / n_child) of the parent's basis, then Onorm (Sec. 4
    requires equal sizes; this generalises it).
  * Onorm: Householder QR with the sign convention diag(R) > 0 (Sec. 4, Eq. HS1).
  * roots: the start matrix of a root block is a supplied random matrix,
    orthonormalised by Onorm (the paper uses the SVD of the first block, Sec. 4).
  * Rayleigh-Ritz (optional, not in the paper): H = V^T L V, ascending Ritz order.
  * dynamic c: relative Frobenius residual, growth by c_step columns
    [e/||e||, counter-hash columns], see ``oi_track_dynamic``; the paper's own
    one-column policy between two thresholds, with the branch directions of
    the text, is ``doi_paper_block`` / ``doi_paper_track``.
  * overlapped parts (Sec. 6.1): induced subgraph per part, copies weighted
    by their degree in the part, see ``weighted_average``.
  * codec (Sec. 7.1, Sec. 8): a uniform quantiser per block and coefficient column
    over [min, max]; NMSVE as printed (unsquared norms, linear value), GL with
    each geometry's own edge lengths, see ``quantize`` and ``nmsve``.
  * fine denoising (Sec. 7.2): face neighbourhood = faces sharing a vertex;
    normals filtered with the input's centroids and areas, see
    ``bilateral_normals``, ``fit_vertices`` and ``normal_angle_error``.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py``, ``tests/test_oracle_codec_pins.py``,
``tests/test_oracle_denoise_pins.py``, ``tests/test_oracle_doi_pins.py`` and
``tests/test_oracle_overlap_pins.py`` against
closed forms, invariants, hand-worked examples or brute force.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

WEIGHT_COMBINATORIAL = 0
WEIGHT_EDGE = 1
WEIGHT_INV_SQ_DIST = 2


# ---------------------------------------------------------------------------
# Sec. 3: mesh, edges, per-block Laplacian
# ---------------------------------------------------------------------------

def undirected_edges(faces: Optional[np.ndarray] = None,
                     edges: Optional[np.ndarray] = None) -> np.ndarray:
    """Edge set E of M = (V, F) (Sec. 3): each triangle contributes its three sides.

    Returns unique undirected edges as (min, max) pairs, sorted
    lexicographically, int64 [E, 2].  With ``edges`` the given list is
    normalised the same way (graphs without faces).
    """
    if faces is not None:
        f = np.asarray(faces, dtype=np.int64)
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
    else:
        e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


@dataclass
class Block:
    """One submesh: its global vertices (in local order) and induced edges."""
    verts: np.ndarray              # int64 [n_b] global vertex ids, local order
    edges: np.ndarray              # int64 [E_b, 2] local (i < j), sorted
    weights: np.ndarray            # float64 [E_b] C_ij per edge


@dataclass
class Mesh:
    """The oracle's view of a partitioned mesh (Sec. 3 and Sec. 4)."""
    n: int
    blocks: List[Block]
    parent: np.ndarray             # int64 [k], -1 for a root; parent[b] < b
    xyz: Optional[np.ndarray] = None
    literal_degree: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def k(self) -> int:
        return len(self.blocks)


def build_mesh(n, block_ptr, block_verts, parent, faces=None, edges=None,
               xyz=None, weight_mode=WEIGHT_COMBINATORIAL, literal_degree=False) -> Mesh:
    """Partition the edge set into per-block induced edge lists (Sec. 4).

    The mesh is split into k non-overlapping parts; block b's Laplacian L[b]
    uses only the edges with both end points in block b (the missing
    neighbours are the edge effect described in Sec. 6.1).  Local edges are
    listed with i < j in lexicographic order; this is also the order of the
    per-edge weights.  ``weight_mode``: combinatorial (C_ij = 1), edge (all
    weights start at 1 and may be replaced), or inverse squared distance
    C_ij = 1 / ||v_i - v_j||^2 (Sec. 3, Eq. for C).
    """
    ptr = np.asarray(block_ptr, dtype=np.int64)
    bv = np.asarray(block_verts, dtype=np.int64)
    k = len(ptr) - 1
    blk_of = np.full(n, -1, dtype=np.int64)
    loc_of = np.full(n, -1, dtype=np.int64)
    for b in range(k):
        vs = bv[ptr[b]:ptr[b + 1]]
        blk_of[vs] = b
        loc_of[vs] = np.arange(vs.size)
    E = undirected_edges(faces=faces, edges=edges)
    same = blk_of[E[:, 0]] == blk_of[E[:, 1]]
    E = E[same]
    eb = blk_of[E[:, 0]]
    li = loc_of[E[:, 0]]
    lj = loc_of[E[:, 1]]
    lo, hi = np.minimum(li, lj), np.maximum(li, lj)
    blocks = []
    for b in range(k):
        m = eb == b
        le = np.stack([lo[m], hi[m]], axis=1)
        order = np.lexsort((le[:, 1], le[:, 0]))
        le = le[order]
        verts = bv[ptr[b]:ptr[b + 1]]
        if weight_mode == WEIGHT_INV_SQ_DIST:
            d = xyz[verts[le[:, 0]]] - xyz[verts[le[:, 1]]]
            w = 1.0 / np.sum(d * d, axis=1)
        else:
            w = np.ones(le.shape[0])
        blocks.append(Block(verts=verts, edges=le, weights=w))
    return Mesh(n=n, blocks=blocks, parent=np.asarray(parent, dtype=np.int64),
                xyz=None if xyz is None else np.asarray(xyz, dtype=np.float64),
                literal_degree=literal_degree)


def laplacian(block: Block, literal_degree: bool = False) -> np.ndarray:
    """Dense L = D - C of one block (Sec. 3, Eqs. for L and C).

    C_ij = C_ji = w_ij on every edge of the block.  D_ii = sum_j C_ij (so that
    L 1 = 0), or, with ``literal_degree``, the neighbour count |N(i)| that the
    paper prints.
    """
    n_b = block.verts.size
    C = np.zeros((n_b, n_b))
    i, j = block.edges[:, 0], block.edges[:, 1]
    C[i, j] = block.weights
    C[j, i] = block.weights
    if literal_degree:
        D = np.diag((C != 0).sum(axis=1).astype(np.float64))
    else:
        D = np.diag(C.sum(axis=1))
    return D - C


def csr_pattern(block: Block, literal_degree: bool = False):
    """Per-block CSR view of L's off-diagonal pattern (for the assembly check).

    Returns (row_ptr int64 [n_b+1], cols int64 [2 E_b] ascending per row,
    vals float64 [2 E_b] = C_ij, diag float64 [n_b] = D_ii), derived from the
    dense Laplacian so that it restates Sec. 3's definition and nothing else.
    """
    L = laplacian(block, literal_degree)
    off = -L.copy()
    np.fill_diagonal(off, 0.0)
    A = np.zeros_like(off, dtype=bool)
    i, j = block.edges[:, 0], block.edges[:, 1]
    A[i, j] = True
    A[j, i] = True
    rows, cols = np.nonzero(A)           # row-major, columns ascending
    row_ptr = np.zeros(L.shape[0] + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, cols.astype(np.int64), off[rows, cols], np.diag(L).copy()


# ---------------------------------------------------------------------------
# Sec. 4: the iteration operator, Onorm, Algorithm 1
# ---------------------------------------------------------------------------

def apply_S(L: np.ndarray, V: np.ndarray, delta: float, z: int) -> np.ndarray:
    """S V with S = R^z and R = (L + delta I)^{-1} (Sec. 4, below Alg. 1).

    Applied as z successive dense linear solves (the paper applies R^z with
    linear-system solvers).
    """
    A = L + delta * np.eye(L.shape[0])
    Y = np.array(V, dtype=np.float64)
    for _ in range(z):
        Y = np.linalg.solve(A, Y)
    return Y


def onorm(Y: np.ndarray):
    """Onorm: thin QR by Householder reflections, keep Q (Sec. 4, Eq. HS1).

    Q_qr = H_1^T ... H_c^T restricted to its first c columns (LAPACK geqrf via
    numpy).  Signs are fixed so that diag(R) > 0, which makes Q unique for a
    full-rank Y.  Returns (Q [n x c], R [c x c]).
    """
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def rayleigh_ritz(L: np.ndarray, V: np.ndarray):
    """Rayleigh-Ritz on span(V): H = V^T L V = W Theta W^T, return (V W, theta).

    Ritz values ascending.  Not part of the paper's Alg. 1; it leaves span(V)
    unchanged and orders the columns from low to high graph frequency.
    """
    H = V.T @ L @ V
    H = 0.5 * (H + H.T)
    theta, W = np.linalg.eigh(H)
    return V @ W, theta


def row_transfer(U_parent: np.ndarray, n_b: int) -> np.ndarray:
    """Warm start for a block of another size: row r <- parent row floor(r n_p / n_b)."""
    n_p = U_parent.shape[0]
    idx = (np.arange(n_b) * n_p) // n_b
    return U_parent[idx]


def oi_block(L: np.ndarray, V0: np.ndarray, delta: float, z: int, t_max: int,
             rr: bool = True):
    """Algorithm 1 (Sec. 4) for one submesh.

    U(0) <- V0; for t = 1..t_max: U(t) <- Onorm(R^z U(t-1)); then optional
    Rayleigh-Ritz.  Returns (U, theta or None).
    """
    U, _ = onorm(V0)
    for _ in range(t_max):
        U, _ = onorm(apply_S(L, U, delta, z))
    theta = None
    if rr:
        U, theta = rayleigh_ritz(L, U)
    return U, theta


def oi_track(mesh: Mesh, c: int, t_max: int, starts: np.ndarray, delta: float = 1e-2,
             z: int = 1, rr: bool = True, block_ids=None):
    """Track U_c[b] for every block in the given topological order (Sec. 4).

    Root blocks (parent -1) start from Onorm of their rows of ``starts``
    (concatenated over roots, in block order); every other block starts from its
    parent's final basis (Alg. 1, first line), row-transferred if the sizes
    differ.  Returns the list of bases U_b [n_b x c].
    """
    k = mesh.k
    U = [None] * k
    root_off = {}
    off = 0
    for b in range(k):
        if mesh.parent[b] < 0:
            root_off[b] = off
            off += mesh.blocks[b].verts.size
    for b in range(k):
        n_b = mesh.blocks[b].verts.size
        if c > n_b:
            raise ValueError(f"c={c} exceeds block {b} size {n_b}")
        L = laplacian(mesh.blocks[b], mesh.literal_degree)
        p = mesh.parent[b]
        if p < 0:
            V0 = starts[root_off[b]:root_off[b] + n_b, :c]
        else:
            V0 = row_transfer(U[p], n_b)
        U[b], _ = oi_block(L, V0, delta, z, t_max, rr)
    return U


def eigh_basis(L: np.ndarray, c: int):
    """The paper's "SVD" baseline: the c eigenvectors of L with the lowest eigenvalues (Sec. 3)."""
    lam, W = np.linalg.eigh(L)
    return W[:, :c], lam


# ---------------------------------------------------------------------------
# Sec. 3 / Sec. 7: GFT projection and reconstruction
# ---------------------------------------------------------------------------

def project(mesh: Mesh, U: List[np.ndarray], X: np.ndarray) -> List[np.ndarray]:
    """Spectral coefficients E[b] = U_c[b]^T v[b] per block (Sec. 3 GFT; Sec. 7.1).

    X holds one row per global vertex (n x m, m = 3 for xyz, 3F for F frames).
    """
    return [U[b].T @ X[mesh.blocks[b].verts] for b in range(mesh.k)]


def reconstruct(mesh: Mesh, U: List[np.ndarray], E: List[np.ndarray], m: int) -> np.ndarray:
    """Inverse GFT per block, v~[b] = U_c[b] E[b], scattered to the global rows (Sec. 7.1, 7.2).

    Non-overlapping partitions: every vertex belongs to exactly one block.
    """
    out = np.zeros((mesh.n, m))
    for b in range(mesh.k):
        out[mesh.blocks[b].verts] = U[b] @ E[b]
    return out


# ---------------------------------------------------------------------------
# Sec. 7.1 compression, with the quantisation, bits per vertex and NMSVE of
# Sec. 8's evaluation
# ---------------------------------------------------------------------------

def quantize(E: List[np.ndarray], bits: int):
    """Uniform scalar quantisation of every block's coefficients to ``bits`` bits (Sec. 7.1, Sec. 8).

    The paper gives the bit count (q_c = 12) but not the range.  Reading: each
    column of each block E[b] (c_b x cols) is coded over its own range
    [lo, hi] = [min, max], kept as side information; with q = 2^bits - 1,
    s = q / (hi - lo) and code = clip(rint((e - lo) s), 0, q), rint rounding
    half to even; s = 0 when hi == lo or when s is not finite.  The codes are
    integers decided by floating point, so the arithmetic runs in the
    coefficients' own dtype (float32 for float32 E), one rounding per
    operation, as the kernel does.

    Returns (codes, ranges): codes[b] uint16 (c_b x cols); ranges[b] (cols x 2).
    """
    codes, ranges = [], []
    for Eb in E:
        Eb = np.asarray(Eb)
        t = Eb.dtype.type
        qmax = t((1 << bits) - 1)
        lo = Eb.min(axis=0)
        hi = Eb.max(axis=0)
        with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
            s = np.where(hi > lo, qmax / (hi - lo), t(0)).astype(Eb.dtype)
        s = np.where(np.isfinite(s), s, t(0)).astype(Eb.dtype)
        q = np.rint((Eb - lo) * s)
        q = np.clip(q, t(0), qmax)
        codes.append(q.astype(np.uint16))
        ranges.append(np.stack([lo, hi], axis=1))
    return codes, ranges


def dequantize(codes: List[np.ndarray], ranges: List[np.ndarray], bits: int,
               dtype=np.float32) -> List[np.ndarray]:
    """Decoder of ``quantize`` (Sec. 7.1): e~ = lo + code (hi - lo) / q, in ``dtype``."""
    out = []
    t = np.dtype(dtype).type
    qmax = t((1 << bits) - 1)
    for Cb, Rb in zip(codes, ranges):
        lo = Rb[:, 0].astype(dtype)
        hi = Rb[:, 1].astype(dtype)
        step = (hi - lo) / qmax
        out.append(lo + Cb.astype(dtype) * step)
    return out


def bits_per_vertex(c_blocks, n: int, bits: int) -> float:
    """Coefficient bits per vertex, 3 q_c c k / n_d of Sec. 8 with per-block c_b.

    Counts the coded xyz coefficients only (no connectivity, no ranges), as
    the paper does.
    """
    return 3.0 * bits * float(np.sum(c_blocks)) / n


def geometric_laplacian(X: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """GL(v_i) = v_i - sum_j v_j / d_ij / sum_j 1 / d_ij over mesh neighbours (Sec. 8, NMSVE).

    Neighbours come from the edges of all faces; d_ij is the edge length in
    the geometry X itself.  Readings: a neighbour at distance 0 gets no
    weight; a vertex with no weighted neighbour keeps GL = v_i.
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    E = undirected_edges(faces=faces)
    num = np.zeros((n, 3))
    den = np.zeros(n)
    for a, b in E:
        d = float(np.linalg.norm(X[a] - X[b]))
        if d > 0.0:
            num[a] += X[b] / d
            den[a] += 1.0 / d
            num[b] += X[a] / d
            den[b] += 1.0 / d
    GL = X.copy()
    has = den > 0
    GL[has] = X[has] - num[has] / den[has, None]
    return GL


def nmsve(X: np.ndarray, X_rec: np.ndarray, faces: np.ndarray):
    """Normalised mean square visual error of Sec. 8.

    (||v - v~|| + ||GL(v) - GL(v~)||) / (2 n) with v, v~ the 3n stacked
    coordinates, norms as printed (unsquared), value linear (the paper's dB
    label comes without a conversion).  Returns (nmsve, ||v - v~||,
    ||GL(v) - GL(v~)||).
    """
    X = np.asarray(X, dtype=np.float64)
    Xr = np.asarray(X_rec, dtype=np.float64)
    n = X.shape[0]
    a = float(np.linalg.norm(X - Xr))
    g = float(np.linalg.norm(geometric_laplacian(X, faces) - geometric_laplacian(Xr, faces)))
    return (a + g) / (2.0 * n), a, g


# ---------------------------------------------------------------------------
# Sec. 7.2: fine denoising after the coarse spectral step (bilateral filter of
# the face normals, then vertex positions fitted to the filtered normals)
# ---------------------------------------------------------------------------

def face_geometry(X: np.ndarray, faces: np.ndarray):
    """Unit normals, centroids and areas of the faces (Sec. 7.2, face normal equation).

    n_i = (v2 - v1) x (v3 - v1) / ||(v2 - v1) x (v3 - v1)||, m_i the centroid,
    A_i = ||(v2 - v1) x (v3 - v1)|| / 2.  Reading: a degenerate face (zero
    cross product) gets the zero vector as its normal and area 0.
    """
    X = np.asarray(X, dtype=np.float64)
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    cr = np.cross(X[f[:, 1]] - X[f[:, 0]], X[f[:, 2]] - X[f[:, 0]])
    ln = np.linalg.norm(cr, axis=1)
    nrm = np.zeros_like(cr)
    ok = ln > 0
    nrm[ok] = cr[ok] / ln[ok, None]
    cen = (X[f[:, 0]] + X[f[:, 1]] + X[f[:, 2]]) / 3.0
    return nrm, cen, 0.5 * ln


def vertex_faces(faces: np.ndarray, n: int) -> List[np.ndarray]:
    """Index set F_v of the faces incident to every vertex (Sec. 7.2)."""
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    lists = [[] for _ in range(n)]
    for i, tri in enumerate(f):
        for v in set(tri.tolist()):
            lists[v].append(i)
    return [np.array(sorted(l), dtype=np.int64) for l in lists]


def face_rings(faces: np.ndarray, n: int) -> List[np.ndarray]:
    """Neighbourhood N(f_i) of every face for the bilateral filter (Sec. 7.2).

    Reading (the paper leaves it open): the faces that share at least one
    vertex with f_i, f_i included.
    """
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    vf = vertex_faces(f, n)
    return [np.unique(np.concatenate([vf[v] for v in tri])) for tri in f]


def bilateral_normals(X: np.ndarray, faces: np.ndarray, sigma_s: float, sigma_r: float,
                      iters: int) -> np.ndarray:
    """Bilateral filter of the face normals (Sec. 7.2, Eqs. BF, Wm, Wn), ``iters`` times.

    n_i <- normalise( sum_{j in N(f_i)} A_j K_s(m_i, m_j) K_r(n_i, n_j) n_j ),
    K_s = exp(-||m_i - m_j||^2 / (2 sigma_s^2)), K_r = exp(-||n_i - n_j||^2 /
    (2 sigma_r^2)); W_i is the normalisation.  Readings: centroids and areas
    stay those of X (the filter moves no vertex); each pass filters the
    previous pass's normals; a face whose weighted sum vanishes keeps its
    normal.
    """
    X = np.asarray(X, dtype=np.float64)
    nrm, cen, area = face_geometry(X, faces)
    rings = face_rings(faces, X.shape[0])
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


def fit_vertices(X: np.ndarray, faces: np.ndarray, normals: np.ndarray, iters: int) -> np.ndarray:
    """Vertex update to match the filtered normals (Sec. 7.2, Eqs. iter1 and iter2), ``iters`` times.

    v <- v + (1 / |F_v|) sum_{z in F_v} n_z [n_z^T (m_z - v)], with m_z the
    centroid of face z at the current positions; every vertex moves from the
    previous iterate's positions.  A vertex in no face stays.
    """
    X = np.asarray(X, dtype=np.float64).copy()
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    vf = vertex_faces(f, X.shape[0])
    for _ in range(iters):
        cen = (X[f[:, 0]] + X[f[:, 1]] + X[f[:, 2]]) / 3.0
        Xn = X.copy()
        for v, F in enumerate(vf):
            if F.size == 0:
                continue
            d = np.sum(normals[F] * (cen[F] - X[v]), axis=1)
            Xn[v] = X[v] + np.sum(normals[F] * d[:, None], axis=0) / F.size
        X = Xn
    return X


def fine_denoise(X: np.ndarray, faces: np.ndarray, sigma_s: float, sigma_r: float,
                 normal_iters: int, vertex_iters: int):
    """The fine step of the coarse-to-fine denoising (Sec. 7.2): filtered normals, fitted vertices."""
    nrm = bilateral_normals(X, faces, sigma_s, sigma_r, normal_iters)
    return fit_vertices(X, faces, nrm, vertex_iters), nrm


def normal_angle_error(X: np.ndarray, X_ref: np.ndarray, faces: np.ndarray) -> float:
    """Mean angle theta (degrees) between corresponding face normals of two meshes (Sec. 8).

    Reading: the angle is atan2(||n x n_ref||, n . n_ref); faces that are
    degenerate in either mesh are left out of the mean (0 if none is left).
    """
    n1, _, _ = face_geometry(X, faces)
    n2, _, _ = face_geometry(X_ref, faces)
    ok = (np.linalg.norm(n1, axis=1) > 0) & (np.linalg.norm(n2, axis=1) > 0)
    if not np.any(ok):
        return 0.0
    ang = np.arctan2(np.linalg.norm(np.cross(n1[ok], n2[ok]), axis=1),
                     np.sum(n1[ok] * n2[ok], axis=1))
    return float(np.degrees(np.mean(ang)))


# ---------------------------------------------------------------------------
# Sec. 6.1: overlapped submeshes and the degree-weighted average (Algorithm 3)
# ---------------------------------------------------------------------------

def build_overlapped_mesh(n, block_ptr, block_verts, parent, faces=None, edges=None) -> Mesh:
    """Parts that may share vertices (Sec. 6.1): each block's Laplacian is that of the
    subgraph induced by its own vertex list, as in ``build_mesh``, but a vertex may
    appear in several blocks (combinatorial weights)."""
    ptr = np.asarray(block_ptr, dtype=np.int64)
    bv = np.asarray(block_verts, dtype=np.int64)
    E = undirected_edges(faces=faces, edges=edges)
    blocks = []
    for b in range(len(ptr) - 1):
        verts = bv[ptr[b]:ptr[b + 1]]
        loc = np.full(n, -1, dtype=np.int64)
        loc[verts] = np.arange(verts.size)
        inside = (loc[E[:, 0]] >= 0) & (loc[E[:, 1]] >= 0)
        li, lj = loc[E[inside, 0]], loc[E[inside, 1]]
        le = np.stack([np.minimum(li, lj), np.maximum(li, lj)], axis=1)
        le = le[np.lexsort((le[:, 1], le[:, 0]))]
        blocks.append(Block(verts=verts, edges=le, weights=np.ones(le.shape[0])))
    return Mesh(n=n, blocks=blocks, parent=np.asarray(parent, dtype=np.int64), xyz=None,
                literal_degree=False)


def block_degrees(block: Block) -> np.ndarray:
    """Degree of every local vertex inside its block: its neighbours in the induced subgraph."""
    d = np.zeros(block.verts.size, dtype=np.int64)
    np.add.at(d, block.edges[:, 0], 1)
    np.add.at(d, block.edges[:, 1], 1)
    return d


def weighted_average(mesh: Mesh, Xb: List[np.ndarray], cols: int) -> np.ndarray:
    """Algorithm 3 (Sec. 6.1): every vertex's position is the average of its copies in the
    parts it belongs to, each weighted by the vertex's degree in that part.

    Reading: a vertex whose weights sum to 0 (isolated in every part holding it)
    takes the plain mean of its copies; a vertex in no part stays 0.
    """
    num = np.zeros((mesh.n, cols))
    den = np.zeros(mesh.n)
    cnt = np.zeros(mesh.n)
    plain = np.zeros((mesh.n, cols))
    for b, blk in enumerate(mesh.blocks):
        w = block_degrees(blk).astype(np.float64)
        np.add.at(num, blk.verts, w[:, None] * Xb[b])
        np.add.at(den, blk.verts, w)
        np.add.at(plain, blk.verts, Xb[b])
        np.add.at(cnt, blk.verts, 1.0)
    out = np.zeros((mesh.n, cols))
    ok = den > 0
    out[ok] = num[ok] / den[ok, None]
    iso = (~ok) & (cnt > 0)
    out[iso] = plain[iso] / cnt[iso, None]
    return out


def reconstruct_overlapped(mesh: Mesh, U: List[np.ndarray], X: np.ndarray) -> np.ndarray:
    """Overlapped reconstruction (Sec. 6.1): every part reconstructs its own copy
    U_b U_b^T X[b]; Algorithm 3 merges the copies."""
    cols = X.shape[1]
    Xb = [U[b] @ (U[b].T @ X[blk.verts]) for b, blk in enumerate(mesh.blocks)]
    return weighted_average(mesh, Xb, cols)


# ---------------------------------------------------------------------------
# Sec. 5: dynamic OI (reading: relative Frobenius residual, growth by c_step)
# ---------------------------------------------------------------------------

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014)."""
    x &= _M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _M64
    return x ^ (x >> 31)


def hash_uniform(seed: int, block: int, rnd: int, row: int, col: int) -> float:
    """Counter-based draw in [-1, 1): chain SplitMix64 over (seed, block, round, row, col).

    h <- seed; for each field f: h <- mix64(h + golden * (f + 1)); the top 53
    bits of h give u in [0, 1); the draw is 2u - 1.
    """
    h = seed & _M64
    for f in (block, rnd, row, col):
        h = _mix64(h + _GOLDEN * (f + 1))
    u = (h >> 11) * (1.0 / (1 << 53))
    return 2.0 * u - 1.0


def residual_ratios(V: np.ndarray, X: np.ndarray, c_step: int):
    """rho(j) = ||X - V_j V_j^T X||_F / ||X||_F for j = c_step, 2 c_step, ..., c.

    V_j is the first j columns of V; computed directly (not by Parseval).
    """
    nx = np.linalg.norm(X)
    out = []
    for j in range(c_step, V.shape[1] + 1, c_step):
        Vj = V[:, :j]
        out.append(np.linalg.norm(X - Vj @ (Vj.T @ X)) / nx)
    return np.asarray(out)


def growth_columns(V: np.ndarray, X: np.ndarray, c_step: int, seed: int, block: int,
                   rnd: int) -> np.ndarray:
    """New columns for a growth round of dynamic OI (Sec. 5, Eq. newU).

    The first is the normalised residual e/||e||, with e summed over the x, y
    and z coordinates (Sec. 5, Eq. residual); the other c_step - 1 are
    counter-hash draws (``hash_uniform``, columns 1 .. c_step-1).  All of them are
    projected off span(V) before they are appended.
    """
    n_b = V.shape[0]
    e = (X - V @ (V.T @ X)).sum(axis=1)
    G = np.empty((n_b, c_step))
    G[:, 0] = e / np.linalg.norm(e)
    for col in range(1, c_step):
        G[:, col] = [hash_uniform(seed, block, rnd, r, col) for r in range(n_b)]
    return G - V @ (V.T @ G)


def oi_dynamic_block(L, X, V0, delta, z, t_max, tol, c_min, c_max, c_step, seed, block,
                     forced_c=-1):
    """Dynamic OI for one submesh (Sec. 5, Alg. 2), with this library's reading.

    Start at the width of V0; run Alg. 1 (t_max steps) and Rayleigh-Ritz; take
    the smallest j in {c_step, 2 c_step, ..., c} with rho(j) <= tol (the Ritz
    prefix, i.e. the shrink step); if none and c < c_max, grow by c_step
    columns (``growth_columns``), orthonormalise, and repeat Alg. 1 warm from the
    grown basis.  The paper's growth direction (append e/||e||, then Onorm of
    R^z [U, e/||e||]) is kept; its two-threshold stop becomes the single
    quality target ``tol``, and growth stops at c_max.  ``forced_c`` >= 0
    replaces the decision by that width (a replay hook for blocks whose rho lies
    at the threshold).
    Returns (U_b [n_b x c_b], c_b, met, rounds, rho at c_b).
    """
    V, _ = oi_block(L, V0, delta, z, t_max, rr=True)
    rnd = 0
    while True:
        c = V.shape[1]
        rho = residual_ratios(V, X, c_step)
        widths = np.arange(c_step, c + 1, c_step)
        if forced_c >= 0:
            if forced_c <= c or c >= c_max:
                j = min(forced_c, c)
                return V[:, :j], j, True, rnd, rho[j // c_step - 1]
        else:
            ok = np.nonzero(rho <= tol)[0]
            if ok.size:
                j = int(widths[ok[0]])
                return V[:, :j], j, True, rnd, rho[ok[0]]
            if c >= c_max:
                return V, c, False, rnd, rho[-1]
        G = growth_columns(V, X, c_step, seed, block, rnd)
        V, _ = onorm(np.concatenate([V, G], axis=1))
        rnd += 1
        V, _ = oi_block(L, V, delta, z, t_max, rr=True)


def oi_track_dynamic(mesh: Mesh, X: np.ndarray, starts: np.ndarray, tol: float = 2e-3,
                     c_min: int = 8, c_max: int = 128, c_step: int = 8, t_max: int = 2,
                     delta: float = 1e-2, z: int = 1, seed: int = 0, forced_c=None,
                     block_ids=None):
    """Dynamic OI over all blocks in topological order (Sec. 5, Alg. 2).

    Roots start at width c_min from their rows of ``starts`` (first c_min
    columns); a child starts at its parent's width c_parent (>= c_min) from the
    parent's basis (Alg. 2, second line).  X: n x 3 coordinates.
    ``block_ids``: the index of every block of ``mesh`` in a larger mesh it was
    cut from, which keys the counter hash of the growth columns (default: its
    position here).
    Returns (U list, c array, met array, rho array).
    """
    k = mesh.k
    U = [None] * k
    cs = np.zeros(k, dtype=np.int64)
    met = np.zeros(k, dtype=bool)
    rhos = np.zeros(k)
    off = 0
    root_off = {}
    for b in range(k):
        if mesh.parent[b] < 0:
            root_off[b] = off
            off += mesh.blocks[b].verts.size
    for b in range(k):
        blk = mesh.blocks[b]
        n_b = blk.verts.size
        L = laplacian(blk, mesh.literal_degree)
        p = mesh.parent[b]
        if p < 0:
            V0 = starts[root_off[b]:root_off[b] + n_b, :c_min]
        else:
            V0 = row_transfer(U[p], n_b)
        fc = -1 if forced_c is None else int(forced_c[b])
        U[b], cs[b], met[b], _, rhos[b] = oi_dynamic_block(
            L, X[blk.verts], V0, delta, z, t_max, tol, c_min,
            min(c_max, (n_b // c_step) * c_step), c_step, seed,
            b if block_ids is None else int(block_ids[b]), fc)
    return U, cs, met, rhos


def doi_paper_block(L: np.ndarray, X: np.ndarray, V0: np.ndarray, delta: float, z: int,
                    eps_l: float, eps_h: float, c_min: int, c_max: int, t_cap: int):
    """The paper's own dynamic OI for one submesh (Sec. 5, Algorithm 2), one column at a time.

    Every iteration applies Algorithm 1 once, U = Onorm(R^z U), and measures
    the summed residual e = sum_{j in x, y, z} (v_j - U U^T v_j) (Sec. 5,
    Eq. residual).  Branch directions as the text states them (Algorithm 2
    prints them swapped): ||e|| > eps_h grows the basis by e/||e|| (the next
    iteration's Onorm(R^z [U, e/||e||]) is Eq. newU), ||e|| < eps_l keeps the
    first c - 1 columns, anything else stops.  Readings: the width stays in
    [c_min, c_max] (a branch that would leave it stops instead), at most
    t_cap iterations run, and a basis left with an appended column at the
    cap is orthonormalised once more.
    Returns (U, c, iterations, ||e|| of the last iteration).
    """
    U = np.asarray(V0, dtype=np.float64)
    ne = 0.0
    for t in range(1, t_cap + 1):
        U, _ = onorm(apply_S(L, U, delta, z))
        e = (X - U @ (U.T @ X)).sum(axis=1)
        ne = float(np.linalg.norm(e))
        c = U.shape[1]
        if ne > eps_h and c < c_max:
            U = np.concatenate([U, (e / ne)[:, None]], axis=1)
        elif ne < eps_l and c > c_min:
            U = U[:, :c - 1]
        else:
            return U, c, t, ne
    U, _ = onorm(U)
    return U, U.shape[1], t_cap, ne


def doi_paper_track(mesh: Mesh, X: np.ndarray, starts: np.ndarray, c0: int, eps_l: float,
                    eps_h: float, c_min: int = 1, c_max: int = 128, t_cap: int = 32,
                    delta: float = 1e-2, z: int = 1):
    """The paper's dynamic OI over all blocks in topological order (Sec. 5, Algorithm 2).

    A root starts from the first c0 columns of its rows of ``starts``; a child
    starts from its parent's final basis and width (c_i <- c_{i-1}, row
    transfer for unequal sizes).  Returns (U list, c array, iterations array).
    """
    k = mesh.k
    U = [None] * k
    cs = np.zeros(k, dtype=np.int64)
    its = np.zeros(k, dtype=np.int64)
    off = 0
    root_off = {}
    for b in range(k):
        if mesh.parent[b] < 0:
            root_off[b] = off
            off += mesh.blocks[b].verts.size
    for b in range(k):
        blk = mesh.blocks[b]
        n_b = blk.verts.size
        p = mesh.parent[b]
        V0 = starts[root_off[b]:root_off[b] + n_b, :c0] if p < 0 else row_transfer(U[p], n_b)
        U[b], cs[b], its[b], _ = doi_paper_block(
            laplacian(blk, mesh.literal_degree), X[blk.verts], V0, delta, z, eps_l, eps_h,
            c_min, min(c_max, n_b), t_cap)
    return U, cs, its


# ---------------------------------------------------------------------------
# Comparison metrics (sign- and rotation-free)
# ---------------------------------------------------------------------------

def principal_sines(U: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Sines of the principal angles between span(U) and span(W) (both orthonormal bases).

    cos(theta_i) are the singular values of U^T W; returned largest angle first.
    """
    cosv = np.linalg.svd(U.T @ W, compute_uv=False)
    cosv = np.clip(cosv, 0.0, 1.0)
    return np.sqrt(np.maximum(0.0, 1.0 - cosv * cosv))[::-1]


def max_sine(U: np.ndarray, W: np.ndarray) -> float:
    """Largest principal-angle sine, computed as ||(I - W W^T) U||_2 (accurate for small angles)."""
    return float(np.linalg.norm(U - W @ (W.T @ U), 2))


def projector_rel_error(U: np.ndarray, W: np.ndarray, X: np.ndarray) -> float:
    """||U U^T X - W W^T X||_F / ||W W^T X||_F."""
    a = U @ (U.T @ X)
    b = W @ (W.T @ X)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# Differentiable block low-pass filter (not in the paper: the coarse denoising
# filter v^ = U_c U_c^T v of Sec. 7.2 made differentiable in the per-edge
# weights of an edge-weighted Laplacian that reduces to Sec. 3's at w = 1)
# ---------------------------------------------------------------------------

def filter_forward_torch(mesh: Mesh, X, w, c: int, t_max: int, starts, delta: float = 1e-2):
    """Dense FP64 torch formulation of the filter, differentiable by torch autograd.

    Per block in order: V0 = the parent's final basis, detached (stop-gradient;
    a root starts from Onorm of its rows of ``starts``); t_max steps of
    Algorithm 1 (Sec. 4) with L(w) = D(w) - C(w), C_ij = w_e on the block's
    edges (``w`` concatenated over blocks in edge order), D_ii = sum_j C_ij,
    exact dense solves and Householder QR with diag(R) > 0; then
    X^_b = U_b U_b^T X_b.  Returns (X^ [n x 3] torch tensor, list of U).
    """
    import torch
    out = torch.zeros_like(X)
    U = [None] * mesh.k
    woff = 0
    root_off = {}
    off = 0
    for b in range(mesh.k):
        if mesh.parent[b] < 0:
            root_off[b] = off
            off += mesh.blocks[b].verts.size
    for b, blk in enumerate(mesh.blocks):
        n_b = blk.verts.size
        E_b = blk.edges.shape[0]
        wb = w[woff:woff + E_b]
        woff += E_b
        i = torch.as_tensor(blk.edges[:, 0])
        j = torch.as_tensor(blk.edges[:, 1])
        C = torch.zeros(n_b, n_b, dtype=torch.float64)
        C = C.index_put((i, j), wb).index_put((j, i), wb)
        L = torch.diag(C.sum(dim=1)) - C
        A = L + delta * torch.eye(n_b, dtype=torch.float64)
        p = mesh.parent[b]
        if p < 0:
            V = torch.as_tensor(starts[root_off[b]:root_off[b] + n_b, :c], dtype=torch.float64)
        else:
            V = torch.as_tensor(row_transfer(U[p].detach().numpy(), n_b))
        Q, R = torch.linalg.qr(V)
        V = Q * torch.sign(torch.diagonal(R))[None, :]
        for _ in range(t_max):
            Y = torch.linalg.solve(A, V)
            Q, R = torch.linalg.qr(Y)
            V = Q * torch.sign(torch.diagonal(R))[None, :]
        U[b] = V
        vb = torch.as_tensor(blk.verts)
        out = out.index_put((vb,), V @ (V.T @ X[vb]))
    return out, U


def filter_loss_grads(mesh: Mesh, X_noisy, X_clean, w, c: int, t_max: int, starts,
                      delta: float = 1e-2):
    """loss = ||filter(X_noisy) - X_clean||^2 and its gradients (d/dX_noisy, d/dw), FP64 autograd."""
    import torch
    X = torch.tensor(X_noisy, dtype=torch.float64, requires_grad=True)
    W = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    Xh, _ = filter_forward_torch(mesh, X, W, c, t_max, starts, delta)
    loss = ((Xh - torch.as_tensor(X_clean, dtype=torch.float64)) ** 2).sum()
    loss.backward()
    return float(loss.detach()), X.grad.numpy().copy(), W.grad.numpy().copy(), Xh.detach().numpy()
