"""Seeded synthetic meshes, partitions and random inputs.

This module only *generates inputs*: vertex positions, triangle faces, block
partitions, block orders (parent arrays) and the random numbers that the method
draws (root start matrices).  It holds none of the method's arithmetic (no
Laplacian, no solve, no orthonormalisation, no projection), so that both the
CUDA path and the CPU oracle can consume exactly the same arrays.

Workload shapes follow the paper's experiments: blocks of a few hundred to a
few thousand vertices (Sec. 6.2, Table "different_part_bunny": 69-1392 vertices
per segment; Sec. 8: ~512 and ~990 vertices per block), triangle meshes
M=(V,F) with edges derived from F (Sec. 3), partitioned into k blocks that are
processed in a topologically sorted order (Sec. 4).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_heightfield", "torus", "tile_partition", "raster_chain",
    "gaussian_starts", "bfs_partition", "block_forest", "torus_frames",
    "noisy_torus", "path_edges", "cycle_edges", "grid_edges", "rect_partition",
    "noisy_torus_patch",
]


def _quad_faces(N: int, M: int, wrap: bool) -> np.ndarray:
    """Triangulate an N x M vertex grid (vertex (i, j) -> i*M + j).

    Every quad (i,j),(i,j+1),(i+1,j),(i+1,j+1) is split along the diagonal
    (i,j)-(i+1,j+1) into two consistently oriented triangles.  With ``wrap``
    the grid closes in both directions (a torus).
    """
    ni = N if wrap else N - 1
    nj = M if wrap else M - 1
    i = np.arange(ni)[:, None]
    j = np.arange(nj)[None, :]
    i1 = (i + 1) % N
    j1 = (j + 1) % M
    v00 = (i * M + j).ravel()
    v01 = (i * M + j1).ravel()
    v10 = (i1 * M + j).ravel()
    v11 = (i1 * M + j1).ravel()
    t1 = np.stack([v00, v01, v11], axis=1)
    t2 = np.stack([v00, v11, v10], axis=1)
    faces = np.empty((2 * t1.shape[0], 3), dtype=np.int32)
    faces[0::2] = t1
    faces[1::2] = t2
    return faces


def grid_heightfield(N: int = 64, seed: int = 0, noise_sigma: float = 0.01):
    """Height-field grid: x, y on a unit N x N grid, z = sum of 3 seeded sinusoids.

    Amplitudes are drawn from U[0.05, 0.2]; spatial frequencies from
    U[0.5, 2.0] cycles per unit length; phases from U[0, 2*pi).  Gaussian noise
    of standard deviation ``noise_sigma`` is added to z.
    Returns (xyz float64 [N*N, 3], faces int32 [2(N-1)^2, 3]).
    """
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.05, 0.2, size=3)
    fx = rng.uniform(0.5, 2.0, size=3)
    fy = rng.uniform(0.5, 2.0, size=3)
    ph = rng.uniform(0.0, 2 * np.pi, size=3)
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    x = jj / (N - 1.0)
    y = ii / (N - 1.0)
    z = np.zeros_like(x)
    for a, u, v, p in zip(amp, fx, fy, ph):
        z += a * np.sin(2 * np.pi * (u * x + v * y) + p)
    z += rng.normal(0.0, noise_sigma, size=z.shape)
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)
    return xyz, _quad_faces(N, N, wrap=False)


def _periodic_gradient_noise(N: int, cells: int, rng) -> np.ndarray:
    """Periodic 2-D gradient (Perlin-style) noise sampled on an N x N grid.

    ``cells`` x ``cells`` lattice with seeded unit gradients, quintic fade
    6t^5 - 15t^4 + 10t^3, wrapping in both directions.  Values are roughly in
    [-0.7, 0.7].
    """
    ang = rng.uniform(0.0, 2 * np.pi, size=(cells, cells))
    gx, gy = np.cos(ang), np.sin(ang)
    s = np.arange(N) * (cells / N)
    u, v = np.meshgrid(s, s, indexing="ij")
    a0 = np.floor(u).astype(np.int64)
    b0 = np.floor(v).astype(np.int64)
    fu, fv = u - a0, v - b0
    a1, b1 = (a0 + 1) % cells, (b0 + 1) % cells
    a0, b0 = a0 % cells, b0 % cells

    def corner(a, b, du, dv):
        return gx[a, b] * du + gy[a, b] * dv

    n00 = corner(a0, b0, fu, fv)
    n10 = corner(a1, b0, fu - 1, fv)
    n01 = corner(a0, b1, fu, fv - 1)
    n11 = corner(a1, b1, fu - 1, fv - 1)
    fade = lambda t: t * t * t * (t * (6 * t - 15) + 10)  # noqa: E731
    wu, wv = fade(fu), fade(fv)
    nx0 = n00 + wu * (n10 - n00)
    nx1 = n01 + wu * (n11 - n01)
    return nx0 + wv * (nx1 - nx0)


def torus(N: int = 1024, R: float = 1.0, r: float = 0.35, amp: float = 0.02,
          seed: int = 0, cells: int = 16):
    """Closed torus from an N x N parametric grid with a seeded radial perturbation.

    Vertex (i, j) sits at angles u = 2*pi*i/N (around the axis) and
    v = 2*pi*j/N (around the tube); its tube radius is r + amp * noise(i, j)
    with periodic gradient noise.  Returns (xyz float64 [N*N, 3],
    faces int32 [2 N^2, 3]).
    """
    rng = np.random.default_rng(seed)
    noise = _periodic_gradient_noise(N, cells, rng)
    u = 2 * np.pi * np.arange(N)[:, None] / N
    v = 2 * np.pi * np.arange(N)[None, :] / N
    rr = r + amp * noise
    x = (R + rr * np.cos(v)) * np.cos(u)
    y = (R + rr * np.cos(v)) * np.sin(u)
    z = rr * np.sin(v) * np.ones_like(u)
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)
    return xyz, _quad_faces(N, N, wrap=True)


def tile_partition(N: int, T: int):
    """Partition an N x N vertex grid into (N/T)^2 square tiles of T x T vertices.

    Tiles are numbered in raster order; inside a tile, vertices are listed in
    row-major order (this is the block's local vertex order).
    Returns (block_ptr int32 [k+1], block_verts int32 [N*N]).
    """
    assert N % T == 0
    nt = N // T
    verts = np.empty(N * N, dtype=np.int32)
    ptr = np.arange(nt * nt + 1, dtype=np.int32) * (T * T)
    li, lj = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    for bi in range(nt):
        for bj in range(nt):
            b = bi * nt + bj
            g = (bi * T + li) * N + (bj * T + lj)
            verts[ptr[b]:ptr[b + 1]] = g.ravel()
    return ptr, verts


def overlapped_tiles(N: int, T: int, r: int):
    """Overlapped equal-size parts of an N x N periodic (torus) vertex grid.

    Every T x T tile is extended by r rings of neighbouring vertices on each
    side (wrapping around), so every part has (T + 2 r)^2 vertices and the
    vertices within r of a tile border appear in 2 or 4 parts.  Parts in
    raster order; inside a part, row-major local order.
    Returns (block_ptr int32 [k+1], block_verts int32 [k (T + 2 r)^2]).
    """
    assert N % T == 0 and 0 <= r and T + 2 * r <= N
    nt = N // T
    S = T + 2 * r
    ptr = np.arange(nt * nt + 1, dtype=np.int32) * (S * S)
    verts = np.empty(nt * nt * S * S, dtype=np.int32)
    li, lj = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    for bi in range(nt):
        for bj in range(nt):
            b = bi * nt + bj
            g = ((bi * T - r + li) % N) * N + ((bj * T - r + lj) % N)
            verts[ptr[b]:ptr[b + 1]] = g.ravel()
    return ptr, verts


def expand_overlapped(block_ptr, block_verts, faces):
    """Non-overlapping copy of an overlapped partition: every (part, vertex) pair
    becomes its own vertex, and every part keeps the mesh edges whose two end
    points it holds, re-indexed to its copies (an edge list, since a part may
    hold an edge without holding a face around it).  A library that needs each
    vertex in one block can then process the parts as they are; the copies are
    merged back afterwards (``orig`` maps each copy to its vertex).
    Returns (block_ptr, block_verts = arange, edges of the copies [E x 2], orig).
    """
    ptr = np.asarray(block_ptr, dtype=np.int64)
    bv = np.asarray(block_verts, dtype=np.int64)
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    n = int(max(bv.max(), f.max())) + 1
    out = []
    for b in range(len(ptr) - 1):
        loc = np.full(n, -1, dtype=np.int64)
        loc[bv[ptr[b]:ptr[b + 1]]] = np.arange(ptr[b], ptr[b + 1])
        le = loc[e]
        out.append(le[np.all(le >= 0, axis=1)])
    return (ptr.astype(np.int32), np.arange(ptr[-1], dtype=np.int32),
            np.concatenate(out).astype(np.int32), bv.astype(np.int32))


def rect_partition(R: int, C: int, TR: int, TC: int):
    """Partition an R x C vertex grid into (R/TR)(C/TC) rectangular tiles of TR x TC.

    Raster tile order; row-major vertex order inside a tile.
    Returns (block_ptr int32 [k+1], block_verts int32 [R*C]).
    """
    assert R % TR == 0 and C % TC == 0
    nr, nc = R // TR, C // TC
    ptr = np.arange(nr * nc + 1, dtype=np.int32) * (TR * TC)
    verts = np.empty(R * C, dtype=np.int32)
    li, lj = np.meshgrid(np.arange(TR), np.arange(TC), indexing="ij")
    for bi in range(nr):
        for bj in range(nc):
            b = bi * nc + bj
            verts[ptr[b]:ptr[b + 1]] = ((bi * TR + li) * C + (bj * TC + lj)).ravel()
    return ptr, verts


def noisy_torus_patch(R: int = 40, C: int = 50, N: int = 512, noise_factor: float = 0.3,
                      seed: int = 0):
    """An open R x C patch (rows/columns 0..R-1, 0..C-1) of the N x N noisy torus.

    Returns (clean xyz [R*C, 3], noisy xyz [R*C, 3], faces of the open R x C grid).
    """
    clean, noisy, _ = noisy_torus(N=N, noise_factor=noise_factor, seed=seed)
    idx = (np.arange(R)[:, None] * N + np.arange(C)[None, :]).ravel()
    return clean[idx].copy(), noisy[idx].copy(), _quad_faces(R, C, wrap=False)


def raster_chain(k: int) -> np.ndarray:
    """Block order as one chain: block b is warm-started from block b-1; block 0 is the root."""
    parent = np.arange(-1, k - 1, dtype=np.int32)
    return parent


def gaussian_starts(block_ptr, parent, c: int, seed: int = 0) -> np.ndarray:
    """Seeded standard-normal start matrices for the root blocks.

    One n_b x c block per root (parent == -1), concatenated row-wise in block
    order, float64.  The method orthonormalises them itself (the paper starts
    from an orthonormal subspace, Sec. 4); these are only the random draws.
    """
    rng = np.random.default_rng(seed)
    sizes = np.diff(np.asarray(block_ptr))
    roots = np.nonzero(np.asarray(parent) < 0)[0]
    rows = int(sizes[roots].sum())
    return rng.standard_normal((rows, c))


# ---------------------------------------------------------------------------
# Edge-list graphs with closed-form spectra (used to pin the oracle).
# ---------------------------------------------------------------------------

def path_edges(n: int) -> np.ndarray:
    """Edges of the path graph P_n (0-1-2-...-(n-1))."""
    a = np.arange(n - 1, dtype=np.int32)
    return np.stack([a, a + 1], axis=1)


def cycle_edges(n: int) -> np.ndarray:
    """Edges of the cycle graph C_n."""
    a = np.arange(n, dtype=np.int32)
    return np.stack([a, (a + 1) % n], axis=1).astype(np.int32)


def grid_edges(a: int, b: int) -> np.ndarray:
    """Edges of the 4-neighbour grid graph P_a x P_b (vertex (i, j) -> i*b + j)."""
    e = []
    for i in range(a):
        for j in range(b):
            v = i * b + j
            if j + 1 < b:
                e.append((v, v + 1))
            if i + 1 < a:
                e.append((v, v + b))
    return np.asarray(e, dtype=np.int32).reshape(-1, 2)


# ---------------------------------------------------------------------------
# Uneven BFS partition and block forest (batched workload).
# ---------------------------------------------------------------------------

def _grid_neighbours(N: int):
    """4-neighbour lattice adjacency of the N x N torus grid as an [N*N, 4] array."""
    idx = np.arange(N * N).reshape(N, N)
    nb = np.stack([
        np.roll(idx, 1, 0).ravel(), np.roll(idx, -1, 0).ravel(),
        np.roll(idx, 1, 1).ravel(), np.roll(idx, -1, 1).ravel(),
    ], axis=1)
    return nb


def bfs_partition(N: int = 1024, target_blocks: int = 2000, min_size: int = 300,
                  max_size: int = 3000, seed: int = 0):
    """Seeded region growing of an N x N torus grid into connected, uneven blocks.

    Seeds are drawn with a density that varies smoothly around the torus, so
    block sizes spread over [min_size, max_size].  Regions grow by a
    multi-source breadth-first search in which every region advances a
    seeded number of rings per round (growth speed 1-4), then blocks smaller
    than ``min_size`` merge into their smallest neighbour and blocks larger
    than ``max_size`` split by BFS from their first vertex.  Every block is
    connected in the 4-neighbour lattice (hence in the triangulation).  Local
    vertex order inside a block is BFS order from the block's seed.
    Returns (block_ptr int32 [k+1], block_verts int32 [N*N]).
    """
    rng = np.random.default_rng(seed)
    n = N * N
    nb = _grid_neighbours(N)
    # Seed density varies with the angle around the axis: 0.25x .. 1.75x.
    i = np.arange(N)
    dens_row = 1.0 + 0.75 * np.sin(2 * np.pi * i / N + rng.uniform(0, 2 * np.pi))
    p = np.repeat(dens_row, N)
    p = p / p.sum()
    seeds = rng.choice(n, size=target_blocks, replace=False, p=p)
    speed = rng.integers(1, 5, size=target_blocks)
    owner = np.full(n, -1, dtype=np.int64)
    owner[seeds] = np.arange(target_blocks)
    fronts = [np.array([s]) for s in seeds]
    active = True
    while active:
        active = False
        for rnd in range(4):
            for b in range(target_blocks):
                if speed[b] <= rnd or fronts[b].size == 0:
                    continue
                cand = np.unique(nb[fronts[b]].ravel())
                cand = cand[owner[cand] < 0]
                owner[cand] = b
                fronts[b] = cand
                if cand.size:
                    active = True
    assert (owner >= 0).all()
    blocks = _components_to_lists(owner, nb, seeds)
    blocks = _merge_small(blocks, nb, n, min_size)
    blocks = _split_large(blocks, nb, n, max_size, min_size)
    # Renumber: order blocks by their first vertex, BFS order inside.
    ptr = np.zeros(len(blocks) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(b) for b in blocks])
    verts = np.concatenate(blocks).astype(np.int32)
    assert np.array_equal(np.sort(verts), np.arange(n))
    return ptr.astype(np.int32), verts


def _bfs_order(members: np.ndarray, start: int, nb: np.ndarray, n: int) -> np.ndarray:
    inside = np.zeros(n, dtype=bool)
    inside[members] = True
    seen = np.zeros(n, dtype=bool)
    order = [start]
    seen[start] = True
    head = 0
    while head < len(order):
        v = order[head]
        head += 1
        for w in nb[v]:
            if inside[w] and not seen[w]:
                seen[w] = True
                order.append(w)
    return np.asarray(order, dtype=np.int64)


def _components_to_lists(owner, nb, seeds):
    n = owner.size
    lists = []
    for b, s in enumerate(seeds):
        members = np.nonzero(owner == b)[0]
        if members.size == 0:
            continue
        order = _bfs_order(members, s, nb, n)
        lists.append(order)
        rest = np.setdiff1d(members, order)
        while rest.size:  # disconnected leftovers become their own pieces
            o = _bfs_order(rest, rest[0], nb, n)
            lists.append(o)
            rest = np.setdiff1d(rest, o)
    return lists


def _merge_small(blocks, nb, n, min_size):
    owner = np.empty(n, dtype=np.int64)
    for b, m in enumerate(blocks):
        owner[m] = b
    sizes = np.array([len(m) for m in blocks])
    alive = np.ones(len(blocks), dtype=bool)
    members = [list(m) for m in blocks]
    changed = True
    while changed:
        changed = False
        for b in np.argsort(sizes):
            if not alive[b] or sizes[b] >= min_size:
                continue
            nbrs = np.unique(owner[nb[np.asarray(members[b])].ravel()])
            nbrs = nbrs[(nbrs != b)]
            nbrs = nbrs[alive[nbrs]]
            if nbrs.size == 0:
                continue
            t = nbrs[np.argmin(sizes[nbrs])]
            members[t].extend(members[b])
            owner[np.asarray(members[b])] = t
            sizes[t] += sizes[b]
            alive[b] = False
            changed = True
    out = []
    for b in range(len(blocks)):
        if alive[b]:
            m = np.asarray(members[b])
            out.append(_bfs_order(m, m[0], nb, n))
    return out


def _split_large(blocks, nb, n, max_size, min_size):
    out = []
    work = list(blocks)
    while work:
        m = work.pop()
        if len(m) <= max_size:
            out.append(m)
            continue
        order = _bfs_order(m, m[0], nb, n)
        half = len(order) // 2
        a = order[:half]
        b = np.setdiff1d(m, a)
        # BFS prefixes are connected; the remainder may not be: re-split pieces.
        rest = b
        pieces = []
        while rest.size:
            o = _bfs_order(rest, rest[0], nb, n)
            pieces.append(o)
            rest = np.setdiff1d(rest, o)
        work.append(_bfs_order(a, a[0], nb, n))
        for pc in pieces:
            work.append(pc)
    # Tiny pieces produced by splits are merged back.
    return _merge_small(out, nb, n, min_size)


def block_forest(block_ptr, block_verts, N: int, roots: int, seed: int = 0):
    """Warm-start forest over the block adjacency graph, in topological order.

    ``roots`` root blocks are picked by farthest-point sampling over block
    adjacency hops (the first one seeded), then a multi-source BFS assigns each
    other block the already-visited neighbour it was reached from as parent.
    Blocks are renumbered in BFS order so that parent[b] < b.
    Returns (block_ptr, block_verts, parent) after renumbering.
    """
    rng = np.random.default_rng(seed)
    k = len(block_ptr) - 1
    owner = np.empty(N * N, dtype=np.int64)
    for b in range(k):
        owner[block_verts[block_ptr[b]:block_ptr[b + 1]]] = b
    nb = _grid_neighbours(N)
    src = np.repeat(owner, 4)
    dst = owner[nb.ravel()]
    mask = src != dst
    pairs = np.unique(np.stack([src[mask], dst[mask]], axis=1), axis=0)
    adj = [[] for _ in range(k)]
    for a, b in pairs:
        adj[a].append(b)

    def hops_from(sources):
        d = np.full(k, np.iinfo(np.int64).max)
        q = list(sources)
        for s in sources:
            d[s] = 0
        h = 0
        while h < len(q):
            v = q[h]
            h += 1
            for w in adj[v]:
                if d[w] > d[v] + 1:
                    d[w] = d[v] + 1
                    q.append(w)
        return d

    chosen = [int(rng.integers(k))]
    dist = hops_from(chosen)
    while len(chosen) < roots:
        nxt = int(np.argmax(dist))
        chosen.append(nxt)
        dist = np.minimum(dist, hops_from([nxt]))
    parent_old = np.full(k, -2, dtype=np.int64)
    order = []
    for r in chosen:
        parent_old[r] = -1
        order.append(r)
    h = 0
    while h < len(order):
        v = order[h]
        h += 1
        for w in adj[v]:
            if parent_old[w] == -2:
                parent_old[w] = v
                order.append(w)
    assert len(order) == k
    new_id = np.empty(k, dtype=np.int64)
    new_id[np.asarray(order)] = np.arange(k)
    sizes = np.diff(block_ptr)
    new_ptr = np.zeros(k + 1, dtype=np.int64)
    new_ptr[1:] = np.cumsum(sizes[np.asarray(order)])
    new_verts = np.concatenate([block_verts[block_ptr[b]:block_ptr[b + 1]] for b in order])
    parent = np.array([-1 if parent_old[b] < 0 else new_id[parent_old[b]] for b in order],
                      dtype=np.int32)
    assert all(parent[b] < b for b in range(k))
    return new_ptr.astype(np.int32), new_verts.astype(np.int32), parent


# ---------------------------------------------------------------------------
# Dynamic mesh (fixed connectivity, many frames) and the noisy torus.
# ---------------------------------------------------------------------------

def torus_frames(N: int = 512, frames: int = 200, seed: int = 0, R: float = 1.0,
                 r: float = 0.35, max_twist: float = 0.5, wave_amp: float = 0.05):
    """A frame sequence of one torus with fixed connectivity.

    Frame f twists the torus about its axis (z): a point at height z turns by
    theta_f * z / r, with theta_f drawn from U[-max_twist, max_twist]; and adds
    a travelling sine wave of amplitude ``wave_amp`` to the tube radius,
    wave_amp * sin(3 u + 2 v - 2 pi f / 25).
    Returns (frames_xyz float64 [frames, N*N, 3], faces int32).
    """
    rng = np.random.default_rng(seed)
    base_noise = _periodic_gradient_noise(N, 16, rng)
    theta = rng.uniform(-max_twist, max_twist, size=frames)
    u = 2 * np.pi * np.arange(N)[:, None] / N
    v = 2 * np.pi * np.arange(N)[None, :] / N
    out = np.empty((frames, N * N, 3), dtype=np.float64)
    for f in range(frames):
        rr = r + 0.02 * base_noise + wave_amp * np.sin(3 * u + 2 * v - 2 * np.pi * f / 25.0)
        x = (R + rr * np.cos(v)) * np.cos(u)
        y = (R + rr * np.cos(v)) * np.sin(u)
        z = rr * np.sin(v)
        ang = theta[f] * z / r
        xr = x * np.cos(ang) - y * np.sin(ang)
        yr = x * np.sin(ang) + y * np.cos(ang)
        out[f] = np.stack([xr.ravel(), yr.ravel(), z.ravel()], axis=1)
    return out, _quad_faces(N, N, wrap=True)


def noisy_torus(N: int = 512, noise_factor: float = 0.3, seed: int = 0):
    """Clean torus plus isotropic Gaussian noise of sigma = noise_factor x mean edge length.

    Returns (clean xyz, noisy xyz, faces).  The mean edge length is measured on
    the clean grid's three edge families (along u, along v, and the quad
    diagonal), each of which holds N*N edges.
    """
    clean, faces = torus(N=N, seed=seed)
    g = clean.reshape(N, N, 3)
    d1 = np.linalg.norm(np.roll(g, -1, 0) - g, axis=2)
    d2 = np.linalg.norm(np.roll(g, -1, 1) - g, axis=2)
    d3 = np.linalg.norm(np.roll(np.roll(g, -1, 0), -1, 1) - g, axis=2)
    mean_len = (d1.mean() + d2.mean() + d3.mean()) / 3.0
    rng = np.random.default_rng(seed + 1)
    noisy = clean + rng.normal(0.0, noise_factor * mean_len, size=clean.shape)
    return clean, noisy, faces
