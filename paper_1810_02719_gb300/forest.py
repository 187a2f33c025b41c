"""Splitting one mesh's block forest across ranks (one process per GPU).

A block warm-starts only from its parent (Sec. 4), so the subtrees of the
block forest are independent problems: whole subtrees go to ranks (largest
first, each to the rank with the fewest vertices so far), every rank tracks
its own sub-forest with its own bsp_mesh, and no data moves between ranks
until the results are assembled.  Each vertex belongs to exactly one block,
hence to exactly one rank; one all-gather of (vertex ids, rows) gives every
rank the whole reconstruction.  Host logic only (numpy and
torch.distributed); the GPU work stays in the library.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np


@dataclass
class RankPart:
    """The blocks one rank tracks, re-indexed as a mesh of their own."""
    blocks: np.ndarray        # global block ids, in global (topological) order
    block_ptr: np.ndarray     # int32 [kr + 1]
    block_verts: np.ndarray   # int32: global vertex ids of the rank's blocks, block by block
    parent: np.ndarray        # int32 [kr]: parents as local block ids (-1 = root)
    roots: np.ndarray         # global block ids of the rank's roots, in local order

    @property
    def n_vertices(self) -> int:
        return int(self.block_verts.size)


def subtree_root(parent) -> np.ndarray:
    """Root block of every block (parents come before their children)."""
    parent = np.asarray(parent)
    root = np.arange(parent.size)
    for b in range(parent.size):
        if parent[b] >= 0:
            if parent[b] >= b:
                raise ValueError("parent[b] must precede b")
            root[b] = root[parent[b]]
    return root


def split_forest(block_ptr, block_verts, parent, world: int) -> List[RankPart]:
    """Whole subtrees per rank, balanced by vertex count (largest subtree first,
    to the least loaded rank; ties to the lowest rank)."""
    ptr = np.asarray(block_ptr, dtype=np.int64)
    bv = np.asarray(block_verts, dtype=np.int64)
    parent = np.asarray(parent, dtype=np.int64)
    k = parent.size
    root = subtree_root(parent)
    sizes = np.diff(ptr)
    roots = np.nonzero(parent < 0)[0]
    load = np.bincount(root, weights=sizes, minlength=k)
    owner_of_root = {}
    totals = np.zeros(world)
    for r in sorted(roots.tolist(), key=lambda r: (-load[r], r)):
        w = int(np.argmin(totals))
        owner_of_root[r] = w
        totals[w] += load[r]
    owner = np.array([owner_of_root[root[b]] for b in range(k)], dtype=np.int64)
    parts = []
    for w in range(world):
        blocks = np.nonzero(owner == w)[0]
        local = np.full(k, -1, dtype=np.int64)
        local[blocks] = np.arange(blocks.size)
        lptr = np.zeros(blocks.size + 1, dtype=np.int64)
        lptr[1:] = np.cumsum(sizes[blocks])
        lverts = np.concatenate([bv[ptr[b]:ptr[b + 1]] for b in blocks]) if blocks.size \
            else np.zeros(0, dtype=np.int64)
        lpar = np.where(parent[blocks] >= 0, local[np.maximum(parent[blocks], 0)], -1)
        parts.append(RankPart(blocks=blocks, block_ptr=lptr.astype(np.int32),
                              block_verts=lverts.astype(np.int32), parent=lpar.astype(np.int32),
                              roots=blocks[parent[blocks] < 0]))
    return parts


def local_starts(starts, block_ptr, parent, part: RankPart) -> np.ndarray:
    """The rows of the global root-start matrix (roots concatenated in global
    block order) that belong to the rank's roots, in the rank's order."""
    ptr = np.asarray(block_ptr, dtype=np.int64)
    parent = np.asarray(parent)
    off, o = {}, 0
    for b in range(parent.size):
        if parent[b] < 0:
            off[b] = o
            o += int(ptr[b + 1] - ptr[b])
    rows = [starts[off[r]:off[r] + int(ptr[r + 1] - ptr[r])] for r in part.roots]
    return np.concatenate(rows) if rows else starts[:0]


def local_mesh_inputs(xyz, faces, part: RankPart):
    """A rank's own mesh: its vertices renumbered 0 .. n_r - 1 in block order and
    every mesh edge (side of a face) with both end points on the rank, as an
    edge list (a face may have a vertex on another rank while its side lies
    inside one of this rank's blocks).  Every block keeps its induced edges.
    Returns (xyz_r, edges_r int32 [E_r x 2], block_ptr, block_verts = arange,
    parent)."""
    gv = part.block_verts.astype(np.int64)
    n = int(np.asarray(xyz).shape[0])
    loc = np.full(n, -1, dtype=np.int64)
    loc[gv] = np.arange(gv.size)
    f = np.asarray(faces, dtype=np.int64).reshape(-1, 3)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    le = loc[e]
    le = le[np.all(le >= 0, axis=1)]
    return (np.asarray(xyz)[gv], le.astype(np.int32), part.block_ptr,
            np.arange(gv.size, dtype=np.int32), part.parent)


def gather_rows(rows, vertex_ids, n: int, group=None):
    """All-gather every rank's rows (torch tensor [n_r x cols], rank-local
    vertex order) with their global vertex ids (int64 [n_r]) into the full
    [n x cols] array on every rank.  Ranks send equal-size padded buffers (one
    all_gather for the ids, one for the rows); vertex ownership must be a
    partition of range(n)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = rows.device
    cnt = torch.tensor([rows.shape[0]], dtype=torch.int64, device=dev)
    cnts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(cnts, cnt, group=group)
    m = int(max(int(c.item()) for c in cnts))
    cols = rows.shape[1]
    pad_rows = torch.zeros((m, cols), dtype=rows.dtype, device=dev)
    pad_rows[:rows.shape[0]] = rows
    pad_ids = torch.full((m,), -1, dtype=torch.int64, device=dev)
    pad_ids[:rows.shape[0]] = torch.as_tensor(vertex_ids, dtype=torch.int64, device=dev)
    all_rows = [torch.empty_like(pad_rows) for _ in range(world)]
    all_ids = [torch.empty_like(pad_ids) for _ in range(world)]
    dist.all_gather(all_rows, pad_rows, group=group)
    dist.all_gather(all_ids, pad_ids, group=group)
    out = torch.zeros((n, cols), dtype=rows.dtype, device=dev)
    seen = torch.zeros(n, dtype=torch.int64, device=dev)
    for r in range(world):
        c = int(cnts[r].item())
        ids = all_ids[r][:c]
        out[ids] = all_rows[r][:c]
        seen[ids] += 1
    if not bool(torch.all(seen == 1)):
        raise ValueError("vertex ownership is not a partition of the mesh")
    return out
