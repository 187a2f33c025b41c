"""Splitting one mesh's block forest across ranks: host logic on the CPU.

Whole subtrees go to ranks (no exchange while tracking); every vertex is owned
by exactly one rank; one all-gather assembles the reconstruction.  Run with
the gloo backend at world size 2: every rank tracks its sub-forest with the
oracle (Algorithm 1 in its own block order) and the gathered reconstruction
must equal the single-process oracle's on the whole mesh.
"""
import os
import socket

import numpy as np
import pytest

from oracle import bsp_oracle as O
from paper_1810_02719_gb300 import forest, synth

torch = pytest.importorskip("torch")


def _mesh():
    N = 48
    xyz, faces = synth.torus(N, seed=2)
    ptr, verts = synth.bfs_partition(N, target_blocks=14, min_size=80, max_size=400, seed=4)
    ptr, verts, parent = synth.block_forest(ptr, verts, N, roots=5, seed=6)
    return N * N, xyz, faces, ptr, verts, parent


def _reconstruct(n, xyz, ptr, verts, parent, starts, c=12, t=2, faces=None, edges=None):
    om = O.build_mesh(n, ptr, verts, parent, faces=faces, edges=edges)
    U = O.oi_track(om, c, t, starts, delta=1e-2)
    return O.reconstruct(om, U, O.project(om, U, xyz), 3)


def test_split_is_a_partition_of_blocks_and_vertices():
    n, xyz, faces, ptr, verts, parent = _mesh()
    for world in (1, 2, 3, 5):
        parts = forest.split_forest(ptr, verts, parent, world)
        blocks = np.sort(np.concatenate([p.blocks for p in parts]))
        assert blocks.tolist() == list(range(len(ptr) - 1))
        owned = np.concatenate([p.block_verts for p in parts])
        assert np.sort(owned).tolist() == list(range(n))
        root = forest.subtree_root(parent)
        for p in parts:   # whole subtrees, parents local and earlier
            assert set(root[p.blocks]) <= set(p.roots.tolist())
            assert all(p.parent[i] < i for i in range(p.parent.size))
        loads = [p.n_vertices for p in parts]
        sub = np.bincount(root, weights=np.diff(ptr))
        assert max(loads) - min(loads) <= sub.max()   # greedy balance bound


def test_local_mesh_keeps_every_block_laplacian():
    n, xyz, faces, ptr, verts, parent = _mesh()
    om = O.build_mesh(n, ptr, verts, parent, faces=faces)
    for p in forest.split_forest(ptr, verts, parent, 2):
        xr, er, lp, lv, lpar = forest.local_mesh_inputs(xyz, faces, p)
        lom = O.build_mesh(xr.shape[0], lp, lv, lpar, edges=er)
        for i, b in enumerate(p.blocks):
            assert np.array_equal(O.laplacian(lom.blocks[i]), O.laplacian(om.blocks[b]))


def _rank(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, xyz, faces, ptr, verts, parent = _mesh()
        starts = synth.gaussian_starts(ptr, parent, 12, seed=3)
        part = forest.split_forest(ptr, verts, parent, world)[rank]
        xr, er, lp, lv, lpar = forest.local_mesh_inputs(xyz, faces, part)
        st = forest.local_starts(starts, ptr, parent, part)
        rows = _reconstruct(xr.shape[0], xr, lp, lv, lpar, st, edges=er)
        full = forest.gather_rows(torch.from_numpy(rows), part.block_verts, n)
        np.save(f"{out_path}.{rank}.npy", full.numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_gather_equals_single_process(tmp_path):
    import torch.multiprocessing as mp
    n, xyz, faces, ptr, verts, parent = _mesh()
    starts = synth.gaussian_starts(ptr, parent, 12, seed=3)
    ref = _reconstruct(n, xyz, ptr, verts, parent, starts, faces=faces)
    out = str(tmp_path / "gathered")
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        got = np.load(f"{out}.{r}.npy")
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _rank_bad(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = np.array([0, 1, 2]) if rank == 0 else np.array([2, 3])   # vertex 2 twice
        try:
            forest.gather_rows(torch.zeros(len(ids), 3, dtype=torch.float64), ids, 4)
            ok = False
        except ValueError:
            ok = True
        np.save(f"{out_path}.{rank}.npy", np.array([ok]))
    finally:
        dist.destroy_process_group()


def test_gather_rejects_overlapping_ownership(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "bad")
    mp.spawn(_rank_bad, args=(2, _free_port(), out), nprocs=2, join=True)
    assert all(bool(np.load(f"{out}.{r}.npy")[0]) for r in range(2))
