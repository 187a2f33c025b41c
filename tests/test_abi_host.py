"""CPU-only checks: the C ABI library loads and exports every declared entry
point, and the host-side input generators produce valid partitions and block
forests (no GPU needed)."""
import os
import re
import ctypes

import numpy as np
import pytest

from paper_1810_02719_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "bsp.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(bsp_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["bsp_mesh_create", "bsp_oi_track", "bsp_oi_track_dynamic", "bsp_project",
                 "bsp_reconstruct", "bsp_mesh_destroy", "bsp_last_error", "bsp_spmm"]:
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_1810_02719_gb300 import build
    build.build()
    from paper_1810_02719_gb300 import bsp
    lib = ctypes.CDLL(bsp.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(bsp.exported_symbols()) <= set(declared_symbols())
    o = bsp.bsp_opts_default()
    assert o.delta == pytest.approx(1e-2) and o.z == 1 and o.precision == bsp.BSP_PREC_MIXED


def test_tile_partition_covers_once():
    ptr, verts = synth.tile_partition(64, 16)
    assert len(ptr) == 17 and ptr[-1] == 4096
    assert np.array_equal(np.sort(verts), np.arange(4096))
    # tile 5 = (1, 1): rows 16..31, cols 16..31, row-major
    t = verts[ptr[5]:ptr[6]].reshape(16, 16)
    assert t[0, 0] == 16 * 64 + 16 and t[0, 1] == 16 * 64 + 17 and t[1, 0] == 17 * 64 + 16


def test_torus_faces_close_the_surface():
    xyz, faces = synth.torus(32)
    assert faces.shape == (2 * 32 * 32, 3) and faces.min() == 0 and faces.max() == 32 * 32 - 1
    # closed surface: every undirected side is shared by exactly two faces
    e = np.sort(np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]]), axis=1)
    _, counts = np.unique(e, axis=0, return_counts=True)
    assert np.all(counts == 2)
    # Euler characteristic of a torus: V - E + F = 0
    assert 32 * 32 - len(counts) + faces.shape[0] == 0


def test_bfs_partition_and_forest_small():
    N = 64
    ptr, verts = synth.bfs_partition(N, target_blocks=20, min_size=60, max_size=600, seed=0)
    sizes = np.diff(ptr)
    assert sizes.min() >= 60 and sizes.max() <= 600
    assert np.array_equal(np.sort(verts), np.arange(N * N))
    # each block is connected in the 4-neighbour lattice
    owner = np.empty(N * N, int)
    for b in range(len(sizes)):
        owner[verts[ptr[b]:ptr[b + 1]]] = b
    for b in range(len(sizes)):
        m = verts[ptr[b]:ptr[b + 1]]
        seen = {int(m[0])}
        stack = [int(m[0])]
        while stack:
            v = stack.pop()
            i, j = divmod(v, N)
            for w in (((i + 1) % N) * N + j, ((i - 1) % N) * N + j, i * N + (j + 1) % N,
                      i * N + (j - 1) % N):
                if owner[w] == b and w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert len(seen) == m.size
    p2, v2, parent = synth.block_forest(ptr, verts, N, roots=3, seed=1)
    assert (parent < np.arange(len(parent))).all() and (parent == -1).sum() == 3
    assert np.array_equal(np.sort(v2), np.arange(N * N))


def test_gaussian_starts_shape():
    ptr = np.array([0, 10, 30, 45])
    parent = np.array([-1, 0, -1])
    g = synth.gaussian_starts(ptr, parent, 4, seed=0)
    assert g.shape == (10 + 15, 4)
