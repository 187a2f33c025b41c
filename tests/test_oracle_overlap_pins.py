"""Pins for the oracle's overlapped parts and degree-weighted average (Sec. 6.1,
Algorithm 3), and for the overlapped-part generator.

Checks: a path graph split into two overlapping parts whose merged values
are worked out by hand, degrees against a brute-force neighbour count, the
non-overlapping case equal to the plain reconstruction, exact recovery with
full bases, and the generator's equal sizes and multiplicities.
``test_overlap_planted_mistakes_are_caught`` plants slips on the CPU.
"""
import numpy as np
import pytest

from oracle import bsp_oracle as O
from paper_1810_02719_gb300 import synth


def path_two_parts():
    """Path 0-1-2-3-4; part A = [0, 1, 2, 3], part B = [2, 3, 4]."""
    ptr = np.array([0, 4, 7])
    verts = np.array([0, 1, 2, 3, 2, 3, 4])
    return O.build_overlapped_mesh(5, ptr, verts, [-1, 0], edges=synth.path_edges(5))


def check_hand_worked_average(O=O):
    mesh = path_two_parts()
    XA = np.array([[1.0], [2.0], [3.0], [4.0]])
    XB = np.array([[30.0], [40.0], [50.0]])
    out = O.weighted_average(mesh, [XA, XB], 1)
    # vertex 2: degree 2 in A (1, 3), 1 in B (3); vertex 3: 1 in A (2), 2 in B (2, 4)
    assert np.allclose(out[:, 0], [1.0, 2.0, (2 * 3 + 1 * 30) / 3, (1 * 4 + 2 * 40) / 3, 50.0])


def check_degrees_brute_force(O=O):
    N, T, r = 12, 4, 1
    xyz, faces = synth.torus(N)
    ptr, verts = synth.overlapped_tiles(N, T, r)
    mesh = O.build_overlapped_mesh(N * N, ptr, verts, synth.raster_chain(len(ptr) - 1),
                                   faces=faces)
    nbr = [set() for _ in range(N * N)]
    for a, b, c in faces.tolist():
        for u, v in ((a, b), (b, c), (c, a)):
            nbr[u].add(v)
            nbr[v].add(u)
    for b, blk in enumerate(mesh.blocks):
        inside = set(blk.verts.tolist())
        ref = [len(nbr[v] & inside) for v in blk.verts.tolist()]
        assert np.array_equal(O.block_degrees(blk), ref), b


def test_hand_worked_average():
    check_hand_worked_average()


def test_degrees_brute_force():
    check_degrees_brute_force()


def test_non_overlapping_parts_give_the_plain_reconstruction():
    N, T, c = 12, 4, 5
    xyz, faces = synth.torus(N, seed=1)
    ptr, verts = synth.overlapped_tiles(N, T, 0)
    parent = synth.raster_chain(len(ptr) - 1)
    om = O.build_overlapped_mesh(N * N, ptr, verts, parent, faces=faces)
    pm = O.build_mesh(N * N, ptr, verts, parent, faces=faces)
    U = [O.eigh_basis(O.laplacian(b), c)[0] for b in pm.blocks]
    ref = O.reconstruct(pm, U, O.project(pm, U, xyz), 3)
    assert np.allclose(O.reconstruct_overlapped(om, U, xyz), ref, atol=1e-13)


def test_full_bases_recover_the_mesh_and_equal_copies_stay():
    N, T, r = 12, 4, 1
    xyz, faces = synth.torus(N, seed=2)
    ptr, verts = synth.overlapped_tiles(N, T, r)
    om = O.build_overlapped_mesh(N * N, ptr, verts, synth.raster_chain(len(ptr) - 1),
                                 faces=faces)
    U = [np.linalg.eigh(O.laplacian(b))[1] for b in om.blocks]      # c = n_b
    assert np.allclose(O.reconstruct_overlapped(om, U, xyz), xyz, atol=1e-12)
    copies = [xyz[b.verts] for b in om.blocks]
    assert np.allclose(O.weighted_average(om, copies, 3), xyz, atol=1e-15)


def test_overlapped_tiles_generator():
    N, T, r = 16, 4, 1
    ptr, verts = synth.overlapped_tiles(N, T, r)
    k = (N // T) ** 2
    assert len(ptr) == k + 1 and np.all(np.diff(ptr) == (T + 2 * r) ** 2)
    mult = np.bincount(verts, minlength=N * N)
    assert set(np.unique(mult).tolist()) == {1, 2, 4}
    # every part holds its own tile
    tp, tv = synth.tile_partition(N, T)
    for b in range(k):
        assert set(tv[tp[b]:tp[b + 1]].tolist()) <= set(verts[ptr[b]:ptr[b + 1]].tolist())
    # r = 0 is the plain tile partition
    p0, v0 = synth.overlapped_tiles(N, T, 0)
    assert np.array_equal(p0, tp) and np.array_equal(v0, tv)


class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(O, k) for k in dir(O) if not k.startswith("__")})
        self.__dict__.update(over)


def test_overlap_planted_mistakes_are_caught():
    def plain_mean(mesh, Xb, cols):
        num = np.zeros((mesh.n, cols))
        cnt = np.zeros(mesh.n)
        for b, blk in enumerate(mesh.blocks):
            np.add.at(num, blk.verts, Xb[b])
            np.add.at(cnt, blk.verts, 1.0)
        return num / np.maximum(cnt, 1)[:, None]

    def degree_first_end_only(block):       # only the first end point of each edge
        d = np.zeros(block.verts.size, dtype=np.int64)
        np.add.at(d, block.edges[:, 0], 1)
        return d

    mutants = [
        (check_hand_worked_average, _Mutant(weighted_average=plain_mean)),
        (check_degrees_brute_force, _Mutant(block_degrees=degree_first_end_only)),
    ]
    for check, mut in mutants:
        with pytest.raises(AssertionError):
            check(O=mut)


def test_expanded_copies_keep_edges_without_faces():
    """A part holding both ends of an edge but no face around it keeps the edge."""
    faces = np.array([[0, 1, 2], [1, 3, 2]])
    ptr, verts = np.array([0, 3, 5]), np.array([0, 1, 2, 1, 2])     # part 1 = edge 1-2 only
    eptr, everts, eedges, orig = synth.expand_overlapped(ptr, verts, faces)
    assert np.array_equal(orig, verts)
    assert sorted(map(tuple, eedges.tolist())) == [(0, 1), (0, 2), (1, 2), (3, 4)]


def test_expanded_copies_reproduce_the_overlapped_parts():
    """Running the non-overlapping path on the expanded copies gives every part the same
    Laplacian as the overlapped part, and merging the copies' reconstructions by
    Algorithm 3 equals the overlapped reconstruction."""
    N, T, r, c = 12, 4, 1, 6
    xyz, faces = synth.torus(N, seed=3)
    ptr, verts = synth.overlapped_tiles(N, T, r)
    parent = synth.raster_chain(len(ptr) - 1)
    om = O.build_overlapped_mesh(N * N, ptr, verts, parent, faces=faces)
    eptr, everts, eedges, orig = synth.expand_overlapped(ptr, verts, faces)
    em = O.build_mesh(len(everts), eptr, everts, parent, edges=eedges)
    for a, b in zip(om.blocks, em.blocks):
        assert np.array_equal(O.laplacian(a), O.laplacian(b))
    U = [O.eigh_basis(O.laplacian(b), c)[0] for b in om.blocks]
    X_copies = xyz[orig]
    rec = O.reconstruct(em, U, O.project(em, U, X_copies), 3)        # one row per copy
    Xb = [rec[eb.verts] for eb in em.blocks]
    assert np.allclose(O.weighted_average(om, Xb, 3), O.reconstruct_overlapped(om, U, xyz),
                       atol=1e-13)
