"""Pins for the oracle's octree: interaction lists against brute force and
the FMM partition property (every leaf pair is near exactly once or far at
exactly one level)."""
import numpy as np

from oracle import octree


def _setup(seed, n=400, level=None):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3)) * np.array([3.0, 2.4, 2.0])
    T = octree.Octree(pts, pts, rc=0.05, leaf_max=8, level=level)
    return T, pts


def test_morton_roundtrip():
    rng = np.random.default_rng(0)
    ix, iy, iz = rng.integers(0, 1 << 10, (3, 100))
    k = octree.morton(ix, iy, iz, 10)
    a, b, c = octree.demorton(k, 10)
    assert np.all(a == ix) and np.all(b == iy) and np.all(c == iz)
    assert octree.morton(1, 0, 0, 1) == 1 and octree.morton(0, 1, 0, 1) == 2 and octree.morton(0, 0, 1, 1) == 4


def test_leaf_assignment_and_level_rule():
    T, pts = _setup(1)
    d = T.delta(T.L)
    c = np.floor((pts - T.origin) / d).astype(int)
    key = octree.morton(c[:, 0], c[:, 1], c[:, 2], T.L)
    assert np.all(key == T.elem_key)
    assert T.leaf_count.max() <= 8 or T.delta(T.L + 1) <= 0.05
    # sorted order is stable by index inside a leaf
    for s, n in zip(T.leaf_start, T.leaf_count):
        seg = T.perm[s:s + n]
        assert np.all(np.diff(seg) > 0)


def test_lists_brute_force():
    T, _ = _setup(2)
    L = T.L
    coords = {l: np.stack(octree.demorton(T.levels[l], l), 1) for l in range(L + 1)}
    U = set(map(tuple, T.ulist()))
    cl = coords[L]
    for a in range(len(cl)):
        for b in range(len(cl)):
            near = max(abs(int(cl[a][i]) - int(cl[b][i])) for i in range(3)) <= 1
            assert ((a, b) in U) == near
    for l in range(2, L + 1):
        V = set(map(tuple, T.vlist(l)))
        c = coords[l]
        for a in range(len(c)):
            for b in range(len(c)):
                adj = max(abs(int(c[a][i]) - int(c[b][i])) for i in range(3)) <= 1
                padj = max(abs(int(c[a][i]) // 2 - int(c[b][i]) // 2) for i in range(3)) <= 1
                assert ((a, b) in V) == ((not adj) and padj)
        assert len(V) == 0 or max(sum(1 for (t, s) in V if t == a) for a in range(len(c))) <= 189


def test_partition_property():
    T, _ = _setup(3, n=600)
    L = T.L
    U = set(map(tuple, T.ulist()))
    V = {l: set(map(tuple, T.vlist(l))) for l in range(2, L + 1)}
    anc = {L: np.arange(len(T.levels[L]))}
    for l in range(L - 1, 1, -1):
        anc[l] = T.parent_index(l + 1)[anc[l + 1]]
    nl = len(T.levels[L])
    for t in range(nl):
        for s in range(nl):
            hits = int((t, s) in U)
            for l in range(2, L + 1):
                hits += int((int(anc[l][t]), int(anc[l][s])) in V[l])
            assert hits == 1
