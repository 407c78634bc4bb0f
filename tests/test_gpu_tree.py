"""GPU octree vs the oracle octree: element order, leaves, boxes of every
level, U-lists and V-lists must agree exactly (integer work)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import oracle_mesh, workload


@pytest.mark.parametrize("name", ["small", "sub", "ragged", "full"])
def test_tree_bit_exact(name):
    from oracle.octree import Octree
    wl = workload(name)
    om = oracle_mesh(name)
    el = om.el
    T = Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, om.rc, 64)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    tree = fb.fb_tree_build(mesh, 64)
    try:
        L, org, side, nb = fb.fb_tree_info(tree)
        assert L == T.L
        assert side == T.side and np.array_equal(org, T.origin)
        assert np.array_equal(fb.fb_tree_export(tree, 0), T.perm)
        ls = fb.fb_tree_export(tree, 1)
        assert np.array_equal(ls[:-1], T.leaf_start) and ls[-1] == wl.n
        for lev in range(L + 1):
            assert np.array_equal(fb.fb_tree_export(tree, 2, lev), T.levels[lev])
        if name != "full":
            assert np.array_equal(fb.fb_tree_export(tree, 3), T.ulist())
            for lev in range(2, L + 1):
                assert np.array_equal(fb.fb_tree_export(tree, 4, lev), T.vlist(lev))
    finally:
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
