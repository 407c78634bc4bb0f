"""Expansion orders beyond one shared-memory tile: a coarse 3,072-element
shoebox at 7.5 kHz has order 116 at level 2 and 66 at level 3, so its RCR
translations run with the global-scratch working set (FP64 at both levels,
FP32 at level 2) and its rotation factors come from the quarter-turn
identity at orders never checked by the composed-matrix export.  Both FMM
precisions match the oracle's dense matrix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import oracle_dense, rel, seeded_vector, workload


def test_high_order_fmm_matches_dense():
    wl = workload("high_order")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    ops = []
    try:
        A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
        ops.append(A64)
        A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
        ops.append(A32)
        n, L, p = fb.fb_operator_info(A64)
        assert L == 3 and p[2] >= 114 and p[3] >= 60, (L, p)
        Ad = oracle_dense("high_order")["A"]
        X = np.stack([seeded_vector(wl.n, 300 + r) for r in range(3)])
        xd = torch.tensor(X, device="cuda")
        y = torch.empty_like(xd[0])
        for op, tol in ((A64, 1e-5), (A32, 2e-5)):
            for r in range(3):
                fb.fb_operator_apply(op, xd[r].contiguous(), y)
                torch.cuda.synchronize()
                assert rel(y.cpu().numpy(), Ad @ X[r]) < tol, (op is A64, r)
        # several right-hand sides per call take the same large-order path
        Y = torch.empty_like(xd)
        fb.fb_operator_apply_multi(A32, xd, Y)
        for r in range(3):
            assert rel(Y[r].cpu().numpy(), Ad @ X[r]) < 2e-5
    finally:
        for op in ops:
            fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


@pytest.mark.parametrize("freq", [7500.0, 10800.0])
def test_high_order_rotation_factors_match_oracle(freq):
    """The device's real rotation factors (quarter-turn identity on the
    device) entry by entry against the oracle's factors from the rotation
    generator, on the same coarse shoebox at 7.5 kHz (orders 116 / 66) and
    at 10.8 kHz (orders 159 / 89, the largest room's top two levels; the
    mesh is too coarse for that frequency, which the rotation data do not
    depend on)."""
    import math
    from oracle import sph
    from paper_2103_16073_gb300 import workloads as W
    wl = W.shoebox_workload("shoebox-3.0x2.4x2.0-N3072", 3.0, 2.4, 2.0, (16, 16, 16), freq, 0.2,
                            (0.7, 0.6, 0.5), 8, 0)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A64 = None
    try:
        A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
        top = max(fb.fb_operator_info(A64)[2]) - 1
        assert top >= (158 if freq > 1e4 else 113)
        worst, found = 0.0, 0
        for d in ((2, 0, 0), (2, 2, 2), (3, -1, 2), (-2, 3, -3), (0, -2, 1)):
            code = (d[0] + 3) * 49 + (d[1] + 3) * 7 + (d[2] + 3)
            try:
                fb.fb_operator_export(A64, 8, 0, code)
            except fb.FBError:
                continue   # no M2L pair of this tree has that offset
            found += 1
            th = math.acos(d[2] / math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2))
            for n in (0, 1, 40, 80, top):
                w = 2 * n + 1
                dn = fb.fb_operator_export(A64, 8, n, code).real.reshape(w, w)
                worst = max(worst, float(np.max(np.abs(dn - sph.rotation_factor(n, th)))))
        print(f"degree <= {top}, {found} directions: max |d_gpu - d_oracle| = {worst:.3e}")
        assert found >= 2
        assert worst < 1e-10
    finally:
        if A64 is not None:
            fb.fb_operator_destroy(A64)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
