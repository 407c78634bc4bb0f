"""GPU FMM vs the oracle: every setup stage entry by entry (near field,
P2M, L2P, M2M / M2L / L2L translation matrices built by rotation - coaxial
- back-rotation), the FP64 FMM matvec against the oracle FMM (same
truncation) and against the dense operator (1e-5), and the mixed path
against the FP64 FMM."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import maxrel, oracle_dense, oracle_fmm, rel, seeded_vector, workload

KINDS = {"L": fb.FB_OP_L, "M": fb.FB_OP_M, "LP": fb.FB_OP_LP, "A": fb.FB_OP_A}
# p_min per operator: 12 keeps L and A within 1e-5 of the dense matrix; the
# derivative kernels M and L' converge more slowly and need 14.
PMIN = {"A": 12, "L": 12, "M": 14, "LP": 14}


class GpuCase:
    def __init__(self, name):
        wl = workload(name)
        self.wl = wl
        self.mesh = fb.fb_mesh_create(wl.verts, wl.tris)
        fb.fb_mesh_set_admittance(self.mesh, wl.beta)
        self.tree = fb.fb_tree_build(self.mesh, 64)
        self.ops = {}

    def op(self, kind, prec):
        key = (kind, prec)
        if key not in self.ops:
            self.ops[key] = fb.fb_operator_create(self.mesh, self.tree, self.wl.k, KINDS[kind], prec, 6.0,
                                                  PMIN[kind])
        return self.ops[key]

    def close(self):
        for op in self.ops.values():
            fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(self.tree)
        fb.fb_mesh_destroy(self.mesh)

    def apply(self, op, x):
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        fb.fb_operator_apply(op, xd, yd)
        torch.cuda.synchronize()
        return yd.cpu().numpy()


@pytest.fixture(scope="module", params=["small", "ragged"])
def case(request):
    c = GpuCase(request.param)
    c.name = request.param
    yield c
    c.close()


def test_orders_match_oracle(case):
    F = oracle_fmm(case.name, "A")
    n, L, p = fb.fb_operator_info(case.op("A", fb.FB_PREC_FP64_FMM))
    assert L == F.L
    for lev in range(2, L + 1):
        assert p[lev] == F.p[lev]


@pytest.mark.parametrize("kind", ["A", "LP"])
def test_setup_stages_match_oracle(case, kind):
    F = oracle_fmm(case.name, kind, 6.0, PMIN[kind])
    op = case.op(kind, fb.FB_PREC_FP64_FMM)
    nleaf = len(F.leaf_elems)
    for b in sorted(set([0, 1, nleaf // 2, nleaf - 1])):
        cols, ent = F.near[b]
        g = fb.fb_operator_export(op, 0, 0, b).reshape(ent.shape)
        assert maxrel(g, ent) < 1e-12, ("near", b)
        g = fb.fb_operator_export(op, 1, 0, b).reshape(F.W[b].T.shape)
        assert maxrel(g, F.W[b].T) < 1e-11, ("P2M", b)
        g = fb.fb_operator_export(op, 2, 0, b).reshape(F.V[b].shape)
        assert maxrel(g, F.V[b]) < 1e-11, ("L2P", b)
    L = F.L
    T = F.tree
    for lev in range(2, L + 1):
        P = F.p[lev] ** 2
        d = T.delta(lev)
        codes = sorted(set((int(dx) + 3) * 49 + (int(dy) + 3) * 7 + (int(dz) + 3)
                           for (t, s) in F.vl[lev][:: max(1, len(F.vl[lev]) // 5)]
                           for dx, dy, dz in [np.round((F.centers[lev][t] - F.centers[lev][s]) / d)]))
        for c in codes[:4]:
            off = np.array([c // 49 - 3, (c // 7) % 7 - 3, c % 7 - 3], float) * d
            ref = F._T(lev, lev, off, "SR")
            g = fb.fb_operator_export(op, 3, lev, c).reshape(P, P)
            assert maxrel(g, ref) < 1e-11, ("M2L", lev, c)
    for lev in range(3, L + 1):
        d = T.delta(lev)
        for o in (0, 5, 7):
            b = np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1], float)
            try:
                g = fb.fb_operator_export(op, 4, lev, o)
            except fb.FBError:
                continue
            ref = F._T(lev - 1, lev, (0.5 - b) * d, "RR")
            assert maxrel(g.reshape(ref.shape), ref) < 1e-11, ("M2M", lev, o)
            g = fb.fb_operator_export(op, 5, lev, o)
            ref = F._T(lev, lev - 1, (b - 0.5) * d, "RR")
            assert maxrel(g.reshape(ref.shape), ref) < 1e-11, ("L2L", lev, o)


def test_rotation_factor_export_matches_oracle(case):
    """The device rotation data (every direction's real factors from the
    quarter-turn identity) entry by entry against the oracle's factors from
    the rotation generator, for M2L directions of the tree and degrees up
    to the largest order: both give d^n(theta) of the direction, row mu,
    column m."""
    import math
    from oracle import sph
    op = case.op("A", fb.FB_PREC_FP64_FMM)
    top = max(fb.fb_operator_info(op)[2]) - 1
    found = 0
    for d in ((2, 0, 0), (2, 2, 2), (3, -1, 2), (-2, 3, -3), (0, -2, 1), (-3, -3, -2)):
        code = (d[0] + 3) * 49 + (d[1] + 3) * 7 + (d[2] + 3)
        th = math.acos(d[2] / math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2))
        try:
            fb.fb_operator_export(op, 8, 0, code)
        except fb.FBError:
            continue   # no M2L pair of this tree has that offset
        found += 1
        for n in sorted({0, 1, 2, 7, top // 2, top}):
            w = 2 * n + 1
            dn = fb.fb_operator_export(op, 8, n, code).real.reshape(w, w)
            assert np.max(np.abs(dn - sph.rotation_factor(n, th))) < 1e-11, (d, n)
    assert found >= 2


@pytest.mark.parametrize("method", [fb.FB_TRANS_RCR, fb.FB_TRANS_COMPOSED])
@pytest.mark.parametrize("kind", ["A", "L", "M", "LP"])
def test_fp64_fmm_matvec(case, kind, method):
    x = seeded_vector(case.wl.n, 11)
    op = case.op(kind, fb.FB_PREC_FP64_FMM)
    fb.fb_operator_set_translation(op, method)
    try:
        y = case.apply(op, x)
    finally:
        fb.fb_operator_set_translation(op, fb.FB_TRANS_AUTO)
    yo = oracle_fmm(case.name, kind, 6.0, PMIN[kind]).matvec(x)
    assert rel(y, yo) < 1e-11                                   # same truncation
    assert rel(y, oracle_dense(case.name)[kind] @ x) < 1e-5     # FMM accuracy


@pytest.mark.parametrize("method", [fb.FB_TRANS_AUTO, fb.FB_TRANS_RCR, fb.FB_TRANS_COMPOSED,
                                    fb.FB_TRANS_TENSOR])
@pytest.mark.parametrize("kind", ["A", "L"])
def test_mixed_fmm_matvec(case, kind, method):
    x = seeded_vector(case.wl.n, 12)
    y64 = case.apply(case.op(kind, fb.FB_PREC_FP64_FMM), x)
    op = case.op(kind, fb.FB_PREC_MIXED_FMM)
    fb.fb_operator_set_translation(op, method)
    try:
        y32 = case.apply(op, x)
    finally:
        fb.fb_operator_set_translation(op, fb.FB_TRANS_AUTO)
    assert rel(y32, y64) < 1e-5
    assert rel(y32, oracle_dense(case.name)[kind] @ x) < 2e-5


def test_fmm_fgmres_solution(case):
    from oracle import bem
    wl = case.wl
    D = oracle_dense(case.name)
    om_g = bem.gamma_monopole(__import__("_cases").oracle_mesh(case.name), wl.k, wl.beta, wl.sources[0])
    b_ref = D["L"] @ om_g
    x_ref = np.linalg.solve(D["A"], b_ref)
    A64 = case.op("A", fb.FB_PREC_FP64_FMM)
    Amx = case.op("A", fb.FB_PREC_MIXED_FMM)
    L64 = case.op("L", fb.FB_PREC_FP64_FMM)
    g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
    fb.fb_gamma_monopole(case.mesh, wl.k, wl.sources[0], g)
    b = torch.empty_like(g)
    fb.fb_operator_apply(L64, g, b)
    assert rel(b.cpu().numpy(), b_ref) < 1e-5
    x = torch.zeros_like(b)
    info = fb.fb_fgmres_solve(A64, b, x, tol=1e-8, restart=40)
    assert info["status"] == 0 and info["true_relres"] <= 1e-8
    assert rel(x.cpu().numpy(), x_ref) < 1e-4
    pc = fb.fb_precond_create(Amx, fb.FB_PC_BLOCK_JACOBI)
    x2 = torch.zeros_like(b)
    info2 = fb.fb_fgmres_solve(Amx, b, x2, pc=pc, tol=1e-4, restart=40, true_op=A64)
    fb.fb_precond_destroy(pc)
    assert info2["status"] == 0 and info2["true_relres"] <= 1e-4
    assert rel(x2.cpu().numpy(), x_ref) < 1e-3


def test_tensor_core_translations_large_p():
    """All M2L levels on the tensor cores for the 4k sub-instance of the 1 kHz
    room (p = 26 and 17: 11 row tiles x 43 K chunks per matrix) against the
    FP64 RCR path."""
    c = GpuCase("sub")
    try:
        x = seeded_vector(c.wl.n, 13)
        y64 = c.apply(c.op("A", fb.FB_PREC_FP64_FMM), x)
        op = c.op("A", fb.FB_PREC_MIXED_FMM)
        fb.fb_operator_set_translation(op, fb.FB_TRANS_TENSOR)
        yt = c.apply(op, x)
        fb.fb_operator_set_translation(op, fb.FB_TRANS_RCR)
        yr = c.apply(op, x)
        assert rel(yt, y64) < 1e-5
        assert rel(yr, y64) < 1e-5
        assert rel(yt, oracle_dense("sub")["A"] @ x) < 2e-5
    finally:
        c.close()
