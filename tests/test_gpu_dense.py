"""GPU dense FP64 collocation path vs the oracle (small shoebox, N = 3,072,
125 Hz, uniform admittance 0.2): matrix entries, matvec, boundary data,
FGMRES solution (tolerance 1e-10 relative L2 for the FP64 path without FMM),
receiver field and the exterior-source test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import maxrel, oracle_dense, oracle_mesh, rel, seeded_vector, workload


@pytest.fixture(scope="module")
def dense_small():
    wl = workload("small")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    ops = {k: fb.fb_operator_create(mesh, None, wl.k, kind, fb.FB_PREC_FP64_DENSE)
           for k, kind in (("L", fb.FB_OP_L), ("M", fb.FB_OP_M), ("LP", fb.FB_OP_LP), ("A", fb.FB_OP_A))}
    yield wl, mesh, ops
    for op in ops.values():
        fb.fb_operator_destroy(op)
    fb.fb_mesh_destroy(mesh)


def test_mesh_geometry_matches_oracle(dense_small):
    wl, mesh, _ = dense_small
    om = oracle_mesh("small")
    n, rc, me = fb.fb_mesh_info(mesh)
    assert n == om.n and me == float(om.el.max_edge.max()) and rc == om.rc
    c, nn = fb.fb_mesh_geometry(mesh)
    assert np.array_equal(c, om.el.centroid)          # bit-exact collocation points
    assert np.max(np.abs(nn - om.el.normal)) < 1e-15


@pytest.mark.parametrize("kind", ["L", "M", "LP", "A"])
def test_dense_rows_match_oracle(dense_small, kind):
    wl, mesh, ops = dense_small
    ref = oracle_dense("small")[kind]
    rows = [0, 1, 777, 1536, 2047, wl.n - 1]
    for r in rows:
        g = fb.fb_operator_export(ops[kind], 6, 0, r)
        assert maxrel(g, ref[r]) < 1e-12, (kind, r)


@pytest.mark.parametrize("kind", ["L", "M", "LP", "A"])
def test_dense_matvec_matches_oracle(dense_small, kind):
    wl, mesh, ops = dense_small
    ref = oracle_dense("small")[kind]
    x = seeded_vector(wl.n, 3)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    fb.fb_operator_apply(ops[kind], xd, yd)
    torch.cuda.synchronize()
    assert rel(yd.cpu().numpy(), ref @ x) < 1e-12
    # host memspace through the same call
    yh = np.zeros(wl.n, np.complex128)
    fb.fb_operator_apply(ops[kind], x, yh)
    assert rel(yh, ref @ x) < 1e-12


def test_gamma_and_solution_match_oracle(dense_small):
    from oracle import bem, fgmres
    wl, mesh, ops = dense_small
    om = oracle_mesh("small")
    D = oracle_dense("small")
    g_ref = bem.gamma_monopole(om, wl.k, wl.beta, wl.sources[0])
    g = np.zeros(wl.n, np.complex128)
    fb.fb_gamma_monopole(mesh, wl.k, wl.sources[0], g)
    assert rel(g, g_ref) < 1e-13
    b_ref = D["L"] @ g_ref
    x_ref = np.linalg.solve(D["A"], b_ref)
    b = torch.tensor(g, device="cuda")
    bb = torch.empty_like(b)
    fb.fb_operator_apply(ops["L"], b, bb)
    x = torch.zeros_like(bb)
    info = fb.fb_fgmres_solve(ops["A"], bb, x, tol=1e-12, restart=40, maxit=500)
    assert info["status"] == 0 and info["true_relres"] <= 1e-12
    assert rel(x.cpu().numpy(), x_ref) < 1e-10
    # the oracle's own FGMRES agrees with LU too
    xo, io = fgmres.fgmres(lambda v: D["A"] @ v, b_ref, tol=1e-12)
    assert rel(xo, x_ref) < 1e-10


def test_receivers_and_exterior_source(dense_small):
    from oracle import bem
    wl, mesh, ops = dense_small
    om = oracle_mesh("small")
    D = oracle_dense("small")
    xe = np.array([3.6, 0.9, 1.2])
    u, gu = bem.incident(om.el.centroid, xe, wl.k)
    gam = bem.gamma_field(om, wl.k, wl.beta, u, np.sum(gu * om.el.normal, 1))
    gd = torch.tensor(gam, device="cuda")
    bd = torch.empty_like(gd)
    fb.fb_operator_apply(ops["L"], gd, bd)
    x = torch.zeros_like(bd)
    info = fb.fb_fgmres_solve(ops["A"], bd, x, tol=1e-10)
    psi = x.cpu().numpy()
    # exterior-source test: discretisation-limited agreement with u
    assert rel(psi, u) < 0.01
    # receiver field by Eq. (dbem1) vs oracle, and vs the exact exterior field
    rcv = wl.receivers
    out = torch.empty(rcv.shape[0], dtype=torch.complex128, device="cuda")
    fb.fb_eval_field(mesh, wl.k, x, gd, torch.tensor(rcv, device="cuda"), out)
    ref = bem.receiver_field(om, wl.k, wl.beta, psi, gam, rcv)
    assert rel(out.cpu().numpy(), ref) < 1e-12
    ue, _ = bem.incident(rcv, xe, wl.k)
    assert rel(out.cpu().numpy(), ue) < 0.01
