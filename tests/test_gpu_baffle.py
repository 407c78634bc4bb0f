"""The door-and-baffle room (shoebox 5x4x3 m, door of admittance 1.0, a
closed 2 cm baffle box of admittance 1.0): parity of the dense and FMM
operators with the oracle on a small instance (N = 3,280), the
exterior-source test through the GPU solver, and at full size (2 kHz,
N = 685,272) sampled rows of the matvec and of the solve's residual in the
configuration a solve uses (mixed FMM, block-Jacobi FGMRES, FP64 FMM true
residual)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W
from _cases import oracle_dense, oracle_mesh, rel, seeded_vector, workload


def _handles(name):
    wl = workload(name)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    return wl, mesh, tree


@pytest.fixture(scope="module")
def small():
    wl, mesh, tree = _handles("baffle_sub")
    ops = {
        "D": fb.fb_operator_create(mesh, None, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_DENSE),
        "DL": fb.fb_operator_create(mesh, None, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_DENSE),
        "A64": fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12),
        "A32": fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12),
    }
    yield wl, mesh, ops
    for op in ops.values():
        fb.fb_operator_destroy(op)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def test_small_operators_match_oracle(small):
    wl, mesh, ops = small
    A = oracle_dense("baffle_sub")["A"]
    x = seeded_vector(wl.n, 11)
    ref = A @ x
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    for name, tol in (("D", 1e-10), ("A64", 1e-5), ("A32", 2e-5)):
        fb.fb_operator_apply(ops[name], xd, yd)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), ref) < tol, name


def test_small_exterior_source_and_solve(small):
    """The field of a monopole outside the room solves the boundary equation
    on walls, door and baffle alike: the mixed solve (FP64 true residual)
    matches the oracle's direct solve and approaches the field."""
    from oracle import bem
    wl, mesh, ops = small
    om = oracle_mesh("baffle_sub")
    D = oracle_dense("baffle_sub")
    xe = W.exterior_source(wl.room)
    u, gu = bem.incident(om.el.centroid, xe, wl.k)
    gam = bem.gamma_field(om, wl.k, wl.beta, u, np.sum(gu * om.el.normal, 1))
    b_ref = D["L"] @ gam
    x_ref = np.linalg.solve(D["A"], b_ref)
    gd = torch.tensor(gam, device="cuda")
    bd = torch.empty_like(gd)
    fb.fb_operator_apply(ops["DL"], gd, bd)
    assert rel(bd.cpu().numpy(), b_ref) < 1e-10
    pc = fb.fb_precond_create(ops["A32"], fb.FB_PC_BLOCK_JACOBI)
    x = torch.zeros_like(bd)
    info = fb.fb_fgmres_solve(ops["A32"], bd, x, pc=pc, tol=1e-6, restart=40, max_refine=6, true_op=ops["A64"])
    fb.fb_precond_destroy(pc)
    assert info["status"] == 0 and info["true_relres"] <= 1e-6
    xs = x.cpu().numpy()
    assert rel(xs, x_ref) < 1e-4
    assert rel(xs, u) < 0.05


def _rows(n, count, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=count, replace=False))


@pytest.fixture(scope="module")
def full():
    wl, mesh, tree = _handles("baffle")
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    L64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, 6.0, 12)
    yield wl, mesh, A32, A64, L64
    for op in (A32, A64, L64):
        fb.fb_operator_destroy(op)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def test_full_matvec_sampled_rows(full):
    from oracle import bem
    wl, mesh, A32, A64, L64 = full
    assert wl.n == 685272
    om = oracle_mesh("baffle")
    rows = _rows(wl.n, 32, 5)
    Ar = bem.system_rows(om, wl.k, wl.beta, rows)
    x = seeded_vector(wl.n, 31)
    xd = torch.tensor(x, device="cuda")
    for op, tol in ((A64, 1e-5), (A32, 2e-5)):
        yd = torch.empty_like(xd)
        fb.fb_operator_apply(op, xd, yd)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy()[rows], Ar @ x) < tol


def test_full_solve_residual_sampled_rows(full):
    from oracle import bem
    wl, mesh, A32, A64, L64 = full
    om = oracle_mesh("baffle")
    g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
    fb.fb_gamma_monopole(mesh, wl.k, wl.sources[0], g)
    b = torch.empty_like(g)
    fb.fb_operator_apply(L64, g, b)
    pc = fb.fb_precond_create(A32, fb.FB_PC_BLOCK_JACOBI)
    x = torch.zeros_like(b)
    info = fb.fb_fgmres_solve(A32, b, x, pc=pc, tol=1e-4, restart=40, max_refine=4, true_op=A64)
    fb.fb_precond_destroy(pc)
    assert info["status"] == 0 and info["true_relres"] <= 1e-4
    rows = _rows(wl.n, 32, 6)
    Ar = bem.system_rows(om, wl.k, wl.beta, rows)
    Lr, _, _ = bem.operator_rows(om, wl.k, om.el.centroid[rows], om.el.normal[rows], rows)
    gam = bem.gamma_monopole(om, wl.k, wl.beta, wl.sources[0])
    b_rows = Lr @ gam
    r = b_rows - Ar @ x.cpu().numpy()
    assert np.linalg.norm(r) / np.linalg.norm(b_rows) < 5e-4
