"""Full-size parity for the 1 kHz shoebox (N = 39,368) in the launch
configuration bench.py times (mixed FMM, automatic translation method,
block-Jacobi FGMRES): sampled rows of the matvec and of the residual against
the oracle's dense rows, which it can compute one by one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import oracle_mesh, rel, seeded_vector, workload


@pytest.fixture(scope="module")
def full():
    wl = workload("full")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    L64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, 6.0, 12)
    yield wl, mesh, A32, A64, L64
    for op in (A32, A64, L64):
        fb.fb_operator_destroy(op)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def _rows(n, count, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=count, replace=False))


def test_full_matvec_sampled_rows(full):
    from oracle import bem
    wl, mesh, A32, A64, L64 = full
    om = oracle_mesh("full")
    rows = _rows(wl.n, 48, 5)
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
    om = oracle_mesh("full")
    g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
    fb.fb_gamma_monopole(mesh, wl.k, wl.sources[0], g)
    b = torch.empty_like(g)
    fb.fb_operator_apply(L64, g, b)
    pc = fb.fb_precond_create(A32, fb.FB_PC_BLOCK_JACOBI)
    x = torch.zeros_like(b)
    info = fb.fb_fgmres_solve(A32, b, x, pc=pc, tol=1e-4, restart=40, max_refine=4, true_op=A64)
    fb.fb_precond_destroy(pc)
    assert info["status"] == 0 and info["true_relres"] <= 1e-4
    rows = _rows(wl.n, 48, 6)
    Ar = bem.system_rows(om, wl.k, wl.beta, rows)
    Lr, _, _ = bem.operator_rows(om, wl.k, om.el.centroid[rows], om.el.normal[rows], rows)
    gam = bem.gamma_monopole(om, wl.k, wl.beta, wl.sources[0])
    b_rows = Lr @ gam
    r = b_rows - Ar @ x.cpu().numpy()
    assert np.linalg.norm(r) / np.linalg.norm(b_rows) < 5e-4
