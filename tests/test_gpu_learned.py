"""Learned octree preconditioner: GPU loss and gradient (BF16 tensor-core
kernels, FP32 accumulation) against the FP64 reference network on the same
weights, tree and inputs; training on pairs logged from block-Jacobi solves
lowers the loss; FGMRES with the trained network meets the true-residual
tolerance, and its iteration count is reported against block Jacobi."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import oracle_dense, oracle_mesh, rel, seeded_vector, workload


@pytest.fixture(scope="module")
def small():
    wl = workload("small")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    bj = fb.fb_precond_create(A, fb.FB_PC_BLOCK_JACOBI)
    yield wl, mesh, tree, A, bj
    fb.fb_precond_destroy(bj)
    fb.fb_operator_destroy(A)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def test_loss_and_gradient_match_reference(small):
    from oracle import learned
    from oracle.octree import Octree
    wl, mesh, tree, A, bj = small
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        _, total = learned.layout()
        rng = np.random.default_rng(4)
        theta = (rng.standard_normal(total) * 0.15).astype(np.float32)
        got = fb.fb_learned_params(pc, theta)
        assert got.size == total and np.array_equal(got, theta)
        r = seeded_vector(wl.n, 41)
        e = seeded_vector(wl.n, 42)
        loss_g, grad_g = fb.fb_learned_loss_and_grad(pc, torch.tensor(r[None], device="cuda"),
                                                     torch.tensor(e[None], device="cuda"))
        om = oracle_mesh("small")
        el = om.el
        T = learned.TreeInfo(Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, om.rc, 64))
        Ad = oracle_dense("small")["A"]
        u = learned.block_jacobi(lambda i, j: Ad[np.ix_(i, j)], T, r)
        loss_o, grad_o = learned.loss_grad(theta.astype(np.float64), T, r, e, u, el.normal)
        assert abs(loss_g - loss_o) < 1e-2 * loss_o
        assert rel(grad_g, grad_o) < 3e-2
    finally:
        fb.fb_precond_destroy(pc)


def test_training_lowers_loss_and_preconditions(small):
    from paper_2103_16073_gb300 import training
    from paper_2103_16073_gb300 import workloads as W
    wl, mesh, tree, A, bj = small
    rng = W.seeded_rng(50)
    srcs = W.uniform_points_in_box(rng, [0, 0, 0], list(wl.room), 3, 0.3)
    Rs, Es = [], []
    for s in srcs:
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(mesh, wl.k, s, g)
        b = torch.empty_like(g)
        fb.fb_operator_apply(A, g, b)       # right-hand side shape, same operator
        R, E = training.collect_pairs(A, bj, b, iterates=(1, 2, 3, 5, 8))
        Rs.append(R)
        Es.append(E)
    R = torch.cat(Rs)
    E = torch.cat(Es)
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        before = training.evaluate(pc, R, E)
        hist = training.train(pc, R, E, steps=60, lr=2e-3, batch=5)
        after = training.evaluate(pc, R, E)
        assert np.isfinite(after) and after < before
        # solve the canonical source with both preconditioners
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(mesh, wl.k, wl.sources[0], g)
        b = torch.empty_like(g)
        fb.fb_operator_apply(A, g, b)
        iters = {}
        for name, p in (("block_jacobi", bj), ("learned", pc)):
            x = torch.zeros_like(b)
            info = fb.fb_fgmres_solve(A, b, x, pc=p, tol=1e-4, restart=40)
            assert info["status"] == 0 and info["true_relres"] <= 1e-4
            iters[name] = info["iters"]
        print(f"loss {before:.4f} -> {after:.4f}; FGMRES iterations {iters}")
    finally:
        fb.fb_precond_destroy(pc)
