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


@pytest.mark.parametrize("objective", ["error", "residual"])
def test_loss_and_gradient_match_reference(small, objective):
    """Same weights, tree and pair on both sides.  The error objective's
    gradient is exact on both; the residual objective pulls back through the
    area-scaled single/adjoint-double-layer stand-in for A^H (FMM on the GPU,
    dense in the reference)."""
    from oracle import learned
    from oracle.octree import Octree
    wl, mesh, tree, A, bj = small
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        fb.fb_learned_set_objective(pc, fb.FB_LOSS_ERROR if objective == "error" else fb.FB_LOSS_RESIDUAL)
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
        D = oracle_dense("small")
        Ad = D["A"]
        u = learned.block_jacobi(lambda i, j: Ad[np.ix_(i, j)], T, r)
        adj = learned.approx_adjoint(D["L"], D["LP"], el.area, wl.beta, wl.k)
        loss_o, grad_o = learned.loss_grad(theta.astype(np.float64), T, r, e, u, el.normal, objective, Ad, adj,
                                           beta=wl.beta, k=wl.k)
        print(f"{objective}: loss {loss_g:.6f} vs {loss_o:.6f}; grad rel {rel(grad_g, grad_o):.2e}")
        assert abs(loss_g - loss_o) < 1e-2 * loss_o
        assert rel(grad_g, grad_o) < 3e-2
    finally:
        fb.fb_precond_destroy(pc)


def test_training_lowers_loss_and_preconditions(small):
    """Trained on logged pairs (plus white-noise inputs) under the residual
    objective, the network leaves a smaller residual ||A P(r) - r|| than block
    Jacobi on pairs from a source it never saw; FGMRES with it meets the true-
    residual tolerance.  Both iteration counts are reported."""
    from paper_2103_16073_gb300 import training
    from paper_2103_16073_gb300 import workloads as W
    wl, mesh, tree, A, bj = small
    rng = W.seeded_rng(50)
    srcs = W.uniform_points_in_box(rng, [0, 0, 0], list(wl.room), 4, 0.3)

    def rhs(s):
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(mesh, wl.k, s, g)
        b = torch.empty_like(g)
        fb.fb_operator_apply(A, g, b)
        return b

    Rs, Es = [], []
    for s in srcs[:3]:
        R, E = training.collect_pairs(A, bj, rhs(s), iterates=(1, 2, 3, 5, 8))
        Rs.append(R)
        Es.append(E)
    R, E = torch.cat(Rs), torch.cat(Es)
    Rt, Et = training.collect_pairs(A, bj, rhs(srcs[3]), iterates=(1, 2, 3, 5, 8))   # held out
    Ra, Ea = training.augment_noise(R, E, R.shape[0], seed=3)
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        fb.fb_learned_set_objective(pc, fb.FB_LOSS_RESIDUAL)
        before = training.evaluate(pc, Ra, Ea)
        hist, _ = training.train(pc, Ra, Ea, steps=100, lr=1e-3, batch=6)
        after = training.evaluate(pc, Ra, Ea)
        assert np.isfinite(after) and after < before
        res_bj = training.residual_error(A, bj, Rt)
        res_l = training.residual_error(A, pc, Rt)
        assert res_l < res_bj
        b = rhs(wl.sources[0])
        iters = {}
        for name, p in (("block_jacobi", bj), ("learned", pc)):
            x = torch.zeros_like(b)
            info = fb.fb_fgmres_solve(A, b, x, pc=p, tol=1e-4, restart=40)
            assert info["status"] == 0 and info["true_relres"] <= 1e-4
            iters[name] = info["iters"]
        print(f"objective {before:.4f} -> {after:.4f}; held-out ||A P r - r||/||r|| "
              f"block Jacobi {res_bj:.4f}, learned {res_l:.4f}; FGMRES iterations {iters}")
    finally:
        fb.fb_precond_destroy(pc)


def test_block_jacobi_fallback_on_bad_network(small):
    """A network whose output overflows makes the Arnoldi estimate non-finite;
    the solve discards that sweep and finishes under block Jacobi."""
    from oracle import learned
    wl, mesh, tree, A, bj = small
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        _, total = learned.layout()
        fb.fb_learned_params(pc, np.full(total, 1e30, np.float32))
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(mesh, wl.k, wl.sources[0], g)
        b = torch.empty_like(g)
        fb.fb_operator_apply(A, g, b)
        x = torch.zeros_like(b)
        info = fb.fb_fgmres_solve(A, b, x, pc=pc, tol=1e-4, restart=40)
        assert info["pc_fallbacks"] >= 1
        assert info["status"] == 0 and info["true_relres"] <= 1e-4
        assert torch.isfinite(torch.view_as_real(x)).all()
    finally:
        fb.fb_precond_destroy(pc)


def test_inference_apply_matches_reference(small):
    """The fused inference path used inside FGMRES (fb_precond_apply) against
    the FP64 reference network on the same weights and input."""
    from oracle import learned
    from oracle.octree import Octree
    wl, mesh, tree, A, bj = small
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        _, total = learned.layout()
        rng = np.random.default_rng(8)
        theta = (rng.standard_normal(total) * 0.15).astype(np.float32)
        fb.fb_learned_params(pc, theta)
        v = seeded_vector(wl.n, 77)
        z = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_precond_apply(pc, torch.tensor(v, device="cuda"), z)
        om = oracle_mesh("small")
        el = om.el
        T = learned.TreeInfo(Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, om.rc, 64))
        Ad = oracle_dense("small")["A"]
        u = learned.block_jacobi(lambda i, j: Ad[np.ix_(i, j)], T, v)
        zo, _ = learned.forward(theta.astype(np.float64), T, v, u, el.normal, wl.beta, wl.k)
        # the network's correction z - u carries the BF16 error; u itself is exact to FP32
        err = rel(z.cpu().numpy() - u, zo - u)
        print(f"inference correction rel err {err:.2e}; total {rel(z.cpu().numpy(), zo):.2e}")
        assert err < 2e-2
        assert rel(z.cpu().numpy(), zo) < 5e-3
    finally:
        fb.fb_precond_destroy(pc)


def test_learned_gain_measured_on_held_out_source(small):
    """What the trained network gains over block Jacobi.  Trained on the
    inputs FGMRES feeds a preconditioner (Arnoldi vectors of block-Jacobi
    solves for three training sources, plus as many white-noise inputs;
    residual objective), with the parameters selected by FGMRES iterations
    on a fourth source (the initial, block-Jacobi-like state included), then
    measured on a fifth: outer iterations and device time to a true relative
    residual of 1e-4, with and without the network.  The selection
    guarantees the kept network needs no more iterations than its initial,
    block-Jacobi-like state on the validation source; the measured gain on the held-out source is
    printed (on the rooms studied it is zero or negative: the network fits
    the Krylov vectors it was shown but not those of an unseen solve)."""
    import time
    from paper_2103_16073_gb300 import training
    from paper_2103_16073_gb300 import workloads as W
    wl, mesh, tree, A, bj = small
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    rng = W.seeded_rng(51)
    srcs = W.uniform_points_in_box(rng, [0, 0, 0], list(wl.room), 5, 0.3)

    def rhs(s):
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(mesh, wl.k, s, g)
        b = torch.empty_like(g)
        fb.fb_operator_apply(A64, g, b)
        return b

    B = [rhs(s) for s in srcs]

    def solve(pc, b):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = fb.fb_fgmres_solve(A, b, x, pc=pc, tol=1e-4, restart=40, maxit=400, max_refine=4, true_op=A64)
        torch.cuda.synchronize()
        assert info["status"] == 0 and info["true_relres"] <= 1e-4
        return info["iters"], time.perf_counter() - t0

    V = torch.cat([training.krylov_inputs(A, bj, B[i], k=12)[0] for i in range(3)])
    E = torch.zeros_like(V)
    V, E = training.augment_noise(V, E, V.shape[0], seed=9)
    pc = fb.fb_precond_create_learned(A, bj)
    try:
        fb.fb_learned_set_objective(pc, fb.FB_LOSS_RESIDUAL)
        base_val = solve(bj, B[3])[0]
        hist, vlog = training.train(pc, V, E, steps=80, lr=1e-3, batch=8, validate=lambda: solve(pc, B[3])[0],
                                    every=20)
        kept = solve(pc, B[3])[0]
        # the selection never keeps a network worse than its initial, block-
        # Jacobi-like state (up to the run-to-run rounding of the FMM's atomic
        # sums, which can move a count by one)
        assert kept <= vlog[0][1] + 1 and kept <= base_val + 1
        assert hist[-1] < hist[0]                    # training lowers the objective on its inputs
        it_bj, t_bj = solve(bj, B[4])
        it_l, t_l = solve(pc, B[4])
        print(f"validation iterations {vlog}; held-out source: block Jacobi {it_bj} iterations "
              f"{t_bj * 1e3:.1f} ms, learned {it_l} iterations {t_l * 1e3:.1f} ms; "
              f"gain {it_bj - it_l} iterations, {(t_bj - t_l) * 1e3:.1f} ms")
        assert it_l <= it_bj + 2
    finally:
        fb.fb_precond_destroy(pc)
        fb.fb_operator_destroy(A64)
