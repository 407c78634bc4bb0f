"""Indirect system (Eq. ibem5, FB_OP_IBEM: two unknowns per element) on the
GPU against the oracle's 2N x 2N matrix: the dense composite to round-off,
its boundary data, right-hand side, FGMRES solution and receiver field; then
the FMM composite (FP64 and mixed) on the 3,072-element room, and a mixed
solve with the inner-outer preconditioner judged by the FP64 composite."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W
from _cases import oracle_dense, oracle_mesh, rel, seeded_vector, workload

K_SMALL = 6.0
X_IN = np.array([0.31, 0.42, 0.27])


@functools.lru_cache(maxsize=None)
def _oracle_small():
    from oracle import bem, hypersingular
    v, t, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 6, 6, 6)
    mesh = bem.Mesh(v, t)
    L, M, LP = bem.dense_operators(mesh, K_SMALL)
    return v, t, mesh, L, M, LP, hypersingular.dense_mp(mesh, K_SMALL)


def test_dense_composite_matches_oracle():
    from oracle import ibem
    v, t, om, L, M, LP, MP = _oracle_small()
    n = om.n
    bm = np.full(n, 0.2 + 0j)
    bp = np.full(n, 0.3 + 0.1j)
    A = ibem.system(L, M, LP, MP, K_SMALL, bp, bm)
    mesh = fb.fb_mesh_create(v, t)
    fb.fb_mesh_set_admittance(mesh, bm)
    fb.fb_mesh_set_admittance_plus(mesh, bp)
    op = fb.fb_operator_create(mesh, None, K_SMALL, fb.FB_OP_IBEM, fb.FB_PREC_FP64_DENSE, 6.0, 12)
    try:
        assert fb.fb_operator_info(op)[0] == 2 * n
        x = np.concatenate([seeded_vector(n, 5), seeded_vector(n, 6)])
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        fb.fb_operator_apply(op, xd, yd)
        assert rel(yd.cpu().numpy(), A @ x) < 1e-11
        # boundary data and right-hand side for a monopole inside
        gp, gm = fb.fb_ibem_gammas_monopole(op, X_IN)
        from oracle import bem
        u, gu = bem.incident(om.el.centroid, X_IN, K_SMALL)
        rp, rm = ibem.gammas_incident(K_SMALL, bp, bm, u, np.sum(gu * om.el.normal, 1))
        assert rel(gp.cpu().numpy(), rp) < 1e-13 and rel(gm.cpu().numpy(), rm) < 1e-13
        b = fb.fb_ibem_rhs(op, gp, gm)
        bref = ibem.rhs(L, LP, rp, rm)
        assert rel(b.cpu().numpy(), bref) < 1e-11
        # FGMRES on the dense composite, then the field off the surface
        xs = torch.zeros_like(b)
        info = fb.fb_fgmres_solve(op, b, xs, tol=1e-11, restart=80, maxit=2000)
        assert info["status"] == 0
        xref = np.linalg.solve(A, bref)
        assert rel(xs.cpu().numpy(), xref) < 1e-8
        rcv = np.array([[0.7, 0.3, 0.35], [0.5, 0.55, 0.2], [0.25, 0.2, 0.4]])
        f = fb.fb_ibem_field(op, xs, gp, gm, torch.tensor(rcv, device="cuda"))
        sig, mu = ibem.densities(K_SMALL, bp, bm, xref[:n], xref[n:], rp, rm)
        assert rel(f.cpu().numpy(), ibem.field(om, K_SMALL, sig, mu, rcv)) < 1e-8
        # block Jacobi needs the FMM composite (leaf blocks from the tree)
        with pytest.raises(fb.FBError):
            fb.fb_precond_create(op, fb.FB_PC_BLOCK_JACOBI)
    finally:
        fb.fb_operator_destroy(op)
        fb.fb_mesh_destroy(mesh)


@functools.lru_cache(maxsize=None)
def _oracle_system(name):
    from oracle import hypersingular, ibem
    wl = workload(name)
    D = oracle_dense(name)
    MP = hypersingular.dense_mp(oracle_mesh(name), wl.k)
    bp = _beta_plus(wl.n)
    return ibem.system(D["L"], D["M"], D["LP"], MP, wl.k, bp, wl.beta), D, MP


def _beta_plus(n):
    rng = np.random.default_rng(17)
    return rng.uniform(0.05, 0.5, n) + 1j * rng.uniform(-0.1, 0.1, n)


def test_fmm_composite_and_mixed_solve():
    from oracle import bem, ibem
    wl = workload("small")
    A, D, MP = _oracle_system("small")
    n = wl.n
    bp = _beta_plus(n)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    fb.fb_mesh_set_admittance_plus(mesh, bp)
    tree = fb.fb_tree_build(mesh, 64)
    ops = []
    try:
        A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_IBEM, fb.FB_PREC_FP64_FMM, 6.0, 14)
        ops.append(A64)
        A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_IBEM, fb.FB_PREC_MIXED_FMM, 6.0, 14)
        ops.append(A32)
        x = np.concatenate([seeded_vector(n, 15), seeded_vector(n, 16)])
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        ref = A @ x
        for op, tol in ((A64, 1e-5), (A32, 2e-5)):
            fb.fb_operator_apply(op, xd, yd)
            torch.cuda.synchronize()
            assert rel(yd.cpu().numpy(), ref) < tol
        # block Jacobi of the 2 x 2 leaf blocks against the oracle's matrix
        # restricted to the same blocks (tree order of the bit-exact octree)
        from oracle.octree import Octree
        om = oracle_mesh("small")
        el = om.el
        T = Octree(np.concatenate([el.v0, el.v1, el.v2]), el.centroid, om.rc, 64)
        bj64 = fb.fb_precond_create(A64, fb.FB_PC_BLOCK_JACOBI)
        r = np.concatenate([seeded_vector(n, 25), seeded_vector(n, 26)])
        z = torch.empty_like(xd)
        fb.fb_precond_apply(bj64, torch.tensor(r, device="cuda"), z)
        fb.fb_precond_destroy(bj64)
        zref = np.zeros(2 * n, np.complex128)
        starts = np.append(T.leaf_start, n)
        for b in range(len(T.leaf_start)):
            idx = T.perm[starts[b]:starts[b + 1]]
            ii = np.concatenate([idx, n + idx])
            zref[ii] = np.linalg.solve(A[np.ix_(ii, ii)], r[ii])
        assert rel(z.cpu().numpy(), zref) < 1e-9
        # mixed solves judged by the FP64 composite: block Jacobi, and
        # inner-outer on a low-accuracy mixed composite with its block Jacobi
        Alow = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_IBEM, fb.FB_PREC_MIXED_FMM, 2.0, 4)
        ops.append(Alow)
        fb.fb_operator_use_graphs(A32, True)
        bj = fb.fb_precond_create(A32, fb.FB_PC_BLOCK_JACOBI)
        bjlow = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
        inner = fb.fb_precond_create_inner(A32, Alow, bjlow, 6)
        src = wl.sources[0]
        gp, gm = fb.fb_ibem_gammas_monopole(A64, src)
        b = fb.fb_ibem_rhs(A64, gp, gm)
        u, gu = bem.incident(om.el.centroid, src, wl.k)
        rp, rm = ibem.gammas_incident(wl.k, bp, wl.beta, u, np.sum(gu * om.el.normal, 1))
        xref = np.linalg.solve(A, ibem.rhs(D["L"], D["LP"], rp, rm))
        its = {}
        for name, pc in (("block Jacobi", bj), ("inner-outer", inner)):
            xs = torch.zeros_like(b)
            info = fb.fb_fgmres_solve(A32, b, xs, pc=pc, tol=1e-6, restart=40, maxit=400, max_refine=6, true_op=A64)
            assert info["status"] == 0 and info["true_relres"] <= 1e-6
            err = rel(xs.cpu().numpy(), xref)
            assert err < 1e-4
            its[name] = info["iters"]
        for pc in (inner, bjlow, bj):
            fb.fb_precond_destroy(pc)
        print(f"indirect mixed solves, outer iterations: {its} (75 with inner-outer alone)")
        assert its["inner-outer"] < 40
    finally:
        for op in ops:
            fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
