"""Several right-hand sides per call: the batched FMM matvec against one
call per right-hand side (every translation method, mixed and FP64), and the
lockstep batched FGMRES against single solves (each system meets its own
true-residual tolerance; solutions and iteration counts agree)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from _cases import rel, seeded_vector, workload


@pytest.fixture(scope="module", params=["small", "sub"])
def setup(request):
    wl = workload(request.param)
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    ops = {}

    def op(prec):
        if prec not in ops:
            ops[prec] = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, prec, 6.0, 12)
        return ops[prec]

    yield wl, mesh, op
    for o in ops.values():
        fb.fb_operator_destroy(o)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


METHODS = {"auto": fb.FB_TRANS_AUTO, "rcr": fb.FB_TRANS_RCR, "tensor": fb.FB_TRANS_TENSOR,
           "composed": fb.FB_TRANS_COMPOSED}


@pytest.mark.parametrize("prec,method", [("mixed", "auto"), ("mixed", "rcr"), ("mixed", "tensor"),
                                         ("mixed", "composed"), ("fp64", "auto")])
def test_apply_multi_matches_single(setup, prec, method):
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM if prec == "mixed" else fb.FB_PREC_FP64_FMM)
    fb.fb_operator_set_translation(A, METHODS[method])
    try:
        R = 5   # a full chunk of four and a ragged one
        X = torch.tensor(np.stack([seeded_vector(wl.n, 100 + r) for r in range(R)]), device="cuda")
        Y = torch.empty_like(X)
        fb.fb_operator_apply_multi(A, X, Y)
        y1 = torch.empty_like(X[0])
        tol = 1e-6 if prec == "mixed" else 1e-13
        for r in range(R):
            fb.fb_operator_apply(A, X[r].contiguous(), y1)
            assert rel(Y[r].cpu().numpy(), y1.cpu().numpy()) < tol, (prec, method, r)
    finally:
        fb.fb_operator_set_translation(A, fb.FB_TRANS_AUTO)


def test_fgmres_multi_matches_single(setup):
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    A64 = op(fb.FB_PREC_FP64_FMM)
    bj = fb.fb_precond_create(A, fb.FB_PC_BLOCK_JACOBI)
    try:
        from paper_2103_16073_gb300 import workloads as W
        rng = W.seeded_rng(60)
        srcs = W.uniform_points_in_box(rng, [0, 0, 0], list(wl.room), 3, 0.3)
        B = torch.empty((3, wl.n), dtype=torch.complex128, device="cuda")
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        for r, s in enumerate(srcs):
            fb.fb_gamma_monopole(mesh, wl.k, s, g)
            fb.fb_operator_apply(A64, g, B[r])
        X = torch.zeros_like(B)
        infos = fb.fb_fgmres_solve_multi(A, B, X, pc=bj, tol=1e-6, restart=20, true_op=A64)
        for r in range(3):
            x1 = torch.zeros_like(g)
            i1 = fb.fb_fgmres_solve(A, B[r].contiguous(), x1, pc=bj, tol=1e-6, restart=20, true_op=A64)
            assert infos[r]["status"] == 0 and infos[r]["true_relres"] <= 1e-6
            assert abs(infos[r]["iters"] - i1["iters"]) <= 1
            assert rel(X[r].cpu().numpy(), x1.cpu().numpy()) < 1e-4
        print("iterations", [i["iters"] for i in infos])
    finally:
        fb.fb_precond_destroy(bj)


def test_autotune_keeps_results(setup):
    """After the autotuner installs its per-level choice the matvec still
    agrees with the all-RCR form (single and multi right-hand side)."""
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    X = torch.tensor(np.stack([seeded_vector(wl.n, 300 + r) for r in range(3)]), device="cuda")
    fb.fb_operator_set_translation(A, fb.FB_TRANS_RCR)
    Yref = torch.empty_like(X)
    fb.fb_operator_apply_multi(A, X, Yref)
    fb.fb_operator_set_translation(A, fb.FB_TRANS_AUTO)
    rep = fb.fb_operator_autotune(A, nrhs=3)
    assert rep and all(v["m2l_rcr"] is not None for l, v in rep.items() if l >= 2)
    Y = torch.empty_like(X)
    fb.fb_operator_apply_multi(A, X, Y)
    y1 = torch.empty_like(X[0])
    fb.fb_operator_apply(A, X[0].contiguous(), y1)
    # both are FP32 forms of the same translations (tensor-core composed
    # matrices vs rotation-coaxial-rotation), equal up to FP32 rounding
    for r in range(3):
        assert rel(Y[r].cpu().numpy(), Yref[r].cpu().numpy()) < 1e-5
    assert rel(y1.cpu().numpy(), Yref[0].cpu().numpy()) < 1e-5
    # the tuned choice can be saved and installed again without timing
    fb.fb_operator_set_forms(A, [0] * 13)
    fb.fb_operator_set_forms(A, rep)
    y2 = torch.empty_like(X[0])
    fb.fb_operator_apply(A, X[0].contiguous(), y2)
    assert rel(y2.cpu().numpy(), y1.cpu().numpy()) < 1e-6
    print(rep)


def test_graph_replay_matches(setup):
    """The captured-graph replay of the matvec (single and multi right-hand
    side) and of the learned preconditioner gives the same results as direct
    launches, and a solve through it converges the same way."""
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    X = torch.tensor(np.stack([seeded_vector(wl.n, 500 + r) for r in range(2)]), device="cuda")
    Yd = torch.empty_like(X)
    fb.fb_operator_apply_multi(A, X, Yd)
    y1d = torch.empty_like(X[0])
    fb.fb_operator_apply(A, X[0].contiguous(), y1d)
    fb.fb_operator_use_graphs(A, True)
    try:
        for _ in range(2):   # capture, then replay
            Yg = torch.empty_like(X)
            fb.fb_operator_apply_multi(A, X, Yg)
            y1g = torch.empty_like(X[0])
            fb.fb_operator_apply(A, X[0].contiguous(), y1g)
            for r in range(2):
                assert rel(Yg[r].cpu().numpy(), Yd[r].cpu().numpy()) < 1e-6
            assert rel(y1g.cpu().numpy(), y1d.cpu().numpy()) < 1e-6
        # more right-hand sides than ever before grow the expansion buffers;
        # the graphs captured on the old buffers must be captured again
        X9 = torch.tensor(np.stack([seeded_vector(wl.n, 600 + r) for r in range(9)]), device="cuda")
        Y9 = torch.empty_like(X9)
        fb.fb_operator_apply_multi(A, X9, Y9)
        y1g = torch.empty_like(X[0])
        fb.fb_operator_apply(A, X[0].contiguous(), y1g)
        assert rel(y1g.cpu().numpy(), y1d.cpu().numpy()) < 1e-6
        bj = fb.fb_precond_create(A, fb.FB_PC_BLOCK_JACOBI)
        pcl = fb.fb_precond_create_learned(A, bj)
        z0 = torch.empty_like(X[0])
        fb.fb_precond_apply(pcl, X[0].contiguous(), z0)
        fb.fb_precond_use_graphs(pcl, True)
        for _ in range(2):
            zg = torch.empty_like(X[0])
            fb.fb_precond_apply(pcl, X[0].contiguous(), zg)
            assert rel(zg.cpu().numpy(), z0.cpu().numpy()) < 1e-6
        b = Yd[1].contiguous()
        infos = []
        for g in (False, True):
            fb.fb_operator_use_graphs(A, g)
            x = torch.zeros_like(b)
            infos.append(fb.fb_fgmres_solve(A, b, x, pc=pcl, tol=1e-6, restart=30))
        assert all(i["status"] == 0 for i in infos)
        assert abs(infos[0]["iters"] - infos[1]["iters"]) <= 1
        fb.fb_precond_destroy(pcl)
        fb.fb_precond_destroy(bj)
    finally:
        fb.fb_operator_use_graphs(A, False)


def test_inner_outer_preconditioner(setup):
    """FGMRES preconditioned by a few GMRES steps on a low-accuracy FMM
    (Sec. 4): one inner step reproduces block Jacobi (a scaled copy of its
    output, so the same outer iterations); four inner steps need fewer outer
    iterations; both meet the FP64 true-residual tolerance."""
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    A64 = op(fb.FB_PREC_FP64_FMM)
    tree = fb.fb_tree_build(mesh, 64)
    Alow = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 2.0, 6)
    bj = fb.fb_precond_create(A, fb.FB_PC_BLOCK_JACOBI)
    bjl = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
    pcs = {k: fb.fb_precond_create_inner(A, Alow, bjl, k) for k in (1, 4)}
    try:
        b = torch.tensor(seeded_vector(wl.n, 77), device="cuda")
        its = {}
        for name, pc in (("bj", bj), ("inner1", pcs[1]), ("inner4", pcs[4])):
            x = torch.zeros_like(b)
            info = fb.fb_fgmres_solve(A, b, x, pc=pc, tol=1e-6, restart=30, true_op=A64)
            assert info["status"] == 0 and info["true_relres"] <= 1e-6, name
            its[name] = info["iters"]
        # the learned network over the inner-outer base (graph replay of both)
        pcl = fb.fb_precond_create_learned(A, pcs[4])
        fb.fb_precond_use_graphs(pcl, True)
        x = torch.zeros_like(b)
        info = fb.fb_fgmres_solve(A, b, x, pc=pcl, tol=1e-6, restart=30, true_op=A64)
        fb.fb_precond_destroy(pcl)
        assert info["status"] == 0 and info["true_relres"] <= 1e-6
        its["learned_over_inner4"] = info["iters"]
        print("outer iterations", its)
        assert abs(its["inner1"] - its["bj"]) <= 1
        assert its["inner4"] < its["bj"]
    finally:
        for pc in pcs.values():
            fb.fb_precond_destroy(pc)
        fb.fb_precond_destroy(bjl)
        fb.fb_precond_destroy(bj)
        fb.fb_operator_destroy(Alow)
        fb.fb_tree_destroy(tree)


def test_create_like_copies_near_field(setup):
    """An operator made from an FP64 donor (fb_operator_create_like) copies
    the donor's near-field entries: the same matvec as an operator created
    from scratch, FP64 to round-off and mixed to FP32 summation order, and
    at another order rule; dense donors and precisions are refused."""
    wl, mesh, op = setup
    A64 = op(fb.FB_PREC_FP64_FMM)
    A32 = op(fb.FB_PREC_MIXED_FMM)
    tree = fb.fb_tree_build(mesh, 64)
    made = []
    try:
        x = torch.tensor(seeded_vector(wl.n, 84), device="cuda")

        def mv(o):
            y = torch.empty_like(x)
            fb.fb_operator_apply(o, x, y)
            torch.cuda.synchronize()
            return y.cpu().numpy()
        B64 = fb.fb_operator_create_like(A64, fb.FB_PREC_FP64_FMM, 6.0, 12)
        made.append(B64)
        assert rel(mv(B64), mv(A64)) < 1e-13
        B32 = fb.fb_operator_create_like(A64, fb.FB_PREC_MIXED_FMM, 6.0, 12)
        made.append(B32)
        assert rel(mv(B32), mv(A32)) < 1e-6
        Low = fb.fb_operator_create_like(A64, fb.FB_PREC_MIXED_FMM, 0.5, 2)
        made.append(Low)
        Ref = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 0.5, 2)
        made.append(Ref)
        assert rel(mv(Low), mv(Ref)) < 1e-6
        with pytest.raises(fb.FBError):
            fb.fb_operator_create_like(A64, fb.FB_PREC_FP64_DENSE, 6.0, 12)
    finally:
        for o in made:
            fb.fb_operator_destroy(o)
        fb.fb_tree_destroy(tree)


def test_inner_operator_bf16_near_field(setup):
    """The low-accuracy inner operator with its near-field entries in BF16:
    its matvec moves from the FP32-entry one by the BF16 rounding only (well
    under 1e-2, and not zero: the 16-bit path runs), the inner-outer solve
    meets the FP64 true-residual tolerance in the same outer iterations
    (+-1), and FP64 operators refuse the setting."""
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    A64 = op(fb.FB_PREC_FP64_FMM)
    tree = fb.fb_tree_build(mesh, 64)
    Alow = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 0.5, 2)
    bjl = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
    inner = fb.fb_precond_create_inner(A, Alow, bjl, 6)
    try:
        x = torch.tensor(seeded_vector(wl.n, 78), device="cuda")
        y32, y16 = torch.empty_like(x), torch.empty_like(x)
        fb.fb_operator_apply(Alow, x, y32)
        b = torch.tensor(seeded_vector(wl.n, 79), device="cuda")
        xs = torch.zeros_like(b)
        it32 = fb.fb_fgmres_solve(A, b, xs, pc=inner, tol=1e-6, restart=30, true_op=A64)["iters"]
        fb.fb_operator_set_near_bf16(Alow, True)
        fb.fb_operator_apply(Alow, x, y16)
        torch.cuda.synchronize()
        d = rel(y16.cpu().numpy(), y32.cpu().numpy())
        assert 1e-6 < d < 1e-2
        xs = torch.zeros_like(b)
        info = fb.fb_fgmres_solve(A, b, xs, pc=inner, tol=1e-6, restart=30, true_op=A64)
        assert info["status"] == 0 and info["true_relres"] <= 1e-6
        assert abs(info["iters"] - it32) <= 1
        fb.fb_operator_set_near_bf16(Alow, False)
        y = torch.empty_like(x)
        fb.fb_operator_apply(Alow, x, y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), y32.cpu().numpy()) < 1e-6   # FP32 atomics: summation order only
        with pytest.raises(fb.FBError):
            fb.fb_operator_set_near_bf16(A64, True)
    finally:
        fb.fb_precond_destroy(inner)
        fb.fb_precond_destroy(bjl)
        fb.fb_operator_destroy(Alow)
        fb.fb_tree_destroy(tree)


def test_inner_outer_several_rhs_and_graphs(setup):
    """The inner-outer preconditioner on several right-hand sides runs one
    lockstep inner GMRES (one multi-RHS matvec per inner step): in a batched
    solve each system needs the outer iterations of its single solve (+-1)
    and meets the tolerance; replayed as captured graphs (one per number of
    right-hand sides) it gives the same solutions up to the rounding of the
    FMM's FP32 atomic scatter-adds, whose order varies from run to run."""
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    A64 = op(fb.FB_PREC_FP64_FMM)
    tree = fb.fb_tree_build(mesh, 64)
    Alow = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 0.5, 2)
    bjl = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
    inner = fb.fb_precond_create_inner(A, Alow, bjl, 6)
    try:
        R = 3
        B = torch.tensor(np.stack([seeded_vector(wl.n, 130 + r) for r in range(R)]), device="cuda")
        single = []
        for r in range(R):
            x = torch.zeros_like(B[0])
            info = fb.fb_fgmres_solve(A, B[r].contiguous(), x, pc=inner, tol=1e-6, restart=30, true_op=A64)
            assert info["status"] == 0
            single.append((x.cpu().numpy(), info["iters"]))
        X = torch.zeros_like(B)
        infos = fb.fb_fgmres_solve_multi(A, B, X, pc=inner, tol=1e-6, restart=30, true_op=A64)
        for r in range(R):
            assert infos[r]["status"] == 0 and infos[r]["true_relres"] <= 1e-6
            assert abs(infos[r]["iters"] - single[r][1]) <= 1
            assert rel(X[r].cpu().numpy(), single[r][0]) < 1e-5
        fb.fb_operator_use_graphs(Alow, True)
        fb.fb_precond_use_graphs(inner, True)
        for _ in range(2):   # capture, then replay
            X2 = torch.zeros_like(B)
            infos2 = fb.fb_fgmres_solve_multi(A, B, X2, pc=inner, tol=1e-6, restart=30, true_op=A64)
            for r in range(R):
                assert infos2[r]["status"] == 0 and abs(infos2[r]["iters"] - infos[r]["iters"]) <= 1
                assert rel(X2[r].cpu().numpy(), X[r].cpu().numpy()) < 1e-6
            x = torch.zeros_like(B[0])
            info = fb.fb_fgmres_solve(A, B[0].contiguous(), x, pc=inner, tol=1e-6, restart=30, true_op=A64)
            assert info["status"] == 0
            assert rel(x.cpu().numpy(), single[0][0]) < 1e-6
    finally:
        fb.fb_precond_destroy(inner)
        fb.fb_precond_destroy(bjl)
        fb.fb_operator_destroy(Alow)
        fb.fb_tree_destroy(tree)


def test_krylov_basis_is_arnoldi(setup):
    """fb_krylov_basis returns an orthonormal basis that starts at b/||b||
    and satisfies the Arnoldi relation A V_j in span(V_0..V_{j+1})."""
    wl, mesh, op = setup
    A = op(fb.FB_PREC_MIXED_FMM)
    b = torch.tensor(seeded_vector(wl.n, 77), device="cuda")
    k = 5
    V = fb.fb_krylov_basis(A, None, b, k)
    assert V.shape == (k + 1, wl.n)
    Vn = V.cpu().numpy()
    G = Vn.conj() @ Vn.T
    assert np.max(np.abs(G - np.eye(k + 1))) < 1e-10
    bn = b.cpu().numpy()
    assert rel(Vn[0], bn / np.linalg.norm(bn)) < 1e-13
    y = torch.empty_like(b)
    for j in range(k):
        fb.fb_operator_apply(A, V[j].contiguous(), y)
        w = y.cpu().numpy()
        proj = Vn[:j + 2].T @ (Vn[:j + 2].conj() @ w)
        assert rel(proj, w) < 1e-6, j
    with pytest.raises(fb.FBError):
        fb.fb_krylov_basis(A, None, b, 0)
