"""Edge and degenerate cases on the GPU, each against the oracle: the
smallest closed mesh (a cube of 12 triangles: too coarse for an octree), a curved
surface (icosphere: normals in every direction), rigid walls (beta = 0), a
zero right-hand side, the largest number of right-hand sides per call, and a
2 kHz room four times the bench's size (sampled rows)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W
from _cases import rel, seeded_vector


def _setup(verts, tris, beta, k):
    mesh = fb.fb_mesh_create(verts, tris)
    fb.fb_mesh_set_admittance(mesh, beta)
    tree = fb.fb_tree_build(mesh, 64)
    return mesh, tree


def _dense_oracle(verts, tris, k, beta):
    from oracle import bem
    m = bem.Mesh(verts, tris)
    L, M, LP = bem.dense_operators(m, k)
    return m, L, M, LP, bem.system_matrix(L, M, k, beta)


def test_smallest_mesh_dense_and_tree_refusal():
    """A cube of 12 triangles: every pair is within r_c of each other, no
    octree level >= 2 has boxes wider than r_c, so the FMM tree is refused
    (argument error, no device work) while the dense operator and solve
    still match the oracle."""
    v, t, _ = W.shoebox_mesh(1.0, 1.0, 1.0, 1, 1, 1)
    k, beta = 2.0, np.full(t.shape[0], 0.3 + 0.1j)
    m, L, M, LP, A = _dense_oracle(v, t, k, beta)
    mesh = fb.fb_mesh_create(v, t)
    fb.fb_mesh_set_admittance(mesh, beta)
    try:
        with pytest.raises(fb.FBError):
            fb.fb_tree_build(mesh, 64)
        op = fb.fb_operator_create(mesh, None, k, fb.FB_OP_A, fb.FB_PREC_FP64_DENSE, 6.0, 12)
        x = seeded_vector(12, 3)
        y = torch.empty(12, dtype=torch.complex128, device="cuda")
        fb.fb_operator_apply(op, torch.tensor(x, device="cuda"), y)
        assert rel(y.cpu().numpy(), A @ x) < 1e-12
        b = A @ seeded_vector(12, 4)
        xs = torch.zeros(12, dtype=torch.complex128, device="cuda")
        info = fb.fb_fgmres_solve(op, torch.tensor(b, device="cuda"), xs, tol=1e-12, restart=12)
        assert info["status"] == 0
        assert rel(xs.cpu().numpy(), np.linalg.solve(A, b)) < 1e-10
        fb.fb_operator_destroy(op)
    finally:
        fb.fb_mesh_destroy(mesh)


@pytest.mark.parametrize("geom", ["sphere", "rigid"])
def test_fmm_matvec_and_solve_against_dense(geom):
    if geom == "sphere":
        v, t, _ = W.sphere_mesh(1.0, 3)
        k, beta = 3.0, np.full(t.shape[0], 0.2 + 0.0j)
    else:
        v, t, _ = W.shoebox_mesh(1.3, 1.1, 0.9, 11, 9, 7)
        k, beta = 5.0, np.zeros(t.shape[0], np.complex128)
    m, L, M, LP, A = _dense_oracle(v, t, k, beta)
    mesh, tree = _setup(v, t, beta, k)
    ops = []
    try:
        x = seeded_vector(t.shape[0], 11)
        for prec, tol in ((fb.FB_PREC_FP64_FMM, 1e-5), (fb.FB_PREC_MIXED_FMM, 1e-5)):
            op = fb.fb_operator_create(mesh, tree, k, fb.FB_OP_A, prec, 6.0, 12)
            ops.append(op)
            xd = torch.tensor(x, device="cuda")
            y = torch.empty_like(xd)
            fb.fb_operator_apply(op, xd, y)
            assert rel(y.cpu().numpy(), A @ x) < tol, (geom, prec)
        # solve A x = b to 1e-8 with the FP64 FMM and compare with the dense solution
        b = A @ seeded_vector(t.shape[0], 12)
        pc = fb.fb_precond_create(ops[0], fb.FB_PC_BLOCK_JACOBI)
        xs = torch.zeros(t.shape[0], dtype=torch.complex128, device="cuda")
        info = fb.fb_fgmres_solve(ops[0], torch.tensor(b, device="cuda"), xs, pc=pc, tol=1e-8, restart=30)
        fb.fb_precond_destroy(pc)
        assert info["status"] == 0
        assert rel(xs.cpu().numpy(), np.linalg.solve(A, b)) < 1e-4
    finally:
        for op in ops:
            fb.fb_operator_destroy(op)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


def test_zero_rhs_and_max_rhs():
    wl_v, wl_t, _ = W.shoebox_mesh(1.3, 1.1, 0.9, 11, 9, 7)
    n = wl_t.shape[0]
    beta = np.full(n, 0.2 + 0.0j)
    mesh, tree = _setup(wl_v, wl_t, beta, 5.0)
    A = fb.fb_operator_create(mesh, tree, 5.0, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    try:
        # b = 0: x = 0 at once
        b = torch.zeros(n, dtype=torch.complex128, device="cuda")
        x = torch.ones_like(b)
        info = fb.fb_fgmres_solve(A, b, x, tol=1e-6)
        assert info["status"] == 0 and info["iters"] == 0 and float(x.abs().max()) == 0.0
        # the largest number of right-hand sides per call, against single applies
        R = fb.FB_MAX_RHS
        X = torch.tensor(np.stack([seeded_vector(n, 200 + r) for r in range(R)]), device="cuda")
        Y = torch.empty_like(X)
        fb.fb_operator_apply_multi(A, X, Y)
        y1 = torch.empty_like(X[0])
        for r in (0, 17, R - 1):
            fb.fb_operator_apply(A, X[r].contiguous(), y1)
            assert rel(Y[r].cpu().numpy(), y1.cpu().numpy()) < 1e-6
        with pytest.raises(fb.FBError):
            fb.fb_operator_apply_multi(A, torch.zeros((R + 1, n), dtype=torch.complex128, device="cuda"),
                                       torch.zeros((R + 1, n), dtype=torch.complex128, device="cuda"))
    finally:
        fb.fb_operator_destroy(A)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)


def test_2khz_room_sampled_rows():
    """3.0 x 2.4 x 2.0 m at 2 kHz, legs lambda/8 (N = 157,472): mixed FMM rows
    against the oracle's dense rows computed one by one."""
    from oracle import bem
    counts = W.shoebox_counts_for_h(3.0, 2.4, 2.0, W.SOUND_SPEED / 2000.0 / 8.0)
    wl = W.shoebox_workload("shoebox-2kHz", 3.0, 2.4, 2.0, counts, 2000.0, 0.2, (0.7, 0.6, 0.5), 4, 3)
    mesh, tree = _setup(wl.verts, wl.tris, wl.beta, wl.k)
    A = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    try:
        x = seeded_vector(wl.n, 31)
        y = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_operator_apply(A, torch.tensor(x, device="cuda"), y)
        rows = np.sort(np.random.default_rng(3).choice(wl.n, 12, replace=False))
        ref = bem.system_rows(bem.Mesh(wl.verts, wl.tris), wl.k, wl.beta, rows) @ x
        print("N", wl.n, "sampled-row rel err", rel(y.cpu().numpy()[rows], ref))
        assert rel(y.cpu().numpy()[rows], ref) < 1e-4
    finally:
        fb.fb_operator_destroy(A)
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
