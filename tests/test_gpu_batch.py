"""Batch scheduler: a small L-room frequency sweep (uneven N, several
sources per frequency) through fb_batch_solve; every solve meets its true-
residual tolerance, jobs run largest first, and one job's solutions agree
with single solves of the same systems built through the public API."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import sweep
from _cases import rel


@pytest.mark.parametrize("lookahead,inner", [(True, 0), (False, 0), (True, 8)])
def test_sweep_batch(lookahead, inner):
    """inner = 0: block Jacobi; inner = 8: the inner-outer preconditioner
    (8 lockstep GMRES steps on a low-accuracy FMM for all sources of a batch,
    replayed as captured graphs)."""
    wls = sweep.W.lroom_sweep(nfreq=3, f_lo=100.0, f_hi=200.0, nsrc=3)
    built = []
    for wl in wls:
        mesh = fb.fb_mesh_create(wl.verts, wl.tris)
        fb.fb_mesh_set_admittance(mesh, wl.beta)
        tree = fb.fb_tree_build(mesh, 64)
        built.append(dict(mesh=mesh, tree=tree, k=wl.k, src=wl.sources,
                          x=torch.zeros((3, wl.n), dtype=torch.complex128, device="cuda")))
    try:
        res = fb.fb_batch_solve(built, tol=1e-5, max_rhs=2, autotune=True, lookahead=lookahead, inner_iters=inner)
        for r in res:
            assert r["status"] == 0
            assert all(i["status"] == 0 and i["true_relres"] <= 1e-5 for i in r["infos"])
        # largest job first
        order = sorted(range(3), key=lambda i: res[i]["order"])
        assert [wls[i].n for i in order] == sorted([w.n for w in wls], reverse=True)
        # job 1 against single solves
        wl, b = wls[1], built[1]
        A32 = fb.fb_operator_create(b["mesh"], b["tree"], wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
        A64 = fb.fb_operator_create(b["mesh"], b["tree"], wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
        L64 = fb.fb_operator_create(b["mesh"], b["tree"], wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, 6.0, 12)
        pc = fb.fb_precond_create(A32, fb.FB_PC_BLOCK_JACOBI)
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        rhs = torch.empty_like(g)
        for q in range(3):
            fb.fb_gamma_monopole(b["mesh"], wl.k, wl.sources[q], g)
            fb.fb_operator_apply(L64, g, rhs)
            x = torch.zeros_like(g)
            info = fb.fb_fgmres_solve(A32, rhs, x, pc=pc, tol=1e-5, restart=40, true_op=A64)
            assert info["status"] == 0
            assert rel(b["x"][q].cpu().numpy(), x.cpu().numpy()) < 1e-4
        fb.fb_precond_destroy(pc)
        for o in (A32, A64, L64):
            fb.fb_operator_destroy(o)
        print([(wl.n, r["order"], round(r["setup_ms"], 1), round(r["solve_ms"], 1)) for wl, r in zip(wls, res)])
    finally:
        for b in built:
            fb.fb_tree_destroy(b["tree"])
            fb.fb_mesh_destroy(b["mesh"])


def test_sweep_top_frequency_full_size():
    """The sweep's largest job at full size (2 kHz, legs lambda/8,
    N = 567,592, 8 sources in one lockstep batch, orders above one shared-
    memory tile in FP64): every solve meets the FP64 true residual, and one
    solution's residual on sampled rows of the oracle's A and L stays at
    the tolerance."""
    from oracle import bem
    wl = sweep.W.lroom_sweep(nfreq=64, f_lo=100.0, f_hi=2000.0, nsrc=8)[-1]
    assert wl.n == 567592
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    job = dict(mesh=mesh, tree=tree, k=wl.k, src=wl.sources,
               x=torch.zeros((8, wl.n), dtype=torch.complex128, device="cuda"))
    try:
        (r,) = fb.fb_batch_solve([job], tol=1e-4, max_rhs=8, autotune=True, lookahead=False)
        assert r["status"] == 0
        assert all(i["status"] == 0 and i["true_relres"] <= 1e-4 for i in r["infos"])
        om = bem.Mesh(wl.verts, wl.tris)
        rows = np.sort(np.random.default_rng(12).choice(wl.n, size=16, replace=False))
        Ar = bem.system_rows(om, wl.k, wl.beta, rows)
        Lr, _, _ = bem.operator_rows(om, wl.k, om.el.centroid[rows], om.el.normal[rows], rows)
        q = 5
        gam = bem.gamma_monopole(om, wl.k, wl.beta, wl.sources[q])
        b_rows = Lr @ gam
        res = b_rows - Ar @ job["x"][q].cpu().numpy()
        err = np.linalg.norm(res) / np.linalg.norm(b_rows)
        print(f"iterations {[i['iters'] for i in r['infos']]}, sampled-row residual {err:.2e}")
        assert err < 5e-4
    finally:
        fb.fb_tree_destroy(tree)
        fb.fb_mesh_destroy(mesh)
