"""The largest room (shoebox 6.5 x 5.5 x 4.2 m at 5 kHz, legs lambda/6,
N = 2,644,104, expansion orders up to 159) in the launch configuration of a
solve (mixed FMM with autotuned forms and graph replay, FP64 FMM true
residual): sampled rows of both matvecs against the oracle's rows, and the
exterior-source test on the full mesh, on the surface and at receivers
(the field of a monopole outside the room solves the interior problem
exactly, so the discrete solution and the receiver field of Eq. (dbem1)
approach it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_16073_gb300 as fb
from paper_2103_16073_gb300 import workloads as W
from _cases import oracle_mesh, rel, seeded_vector, workload


@pytest.fixture(scope="module")
def largest():
    wl = workload("largest")
    mesh = fb.fb_mesh_create(wl.verts, wl.tris)
    fb.fb_mesh_set_admittance(mesh, wl.beta)
    tree = fb.fb_tree_build(mesh, 64)
    A32 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 6.0, 12)
    fb.fb_operator_autotune(A32, 1)
    fb.fb_operator_use_graphs(A32, True)
    A64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_FP64_FMM, 6.0, 12)
    yield wl, mesh, tree, A32, A64
    for op in (A32, A64):
        fb.fb_operator_destroy(op)
    fb.fb_tree_destroy(tree)
    fb.fb_mesh_destroy(mesh)


def test_largest_matvec_sampled_rows(largest):
    from oracle import bem
    wl, mesh, tree, A32, A64 = largest
    assert wl.n == 2644104
    n, L, p = fb.fb_operator_info(A64)
    assert max(p) >= 150
    om = oracle_mesh("largest")
    rows = np.sort(np.random.default_rng(9).choice(wl.n, size=16, replace=False))
    Ar = bem.system_rows(om, wl.k, wl.beta, rows)
    x = seeded_vector(wl.n, 91)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    for op, tol in ((A64, 1e-5), (A32, 2e-5)):
        fb.fb_operator_apply(op, xd, yd)
        torch.cuda.synchronize()
        err = rel(yd.cpu().numpy()[rows], Ar @ x)
        print(f"sampled rows rel err {err:.2e}")
        assert err < tol


def test_largest_exterior_source(largest):
    from oracle import bem
    wl, mesh, tree, A32, A64 = largest
    om = oracle_mesh("largest")
    xe = W.exterior_source(wl.room)
    u, gu = bem.incident(om.el.centroid, xe, wl.k)
    gam = bem.gamma_field(om, wl.k, wl.beta, u, np.sum(gu * om.el.normal, 1))
    gd = torch.tensor(gam, device="cuda")
    L64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, 6.0, 12)
    Alow = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 2.0, 4)
    pclow = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
    inner = fb.fb_precond_create_inner(A32, Alow, pclow, 8)
    try:
        b = torch.empty_like(gd)
        fb.fb_operator_apply(L64, gd, b)
        x = torch.zeros_like(b)
        info = fb.fb_fgmres_solve(A32, b, x, pc=inner, tol=1e-5, restart=40, maxit=400, max_refine=6,
                                  true_op=A64)
        assert info["status"] == 0 and info["true_relres"] <= 1e-5
        psi = x.cpu().numpy()
        e_surf = rel(psi, u)
        rcv = wl.receivers
        out = torch.empty(rcv.shape[0], dtype=torch.complex128, device="cuda")
        fb.fb_eval_field(mesh, wl.k, x, gd, torch.tensor(rcv, device="cuda"), out)
        got = out.cpu().numpy()
        ue, _ = bem.incident(rcv, xe, wl.k)
        e_rcv = rel(got, ue)
        ref = bem.receiver_field(om, wl.k, wl.beta, psi, gam, rcv[:8])
        e_par = rel(got[:8], ref)
        print(f"iterations {info['iters']}; exterior source: surface {e_surf:.3e}, 1024 receivers {e_rcv:.3e}; "
              f"receiver field vs oracle {e_par:.1e}")
        assert e_par < 1e-10
        assert e_surf < 0.045 and e_rcv < 0.04   # discretisation error at 6 elements per wavelength
    finally:
        fb.fb_precond_destroy(inner)
        fb.fb_precond_destroy(pclow)
        fb.fb_operator_destroy(Alow)
        fb.fb_operator_destroy(L64)


def test_largest_rotation_factors_to_degree_158(largest):
    """The rotation data at the largest room's degrees (up to 158; every
    direction from the quarter-turn identity on the device): each real factor
    block d^n is orthogonal, obeys d_{-mu,-m} = d_{mu,m} (the folding of the
    translation kernels relies on it), and its column m = 0 matches the
    closed form sqrt(4 pi/(2n+1)) conj(Y_n^mu(Q z)) evaluated by the oracle's
    spherical harmonics at one point (Q: the rotation taking the direction to
    +z); and the whole block matches the oracle's factors from the rotation
    generator entry by entry (2.7e-13 measured at degrees up to 158 on the
    3,072-element shoebox at 10.8 kHz, which has the same orders)."""
    import math
    from oracle import sph
    wl, mesh, tree, A32, A64 = largest
    n_, L, p = fb.fb_operator_info(A64)
    top = max(p) - 1
    worst = {"orth": 0.0, "sym": 0.0, "col": 0.0, "oracle": 0.0}
    for d in ((2, 0, 0), (2, 2, 2), (3, -1, 2), (-2, 3, -3)):
        code = (d[0] + 3) * 49 + (d[1] + 3) * 7 + (d[2] + 3)
        Q = sph.rotation_to_z(np.array(d, float))
        qz = Q @ np.array([0.0, 0.0, 1.0])
        th = math.acos(d[2] / math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2))
        Y = sph.ylm(top + 1, np.array([math.acos(max(-1.0, min(1.0, qz[2])))]),
                    np.array([math.atan2(qz[1], qz[0])]))[:, 0]
        for n in (0, 1, 40, 97, 131, top):
            w = 2 * n + 1
            dn = fb.fb_operator_export(A64, 8, n, code).real.reshape(w, w)
            worst["orth"] = max(worst["orth"], float(np.max(np.abs(dn @ dn.T - np.eye(w)))))
            worst["sym"] = max(worst["sym"], float(np.max(np.abs(dn[::-1, ::-1] - dn))))
            col = math.sqrt(4 * math.pi / w) * np.conj(Y[n * n:(n + 1) ** 2])
            worst["col"] = max(worst["col"], float(np.max(np.abs(dn[:, n] - col.real))))
            worst["oracle"] = max(worst["oracle"], float(np.max(np.abs(dn - sph.rotation_factor(n, th)))))
            assert np.max(np.abs(col.imag)) < 1e-12   # the m = 0 column carries no phase
    print(f"degree <= {top}: {worst}")
    assert top >= 150
    assert worst["orth"] < 1e-11 and worst["sym"] < 1e-12 and worst["col"] < 1e-11
    assert worst["oracle"] < 1e-11


def test_largest_image_source_sanity(largest):
    """The room's own monopole against the truncated image-source sum of
    Eq. (an2) (images of the shoebox, amplitudes the products of the wall
    reflection coefficients R = (1 - beta)/(1 + beta), dropped below 1e-5;
    the 1e-7 of Sec. 4 would need more than the 64 image orders per axis
    the library allows at these nearly rigid walls):
    the image model's angle-independent reflection is not the impedance
    boundary condition the BEM solves, so the two differ at a model level,
    not to rounding (Sec. 4 reports 16 % for R = 0.8 to 2.56 kHz; here the
    walls reflect more, R = 0.59 to 0.88, at 5 kHz with 6 elements per
    wavelength, and the measured difference is 0.39).  A sanity bound of 0.5
    in relative L2 over the 1,024 receivers, and the check must discriminate:
    the image sum with the reflection coefficients' sign flipped lies far
    outside it."""
    wl, mesh, tree, A32, A64 = largest
    L64 = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_L, fb.FB_PREC_FP64_FMM, 6.0, 12)
    Alow = fb.fb_operator_create(mesh, tree, wl.k, fb.FB_OP_A, fb.FB_PREC_MIXED_FMM, 0.5, 2)
    pclow = fb.fb_precond_create(Alow, fb.FB_PC_BLOCK_JACOBI)
    inner = fb.fb_precond_create_inner(A32, Alow, pclow, 14)
    try:
        src = wl.sources[0]
        g = torch.empty(wl.n, dtype=torch.complex128, device="cuda")
        fb.fb_gamma_monopole(mesh, wl.k, src, g)
        b = torch.empty_like(g)
        fb.fb_operator_apply(L64, g, b)
        x = torch.zeros_like(b)
        info = fb.fb_fgmres_solve(A32, b, x, pc=inner, tol=1e-5, restart=40, maxit=400, max_refine=6, true_op=A64)
        assert info["status"] == 0 and info["true_relres"] <= 1e-5
        rcv = torch.tensor(wl.receivers, device="cuda")
        bem_field = torch.empty(wl.receivers.shape[0], dtype=torch.complex128, device="cuda")
        fb.fb_eval_field(mesh, wl.k, x, g, rcv, bem_field, src=src)
        beta_wall = np.array([wl.beta[wl.wall == w][0] for w in range(6)])
        R = (1 - beta_wall) / (1 + beta_wall)
        img = fb.fb_image_field(wl.room, src, R, wl.k, rcv, a_th=1e-5)[0]
        e = rel(bem_field.cpu().numpy(), img.cpu().numpy())
        bad = fb.fb_image_field(wl.room, src, -R, wl.k, rcv, a_th=1e-5)[0]
        e_bad = rel(bem_field.cpu().numpy(), bad.cpu().numpy())
        print(f"BEM vs image sources at 1,024 receivers: {e:.3f} (reflection signs flipped: {e_bad:.3f}); "
              f"iterations {info['iters']}")
        assert e <= 0.5
        assert e_bad > 1.5 * 0.5
    finally:
        fb.fb_precond_destroy(inner)
        fb.fb_precond_destroy(pclow)
        fb.fb_operator_destroy(Alow)
        fb.fb_operator_destroy(L64)
