"""Pins for the oracle's dense collocation BEM against closed forms and
exact solutions: exterior-source test, rigid-room image sums (exact Neumann
Green's function for complex k), the interior sphere series, reciprocity and
the paper's approximate image model for absorbing walls."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import bem, fgmres, images, integrals
from paper_2103_16073_gb300 import workloads as W


def _solve(mesh, k, beta, gamma):
    L, M, _ = bem.dense_operators(mesh, k)
    A = bem.system_matrix(L, M, k, beta)
    return np.linalg.solve(A, L @ gamma), L, M


def test_near_entries_reduce_to_closed_forms_at_k0():
    """At k = 0 the smooth remainders vanish: near entries are exactly
    (1/4pi) int 1/R, -(1/4pi) Omega and (1/4pi) n_x . int grad(1/R)."""
    v, t, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 5, 4, 3)
    mesh = bem.Mesh(v, t)
    el = mesh.el
    L, M, LP = bem.dense_operators(mesh, 0.0)
    d = np.linalg.norm(el.centroid[:, None] - el.centroid[None], axis=-1)
    ii, jj = np.nonzero((d < mesh.rc) & (d > 0))
    x = el.centroid[ii]
    I1 = integrals.inv_r(x, el.v0[jj], el.v1[jj], el.v2[jj]) / (4 * math.pi)
    Om = integrals.solid_angle(x, el.v0[jj], el.v1[jj], el.v2[jj]) / (4 * math.pi)
    V = integrals.grad_inv_r(x, el.v0[jj], el.v1[jj], el.v2[jj])
    assert np.max(np.abs(L[ii, jj] - I1)) < 1e-15
    assert np.max(np.abs(M[ii, jj] + Om)) < 1e-15
    assert np.max(np.abs(LP[ii, jj] - np.sum(el.normal[ii] * V, -1) / (4 * math.pi))) < 1e-15
    # self terms: M = L' = 0, L = (1/4pi) int 1/R
    s = np.arange(mesh.n)
    assert np.all(M[s, s] == 0) and np.all(LP[s, s] == 0)
    I1s = integrals.inv_r(el.centroid, el.v0, el.v1, el.v2) / (4 * math.pi)
    assert np.max(np.abs(L[s, s] - I1s)) < 1e-15


def test_exterior_source_converges():
    """u = G(r, r_e) with r_e outside the room is regular inside, so it solves
    Eq. (dbem4) with gamma := du/dn - ik beta u; the discrete solution must
    approach u at the centroids under refinement."""
    room = (3.0, 2.4, 2.0)
    k = W.wavenumber(125.0)
    xe = W.exterior_source(room)
    errs = []
    for n in (6, 9, 12):
        v, t, _ = W.shoebox_mesh(*room, n, n, n)
        mesh = bem.Mesh(v, t)
        el = mesh.el
        beta = np.full(mesh.n, 0.2 + 0j)
        u, gu = bem.incident(el.centroid, xe, k)
        g = bem.gamma_field(mesh, k, beta, u, np.sum(gu * el.normal, 1))
        psi, _, _ = _solve(mesh, k, beta, g)
        errs.append(np.linalg.norm(psi - u) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02
    # observed order (h ratio 2/3 then 3/4) at least 1
    assert math.log(errs[0] / errs[2]) / math.log(12 / 6) > 1.0


def test_rigid_room_matches_image_sum_complex_k():
    """beta = 0, complex k: the image sum of Allen & Berkley with A_j = 1 is
    the exact Neumann Green's function of the box (Eq. an2)."""
    room = (1.0, 0.8, 0.6)
    k = 4.0 + 1.5j
    xs = np.array([0.3, 0.35, 0.2])
    rng = np.random.default_rng(3)
    xr = 0.2 + rng.random((16, 3)) * (np.array(room) - 0.4)
    ref = images.image_field(xr, xs, room, k, decay_tol=1e-10)
    errs = []
    for n in ((5, 4, 3), (10, 8, 6), (15, 12, 9)):
        v, t, _ = W.shoebox_mesh(*room, *n)
        mesh = bem.Mesh(v, t)
        beta = np.zeros(mesh.n)
        g = bem.gamma_monopole(mesh, k, beta, xs)
        psi, _, _ = _solve(mesh, k, beta, g)
        f = bem.receiver_field(mesh, k, beta, psi, g, xr, xs)
        errs.append(np.linalg.norm(f - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3


def test_sphere_series():
    """Interior of a sphere of radius a with admittance beta, source r_s:
    psi_sc = sum_n c_n j_n(kr) P_n(cos g),
    c_n = -ik (2n+1)/(4pi) j_n(k r_s) [h_n'(ka) - i beta h_n(ka)] / [j_n'(ka) - i beta j_n(ka)]."""
    a, k, beta0 = 1.0, 2.0, 0.5 + 0.1j
    xs = np.array([0.2, 0.1, -0.3])
    rng = np.random.default_rng(5)
    d = rng.standard_normal((12, 3))
    xr = d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(0.1, 0.6, (12, 1))
    rs = np.linalg.norm(xs)
    r = np.linalg.norm(xr, axis=1)
    cg = (xr @ xs) / (r * rs)
    ka = k * a
    ref = np.zeros(len(xr), np.complex128)
    for n in range(40):
        jn, jnp = special.spherical_jn(n, ka), special.spherical_jn(n, ka, derivative=True)
        hn = jn + 1j * special.spherical_yn(n, ka)
        hnp = jnp + 1j * special.spherical_yn(n, ka, derivative=True)
        c = -1j * k * (2 * n + 1) / (4 * np.pi) * special.spherical_jn(n, k * rs) \
            * (hnp - 1j * beta0 * hn) / (jnp - 1j * beta0 * jn)
        ref += c * special.spherical_jn(n, k * r) * special.eval_legendre(n, cg)
    errs = []
    for sub in (2, 3):
        v, t, _ = W.sphere_mesh(a, sub)
        mesh = bem.Mesh(v, t)
        beta = np.full(mesh.n, beta0)
        g = bem.gamma_monopole(mesh, k, beta, xs)
        psi, _, _ = _solve(mesh, k, beta, g)
        f = bem.receiver_field(mesh, k, beta, psi, g, xr)      # scattered part only
        errs.append(np.linalg.norm(f - ref) / np.linalg.norm(ref))
    assert errs[1] < 0.6 * errs[0]
    assert errs[1] < 0.05


def test_reciprocity():
    room = (1.0, 0.8, 0.6)
    k = W.wavenumber(600.0)
    v, t, _ = W.shoebox_mesh(*room, 12, 10, 8)
    mesh = bem.Mesh(v, t)
    beta = np.full(mesh.n, 0.3 + 0j)
    L, M, _ = bem.dense_operators(mesh, k)
    A = bem.system_matrix(L, M, k, beta)
    ra, rb = np.array([0.25, 0.3, 0.2]), np.array([0.7, 0.5, 0.4])
    out = []
    for src, rec in ((ra, rb), (rb, ra)):
        g = bem.gamma_monopole(mesh, k, beta, src)
        psi = np.linalg.solve(A, L @ g)
        out.append(bem.receiver_field(mesh, k, beta, psi, g, rec[None], src)[0])
    assert abs(out[0] - out[1]) < 0.01 * abs(out[0])


def test_absorbing_room_image_model_sanity():
    """Sec. 4 compares the BEM with the image model (A_j = R^{n_j},
    A_th = 1e-7) and reports ~16% relative L2 mismatch for absorbing walls;
    only a loose sanity bound holds."""
    room = (1.5, 1.2, 1.0)
    k = W.wavenumber(400.0)
    v, t, _ = W.shoebox_mesh(*room, 15, 12, 10)
    mesh = bem.Mesh(v, t)
    beta = np.full(mesh.n, 0.2 + 0j)
    xs = np.array([0.4, 0.5, 0.3])
    rng = np.random.default_rng(9)
    xr = 0.25 + rng.random((24, 3)) * (np.array(room) - 0.5)
    g = bem.gamma_monopole(mesh, k, beta, xs)
    psi, _, _ = _solve(mesh, k, beta, g)
    f = bem.receiver_field(mesh, k, beta, psi, g, xr, xs)
    R = complex(images.reflection_from_admittance(0.2))
    ref = images.image_field(xr, xs, room, k, R_walls=(R,) * 6, a_th=1e-7)
    assert np.linalg.norm(f - ref) / np.linalg.norm(ref) < 0.3


def test_system_rows_match_dense():
    wl = W.shoebox_workload("t", 1.0, 0.8, 0.6, (6, 5, 4), 500.0, 0.2, (0.3, 0.3, 0.3), 4, 0)
    mesh = bem.Mesh(wl.verts, wl.tris)
    L, M, _ = bem.dense_operators(mesh, wl.k)
    A = bem.system_matrix(L, M, wl.k, wl.beta)
    rows = np.array([0, 5, 77, mesh.n - 1])
    assert np.max(np.abs(bem.system_rows(mesh, wl.k, wl.beta, rows) - A[rows])) < 1e-15


def test_fgmres_matches_direct_solve():
    rng = np.random.default_rng(2)
    n = 300
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = fgmres.fgmres(lambda v: A @ v, b, tol=1e-12, restart=20)
    xd = np.linalg.solve(A, b)
    assert info["relres"] <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    # a preconditioner that changes every call (flexible GMRES admits it)
    calls = [0]

    def prec(v):
        calls[0] += 1
        return v / (3.0 + 0.1 * (calls[0] % 3))
    x2, info2 = fgmres.fgmres(lambda v: A @ v, b, tol=1e-12, restart=20, precond=prec)
    assert info2["relres"] <= 1e-12
    assert np.linalg.norm(x2 - xd) / np.linalg.norm(xd) < 1e-10
    # exact solution in one step for A = I (happy breakdown)
    x3, info3 = fgmres.fgmres(lambda v: v, b, tol=1e-14)
    assert info3["iters"] == 1 and np.allclose(x3, b)


def test_baffle_room_exterior_source():
    """Door-and-baffle room (a closed thin box inside the room, its normals
    pointing into the box, out of the air): the exterior-source field solves
    Eq. (dbem4) on the whole boundary, baffle included, and the error falls
    under refinement; with the baffle's normals flipped it does not."""
    room = W.BAFFLE_ROOM
    k = W.wavenumber(125.0)
    xe = W.exterior_source(room)

    def err(h, flip=False):
        v, t, wall = W.baffle_room_mesh(h)
        bf = wall == W.WALL_BAFFLE
        if flip:
            t = t.copy()
            t[bf] = t[bf][:, [0, 2, 1]]
        mesh = bem.Mesh(v, t)
        el = mesh.el
        beta = np.where(bf, 1.0, 0.2).astype(complex)
        u, gu = bem.incident(el.centroid, xe, k)
        g = bem.gamma_field(mesh, k, beta, u, np.sum(gu * el.normal, 1))
        psi, _, _ = _solve(mesh, k, beta, g)
        return np.linalg.norm(psi - u) / np.linalg.norm(u), np.linalg.norm((psi - u)[bf]) / np.linalg.norm(u[bf])

    e0, b0 = err(0.5)
    e1, b1 = err(0.35)
    assert e1 < 0.6 * e0 and b1 < 0.6 * b0 and e1 < 0.03
    ef, _ = err(0.5, flip=True)
    assert ef > 0.3


def test_dbem5_formulation():
    """Eq. (dbem5) (unknown d psi/dn): with constant zeta its matrix is the
    matrix of Eq. (dbem4) and its right-hand side (1/2 I + M) gamma, as the
    paper states; with zeta varying per wall the collocated system is
    diag(beta) A4 diag(1/beta), so psi recovered from its solution through
    the boundary condition equals the dbem4 solution to round-off; and in the
    exterior-source test its solution approaches du/dn under refinement."""
    room = (1.0, 0.8, 0.6)
    k = 6.0
    xs = np.array([0.31, 0.42, 0.27])
    v, t, wall = W.shoebox_mesh(*room, 6, 6, 6)
    mesh = bem.Mesh(v, t)
    L, M, _ = bem.dense_operators(mesh, k)
    beta0 = np.full(mesh.n, 0.2 + 0.05j)
    A4 = bem.system_matrix(L, M, k, beta0)
    assert np.max(np.abs(bem.system_matrix_dbem5(L, M, k, beta0) - A4)) < 1e-14
    g = bem.gamma_monopole(mesh, k, beta0, xs)
    b5 = bem.rhs_dbem5(M, beta0, g)
    assert np.max(np.abs(b5 - (0.5 * g + M @ g))) < 1e-14
    beta = np.array([1.0, 0.002, 0.5, 0.01, 0.3, 0.05 + 0.02j])[wall]
    g = bem.gamma_monopole(mesh, k, beta, xs)
    psi4 = np.linalg.solve(bem.system_matrix(L, M, k, beta), L @ g)
    q = np.linalg.solve(bem.system_matrix_dbem5(L, M, k, beta), bem.rhs_dbem5(M, beta, g))
    assert np.linalg.norm(bem.psi_from_dnpsi(q, g, k, beta) - psi4) < 1e-11 * np.linalg.norm(psi4)
    xe = W.exterior_source(room)
    errs = []
    for nn in (4, 6):
        v, t, wall = W.shoebox_mesh(*room, nn, nn, nn)
        m = bem.Mesh(v, t)
        Lm, Mm, _ = bem.dense_operators(m, k)
        bm = np.array([1.0, 0.002, 0.5, 0.01, 0.3, 0.05 + 0.02j])[wall]
        u, gu = bem.incident(m.el.centroid, xe, k)
        dudn = np.sum(gu * m.el.normal, 1)
        gam = bem.gamma_field(m, k, bm, u, dudn)
        qq = np.linalg.solve(bem.system_matrix_dbem5(Lm, Mm, k, bm), bem.rhs_dbem5(Mm, bm, gam))
        errs.append(np.linalg.norm(qq - dudn) / np.linalg.norm(dudn))
    assert errs[1] < 0.8 * errs[0]
