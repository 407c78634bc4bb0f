"""Pins for the hypersingular operator M' (Eq. ibem3) of the oracle: the
point kernel against finite differences of dG/dn_y, the self (finite-part)
entry against a polar-coordinate finite-part integral (Laplace and
Helmholtz), and near entries against finite differences of an accurately
integrated double-layer potential."""
import numpy as np
import pytest

from oracle import bem, hypersingular as hs, integrals
from paper_2103_16073_gb300 import workloads as W


def test_kernel_matches_finite_difference():
    rng = np.random.default_rng(0)
    for k in (0.0, 3.0):
        for _ in range(5):
            x = rng.standard_normal(3)
            y = rng.standard_normal(3) + 2.0
            nx = rng.standard_normal(3); nx /= np.linalg.norm(nx)
            ny = rng.standard_normal(3); ny /= np.linalg.norm(ny)
            h = 1e-5

            def dny(xx):
                _, d, _ = bem._kernels(xx, y, ny, nx, k, smooth=False)
                return d
            fd = (dny(x + h * nx) - dny(x - h * nx)) / (2 * h)
            got = hs.kernel_nn(k, y - x, nx, ny)
            assert abs(got - fd) < 1e-7 * abs(got)


def _polar_fp(k, x, verts, nth=4000):
    """(FP int_T d2G/dn dn' dS, int_T G dS) for x inside the flat triangle
    (coplanar: kernel -(ikR-1) e^{ikR}/(4 pi R^3)) in polar coordinates
    around x: (1/4pi) int dtheta [ int_0^rho ((1-ikR)e^{ikR} - 1)/R^2 dR - 1/rho ]
    and (1/4pi) int dtheta (e^{ik rho} - 1)/(ik) (rho at k = 0)."""
    n = np.cross(verts[1] - verts[0], verts[2] - verts[0])
    n /= np.linalg.norm(n)
    e1 = (verts[0] - x) / np.linalg.norm(verts[0] - x)
    e2 = np.cross(n, e1)
    ang = np.sort(np.mod([np.arctan2((v - x) @ e2, (v - x) @ e1) for v in verts], 2 * np.pi))
    bounds = np.append(ang, ang[0] + 2 * np.pi)
    gx, gw = np.polynomial.legendre.leggauss(nth)
    rx, rw = np.polynomial.legendre.leggauss(200)
    total = 0.0 + 0.0j
    single = 0.0 + 0.0j
    for a, b in zip(bounds[:-1], bounds[1:]):
        th = 0.5 * (b - a) * gx + 0.5 * (a + b)
        wt = 0.5 * (b - a) * gw
        dirs = np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2
        rho = np.full(th.size, np.inf)
        for i in range(3):
            p0, p1 = verts[i], verts[(i + 1) % 3]
            d = p1 - p0
            # x + s dir = p0 + u d  (in-plane)
            M = np.stack([dirs, -np.broadcast_to(d, dirs.shape)], axis=-1)   # [nth,3,2]
            sol = np.array([np.linalg.lstsq(Mi, p0 - x, rcond=None)[0] for Mi in M])
            ok = (sol[:, 0] > 0) & (sol[:, 1] >= -1e-12) & (sol[:, 1] <= 1 + 1e-12)
            rho = np.where(ok, np.minimum(rho, sol[:, 0]), rho)
        R = 0.5 * rho[:, None] * (rx[None, :] + 1.0)
        ikR = 1j * k * R
        smooth = np.where(R > 0, ((1.0 - ikR) * np.exp(ikR) - 1.0) / R ** 2, 0.0)
        reg = 0.5 * rho * np.sum(rw[None, :] * smooth, axis=1)
        total += np.sum(wt * (reg - 1.0 / rho))
        single += np.sum(wt * ((np.exp(1j * k * rho) - 1.0) / (1j * k) if k else rho))
    return total / (4 * np.pi), single / (4 * np.pi)


@pytest.mark.parametrize("k", [0.0, 4.0])
def test_self_entry_is_the_finite_part(k):
    v, t, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 4, 3, 3)
    mesh = bem.Mesh(v, t)
    el = mesh.el
    for j in (0, 7, 20):
        got = hs.mp_rows(mesh, k, [j], [j])[0, 0]
        verts = np.stack([el.v0[j], el.v1[j], el.v2[j]])
        ref, s_exact = _polar_fp(k, el.centroid[j], verts)
        # the entry carries k^2 x (error of the single-layer self rule); remove it
        s_rule = bem._self_terms(mesh, k, np.array([j]))[0]
        assert abs(s_rule - s_exact) < 1e-3 * abs(s_exact)   # self rule of L at k h ~ 1.3
        assert abs(got - k * k * (s_rule - s_exact) - ref) < 2e-6 * abs(ref), (j, got, ref)


def _w_accurate(k, x, verts, n, depth=4):
    """Double-layer potential of unit density, int_T dG/dn_y dS, at an
    off-surface point: the closed-form Laplace part (solid angle) plus the
    smooth remainder on 4^depth sub-triangles with the 7-point rule."""
    b7, w7 = bem.rule7()
    tris = [verts]
    for _ in range(depth):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nxt
    om = integrals.solid_angle(x[None], verts[0][None], verts[1][None], verts[2][None])[0]
    val = -om / (4 * np.pi)
    for a, b, c in tris:
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        pts = b7[:, 0, None] * a + b7[:, 1, None] * b + b7[:, 2, None] * c
        _, dny, _ = bem._kernels(x[None], pts, n[None], n[None], k, smooth=True)
        val += area * np.sum(w7 * dny)
    return val


def _s_accurate(k, x, verts, depth=4):
    """int_T G dS at x: closed-form 1/R part plus the smooth remainder on
    4^depth sub-triangles with the 7-point rule."""
    b7, w7 = bem.rule7()
    tris = [verts]
    for _ in range(depth):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nxt
    val = integrals.inv_r(x[None], verts[0][None], verts[1][None], verts[2][None])[0] / (4 * np.pi)
    for a, b, c in tris:
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        pts = b7[:, 0, None] * a + b7[:, 1, None] * b + b7[:, 2, None] * c
        g, _, _ = bem._kernels(x[None], pts, x[None], x[None], k, smooth=True)
        val += area * np.sum(w7 * g)
    return val


@pytest.mark.parametrize("k", [0.0, 3.0])
def test_near_entries_match_finite_differences(k):
    v, t, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 4, 3, 3)
    mesh = bem.Mesh(v, t)
    el = mesh.el
    rng = np.random.default_rng(1)
    checked = 0
    for i in rng.choice(mesh.n, 6, replace=False):
        d = np.linalg.norm(el.centroid - el.centroid[i], axis=1)
        for j in np.nonzero((d < mesh.rc) & (d > 0))[0][:4]:
            got = hs.mp_rows(mesh, k, [i], [j])[0, 0]
            verts = np.stack([el.v0[j], el.v1[j], el.v2[j]])
            x, nx, n = el.centroid[i], el.normal[i], el.normal[j]
            h = 1e-3 * el.max_edge[j]
            f = lambda s: _w_accurate(k, x + s * nx, verts, n)
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
            fd = (4 * d1 - d2) / 3
            # the entry carries (n_x.n) k^2 x (error of the single-layer near rule); remove it
            L, _, _ = bem.operator_rows(mesh, k, x[None], nx[None], [i], [j])
            s_err = L[0, 0] - _s_accurate(k, x, verts)
            assert abs(s_err) < 1e-3 * abs(L[0, 0])   # near rule of L (7-point remainder)
            got = got - np.dot(nx, n) * k * k * s_err
            assert abs(got - fd) < 2e-6 * max(abs(fd), 1e-3 / el.max_edge[j]), (i, j, got, fd)
            checked += 1
    assert checked >= 10
