"""Dense collocation BEM for the interior impedance problem (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Problem (Sec. 2): Helmholtz equation, Eq. (sp2), with the impedance wall
condition Eq. (sp3), normal out of the room, time factor e^{-i omega t} and
Green's function G = e^{ikR}/(4 pi R), Eq. (sp6).  With the admittance
beta = 1/zeta the boundary data Eq. (sp7) reads
    dpsi/dn - i k beta psi = gamma,   gamma = -(dpsi_in/dn - i k beta psi_in).
Direct BEM, Eq. (dbem4), with k/(i zeta) = -i k beta:
    A psi = L gamma,   A = 1/2 I + M - i k L diag(beta).
Operators (Eqs. dbem2, ibem3):
    L[s](x)  = int s(y) G(x,y) dS_y
    M[s](x)  = int s(y) dG/dn_y dS_y
    L'[s](x) = int s(y) dG/dn_x dS_y
Discretisation: piecewise-constant values on flat triangles, collocation at
the centroids (free term 1/2: centroids are smooth points, Eq. dbem3).

Entry rule for collocation point x and element T (same rule on every path):
  * self (x is T's own centroid):  L = (1/4pi) int 1/R (closed form)
        + int (G - 1/(4pi R)) by the 7-point rule on the three sub-triangles
        (x, v_a, v_b);  M = L' = 0 (flat element: (y-x).n = 0).
  * near (|x - c_T| < r_c):  closed-form singular part (1/R, solid angle,
        int grad 1/R) + 7-point rule on the smooth remainder.
  * far:  3-point rule.
"""
from __future__ import annotations

import numpy as np

from . import integrals
from .geometry import Elements, rule3, rule7, cutoff_radius

FOUR_PI = 4.0 * np.pi


def expm1c(z):
    """e^z - 1 for complex z without cancellation at small |z|."""
    z = np.asarray(z, dtype=np.complex128)
    a, b = z.real, z.imag
    ea = np.exp(a)
    return (ea * (-2.0 * np.sin(0.5 * b) ** 2) + np.expm1(a)) + 1j * ea * np.sin(b)


def green(x, y, k):
    """Free-space Green's function G = e^{ikR} / (4 pi R), R = |x - y| (Sec. 2,
    the kernel of the boundary integrals of Eq. dbem2)."""
    R = np.linalg.norm(x - y, axis=-1)
    return np.exp(1j * k * R) / (FOUR_PI * R)


def _kernels(x, y, ny, nx, k, smooth):
    """(G, dG/dn_y, dG/dn_x) at point pairs; if smooth, the singular
    Laplace parts 1/(4piR), d/dn_y 1/(4piR), d/dn_x 1/(4piR) are removed."""
    r = y - x
    R = np.linalg.norm(r, axis=-1)
    ikR = 1j * k * R
    E = np.exp(ikR)
    if smooth:
        g = expm1c(ikR) / (FOUR_PI * R)
        f = ikR * E - expm1c(ikR)          # E(ikR-1) + 1
    else:
        g = E / (FOUR_PI * R)
        f = E * (ikR - 1.0)
    inv = 1.0 / (FOUR_PI * R ** 3)
    dny = np.sum(ny * r, axis=-1) * f * inv
    dnx = -np.sum(nx * r, axis=-1) * f * inv
    return g, dny, dnx


class Mesh:
    """Geometry + quadrature data for one mesh."""

    def __init__(self, verts, tris, rc=None):
        self.el = Elements(verts, tris)
        self.n = self.el.n
        self.rc = cutoff_radius(self.el.max_edge.max()) if rc is None else float(rc)
        b3, self.w3 = rule3()
        b7, self.w7 = rule7()
        self.b7 = b7
        self.q3 = self.el.points(b3)     # [n,3,3]
        self.q7 = self.el.points(b7)     # [n,7,3]


def _self_terms(mesh, k, idx):
    """L_ii for elements idx (M_ii = L'_ii = 0)."""
    el = mesh.el
    c = el.centroid[idx]
    out = integrals.inv_r(c, el.v0[idx], el.v1[idx], el.v2[idx]) / FOUR_PI
    out = out.astype(np.complex128)
    verts = (el.v0[idx], el.v1[idx], el.v2[idx])
    for s in range(3):
        a, b = verts[s], verts[(s + 1) % 3]
        cr = np.cross(a - c, b - c)
        asub = 0.5 * np.linalg.norm(cr, axis=-1)
        pts = (mesh.b7[None, :, 0, None] * c[:, None, :]
               + mesh.b7[None, :, 1, None] * a[:, None, :]
               + mesh.b7[None, :, 2, None] * b[:, None, :])
        R = np.linalg.norm(pts - c[:, None, :], axis=-1)
        g = expm1c(1j * k * R) / (FOUR_PI * R)
        out = out + asub * np.sum(mesh.w7[None, :] * g, axis=1)
    return out


def operator_rows(mesh, k, xt, nt, self_idx, cols=None):
    """Rows of (L, M, L') for target points xt[r,3] with normals nt[r,3].

    self_idx[r] = element index whose centroid is xt[r], or -1.
    Returns three complex arrays [r, ncols].
    """
    el = mesh.el
    if cols is None:
        cols = np.arange(mesh.n)
    cols = np.asarray(cols)
    xt = np.asarray(xt, float)
    nt = np.asarray(nt, float)
    r, c = xt.shape[0], cols.size
    X = xt[:, None, None, :]
    NX = nt[:, None, None, :]
    NY = el.normal[cols][None, :, None, :]
    A = el.area[cols][None, :]
    # far rule everywhere first
    g, dny, dnx = _kernels(X, mesh.q3[cols][None], NY, NX, k, smooth=False)
    L = A * np.sum(mesh.w3 * g, axis=-1)
    M = A * np.sum(mesh.w3 * dny, axis=-1)
    LP = A * np.sum(mesh.w3 * dnx, axis=-1)
    # near and self corrections
    dist = np.linalg.norm(xt[:, None, :] - el.centroid[cols][None, :, :], axis=-1)
    is_self = (np.asarray(self_idx)[:, None] == cols[None, :])
    near = (dist < mesh.rc) & ~is_self
    ri, ci = np.nonzero(near)
    if ri.size:
        j = cols[ci]
        x = xt[ri]
        v0, v1, v2 = el.v0[j], el.v1[j], el.v2[j]
        g7, dny7, dnx7 = _kernels(x[:, None, :], mesh.q7[j], el.normal[j][:, None, :],
                                  nt[ri][:, None, :], k, smooth=True)
        aj = el.area[j]
        I1 = integrals.inv_r(x, v0, v1, v2)
        Om = integrals.solid_angle(x, v0, v1, v2)
        V = integrals.grad_inv_r(x, v0, v1, v2)
        L[ri, ci] = I1 / FOUR_PI + aj * np.sum(mesh.w7 * g7, axis=-1)
        M[ri, ci] = -Om / FOUR_PI + aj * np.sum(mesh.w7 * dny7, axis=-1)
        LP[ri, ci] = np.sum(nt[ri] * V, axis=-1) / FOUR_PI + aj * np.sum(mesh.w7 * dnx7, axis=-1)
    si, sc = np.nonzero(is_self)
    if si.size:
        L[si, sc] = _self_terms(mesh, k, cols[sc])
        M[si, sc] = 0.0
        LP[si, sc] = 0.0
    return L, M, LP


def dense_operators(mesh, k, chunk=64):
    """Full N x N matrices (L, M, L') at the centroids."""
    n = mesh.n
    L = np.empty((n, n), np.complex128)
    M = np.empty((n, n), np.complex128)
    LP = np.empty((n, n), np.complex128)
    el = mesh.el
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(s, e)
        L[s:e], M[s:e], LP[s:e] = operator_rows(mesh, k, el.centroid[s:e], el.normal[s:e], idx)
    return L, M, LP


def system_matrix(L, M, k, beta):
    """A = 1/2 I + M - i k L diag(beta)   (Eq. dbem4 with k/(i zeta) = -ik beta)."""
    A = M - 1j * k * L * np.asarray(beta)[None, :]
    A[np.diag_indices_from(A)] += 0.5
    return A


def system_matrix_dbem5(L, M, k, beta):
    """Eq. (dbem5) for the unknown q = d psi_sc/dn:
    1/2 q + (1/zeta) M[zeta q] + (k/(i zeta)) L[q] with zeta = 1/beta, i.e.
    1/2 I + diag(beta) M diag(1/beta) - i k diag(beta) L (beta != 0)."""
    b = np.asarray(beta, dtype=np.complex128)
    A = b[:, None] * M / b[None, :] - 1j * k * b[:, None] * L
    A[np.diag_indices_from(A)] += 0.5
    return A


def rhs_dbem5(M, beta, gamma):
    """Right-hand side of Eq. (dbem5): 1/2 gamma + (1/zeta) M[zeta gamma]."""
    b = np.asarray(beta, dtype=np.complex128)
    return 0.5 * gamma + b * (M @ (gamma / b))


def psi_from_dnpsi(q, gamma, k, beta):
    """psi_sc from q = d psi_sc/dn by the boundary condition of Eq. (sp7):
    q - i k beta psi_sc = gamma."""
    return (q - gamma) / (1j * k * np.asarray(beta))


def system_rows(mesh, k, beta, rows):
    """Rows of A (Eq. dbem4) for element indices ``rows`` (for sampled checks)."""
    rows = np.asarray(rows)
    el = mesh.el
    L, M, _ = operator_rows(mesh, k, el.centroid[rows], el.normal[rows], rows)
    A = M - 1j * k * L * np.asarray(beta)[None, :]
    A[np.arange(rows.size), rows] += 0.5
    return A


def incident(x, xs, k):
    """psi_in = G(x, r_s) and grad_x psi_in, Eq. (sp6)."""
    r = x - xs
    R = np.linalg.norm(r, axis=-1)
    E = np.exp(1j * k * R)
    g = E / (FOUR_PI * R)
    grad = r * (E * (1j * k * R - 1.0) / (FOUR_PI * R ** 3))[..., None]
    return g, grad


def gamma_monopole(mesh, k, beta, xs):
    """gamma = -(dpsi_in/dn - i k beta psi_in) at the centroids, Eq. (sp7)."""
    el = mesh.el
    g, grad = incident(el.centroid, np.asarray(xs, float), k)
    dn = np.sum(grad * el.normal, axis=-1)
    return -(dn - 1j * k * np.asarray(beta) * g)


def gamma_field(mesh, k, beta, u, dudn):
    """Boundary data for a prescribed field u regular in the room:
    gamma = du/dn - i k beta u (the exterior-source test)."""
    return dudn - 1j * k * np.asarray(beta) * u


def receiver_field(mesh, k, beta, psi_sc, gamma, xr, xs=None, chunk=64):
    """Field at interior points by Green's identity, Eq. (dbem1):
    psi_sc(r) = L[dpsi_sc/dn](r) - M[psi_sc](r), dpsi_sc/dn = gamma + ik beta psi_sc.
    Adds psi_in if a source xs is given."""
    xr = np.asarray(xr, float)
    q = gamma + 1j * k * np.asarray(beta) * psi_sc
    out = np.empty(xr.shape[0], np.complex128)
    dummy_n = np.zeros_like(xr)
    for s in range(0, xr.shape[0], chunk):
        e = min(xr.shape[0], s + chunk)
        L, M, _ = operator_rows(mesh, k, xr[s:e], dummy_n[s:e], -np.ones(e - s, int))
        out[s:e] = L @ q - M @ psi_sc
    if xs is not None:
        g, _ = incident(xr, np.asarray(xs, float), k)
        out = out + g
    return out
