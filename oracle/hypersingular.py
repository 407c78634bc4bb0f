"""Hypersingular operator M'_k (Eq. ibem3) at the element centroids of flat
triangles with piecewise-constant density (oracle, test infrastructure).

    M'[mu](x) = d/dn_x int_S mu(y) dG(x,y)/dn_y dS_y      (finite part on S)

Entry rule (the GPU path implements the same rule in its own code):
  far (|x - c_j| >= r_c):   three-point rule of the point kernel
      d2G/dn_x dn_y = -e^{ikR}/(4 pi R^3) [(3 - 3ikR - k^2R^2)(n_x.r)(n_y.r)/R^2
                                           + (ikR - 1)(n_x.n_y)],   r = y - x;
  near and self: the double-layer potential of a unit density on the flat
      element is W = -n.grad S with S(x) = int_T G dS, so
      M' = -n_x^T Hess(S) n.  Splitting n_x = (n_x.n) n + t and using
      Helmholtz's equation for the normal-normal part and the in-plane
      divergence theorem (int_T grad_T f dS = sum over edges of int f m dl, m
      the outward in-plane edge normal) for the tangential ones:
        M' = (n_x.n) [k^2 S + sum_e int_e grad_y G . m dl]
             + sum_e int_e (n . grad_x G)(t . m) dl,
      with S the single-layer entry of the same pair (its own closed-form
      rule) and the edge integrals by 8-point Gauss-Legendre on
      min(16, ceil(2 l_e / d_e)) equal segments (d_e = distance from x to the
      edge).  At the element's own centroid (t = 0) this is the finite-part
      value.
"""
from __future__ import annotations

import numpy as np

from . import bem

FOUR_PI = 4.0 * np.pi
GL_X, GL_W = np.polynomial.legendre.leggauss(8)


def kernel_nn(k, r, nx, ny):
    """d2G/dn_x dn_y at point pairs, r = y - x (last axis 3)."""
    R = np.linalg.norm(r, axis=-1)
    ikR = 1j * k * R
    E = np.exp(ikR)
    a = np.sum(nx * r, axis=-1) * np.sum(ny * r, axis=-1) / R ** 2
    b = np.sum(nx * ny, axis=-1)
    return -E / (FOUR_PI * R ** 3) * ((3.0 - 3.0 * ikR + ikR * ikR) * a + (ikR - 1.0) * b)


def _seg_dist(x, p0, p1):
    d = p1 - p0
    s = np.clip(np.dot(x - p0, d) / np.dot(d, d), 0.0, 1.0)
    return np.linalg.norm(x - (p0 + s * d))


def edge_integrals(k, x, nx, verts, n):
    """(A, B): A = sum_e int_e grad_y G . m dl, B = sum_e int_e (n . grad_x G)(t . m) dl
    for one target point x (normal nx) and one triangle (verts[3,3], normal n)."""
    t = nx - np.dot(nx, n) * n
    A = 0.0 + 0.0j
    B = 0.0 + 0.0j
    for e in range(3):
        p0, p1 = verts[e], verts[(e + 1) % 3]
        d = p1 - p0
        le = np.linalg.norm(d)
        tg = d / le
        m = np.cross(tg, n)
        ns = int(min(16, max(1, np.ceil(2.0 * le / _seg_dist(x, p0, p1)))))
        s = (np.arange(ns)[:, None] + 0.5 * (GL_X[None, :] + 1.0)) / ns     # [ns, 8] in (0,1)
        w = np.broadcast_to(GL_W[None, :] * 0.5 / ns * le, s.shape)
        y = p0 + s[..., None] * d
        r = y - x
        R = np.linalg.norm(r, axis=-1)
        ikR = 1j * k * R
        gp = np.exp(ikR) * (ikR - 1.0) / (FOUR_PI * R ** 2)      # g'(R)
        A += np.sum(w * gp * (r @ m) / R)
        B += np.sum(w * (-gp * (r @ n) / R)) * np.dot(t, m)
    return A, B


def mp_rows(mesh, k, rows, cols=None):
    """Rows of M' for collocation at the centroids of elements `rows`."""
    el = mesh.el
    rows = np.asarray(rows)
    cols = np.arange(mesh.n) if cols is None else np.asarray(cols)
    xt = el.centroid[rows]
    nt = el.normal[rows]
    X = xt[:, None, None, :]
    r = mesh.q3[cols][None] - X
    K = kernel_nn(k, r, nt[:, None, None, :], el.normal[cols][None, :, None, :])
    out = el.area[cols][None, :] * np.sum(mesh.w3 * K, axis=-1)
    L, _, _ = bem.operator_rows(mesh, k, xt, nt, rows, cols)
    dist = np.linalg.norm(xt[:, None, :] - el.centroid[cols][None, :, :], axis=-1)
    special = (dist < mesh.rc) | (rows[:, None] == cols[None, :])
    for ri, ci in zip(*np.nonzero(special)):
        j = cols[ci]
        verts = np.stack([el.v0[j], el.v1[j], el.v2[j]])
        n = el.normal[j]
        A, B = edge_integrals(k, xt[ri], nt[ri], verts, n)
        out[ri, ci] = np.dot(nt[ri], n) * (k * k * L[ri, ci] + A) + B
    return out


def dense_mp(mesh, k, chunk=64):
    """Dense hypersingular operator M' of Eq. ibem3 (all collocation rows,
    built in row chunks by mp_rows)."""
    out = np.empty((mesh.n, mesh.n), np.complex128)
    for s in range(0, mesh.n, chunk):
        e = min(mesh.n, s + chunk)
        out[s:e] = mp_rows(mesh, k, np.arange(s, e))
    return out
