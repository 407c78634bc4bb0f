"""Closed-form integrals over a flat triangle (oracle, test infrastructure).

Sec. 3.3 computes the matrix entries between closely located elements "using
analytical formulae"; the formulas themselves are not in the paper.  This
module states the classical closed forms used in their place:

* ``inv_r``:    int_T 1/|x-y| dS_y, by the divergence theorem in the plane of
  T (Wilton et al. 1984; Graglia 1993):
      sum_i [ P_i (asinh(l+_i/R0_i) - asinh(l-_i/R0_i))
              - |d| (atan(P_i l+_i/(R0_i^2+|d|R+_i)) - atan(P_i l-_i/(R0_i^2+|d|R-_i))) ]
  where d is the signed height of x above the plane, P_i the in-plane
  distance from the projection of x to edge line i (positive inside),
  l+-_i the edge-tangent coordinates of the edge end points and
  R0_i^2 = P_i^2 + d^2.
* ``solid_angle``: Omega = int_T (y-x).n / |y-x|^3 dS_y, signed, by the
  Van Oosterom & Strackee (1983) formula
      tan(Omega/2) = r0.(r1 x r2) / (r0 r1 r2 + (r0.r1) r2 + (r0.r2) r1 + (r1.r2) r0).
* ``grad_inv_r``: int_T (y-x)/|y-x|^3 dS_y = n Omega - sum_i m_i E_i where
  m_i is the outward in-plane edge normal and E_i = int_edge dl/R.

All functions are vectorised over leading axes and work in FP64.
"""
from __future__ import annotations

import numpy as np


def _edges(v0, v1, v2):
    return ((v0, v1), (v1, v2), (v2, v0))


def _frame(v0, v1, v2):
    cr = np.cross(v1 - v0, v2 - v0)
    n = cr / np.linalg.norm(cr, axis=-1, keepdims=True)
    return n


def _edge_terms(x, v0, v1, v2):
    """Per-edge quantities (P, l-, l+, R0, R-, R+, m, E) for the three edges."""
    n = _frame(v0, v1, v2)
    d = np.sum((x - v0) * n, axis=-1)
    x0 = x - d[..., None] * n
    out = []
    for a, b in _edges(v0, v1, v2):
        e = b - a
        le = np.linalg.norm(e, axis=-1, keepdims=True)
        t = e / le
        m = np.cross(t, n)
        lm = np.sum((a - x0) * t, axis=-1)
        lp = np.sum((b - x0) * t, axis=-1)
        P = np.sum((a - x0) * m, axis=-1)
        R0 = np.sqrt(P * P + d * d)
        R0s = np.maximum(R0, 1e-30 * le[..., 0])
        Rm = np.sqrt(R0 * R0 + lm * lm)
        Rp = np.sqrt(R0 * R0 + lp * lp)
        E = np.arcsinh(lp / R0s) - np.arcsinh(lm / R0s)
        out.append((P, lm, lp, R0, Rm, Rp, m, E))
    return n, d, out


def inv_r(x, v0, v1, v2):
    """int_T 1/|x-y| dS_y for points x and triangles (v0,v1,v2)."""
    n, d, edges = _edge_terms(x, v0, v1, v2)
    ad = np.abs(d)
    total = np.zeros(d.shape)
    for P, lm, lp, R0, Rm, Rp, m, E in edges:
        total += P * E
        total -= ad * (np.arctan2(P * lp, R0 * R0 + ad * Rp)
                       - np.arctan2(P * lm, R0 * R0 + ad * Rm))
    return total


def solid_angle(x, v0, v1, v2):
    """Signed solid angle int_T (y-x).n/|y-x|^3 dS_y (n = right-hand normal)."""
    r0 = v0 - x
    r1 = v1 - x
    r2 = v2 - x
    a0 = np.linalg.norm(r0, axis=-1)
    a1 = np.linalg.norm(r1, axis=-1)
    a2 = np.linalg.norm(r2, axis=-1)
    num = np.sum(r0 * np.cross(r1, r2), axis=-1)
    den = (a0 * a1 * a2 + np.sum(r0 * r1, axis=-1) * a2
           + np.sum(r0 * r2, axis=-1) * a1 + np.sum(r1 * r2, axis=-1) * a0)
    return 2.0 * np.arctan2(num, den)


def grad_inv_r(x, v0, v1, v2):
    """int_T (y-x)/|y-x|^3 dS_y (a 3-vector per pair)."""
    n, d, edges = _edge_terms(x, v0, v1, v2)
    om = solid_angle(x, v0, v1, v2)
    vec = om[..., None] * n
    for P, lm, lp, R0, Rm, Rp, m, E in edges:
        vec = vec - m * E[..., None]
    return vec
