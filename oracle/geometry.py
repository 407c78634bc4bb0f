"""Flat-triangle element geometry and Gauss rules (oracle, test infrastructure).

Piecewise-constant collocation on flat triangles (Sec. 4: meshes of flat
triangles; one unknown per element, collocation at the centroid).

Quadrature rules (symmetric Gauss rules on a triangle, Strang & Fix /
Dunavant 1985), written here in barycentric form:
  * 3-point, degree 2: barycentric (2/3,1/6,1/6) and permutations, w = 1/3.
  * 7-point, degree 5 (Radon): centroid w = 9/40; (a,a,1-2a) with
    a = (6-sqrt15)/21, w = (155-sqrt15)/1200; (b,b,1-2b) with
    b = (6+sqrt15)/21, w = (155+sqrt15)/1200.
Weights sum to 1 and are multiplied by the element area.
"""
from __future__ import annotations

import math

import numpy as np


def rule3():
    """Symmetric 3-point rule on a triangle (barycentric points, weights
    summing to 1), exact for polynomials of degree 2: the far-field rule of
    the collocation (the paper leaves the quadrature to the implementer)."""
    bary = np.array([[2 / 3, 1 / 6, 1 / 6],
                     [1 / 6, 2 / 3, 1 / 6],
                     [1 / 6, 1 / 6, 2 / 3]])
    w = np.full(3, 1.0 / 3.0)
    return bary, w


def rule7():
    """Radon's 7-point rule on a triangle (barycentric points, weights
    summing to 1), exact for polynomials of degree 5: the rule for the
    smooth remainder of near and self entries."""
    s15 = math.sqrt(15.0)
    a = (6.0 - s15) / 21.0
    b = (6.0 + s15) / 21.0
    wa = (155.0 - s15) / 1200.0
    wb = (155.0 + s15) / 1200.0
    bary = np.array([[1 / 3, 1 / 3, 1 / 3],
                     [a, a, 1 - 2 * a], [a, 1 - 2 * a, a], [1 - 2 * a, a, a],
                     [b, b, 1 - 2 * b], [b, 1 - 2 * b, b], [1 - 2 * b, b, b]])
    w = np.array([9 / 40, wa, wa, wa, wb, wb, wb])
    return bary, w


class Elements:
    """Per-element geometry in FP64."""

    def __init__(self, verts, tris):
        v = np.asarray(verts, dtype=np.float64)
        t = np.asarray(tris, dtype=np.int64)
        self.v0 = v[t[:, 0]]
        self.v1 = v[t[:, 1]]
        self.v2 = v[t[:, 2]]
        self.centroid = (self.v0 + self.v1 + self.v2) / 3.0
        cr = np.cross(self.v1 - self.v0, self.v2 - self.v0)
        dbl = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * dbl
        self.normal = cr / dbl[:, None]
        e0 = np.linalg.norm(self.v1 - self.v0, axis=1)
        e1 = np.linalg.norm(self.v2 - self.v1, axis=1)
        e2 = np.linalg.norm(self.v0 - self.v2, axis=1)
        self.max_edge = np.maximum(np.maximum(e0, e1), e2)
        self.n = t.shape[0]

    def points(self, bary):
        """Quadrature points [n, q, 3] for barycentric coordinates [q, 3]."""
        return (bary[None, :, 0, None] * self.v0[:, None, :]
                + bary[None, :, 1, None] * self.v1[:, None, :]
                + bary[None, :, 2, None] * self.v2[:, None, :])


def cutoff_radius(max_edge: float) -> float:
    """Near-field cutoff r_c (Sec. 3.3: entries for closely located elements
    use closed-form integrals).  The paper does not state r_c; the reading
    used throughout is r_c = 1.5 x (longest edge in the mesh), measured
    from the collocation point to the source element's centroid."""
    return 1.5 * float(max_edge)
