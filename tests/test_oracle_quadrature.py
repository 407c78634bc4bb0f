"""Pins for the oracle's element quadrature and closed-form integrals."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import geometry, integrals
from paper_2103_16073_gb300 import workloads as W


def _tri_monomial_exact(a, b):
    # int over the unit right triangle of x^a y^b = a! b! / (a+b+2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("rule,deg", [(geometry.rule3, 2), (geometry.rule7, 5)])
def test_gauss_rules_exact_to_degree(rule, deg):
    bary, w = rule()
    assert abs(w.sum() - 1.0) < 1e-15
    # unit right triangle v0=(0,0) v1=(1,0) v2=(0,1), area 1/2
    x = bary[:, 1]
    y = bary[:, 2]
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            q = 0.5 * np.sum(w * x ** a * y ** b)
            assert abs(q - _tri_monomial_exact(a, b)) < 1e-15
    # and not exact one degree higher for some monomial
    errs = [abs(0.5 * np.sum(w * x ** a * y ** (deg + 1 - a)) - _tri_monomial_exact(a, deg + 1 - a))
            for a in range(deg + 2)]
    assert max(errs) > 1e-6


def _brute_tri(f, v0, v1, v2, levels=5):
    """Composite 7-point rule on 4^levels sub-triangles."""
    bary, w = geometry.rule7()
    tris = [(v0, v1, v2)]
    for _ in range(levels):
        nt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nt += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = nt
    A = np.array([t[0] for t in tris])
    B = np.array([t[1] for t in tris])
    C = np.array([t[2] for t in tris])
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A), axis=1)
    pts = bary[None, :, 0, None] * A[:, None] + bary[None, :, 1, None] * B[:, None] + bary[None, :, 2, None] * C[:, None]
    vals = f(pts)
    return np.sum(area[:, None, ...] * (w[None, :, None] if vals.ndim == 3 else w[None, :]) * vals,
                  axis=(0, 1))


def _random_tri(rng):
    v = rng.standard_normal((3, 3))
    return v[0], v[1], v[2]


def test_inv_r_against_brute_force_off_element():
    rng = np.random.default_rng(11)
    for _ in range(12):
        v0, v1, v2 = _random_tri(rng)
        c = (v0 + v1 + v2) / 3
        n = np.cross(v1 - v0, v2 - v0)
        n /= np.linalg.norm(n)
        r = rng.standard_normal(3) * 0.7
        r -= (r @ n) * n                      # in-plane offset, height >= 0.3
        x = c + r + n * (0.3 + rng.random()) * rng.choice([-1.0, 1.0])
        exact = integrals.inv_r(x, v0, v1, v2)
        brute = _brute_tri(lambda p: 1.0 / np.linalg.norm(p - x, axis=-1), v0, v1, v2)
        assert abs(exact - brute) < 1e-9 * abs(brute)


def test_inv_r_in_plane_point_inside_polar_quadrature():
    # x in the plane, inside T: int 1/R dS = int_0^{2pi} rho(theta) dtheta,
    # rho(theta) = distance from x to the boundary along direction theta.
    rng = np.random.default_rng(12)
    for _ in range(5):
        v0, v1, v2 = _random_tri(rng)
        bc = rng.dirichlet([2, 2, 2])
        x = bc[0] * v0 + bc[1] * v1 + bc[2] * v2
        e1 = (v1 - v0) / np.linalg.norm(v1 - v0)
        n = np.cross(v1 - v0, v2 - v0)
        n /= np.linalg.norm(n)
        e2 = np.cross(n, e1)
        P = [np.array([(v - x) @ e1, (v - x) @ e2]) for v in (v0, v1, v2)]

        def rho(th):
            d = np.array([math.cos(th), math.sin(th)])
            best = np.inf
            for i in range(3):
                a, b = P[i], P[(i + 1) % 3]
                M = np.array([d, a - b]).T
                s, t = np.linalg.solve(M, a)
                if s > 0 and -1e-12 <= t <= 1 + 1e-12:
                    best = min(best, s)
            return best
        angs = sorted(math.atan2(p[1], p[0]) % (2 * math.pi) for p in P)
        pts = [0.0] + angs + [2 * math.pi]
        val = sum(integrate.quad(rho, pts[i], pts[i + 1], epsabs=1e-13, epsrel=1e-13)[0]
                  for i in range(len(pts) - 1))
        assert abs(integrals.inv_r(x, v0, v1, v2) - val) < 1e-10 * val


def test_grad_inv_r_is_gradient_of_inv_r():
    rng = np.random.default_rng(13)
    h = 1e-5
    for _ in range(10):
        v0, v1, v2 = _random_tri(rng)
        x = (v0 + v1 + v2) / 3 + rng.standard_normal(3) * 0.8
        g = integrals.grad_inv_r(x, v0, v1, v2)
        fd = np.array([(integrals.inv_r(x + h * e, v0, v1, v2) - integrals.inv_r(x - h * e, v0, v1, v2)) / (2 * h)
                       for e in np.eye(3)])
        # grad_x int 1/|x-y| = int (y-x)/|x-y|^3
        assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_solid_angle_closed_surface():
    """Gauss: a closed outward-oriented surface subtends 4 pi at interior
    points, 2 pi at a smooth surface point (element's own plane excluded),
    0 outside."""
    verts, tris, _ = W.shoebox_mesh(1.0, 0.8, 0.6, 5, 4, 3)
    v = verts[tris]
    v0, v1, v2 = v[:, 0], v[:, 1], v[:, 2]

    def total(x):
        return integrals.solid_angle(np.broadcast_to(x, v0.shape), v0, v1, v2)
    assert abs(total(np.array([0.3, 0.5, 0.2])).sum() - 4 * math.pi) < 1e-12
    assert abs(total(np.array([1.7, 0.5, 0.2])).sum()) < 1e-12
    c = v.mean(axis=1)
    for i in (0, 17, 55):
        om = total(c[i])
        om[i] = 0.0
        assert abs(om.sum() - 2 * math.pi) < 1e-12


def test_paper_mesh_count_golden():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_mesh_counts.json")))
    c = W.paper_shoebox_counts(*g["room_m"], g["max_edge_m"])
    verts, tris, _ = W.shoebox_mesh(*g["room_m"], *c) if False else (None, None, None)
    n = 4 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2])
    assert n == g["n_triangles"]
