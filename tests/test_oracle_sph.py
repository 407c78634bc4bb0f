"""Pins for the oracle's spherical basis, coaxial recursions (Sec. 3.3.1),
rotations and composed RCR translations."""
import functools
import math

import numpy as np
import pytest
from scipy import special

from oracle import sph


def _nm(p):
    n_of = np.repeat(np.arange(p), 2 * np.arange(p) + 1)
    m_of = np.concatenate([np.arange(-n, n + 1) for n in range(p)])
    return n_of, m_of


def test_ylm_matches_library_with_convention_factor():
    p = 25
    rng = np.random.default_rng(0)
    th = rng.random(40) * np.pi
    ph = rng.random(40) * 2 * np.pi - np.pi
    n_of, m_of = _nm(p)
    Ys = special.sph_harm_y(n_of[:, None], m_of[:, None], th[None], ph[None])
    eps = np.where(m_of >= 0, (-1.0) ** np.abs(m_of), 1.0)
    assert np.max(np.abs(eps[:, None] * Ys - sph.ylm(p, th, ph))) < 1e-13
    # Y_n^{-m} = conj(Y_n^m)
    Y = sph.ylm(p, th, ph)
    neg = np.array([sph.idx(n, -m) for n, m in zip(n_of, m_of)])
    assert np.max(np.abs(Y[neg] - np.conj(Y))) < 1e-15


@pytest.mark.parametrize("k", [0.7, 2.0, 9.0])
def test_green_addition_theorem(k):
    """G(x,y) = ik sum S_n^m(x-c) R_n^{-m}(y-c) for |x-c| > |y-c|."""
    rng = np.random.default_rng(1)
    c = rng.standard_normal(3)
    p = 45
    n_of, m_of = _nm(p)
    neg = np.array([sph.idx(n, -m) for n, m in zip(n_of, m_of)])
    for _ in range(4):
        y = c + rng.standard_normal(3) * 0.1
        x = c + rng.standard_normal(3)
        x = c + (x - c) / np.linalg.norm(x - c) * 1.3
        S = sph.singular(p, k, x - c)
        R = sph.regular(p, k, y - c)
        G = np.exp(1j * k * np.linalg.norm(x - y)) / (4 * np.pi * np.linalg.norm(x - y))
        assert abs(1j * k * np.sum(S * R[neg]) - G) < 1e-13 * abs(G)


def test_grad_regular_finite_difference():
    p, k = 10, 3.0
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(5):
        r = rng.standard_normal(3) * 0.4
        g = sph.grad_regular(p, k, r)
        fd = np.stack([(sph.regular(p, k, r + h * e) - sph.regular(p, k, r - h * e)) / (2 * h)
                       for e in np.eye(3)], -1)
        assert np.max(np.abs(g - fd)) < 1e-8


@pytest.mark.parametrize("ktau", [0.3, 0.9, 3.0, 12.0])
@pytest.mark.parametrize("kind", ["SR", "RR"])
@pytest.mark.parametrize("scheme", ["original", "stabilized"])
def test_coaxial_addition_theorem(ktau, kind, scheme):
    """F_n^m(r + tau z) = sum_n' (E|F)^m_{n'n} R_n'^m(r): checked column by
    column against direct evaluation (truncation made negligible by a large
    row count and |r| = 0.1 tau)."""
    k = 1.7
    tau = ktau / k
    p, big = 10, 36
    X = sph.coaxial(big, ktau, kind, scheme)
    r = np.array([0.06, -0.05, 0.055]) * tau
    F = sph.singular if kind == "SR" else sph.regular
    lhs = F(p, k, r + np.array([0.0, 0.0, tau]))
    Rv = sph.regular(big, k, r)
    n_of, m_of = _nm(p)
    for q, (n, m) in enumerate(zip(n_of, m_of)):
        s = sum(X[abs(m), n1, n] * Rv[sph.idx(n1, m)] for n1 in range(abs(m), big))
        assert abs(s - lhs[q]) <= 1e-11 * max(1.0, abs(lhs[q]))


def test_coaxial_projection_quadrature():
    """(S|R)^m_{n'n}(tau) = int conj(Y_n'^m) S_n^m(a u + tau z) dOmega / j_n'(ka)."""
    k, tau, a, p = 2.0, 1.5, 0.5, 8
    X = sph.coaxial(p, k * tau, "SR")
    nq = 40
    xg, wg = np.polynomial.legendre.leggauss(nq)
    phis = 2 * np.pi * np.arange(2 * nq) / (2 * nq)
    TH, PH = np.meshgrid(np.arccos(xg), phis, indexing="ij")
    W = (wg[:, None] * np.full(2 * nq, np.pi / nq)).ravel()
    u = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    S = sph.singular(p, k, a * u + np.array([0, 0, tau]))
    Y = sph.ylm(p, np.arccos(u[:, 2]), np.arctan2(u[:, 1], u[:, 0]))
    j = special.spherical_jn(np.arange(p), k * a)
    for n in range(p):
        for n1 in range(p):
            for m in range(-min(n, n1), min(n, n1) + 1):
                proj = np.sum(W * np.conj(Y[sph.idx(n1, m)]) * S[sph.idx(n, m)]) / j[n1]
                assert abs(proj - X[abs(m), n1, n]) < 1e-9 * max(1.0, abs(proj))


def test_printed_shft8_third_formula_fails_corrected_holds():
    """The third formula of Eq. (shft8) as printed (last coefficient
    b_{n+1}^{-m-1}) does not reproduce exact coefficients; with b_n^{-m-1}
    it does (the reading the oracle uses)."""
    p, ktau = 24, 20.0
    ref = sph.coaxial(p, ktau, "SR", "original")
    good = sph.coaxial(p, ktau, "SR", "stabilized")
    bad = sph.coaxial(p, ktau, "SR", "stabilized", misprint=True)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(good - ref)) < 1e-13 * scale
    assert np.max(np.abs(bad - ref)) > 1e-6 * scale


def test_stabilized_scheme_stable_where_original_is_not():
    """Sec. 3.3.1: n-propagation (original step 3) is CFL-unstable for n' > n
    at large k tau; the stabilized scheme is not.  Reference: the stabilized
    steps run in 40-digit arithmetic (their values are pinned independently
    by the projection test at order 159)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    p, ktau = 100, 300.0
    ref = sph.coaxial(p, ktau, "SR", "stabilized", mp=mpmath.mp)
    R = np.vectorize(complex)(ref)
    scale = np.max(np.abs(R))
    e_orig = np.max(np.abs(sph.coaxial(p, ktau, "SR", "original") - R)) / scale
    e_stab = np.max(np.abs(sph.coaxial(p, ktau, "SR", "stabilized") - R)) / scale
    assert e_stab < 1e-13
    assert e_orig > 1e3 * e_stab


@functools.lru_cache(maxsize=None)
def _gauss_legendre(nodes):
    return np.polynomial.legendre.leggauss(nodes)


def _coax_by_projection(kind, m, n1, n, ktau, nodes=3000):
    """(E|F)^m_{n'n}(tau) from its definition by projection, reduced to one
    dimension: a coaxial shift keeps the azimuth of a u + tau z equal to
    that of u, so with Y_n^m = P_n^m(theta) e^{i m phi} (scipy's normalised
    P_n^m; its (-1)^m cancels in the product of two equal-m functions)
        (E|F)^m_{n'n} j_n'(k a) = 2 pi int_{-1}^{1} P_n'^m(x) f_n(k rho) P_n^m(theta') dx,
    rho = |a u + tau z|, cos theta' = (a x + tau) / rho, f = h (S|R) or j
    (R|R); Gauss-Legendre in x.  k = 1 (only k tau matters).  The radius a
    puts k a just past the first maximum of j_n' (so the division does not
    amplify), below tau for S|R (where the expansion converges); returns the
    value and the rounding floor eps sqrt(nodes) max|integrand| / |j_n'(k a)|."""
    tau = ktau
    a = n1 + 0.81 * n1 ** (1.0 / 3.0) + 1.0
    if kind == "SR":
        assert a < 0.9 * tau
    elif abs(a - tau) < 0.05 * tau:
        a = 1.1 * tau if a > tau else 0.9 * tau
    x, w = _gauss_legendre(nodes)
    rho = np.sqrt(a * a + tau * tau + 2 * a * tau * x)
    th2 = np.arccos(np.clip((a * x + tau) / rho, -1.0, 1.0))
    f = special.spherical_jn(n, rho).astype(np.complex128)
    if kind == "SR":
        f += 1j * special.spherical_yn(n, rho)
    g = 2 * np.pi * special.sph_legendre_p(n1, m, np.arccos(x)) * f * special.sph_legendre_p(n, m, th2)
    j1 = special.spherical_jn(n1, a)
    return np.sum(w * g) / j1, 2.2e-16 * math.sqrt(nodes) * np.max(np.abs(g)) / abs(j1)


@pytest.mark.parametrize("kind, ktau", [("SR", 300.0), ("SR", 773.0), ("RR", 64.0)])
def test_coaxial_projection_at_order_159(kind, ktau):
    """Coaxial coefficients at order 159 against their projection definition
    (sampled entries: corners, sectorial, the high-degree corner at middle
    orders, random): the 6.5 x 5.5 x 4.2 m room
    at 5 kHz translates its level-2 M2L at k tau = 298..773 and its level-3
    M2M / L2L at k tau = 64 with these orders.  Tolerance: 1e-12 of the
    largest entry plus 50x the projection's own rounding floor (which is
    loose only where n' + n exceeds k tau, for the reference's sake)."""
    p = 159
    X = sph.coaxial(p, ktau, kind)
    scale = np.max(np.abs(X))
    rng = np.random.default_rng(15)
    picks = [(0, 0, 0), (0, p - 1, p - 1), (0, 0, p - 1), (0, p - 1, 0), (p - 1, p - 1, p - 1),
             (100, 158, 120), (1, 2, 157)]
    # the high-degree corner at middle orders, where an unstable recursion
    # goes wrong first
    picks += [(m, n1, n) for m in (20, 39, 59, 80, 120) for n1, n in ((157, 158), (158, 158), (158, 140))]
    for _ in range(16):
        m = int(rng.integers(0, p))
        a, b = rng.integers(m, p, 2)
        picks.append((m, int(a), int(b)))
    for m, n1, n in picks:
        ref, floor = _coax_by_projection(kind, m, n1, n, ktau)
        assert abs(X[m, n1, n] - ref) <= 1e-12 * scale + 50 * floor, (m, n1, n)


def _rcr_apply(cin, t, k, p, kind):
    """Rotation - coaxial - back-rotation (Sec. 3.3) applied to coefficient
    vectors (columns of cin, flat index n^2 + n + m) degree by degree, as the
    composed matrix of sph.translation would (which is p^2 x p^2 and too
    large at order 159): u^n = D^n c^n, v = (E|F) u per order m,
    out^n = D^n^H v^n, with D^n = d^n(theta) e^{i m phi} of t's direction."""
    tau = float(np.linalg.norm(t))
    th, ph = math.acos(t[2] / tau), math.atan2(t[1], t[0])
    X = sph.coaxial(p, k * tau, kind)
    D = []
    u = np.zeros_like(cin)
    for n in range(p):
        m = np.arange(-n, n + 1)
        D.append(sph.rotation_factor(n, th) * np.exp(1j * m * ph)[None, :])
        u[n * n:(n + 1) ** 2] = D[n] @ cin[n * n:(n + 1) ** 2]
    v = np.zeros_like(cin)
    for mm in range(-(p - 1), p):
        a = abs(mm)
        rows = [sph.idx(n, mm) for n in range(a, p)]
        v[rows] = X[a, a:p, a:p] @ u[rows]
    out = np.zeros_like(cin)
    for n in range(p):
        out[n * n:(n + 1) ** 2] = D[n].conj().T @ v[n * n:(n + 1) ** 2]
    return out


@pytest.mark.parametrize("kind", ["SR", "RR"])
def test_rcr_translation_addition_theorem_at_order_159(kind):
    """The whole RCR chain at order 159 (generator-form rotations, stabilized
    coaxial coefficients) against the Green's function of point sources:
    S|R (M2L) at k tau = 300 along (2, -1, 2) with sources and receivers
    within k r = 60 of the two centres; R|R (M2M, t = parent - child) at
    k tau = 64 along (1, 1, -1) with sources within k r = 20 of the child
    and receivers at k r = 200 from the parent (the 6.5 x 5.5 x 4.2 m room's
    level-2 M2L and level-3 M2M at 5 kHz, with k = 1)."""
    p, k = 159, 1.0
    rng = np.random.default_rng(16)

    def around(c, r, count):
        v = rng.standard_normal((count, 3))
        return c + r * v / np.linalg.norm(v, axis=1)[:, None]

    neg = np.array([sph.idx(n, -m) for n in range(p) for m in range(-n, n + 1)])
    c1 = np.zeros(3)
    if kind == "SR":
        t = np.array([2.0, -1.0, 2.0]) * 100.0
        src, rcv = around(c1, 60.0, 3), around(c1 + t, 60.0, 3)
    else:
        t = np.array([1.0, 1.0, -1.0]) / math.sqrt(3.0) * 64.0
        src, rcv = around(c1, 20.0, 3), around(c1 + t, 200.0, 3)
    # multipole coefficients of each source about c1: G(x, y) = ik sum S_n^m(x - c) R_n^-m(y - c)
    C = np.stack([1j * k * sph.regular(p, k, y - c1)[neg] for y in src], axis=1)
    out = _rcr_apply(C, t, k, p, kind)
    F = sph.regular if kind == "SR" else sph.singular
    for x in rcv:
        basis = F(p, k, x - (c1 + t))
        for j, y in enumerate(src):
            r = np.linalg.norm(x - y)
            g = np.exp(1j * k * r) / (4 * math.pi * r)
            assert abs(np.sum(out[:, j] * basis) - g) < 1e-12 * abs(g)


def _random_rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def test_rotation_blocks_definition_unitarity_composition():
    rng = np.random.default_rng(4)
    p = 12
    Q1, Q2 = _random_rotation(rng), _random_rotation(rng)
    D1 = sph.rotation_blocks(Q1, p)
    D2 = sph.rotation_blocks(Q2, p)
    D12 = sph.rotation_blocks(Q2 @ Q1, p)
    # pointwise definition: Y_n^m(x) = sum_m' D_{m'm} Y_n^m'(Q x)
    x = rng.standard_normal((20, 3))
    x /= np.linalg.norm(x, axis=1)[:, None]
    qx = x @ Q1.T
    Y = sph.ylm(p, np.arccos(x[:, 2]), np.arctan2(x[:, 1], x[:, 0]))
    Yq = sph.ylm(p, np.arccos(qx[:, 2]), np.arctan2(qx[:, 1], qx[:, 0]))
    for n in range(p):
        s = slice(n * n, (n + 1) ** 2)
        assert np.max(np.abs(D1[n].T @ Yq[s] - Y[s])) < 1e-13
        assert np.max(np.abs(D1[n] @ D1[n].conj().T - np.eye(2 * n + 1))) < 1e-13
        # first Q1 then Q2: coefficients transform by D(Q2) D(Q1)
        assert np.max(np.abs(D2[n] @ D1[n] - D12[n])) < 1e-13
    # rotation about z by a: Y^m(R_z x) = e^{ima} Y^m(x), so D = diag(e^{-ima})
    a = 0.7
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Dz = sph.rotation_blocks(Rz, p)
    for n in range(p):
        m = np.arange(-n, n + 1)
        assert np.max(np.abs(Dz[n] - np.diag(np.exp(-1j * m * a)))) < 1e-13


@pytest.mark.parametrize("kind", ["SR", "RR"])
def test_composed_translation_addition_theorem(kind):
    """RCR-composed translation reproduces S (or R) about a shifted centre."""
    rng = np.random.default_rng(6)
    k = 2.3
    p_in, p_out = 9, 34
    for _ in range(3):
        t = rng.standard_normal(3)
        t *= 1.2 / np.linalg.norm(t)
        T = sph.translation(t, k, p_out, p_in, kind)
        r = rng.standard_normal(3) * 0.05
        F = sph.singular if kind == "SR" else sph.regular
        lhs = F(p_in, k, r + t)
        rhs = T.T @ sph.regular(p_out, k, r)
        assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(lhs))


def test_multipole_to_multipole_translation():
    """(S|S) = (R|R): S_n^m(r + t) = sum (R|R)_{n'n}(t) S_n'^m(r), |r| > |t|."""
    rng = np.random.default_rng(7)
    k = 1.9
    t = rng.standard_normal(3)
    t *= 0.2 / np.linalg.norm(t)
    p_in, p_out = 8, 40
    T = sph.translation(t, k, p_out, p_in, "RR")
    r = rng.standard_normal(3)
    r *= 2.0 / np.linalg.norm(r)
    lhs = sph.singular(p_in, k, r + t)
    rhs = T.T @ sph.singular(p_out, k, r)
    assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(lhs))


def test_rotation_factors_from_quarter_turn_identity():
    """The real factors d^n(theta) of the rotation blocks (D = d e^{i m phi})
    follow from the single matrix Delta^n = d^n(pi/2) by
    d_{mu,m}(theta) = sum_k Delta_{mu,k} Delta_{m,k} cos(k theta + (mu - m) pi/2)
    (a rotation about y written as a rotation about z between quarter turns);
    checked against the projection of the rotation definition for axis,
    diagonal and general directions up to degree 39."""
    p = 40
    Dl = [b.real for b in sph.rotation_blocks(sph.rotation_to_z(np.array([1.0, 0.0, 0.0])), p)]
    worst = 0.0
    for t in ([0, 0, 1.0], [0, 0, -1.0], [2, -3, 1.0], [-1, -1, -3.0], [3, 3, 3.0], [1, 0, -2.0]):
        t = np.asarray(t)
        th = np.arccos(t[2] / np.linalg.norm(t))
        ph = np.arctan2(t[1], t[0])
        D = sph.rotation_blocks(sph.rotation_to_z(t), p)
        for n in range(p):
            m = np.arange(-n, n + 1)
            C = np.cos(m[None, None, :] * th + (m[:, None, None] - m[None, :, None]) * np.pi / 2)
            d = np.einsum("ak,bk,abk->ab", Dl[n], Dl[n], C)
            worst = max(worst, float(np.max(np.abs(d * np.exp(1j * m[None, :] * ph) - D[n]))))
    assert worst < 1e-12


def _real_factor(t, p):
    """d^n of direction t: the rotation blocks with the phase e^{i m phi} of
    the input index removed (D^n_{mu,m} = d^n_{mu,m} e^{i m phi})."""
    t = np.asarray(t, float)
    ph = math.atan2(t[1], t[0])
    D = sph.rotation_blocks(sph.rotation_to_z(t), p)
    out = []
    for n in range(p):
        m = np.arange(-n, n + 1)
        d = D[n] * np.exp(-1j * m[None, :] * ph)
        assert np.max(np.abs(d.imag)) < 1e-13
        out.append(d.real)
    return out


def test_rotation_factor_symmetry_and_polar_angle_sharing():
    """The folded rotations of the translation kernels rest on two facts of
    the definition: d^n_{-mu,-m} = d^n_{mu,m}, and d^n depends on the polar
    angle of the direction only (directions of equal theta share it)."""
    p = 24
    base = _real_factor([2.0, 1.0, 2.0], p)
    same = [[1.0, 2.0, 2.0], [-2.0, 1.0, 2.0], [2.0, -1.0, 2.0]]   # |t| = 3, t_z = 2: same theta
    for t in same:
        d = _real_factor(t, p)
        for n in range(p):
            assert np.max(np.abs(d[n] - base[n])) < 1e-13
    for t in ([2.0, 1.0, 2.0], [1.0, -3.0, -1.0], [0.0, 0.0, 1.0], [1.0, 1.0, 0.0]):
        d = _real_factor(t, p)
        for n in range(p):
            assert np.max(np.abs(d[n][::-1, ::-1] - d[n])) < 1e-13


def test_folded_rotation_reproduces_plain_rotation():
    """Even / odd folding of one rotation block, as the kernels compute it:
    with s_m = x_m + x_{-m}, t_m = x_m - x_{-m}, s_0 = x_0,
    E_mu = 2 d_{mu,0} s_0 + sum_{m>0} (d_{mu,m} + d_{mu,-m}) s_m = u_mu + u_{-mu}
    and O_mu = sum_{m>0} (d_{mu,m} - d_{mu,-m}) t_m = u_mu - u_{-mu} for
    u = d x; the back-rotation folds the same way with d^T."""
    rng = np.random.default_rng(11)
    p = 20
    d_all = _real_factor([1.0, -2.0, 3.0], p)
    for n in (0, 1, 7, 19):
        d = d_all[n]
        x = rng.standard_normal(2 * n + 1) + 1j * rng.standard_normal(2 * n + 1)
        u = d @ x
        c = n   # index of m = 0
        s = np.array([x[c]] + [x[c + m] + x[c - m] for m in range(1, n + 1)])
        tt = np.array([x[c + m] - x[c - m] for m in range(1, n + 1)])
        for mu in range(0, n + 1):
            E = 2 * d[c + mu, c] * s[0] + sum((d[c + mu, c + m] + d[c + mu, c - m]) * s[m] for m in range(1, n + 1))
            assert abs(E - (u[c + mu] + u[c - mu])) < 1e-12 * (1 + np.abs(u).max())
            if mu > 0:
                O = sum((d[c + mu, c + m] - d[c + mu, c - m]) * tt[m - 1] for m in range(1, n + 1))
                assert abs(O - (u[c + mu] - u[c - mu])) < 1e-12 * (1 + np.abs(u).max())
        # back-rotation y = d^T v from the folded v
        v = rng.standard_normal(2 * n + 1) + 1j * rng.standard_normal(2 * n + 1)
        y = d.T @ v
        Ev = np.array([2 * v[c]] + [v[c + mu] + v[c - mu] for mu in range(1, n + 1)])
        Ov = np.array([v[c + mu] - v[c - mu] for mu in range(1, n + 1)])
        for mp in range(0, n + 1):
            Yp = d[c, c + mp] * Ev[0] + sum((d[c + mu, c + mp] + d[c - mu, c + mp]) * Ev[mu] for mu in range(1, n + 1))
            Ym = sum((d[c + mu, c + mp] - d[c - mu, c + mp]) * Ov[mu - 1] for mu in range(1, n + 1))
            assert abs((Yp + Ym) / 2 - y[c + mp]) < 1e-12 * (1 + np.abs(y).max())
            assert abs((Yp - Ym) / 2 - y[c - mp]) < 1e-12 * (1 + np.abs(y).max())


def test_rotation_column_closed_form():
    """Column m = 0 of every block from the addition theorem:
    D^n_{mu,0} = sqrt(4 pi / (2n+1)) conj(Y_n^mu(Q z)) (the projection of
    Y_n^0(Q^T y) = sqrt((2n+1)/(4 pi)) P_n((Q z).y) on Y_n^mu), against the
    projection quadrature of the definition; the closed form needs Y_n^mu at
    one point only, so it also checks rotation data at degrees the
    projection cannot reach here."""
    p = 30
    rng = np.random.default_rng(12)
    for t in (rng.standard_normal(3), [1.0, 1.0, 1.0], [0.0, -2.0, 1.0]):
        t = np.asarray(t, float)
        Q = sph.rotation_to_z(t)
        D = sph.rotation_blocks(Q, p)
        qz = Q @ np.array([0.0, 0.0, 1.0])
        Y = sph.ylm(p, np.array([math.acos(max(-1.0, min(1.0, qz[2])))]), np.array([math.atan2(qz[1], qz[0])]))[:, 0]
        for n in range(p):
            col = math.sqrt(4 * math.pi / (2 * n + 1)) * np.conj(Y[n * n:(n + 1) ** 2])
            assert np.max(np.abs(D[n][:, n] - col)) < 1e-13


def test_ylm_unsold_identity_to_degree_158():
    """Unsold's theorem, sum_m |Y_n^m(x)|^2 = (2n+1)/(4 pi), at every degree
    below 159 and several points: the spherical harmonics the closed-form
    rotation check evaluates at the largest room's degrees."""
    p = 159
    rng = np.random.default_rng(13)
    th = np.concatenate([[0.0, math.pi / 2, 1e-3], rng.uniform(0, math.pi, 5)])
    ph = rng.uniform(-math.pi, math.pi, th.size)
    Y = sph.ylm(p, th, ph)
    for n in range(p):
        s = np.sum(np.abs(Y[n * n:(n + 1) ** 2]) ** 2, axis=0)
        assert np.max(np.abs(s - (2 * n + 1) / (4 * math.pi))) < 1e-11 * (2 * n + 1)


# Degrees for the high-degree rotation pins: the largest room's orders reach
# 159 (rotation degree 158), the GPU setup accepts orders to 256, and 318 is
# twice the largest room's order.
_HIGH_DEGREES = (0, 1, 2, 17, 40, 64, 101, 158, 159, 200, 255, 318)
_THETAS = (1e-3, 0.4, math.pi / 2, 2.2, math.pi - 1e-3)


def test_rotation_factor_generator_matches_projection():
    """The generator form of the real factors against the projection of the
    rotation definition (rotation_blocks) for general, axis-near and
    lower-hemisphere directions, every degree below 40."""
    p = 40
    for t in ([1.0, -2.0, 0.7], [0.3, 0.1, 5.0], [-1.0, 2.0, -3.0], [2.0, 1.0, 0.0]):
        t = np.asarray(t)
        th = math.acos(t[2] / np.linalg.norm(t))
        ph = math.atan2(t[1], t[0])
        D = sph.rotation_blocks(sph.rotation_to_z(t), p)
        for n in range(p):
            m = np.arange(-n, n + 1)
            assert np.max(np.abs(sph.rotation_factor(n, th) * np.exp(1j * m[None, :] * ph) - D[n])) < 1e-12


def test_rotation_factor_column_closed_form_to_degree_318():
    """Column m = 0 at high degree: with Q z at polar angle theta and azimuth
    pi, D^n_{mu,0} = sqrt(4 pi / (2n+1)) conj(Y_n^mu(Q z)) (the addition
    theorem), so d^n_{mu,0}(theta) = sqrt(4 pi / (2n+1)) (-1)^mu Q_n^|mu|(theta)
    from the Legendre recursion of ylm, independent of the generator."""
    p = 319
    th = np.array(_THETAS)
    Y = sph.ylm(p, th, np.full(th.size, math.pi))
    for n in _HIGH_DEGREES:
        col_ref = math.sqrt(4 * math.pi / (2 * n + 1)) * np.conj(Y[n * n:(n + 1) ** 2])
        assert np.max(np.abs(col_ref.imag)) < 1e-12
        for i, t in enumerate(_THETAS):
            d = sph.rotation_factor(n, t)
            assert np.max(np.abs(d[:, n] - col_ref[:, i].real)) < 1e-12, (n, t)


def _wigner_sum(n, mu, m, beta, digits=300):
    """d^n_{mu,m}(beta) of the Condon-Shortley convention by Wigner's
    explicit finite sum, in `digits`-digit arithmetic (its terms reach about
    4^n before they cancel)."""
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(digits):
        f = [mpmath.factorial(i) for i in range(2 * n + 1)]
        c, s = mpmath.cos(mpmath.mpf(beta) / 2), mpmath.sin(mpmath.mpf(beta) / 2)
        pre = mpmath.sqrt(f[n + mu] * f[n - mu] * f[n + m] * f[n - m])
        acc = mpmath.mpf(0)
        for k in range(max(0, m - mu), min(n + m, n - mu) + 1):
            term = pre / (f[n + m - k] * f[k] * f[mu - m + k] * f[n - mu - k])
            term *= c ** (2 * n + m - mu - 2 * k) * s ** (mu - m + 2 * k)
            acc += -term if (mu - m + k) % 2 else term
        return float(acc)


def test_rotation_factor_exact_sum_at_high_degree():
    """Sampled entries (corners, centre, random) of d^n(theta) at degrees 158
    and 318 against Wigner's explicit sum in 300-digit arithmetic:
    d^n_{mu,m}(theta) = eps_mu eps_m d_CS^n_{mu,m}(-theta)."""
    rng = np.random.default_rng(14)
    for n in (158, 318):
        for th in (0.4, 2.2):
            d = sph.rotation_factor(n, th)
            picks = [(n, n), (-n, -n), (n, -n), (0, 0), (1, -1), (n, 0)]
            picks += [tuple(int(v) for v in rng.integers(-n, n + 1, 2)) for _ in range(6)]
            for mu, m in picks:
                eps = (-1.0) ** mu if mu > 0 else 1.0
                eps *= (-1.0) ** m if m > 0 else 1.0
                ref = eps * _wigner_sum(n, mu, m, -th)
                assert abs(d[mu + n, m + n] - ref) < 1e-12, (n, th, mu, m)


def test_rotation_factor_orthogonal_composes_symmetric_to_degree_318():
    """d^n(theta) is orthogonal, d^n(0) = I, rotations about one axis compose
    by adding angles, d^n(-theta) = d^n(theta)^T, and the folded kernels'
    symmetry d^n_{-mu,-m} = d^n_{mu,m} holds, at every sampled degree."""
    for n in _HIGH_DEGREES:
        w = 2 * n + 1
        I = np.eye(w)
        assert np.max(np.abs(sph.rotation_factor(n, 0.0) - I)) < 1e-13
        a, b = 0.7, 1.9
        da, db, dab = sph.rotation_factor(n, a), sph.rotation_factor(n, b), sph.rotation_factor(n, a + b)
        assert np.max(np.abs(da @ da.T - I)) < 1e-12
        assert np.max(np.abs(da @ db - dab)) < 1e-12
        assert np.max(np.abs(sph.rotation_factor(n, -a) - da.T)) < 1e-12
        assert np.max(np.abs(da[::-1, ::-1] - da)) < 1e-12


def test_quarter_turn_identity_to_degree_318():
    """The identity the GPU setup builds every direction's factors from,
    d^n_{mu,m}(theta) = sum_k Delta_{mu,k} Delta_{m,k} cos(k theta + (mu - m) pi/2)
    with Delta = d^n(pi/2), at every sampled degree up to twice the largest
    room's order (the GPU accepts orders to 256)."""
    for n in _HIGH_DEGREES:
        Dl = sph.rotation_factor(n, math.pi / 2)
        k = np.arange(-n, n + 1)
        j = (k[:, None] - k[None, :]) % 4          # (mu - m) mod 4
        for th in _THETAS:
            # cos(x + j pi/2) is cos x, -sin x, -cos x, sin x for j = 0..3
            A = (Dl * np.cos(k * th)[None, :]) @ Dl.T
            B = (Dl * np.sin(k * th)[None, :]) @ Dl.T
            d = np.select([j == 0, j == 1, j == 2], [A, -B, -A], B)
            assert np.max(np.abs(d - sph.rotation_factor(n, th))) < 1e-12, (n, th)
