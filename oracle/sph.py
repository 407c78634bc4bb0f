"""Spherical basis functions and FMM translations (oracle, test infrastructure).

Sec. 3.3.1, Eq. (shft0): multipole and local expansions
    psi = sum_{n<p} sum_{|m|<=n} C_n^m S_n^m(r),   psi = sum D_n^m R_n^m(r),
    S_n^m = h_n(kr) Y_n^m(theta,phi),  R_n^m = j_n(kr) Y_n^m(theta,phi).
Spherical harmonics follow the convention of the book the paper cites for
them: Y_n^m = sqrt((2n+1)/(4pi) (n-|m|)!/(n+|m|)!) P_n^{|m|}(cos theta) e^{im phi}
with P_n^{|m|} WITHOUT the Condon-Shortley phase, so Y_n^{-m} = conj(Y_n^m).
With it the Green's function expands as
    G(x,y) = ik sum_{n,m} S_n^m(x-c) R_n^{-m}(y-c),   |x-c| > |y-c|.
Coefficient vectors are stored with the flat index n^2 + n + m.

Coaxial coefficients (Eq. shft0.1):
    S_n^m(r + tau i_z) = sum_{n'} (S|R)^m_{n'n}(tau) R_{n'}^m(r),
    R_n^m(r + tau i_z) = sum_{n'} (R|R)^m_{n'n}(tau) R_{n'}^m(r),  (S|S) = (R|R).
``coaxial`` implements the paper's algorithm: seeds Eq. (shft1), sectorial
recursion Eq. (shft2), then either the original n-propagation Eqs.
(shft3)-(shft5) with the symmetry of step 4 (k tau < 1) or the stabilised
scheme: zonal Eq. (shft7), diagonal/subdiagonal Eq. (shft8), n'-propagation
Eq. (shift6) (k tau >= 1).  The third formula of Eq. (shft8) is used with its
last coefficient read as b_n^{-m-1} (as printed, b_{n+1}^{-m-1}, the relation
does not hold for exact coefficients).

Rotation blocks are not given in the paper (Sec. 3.3 cites a separate
chapter); the oracle uses their definition: for a rotation Q (x_new = Q x),
D^n_{m'm} = int conj(Y_n^{m'}(y)) Y_n^m(Q^T y) dOmega(y), evaluated with a
product Gauss-Legendre x trapezoid rule that is exact for the band limit.
At the degrees of the largest orders, where that grid is too large,
``rotation_factor`` gives the real factor of one degree from the generator
of rotations about y; the two agree at low degree, and the generator form is
pinned at high degree by the closed-form m = 0 column, Wigner's explicit sum
in high precision and the quarter-turn identity the GPU setup uses.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def idx(n, m):
    """Flat index n^2 + n + m of coefficient (n, m), |m| <= n."""
    return n * n + n + m


def a_coef(n, m):
    """a_n^m = sqrt((n+1+|m|)(n+1-|m|)/((2n+1)(2n+3))), 0 if n < |m|."""
    am = abs(m)
    if n < am or n < 0:
        return 0.0
    return math.sqrt((n + 1 + am) * (n + 1 - am) / ((2 * n + 1) * (2 * n + 3)))


def b_coef(n, m):
    """b_n^m = +-sqrt((n-m-1)(n-m)/((2n-1)(2n+1))), + for 0<=m<=n, - for
    -n<=m<0, 0 for |m| > n."""
    if n < 0 or abs(m) > n:
        return 0.0
    v = math.sqrt((n - m - 1) * (n - m) / ((2 * n - 1) * (2 * n + 1)))
    return v if m >= 0 else -v


def sph_j(nmax, x):
    """Spherical Bessel functions j_n(x), n = 0..nmax (the radial part of
    R_n^m, Eq. shft0); shape [nmax+1, ...]."""
    n = np.arange(nmax + 1)
    x = np.asarray(x)
    return special.spherical_jn(n[:, None], x.ravel()[None, :]).reshape((nmax + 1,) + x.shape)


def sph_jp(nmax, x):
    """Derivatives j_n'(x), n = 0..nmax; shape [nmax+1, ...]."""
    n = np.arange(nmax + 1)
    x = np.asarray(x)
    return special.spherical_jn(n[:, None], x.ravel()[None, :], derivative=True).reshape(
        (nmax + 1,) + x.shape)


def sph_h(nmax, x):
    """Spherical Hankel functions h_n(x) = j_n(x) + i y_n(x), n = 0..nmax (the
    radial part of S_n^m, Eq. shft0); shape [nmax+1, ...]."""
    n = np.arange(nmax + 1)
    x = np.asarray(x)
    j = special.spherical_jn(n[:, None], x.ravel()[None, :])
    y = special.spherical_yn(n[:, None], x.ravel()[None, :])
    return (j + 1j * y).reshape((nmax + 1,) + x.shape)


def _norm(n, am):
    return math.sqrt((2 * n + 1) / (4 * math.pi)
                     * math.exp(math.lgamma(n - am + 1) - math.lgamma(n + am + 1)))


def ylm(p, theta, phi):
    """Y_n^m(theta,phi) for n < p, flat index; shape [p^2, ...].

    Fully normalised associated Legendre functions without the
    Condon-Shortley phase by the standard three-term recursion in n
    (x = cos theta, s = sin theta):
        Q_0^0 = 1/sqrt(4pi),  Q_m^m = sqrt((2m+1)/(2m)) s Q_{m-1}^{m-1},
        Q_{m+1}^m = sqrt(2m+3) x Q_m^m,
        Q_n^m = sqrt((4n^2-1)/(n^2-m^2)) x Q_{n-1}^m
                - sqrt(((n-1)^2-m^2)(2n+1)/((2n-3)(n^2-m^2))) Q_{n-2}^m,
    then Y_n^m = Q_n^{|m|} e^{i m phi}."""
    theta = np.asarray(theta, float)
    phi = np.asarray(phi, float)
    x = np.cos(theta)
    s = np.sin(theta)
    Q = np.zeros((p, p) + theta.shape)
    Q[0, 0] = 1.0 / math.sqrt(4.0 * math.pi)
    for m in range(1, p):
        Q[m, m] = math.sqrt((2 * m + 1) / (2.0 * m)) * s * Q[m - 1, m - 1]
    for m in range(p - 1):
        Q[m + 1, m] = math.sqrt(2 * m + 3) * x * Q[m, m]
    for m in range(p):
        for n in range(m + 2, p):
            a = math.sqrt((4.0 * n * n - 1) / (n * n - m * m))
            b = math.sqrt(((n - 1) ** 2 - m * m) * (2.0 * n + 1) / ((2.0 * n - 3) * (n * n - m * m)))
            Q[n, m] = a * x * Q[n - 1, m] - b * Q[n - 2, m]
    out = np.zeros((p * p,) + theta.shape, np.complex128)
    for n in range(p):
        for m in range(-n, n + 1):
            out[idx(n, m)] = Q[n, abs(m)] * np.exp(1j * m * phi)
    return out


def _dylm_dtheta(p, theta, phi):
    theta = np.asarray(theta, float)
    phi = np.asarray(phi, float)
    x = np.cos(theta)
    s = np.sin(theta)
    out = np.zeros((p * p,) + theta.shape, np.complex128)
    for n in range(p):
        for m in range(-n, n + 1):
            am = abs(m)
            Pn = special.lpmv(am, n, x)
            Pn1 = special.lpmv(am, n - 1, x) if n - 1 >= am else 0.0
            dP = (n * x * Pn - (n + am) * Pn1) / s
            out[idx(n, m)] = _norm(n, am) * (-1.0) ** am * dP * np.exp(1j * m * phi)
    return out


def _spherical(r):
    r = np.asarray(r, float)
    rho = np.linalg.norm(r, axis=-1)
    theta = np.arccos(np.clip(r[..., 2] / np.where(rho > 0, rho, 1.0), -1.0, 1.0))
    phi = np.arctan2(r[..., 1], r[..., 0])
    return rho, theta, phi


def regular(p, k, r):
    """R_n^m(r) = j_n(k|r|) Y_n^m(r/|r|), shape [p^2, ...]."""
    rho, th, ph = _spherical(r)
    j = sph_j(p - 1, k * rho)
    Y = ylm(p, th, ph)
    n_of = np.repeat(np.arange(p), 2 * np.arange(p) + 1)
    return j[n_of] * Y


def singular(p, k, r):
    """S_n^m(r) = h_n(k|r|) Y_n^m(r/|r|), shape [p^2, ...]."""
    rho, th, ph = _spherical(r)
    h = sph_h(p - 1, k * rho)
    Y = ylm(p, th, ph)
    n_of = np.repeat(np.arange(p), 2 * np.arange(p) + 1)
    return h[n_of] * Y


def grad_regular(p, k, r):
    """grad R_n^m(r) by the chain rule in spherical coordinates, [p^2, ..., 3]."""
    rho, th, ph = _spherical(r)
    j = sph_j(p - 1, k * rho)
    jp = sph_jp(p - 1, k * rho)
    Y = ylm(p, th, ph)
    dY = _dylm_dtheta(p, th, ph)
    n_of = np.repeat(np.arange(p), 2 * np.arange(p) + 1)
    m_of = np.concatenate([np.arange(-n, n + 1) for n in range(p)])
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    rhat = np.stack([st * cp, st * sp, ct], axis=-1)
    that = np.stack([ct * cp, ct * sp, -st], axis=-1)
    phat = np.stack([-sp, cp, np.zeros_like(sp)], axis=-1)
    mshape = (slice(None),) + (None,) * rho.ndim
    dr = k * jp[n_of] * Y
    dt = j[n_of] * dY / rho
    dp = j[n_of] * (1j * m_of[mshape]) * Y / (rho * st)
    return dr[..., None] * rhat + dt[..., None] * that + dp[..., None] * phat


# ---------------------------------------------------------------------------
# Coaxial translation coefficients, Sec. 3.3.1
# ---------------------------------------------------------------------------

def _seeds(nmax, ktau, kind, mp):
    """f_n(k tau), n = 0..nmax: h_n for S|R, j_n for R|R."""
    if mp is None:
        if kind == "SR":
            return sph_h(nmax, ktau)
        return sph_j(nmax, ktau).astype(np.complex128)
    x = mp.mpf(ktau)
    out = []
    for n in range(nmax + 1):
        j = mp.sqrt(mp.pi / (2 * x)) * mp.besselj(n + mp.mpf(1) / 2, x)
        if kind == "SR":
            y = mp.sqrt(mp.pi / (2 * x)) * mp.bessely(n + mp.mpf(1) / 2, x)
            out.append(mp.mpc(j, y))
        else:
            out.append(mp.mpc(j, 0))
    return out


def coaxial(p, ktau, kind="SR", scheme="auto", mp=None, misprint=False):
    """(E|F)^m_{n'n}(tau) for m = 0..p-1, n', n = m..p-1.

    kind: "SR" (seeds h_n) or "RR" (seeds j_n).  scheme: "original",
    "stabilized" or "auto" (original if k tau < 1, Sec. 3.3.1 last paragraph).
    mp: optional mpmath module; the same steps then run in its arithmetic
    (used to reproduce the paper's stability comparison).  misprint: use the
    third formula of Eq. (shft8) exactly as printed (for tests only).
    Returns X with X[m, n', n] (zero outside |m| <= n', n < p).
    """
    if scheme == "auto":
        scheme = "original" if ktau < 1.0 else "stabilized"
    P2 = 2 * p
    sqrt = math.sqrt if mp is None else mp.sqrt
    if mp is None:
        X = np.zeros((p + 1, P2 + 2, p + 2), np.complex128)
    else:
        X = np.empty((p + 1, P2 + 2, p + 2), dtype=object)
        X.fill(mp.mpc(0))

    def a(n, m):
        am = abs(m)
        if n < am or n < 0:
            return 0.0
        return sqrt((n + 1 + am) * (n + 1 - am) / ((2 * n + 1) * (2 * n + 3)))

    def b(n, m):
        if n < 0 or abs(m) > n:
            return 0.0
        v = sqrt((n - m - 1) * (n - m) / ((2 * n - 1) * (2 * n + 1)))
        return v if m >= 0 else -v

    f = _seeds(P2 - 1, ktau, kind, mp)
    # Step 1, Eq. (shft1): zero-order seeds, n' = 0..2p-1
    for n1 in range(P2):
        X[0, n1, 0] = (-1) ** n1 * sqrt(2 * n1 + 1) * f[n1]
    # Step 2, Eq. (shft2): sectorial coefficients (E|F)^m_{n',m}
    for m in range(p - 1):
        for n1 in range(m + 1, P2 - 1 - m):
            X[m + 1, n1, m + 1] = (b(n1, -m - 1) * X[m, n1 - 1, m]
                                   - b(n1 + 1, m) * X[m, n1 + 1, m]) / b(m + 1, -m - 1)
    if scheme == "original":
        # Step 3, Eqs. (shft3)-(shft5): propagation in n for n' >= n
        for m in range(p):
            for n in range(m, p - 1):
                for n1 in range(n, 2 * p - 1 - n):
                    X[m, n1, n + 1] = (a(n - 1, m) * X[m, n1, n - 1]
                                       - a(n1, m) * X[m, n1 + 1, n]
                                       + a(n1 - 1, m) * X[m, n1 - 1, n]) / a(n, m)
    else:
        # Step 3.1, Eq. (shft7): zonal coefficients by propagation in n
        for n in range(p - 1):
            for n1 in range(n + 1, 2 * p - n - 2):
                X[0, n1, n + 1] = (a(n - 1, 0) * X[0, n1, n - 1]
                                   - a(n1, 0) * X[0, n1 + 1, n]
                                   + a(n1 - 1, 0) * X[0, n1 - 1, n]) / a(n, 0)
        # Step 3.2, Eq. (shft8): diagonal and the two subdiagonals, up in m
        for m in range(p - 2):
            for n in range(m + 1, p - 1):
                if n >= m + 2:
                    X[m + 1, n + 1, n] = (b(n + 1, m) * X[m, n + 1, n]
                                          + b(n, -m - 1) * X[m, n, n - 1]
                                          - b(n, m) * X[m + 1, n, n - 1]) / b(n + 1, -m - 1)
                X[m + 1, n + 1, n + 1] = (b(n, m) * X[m + 1, n + 1, n - 1]
                                          - b(n + 2, m) * X[m, n + 2, n]
                                          + b(n + 1, -m - 1) * X[m, n, n]) / b(n + 1, -m - 1)
                if n >= m + 2:
                    last = b(n + 1, -m - 1) if misprint else b(n, -m - 1)
                    X[m + 1, n + 2, n] = (b(n + 1, m) * X[m + 1, n, n]
                                          - b(n + 1, m) * X[m, n + 1, n + 1]
                                          + last * X[m, n + 1, n - 1]) / b(n + 2, -m - 1)
        # Step 3 (modified), Eq. (shift6): propagation in n'
        for m in range(1, p):
            for n1 in range(m + 3, p - 1):
                for n in range(m + 1, n1 - 1):
                    X[m, n1 + 1, n] = (a(n - 1, m) * X[m, n1, n - 1]
                                       - a(n, m) * X[m, n1, n + 1]
                                       + a(n1 - 1, m) * X[m, n1 - 1, n]) / a(n1, m)
    # Step 4: symmetry for n' < n
    out = np.zeros((p, p, p), np.complex128 if mp is None else object)
    for m in range(p):
        for n1 in range(m, p):
            for n in range(m, p):
                if n1 >= n:
                    out[m, n1, n] = X[m, n1, n]
                else:
                    out[m, n1, n] = (-1) ** (n + n1) * X[m, n, n1]
    return out


# ---------------------------------------------------------------------------
# Rotations
# ---------------------------------------------------------------------------

def rotation_to_z(t):
    """Q = R_y(-theta) R_z(-phi): the rotation that maps the unit vector of
    t (polar angle theta, azimuth phi) to +z."""
    t = np.asarray(t, float)
    rho = np.linalg.norm(t)
    th = math.acos(max(-1.0, min(1.0, t[2] / rho)))
    ph = math.atan2(t[1], t[0])
    cz, sz = math.cos(-ph), math.sin(-ph)
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1.0]])
    cy, sy = math.cos(-th), math.sin(-th)
    Ry = np.array([[cy, 0, sy], [0, 1.0, 0], [-sy, 0, cy]])
    return Ry @ Rz


def rotation_blocks(Q, p):
    """D^n (n < p) for rotation Q by projection quadrature; list of
    (2n+1)x(2n+1) arrays with D[n][m'+n, m+n]."""
    nq = p + 1
    xg, wg = np.polynomial.legendre.leggauss(nq)
    nphi = 2 * p + 1
    phis = 2 * np.pi * np.arange(nphi) / nphi
    TH, PH = np.meshgrid(np.arccos(xg), phis, indexing="ij")
    W = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    yv = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    yr = yv @ np.asarray(Q)          # rows: Q^T y
    _, th2, ph2 = _spherical(yr)
    Y = ylm(p, np.arccos(yv[:, 2].clip(-1, 1)), np.arctan2(yv[:, 1], yv[:, 0]))
    Y2 = ylm(p, th2, ph2)
    out = []
    for n in range(p):
        s = slice(n * n, (n + 1) * (n + 1))
        out.append((np.conj(Y[s]) * W[None, :]) @ Y2[s].T)
    return out


def _eps(m):
    """(-1)^m for m > 0, else 1: Y_n^m of the Condon-Shortley convention
    over Y_n^m of this one."""
    m = np.asarray(m)
    return np.where(m > 0, (-1.0) ** m, 1.0)


def rotation_factor(n, theta):
    """Real factor d^n(theta), [mu + n, m + n], of the rotation blocks at one
    degree n: for the rotation Q = rotation_to_z(t) of a direction with polar
    angle theta and azimuth phi, rotation_blocks gives
    D^n_{mu,m} = d^n_{mu,m}(theta) e^{i m phi}.

    Computed from the generator of rotations about y, not by projection (the
    projection grid of rotation_blocks grows as p^2 points x p^2 harmonics and
    stops near degree 40 here, far below the orders of Sec. 3.3's largest
    boxes).  In the Condon-Shortley basis |n, m>, a rotation by beta about y
    acts as exp(-i beta J_y), J_y = (J_+ - J_-) / (2i) with the ladder
    elements <m+1|J_+|m> = <m|J_-|m+1> = sqrt(n(n+1) - m(m+1)).  Q turns by
    -theta about y after a turn about z, and the harmonics here drop the
    (-1)^m of positive orders, so
        d^n_{mu,m}(theta) = eps_mu eps_m [exp(i theta J_y)]_{mu,m}.
    J_y is Hermitian with eigenvalues exactly -n..n; the exponential is
    formed from its eigenvectors with the eigenvalues rounded to those
    integers."""
    w = 2 * n + 1
    m = np.arange(-n, n + 1)
    lad = np.sqrt(n * (n + 1.0) - m[:-1] * (m[:-1] + 1.0))    # <m+1|J_+|m>
    Jy = np.zeros((w, w), np.complex128)
    Jy[np.arange(1, w), np.arange(w - 1)] = lad / 2j           # J_+ / (2i)
    Jy[np.arange(w - 1), np.arange(1, w)] = -lad / 2j          # -J_- / (2i)
    lam, V = np.linalg.eigh(Jy)
    E = (V * np.exp(1j * theta * np.round(lam))[None, :]) @ V.conj().T
    e = _eps(m)
    return e[:, None] * E.real * e[None, :]


def block_diag_rot(D, p):
    """The rotation blocks D^n, n < p, as one block-diagonal [p^2, p^2]
    matrix acting on flat coefficient vectors."""
    Mx = np.zeros((p * p, p * p), np.complex128)
    for n in range(p):
        s = slice(n * n, (n + 1) * (n + 1))
        Mx[s, s] = D[n]
    return Mx


def coax_matrix(X, p_out, p_in):
    """Coaxial coefficients as a [p_out^2, p_in^2] matrix (diagonal in m)."""
    T = np.zeros((p_out * p_out, p_in * p_in), np.complex128)
    for n1 in range(p_out):
        for n in range(p_in):
            for m in range(-min(n1, n), min(n1, n) + 1):
                T[idx(n1, m), idx(n, m)] = X[abs(m), n1, n]
    return T


def translation(t, k, p_out, p_in, kind, rot=None, coax=None):
    """Full translation matrix by rotation - coaxial - back-rotation (Sec. 3.3).

    kind "SR" (multipole-to-local, t = c_target - c_source) or "RR"
    (multipole-to-multipole with t = c_parent - c_child, and
    local-to-local with t = c_child - c_parent).
    rot: optional precomputed rotation blocks for t's direction (>= max p);
    coax: optional precomputed ``coaxial`` array (size >= max p).
    Returns T [p_out^2, p_in^2] with out = T @ in.
    """
    t = np.asarray(t, float)
    tau = float(np.linalg.norm(t))
    p = max(p_out, p_in)
    X = coaxial(p, k * tau, kind) if coax is None else coax
    D = rotation_blocks(rotation_to_z(t), p) if rot is None else rot
    Din = block_diag_rot(D[:p_in], p_in)
    Dout = block_diag_rot(D[:p_out], p_out)
    C = coax_matrix(X, p_out, p_in)
    return Dout.conj().T @ C @ Din
