// FP64 spherical basis functions on the device (Sec. 3.3.1, Eq. shft0):
//   R_n^m(r) = j_n(k|r|) Y_n^m(theta, phi),  S_n^m = h_n Y_n^m,
//   Y_n^m = sqrt((2n+1)/(4pi) (n-|m|)!/(n+|m|)!) P_n^{|m|}(cos theta) e^{i m phi}
// with P_n^{|m|} free of the Condon-Shortley phase (so Y_n^{-m} = conj Y_n^m).
// Coefficient vectors use the flat index n^2 + n + m.
#pragma once

#include "quad.cuh"

__device__ __forceinline__ int nm_idx(int n, int m) { return n * n + n + m; }

// a_n^m and b_n^m of the translation recursions (zero outside their range).
__device__ __forceinline__ double coef_a(int n, int m) {
    int am = abs(m);
    if (n < am || n < 0) return 0.0;
    return sqrt((double)((n + 1 + am) * (n + 1 - am)) / (double)((2 * n + 1) * (2 * n + 3)));
}
__device__ __forceinline__ double coef_b(int n, int m) {
    if (n < 0 || abs(m) > n) return 0.0;
    double v = sqrt((double)((n - m - 1) * (n - m)) / (double)((2 * n - 1) * (2 * n + 1)));
    return m >= 0 ? v : -v;
}

// Normalised associated Legendre functions (no Condon-Shortley phase) for
// n < P at x = cos theta, s = sin theta: out[n(n+1)/2 + m], 0 <= m <= n.
//   Q_0^0 = 1/sqrt(4pi);  Q_m^m = sqrt((2m+1)/(2m)) s Q_{m-1}^{m-1};
//   Q_{m+1}^m = sqrt(2m+3) x Q_m^m;
//   Q_n^m = A x Q_{n-1}^m - B Q_{n-2}^m,
//     A = sqrt((4n^2-1)/(n^2-m^2)),  B = sqrt(((n-1)^2-m^2)(2n+1)/((2n-3)(n^2-m^2))).
__device__ inline void legendre_q(int P, double x, double s, double* out) {
    out[0] = 0.28209479177387814347;   // 1/sqrt(4 pi)
    double diag = out[0];
    for (int m = 0; m < P; ++m) {
        if (m > 0) {
            diag *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
            out[m * (m + 1) / 2 + m] = diag;
        }
        if (m + 1 < P) out[(m + 1) * (m + 2) / 2 + m] = sqrt(2.0 * m + 3.0) * x * diag;
        for (int n = m + 2; n < P; ++n) {
            double nn = (double)n * n, mm = (double)m * m;
            double A = sqrt((4.0 * nn - 1.0) / (nn - mm));
            double B = sqrt(((n - 1.0) * (n - 1.0) - mm) * (2.0 * n + 1.0) / ((2.0 * n - 3.0) * (nn - mm)));
            out[n * (n + 1) / 2 + m] = A * x * out[(n - 1) * n / 2 + m] - B * out[(n - 2) * (n - 1) / 2 + m];
        }
    }
}

// Spherical Bessel j_n(x), n = 0..nmax, by downward recurrence (Miller)
// normalised with j_0 or j_1, whichever is larger in magnitude.
__device__ inline void sph_bessel_j(int nmax, double x, double* j) {
    if (x == 0.0) {
        j[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) j[n] = 0.0;
        return;
    }
    int start = nmax + 24 + (int)x;
    double fp = 0.0, f = 1e-280;
    for (int n = 0; n <= nmax; ++n) j[n] = 0.0;
    for (int n = start; n >= 1; --n) {
        double fm = (2.0 * n + 1.0) / x * f - fp;
        fp = f;
        f = fm;             // f = f_{n-1}, fp = f_n
        if (n - 1 <= nmax) j[n - 1] = f;
        if (n <= nmax) j[n] = fp;
        if (fabs(f) > 1e200) {
            f *= 1e-200;
            fp *= 1e-200;
            for (int q = n - 1; q <= nmax; ++q) j[q] *= 1e-200;
        }
    }
    double sn, cs;
    sincos(x, &sn, &cs);
    double j0 = sn / x;
    double j1 = sn / (x * x) - cs / x;
    double scale = (fabs(j0) >= fabs(j1) || nmax < 1) ? j0 / j[0] : j1 / j[1];
    for (int n = 0; n <= nmax; ++n) j[n] *= scale;
}

// Spherical Bessel y_n(x), n = 0..nmax, by upward recurrence (stable for y).
__device__ inline void sph_bessel_y(int nmax, double x, double* y) {
    double sn, cs;
    sincos(x, &sn, &cs);
    y[0] = -cs / x;
    if (nmax >= 1) y[1] = -cs / (x * x) - sn / x;
    for (int n = 1; n < nmax; ++n) y[n + 1] = (2.0 * n + 1.0) / x * y[n] - y[n - 1];
}

// Y_n^m(u) for n < P at unit vector u: out[nm_idx(n,m)].  q: scratch of
// P(P+1)/2 doubles.
__device__ inline void ylm_unit(int P, double ux, double uy, double uz, double* q, cd* out) {
    double s = sqrt(ux * ux + uy * uy);
    cd e1 = s > 0.0 ? mk(ux / s, uy / s) : mk(1.0, 0.0);
    legendre_q(P, uz, s, q);
    cd em = mk(1.0, 0.0);
    for (int m = 0; m < P; ++m) {
        for (int n = m; n < P; ++n) {
            double v = q[n * (n + 1) / 2 + m];
            out[nm_idx(n, m)] = v * em;
            if (m > 0) out[nm_idx(n, -m)] = v * conjg(em);
        }
        em = em * e1;
    }
}

// R_n^m(r) for n < P: out[nm_idx(n,m)].  scratch: P(P+1)/2 + P + 24 doubles.
__device__ inline void regular_all(int P, double k, V3 r, double* scratch, cd* out) {
    double rho = norm(r);
    double* q = scratch;
    double* jn = scratch + P * (P + 1) / 2;
    if (rho == 0.0) {
        for (int i = 0; i < P * P; ++i) out[i] = mk(0.0, 0.0);
        out[0] = mk(0.28209479177387814347, 0.0);
        return;
    }
    ylm_unit(P, r.x / rho, r.y / rho, r.z / rho, q, out);
    sph_bessel_j(P - 1, k * rho, jn);
    for (int n = 0; n < P; ++n)
        for (int m = -n; m <= n; ++m) out[nm_idx(n, m)] = jn[n] * out[nm_idx(n, m)];
}

// n . grad R_n^mu for n < P from R up to degree P (array Rv of (P+1)^2):
//   dz R_n^u      = k [a_{n-1}^u R_{n-1}^u - a_n^u R_{n+1}^u]
//   (dx+idy) R_n^u = k [-b_n^u R_{n-1}^{u+1} + b_{n+1}^{-u-1} R_{n+1}^{u+1}]
//   (dx-idy) R_n^u = k [-b_n^{-u} R_{n-1}^{u-1} + b_{n+1}^{u-1} R_{n+1}^{u-1}]
//   n.grad = (nx - i ny)/2 (dx+idy) + (nx + i ny)/2 (dx-idy) + nz dz
__device__ __forceinline__ cd rget(const cd* Rv, int Pp1, int n, int m) {
    if (n < 0 || n >= Pp1 || abs(m) > n) return mk(0.0, 0.0);
    return Rv[nm_idx(n, m)];
}
__device__ inline cd ndot_grad_regular(const cd* Rv, int P, double k, V3 nv, int n, int u) {
    int Pp1 = P + 1;
    cd dz = k * (coef_a(n - 1, u) * rget(Rv, Pp1, n - 1, u) - coef_a(n, u) * rget(Rv, Pp1, n + 1, u));
    cd dp = k * ((-coef_b(n, u)) * rget(Rv, Pp1, n - 1, u + 1) + coef_b(n + 1, -u - 1) * rget(Rv, Pp1, n + 1, u + 1));
    cd dm = k * ((-coef_b(n, -u)) * rget(Rv, Pp1, n - 1, u - 1) + coef_b(n + 1, u - 1) * rget(Rv, Pp1, n + 1, u - 1));
    cd hp = mk(0.5 * nv.x, -0.5 * nv.y), hm = mk(0.5 * nv.x, 0.5 * nv.y);
    return hp * dp + hm * dm + nv.z * dz;
}
