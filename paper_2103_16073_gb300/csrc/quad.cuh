// FP64 element integrals of the Helmholtz kernels over flat triangles.
//
// Entry rule for collocation point x and element T (Sec. 3.3: entries of
// closely located elements by closed-form integrals, far ones by quadrature):
//   self (x = centroid of T): L = (1/4pi) int_T 1/R (closed form) + smooth
//        remainder (e^{ikR}-1)/(4piR) by the degree-5 rule on the three
//        sub-triangles (x, v_a, v_b);  M = L' = 0 on a flat element.
//   near (|x - c_T| < r_c): closed-form singular parts (int 1/R, the solid
//        angle, int grad 1/R) + the smooth remainders by the degree-5 rule.
//   far: degree-2 three-point rule.
// Closed forms: int_T 1/R dS by the in-plane divergence theorem (Wilton et
// al. 1984, Graglia 1993); signed solid angle by Van Oosterom & Strackee
// (1983); int_T (y-x)/R^3 dS = n Omega - sum_edges m_e int_e dl/R.
#pragma once

#include "common.cuh"

#define FB_PI 3.14159265358979323846
#define FB_INV4PI 0.079577471545947667884

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 v3(double x, double y, double z) { V3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double norm(V3 a) { return sqrt(dot(a, a)); }

struct Tri {
    V3 a, b, c, n;
    double area;
};

__device__ __forceinline__ Tri load_tri(const Geom& g, int64_t j) {
    Tri t;
    t.a = v3(g.ax[j], g.ay[j], g.az[j]);
    t.b = v3(g.bx[j], g.by[j], g.bz[j]);
    t.c = v3(g.qx[j], g.qy[j], g.qz[j]);
    t.n = v3(g.nx[j], g.ny[j], g.nz[j]);
    t.area = g.area[j];
    return t;
}

// Per-edge closed-form pieces: P (in-plane distance, positive inside), E =
// int_edge dl/R, and the atan term of int 1/R.
struct EdgeSums {
    double inv_r;   // int_T 1/R
    V3 medge;       // sum_e m_e E_e
};

__device__ __forceinline__ EdgeSums edge_sums(V3 x, const Tri& t) {
    double d = dot(x - t.a, t.n);
    double ad = fabs(d);
    V3 x0 = x - d * t.n;
    EdgeSums s;
    s.inv_r = 0.0;
    s.medge = v3(0, 0, 0);
    V3 vs[3] = {t.a, t.b, t.c};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        V3 p0 = vs[e], p1 = vs[(e + 1) % 3];
        V3 ed = p1 - p0;
        double le = norm(ed);
        V3 tg = (1.0 / le) * ed;
        V3 m = cross(tg, t.n);
        double lm = dot(p0 - x0, tg);
        double lp = dot(p1 - x0, tg);
        double P = dot(p0 - x0, m);
        double R0sq = P * P + d * d;
        double R0 = sqrt(R0sq);
        double R0s = fmax(R0, 1e-30 * le);
        double Rm = sqrt(R0sq + lm * lm);
        double Rp = sqrt(R0sq + lp * lp);
        double E = asinh(lp / R0s) - asinh(lm / R0s);
        s.inv_r += P * E - ad * (atan2(P * lp, R0sq + ad * Rp) - atan2(P * lm, R0sq + ad * Rm));
        s.medge = s.medge + E * m;
    }
    return s;
}

// Signed solid angle int_T (y-x).n / |y-x|^3 dS (Van Oosterom & Strackee).
__device__ __forceinline__ double solid_angle(V3 x, const Tri& t) {
    V3 r0 = t.a - x, r1 = t.b - x, r2 = t.c - x;
    double l0 = norm(r0), l1 = norm(r1), l2 = norm(r2);
    double num = dot(r0, cross(r1, r2));
    double den = l0 * l1 * l2 + dot(r0, r1) * l2 + dot(r0, r2) * l1 + dot(r1, r2) * l0;
    return 2.0 * atan2(num, den);
}

// e^{i kR} - 1 without cancellation: (cos kR - 1) + i sin kR.
__device__ __forceinline__ cd em1(double kr) {
    double s2, c2;
    sincos(0.5 * kr, &s2, &c2);
    return mk(-2.0 * s2 * s2, 2.0 * s2 * c2);
}

// Kernel values at one point pair (r = y - x):
//   g = G or G - 1/(4piR);  f such that dG/dn_y = (n_y.r) f / (4pi R^3),
//   dG/dn_x = -(n_x.r) f / (4pi R^3);  f = e^{ikR}(ikR - 1) (+1 if smooth).
__device__ __forceinline__ void kernel_pt(double k, V3 r, bool smooth, cd& g, cd& f, double& inv4piR3) {
    double R = norm(r);
    double kr = k * R;
    double s, c;
    sincos(kr, &s, &c);
    cd E = mk(c, s);
    cd ikR = mk(0.0, kr);
    double i4R = FB_INV4PI / R;
    if (smooth) {
        cd e1 = em1(kr);
        g = i4R * e1;
        f = ikR * E - e1;
    } else {
        g = i4R * E;
        f = E * mk(-1.0, kr);
    }
    inv4piR3 = i4R / (R * R);
}

// Degree-5 seven-point rule (Radon): barycentrics and weights.
__device__ __forceinline__ void rule7(int q, double& b0, double& b1, double& b2, double& w) {
    const double s15 = 3.872983346207416885;   // sqrt(15)
    const double a = (6.0 - s15) / 21.0, b = (6.0 + s15) / 21.0;
    const double wa = (155.0 - s15) / 1200.0, wb = (155.0 + s15) / 1200.0;
    switch (q) {
        case 0: b0 = 1.0 / 3.0; b1 = 1.0 / 3.0; b2 = 1.0 / 3.0; w = 9.0 / 40.0; break;
        case 1: b0 = a; b1 = a; b2 = 1 - 2 * a; w = wa; break;
        case 2: b0 = a; b1 = 1 - 2 * a; b2 = a; w = wa; break;
        case 3: b0 = 1 - 2 * a; b1 = a; b2 = a; w = wa; break;
        case 4: b0 = b; b1 = b; b2 = 1 - 2 * b; w = wb; break;
        case 5: b0 = b; b1 = 1 - 2 * b; b2 = b; w = wb; break;
        default: b0 = 1 - 2 * b; b1 = b; b2 = b; w = wb; break;
    }
}

struct Entry {
    cd L, M, LP;
};

// (L, M, L') entries for target point x (normal nx), element j.
// self: x is the centroid of j.
__device__ inline Entry pair_entry(const Geom& g, int64_t j, V3 x, V3 nxv, bool self, double k,
                                   double rc) {
    Entry out;
    Tri t = load_tri(g, j);
    V3 cj = v3(g.cx[j], g.cy[j], g.cz[j]);
    if (self) {
        EdgeSums es = edge_sums(x, t);
        cd L = mk(es.inv_r * FB_INV4PI, 0.0);
        V3 vs[3] = {t.a, t.b, t.c};
        for (int s = 0; s < 3; ++s) {
            V3 pa = vs[s], pb = vs[(s + 1) % 3];
            double asub = 0.5 * norm(cross(pa - x, pb - x));
            for (int q = 0; q < 7; ++q) {
                double b0, b1, b2, w;
                rule7(q, b0, b1, b2, w);
                V3 y = b0 * x + b1 * pa + b2 * pb;
                double R = norm(y - x);
                cd e1 = em1(k * R);
                L = L + (asub * w * FB_INV4PI / R) * e1;
            }
        }
        out.L = L;
        out.M = mk(0.0, 0.0);
        out.LP = mk(0.0, 0.0);
        return out;
    }
    V3 dc = x - cj;
    if (dot(dc, dc) < rc * rc) {
        EdgeSums es = edge_sums(x, t);
        double om = solid_angle(x, t);
        V3 gv = om * t.n - es.medge;            // int (y-x)/R^3
        cd L = mk(es.inv_r * FB_INV4PI, 0.0);
        cd M = mk(-om * FB_INV4PI, 0.0);
        cd LP = mk(dot(nxv, gv) * FB_INV4PI, 0.0);
        for (int q = 0; q < 7; ++q) {
            double b0, b1, b2, w;
            rule7(q, b0, b1, b2, w);
            V3 y = b0 * t.a + b1 * t.b + b2 * t.c;
            V3 r = y - x;
            cd gk, f;
            double i3;
            kernel_pt(k, r, true, gk, f, i3);
            double aw = t.area * w;
            L = L + aw * gk;
            M = M + (aw * dot(t.n, r) * i3) * f;
            LP = LP + (-aw * dot(nxv, r) * i3) * f;
        }
        out.L = L;
        out.M = M;
        out.LP = LP;
        return out;
    }
    cd L = mk(0.0, 0.0), M = mk(0.0, 0.0), LP = mk(0.0, 0.0);
    const double w3 = 1.0 / 3.0;
    for (int q = 0; q < 3; ++q) {
        V3 y = v3(g.gx[3 * j + q], g.gy[3 * j + q], g.gz[3 * j + q]);
        V3 r = y - x;
        cd gk, f;
        double i3;
        kernel_pt(k, r, false, gk, f, i3);
        double aw = t.area * w3;
        L = L + aw * gk;
        M = M + (aw * dot(t.n, r) * i3) * f;
        LP = LP + (-aw * dot(nxv, r) * i3) * f;
    }
    out.L = L;
    out.M = M;
    out.LP = LP;
    return out;
}

// ------------------------------------------------ hypersingular M' ----
// Point kernel d2G/dn_x dn_y (r = y - x):
//   -e^{ikR}/(4 pi R^3) [(3 - 3ikR - k^2R^2)(n_x.r)(n_y.r)/R^2 + (ikR - 1)(n_x.n_y)]
__device__ __forceinline__ cd kernel_nn(double k, V3 r, V3 nx, V3 ny) {
    double R = norm(r);
    double kr = k * R;
    double s, c;
    sincos(kr, &s, &c);
    double a = dot(nx, r) * dot(ny, r) / (R * R);
    double b = dot(nx, ny);
    cd t = mk((3.0 - kr * kr) * a - b, -3.0 * kr * a + kr * b);   // (3 - 3ikR - k^2R^2) a + (ikR - 1) b
    cd e = mk(c, s);
    double f = -FB_INV4PI / (R * R * R);
    return (f * e) * t;
}

// Gauss-Legendre, 8 points on [-1, 1]
__device__ __forceinline__ void gl8(int q, double& x, double& w) {
    const double X[4] = {0.18343464249564978, 0.525532409916329, 0.7966664774136267, 0.9602898564975362};
    const double Wt[4] = {0.36268378337836166, 0.3137066458778869, 0.22238103445337443, 0.10122853629037706};
    int h = q < 4 ? 3 - q : q - 4;
    x = q < 4 ? -X[h] : X[h];
    w = Wt[h];
}

// Edge integrals of the flat-element form of M' for target x (normal nx):
//   A = sum_e int_e grad_y G . m dl,   B = sum_e int_e (n . grad_x G)(t . m) dl,
// t = nx - (nx.n) n, m the outward in-plane edge normal; 8-point
// Gauss-Legendre on min(16, ceil(2 l_e / d_e)) segments (d_e = distance from
// x to the edge).
__device__ inline void mp_edges(double k, V3 x, V3 nxv, const Tri& t, cd& A, cd& B) {
    A = mk(0.0, 0.0);
    B = mk(0.0, 0.0);
    V3 tv = nxv - dot(nxv, t.n) * t.n;
    V3 vs[3] = {t.a, t.b, t.c};
    for (int e = 0; e < 3; ++e) {
        V3 p0 = vs[e], p1 = vs[(e + 1) % 3];
        V3 d = p1 - p0;
        double le = norm(d);
        V3 m = cross((1.0 / le) * d, t.n);
        double sp = fmin(fmax(dot(x - p0, d) / dot(d, d), 0.0), 1.0);
        double de = norm(x - (p0 + sp * d));
        int ns = (int)fmin(16.0, fmax(1.0, ceil(2.0 * le / de)));
        double tm = dot(tv, m);
        for (int sgi = 0; sgi < ns; ++sgi)
            for (int q = 0; q < 8; ++q) {
                double gx, gw;
                gl8(q, gx, gw);
                double u = (sgi + 0.5 * (gx + 1.0)) / ns;
                double w = gw * 0.5 / ns * le;
                V3 r = (p0 + u * d) - x;
                double R = norm(r);
                double kr = k * R;
                double s, c;
                sincos(kr, &s, &c);
                // g'(R) = e^{ikR}(ikR - 1)/(4 pi R^2)
                cd gp = (FB_INV4PI / (R * R)) * (mk(c, s) * mk(-1.0, kr));
                A = A + (w * dot(r, m) / R) * gp;
                B = B + (-w * dot(r, t.n) / R * tm) * gp;
            }
    }
}

// M' entry for target point x (normal nx), element j (self: x = centroid of j):
//   far:  three-point rule of d2G/dn_x dn_y;
//   near / self:  (nx.n)[k^2 S + A] + B, S the single-layer entry of the pair.
__device__ inline cd mp_entry(const Geom& g, int64_t j, V3 x, V3 nxv, bool self, double k, double rc) {
    Tri t = load_tri(g, j);
    V3 cj = v3(g.cx[j], g.cy[j], g.cz[j]);
    V3 dc = x - cj;
    if (self || dot(dc, dc) < rc * rc) {
        Entry e = pair_entry(g, j, x, nxv, self, k, rc);
        cd A, B;
        mp_edges(k, x, nxv, t, A, B);
        return dot(nxv, t.n) * (((k * k) * e.L) + A) + B;
    }
    cd out = mk(0.0, 0.0);
    for (int q = 0; q < 3; ++q) {
        V3 y = v3(g.gx[3 * j + q], g.gy[3 * j + q], g.gz[3 * j + q]);
        out = out + (t.area / 3.0) * kernel_nn(k, y - x, nxv, t.n);
    }
    return out;
}

// Operator entry of kind FB_OP_* for collocation row i (element i) and column j.
__device__ __forceinline__ cd op_entry(const Geom& g, int kind, int64_t i, int64_t j, double k,
                                       double rc) {
    V3 x = v3(g.cx[i], g.cy[i], g.cz[i]);
    V3 nv = v3(g.nx[i], g.ny[i], g.nz[i]);
    if (kind == FB_OP_MP) return mp_entry(g, j, x, nv, i == j, k, rc);
    Entry e = pair_entry(g, j, x, nv, i == j, k, rc);
    switch (kind) {
        case FB_OP_L: return e.L;
        case FB_OP_M: return e.M;
        case FB_OP_LP: return e.LP;
        default: {
            // A = 1/2 I + M - i k beta_j L
            cd b = g.beta[j];
            cd ikb = mk(-k * b.im, k * b.re);   // i k beta
            cd a = e.M - ikb * e.L;
            if (i == j) a.re += 0.5;
            return a;
        }
    }
}
