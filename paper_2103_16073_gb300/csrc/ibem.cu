// Indirect boundary-element system (Sec. 2.3, Eqs. ibem1-ibem5) with two
// unknowns per element, psi+ and psi- (the scattered field on the side the
// normal points to and on the other side).  With a = k/(i zeta) = -i k beta
// per side,
//   s  = a- psi- + a+ psi+,   mu = psi+ - psi-
//   y+ = (psi- + psi+)/2 - M[mu] + L[s]
//   y- = -M'[mu] + (a+ psi+ - a- psi-)/2 + L'[s]
// i.e. the two rows of Eq. (ibem5); unknown and result vectors are
// [psi+ (N), psi- (N)] and [row 1 (N), row 2 (N)] in element order.  The
// operator is composed of the four FMM (or dense) operators L, M, L', M' on
// the same mesh and tree, so one product costs four operator applications
// plus two element-wise passes.
#include "common.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ cd side_a(double k, cd beta) { return mk(k * beta.im, -k * beta.re); }   // -i k beta

__global__ void k_ibem_pre(const cd* __restrict__ x, const cd* __restrict__ bp, const cd* __restrict__ bm,
                           double k, int64_t n, cd* __restrict__ s, cd* __restrict__ mu) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd pp = x[i], pm = x[n + i];
    s[i] = side_a(k, bm[i]) * pm + side_a(k, bp[i]) * pp;
    mu[i] = pp - pm;
}

// t = [M mu, L s, M' mu, L' s]
__global__ void k_ibem_post(const cd* __restrict__ x, const cd* __restrict__ bp, const cd* __restrict__ bm,
                            double k, int64_t n, const cd* __restrict__ t, cd* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd pp = x[i], pm = x[n + i];
    cd ap = side_a(k, bp[i]), am = side_a(k, bm[i]);
    y[i] = mk(0.5, 0.0) * (pm + pp) - t[i] + t[n + i];
    y[n + i] = mk(0.5, 0.0) * (ap * pp - am * pm) - t[2 * n + i] + t[3 * n + i];
}

// gamma+ = d psi_in/dn - a+ psi_in, gamma- = -d psi_in/dn - a- psi_in for a
// monopole psi_in = e^{ikR}/(4 pi R) at the centroids (Eq. ibem4)
__global__ void k_ibem_gammas(Geom g, const cd* __restrict__ bp, const cd* __restrict__ bm, double k, double sx,
                              double sy, double sz, cd* __restrict__ gp, cd* __restrict__ gm) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    double rx = g.cx[i] - sx, ry = g.cy[i] - sy, rz = g.cz[i] - sz;
    double R = sqrt(rx * rx + ry * ry + rz * rz);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    cd G = mk(cs / (4.0 * kPi * R), sn / (4.0 * kPi * R));
    // dG/dR = G (ik R - 1) / R;  d/dn = dG/dR (r . n) / R
    double rn = (rx * g.nx[i] + ry * g.ny[i] + rz * g.nz[i]) / R;
    cd dG = G * mk(-rn / R, k * rn);
    gp[i] = dG - side_a(k, bp[i]) * G;
    gm[i] = mk(-dG.re, -dG.im) - side_a(k, bm[i]) * G;
}

// right-hand side pieces: w = gamma- + gamma+, d = (gamma+ - gamma-)/2
__global__ void k_ibem_rhs_pre(const cd* __restrict__ gp, const cd* __restrict__ gm, int64_t n, cd* __restrict__ w) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    w[i] = gm[i] + gp[i];
}
__global__ void k_ibem_rhs_post(const cd* __restrict__ gp, const cd* __restrict__ gm, const cd* __restrict__ Lw,
                                const cd* __restrict__ LPw, int64_t n, cd* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = Lw[i];
    b[n + i] = mk(0.5, 0.0) * (gp[i] - gm[i]) + LPw[i];
}

// densities for the field off the surface, written for the direct-formula
// evaluator psi(r) = L[q + i k beta- p](r) - M[p](r):  p = -mu and
// q = sigma + i k beta- mu, so that it returns L[sigma] + M[mu] (Eq. ibem1);
// sigma = gamma- + gamma+ - a- psi- - a+ psi+
__global__ void k_ibem_field_dens(const cd* __restrict__ x, const cd* __restrict__ gp, const cd* __restrict__ gm,
                                  const cd* __restrict__ bp, const cd* __restrict__ bm, double k, int64_t n,
                                  cd* __restrict__ p, cd* __restrict__ q) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd pp = x[i], pm = x[n + i];
    cd mu = pp - pm;
    cd sigma = gm[i] + gp[i] - side_a(k, bm[i]) * pm - side_a(k, bp[i]) * pp;
    p[i] = mk(-mu.re, -mu.im);
    q[i] = sigma - side_a(k, bm[i]) * mu;   // i k beta- mu = -a- mu
}

}  // namespace


// Builds the four constituent operators and the work buffers.
fb_status fb_ibem_create(fb_op* op, cudaStream_t s) {
    const int kinds[4] = {FB_OP_M, FB_OP_L, FB_OP_MP, FB_OP_LP};
    for (int q = 0; q < 4; ++q)
        FB_CHECK(fb_operator_create_impl(op->mesh, op->tree, op->k, kinds[q], op->prec, op->d0, op->pmin, s,
                                         &op->sub[q]));
    const int64_t n = op->mesh->n;
    FB_CHECK(dalloc(&op->ib_work, (size_t)6 * n));
    FB_CHECK(dalloc(&op->ib_beta_p, (size_t)n));
    const cd* src = op->mesh->beta_p ? op->mesh->beta_p : op->mesh->beta;
    FB_CUDA(cudaMemcpyAsync(op->ib_beta_p, src, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s));
    FB_CHECK(dalloc(&op->ib_beta_m, (size_t)n));
    FB_CUDA(cudaMemcpyAsync(op->ib_beta_m, op->mesh->beta, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s));
    op->n = 2 * n;
    return FB_OK;
}

void fb_ibem_free(fb_op* op) {
    for (int q = 0; q < 4; ++q) {
        fb_operator_destroy(op->sub[q]);
        op->sub[q] = nullptr;
    }
    dfree(op->ib_work);
    dfree(op->ib_beta_p);
    dfree(op->ib_beta_m);
}

fb_status fb_ibem_apply(fb_op* op, const cd* x, cd* y, cudaStream_t s, int nrhs) {
    const int64_t n = op->n / 2;
    cd* sv = op->ib_work;
    cd* mu = op->ib_work + n;
    cd* t = op->ib_work + 2 * n;   // 4 n
    const int g = (int)div_up(n, 256);
    for (int r = 0; r < nrhs; ++r) {
        const cd* xr = x + (int64_t)r * op->n;
        cd* yr = y + (int64_t)r * op->n;
        k_ibem_pre<<<g, 256, 0, s>>>(xr, op->ib_beta_p, op->ib_beta_m, op->k, n, sv, mu);
        FB_LAUNCH_CHECK();
        fb_count_launch();
        FB_CHECK(fb_apply_any(op->sub[0], mu, t, s));
        FB_CHECK(fb_apply_any(op->sub[1], sv, t + n, s));
        FB_CHECK(fb_apply_any(op->sub[2], mu, t + 2 * n, s));
        FB_CHECK(fb_apply_any(op->sub[3], sv, t + 3 * n, s));
        k_ibem_post<<<g, 256, 0, s>>>(xr, op->ib_beta_p, op->ib_beta_m, op->k, n, t, yr);
        FB_LAUNCH_CHECK();
        fb_count_launch();
    }
    return FB_OK;
}

fb_status fb_ibem_gammas_impl(fb_op* op, const double* src, cd* gp, cd* gm, cudaStream_t s) {
    const int64_t n = op->n / 2;
    k_ibem_gammas<<<div_up(n, 256), 256, 0, s>>>(op->mesh->g, op->ib_beta_p, op->ib_beta_m, op->k, src[0], src[1],
                                                  src[2], gp, gm);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

fb_status fb_ibem_rhs_impl(fb_op* op, const cd* gp, const cd* gm, cd* b, cudaStream_t s) {
    const int64_t n = op->n / 2;
    cd* w = op->ib_work;
    cd* Lw = op->ib_work + n;
    cd* LPw = op->ib_work + 2 * n;
    const int g = (int)div_up(n, 256);
    k_ibem_rhs_pre<<<g, 256, 0, s>>>(gp, gm, n, w);
    FB_LAUNCH_CHECK();
    FB_CHECK(fb_apply_any(op->sub[1], w, Lw, s));
    FB_CHECK(fb_apply_any(op->sub[3], w, LPw, s));
    k_ibem_rhs_post<<<g, 256, 0, s>>>(gp, gm, Lw, LPw, n, b);
    FB_LAUNCH_CHECK();
    fb_count_launch(2);
    return FB_OK;
}

fb_status fb_eval_impl(const fb_mesh*, double, const cd*, const cd*, const double*, const double*, int64_t, cd*,
                       cudaStream_t);

fb_status fb_ibem_field_impl(fb_op* op, const cd* x, const cd* gp, const cd* gm, const double* rcv, int64_t nr,
                             cd* out, cudaStream_t s) {
    const int64_t n = op->n / 2;
    cd* p = op->ib_work;
    cd* q = op->ib_work + n;
    k_ibem_field_dens<<<div_up(n, 256), 256, 0, s>>>(x, gp, gm, op->ib_beta_p, op->ib_beta_m, op->k, n, p, q);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return fb_eval_impl(op->mesh, op->k, p, q, nullptr, rcv, nr, out, s);
}
