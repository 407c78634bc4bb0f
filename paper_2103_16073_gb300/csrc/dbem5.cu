// Direct formulation for the unknown q = d psi_sc/dn (Sec. 2.2, Eq. dbem5):
//   1/2 q + (1/zeta) M[zeta q] + (k/(i zeta)) L[q] = 1/2 gamma + (1/zeta) M[zeta gamma]
// with zeta = 1/beta per element (beta != 0 everywhere), i.e.
//   A5 q = 1/2 q + beta M[q / beta] - i k beta L[q].
// psi_sc follows from the boundary condition q - i k beta psi_sc = gamma.
// Composed of the M and L operators (dense or FMM) of the same mesh and tree.
#include <vector>

#include "common.cuh"

namespace {

__device__ __forceinline__ cd cdiv(cd a, cd b) {
    double d = b.re * b.re + b.im * b.im;
    return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

__global__ void k_d5_div(const cd* __restrict__ x, const cd* __restrict__ beta, int64_t n, cd* __restrict__ t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) t[i] = cdiv(x[i], beta[i]);
}

// y = 1/2 q + beta (M t) - i k beta (L q)
__global__ void k_d5_post(const cd* __restrict__ q, const cd* __restrict__ beta, double k, int64_t n,
                          const cd* __restrict__ Mt, const cd* __restrict__ Lq, cd* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd b = beta[i];
    cd ikb = mk(-k * b.im, k * b.re);
    y[i] = mk(0.5, 0.0) * q[i] + b * Mt[i] - ikb * Lq[i];
}

// b = 1/2 gamma + beta (M t), t = gamma / beta
__global__ void k_d5_rhs(const cd* __restrict__ g, const cd* __restrict__ beta, int64_t n, const cd* __restrict__ Mt,
                         cd* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = mk(0.5, 0.0) * g[i] + beta[i] * Mt[i];
}

__global__ void k_d5_psi(const cd* __restrict__ q, const cd* __restrict__ g, const cd* __restrict__ beta, double k,
                         int64_t n, cd* __restrict__ psi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd b = beta[i];
    psi[i] = cdiv(q[i] - g[i], mk(-k * b.im, k * b.re));
}

}  // namespace


fb_status fb_dbem5_create(fb_op* op, cudaStream_t s) {
    const int64_t n = op->mesh->n;
    std::vector<cd> hb(n);
    FB_CUDA(cudaMemcpy(hb.data(), op->mesh->beta, sizeof(cd) * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
        if (hb[i].re == 0.0 && hb[i].im == 0.0)
            return fb_fail(FB_ERR_ARG, "Eq. dbem5 needs a finite impedance (admittance != 0) on every element");
    FB_CHECK(fb_operator_create_impl(op->mesh, op->tree, op->k, FB_OP_M, op->prec, op->d0, op->pmin, s, &op->sub[0]));
    FB_CHECK(fb_operator_create_impl(op->mesh, op->tree, op->k, FB_OP_L, op->prec, op->d0, op->pmin, s, &op->sub[1]));
    FB_CHECK(dalloc(&op->ib_work, (size_t)3 * n));
    FB_CHECK(dalloc(&op->ib_beta_m, (size_t)n));
    FB_CUDA(cudaMemcpyAsync(op->ib_beta_m, op->mesh->beta, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s));
    return FB_OK;
}

fb_status fb_dbem5_apply(fb_op* op, const cd* x, cd* y, cudaStream_t s, int nrhs) {
    const int64_t n = op->n;
    cd* t = op->ib_work;
    cd* Mt = op->ib_work + n;
    cd* Lq = op->ib_work + 2 * n;
    const int g = (int)div_up(n, 256);
    for (int r = 0; r < nrhs; ++r) {
        const cd* q = x + (int64_t)r * n;
        k_d5_div<<<g, 256, 0, s>>>(q, op->ib_beta_m, n, t);
        FB_LAUNCH_CHECK();
        FB_CHECK(fb_apply_any(op->sub[0], t, Mt, s));
        FB_CHECK(fb_apply_any(op->sub[1], q, Lq, s));
        k_d5_post<<<g, 256, 0, s>>>(q, op->ib_beta_m, op->k, n, Mt, Lq, y + (int64_t)r * n);
        FB_LAUNCH_CHECK();
        fb_count_launch(2);
    }
    return FB_OK;
}

fb_status fb_dbem5_rhs_impl(fb_op* op, const cd* gamma, cd* b, cudaStream_t s) {
    const int64_t n = op->n;
    cd* t = op->ib_work;
    cd* Mt = op->ib_work + n;
    const int g = (int)div_up(n, 256);
    k_d5_div<<<g, 256, 0, s>>>(gamma, op->ib_beta_m, n, t);
    FB_LAUNCH_CHECK();
    FB_CHECK(fb_apply_any(op->sub[0], t, Mt, s));
    k_d5_rhs<<<g, 256, 0, s>>>(gamma, op->ib_beta_m, n, Mt, b);
    FB_LAUNCH_CHECK();
    fb_count_launch(2);
    return FB_OK;
}

fb_status fb_dbem5_psi_impl(fb_op* op, const cd* q, const cd* gamma, cd* psi, cudaStream_t s) {
    k_d5_psi<<<div_up(op->n, 256), 256, 0, s>>>(q, gamma, op->ib_beta_m, op->k, op->n, psi);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}
