// Flexible GMRES (Sec. 3.1, Sec. 4: the paper solves Eq. (dbem4) by flexible
// GMRES, which admits a preconditioner that changes between iterations) and
// the block-Jacobi preconditioner.  All Krylov vectors, the Hessenberg matrix
// and the Givens rotations are FP64; the operator may compute in FP32.
//
// Arnoldi orthogonalisation: classical Gram-Schmidt applied twice (CGS2),
// two fused kernels per pass instead of j sequential dot products.
#include <cmath>
#include <vector>

#include "common.cuh"

// ---------------------------------------------------------- vector ops ----
constexpr int KB = 256;

__device__ __forceinline__ void block_reduce_add(double v, double* target) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(target, v);
    }
    __syncthreads();
}

// h[i] += sum_n conj(V_i[n]) w[n], i = blockIdx.y
__global__ void k_mdot(const cd* __restrict__ V, int64_t n, const cd* __restrict__ w, cd* h) {
    int i = blockIdx.y;
    const cd* v = V + (int64_t)i * n;
    cd acc = mk(0.0, 0.0);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        cmacc(acc, v[q], w[q]);
    block_reduce_add(acc.re, &h[i].re);
    block_reduce_add(acc.im, &h[i].im);
}

// w -= sum_{i<=j} V_i h[i]
__global__ void k_gs_update(const cd* __restrict__ V, int64_t n, int j1, const cd* __restrict__ h, cd* w) {
    __shared__ cd hs[1024];
    for (int i = threadIdx.x; i < j1; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        cd a = w[q];
        for (int i = 0; i < j1; ++i) {
            cd v = V[(int64_t)i * n + q];
            a.re -= v.re * hs[i].re - v.im * hs[i].im;
            a.im -= v.re * hs[i].im + v.im * hs[i].re;
        }
        w[q] = a;
    }
}

__global__ void k_norm2(const cd* __restrict__ w, int64_t n, double* out) {
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        acc += abs2(w[q]);
    block_reduce_add(acc, out);
}

__global__ void k_scale(cd* __restrict__ out, const cd* __restrict__ in, int64_t n, const double* s) {
    double f = *s;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = f * in[q];
}

// out = a - b
__global__ void k_sub(cd* out, const cd* a, const cd* b, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = a[q] - b[q];
}
__global__ void k_add(cd* out, const cd* a, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = out[q] + a[q];
}

// x += sum_i Z_i y[i]
__global__ void k_update_x(cd* x, const cd* __restrict__ Z, int64_t n, int j1, const cd* __restrict__ y) {
    __shared__ cd ys[1024];
    for (int i = threadIdx.x; i < j1; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        cd a = x[q];
        for (int i = 0; i < j1; ++i) cmac(a, Z[(int64_t)i * n + q], ys[i]);
        x[q] = a;
    }
}

// Small dense state of one restart cycle (device).
struct Hess {
    int m;
    cd* H;      // (m+1) x m, column-major: H[j*(m+1) + i]
    cd* cs;     // m (real part used)
    cd* sn;     // m
    cd* g;      // m+1
    cd* h;      // m+1 scratch (CGS pass)
    cd* y;      // m
    double* nrm2;
    double* inv;      // 1 / H[j+1][j]
    double* est;      // |g[j+1]|
};

// Starts a cycle: g = (beta, 0, ...), inv = 1/beta (beta = sqrt(nrm2)).
__device__ void cycle_start(const Hess& hs) {
    double beta = sqrt(*hs.nrm2);
    for (int i = 0; i <= hs.m; ++i) hs.g[i] = mk(0.0, 0.0);
    for (int i = 0; i < (hs.m + 1) * hs.m; ++i) hs.H[i] = mk(0.0, 0.0);
    hs.g[0] = mk(beta, 0.0);
    *hs.inv = beta > 0.0 ? 1.0 / beta : 0.0;
    *hs.est = beta;
}
__global__ void k_cycle_start(Hess hs) { cycle_start(hs); }

// Adds the CGS pass coefficients into column j.
__global__ void k_accum_h(Hess hs, int j) {
    int i = threadIdx.x;
    if (i <= j) hs.H[j * (hs.m + 1) + i] = hs.H[j * (hs.m + 1) + i] + hs.h[i];
}

// Completes column j: H[j+1][j] = ||w||, previous rotations, new rotation,
// residual estimate |g[j+1]|, inv = 1/H[j+1][j].
__device__ void arnoldi_close(const Hess& hs, int j) {
    int ld = hs.m + 1;
    cd* col = hs.H + j * ld;
    double hn = sqrt(*hs.nrm2);
    col[j + 1] = mk(hn, 0.0);
    *hs.inv = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
        cd c = hs.cs[i], s = hs.sn[i];
        cd a = col[i], b = col[i + 1];
        col[i] = c * a + s * b;
        col[i + 1] = conjg(s) * mk(-a.re, -a.im) + conjg(c) * b;
    }
    cd a = col[j], b = col[j + 1];
    double na = sqrt(abs2(a)), nb = sqrt(abs2(b));
    double den = sqrt(na * na + nb * nb);
    cd c, s;
    if (den == 0.0) { c = mk(1.0, 0.0); s = mk(0.0, 0.0); }
    else if (na == 0.0) { c = mk(0.0, 0.0); s = mk(1.0, 0.0); }
    else {
        c = mk(na / den, 0.0);
        s = (1.0 / (na * den)) * (a * conjg(b));
    }
    hs.cs[j] = c;
    hs.sn[j] = s;
    col[j] = c * a + s * b;
    col[j + 1] = mk(0.0, 0.0);
    cd gj = hs.g[j];
    hs.g[j + 1] = conjg(s) * mk(-gj.re, -gj.im);
    hs.g[j] = c * gj;
    *hs.est = sqrt(abs2(hs.g[j + 1]));
}
__global__ void k_arnoldi_close(Hess hs, int j) { arnoldi_close(hs, j); }

// Back substitution H y = g for the first j1 columns.
__device__ void backsolve(const Hess& hs, int j1) {
    int ld = hs.m + 1;
    for (int i = j1 - 1; i >= 0; --i) {
        cd acc = hs.g[i];
        for (int q = i + 1; q < j1; ++q) acc = acc - hs.H[q * ld + i] * hs.y[q];
        cd d = hs.H[i * ld + i];
        double dd = abs2(d);
        // a zero pivot only follows an exact breakdown (or a zero right-hand
        // side); the Krylov space ended there, so the coefficient is 0
        hs.y[i] = dd > 0.0 ? (1.0 / dd) * (acc * conjg(d)) : mk(0.0, 0.0);
    }
}
__global__ void k_backsolve(Hess hs, int j1) { backsolve(hs, j1); }

static inline void cnt(long long n = 1) { fb_count_launch(n); }

static int grid_for(int64_t n) { return (int)std::min<int64_t>(div_up(n, KB), 152 * 8); }

static fb_status norm2(const cd* v, int64_t n, double* d_out, cudaStream_t s) {
    FB_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), s));
    k_norm2<<<grid_for(n), KB, 0, s>>>(v, n, d_out);
    FB_LAUNCH_CHECK();
    cnt();
    return FB_OK;
}

static fb_status read_scalar(const double* d, double* h, cudaStream_t s) {
    FB_CUDA(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    FB_CUDA(cudaStreamSynchronize(s));
    return FB_OK;
}

struct Work {
    int64_t n = 0;
    int m = 0;
    cd *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *d = nullptr, *tmp = nullptr;
    cd* small = nullptr;
    double* scal = nullptr;
    double* host = nullptr;   // pinned scalar
    Hess hs{};
    ~Work() {
        dfree(V); dfree(Z); dfree(w); dfree(r); dfree(d); dfree(tmp); dfree(small); dfree(scal);
        if (host) cudaFreeHost(host);
    }
};

static fb_status work_alloc(Work& W, int64_t n, int m, bool with_z) {
    W.n = n;
    W.m = m;
    FB_CHECK(dalloc(&W.V, (size_t)(m + 1) * n));
    if (with_z) FB_CHECK(dalloc(&W.Z, (size_t)m * n));
    FB_CHECK(dalloc(&W.w, n));
    FB_CHECK(dalloc(&W.r, n));
    FB_CHECK(dalloc(&W.d, n));
    FB_CHECK(dalloc(&W.tmp, n));
    size_t nsmall = (size_t)(m + 1) * m + 4 * (m + 1) + 2 * m + 8;
    FB_CHECK(dalloc(&W.small, nsmall));
    FB_CHECK(dalloc(&W.scal, 8));
    FB_CUDA(cudaMallocHost((void**)&W.host, sizeof(double) * 4));
    cd* sp = W.small;
    W.hs.m = m;
    W.hs.H = sp; sp += (size_t)(m + 1) * m;
    W.hs.cs = sp; sp += m + 1;
    W.hs.sn = sp; sp += m + 1;
    W.hs.g = sp; sp += m + 1;
    W.hs.h = sp; sp += m + 1;
    W.hs.y = sp;
    W.hs.nrm2 = W.scal;
    W.hs.inv = W.scal + 1;
    W.hs.est = W.scal + 2;
    return FB_OK;
}

// k steps of GMRES (one cycle, no restart, no host synchronisation) on
// A d = rhs from d = 0, right-preconditioned by pc; the result in W.d.  Used
// as the inner solver of the inner-outer preconditioner (Sec. 4: FGMRES
// preconditioned by a few GMRES iterations on a low-accuracy FMM).
static fb_status gmres_fixed(fb_op* A, const fb_precond* pc, Work& W, const cd* rhs, int k, cudaStream_t s) {
    const int64_t n = W.n;
    FB_CUDA(cudaMemsetAsync(W.d, 0, sizeof(cd) * n, s));
    FB_CHECK(norm2(rhs, n, W.hs.nrm2, s));
    k_cycle_start<<<1, 1, 0, s>>>(W.hs);
    k_scale<<<grid_for(n), KB, 0, s>>>(W.V, rhs, n, W.hs.inv);
    FB_LAUNCH_CHECK();
    cnt(2);
    for (int j = 0; j < k; ++j) {
        cd* vj = W.V + (int64_t)j * n;
        cd* zj = vj;
        if (pc) {
            zj = W.Z + (int64_t)j * n;
            FB_CHECK(fb_pc_apply(pc, vj, zj, s));
        }
        FB_CHECK(fb_apply_any(A, zj, W.w, s));
        for (int pass = 0; pass < 2; ++pass) {
            FB_CUDA(cudaMemsetAsync(W.hs.h, 0, sizeof(cd) * (j + 1), s));
            dim3 g(std::min(grid_for(n), 64), j + 1);
            k_mdot<<<g, KB, 0, s>>>(W.V, n, W.w, W.hs.h);
            k_gs_update<<<grid_for(n), KB, 0, s>>>(W.V, n, j + 1, W.hs.h, W.w);
            k_accum_h<<<1, 1024, 0, s>>>(W.hs, j);
            cnt(3);
        }
        FB_CHECK(norm2(W.w, n, W.hs.nrm2, s));
        k_arnoldi_close<<<1, 1, 0, s>>>(W.hs, j);
        k_scale<<<grid_for(n), KB, 0, s>>>(W.V + (int64_t)(j + 1) * n, W.w, n, W.hs.inv);
        FB_LAUNCH_CHECK();
        cnt(2);
    }
    k_backsolve<<<1, 1, 0, s>>>(W.hs, k);
    k_update_x<<<grid_for(n), KB, 0, s>>>(W.d, pc ? W.Z : W.V, n, k, W.hs.y);
    FB_LAUNCH_CHECK();
    cnt(2);
    return FB_OK;
}

struct InnerBatch;
// Work buffers of the inner-outer preconditioner: the single-system GMRES
// and, per number of right-hand sides, the lockstep batch (created on first
// use outside any capture).
struct InnerSolver {
    Work W;
    std::map<int, InnerBatch*> batch;
    ~InnerSolver();
};

// Workspace of fb_fgmres_solve on operator A with restart m, kept on A and
// reused while (N, m) match and it holds the Z block a preconditioned solve
// needs; otherwise it is replaced.  Every solve ends with a host read of a
// device scalar, so no kernel of the previous solve still uses it.
static fb_status work_get(fb_op* A, int m, bool with_z, Work** out) {
    Work* W = (Work*)A->fg_work;
    if (W && W->n == A->n && W->m == m && (W->Z || !with_z)) {
        *out = W;
        return FB_OK;
    }
    delete W;
    A->fg_work = nullptr;
    W = new Work();
    fb_status st = work_alloc(*W, A->n, m, with_z);
    if (st != FB_OK) {
        delete W;
        return st;
    }
    A->fg_work = W;
    *out = W;
    return FB_OK;
}

// The first k+1 Arnoldi vectors of the right-preconditioned Krylov space of
// A for the start vector b (the inputs a preconditioner sees in the first k
// iterations of a solve), written to V [(k+1) x N].
fb_status fb_krylov_basis_impl(fb_op* A, const fb_precond* pc, const cd* b, int k, cd* V, cudaStream_t s) {
    Work W;
    FB_CHECK(work_alloc(W, A->n, k, pc != nullptr));
    FB_CHECK(gmres_fixed(A, pc, W, b, k, s));
    FB_CUDA(cudaMemcpyAsync(V, W.V, sizeof(cd) * (size_t)(k + 1) * A->n, cudaMemcpyDeviceToDevice, s));
    FB_CUDA(cudaStreamSynchronize(s));
    return FB_OK;
}

fb_status fb_inner_create(fb_precond* pc, cudaStream_t s) {
    InnerSolver* in = new InnerSolver();
    fb_status st = work_alloc(in->W, pc->n, pc->inner_its, pc->base != nullptr);
    if (st != FB_OK) {
        delete in;
        return st;
    }
    pc->inner = in;
    return FB_OK;
}

void fb_inner_free(void*& inner) {
    delete (InnerSolver*)inner;
    inner = nullptr;
}

// Inner restarted FGMRES on A d = rhs from d = 0 until the Arnoldi estimate
// reaches rel_tol * ||rhs|| or the iteration budget is spent.
static fb_status fgmres_inner(fb_op* A, fb_precond* pc, Work& W, const cd* rhs, double rhs_norm,
                              double rel_tol, int budget, int* iters, double* est_rel, int* status,
                              cudaStream_t s) {
    int64_t n = W.n;
    int m = W.m;
    FB_CUDA(cudaMemsetAsync(W.d, 0, sizeof(cd) * n, s));
    *status = FB_OK;
    int it = 0;
    bool first = true;
    double est = rhs_norm;
    while (true) {
        // r_c = rhs - A d
        if (first) {
            FB_CUDA(cudaMemcpyAsync(W.w, rhs, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s));
        } else {
            FB_CHECK(fb_apply_any(A, W.d, W.tmp, s));
            k_sub<<<grid_for(n), KB, 0, s>>>(W.w, rhs, W.tmp, n);
            cnt();
        }
        first = false;
        FB_CHECK(norm2(W.w, n, W.hs.nrm2, s));
        k_cycle_start<<<1, 1, 0, s>>>(W.hs);
        k_scale<<<grid_for(n), KB, 0, s>>>(W.V, W.w, n, W.hs.inv);
        FB_LAUNCH_CHECK();
        cnt(2);
        FB_CHECK(read_scalar(W.hs.est, W.host, s));
        est = *W.host;
        if (!std::isfinite(est)) { *status = FB_ERR_NAN; break; }
        if (est <= rel_tol * rhs_norm || it >= budget) break;
        int j = 0;
        bool breakdown = false;
        for (; j < m && it < budget; ++j) {
            cd* vj = W.V + (int64_t)j * n;
            cd* zj = vj;
            if (pc) {
                zj = W.Z + (int64_t)j * n;
                FB_CHECK(fb_pc_apply(pc, vj, zj, s));
            }
            FB_CHECK(fb_apply_any(A, zj, W.w, s));
            for (int pass = 0; pass < 2; ++pass) {
                FB_CUDA(cudaMemsetAsync(W.hs.h, 0, sizeof(cd) * (j + 1), s));
                dim3 g(std::min(grid_for(n), 64), j + 1);
                k_mdot<<<g, KB, 0, s>>>(W.V, n, W.w, W.hs.h);
                k_gs_update<<<grid_for(n), KB, 0, s>>>(W.V, n, j + 1, W.hs.h, W.w);
                k_accum_h<<<1, 1024, 0, s>>>(W.hs, j);
                cnt(3);
            }
            FB_CHECK(norm2(W.w, n, W.hs.nrm2, s));
            k_arnoldi_close<<<1, 1, 0, s>>>(W.hs, j);
            k_scale<<<grid_for(n), KB, 0, s>>>(W.V + (int64_t)(j + 1) * n, W.w, n, W.hs.inv);
            FB_LAUNCH_CHECK();
            cnt(2);
            // one read per step: nrm2, inv, est are adjacent
            FB_CUDA(cudaMemcpyAsync(W.host, W.hs.nrm2, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
            FB_CUDA(cudaStreamSynchronize(s));
            est = W.host[2];
            double hn = W.host[0];
            ++it;
            if (!std::isfinite(est)) { *status = FB_ERR_NAN; break; }
            if (hn == 0.0) { breakdown = true; ++j; break; }
            if (est <= rel_tol * rhs_norm) { ++j; break; }
        }
        if (*status != FB_OK) break;
        int j1 = j;
        if (j1 > 0) {
            k_backsolve<<<1, 1, 0, s>>>(W.hs, j1);
            k_update_x<<<grid_for(n), KB, 0, s>>>(W.d, pc ? W.Z : W.V, n, j1, W.hs.y);
            FB_LAUNCH_CHECK();
            cnt(2);
        }
        if (breakdown || est <= rel_tol * rhs_norm || it >= budget) break;
    }
    *iters = it;
    *est_rel = rhs_norm > 0 ? est / rhs_norm : 0.0;
    return FB_OK;
}

fb_status fb_fgmres_impl(fb_op* A, fb_precond* pc, const cd* b, cd* x, const fb_solver_opts* o,
                         fb_solve_info* info, cudaStream_t s) {
    fb_solver_opts opts = *o;
    if (opts.restart < 1 || opts.restart > 1000) return fb_fail(FB_ERR_ARG, "restart must be in [1, 1000]");
    if (opts.maxit < 1) return fb_fail(FB_ERR_ARG, "maxit must be >= 1");
    if (opts.max_refine < 1) opts.max_refine = 1;
    fb_op* T = opts.true_op ? const_cast<fb_op*>(opts.true_op) : A;
    if (T->n != A->n) return fb_fail(FB_ERR_ARG, "true_op size differs");
    int64_t n = A->n;
    int m = opts.restart;
    Work* Wp = nullptr;
    FB_CHECK(work_get(A, m, pc != nullptr, &Wp));
    Work& W = *Wp;
    double* bnorm2 = W.scal + 3;

    fb_solve_info inf{};
    FB_CUDA(cudaMemsetAsync(x, 0, sizeof(cd) * n, s));
    FB_CHECK(norm2(b, n, bnorm2, s));
    double bn2 = 0;
    FB_CHECK(read_scalar(bnorm2, &bn2, s));
    double bn = std::sqrt(bn2);
    if (bn == 0.0) {
        inf.status = FB_OK;
        if (info) *info = inf;
        return FB_OK;
    }
    FB_CUDA(cudaMemcpyAsync(W.r, b, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s));
    double rn = bn;
    double inner_floor = opts.inner_tol > 0 ? opts.inner_tol : 0.0;
    int status = FB_OK;
    fb_precond* cur = pc;
    for (int sweep = 0; sweep < opts.max_refine; ++sweep) {
        if (rn <= opts.tol * bn) break;
        double rel = std::max(inner_floor, 0.5 * opts.tol * bn / rn);
        int its = 0, st = FB_OK;
        double est_rel = 0;
        FB_CHECK(fgmres_inner(A, cur, W, W.r, rn, rel, opts.maxit - inf.iters, &its, &est_rel, &st, s));
        inf.iters += its;
        inf.est_relres = est_rel * rn / bn;
        inf.refinements = sweep + 1;
        const bool learned = cur && cur->net && cur->base;
        if (learned && st == FB_ERR_NAN) {
            // discard the correction and continue under the block-Jacobi base
            cur = const_cast<fb_precond*>(cur->base);
            inf.pc_fallbacks++;
            if (inf.iters >= opts.maxit) break;
            continue;
        }
        k_add<<<grid_for(n), KB, 0, s>>>(x, W.d, n);
        cnt();
        // true residual r = b - T x
        FB_CHECK(fb_apply_any(T, x, W.tmp, s));
        k_sub<<<grid_for(n), KB, 0, s>>>(W.r, b, W.tmp, n);
        FB_LAUNCH_CHECK();
        cnt();
        inf.true_matvecs++;
        double r2 = 0;
        FB_CHECK(norm2(W.r, n, W.scal + 4, s));
        FB_CHECK(read_scalar(W.scal + 4, &r2, s));
        const double rn_prev = rn;
        rn = std::sqrt(r2);
        if (st != FB_OK) { status = st; break; }
        if (learned && std::isfinite(rn) && rn > opts.tol * bn && !(rn <= 0.5 * rn_prev)) {
            cur = const_cast<fb_precond*>(cur->base);
            inf.pc_fallbacks++;
        }
        if (!std::isfinite(rn)) { status = FB_ERR_NAN; break; }
        if (inf.iters >= opts.maxit) break;
    }
    inf.true_relres = rn / bn;
    if (status == FB_OK && !(inf.true_relres <= opts.tol)) status = FB_ERR_NOCONV;
    {
        // a bounded device wait that ran out invalidates the products it fed
        fb_status ws = fb_op_wait_status(A);
        if (ws == FB_OK && T != A) ws = fb_op_wait_status(T);
        if (ws == FB_OK && pc && pc->inner_op) ws = fb_op_wait_status(pc->inner_op);
        if (ws != FB_OK) status = ws;
    }
    inf.status = status;
    if (info) *info = inf;
    if (status != FB_OK) {
        fb_set_error(status, status == FB_ERR_NOCONV ? "FGMRES did not reach the tolerance"
                                                     : "FGMRES stopped on a non-finite residual");
    }
    return status;
}

// ------------------------------------------------------- block Jacobi ----
// In-place Gauss-Jordan inversion with partial pivoting of each leaf block.
__global__ void k_bj_extract(const cd* nf, const int64_t* nf_off, const int32_t* nf_ncol,
                             const int32_t* leaf_start, const int32_t* ucnt, const int32_t* ulist,
                             const int64_t* blk_off, cd* out) {
    int t = blockIdx.x;
    int nr = leaf_start[t + 1] - leaf_start[t];
    int K = nf_ncol[t];
    int c0 = 0;
    for (int i = 0; i < ucnt[t]; ++i) {
        int sl = ulist[(int64_t)t * FB_ULIST + i];
        if (sl == t) break;
        c0 += leaf_start[sl + 1] - leaf_start[sl];
    }
    for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) {
        int r = e / nr, c = e % nr;
        out[blk_off[t] + e] = nf[nf_off[t] + (int64_t)r * K + c0 + c];
    }
}

fb_status fb_self_blocks(const fb_op* op, const int64_t* d_off, cd* out, cudaStream_t s) {
    const fb_tree* t = op->tree;
    int nleaf = t->nbox[t->L];
    k_bj_extract<<<nleaf, 256, 0, s>>>(op->nf64, op->nf_off, op->nf_ncol, t->leaf_start, t->ucnt, t->ulist, d_off,
                                       out);
    FB_LAUNCH_CHECK();
    return FB_OK;
}

// In-place Gauss-Jordan inverse with partial pivoting of the block of leaf t
// (order `scale` x its element count; scale 2 for the indirect system).
__global__ void k_bj_invert(const int32_t* leaf_start, const int64_t* blk_off, cd* blocks, int* piv_scr,
                            int* singular, int scale) {
    int t = blockIdx.x;
    int n = scale * (leaf_start[t + 1] - leaf_start[t]);
    cd* a = blocks + blk_off[t];
    int* piv = piv_scr + scale * leaf_start[t];
    extern __shared__ cd fcol[];
    __shared__ int s_p;
    __shared__ cd s_inv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            double best = abs2(a[(int64_t)k * n + k]);
            for (int i = k + 1; i < n; ++i) {
                double v = abs2(a[(int64_t)i * n + k]);
                if (v > best) { best = v; p = i; }
            }
            piv[k] = p;
            s_p = p;
            if (best == 0.0) { atomicExch(singular, 1); s_inv = mk(0.0, 0.0); }
            else {
                cd d = a[(int64_t)p * n + k];
                s_inv = (1.0 / best) * conjg(d);
            }
        }
        __syncthreads();
        int p = s_p;
        if (p != k)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                cd tmp = a[(int64_t)k * n + j];
                a[(int64_t)k * n + j] = a[(int64_t)p * n + j];
                a[(int64_t)p * n + j] = tmp;
            }
        __syncthreads();
        cd inv = s_inv;
        if (threadIdx.x == 0) a[(int64_t)k * n + k] = mk(1.0, 0.0);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) a[(int64_t)k * n + j] = inv * a[(int64_t)k * n + j];
        for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = (i == k) ? mk(0.0, 0.0) : a[(int64_t)i * n + k];
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int i = e / n, j = e % n;
            if (i == k) continue;
            cd f = fcol[i];
            if (j == k) a[(int64_t)i * n + j] = mk(0.0, 0.0) - f * a[(int64_t)k * n + j];
            else a[(int64_t)i * n + j] = a[(int64_t)i * n + j] - f * a[(int64_t)k * n + j];
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                cd tmp = a[(int64_t)i * n + k];
                a[(int64_t)i * n + k] = a[(int64_t)i * n + p];
                a[(int64_t)i * n + p] = tmp;
            }
        __syncthreads();
    }
}

template <class R>
__global__ void k_bj_apply(const int32_t* leaf_start, const int32_t* perm, const int64_t* blk_off,
                           const cx<R>* blocks, const cd* __restrict__ x, cd* __restrict__ y, int64_t stride) {
    x += blockIdx.y * stride;   // right-hand side blockIdx.y
    y += blockIdx.y * stride;
    int t = blockIdx.x;
    int r0 = leaf_start[t], n = leaf_start[t + 1] - r0;
    extern __shared__ unsigned char raw[];
    cx<R>* xs = (cx<R>*)raw;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = from_d<R>(x[perm[r0 + i]]);
    __syncthreads();
    const cx<R>* a = blocks + blk_off[t];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < n; r += nw) {
        cx<R> acc = mk<R>(0, 0);
        for (int c = lane; c < n; c += 32) cmac(acc, a[(int64_t)r * n + c], xs[c]);
        for (int o = 16; o > 0; o >>= 1) {
            acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
            acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
        }
        if (lane == 0) y[perm[r0 + r]] = mk<double>((double)acc.re, (double)acc.im);
    }
}

// Block Jacobi of the indirect system (FB_OP_IBEM, Eq. ibem5): per leaf the
// 2n x 2n matrix coupling its n elements' two equations to their psi+ and
// psi-, from the self-blocks of M, L, M', L' (tree order, row = target):
//   [ I/2 - M + L a+      I/2 + M + L a-     ]   a = -i k beta of the
//   [ -M' + a+/2 + L' a+   M' - a-/2 + L' a- ]   column (diagonal: row) element
__global__ void k_ibem_bj_assemble(const int32_t* leaf_start, const int32_t* perm, const int64_t* off1,
                                   const int64_t* off2, const cd* Mb, const cd* Lb, const cd* MPb, const cd* LPb,
                                   const cd* bp, const cd* bm, double k, cd* out) {
    int t = blockIdx.x;
    int r0 = leaf_start[t], n = leaf_start[t + 1] - r0, w = 2 * n;
    cd* B = out + off2[t];
    const int64_t o = off1[t];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        int ei = perm[r0 + i], ej = perm[r0 + j];
        cd apj = mk(k * bp[ej].im, -k * bp[ej].re), amj = mk(k * bm[ej].im, -k * bm[ej].re);
        cd m = Mb[o + e], l = Lb[o + e], mp = MPb[o + e], lp = LPb[o + e];
        cd h = mk(i == j ? 0.5 : 0.0, 0.0);
        B[(int64_t)i * w + j] = h - m + l * apj;
        B[(int64_t)i * w + n + j] = h + m + l * amj;
        cd d21 = mk(0.0, 0.0), d22 = mk(0.0, 0.0);
        if (i == j) {
            d21 = mk(0.5 * k * bp[ei].im, -0.5 * k * bp[ei].re);    // a+/2
            d22 = mk(-0.5 * k * bm[ei].im, 0.5 * k * bm[ei].re);    // -a-/2
        }
        B[(int64_t)(n + i) * w + j] = d21 - mp + lp * apj;
        B[(int64_t)(n + i) * w + n + j] = d22 + mp + lp * amj;
    }
}

// z = B^-1 r per leaf: rows 0..n-1 of r are the first equations of the
// leaf's elements (r[e]), rows n..2n-1 the second (r[N + e]); columns map to
// psi+ (z[e]) and psi- (z[N + e]).
__global__ void k_ibem_bj_apply(const int32_t* leaf_start, const int32_t* perm, const int64_t* off2, const cd* inv,
                                const cd* __restrict__ x, cd* __restrict__ y, int64_t N) {
    int t = blockIdx.x;
    int r0 = leaf_start[t], n = leaf_start[t + 1] - r0, w = 2 * n;
    extern __shared__ unsigned char raw[];
    cd* xs = (cd*)raw;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int e = perm[r0 + i];
        xs[i] = x[e];
        xs[n + i] = x[N + e];
    }
    __syncthreads();
    const cd* a = inv + off2[t];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < w; r += nw) {
        cd acc = mk(0.0, 0.0);
        for (int c = lane; c < w; c += 32) cmac(acc, a[(int64_t)r * w + c], xs[c]);
        for (int q = 16; q > 0; q >>= 1) {
            acc.re += __shfl_xor_sync(0xffffffffu, acc.re, q);
            acc.im += __shfl_xor_sync(0xffffffffu, acc.im, q);
        }
        if (lane == 0) y[r < n ? perm[r0 + r] : N + perm[r0 + r - n]] = acc;
    }
}

void fb_precond_free(fb_precond* pc);

// Block Jacobi of Eq. (dbem5) (FB_OP_DBEM5): per leaf
//   B_ij = delta_ij / 2 + beta_i M_ij / beta_j - i k beta_i L_ij
// from the self-blocks of M and L (tree order, row = target).
__global__ void k_d5_bj_assemble(const int32_t* leaf_start, const int32_t* perm, const int64_t* off1,
                                 const cd* Mb, const cd* Lb, const cd* beta, double k, cd* out) {
    int t = blockIdx.x;
    int r0 = leaf_start[t], n = leaf_start[t + 1] - r0;
    const int64_t o = off1[t];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        cd bi = beta[perm[r0 + i]], bj = beta[perm[r0 + j]];
        double d = bj.re * bj.re + bj.im * bj.im;
        cd ratio = bi * mk(bj.re / d, -bj.im / d);
        cd ikb = mk(-k * bi.im, k * bi.re);
        out[o + e] = mk(i == j ? 0.5 : 0.0, 0.0) + ratio * Mb[o + e] - ikb * Lb[o + e];
    }
}

static fb_status dbem5_bj_create(fb_op* op, cudaStream_t s, fb_precond** out) {
    const fb_tree* t = op->tree;
    if (!t || op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "block Jacobi needs an FMM operator");
    const int nleaf = t->nbox[t->L];
    std::vector<int64_t> off(nleaf + 1, 0);
    int maxn = 0;
    for (int b = 0; b < nleaf; ++b) {
        int64_t nb = t->h_leaf_start[b + 1] - t->h_leaf_start[b];
        maxn = std::max<int>(maxn, (int)nb);
        off[b + 1] = off[b] + nb * nb;
    }
    fb_precond* pc = new fb_precond();
    pc->op = op;
    pc->kind = FB_PC_BLOCK_JACOBI;
    pc->n = op->n;
    cd* tmp[2] = {nullptr, nullptr};
    const cd* self[2] = {nullptr, nullptr};
    int* piv = nullptr;
    int* sing = nullptr;
    auto cleanup = [&]() { dfree(tmp[0]); dfree(tmp[1]); dfree(piv); dfree(sing); };
    fb_status st = FB_OK;
    if ((st = dalloc(&pc->blk_off, nleaf + 1)) || (st = dalloc(&pc->inv64, std::max<int64_t>(off[nleaf], 1))) ||
        (st = dalloc(&piv, op->n)) || (st = dalloc(&sing, 1))) {
        cleanup();
        fb_precond_free(pc);
        return st;
    }
    cudaMemcpyAsync(pc->blk_off, off.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(sing, 0, sizeof(int), s);
    for (int q = 0; q < 2 && st == FB_OK; ++q) {   // sub-operators: 0 = M, 1 = L
        const fb_op* sub = op->sub[q];
        if (sub->nf64) {
            if ((st = dalloc(&tmp[q], std::max<int64_t>(off[nleaf], 1))) == FB_OK)
                st = fb_self_blocks(sub, pc->blk_off, tmp[q], s);
            self[q] = tmp[q];
        } else {
            self[q] = sub->self64;
        }
    }
    if (st == FB_OK) {
        k_d5_bj_assemble<<<nleaf, 256, 0, s>>>(t->leaf_start, t->perm, pc->blk_off, self[0], self[1], op->ib_beta_m,
                                               op->k, pc->inv64);
        st = fb_smem_cap((const void*)k_bj_invert, sizeof(cd) * std::max(maxn, 1));
    }
    if (st == FB_OK) {
        k_bj_invert<<<nleaf, 256, sizeof(cd) * std::max(maxn, 1), s>>>(t->leaf_start, pc->blk_off, pc->inv64, piv,
                                                                        sing, 1);
        int hs = 0;
        cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fb_fail(FB_ERR_CUDA, std::string("dbem5 block Jacobi: ") + cudaGetErrorString(e));
        else if (hs) st = fb_fail(FB_ERR_BREAKDOWN, "singular leaf block in the dbem5 block-Jacobi setup");
    }
    cleanup();
    if (st != FB_OK) {
        fb_precond_free(pc);
        return st;
    }
    fb_count_launch(2);
    *out = pc;
    return FB_OK;
}

static fb_status ibem_bj_create(fb_op* op, cudaStream_t s, fb_precond** out) {
    const fb_tree* t = op->tree;
    if (!t || op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "block Jacobi needs an FMM operator");
    const int nleaf = t->nbox[t->L];
    std::vector<int64_t> off1(nleaf + 1, 0), off2(nleaf + 1, 0);
    int maxn = 0;
    for (int b = 0; b < nleaf; ++b) {
        int64_t nb = t->h_leaf_start[b + 1] - t->h_leaf_start[b];
        maxn = std::max<int>(maxn, (int)nb);
        off1[b + 1] = off1[b] + nb * nb;
        off2[b + 1] = off2[b] + 4 * nb * nb;
    }
    fb_precond* pc = new fb_precond();
    pc->op = op;
    pc->kind = FB_PC_BLOCK_JACOBI;
    pc->n = op->n;
    pc->ibem = 1;
    int64_t* d_off1 = nullptr;
    cd* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
    const cd* self[4] = {nullptr, nullptr, nullptr, nullptr};
    int* piv = nullptr;
    int* sing = nullptr;
    auto cleanup = [&]() {
        dfree(d_off1);
        for (int q = 0; q < 4; ++q) dfree(tmp[q]);
        dfree(piv);
        dfree(sing);
    };
    fb_status st = FB_OK;
    if ((st = dalloc(&d_off1, nleaf + 1)) || (st = dalloc(&pc->blk_off, nleaf + 1)) ||
        (st = dalloc(&pc->inv64, off2[nleaf])) || (st = dalloc(&piv, 2 * op->n)) || (st = dalloc(&sing, 1))) {
        cleanup();
        fb_precond_free(pc);
        return st;
    }
    cudaMemcpyAsync(d_off1, off1.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(pc->blk_off, off2.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(sing, 0, sizeof(int), s);
    for (int q = 0; q < 4 && st == FB_OK; ++q) {
        const fb_op* sub = op->sub[q];
        if (sub->nf64) {
            if ((st = dalloc(&tmp[q], std::max<int64_t>(off1[nleaf], 1))) == FB_OK)
                st = fb_self_blocks(sub, d_off1, tmp[q], s);
            self[q] = tmp[q];
        } else {
            self[q] = sub->self64;
        }
    }
    if (st == FB_OK) {
        // sub-operators: 0 = M, 1 = L, 2 = M', 3 = L'
        k_ibem_bj_assemble<<<nleaf, 256, 0, s>>>(t->leaf_start, t->perm, d_off1, pc->blk_off, self[0], self[1],
                                                 self[2], self[3], op->ib_beta_p, op->ib_beta_m, op->k, pc->inv64);
        st = fb_smem_cap((const void*)k_bj_invert, sizeof(cd) * 2 * std::max(maxn, 1));
    }
    if (st == FB_OK) {
        k_bj_invert<<<nleaf, 256, sizeof(cd) * 2 * std::max(maxn, 1), s>>>(t->leaf_start, pc->blk_off, pc->inv64,
                                                                            piv, sing, 2);
        int hs = 0;
        cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fb_fail(FB_ERR_CUDA, std::string("indirect block Jacobi: ") + cudaGetErrorString(e));
        else if (hs) st = fb_fail(FB_ERR_BREAKDOWN, "singular leaf block in the indirect block-Jacobi setup");
    }
    cleanup();
    if (st != FB_OK) {
        fb_precond_free(pc);
        return st;
    }
    fb_count_launch(2);
    *out = pc;
    return FB_OK;
}

__global__ void k_d2f_bj(const cd* a, cf* b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = to_f(a[i]);
}

// ------------------------------------------------------ batched FGMRES ----
// nrhs independent systems A x_r = b_r with one operator solved in lockstep:
// every Arnoldi step applies the preconditioner and the operator to the nrhs
// current basis vectors in one batched call (fb_pc_apply / fb_apply_any with
// nrhs), so the operator's data are read once per step for all systems.  Each
// system keeps its own Hessenberg matrix, Givens rotations, restart cycle,
// convergence test and true-residual refinement; a system that has converged
// is masked out of the Krylov updates (its matvec column is still computed
// until the whole batch finishes).  Layouts: V [(m+1)][R][N], Z [m][R][N],
// vectors [R][N]; Hessenberg state [R][...].
namespace {

__global__ void k_bmdot(const cd* __restrict__ V, int64_t n, int R, const cd* __restrict__ w, cd* h, int hstride,
                        const int* act) {
    int r = blockIdx.z, i = blockIdx.y;
    if (!act[r]) return;
    const cd* v = V + ((int64_t)i * R + r) * n;
    const cd* wr = w + (int64_t)r * n;
    cd acc = mk(0.0, 0.0);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        cmacc(acc, v[q], wr[q]);
    block_reduce_add(acc.re, &h[r * hstride + i].re);
    block_reduce_add(acc.im, &h[r * hstride + i].im);
}

__global__ void k_bgs_update(const cd* __restrict__ V, int64_t n, int R, int j1, const cd* __restrict__ h,
                             int hstride, cd* w, const int* act) {
    int r = blockIdx.y;
    if (!act[r]) return;
    __shared__ cd hs[1024];
    for (int i = threadIdx.x; i < j1; i += blockDim.x) hs[i] = h[r * hstride + i];
    __syncthreads();
    cd* wr = w + (int64_t)r * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        cd a = wr[q];
        for (int i = 0; i < j1; ++i) {
            cd v = V[((int64_t)i * R + r) * n + q];
            a.re -= v.re * hs[i].re - v.im * hs[i].im;
            a.im -= v.re * hs[i].im + v.im * hs[i].re;
        }
        wr[q] = a;
    }
}

__global__ void k_bnorm2(const cd* __restrict__ w, int64_t n, double* out, int ostride, const int* act) {
    int r = blockIdx.y;
    if (act && !act[r]) return;
    const cd* wr = w + (int64_t)r * n;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        acc += abs2(wr[q]);
    block_reduce_add(acc, out + r * ostride);
}

// out_r = f_r in_r with f_r = scal[r * ostride]
__global__ void k_bscale(cd* __restrict__ out, const cd* __restrict__ in, int64_t n, const double* f, int fstride,
                         const int* act) {
    int r = blockIdx.y;
    if (!act[r]) return;
    double a = f[r * fstride];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[r * n + q] = a * in[r * n + q];
}

// out_r = a_r - b_r (masked)
__global__ void k_bsub(cd* out, const cd* a, const cd* b, int64_t n, const int* act) {
    int r = blockIdx.y;
    if (act && !act[r]) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[r * n + q] = a[r * n + q] - b[r * n + q];
}
__global__ void k_badd(cd* out, const cd* a, int64_t n, const int* act) {
    int r = blockIdx.y;
    if (!act[r]) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[r * n + q] = out[r * n + q] + a[r * n + q];
}

// x_r += sum_{i < j1_r} Z_{i,r} y_r[i]
__global__ void k_bupdate_x(cd* x, const cd* __restrict__ Z, int64_t n, int R, const int* j1, const cd* y,
                            int ystride) {
    int r = blockIdx.y;
    int jr = j1[r];
    if (jr <= 0) return;
    __shared__ cd ys[1024];
    for (int i = threadIdx.x; i < jr; i += blockDim.x) ys[i] = y[r * ystride + i];
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        cd a = x[r * n + q];
        for (int i = 0; i < jr; ++i) cmac(a, Z[((int64_t)i * R + r) * n + q], ys[i]);
        x[r * n + q] = a;
    }
}

__global__ void k_bcycle_start(const Hess* hs, const int* act) {
    int r = blockIdx.x;
    if (act[r]) cycle_start(hs[r]);
}
__global__ void k_baccum_h(const Hess* hs, int j, const int* act) {
    int r = blockIdx.x, i = threadIdx.x;
    if (!act[r]) return;
    const Hess& h = hs[r];
    if (i <= j) h.H[j * (h.m + 1) + i] = h.H[j * (h.m + 1) + i] + h.h[i];
}
__global__ void k_barnoldi_close(const Hess* hs, int j, const int* act) {
    int r = blockIdx.x;
    if (act[r]) arnoldi_close(hs[r], j);
}
__global__ void k_bbacksolve(const Hess* hs, const int* j1) {
    int r = blockIdx.x;
    if (j1[r] > 0) backsolve(hs[r], j1[r]);
}

}  // namespace

struct BatchWork {
    int64_t n = 0;
    int m = 0, R = 0;
    cd *V = nullptr, *Z = nullptr, *W = nullptr, *Rs = nullptr, *D = nullptr, *T = nullptr;
    cd* small = nullptr;
    double* scal = nullptr;     // [R][4]: nrm2, inv, est, spare
    int* dint = nullptr;        // act [R], j1 [R]
    Hess* dhs = nullptr;
    double* host = nullptr;     // pinned [R][4]
    int* hint = nullptr;        // pinned act [R], j1 [R]
    ~BatchWork() {
        dfree(V); dfree(Z); dfree(W); dfree(Rs); dfree(D); dfree(T); dfree(small); dfree(scal); dfree(dint);
        dfree(dhs);
        if (host) cudaFreeHost(host);
        if (hint) cudaFreeHost(hint);
    }
};

static fb_status bwork_alloc(BatchWork& B, int64_t n, int m, int R, bool with_z) {
    B.n = n;
    B.m = m;
    B.R = R;
    FB_CHECK(dalloc(&B.V, (size_t)(m + 1) * R * n));
    if (with_z) FB_CHECK(dalloc(&B.Z, (size_t)m * R * n));
    FB_CHECK(dalloc(&B.W, (size_t)R * n));
    FB_CHECK(dalloc(&B.Rs, (size_t)R * n));
    FB_CHECK(dalloc(&B.D, (size_t)R * n));
    FB_CHECK(dalloc(&B.T, (size_t)R * n));
    // small state: H [R][(m+1) m] | h, cs, sn, g, y, spare [R][m+1] each
    FB_CHECK(dalloc(&B.small, (size_t)R * (m + 1) * m + (size_t)R * (m + 1) * 6));
    FB_CHECK(dalloc(&B.scal, (size_t)4 * R));
    FB_CHECK(dalloc(&B.dint, (size_t)2 * R));
    FB_CHECK(dalloc(&B.dhs, (size_t)R));
    FB_CUDA(cudaMallocHost((void**)&B.host, sizeof(double) * 4 * R));
    FB_CUDA(cudaMallocHost((void**)&B.hint, sizeof(int) * 2 * R));
    return FB_OK;
}

// Workspace of fb_fgmres_solve_multi, cached on A like work_get's (reused
// while N, m and the number of systems match).
static fb_status bwork_get(fb_op* A, int m, int R, bool with_z, BatchWork** out) {
    BatchWork* B = (BatchWork*)A->fg_bwork;
    if (B && B->n == A->n && B->m == m && B->R == R && (B->Z || !with_z)) {
        *out = B;
        return FB_OK;
    }
    delete B;
    A->fg_bwork = nullptr;
    B = new BatchWork();
    fb_status st = bwork_alloc(*B, A->n, m, R, with_z);
    if (st != FB_OK) {
        delete B;
        return st;
    }
    A->fg_bwork = B;
    *out = B;
    return FB_OK;
}

void fb_krylov_free(fb_op* op) {
    delete (Work*)op->fg_work;
    delete (BatchWork*)op->fg_bwork;
    op->fg_work = nullptr;
    op->fg_bwork = nullptr;
}

// Lockstep fixed-step GMRES of the inner-outer preconditioner on R
// right-hand sides: the batch workspace with its Hessenberg states, every
// system active and taking exactly k = B.m steps (set once at creation, so
// an application uploads nothing and can be captured into a graph).
struct InnerBatch {
    BatchWork B;
};
InnerSolver::~InnerSolver() {
    for (auto& kv : batch) delete kv.second;
}

static fb_status bwork_hess(BatchWork& B) {
    const int R = B.R, m = B.m;
    std::vector<Hess> hh(R);
    cd* H0 = B.small;
    cd* blk = B.small + (size_t)R * (m + 1) * m;
    for (int r = 0; r < R; ++r) {
        Hess& h = hh[r];
        h.m = m;
        h.H = H0 + (size_t)r * (m + 1) * m;
        h.h = blk + (size_t)0 * R * (m + 1) + (size_t)r * (m + 1);
        h.cs = blk + (size_t)1 * R * (m + 1) + (size_t)r * (m + 1);
        h.sn = blk + (size_t)2 * R * (m + 1) + (size_t)r * (m + 1);
        h.g = blk + (size_t)3 * R * (m + 1) + (size_t)r * (m + 1);
        h.y = blk + (size_t)5 * R * (m + 1) + (size_t)r * (m + 1);
        h.nrm2 = B.scal + 4 * r;
        h.inv = B.scal + 4 * r + 1;
        h.est = B.scal + 4 * r + 2;
    }
    FB_CUDA(cudaMemcpy(B.dhs, hh.data(), sizeof(Hess) * R, cudaMemcpyHostToDevice));
    return FB_OK;
}

static fb_status inner_batch_get(InnerSolver* in, int64_t n, int k, int R, bool with_z, InnerBatch** out) {
    auto it = in->batch.find(R);
    if (it != in->batch.end()) {
        *out = it->second;
        return FB_OK;
    }
    InnerBatch* ib = new InnerBatch();
    fb_status st = bwork_alloc(ib->B, n, k, R, with_z);
    if (st == FB_OK) st = bwork_hess(ib->B);
    if (st == FB_OK) {
        std::vector<int> flags(2 * R);
        for (int r = 0; r < R; ++r) {
            flags[r] = 1;        // active
            flags[R + r] = k;    // steps taken
        }
        if (cudaMemcpy(ib->B.dint, flags.data(), sizeof(int) * 2 * R, cudaMemcpyHostToDevice) != cudaSuccess)
            st = fb_fail(FB_ERR_CUDA, "inner batch flags upload failed");
    }
    if (st != FB_OK) {
        delete ib;
        return st;
    }
    in->batch[R] = ib;
    *out = ib;
    return FB_OK;
}

// k = B.m steps of GMRES on A d_r = rhs_r for the R systems of B at once
// (one multi-RHS matvec and one batched preconditioner application per
// step, CGS2, no host synchronisation); the results in B.D.
static fb_status gmres_fixed_multi(fb_op* A, const fb_precond* pc, BatchWork& B, const cd* rhs, cudaStream_t s) {
    const int64_t n = B.n;
    const int R = B.R, m = B.m;
    const int* dact = B.dint;
    const int* dj1 = B.dint + R;
    const int gx = std::min(grid_for(n), 64);
    FB_CUDA(cudaMemsetAsync(B.D, 0, sizeof(cd) * n * R, s));
    FB_CUDA(cudaMemsetAsync(B.scal, 0, sizeof(double) * 4 * R, s));
    k_bnorm2<<<dim3(grid_for(n), R), KB, 0, s>>>(rhs, n, B.scal, 4, nullptr);
    k_bcycle_start<<<R, 1, 0, s>>>(B.dhs, dact);
    k_bscale<<<dim3(grid_for(n), R), KB, 0, s>>>(B.V, rhs, n, B.scal + 1, 4, dact);
    FB_LAUNCH_CHECK();
    cnt(3);
    cd* h = B.small + (size_t)R * (m + 1) * m;    // [R][m+1] CGS coefficients (Hess.h)
    for (int j = 0; j < m; ++j) {
        cd* Vj = B.V + (int64_t)j * R * n;
        cd* Zj = Vj;
        if (pc) {
            Zj = B.Z + (int64_t)j * R * n;
            FB_CHECK(fb_pc_apply(pc, Vj, Zj, s, R));
        }
        FB_CHECK(fb_apply_any(A, Zj, B.W, s, R));
        for (int pass = 0; pass < 2; ++pass) {
            FB_CUDA(cudaMemsetAsync(h, 0, sizeof(cd) * R * (m + 1), s));
            k_bmdot<<<dim3(gx, j + 1, R), KB, 0, s>>>(B.V, n, R, B.W, h, m + 1, dact);
            k_bgs_update<<<dim3(grid_for(n), R), KB, 0, s>>>(B.V, n, R, j + 1, h, m + 1, B.W, dact);
            k_baccum_h<<<R, 1024, 0, s>>>(B.dhs, j, dact);
            cnt(3);
        }
        FB_CUDA(cudaMemsetAsync(B.scal, 0, sizeof(double) * 4 * R, s));
        k_bnorm2<<<dim3(grid_for(n), R), KB, 0, s>>>(B.W, n, B.scal, 4, dact);
        k_barnoldi_close<<<R, 1, 0, s>>>(B.dhs, j, dact);
        k_bscale<<<dim3(grid_for(n), R), KB, 0, s>>>(B.V + (int64_t)(j + 1) * R * n, B.W, n, B.scal + 1, 4, dact);
        FB_LAUNCH_CHECK();
        cnt(3);
    }
    k_bbacksolve<<<R, 1, 0, s>>>(B.dhs, dj1);
    cd* ys = B.small + (size_t)R * (m + 1) * m + (size_t)R * (m + 1) * 5;   // Hess.y block
    k_bupdate_x<<<dim3(grid_for(n), R), KB, 0, s>>>(B.D, pc ? B.Z : B.V, n, R, dj1, ys, m + 1);
    FB_LAUNCH_CHECK();
    cnt(2);
    return FB_OK;
}

static fb_status upload_ints(BatchWork& B, cudaStream_t s) {
    FB_CUDA(cudaMemcpyAsync(B.dint, B.hint, sizeof(int) * 2 * B.R, cudaMemcpyHostToDevice, s));
    return FB_OK;
}

// Inner lockstep FGMRES on A d_r = rhs_r (r with in[r]) from d = 0.
static fb_status bfgmres_inner(fb_op* A, fb_precond* pc, BatchWork& B, const std::vector<char>& in,
                               const std::vector<double>& rhs_norm, const std::vector<double>& rel_tol,
                               const std::vector<int>& budget, std::vector<int>& iters, std::vector<double>& est_rel,
                               std::vector<int>& status, cudaStream_t s) {
    const int64_t n = B.n;
    const int m = B.m, R = B.R;
    const int gx = std::min(grid_for(n), 64);
    int* act = B.hint;
    int* j1 = B.hint + R;
    int* dact = B.dint;
    int* dj1 = B.dint + R;
    std::vector<char> fin(R, 1);
    for (int r = 0; r < R; ++r) {
        fin[r] = !in[r];
        iters[r] = 0;
        est_rel[r] = 0.0;
        status[r] = FB_OK;
    }
    FB_CUDA(cudaMemsetAsync(B.D, 0, sizeof(cd) * n * R, s));
    std::vector<double> est(R, 0.0);
    bool first = true;
    while (true) {
        for (int r = 0; r < R; ++r) act[r] = !fin[r];
        FB_CHECK(upload_ints(B, s));
        if (first) {
            FB_CUDA(cudaMemcpyAsync(B.W, B.Rs, sizeof(cd) * n * R, cudaMemcpyDeviceToDevice, s));
        } else {
            FB_CHECK(fb_apply_any(A, B.D, B.T, s, R));
            k_bsub<<<dim3(grid_for(n), R), KB, 0, s>>>(B.W, B.Rs, B.T, n, dact);
            cnt();
        }
        first = false;
        FB_CUDA(cudaMemsetAsync(B.scal, 0, sizeof(double) * 4 * R, s));
        k_bnorm2<<<dim3(grid_for(n), R), KB, 0, s>>>(B.W, n, B.scal, 4, dact);
        k_bcycle_start<<<R, 1, 0, s>>>(B.dhs, dact);
        k_bscale<<<dim3(grid_for(n), R), KB, 0, s>>>(B.V, B.W, n, B.scal + 1, 4, dact);
        FB_LAUNCH_CHECK();
        cnt(3);
        FB_CUDA(cudaMemcpyAsync(B.host, B.scal, sizeof(double) * 4 * R, cudaMemcpyDeviceToHost, s));
        FB_CUDA(cudaStreamSynchronize(s));
        bool any = false;
        for (int r = 0; r < R; ++r) {
            j1[r] = 0;
            if (fin[r]) { act[r] = 0; continue; }
            est[r] = B.host[4 * r + 2];
            if (!std::isfinite(est[r])) { status[r] = FB_ERR_NAN; fin[r] = 1; act[r] = 0; continue; }
            if (est[r] <= rel_tol[r] * rhs_norm[r] || iters[r] >= budget[r]) { fin[r] = 1; act[r] = 0; continue; }
            act[r] = 1;
            any = true;
        }
        FB_CHECK(upload_ints(B, s));
        if (!any) break;
        for (int j = 0; j < m; ++j) {
            cd* Vj = B.V + (int64_t)j * R * n;
            cd* Zj = Vj;
            if (pc) {
                Zj = B.Z + (int64_t)j * R * n;
                FB_CHECK(fb_pc_apply(pc, Vj, Zj, s, R));
            }
            FB_CHECK(fb_apply_any(A, Zj, B.W, s, R));
            for (int pass = 0; pass < 2; ++pass) {
                FB_CUDA(cudaMemsetAsync(B.small + (size_t)R * (m + 1) * m, 0, sizeof(cd) * R * (m + 1), s));
                cd* h = B.small + (size_t)R * (m + 1) * m;    // [R][m+1] CGS scratch (Hess.h)
                k_bmdot<<<dim3(gx, j + 1, R), KB, 0, s>>>(B.V, n, R, B.W, h, m + 1, dact);
                k_bgs_update<<<dim3(grid_for(n), R), KB, 0, s>>>(B.V, n, R, j + 1, h, m + 1, B.W, dact);
                k_baccum_h<<<R, 1024, 0, s>>>(B.dhs, j, dact);
                cnt(3);
            }
            FB_CUDA(cudaMemsetAsync(B.scal, 0, sizeof(double) * 4 * R, s));   // active rows are all rewritten
            k_bnorm2<<<dim3(grid_for(n), R), KB, 0, s>>>(B.W, n, B.scal, 4, dact);
            k_barnoldi_close<<<R, 1, 0, s>>>(B.dhs, j, dact);
            k_bscale<<<dim3(grid_for(n), R), KB, 0, s>>>(B.V + (int64_t)(j + 1) * R * n, B.W, n, B.scal + 1, 4, dact);
            FB_LAUNCH_CHECK();
            cnt(3);
            FB_CUDA(cudaMemcpyAsync(B.host, B.scal, sizeof(double) * 4 * R, cudaMemcpyDeviceToHost, s));
            FB_CUDA(cudaStreamSynchronize(s));
            bool changed = false;
            any = false;
            for (int r = 0; r < R; ++r) {
                if (!act[r]) continue;
                double e = B.host[4 * r + 2], hn = B.host[4 * r];
                iters[r]++;
                j1[r] = j + 1;
                est[r] = e;
                bool stop = false;
                if (!std::isfinite(e)) { status[r] = FB_ERR_NAN; fin[r] = 1; stop = true; }
                else if (hn == 0.0 || e <= rel_tol[r] * rhs_norm[r] || iters[r] >= budget[r]) { fin[r] = 1; stop = true; }
                if (stop) { act[r] = 0; changed = true; } else any = true;
            }
            if (!any) break;
            if (changed) FB_CHECK(upload_ints(B, s));
        }
        // x-update of every system that took steps in this cycle (NaN ones excluded)
        for (int r = 0; r < R; ++r) if (status[r] != FB_OK) j1[r] = 0;
        FB_CHECK(upload_ints(B, s));
        k_bbacksolve<<<R, 1, 0, s>>>(B.dhs, dj1);
        cd* ys = B.small + (size_t)R * (m + 1) * m + (size_t)R * (m + 1) * 5;   // Hess.y block
        k_bupdate_x<<<dim3(grid_for(n), R), KB, 0, s>>>(B.D, pc ? B.Z : B.V, n, R, dj1, ys, m + 1);
        FB_LAUNCH_CHECK();
        cnt(2);
        bool all = true;
        for (int r = 0; r < R; ++r) all = all && fin[r];
        if (all) break;
    }
    for (int r = 0; r < R; ++r) est_rel[r] = rhs_norm[r] > 0 ? est[r] / rhs_norm[r] : 0.0;
    return FB_OK;
}

fb_status fb_fgmres_multi_impl(fb_op* A, fb_precond* pc, const cd* b, cd* x, int R, const fb_solver_opts* o,
                               fb_solve_info* info, cudaStream_t s) {
    fb_solver_opts opts = *o;
    if (opts.restart < 1 || opts.restart > 1000) return fb_fail(FB_ERR_ARG, "restart must be in [1, 1000]");
    if (opts.maxit < 1) return fb_fail(FB_ERR_ARG, "maxit must be >= 1");
    if (opts.max_refine < 1) opts.max_refine = 1;
    fb_op* T = opts.true_op ? const_cast<fb_op*>(opts.true_op) : A;
    if (T->n != A->n) return fb_fail(FB_ERR_ARG, "true_op size differs");
    const int64_t n = A->n;
    const int m = opts.restart;
    BatchWork* Bp = nullptr;
    FB_CHECK(bwork_get(A, m, R, pc != nullptr, &Bp));
    BatchWork& B = *Bp;
    std::vector<Hess> hh(R);
    cd* H0 = B.small;
    cd* blk = B.small + (size_t)R * (m + 1) * m;
    for (int r = 0; r < R; ++r) {
        Hess& h = hh[r];
        h.m = m;
        h.H = H0 + (size_t)r * (m + 1) * m;
        h.h = blk + (size_t)0 * R * (m + 1) + (size_t)r * (m + 1);
        h.cs = blk + (size_t)1 * R * (m + 1) + (size_t)r * (m + 1);
        h.sn = blk + (size_t)2 * R * (m + 1) + (size_t)r * (m + 1);
        h.g = blk + (size_t)3 * R * (m + 1) + (size_t)r * (m + 1);
        h.y = blk + (size_t)5 * R * (m + 1) + (size_t)r * (m + 1);
        h.nrm2 = B.scal + 4 * r;
        h.inv = B.scal + 4 * r + 1;
        h.est = B.scal + 4 * r + 2;
    }
    FB_CUDA(cudaMemcpyAsync(B.dhs, hh.data(), sizeof(Hess) * R, cudaMemcpyHostToDevice, s));

    std::vector<fb_solve_info> inf(R);
    for (auto& q : inf) q = fb_solve_info{};
    FB_CUDA(cudaMemsetAsync(x, 0, sizeof(cd) * n * R, s));
    // ||b_r||
    std::vector<double> bn(R), rn(R);
    FB_CUDA(cudaMemsetAsync(B.scal, 0, sizeof(double) * 4 * R, s));
    k_bnorm2<<<dim3(grid_for(n), R), KB, 0, s>>>(b, n, B.scal, 4, nullptr);
    cnt();
    FB_CUDA(cudaMemcpyAsync(B.host, B.scal, sizeof(double) * 4 * R, cudaMemcpyDeviceToHost, s));
    FB_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < R; ++r) rn[r] = bn[r] = std::sqrt(B.host[4 * r]);
    FB_CUDA(cudaMemcpyAsync(B.Rs, b, sizeof(cd) * n * R, cudaMemcpyDeviceToDevice, s));
    const double inner_floor = opts.inner_tol > 0 ? opts.inner_tol : 0.0;
    std::vector<char> in(R);
    std::vector<double> rel(R);
    std::vector<int> budget(R), its(R), st(R);
    std::vector<double> estr(R);
    std::vector<int> status(R, FB_OK);
    for (int sweep = 0; sweep < opts.max_refine; ++sweep) {
        bool any = false;
        for (int r = 0; r < R; ++r) {
            in[r] = status[r] == FB_OK && bn[r] > 0 && rn[r] > opts.tol * bn[r] && inf[r].iters < opts.maxit;
            any = any || in[r];
            rel[r] = in[r] ? std::max(inner_floor, 0.5 * opts.tol * bn[r] / rn[r]) : 0.0;
            budget[r] = opts.maxit - inf[r].iters;
        }
        if (!any) break;
        FB_CHECK(bfgmres_inner(A, pc, B, in, rn, rel, budget, its, estr, st, s));
        for (int r = 0; r < R; ++r) {
            B.hint[r] = in[r] && st[r] == FB_OK;
            B.hint[R + r] = 0;
        }
        FB_CHECK(upload_ints(B, s));
        k_badd<<<dim3(grid_for(n), R), KB, 0, s>>>(x, B.D, n, B.dint);
        cnt();
        // true residuals r = b - T x (all systems, one batched matvec)
        FB_CHECK(fb_apply_any(T, x, B.T, s, R));
        k_bsub<<<dim3(grid_for(n), R), KB, 0, s>>>(B.Rs, b, B.T, n, nullptr);
        FB_CUDA(cudaMemsetAsync(B.scal, 0, sizeof(double) * 4 * R, s));
        k_bnorm2<<<dim3(grid_for(n), R), KB, 0, s>>>(B.Rs, n, B.scal, 4, nullptr);
        FB_LAUNCH_CHECK();
        cnt(2);
        FB_CUDA(cudaMemcpyAsync(B.host, B.scal, sizeof(double) * 4 * R, cudaMemcpyDeviceToHost, s));
        FB_CUDA(cudaStreamSynchronize(s));
        for (int r = 0; r < R; ++r) {
            if (!in[r]) continue;
            inf[r].iters += its[r];
            inf[r].est_relres = estr[r] * rn[r] / bn[r];
            inf[r].refinements = sweep + 1;
            inf[r].true_matvecs++;
            if (st[r] != FB_OK) status[r] = st[r];
            rn[r] = std::sqrt(B.host[4 * r]);
            if (!std::isfinite(rn[r])) status[r] = FB_ERR_NAN;
        }
    }
    fb_status waits = fb_op_wait_status(A);
    if (waits == FB_OK && T != A) waits = fb_op_wait_status(T);
    if (waits == FB_OK && pc && pc->inner_op) waits = fb_op_wait_status(pc->inner_op);
    fb_status worst = FB_OK;
    for (int r = 0; r < R; ++r) {
        if (waits != FB_OK) status[r] = waits;
        inf[r].true_relres = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
        int stt = status[r];
        if (stt == FB_OK && !(inf[r].true_relres <= opts.tol)) stt = FB_ERR_NOCONV;
        inf[r].status = stt;
        if (worst == FB_OK && stt != FB_OK) worst = stt;
        if (info) info[r] = inf[r];
    }
    if (worst != FB_OK)
        fb_set_error(worst, worst == FB_ERR_NOCONV ? "FGMRES (batched): a system did not reach the tolerance"
                                                   : "FGMRES (batched): a system stopped on a non-finite residual");
    return worst;
}

fb_status fb_precond_create_impl(fb_op* op, int kind, cudaStream_t s, fb_precond** out) {
    *out = nullptr;
    if (kind == FB_PC_NONE) return FB_OK;
    if (kind != FB_PC_BLOCK_JACOBI) return fb_fail(FB_ERR_ARG, "unknown preconditioner kind");
    if (op->kind == FB_OP_IBEM) return ibem_bj_create(op, s, out);
    if (op->kind == FB_OP_DBEM5) return dbem5_bj_create(op, s, out);
    if (op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "block Jacobi needs an FMM operator");
    const fb_tree* t = op->tree;
    int nleaf = t->nbox[t->L];
    fb_precond* pc = new fb_precond();
    pc->op = op;
    pc->kind = kind;
    pc->n = op->n;
    std::vector<int64_t> off(nleaf + 1, 0);
    int maxn = 0;
    for (int b = 0; b < nleaf; ++b) {
        int nb = t->h_leaf_start[b + 1] - t->h_leaf_start[b];
        maxn = std::max(maxn, nb);
        off[b + 1] = off[b] + (int64_t)nb * nb;
    }
    int* piv = nullptr;
    int* sing = nullptr;
    auto fail = [&](fb_status st) { dfree(piv); dfree(sing); fb_precond_destroy(pc); return st; };
    fb_status st;
    if ((st = dalloc(&pc->blk_off, nleaf + 1)) || (st = dalloc(&pc->inv64, off[nleaf])) ||
        (st = dalloc(&piv, op->n)) || (st = dalloc(&sing, 1)))
        return fail(st);
    FB_CUDA(cudaMemcpyAsync(pc->blk_off, off.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
    if (op->nf64) FB_CHECK(fb_self_blocks(op, pc->blk_off, pc->inv64, s));
    else FB_CUDA(cudaMemcpyAsync(pc->inv64, op->self64, sizeof(cd) * off[nleaf], cudaMemcpyDeviceToDevice, s));
    FB_CHECK(fb_smem_cap((const void*)k_bj_invert, sizeof(cd) * std::max(maxn, 1)));
    k_bj_invert<<<nleaf, 256, sizeof(cd) * std::max(maxn, 1), s>>>(t->leaf_start, pc->blk_off, pc->inv64, piv, sing, 1);
    int hs = 0;
    FB_CUDA(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
    FB_CUDA(cudaStreamSynchronize(s));
    dfree(piv);
    dfree(sing);
    if (hs) {
        fb_precond_destroy(pc);
        return fb_fail(FB_ERR_BREAKDOWN, "singular leaf block in block-Jacobi setup");
    }
    if (op->prec == FB_PREC_MIXED_FMM) {
        FB_CHECK(dalloc(&pc->inv32, off[nleaf]));
        k_d2f_bj<<<div_up(off[nleaf], 256), 256, 0, s>>>(pc->inv64, pc->inv32, off[nleaf]);
        FB_LAUNCH_CHECK();
    }
    *out = pc;
    return FB_OK;
}

fb_status fb_pc_apply(const fb_precond* pc, const cd* x, cd* y, cudaStream_t s, int nrhs) {
    const int64_t n = pc->n;
    if (pc->kind == FB_PC_INNER) {
        InnerSolver* in = (InnerSolver*)pc->inner;
        auto body = [pc, in, nrhs, n](const cd* gx, cd* gy, cudaStream_t st) -> fb_status {
            if (nrhs == 1) {
                FB_CHECK(gmres_fixed(pc->inner_op, pc->base, in->W, gx, pc->inner_its, st));
                FB_CUDA(cudaMemcpyAsync(gy, in->W.d, sizeof(cd) * n, cudaMemcpyDeviceToDevice, st));
                return FB_OK;
            }
            // several right-hand sides: one lockstep inner solve, multi-RHS matvecs
            InnerBatch* ib = nullptr;
            FB_CHECK(inner_batch_get(in, n, pc->inner_its, nrhs, pc->base != nullptr, &ib));
            FB_CHECK(gmres_fixed_multi(pc->inner_op, pc->base, ib->B, gx, st));
            FB_CUDA(cudaMemcpyAsync(gy, ib->B.D, sizeof(cd) * n * nrhs, cudaMemcpyDeviceToDevice, st));
            return FB_OK;
        };
        if (pc->use_graphs) {
            // the inner steps synchronise nothing: one captured graph per
            // number of right-hand sides, recaptured when the inner operator
            // reallocates buffers the graph refers to
            fb_precond* mpc = const_cast<fb_precond*>(pc);
            return fb_graph_run(mpc->graphs, nrhs, n * nrhs, n * nrhs, x, y, s, body, &pc->inner_op->buf_gen);
        }
        return body(x, y, s);
    }
    if (pc->net) {
        if (pc->use_graphs) {
            fb_precond* mpc = const_cast<fb_precond*>(pc);
            for (int r = 0; r < nrhs; ++r)
                FB_CHECK(fb_graph_run(mpc->graphs, 1, n, n, x + r * n, y + r * n, s,
                                      [mpc](const cd* gx, cd* gy, cudaStream_t st) {
                                          return fb_learned_apply(mpc->net, gx, gy, st);
                                      }));
            return FB_OK;
        }
        for (int r = 0; r < nrhs; ++r) FB_CHECK(fb_learned_apply(pc->net, x + r * n, y + r * n, s));
        return FB_OK;
    }
    const fb_tree* t = pc->op->tree;
    int nleaf = t->nbox[t->L];
    int maxn = 0;
    for (int b = 0; b < nleaf; ++b) maxn = std::max(maxn, t->h_leaf_start[b + 1] - t->h_leaf_start[b]);
    if (pc->ibem) {
        FB_CHECK(fb_smem_cap((const void*)k_ibem_bj_apply, sizeof(cd) * 2 * maxn));
        for (int r = 0; r < nrhs; ++r)
            k_ibem_bj_apply<<<nleaf, 128, sizeof(cd) * 2 * maxn, s>>>(t->leaf_start, t->perm, pc->blk_off, pc->inv64,
                                                                      x + r * n, y + r * n, n / 2);
        FB_LAUNCH_CHECK();
        fb_count_launch(nrhs);
        return FB_OK;
    }
    dim3 g(nleaf, nrhs);
    FB_CHECK(fb_smem_cap(pc->inv32 ? (const void*)k_bj_apply<float> : (const void*)k_bj_apply<double>,
                         (pc->inv32 ? sizeof(cf) : sizeof(cd)) * maxn));
    if (pc->inv32) {
        k_bj_apply<float><<<g, 128, sizeof(cf) * maxn, s>>>(t->leaf_start, t->perm, pc->blk_off, pc->inv32, x, y, n);
    } else {
        k_bj_apply<double><<<g, 128, sizeof(cd) * maxn, s>>>(t->leaf_start, t->perm, pc->blk_off, pc->inv64, x, y, n);
    }
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

void fb_precond_free(fb_precond* pc) {
    if (!pc) return;
    fb_inner_free(pc->inner);
    fb_graph_free(pc->graphs);
    fb_learned_free(pc->net);
    dfree(pc->blk_off);
    dfree(pc->inv64);
    dfree(pc->inv32);
    delete pc;
}
