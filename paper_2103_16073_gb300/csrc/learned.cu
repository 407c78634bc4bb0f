// Learned octree preconditioner: a small hierarchical network over the FMM
// octree that refines block Jacobi, z = BJ(v) + s * N(v / s), used as the
// variable right preconditioner that flexible GMRES admits (Sec. 3.1, Sec. 4:
// FGMRES with a changing preconditioner).  Trained on residual/error pairs
// (r, e = x* - x) logged from plain block-Jacobi solves, loss
// ||z(r) - e||^2 / ||e||^2.
//
// Network (64-wide features, SiLU, weights W as [in x out], Y = X W + b):
//   features f_i = (Re, Im of v_i conj(ph), u_i conj(ph))/s, n_i, 1,
//                  Re, Im beta_i, k delta_L
//                  (u = BJ(v), s = rms of v, ph = unit phase of sum_i v_i,
//                  beta the admittance, k delta_L the wavenumber times the
//                  leaf side; elements in tree order)
//   H0 = silu(F W0 + b0)                                  elements
//   G_L = mean of H0 over each leaf                       leaves
//   G_l = silu(mean of G_{l+1} over children W_up,k + b)  3 coarser levels
//   D_{L-3} = G_{L-3};  D_l = silu([G_l, D_{l-1}(parent)] W_dn,k + b)
//   H1 = silu([H0, D_L(leaf)] W_h + b_h),  O = H1 W_o + b_o (Re, Im)
//   z_i = u_i + s ph (O_i0 + i O_i1)
// so N(a v) = a N(v) for any complex a, as for a linear preconditioner.
// All GEMMs run on the tensor cores as BF16 x BF16 -> FP32 (mma.sync
// m16n8k16) with FP32 activations rounded to BF16 while staging; master
// weights, gradients and Adam moments are FP32.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int HW = 64;       // feature width
constexpr int NF = 11;       // element input features
constexpr int DEPTH = 3;     // coarser levels above the leaves

// ---------------------------------------------------------------- GEMM ----
// C[M x N] (+)= A[M x K] B[K x N] with arbitrary strides, BF16 operands,
// FP32 accumulation.  Epilogue: optional bias (per column) and SiLU; writes
// the pre-activation to Cpre and the activation to C.
struct GemmArgs {
    const float* A; int64_t a_m, a_k;
    const float* B; int64_t b_k, b_n;
    float* C; int64_t c_m, c_n;
    float* Cpre;                 // pre-activation (may be null)
    const float* bias;           // per column (may be null)
    int M, N, K;
    int act;                     // 0 none, 1 SiLU
    int accumulate;              // C += result
    int kchunk;                  // split-K: K range per blockIdx.z (multiple of 16); 0 = whole K
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float silu(float x) { return x / (1.f + __expf(-x)); }
__device__ __forceinline__ float silu_grad(float x) {
    float sg = 1.f / (1.f + __expf(-x));
    return sg * (1.f + x * (1.f - sg));
}

// 128 threads: 4 warps x 16 rows = 64 rows; 64 columns (8 n-tiles of 8).
__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
    __shared__ uint32_t As[64][8 + 1];   // [row][k pair], 16 k per stage
    __shared__ uint32_t Bs[64][8 + 1];   // [col][k pair]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    const int kb = g.kchunk ? blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk ? min(g.K, kb + g.kchunk) : g.K;
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int i = threadIdx.x; i < 64 * 8; i += blockDim.x) {
            int r = i >> 3, kp = i & 7;
            int m = m0 + r, k = k0 + 2 * kp;
            float x0 = 0.f, x1 = 0.f;
            if (m < g.M) {
                if (k < ke) x0 = g.A[m * g.a_m + k * g.a_k];
                if (k + 1 < ke) x1 = g.A[m * g.a_m + (k + 1) * g.a_k];
            }
            As[r][kp] = pack_bf16(x0, x1);
            int n = n0 + r;
            float y0 = 0.f, y1 = 0.f;
            if (n < g.N) {
                if (k < ke) y0 = g.B[k * g.b_k + n * g.b_n];
                if (k + 1 < ke) y1 = g.B[(k + 1) * g.b_k + n * g.b_n];
            }
            Bs[r][kp] = pack_bf16(y0, y1);
        }
        __syncthreads();
        const int row = warp * 16 + (lane >> 2);
        const int kq = lane & 3;
        uint32_t a0 = As[row][kq], a1 = As[row + 8][kq], a2 = As[row][kq + 4], a3 = As[row + 8][kq + 4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int col = t * 8 + (lane >> 2);
            uint32_t b0 = Bs[col][kq], b1 = Bs[col][kq + 4];
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
        __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int m = m0 + warp * 16 + (lane >> 2) + (q >> 1) * 8;
            int n = n0 + t * 8 + (lane & 3) * 2 + (q & 1);
            if (m >= g.M || n >= g.N) continue;
            float v = acc[t][q];
            float* c = g.C + m * g.c_m + n * g.c_n;
            if (g.kchunk) {              // split-K partial sum (plain accumulation only)
                atomicAdd(c, v);
                continue;
            }
            if (g.bias) v += g.bias[n];
            if (g.accumulate) v += *c;
            if (g.Cpre) g.Cpre[m * g.c_m + n * g.c_n] = v;
            *c = g.act ? silu(v) : v;
        }
}

// --------------------------------------------------------------- helpers ----
// Input statistics: st[0] += sum |v|^2, st[3..4] += sum v (complex).  The
// scale s = rms(v) and the phase of sum v normalise the input, so that the
// network's map is complex-homogeneous: N(a v) = a N(v) for every complex a.
__global__ void k_stats(const cd* v, int64_t n, double* st) {
    __shared__ double sh[3][32];
    double a = 0.0, cr = 0.0, ci = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        cd x = v[i];
        a += abs2(x);
        cr += x.re;
        ci += x.im;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        cr += __shfl_xor_sync(0xffffffffu, cr, o);
        ci += __shfl_xor_sync(0xffffffffu, ci, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a;
        sh[1][threadIdx.x >> 5] = cr;
        sh[2][threadIdx.x >> 5] = ci;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        bool in = threadIdx.x < (blockDim.x >> 5);
        a = in ? sh[0][threadIdx.x] : 0.0;
        cr = in ? sh[1][threadIdx.x] : 0.0;
        ci = in ? sh[2][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            cr += __shfl_xor_sync(0xffffffffu, cr, o);
            ci += __shfl_xor_sync(0xffffffffu, ci, o);
        }
        if (threadIdx.x == 0) {
            atomicAdd(&st[0], a);
            atomicAdd(&st[3], cr);
            atomicAdd(&st[4], ci);
        }
    }
}

// unit phase of sum v (1 when the sum vanishes)
__device__ __forceinline__ cd input_phase(const double* st) {
    double m = hypot(st[3], st[4]);
    return m > 0.0 ? mk(st[3] / m, st[4] / m) : mk(1.0, 0.0);
}

// features in tree order: (v, u) rotated by the conjugate input phase and
// divided by s
__global__ void k_features(Geom g, const int32_t* perm, const cd* v, const cd* u, const double* st,
                           int64_t n, float kd, float* F) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= n) return;
    double s = sqrt(st[0] / (double)n);
    double inv = s > 0.0 ? 1.0 / s : 0.0;
    cd ph = input_phase(st);
    cd rot = mk(ph.re * inv, -ph.im * inv);
    int64_t e = perm[pos];
    cd vv = v[e] * rot, uu = u[e] * rot;
    float* f = F + pos * NF;
    f[0] = (float)vv.re;
    f[1] = (float)vv.im;
    f[2] = (float)uu.re;
    f[3] = (float)uu.im;
    f[4] = (float)g.nx[e];
    f[5] = (float)g.ny[e];
    f[6] = (float)g.nz[e];
    f[7] = 1.f;
    f[8] = (float)g.beta[e].re;
    f[9] = (float)g.beta[e].im;
    f[10] = kd;
}

// mean of rows [start[s], start[s+1]) of X (width HW) -> Y[s]
__global__ void k_segmean(const float* X, const int32_t* start, int nseg, float* Y) {
    int sgi = blockIdx.x;
    int c = threadIdx.x;
    if (sgi >= nseg || c >= HW) return;
    int a = start[sgi], b = start[sgi + 1];
    float acc = 0.f;
    for (int i = a; i < b; ++i) acc += X[(int64_t)i * HW + c];
    Y[(int64_t)sgi * HW + c] = b > a ? acc / (float)(b - a) : 0.f;
}
// backward: dX[i] += dY[seg(i)] / count
__global__ void k_segmean_back(const float* dY, const int32_t* start, int nseg, float* dX) {
    int sgi = blockIdx.x;
    int c = threadIdx.x;
    if (sgi >= nseg || c >= HW) return;
    int a = start[sgi], b = start[sgi + 1];
    if (b <= a) return;
    float d = dY[(int64_t)sgi * HW + c] / (float)(b - a);
    for (int i = a; i < b; ++i) dX[(int64_t)i * HW + c] += d;
}

// C[i] = [X[i], Y[idx[i]]]  (widths HW + HW)
__global__ void k_concat(const float* X, const float* Y, const int32_t* idx, int64_t rows, float* C) {
    int64_t i = blockIdx.x;
    int c = threadIdx.x;
    if (i >= rows) return;
    if (c < HW) C[i * 2 * HW + c] = X[i * HW + c];
    else C[i * 2 * HW + c] = Y[(int64_t)idx[i] * HW + (c - HW)];
}
// backward of k_concat: dX[i] += dC[i][:HW], dY[idx[i]] += dC[i][HW:] (atomic)
__global__ void k_concat_back(const float* dC, const int32_t* idx, int64_t rows, float* dX, float* dY) {
    int64_t i = blockIdx.x;
    int c = threadIdx.x;
    if (i >= rows) return;
    if (c < HW) dX[i * HW + c] += dC[i * 2 * HW + c];
    else atomicAdd(&dY[(int64_t)idx[i] * HW + (c - HW)], dC[i * 2 * HW + c]);
}

__global__ void k_add_f(float* dst, const float* src, int64_t count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) dst[i] += src[i];
}

__global__ void k_silu_back(const float* dA, const float* pre, int64_t count, float* dP) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) dP[i] = dA[i] * silu_grad(pre[i]);
}

// column sums (bias gradients): out[c] += sum_r X[r][c]
__global__ void k_colsum(const float* X, int64_t rows, int cols, float* out) {
    int c = blockIdx.y;
    float a = 0.f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        a += X[r * cols + c];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[c], a);
}

// z (element order) = u + s ph (O0 + i O1)
__global__ void k_output(const int32_t* perm, const cd* u, const float* O, const double* st, int64_t n, cd* z) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= n) return;
    double s = sqrt(st[0] / (double)n);
    cd ph = input_phase(st);
    int64_t e = perm[pos];
    cd o = mk(s * (double)O[pos * 2], s * (double)O[pos * 2 + 1]) * ph;
    z[e] = u[e] + o;
}

// loss pieces: sum |z - e|^2, sum |e|^2; dO = 2 s (z - e) / ||e||^2 (tree order)
__global__ void k_loss_sums(const cd* z, const cd* e, int64_t n, double* sums) {
    __shared__ double s0[32], s1[32];
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        cd d = z[i] - e[i];
        a += abs2(d);
        b += abs2(e[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { s0[threadIdx.x >> 5] = a; s1[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < (blockDim.x >> 5) ? s0[threadIdx.x] : 0.0;
        b = threadIdx.x < (blockDim.x >> 5) ? s1[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (threadIdx.x == 0) { atomicAdd(&sums[0], a); atomicAdd(&sums[1], b); }
    }
}
// dO = 2 s conj(ph) (z - e) / ||e||^2 as (Re, Im), tree order
__global__ void k_loss_grad(const int32_t* perm, const cd* z, const cd* e, const double* st, const double* sums,
                            int64_t n, double scale, float* dO) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= n) return;
    double s = sqrt(st[0] / (double)n);
    cd ph = input_phase(st);
    int64_t i = perm[pos];
    double f = scale * 2.0 * s / sums[1];
    cd d = (z[i] - e[i]) * mk(f * ph.re, -f * ph.im);
    dO[pos * 2] = (float)d.re;
    dO[pos * 2 + 1] = (float)d.im;
}

// Residual objective.  yc = conj((A z - r) / area)
__global__ void k_adj_prep(const cd* az, const cd* r, const double* area, int64_t n, cd* yc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd w = az[i] - r[i];
    double ia = 1.0 / area[i];
    yc[i] = mk(w.re * ia, -w.im * ia);
}
// g = w/2 + a conj(t1) + i k conj(beta) a conj(t2)  (t1 = L' yc, t2 = L yc),
// the stand-in adjoint applied to w = A z - r; dO = 2 s conj(ph) g / ||r||^2
__global__ void k_adj_grad(const int32_t* perm, const cd* az, const cd* r, const cd* t1, const cd* t2,
                           const double* area, const cd* beta, double k, const double* st, const double* sums,
                           int64_t n, double scale, float* dO) {
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= n) return;
    double s = sqrt(st[0] / (double)n);
    cd ph = input_phase(st);
    int64_t i = perm[pos];
    cd w = az[i] - r[i];
    double a = area[i];
    cd c1 = mk(a * t1[i].re, -a * t1[i].im);
    cd c2 = mk(a * t2[i].re, -a * t2[i].im);
    cd ikb = mk(k * beta[i].im, k * beta[i].re);      // i k conj(beta)
    cd g = mk(0.5 * w.re, 0.5 * w.im) + c1 + ikb * c2;
    double f = scale * 2.0 * s / sums[1];
    cd d = g * mk(f * ph.re, -f * ph.im);
    dO[pos * 2] = (float)d.re;
    dO[pos * 2 + 1] = (float)d.im;
}

__global__ void k_adam(float* w, const float* gr, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = gr[i];
    float mi = b1 * m[i] + (1.f - b1) * g;
    float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Packed BF16 copies of the 64-column weight matrices for the inference
// kernels: W (K x 64, K = 64 or 128) -> P[n][kp] = (W[2kp][n], W[2kp+1][n]),
// so a CTA stages a layer's weights with 16-byte loads.  Rebuilt after every
// parameter change (initialisation, upload, Adam step).
__global__ void k_pack_w(const float* __restrict__ W, int K, uint32_t* __restrict__ P) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int KP = K / 2;
    if (i >= HW * KP) return;
    int n = i / KP, kp = i % KP;
    P[i] = pack_bf16(W[(2 * kp) * HW + n], W[(2 * kp + 1) * HW + n]);
}

// Stages a packed K x 64 weight block into shared memory rows of KP + 4 words.
template <int KP>
__device__ __forceinline__ void stage_w(const uint32_t* __restrict__ P, uint32_t (*Ws)[KP + 4], int tid, int nth) {
    constexpr int V = KP / 4;   // uint4 per row
    for (int i = tid; i < HW * V; i += nth) {
        int n = i / V, q = i % V;
        uint4 x = reinterpret_cast<const uint4*>(P + n * KP)[q];
        Ws[n][4 * q] = x.x;
        Ws[n][4 * q + 1] = x.y;
        Ws[n][4 * q + 2] = x.z;
        Ws[n][4 * q + 3] = x.w;
    }
}

// ------------------------------------------------ fused inference path ----
// Applying the trained network inside FGMRES needs no activations for a
// backward pass, so the element-level layers run fused: pass 1 computes the
// element encoder H0 and its leaf means in one CTA per leaf; pass 2
// recomputes H0 per 64-element tile, joins it with the leaf's down-sweep
// feature, runs the W_h layer on the tensor cores (mma.sync BF16, FP32
// accumulation) and the W_o layer and the output z = u + s ph O in
// registers.  Operands are rounded to BF16 where the training path rounds
// them, so both evaluate the same network.
__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void elem_features(const Geom& g, const int32_t* perm, const cd* v, const cd* u,
                                              const double* st, int64_t n, float kd, int64_t pos, float f[NF]) {
    double s = sqrt(st[0] / (double)n);
    double inv = s > 0.0 ? 1.0 / s : 0.0;
    cd ph = input_phase(st);
    cd rot = mk(ph.re * inv, -ph.im * inv);
    int64_t e = perm[pos];
    cd vv = v[e] * rot, uu = u[e] * rot;
    f[0] = bfr((float)vv.re);
    f[1] = bfr((float)vv.im);
    f[2] = bfr((float)uu.re);
    f[3] = bfr((float)uu.im);
    f[4] = bfr((float)g.nx[e]);
    f[5] = bfr((float)g.ny[e]);
    f[6] = bfr((float)g.nz[e]);
    f[7] = 1.f;
    f[8] = bfr((float)g.beta[e].re);
    f[9] = bfr((float)g.beta[e].im);
    f[10] = bfr(kd);
}

// G_L[leaf][c] = mean over the leaf's elements of silu(F W0 + b0)[c]; one CTA
// of 64 threads (one per feature column) per leaf.
__global__ void __launch_bounds__(64) k_inf_pass1(Geom g, const int32_t* perm, const int32_t* leaf_start,
                                                  const cd* v, const cd* u, const double* st, int64_t n,
                                                  float kd, const float* W0, const float* b0, float* GL) {
    int leaf = blockIdx.x, c = threadIdx.x;
    int a = leaf_start[leaf], b = leaf_start[leaf + 1];
    float w[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) w[k] = bfr(W0[k * HW + c]);
    float bias = b0[c];
    __shared__ float fs[64][NF];
    float acc = 0.f;
    for (int e0 = a; e0 < b; e0 += 64) {
        int cnt = min(64, b - e0);
        __syncthreads();
        if (c < cnt) {
            float f[NF];
            elem_features(g, perm, v, u, st, n, kd, e0 + c, f);
#pragma unroll
            for (int k = 0; k < NF; ++k) fs[c][k] = f[k];
        }
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            float h = bias;
#pragma unroll
            for (int k = 0; k < NF; ++k) h = fmaf(fs[i][k], w[k], h);
            acc += silu(h);
        }
    }
    GL[(int64_t)leaf * HW + c] = b > a ? acc / (float)(b - a) : 0.f;
}

// 64 elements per CTA (tree order), 256 threads = 8 warps: warp w computes
// rows 16 (w & 3) .. +16 and the 32 columns 32 (w >> 2) .. +32 of H1.
__global__ void __launch_bounds__(256) k_inf_pass2(Geom g, const int32_t* perm, const int32_t* leaf_of,
                                                   const cd* v, const cd* u, const double* st, int64_t n,
                                                   float kd, const float* W0, const float* b0, const float* DL,
                                                   const uint32_t* Whp, const float* bh, const float* Wo,
                                                   const float* bo, cd* z) {
    __shared__ __align__(16) uint32_t Es[64][HW + 4];   // [row][k pair]: 128 bf16 per row (+pad)
    __shared__ __align__(16) uint32_t Ws[HW][HW + 4];   // W_h as [col n][k pair]
    __shared__ float fs[64][NF];
    __shared__ float w0s[NF][HW];
    __shared__ float opart[2][64][2];                  // output partial sums per column half
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    for (int i = tid; i < NF * HW; i += blockDim.x) w0s[i / HW][i % HW] = bfr(W0[i]);
    stage_w<HW>(Whp, Ws, tid, blockDim.x);   // W_h [128 x 64] packed as [n][k pair]
    if (tid < 64) {
        int64_t pos = r0 + tid;
        float f[NF];
        if (pos < n) elem_features(g, perm, v, u, st, n, kd, pos, f);
        else
            for (int k = 0; k < NF; ++k) f[k] = 0.f;
        for (int k = 0; k < NF; ++k) fs[tid][k] = f[k];
    }
    __syncthreads();
    // E = [H0, D_L(leaf)] as bf16 pairs: H0 pairs, then D_L in 4-float pieces
    for (int i = tid; i < 64 * (HW / 2); i += blockDim.x) {
        int r = i / (HW / 2), kp = i % (HW / 2);
        int c0 = 2 * kp;
        float x0 = 0.f, x1 = 0.f;
        if (r0 + r < n) {
            float h0 = b0[c0], h1 = b0[c0 + 1];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                h0 = fmaf(fs[r][k], w0s[k][c0], h0);
                h1 = fmaf(fs[r][k], w0s[k][c0 + 1], h1);
            }
            x0 = silu(h0);
            x1 = silu(h1);
        }
        Es[r][kp] = pack_bf16(x0, x1);
    }
    for (int i = tid; i < 64 * (HW / 4); i += blockDim.x) {
        int r = i / (HW / 4), q = i % (HW / 4);
        int64_t pos = r0 + r;
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pos < n) d = reinterpret_cast<const float4*>(DL + (int64_t)leaf_of[pos] * HW)[q];
        Es[r][HW / 2 + 2 * q] = pack_bf16(d.x, d.y);
        Es[r][HW / 2 + 2 * q + 1] = pack_bf16(d.z, d.w);
    }
    __syncthreads();
    // H1 = silu(E W_h + b_h)
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    const int row = (warp & 3) * 16 + (lane >> 2), kq = lane & 3;
    const int half = warp >> 2, cbase = half * 32;
#pragma unroll
    for (int k0 = 0; k0 < 2 * HW; k0 += 16) {
        int kb = k0 / 2;
        uint32_t a0 = Es[row][kb + kq], a1 = Es[row + 8][kb + kq], a2 = Es[row][kb + kq + 4],
                 a3 = Es[row + 8][kb + kq + 4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int col = cbase + t * 8 + (lane >> 2);
            uint32_t b0r = Ws[col][kb + kq], b1r = Ws[col][kb + kq + 4];
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0r), "r"(b1r));
        }
    }
    // O = H1 W_o + b_o over this warp's 32 columns; rows (lane >> 2) and +8
    float o[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int col = cbase + t * 8 + (lane & 3) * 2 + (q & 1);
            float h = bfr(silu(acc[t][q] + bh[col]));
            int hr = q >> 1;
            o[hr][0] = fmaf(h, bfr(Wo[col * 2]), o[hr][0]);
            o[hr][1] = fmaf(h, bfr(Wo[col * 2 + 1]), o[hr][1]);
        }
#pragma unroll
    for (int hr = 0; hr < 2; ++hr)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            o[hr][j] += __shfl_xor_sync(0xffffffffu, o[hr][j], 1);
            o[hr][j] += __shfl_xor_sync(0xffffffffu, o[hr][j], 2);
        }
    if ((lane & 3) == 0) {
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {
            opart[half][row + hr * 8][0] = o[hr][0];
            opart[half][row + hr * 8][1] = o[hr][1];
        }
    }
    __syncthreads();
    if (tid < 64) {
        int64_t pos = r0 + tid;
        if (pos < n) {
            double sc = sqrt(st[0] / (double)n);
            cd ph = input_phase(st);
            float oa = opart[0][tid][0] + opart[1][tid][0] + bo[0];
            float ob = opart[0][tid][1] + opart[1][tid][1] + bo[1];
            int64_t e = perm[pos];
            z[e] = u[e] + mk(sc * (double)oa, sc * (double)ob) * ph;
        }
    }
}

// One coarse layer of the inference path, fused: rows b of a level (64 per
// CTA) gather their input, Y[b] = silu(X[b] W + bias), W (K x 64, K = 64 or
// 128) staged once per CTA as BF16, X rounded to BF16, FP32 accumulation.
//   mode 0 (up-sweep):   X[b] = mean of Gc[c], c in [cs[b], cs[b+1])        (K = 64)
//   mode 1 (down-sweep): X[b] = [G[b], Dp[parent[b]]]                        (K = 128)
template <int K>
__global__ void __launch_bounds__(256) k_inf_layer(int mode, int M, const float* __restrict__ G,
                                                   const int32_t* __restrict__ idx, const float* __restrict__ Dp,
                                                   const uint32_t* __restrict__ Wp, const float* __restrict__ bias,
                                                   float* __restrict__ Y) {
    // 32 rows per CTA, 8 warps: warp w computes rows 16 (w & 1) .. +16 and the
    // 16 columns 16 (w >> 1) .. +16 (two n-tiles of 8)
    constexpr int KP = K / 2;
    constexpr int ROWS = 32;
    __shared__ __align__(16) uint32_t Xs[ROWS][KP + 4];
    __shared__ __align__(16) uint32_t Ws[HW][KP + 4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b0 = blockIdx.x * ROWS;
    stage_w<KP>(Wp, Ws, tid, blockDim.x);
    // X rows in 4-float pieces (row-major feature arrays are 16-byte aligned)
    constexpr int Q = K / 4;
    for (int i = tid; i < ROWS * Q; i += blockDim.x) {
        int r = i / Q, q = i % Q;
        int b = b0 + r;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b < M) {
            if (mode == 0) {
                int c0 = idx[b], c1 = idx[b + 1];
                float4 y[8];
#pragma unroll
                for (int c = 0; c < 8; ++c)   // an octree box has at most 8 children
                    y[c] = c0 + c < c1 ? reinterpret_cast<const float4*>(G + (int64_t)(c0 + c) * HW)[q]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    x.x += y[c].x; x.y += y[c].y; x.z += y[c].z; x.w += y[c].w;
                }
                float inv = c1 > c0 ? 1.f / (float)(c1 - c0) : 0.f;
                x.x *= inv; x.y *= inv; x.z *= inv; x.w *= inv;
            } else if (q < HW / 4) {
                x = reinterpret_cast<const float4*>(G + (int64_t)b * HW)[q];
            } else {
                x = reinterpret_cast<const float4*>(Dp + (int64_t)idx[b] * HW)[q - HW / 4];
            }
        }
        Xs[r][2 * q] = pack_bf16(x.x, x.y);
        Xs[r][2 * q + 1] = pack_bf16(x.z, x.w);
    }
    __syncthreads();
    float acc[2][4];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    const int row = (warp & 1) * 16 + (lane >> 2), kq = lane & 3;
    const int cbase = (warp >> 1) * 16;
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        int kb = k0 / 2;
        uint32_t a0 = Xs[row][kb + kq], a1 = Xs[row + 8][kb + kq], a2 = Xs[row][kb + kq + 4],
                 a3 = Xs[row + 8][kb + kq + 4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            int col = cbase + t * 8 + (lane >> 2);
            uint32_t b0r = Ws[col][kb + kq], b1r = Ws[col][kb + kq + 4];
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0r), "r"(b1r));
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int b = b0 + row + (q >> 1) * 8;
            int col = cbase + t * 8 + (lane & 3) * 2 + (q & 1);
            if (b < M) Y[(int64_t)b * HW + col] = silu(acc[t][q] + bias[col]);
        }
}

}  // namespace

// ------------------------------------------------------------------ host ----
// Parameter layout (FP32, one flat array):
//   W0 [8 x 64], b0 [64], Wu[k] [64 x 64], bu[k] [64] (k = 0..2),
//   Wd[k] [128 x 64], bd[k] [64] (k = 0..2), Wh [128 x 64], bh [64], Wo [64 x 2], bo [2]
struct LearnedNet {
    const fb_op* op = nullptr;
    const fb_precond* bj = nullptr;
    int L = 0, depth = 0;
    int64_t n = 0;
    float kd = 0.f;                          // k times the leaf side (input feature)
    int64_t nparam = 0;
    int64_t oW0, ob0, oWu[DEPTH], obu[DEPTH], oWd[DEPTH], obd[DEPTH], oWh, obh, oWo, obo;
    float *w = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    uint32_t* wpk = nullptr;                 // packed BF16 weights for inference
    int64_t pWu[DEPTH], pWd[DEPTH], pWh;     // offsets in wpk
    int64_t adam_t = 0;
    // activations (tree order)
    float *F = nullptr, *pre0 = nullptr, *H0 = nullptr, *E = nullptr, *preh = nullptr, *H1 = nullptr, *O = nullptr;
    float* G[FB_MAXLEV + 1] = {nullptr};
    float* Pm[FB_MAXLEV + 1] = {nullptr};
    float* preu[FB_MAXLEV + 1] = {nullptr};
    float* D[FB_MAXLEV + 1] = {nullptr};
    float* Cc[FB_MAXLEV + 1] = {nullptr};
    float* pred[FB_MAXLEV + 1] = {nullptr};
    // gradients of activations
    float *dH0 = nullptr, *dE = nullptr, *dH1 = nullptr, *dO = nullptr, *dtmp = nullptr;
    float* dG[FB_MAXLEV + 1] = {nullptr};
    float* dD[FB_MAXLEV + 1] = {nullptr};
    float* dC[FB_MAXLEV + 1] = {nullptr};
    float* dPm[FB_MAXLEV + 1] = {nullptr};
    int32_t* child_start[FB_MAXLEV + 1] = {nullptr};   // children of box b at level l: [cs[b], cs[b+1]) at level l+1
    int32_t* leaf_of = nullptr;                         // tree position -> leaf
    cd *u = nullptr, *z = nullptr;
    double* scal = nullptr;    // [0] sum |v|^2, [1..2] loss sums, [3..4] sum v
    // residual objective: single- and adjoint-double-layer operators (mixed
    // FMM, built on first use) for the stand-in adjoint, and work vectors
    int objective = FB_LOSS_RESIDUAL;
    fb_op *opL = nullptr, *opLP = nullptr;
    cd *az = nullptr, *yc = nullptr, *t1 = nullptr, *t2 = nullptr;
};

static void gemm(cudaStream_t s, const float* A, int64_t am, int64_t ak, const float* B, int64_t bk, int64_t bn,
                 float* C, int64_t cm, int64_t cn, int M, int N, int K, const float* bias = nullptr,
                 float* Cpre = nullptr, int act = 0, int accumulate = 0) {
    if (M <= 0 || N <= 0) return;
    GemmArgs g{A, am, ak, B, bk, bn, C, cm, cn, Cpre, bias, M, N, K, act, accumulate, 0};
    dim3 grid(div_up(M, 64), div_up(N, 64));
    // Long reductions into few output tiles (weight gradients, K = elements
    // or boxes): split K over blockIdx.z and add the partial sums atomically.
    const int tiles = (int)(grid.x * grid.y);
    if (accumulate && !bias && !act && !Cpre && K > 1024 && tiles < 256) {
        int splits = std::min(div_up(K, 512), std::max(1, 1024 / tiles));
        g.kchunk = div_up(div_up(K, splits), 16) * 16;
        grid.z = div_up(K, g.kchunk);
    }
    k_gemm_bf16<<<grid, 128, 0, s>>>(g);
    fb_count_launch();
}

__global__ void k_child_start(const int32_t* parent, int nchild, int nparent, int32_t* cs) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nparent) return;
    // first child whose parent index >= p (children are sorted by parent)
    int lo = 0, hi = nchild;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (parent[mid] < p) lo = mid + 1; else hi = mid;
    }
    cs[p] = lo;
}
__global__ void k_leaf_of_pos(const int32_t* leaf_start, int nleaf, int32_t* leaf_of) {
    int b = blockIdx.x;
    if (b >= nleaf) return;
    for (int i = leaf_start[b] + threadIdx.x; i < leaf_start[b + 1]; i += blockDim.x) leaf_of[i] = b;
}

fb_status fb_learned_alloc(LearnedNet*& net, const fb_op* op, const fb_precond* bj, cudaStream_t s) {
    const fb_tree* t = op->tree;
    net = new LearnedNet();
    net->op = op;
    net->bj = bj;
    net->L = t->L;
    net->depth = std::min(DEPTH, t->L);
    net->n = op->n;
    net->kd = (float)(op->k * t->side / (double)(1 << t->L));
    int64_t o = 0;
    auto take = [&](int64_t c) { int64_t r = o; o += c; return r; };
    net->oW0 = take(NF * HW);
    net->ob0 = take(HW);
    for (int k = 0; k < DEPTH; ++k) { net->oWu[k] = take(HW * HW); net->obu[k] = take(HW); }
    for (int k = 0; k < DEPTH; ++k) { net->oWd[k] = take(2 * HW * HW); net->obd[k] = take(HW); }
    net->oWh = take(2 * HW * HW);
    net->obh = take(HW);
    net->oWo = take(HW * 2);
    net->obo = take(2);
    net->nparam = o;
    int64_t n = net->n;
    FB_CHECK(dalloc(&net->w, o));
    FB_CHECK(dalloc(&net->grad, o));
    FB_CHECK(dalloc(&net->m1, o));
    FB_CHECK(dalloc(&net->m2, o));
    {   // packed inference weights: Wu_k (64 x 32 words), Wd_k and Wh (64 x 64 words)
        int64_t q = 0;
        for (int k = 0; k < DEPTH; ++k) { net->pWu[k] = q; q += HW * (HW / 2); }
        for (int k = 0; k < DEPTH; ++k) { net->pWd[k] = q; q += HW * HW; }
        net->pWh = q;
        q += HW * HW;
        FB_CHECK(dalloc(&net->wpk, q));
    }
    FB_CUDA(cudaMemsetAsync(net->m1, 0, sizeof(float) * o, s));
    FB_CUDA(cudaMemsetAsync(net->m2, 0, sizeof(float) * o, s));
    FB_CHECK(dalloc(&net->F, n * NF));
    FB_CHECK(dalloc(&net->pre0, n * HW));
    FB_CHECK(dalloc(&net->H0, n * HW));
    FB_CHECK(dalloc(&net->E, n * 2 * HW));
    FB_CHECK(dalloc(&net->preh, n * HW));
    FB_CHECK(dalloc(&net->H1, n * HW));
    FB_CHECK(dalloc(&net->O, n * 2));
    FB_CHECK(dalloc(&net->dH0, n * HW));
    FB_CHECK(dalloc(&net->dE, n * 2 * HW));
    FB_CHECK(dalloc(&net->dH1, n * HW));
    FB_CHECK(dalloc(&net->dO, n * 2));
    FB_CHECK(dalloc(&net->dtmp, n * 2 * HW));
    int L = net->L;
    for (int l = L - net->depth; l <= L; ++l) {
        int64_t nb = t->nbox[l];
        FB_CHECK(dalloc(&net->G[l], nb * HW));
        FB_CHECK(dalloc(&net->D[l], nb * HW));
        FB_CHECK(dalloc(&net->dG[l], nb * HW));
        FB_CHECK(dalloc(&net->dD[l], nb * HW));
        if (l < L) {
            FB_CHECK(dalloc(&net->Pm[l], nb * HW));
            FB_CHECK(dalloc(&net->preu[l], nb * HW));
            FB_CHECK(dalloc(&net->dPm[l], nb * HW));
            FB_CHECK(dalloc(&net->child_start[l], nb + 1));
            k_child_start<<<div_up(nb + 1, 128), 128, 0, s>>>(t->parent[l + 1], t->nbox[l + 1], (int)nb,
                                                              net->child_start[l]);
        }
        if (l > L - net->depth) {
            FB_CHECK(dalloc(&net->Cc[l], nb * 2 * HW));
            FB_CHECK(dalloc(&net->pred[l], nb * HW));
            FB_CHECK(dalloc(&net->dC[l], nb * 2 * HW));
        }
    }
    FB_CHECK(dalloc(&net->leaf_of, n));
    k_leaf_of_pos<<<t->nbox[L], 64, 0, s>>>(t->leaf_start, t->nbox[L], net->leaf_of);
    FB_CHECK(dalloc(&net->u, n));
    FB_CHECK(dalloc(&net->z, n));
    FB_CHECK(dalloc(&net->scal, 8));
    FB_LAUNCH_CHECK();
    return FB_OK;
}

void fb_learned_free(LearnedNet*& net) {
    if (!net) return;
    float** fl[] = {&net->w, &net->grad, &net->m1, &net->m2, &net->F, &net->pre0, &net->H0, &net->E, &net->preh,
                    &net->H1, &net->O, &net->dH0, &net->dE, &net->dH1, &net->dO, &net->dtmp};
    for (auto p : fl) dfree(*p);
    dfree(net->wpk);
    for (int l = 0; l <= FB_MAXLEV; ++l) {
        dfree(net->G[l]); dfree(net->Pm[l]); dfree(net->preu[l]); dfree(net->D[l]); dfree(net->Cc[l]);
        dfree(net->pred[l]); dfree(net->dG[l]); dfree(net->dD[l]); dfree(net->dC[l]); dfree(net->dPm[l]);
        dfree(net->child_start[l]);
    }
    dfree(net->leaf_of);
    dfree(net->u);
    dfree(net->z);
    dfree(net->scal);
    dfree(net->az); dfree(net->yc); dfree(net->t1); dfree(net->t2);
    fb_operator_destroy(net->opL);
    fb_operator_destroy(net->opLP);
    delete net;
    net = nullptr;
}

// Forward: v (element order, device) -> z = BJ(v) + s N(v/s).
fb_status fb_learned_forward(LearnedNet* net, const cd* v, cd* z, cudaStream_t s) {
    const fb_tree* t = net->op->tree;
    const Geom& g = net->op->mesh->g;
    int L = net->L, Ltop = L - net->depth;
    int64_t n = net->n;
    int nleaf = t->nbox[L];
    FB_CHECK(fb_pc_apply(net->bj, v, net->u, s));
    FB_CUDA(cudaMemsetAsync(net->scal, 0, 8 * sizeof(double), s));
    k_stats<<<std::min<int64_t>(div_up(n, 256), 1024), 256, 0, s>>>(v, n, net->scal);
    k_features<<<div_up(n, 256), 256, 0, s>>>(g, t->perm, v, net->u, net->scal, n, net->kd, net->F);
    fb_count_launch(2);
    const float* w = net->w;
    gemm(s, net->F, NF, 1, w + net->oW0, HW, 1, net->H0, HW, 1, (int)n, HW, NF, w + net->ob0, net->pre0, 1);
    k_segmean<<<nleaf, HW, 0, s>>>(net->H0, t->leaf_start, nleaf, net->G[L]);
    fb_count_launch();
    for (int l = L - 1, k = 0; l >= Ltop; --l, ++k) {
        int nb = t->nbox[l];
        k_segmean<<<nb, HW, 0, s>>>(net->G[l + 1], net->child_start[l], nb, net->Pm[l]);
        fb_count_launch();
        gemm(s, net->Pm[l], HW, 1, w + net->oWu[k], HW, 1, net->G[l], HW, 1, nb, HW, HW, w + net->obu[k],
             net->preu[l], 1);
    }
    FB_CUDA(cudaMemcpyAsync(net->D[Ltop], net->G[Ltop], sizeof(float) * t->nbox[Ltop] * HW,
                            cudaMemcpyDeviceToDevice, s));
    for (int l = Ltop + 1, k = 0; l <= L; ++l, ++k) {
        int nb = t->nbox[l];
        k_concat<<<nb, 2 * HW, 0, s>>>(net->G[l], net->D[l - 1], t->parent[l], nb, net->Cc[l]);
        fb_count_launch();
        gemm(s, net->Cc[l], 2 * HW, 1, w + net->oWd[k], HW, 1, net->D[l], HW, 1, nb, HW, 2 * HW, w + net->obd[k],
             net->pred[l], 1);
    }
    k_concat<<<(unsigned)n, 2 * HW, 0, s>>>(net->H0, net->D[L], net->leaf_of, n, net->E);
    fb_count_launch();
    gemm(s, net->E, 2 * HW, 1, w + net->oWh, HW, 1, net->H1, HW, 1, (int)n, HW, 2 * HW, w + net->obh, net->preh, 1);
    gemm(s, net->H1, HW, 1, w + net->oWo, 2, 1, net->O, 2, 1, (int)n, 2, HW, w + net->obo, nullptr, 0);
    k_output<<<div_up(n, 256), 256, 0, s>>>(t->perm, net->u, net->O, net->scal, n, z);
    fb_count_launch();
    FB_LAUNCH_CHECK();
    return FB_OK;
}

// Inference forward (no stored activations): fused element passes around the
// coarse up/down sweeps.
fb_status fb_learned_apply(LearnedNet* net, const cd* v, cd* z, cudaStream_t s) {
    const fb_tree* t = net->op->tree;
    const Geom& g = net->op->mesh->g;
    int L = net->L, Ltop = L - net->depth;
    int64_t n = net->n;
    int nleaf = t->nbox[L];
    const float* w = net->w;
    FB_CHECK(fb_pc_apply(net->bj, v, net->u, s));
    FB_CUDA(cudaMemsetAsync(net->scal, 0, 8 * sizeof(double), s));
    k_stats<<<std::min<int64_t>(div_up(n, 256), 1024), 256, 0, s>>>(v, n, net->scal);
    k_inf_pass1<<<nleaf, 64, 0, s>>>(g, t->perm, t->leaf_start, v, net->u, net->scal, n, net->kd, w + net->oW0,
                                     w + net->ob0, net->G[L]);
    fb_count_launch(2);
    for (int l = L - 1, k = 0; l >= Ltop; --l, ++k) {
        int nb = t->nbox[l];
        k_inf_layer<HW><<<div_up(nb, 32), 256, 0, s>>>(0, nb, net->G[l + 1], net->child_start[l], nullptr,
                                                       net->wpk + net->pWu[k], w + net->obu[k], net->G[l]);
        fb_count_launch();
    }
    // D_top = G_top: the first down-sweep layer reads G_top as its parent feature
    const float* Dprev = net->G[Ltop];
    for (int l = Ltop + 1, k = 0; l <= L; ++l, ++k) {
        int nb = t->nbox[l];
        k_inf_layer<2 * HW><<<div_up(nb, 32), 256, 0, s>>>(1, nb, net->G[l], t->parent[l], Dprev,
                                                           net->wpk + net->pWd[k], w + net->obd[k], net->D[l]);
        fb_count_launch();
        Dprev = net->D[l];
    }
    k_inf_pass2<<<div_up(n, 64), 256, 0, s>>>(g, t->perm, net->leaf_of, v, net->u, net->scal, n, net->kd,
                                             w + net->oW0,
                                             w + net->ob0, Dprev, net->wpk + net->pWh, w + net->obh, w + net->oWo,
                                             w + net->obo, z);
    fb_count_launch();
    FB_LAUNCH_CHECK();
    return FB_OK;
}

// Loss of one pair and accumulation of its gradient (scaled by `scale`)
// into net->grad.  Returns the loss sums in net->scal[1..2] (device).
fb_status fb_learned_backward(LearnedNet* net, const cd* r, const cd* e, double scale, cudaStream_t s) {
    const fb_tree* t = net->op->tree;
    int L = net->L, Ltop = L - net->depth;
    int64_t n = net->n;
    int nleaf = t->nbox[L];
    FB_CHECK(fb_learned_forward(net, r, net->z, s));
    FB_CUDA(cudaMemsetAsync(net->scal + 1, 0, 2 * sizeof(double), s));
    const int red = std::min<int64_t>(div_up(n, 256), 1024);
    if (net->objective == FB_LOSS_ERROR) {
        k_loss_sums<<<red, 256, 0, s>>>(net->z, e, n, net->scal + 1);
        k_loss_grad<<<div_up(n, 256), 256, 0, s>>>(t->perm, net->z, e, net->scal, net->scal + 1, n, scale,
                                                   net->dO);
        fb_count_launch(2);
    } else {
        FB_CHECK(fb_learned_adjoint_ops(net, s));
        const fb_op* A = net->op;
        const Geom& g = A->mesh->g;
        FB_CHECK(fb_apply_any(const_cast<fb_op*>(A), net->z, net->az, s));
        k_loss_sums<<<red, 256, 0, s>>>(net->az, r, n, net->scal + 1);   // ||A z - r||^2, ||r||^2
        k_adj_prep<<<div_up(n, 256), 256, 0, s>>>(net->az, r, g.area, n, net->yc);
        fb_count_launch(2);
        FB_CHECK(fb_apply_any(net->opLP, net->yc, net->t1, s));
        FB_CHECK(fb_apply_any(net->opL, net->yc, net->t2, s));
        k_adj_grad<<<div_up(n, 256), 256, 0, s>>>(t->perm, net->az, r, net->t1, net->t2, g.area, g.beta, A->k,
                                                  net->scal, net->scal + 1, n, scale, net->dO);
        fb_count_launch();
    }
    float* w = net->w;
    float* gr = net->grad;
    auto colsum = [&](const float* X, int64_t rows, int cols, float* out) {
        dim3 grid((unsigned)std::min<int64_t>(div_up(rows, 256), 256), cols);
        k_colsum<<<grid, 256, 0, s>>>(X, rows, cols, out);
        fb_count_launch();
    };
    // O = H1 Wo + bo
    gemm(s, net->H1, 1, HW, net->dO, 2, 1, gr + net->oWo, 2, 1, HW, 2, (int)n, nullptr, nullptr, 0, 1);
    colsum(net->dO, n, 2, gr + net->obo);
    gemm(s, net->dO, 2, 1, w + net->oWo, 1, 2, net->dH1, HW, 1, (int)n, HW, 2);
    // H1 = silu(E Wh + bh)
    k_silu_back<<<div_up(n * HW, 256), 256, 0, s>>>(net->dH1, net->preh, n * HW, net->dtmp);
    fb_count_launch();
    gemm(s, net->E, 1, 2 * HW, net->dtmp, HW, 1, gr + net->oWh, HW, 1, 2 * HW, HW, (int)n, nullptr, nullptr, 0, 1);
    colsum(net->dtmp, n, HW, gr + net->obh);
    gemm(s, net->dtmp, HW, 1, w + net->oWh, 1, HW, net->dE, 2 * HW, 1, (int)n, 2 * HW, HW);
    // E = [H0, D_L(leaf)]
    FB_CUDA(cudaMemsetAsync(net->dH0, 0, sizeof(float) * n * HW, s));
    for (int l = Ltop; l <= L; ++l) {
        FB_CUDA(cudaMemsetAsync(net->dD[l], 0, sizeof(float) * t->nbox[l] * HW, s));
        FB_CUDA(cudaMemsetAsync(net->dG[l], 0, sizeof(float) * t->nbox[l] * HW, s));
    }
    k_concat_back<<<(unsigned)n, 2 * HW, 0, s>>>(net->dE, net->leaf_of, n, net->dH0, net->dD[L]);
    fb_count_launch();
    // down-sweep backward
    for (int l = L, k = net->depth - 1; l > Ltop; --l, --k) {
        int nb = t->nbox[l];
        k_silu_back<<<div_up((int64_t)nb * HW, 256), 256, 0, s>>>(net->dD[l], net->pred[l], (int64_t)nb * HW, net->dtmp);
        fb_count_launch();
        gemm(s, net->Cc[l], 1, 2 * HW, net->dtmp, HW, 1, gr + net->oWd[k], HW, 1, 2 * HW, HW, nb, nullptr, nullptr,
             0, 1);
        colsum(net->dtmp, nb, HW, gr + net->obd[k]);
        gemm(s, net->dtmp, HW, 1, w + net->oWd[k], 1, HW, net->dC[l], 2 * HW, 1, nb, 2 * HW, HW);
        k_concat_back<<<nb, 2 * HW, 0, s>>>(net->dC[l], t->parent[l], nb, net->dG[l], net->dD[l - 1]);
        fb_count_launch();
    }
    // D_top = G_top: dG_top += dD_top
    {
        int64_t cnt = (int64_t)t->nbox[Ltop] * HW;
        k_add_f<<<div_up(cnt, 256), 256, 0, s>>>(net->dG[Ltop], net->dD[Ltop], cnt);
        fb_count_launch();
    }
    // up-sweep backward (top level first)
    for (int l = Ltop, k = net->depth - 1; l < L; ++l, --k) {
        int nb = t->nbox[l];
        k_silu_back<<<div_up((int64_t)nb * HW, 256), 256, 0, s>>>(net->dG[l], net->preu[l], (int64_t)nb * HW, net->dtmp);
        fb_count_launch();
        gemm(s, net->Pm[l], 1, HW, net->dtmp, HW, 1, gr + net->oWu[k], HW, 1, HW, HW, nb, nullptr, nullptr, 0, 1);
        colsum(net->dtmp, nb, HW, gr + net->obu[k]);
        gemm(s, net->dtmp, HW, 1, w + net->oWu[k], 1, HW, net->dPm[l], HW, 1, nb, HW, HW);
        k_segmean_back<<<nb, HW, 0, s>>>(net->dPm[l], net->child_start[l], nb, net->dG[l + 1]);
        fb_count_launch();
    }
    // leaves: G_L = mean(H0)
    k_segmean_back<<<nleaf, HW, 0, s>>>(net->dG[L], t->leaf_start, nleaf, net->dH0);
    fb_count_launch();
    // H0 = silu(F W0 + b0)
    k_silu_back<<<div_up(n * HW, 256), 256, 0, s>>>(net->dH0, net->pre0, n * HW, net->dtmp);
    fb_count_launch();
    gemm(s, net->F, 1, NF, net->dtmp, HW, 1, gr + net->oW0, HW, 1, NF, HW, (int)n, nullptr, nullptr, 0, 1);
    colsum(net->dtmp, n, HW, gr + net->ob0);
    FB_LAUNCH_CHECK();
    return FB_OK;
}

// Operators of the stand-in adjoint (built once, same tree, k and order rule
// as the served operator, mixed precision).
fb_status fb_learned_adjoint_ops(LearnedNet* net, cudaStream_t s) {
    if (net->opL && net->opLP) return FB_OK;
    const fb_op* A = net->op;
    int64_t n = net->n;
    void* st = (void*)s;
    FB_CHECK(fb_operator_create(A->mesh, A->tree, A->k, FB_OP_L, FB_PREC_MIXED_FMM, A->d0, A->pmin, st, &net->opL));
    FB_CHECK(fb_operator_create(A->mesh, A->tree, A->k, FB_OP_LP, FB_PREC_MIXED_FMM, A->d0, A->pmin, st,
                                &net->opLP));
    FB_CHECK(dalloc(&net->az, n));
    FB_CHECK(dalloc(&net->yc, n));
    FB_CHECK(dalloc(&net->t1, n));
    FB_CHECK(dalloc(&net->t2, n));
    return FB_OK;
}

fb_status fb_learned_set_objective(LearnedNet* net, int objective) {
    if (objective != FB_LOSS_ERROR && objective != FB_LOSS_RESIDUAL) return fb_fail(FB_ERR_ARG, "unknown objective");
    net->objective = objective;
    return FB_OK;
}

// Loss and gradient over a batch of pairs (device arrays, element order,
// pairs stored one after the other).  grad is averaged over the batch.
fb_status fb_learned_loss_grad(LearnedNet* net, const cd* R, const cd* E, int npairs, double* loss,
                               cudaStream_t s) {
    int64_t n = net->n;
    FB_CUDA(cudaMemsetAsync(net->grad, 0, sizeof(float) * net->nparam, s));
    double total = 0.0;
    for (int q = 0; q < npairs; ++q) {
        FB_CHECK(fb_learned_backward(net, R + (int64_t)q * n, E + (int64_t)q * n, 1.0 / npairs, s));
        double h[2];
        FB_CUDA(cudaMemcpyAsync(h, net->scal + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
        FB_CUDA(cudaStreamSynchronize(s));
        total += h[1] > 0 ? h[0] / h[1] : 0.0;
    }
    if (loss) *loss = total / std::max(npairs, 1);
    return FB_OK;
}

// Rebuilds the packed inference weights from the FP32 parameters.
fb_status fb_learned_pack(LearnedNet* net, cudaStream_t s) {
    const float* w = net->w;
    for (int k = 0; k < DEPTH; ++k) {
        k_pack_w<<<div_up(HW * (HW / 2), 256), 256, 0, s>>>(w + net->oWu[k], HW, net->wpk + net->pWu[k]);
        k_pack_w<<<div_up(HW * HW, 256), 256, 0, s>>>(w + net->oWd[k], 2 * HW, net->wpk + net->pWd[k]);
    }
    k_pack_w<<<div_up(HW * HW, 256), 256, 0, s>>>(w + net->oWh, 2 * HW, net->wpk + net->pWh);
    fb_count_launch(2 * DEPTH + 1);
    FB_LAUNCH_CHECK();
    return FB_OK;
}

fb_status fb_learned_adam_step(LearnedNet* net, double lr, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    net->adam_t++;
    float c1 = 1.f - powf(b1, (float)net->adam_t), c2 = 1.f - powf(b2, (float)net->adam_t);
    k_adam<<<div_up(net->nparam, 256), 256, 0, s>>>(net->w, net->grad, net->m1, net->m2, net->nparam, (float)lr, b1,
                                                    b2, eps, c1, c2);
    fb_count_launch();
    FB_LAUNCH_CHECK();
    FB_CHECK(fb_learned_pack(net, s));
    return FB_OK;
}

// Deterministic initialisation: uniform(-a, a), a = sqrt(3 / fan_in) from a
// counter-based hash of the parameter index and seed; biases zero; the output
// layer scaled by 1e-2 so the untrained network is close to block Jacobi.
__global__ void k_init_params(float* w, int64_t n, const int64_t* seg, int nseg, uint64_t seed) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    // segments: (offset, count, fan_in, scale_code) quadruples
    float val = 0.f;
    for (int k = 0; k < nseg; ++k) {
        int64_t off = seg[4 * k], cnt = seg[4 * k + 1], fan = seg[4 * k + 2], code = seg[4 * k + 3];
        if (i >= off && i < off + cnt) {
            if (fan > 0) {
                uint64_t x = (uint64_t)i * 0x9E3779B97F4A7C15ULL ^ seed;
                x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
                float u01 = (float)((x >> 40) & 0xFFFFFF) / 16777216.0f;
                float a = sqrtf(3.f / (float)fan) * (code == 1 ? 1e-2f : 1.f);
                val = (2.f * u01 - 1.f) * a;
            }
            break;
        }
    }
    w[i] = val;
}

fb_status fb_learned_init(LearnedNet* net, uint64_t seed, cudaStream_t s) {
    std::vector<int64_t> seg;
    auto add = [&](int64_t off, int64_t cnt, int64_t fan, int64_t code) {
        seg.push_back(off); seg.push_back(cnt); seg.push_back(fan); seg.push_back(code);
    };
    add(net->oW0, NF * HW, NF, 0);
    add(net->ob0, HW, 0, 0);
    for (int k = 0; k < DEPTH; ++k) { add(net->oWu[k], HW * HW, HW, 0); add(net->obu[k], HW, 0, 0); }
    for (int k = 0; k < DEPTH; ++k) { add(net->oWd[k], 2 * HW * HW, 2 * HW, 0); add(net->obd[k], HW, 0, 0); }
    add(net->oWh, 2 * HW * HW, 2 * HW, 0);
    add(net->obh, HW, 0, 0);
    add(net->oWo, HW * 2, HW, 1);
    add(net->obo, 2, 0, 0);
    int64_t* dseg = nullptr;
    FB_CHECK(dalloc(&dseg, seg.size()));
    FB_CUDA(cudaMemcpyAsync(dseg, seg.data(), sizeof(int64_t) * seg.size(), cudaMemcpyHostToDevice, s));
    k_init_params<<<div_up(net->nparam, 256), 256, 0, s>>>(net->w, net->nparam, dseg, (int)seg.size() / 4, seed);
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(dseg);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, cudaGetErrorString(e));
    net->adam_t = 0;
    FB_CUDA(cudaMemsetAsync(net->m1, 0, sizeof(float) * net->nparam, s));
    FB_CUDA(cudaMemsetAsync(net->m2, 0, sizeof(float) * net->nparam, s));
    FB_CHECK(fb_learned_pack(net, s));
    return FB_OK;
}

int64_t fb_learned_nparam(const LearnedNet* net) { return net->nparam; }
float* fb_learned_weights(LearnedNet* net) { return net->w; }
float* fb_learned_grads(LearnedNet* net) { return net->grad; }

fb_status fb_learned_params_changed(LearnedNet* net, cudaStream_t s) { return fb_learned_pack(net, s); }
