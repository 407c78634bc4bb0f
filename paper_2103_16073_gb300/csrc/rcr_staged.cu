// Rotation - coaxial translation - back-rotation (Sec. 3.3) for large
// expansion orders, staged through global memory as three batched GEMM
// passes per level.  At order p one box pair needs the rotation blocks of its
// direction (sum_n (2n+1)^2 ~ 4p^3/3 coefficients, twice) and the coaxial
// blocks of its |t| (sum_m (p-|m|)^2 ~ 2p^3/3); at p = 159 that is ~40 MB per
// pair, so the translation only runs near the arithmetic roofline when every
// coefficient block is applied to many pairs at once.  The passes group the
// pairs so that it is:
//
//   R  rotate:       u_n = d^n(theta) (e^{i m phi} x_n)       per (theta, n)
//      The real factor d^n depends on the polar angle theta of the
//      translation direction only (D^n_{mu,m} = d^n_{mu,m}(theta) e^{i m phi}
//      for Q = R_y(-theta) R_z(-phi)), so all pairs of a level whose
//      directions share theta (290 directions, 49 polar angles) form the
//      columns of one real GEMM per degree n; the phase e^{i m phi} of each
//      pair's own direction is applied while staging its input.
//   C  coaxial:      v^{+-m} = C^{|m|}(|t|) u^{+-m}             per (|t|, |m|)
//      The coaxial block of order |m| depends on the translation distance
//      only: all pairs of a level with one |t|, both signs of m, are the
//      columns of one complex GEMM per |m|.
//   B  back-rotate:  y_n' = e^{-i m' phi} d^{n'}(theta)^T v_n'   per (theta, n')
//      then scatter-added into the target boxes (atomic adds: several pairs
//      share a target).
//
// The rotations run folded (even / odd in m, see below: half the
// multipliers).  u and v are kept per pair in degree-major order (degree n
// at n^2, folded within the degree: E_0..E_n, then O_1..O_n), so the
// rotations read and write contiguous runs; the coaxial pass, which sums
// over degrees at a fixed order, gathers its inputs and scatters its
// outputs with a stride of one degree block.  One CTA computes a 64 x 64
// tile of one GEMM (256 threads, 4 x 4 complex outputs each, K in chunks
// of 16, three-stage cp.async pipeline).
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "df.cuh"
#include "rcr_staged.cuh"

using namespace stg;

namespace {

constexpr int SBM = 64;   // rows per tile
constexpr int SBN = 64;   // complex columns per tile
constexpr int SBK = 16;   // K chunk
constexpr int STHREADS = 256;

// tile of pass R (degree n) or B (degree n'): slots [col0, col0 + ncol) of
// one polar-angle group, rows [row0, row0 + 64) of the even or odd block
struct StgTile {
    int32_t col0, ncol;
    int32_t n, row0;
    int32_t adir;      // a direction of the group (its real factors d^n)
    int32_t part;      // 0: even (E, Y+) block, 1: odd (O, Y-) block of the folded rotation
};
// tile of pass C: virtual columns [vc0, vc0 + nvc) of one |t| group
// (virtual column v = slot cidx[c0 + v] for m = 0, else (slot cidx[c0 + v/2],
// sign + for even v, - for odd v))
struct StgCTile {
    int64_t a_off;     // C^{|m|}_{|m|,|m|} of the set
    int32_t c0, vc0, nvc;
    int32_t am, row0, pc;
    int32_t M, K;
};

constexpr int SSTAGES = 3;   // shared-memory stages of the copy pipeline

template <class R, bool CA>
struct StgSmem {
    using AT = typename std::conditional<CA, cx<R>, R>::type;
    alignas(16) AT A[SSTAGES][SBK][SBM + (CA ? 2 : 4)];   // padded rows (16-byte aligned, fewer bank conflicts)
    alignas(16) cx<R> X[SSTAGES][SBK][SBN + 2];
    int64_t col_off[SBN];
    int32_t col_aux[SBN];
};

// asynchronous global -> shared copy of one operand (BYTES = 4, 8 or 16),
// zero-filled when `valid` is false (src is then only a valid address)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const int n = valid ? BYTES : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(n));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

template <class R>
__device__ __forceinline__ void fma_ax(cx<R>& acc, R a, const cx<R>& x) {
    acc.re = fma(a, x.re, acc.re);
    acc.im = fma(a, x.im, acc.im);
}
template <class R>
__device__ __forceinline__ void fma_ax(cx<R>& acc, const cx<R>& a, const cx<R>& x) {
    acc.re = fma(a.re, x.re, acc.re);
    acc.re = fma(-a.im, x.im, acc.re);
    acc.im = fma(a.re, x.im, acc.im);
    acc.im = fma(a.im, x.re, acc.im);
}
// four consecutive shared-memory operands (16-byte aligned) in vector loads
__device__ __forceinline__ void ld4(float (&o)[4], const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(double (&o)[4], const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(cf (&o)[4], const cf* p) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 2);
    o[0] = mk(a.x, a.y); o[1] = mk(a.z, a.w); o[2] = mk(b.x, b.y); o[3] = mk(b.z, b.w);
}
__device__ __forceinline__ void ld4(df (&o)[4], const df* p) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 2);
    o[0] = df(a.x, a.y); o[1] = df(a.z, a.w); o[2] = df(b.x, b.y); o[3] = df(b.z, b.w);
}
__device__ __forceinline__ void ld4(cx<df> (&o)[4], const cx<df>* p) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 a = *reinterpret_cast<const float4*>(p + i);
        o[i] = mk(df(a.x, a.y), df(a.z, a.w));
    }
}
__device__ __forceinline__ void ld4(cd (&o)[4], const cd* p) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 a = *reinterpret_cast<const double2*>(p + i);
        o[i] = mk(a.x, a.y);
    }
}

// acc[i][j] (rows ty*4+i, columns tx+16j) += sum_k A[row][k] X[k][col] over
// k < K.  aptr(r, k) / xptr(c, k) give the global address of an operand, or
// nullptr for a zero (outside the block); A is contiguous along k.  The
// operands of chunk kc + SSTAGES - 1 are copied while chunk kc is computed.
template <class R, bool CA, class PA, class PX>
__device__ __forceinline__ void stg_mainloop(StgSmem<R, CA>& sm, int K, PA aptr, PX xptr, const void* dummy,
                                             cx<R> (&acc)[4][4]) {
    using AT = typename StgSmem<R, CA>::AT;
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    auto issue = [&](int b, int k0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + i * STHREADS;
            const int r = e / SBK, k = e % SBK;
            const AT* pa = aptr(r, k0 + k);
            cp_async<sizeof(AT)>(&sm.A[b][k][r], pa ? (const void*)pa : dummy, pa != nullptr);
            const cx<R>* px = xptr(r, k0 + k);   // column r of the X tile, same (e / 16, e % 16) split
            cp_async<sizeof(cx<R>)>(&sm.X[b][k][r], px ? (const void*)px : dummy, px != nullptr);
        }
    };
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mk<R>(0, 0);
    const int nk = (K + SBK - 1) / SBK;
#pragma unroll
    for (int st = 0; st < SSTAGES - 1; ++st) {
        if (st < nk) issue(st, st * SBK);
        cp_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        cp_wait<SSTAGES - 2>();   // chunk kc has landed (this thread's copies)
        __syncthreads();          // ... and every thread's; chunk kc - 1 is no longer read
        const int nxt = kc + SSTAGES - 1;
        if (nxt < nk) issue(nxt % SSTAGES, nxt * SBK);
        cp_commit();
        const int b = kc % SSTAGES;
#pragma unroll
        for (int kk = 0; kk < SBK; ++kk) {
            AT a[4];
            cx<R> x[4];
            ld4(a, &sm.A[b][kk][ty * 4]);
            // columns tx + 16 j: each load of the half-warp reads 16
            // consecutive operands (no bank conflicts)
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = sm.X[b][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) fma_ax(acc[i][j], a[i], x[j]);
        }
    }
    cp_wait<0>();
}

// The real factors obey d^n_{-mu,-m} = d^n_{mu,m} (for Q = R_y(-theta)
// R_z(-phi); equivalently d_{mu,-m} = d_{-mu,m}), so each rotation folds
// into an "even" and an "odd" GEMM of about half the size: with
// s_m = x_m + x_{-m}, t_m = x_m - x_{-m} (m > 0), s_0 = x_0,
//   E_mu = u_mu + u_{-mu} = 2 d_{mu,0} s_0 + sum_{m>0} (d_{mu,m} + d_{mu,-m}) s_m   (mu = 0..n)
//   O_mu = u_mu - u_{-mu} =                  sum_{m>0} (d_{mu,m} - d_{mu,-m}) t_m   (mu = 1..n)
// ((n+1)^2 + n^2 real multipliers instead of (2n+1)^2).  The coaxial blocks
// depend on |m| only, so they map E to E and O to O; the back-rotation
// folds the same way (y_{-m'} = sum_mu d_{mu,m'} v_{-mu}):
//   Y+_{m'} = y_{m'} + y_{-m'} = d_{0,m'} E_0 + sum_{mu>0} (d_{mu,m'} + d_{-mu,m'}) E_mu
//   Y-_{m'} = y_{m'} - y_{-m'} =               sum_{mu>0} (d_{mu,m'} - d_{-mu,m'}) O_mu
// and y_{+-m'} = (Y+ +- Y-)/2.  Folded layout of a degree-n block of u and
// v: E_0..E_n at offsets 0..n, O_1..O_n at n+1..2n.
//
// Folded rotation tables of a polar-angle group (per degree n at fo(n)):
//   R table, part 0: [mu][m] (n+1)^2, m = 0 -> 2 d_{mu,0}, else d_{mu,m} + d_{mu,-m};
//            part 1: [mu-1][m-1] n^2, d_{mu,m} - d_{mu,-m};
//   B table, part 0: [m'][mu] (n+1)^2, mu = 0 -> d_{0,m'}, else d_{mu,m'} + d_{-mu,m'};
//            part 1: [m'-1][mu-1] n^2, d_{mu,m'} - d_{-mu,m'};
// both row-major with K (the summed index) contiguous.  Group g holds its R
// table at g * 2 fper and its B table at g * 2 fper + fper.

template <class R>
__global__ void k_fold_tables(const double* __restrict__ rotd, int64_t per_dir, const int* __restrict__ rep_dirs,
                              int P, R* __restrict__ out, int64_t fper) {
    const int n = blockIdx.x, g = blockIdx.y;
    const int w = 2 * n + 1;
    const double* Dc = rotd + (int64_t)rep_dirs[g] * per_dir + rot_off(n) + (int64_t)n * w + n;   // d_{0,0}
    R* Rt = out + (int64_t)g * 2 * fper + fo(n);
    R* Bt = Rt + fper;
    const int n0 = (n + 1) * (n + 1), n1 = n * n;
    for (int e = threadIdx.x; e < n0 + n1; e += blockDim.x) {
        const int part = e < n0 ? 0 : 1;
        const int q = part ? e - n0 : e;
        const int nb = n + 1 - part;
        const int a = q / nb + part, b = q % nb + part;   // (row, column) indices
        double rv, bv;
        // R: row mu = a, column m = b;  B: row m' = a, column mu = b
        if (part == 0) {
            rv = b == 0 ? 2.0 * Dc[(int64_t)a * w] : Dc[(int64_t)a * w + b] + Dc[(int64_t)a * w - b];
            bv = b == 0 ? Dc[a] : Dc[(int64_t)b * w + a] + Dc[-(int64_t)b * w + a];
        } else {
            rv = Dc[(int64_t)a * w + b] - Dc[(int64_t)a * w - b];
            bv = Dc[(int64_t)b * w + a] - Dc[-(int64_t)b * w + a];
        }
        Rt[e] = real_from<R>(rv);
        Bt[e] = real_from<R>(bv);
    }
}

// ---------------------------------------------------------- pre-pass P ----
// X0[slot][n^2 + j]: the folded phased input of each pair (x_m =
// e^{i m phi_slot} src[slot][n^2 + n + m]; j <= n: s_j, j > n: t_{j-n}),
// written once so that the rotation GEMMs read contiguous columns.
template <class R, class O>
__global__ void k_stg_prep(const StgSlot* __restrict__ slots, int nslot, const cx<O>* __restrict__ src,
                           const cx<O>* __restrict__ rph, int prot, int Pin, int S, cx<R>* __restrict__ X0) {
    const int64_t total = (int64_t)nslot * Pin;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int sl = (int)(q / Pin), e = (int)(q % Pin);
        const StgSlot s = slots[sl];
        int n = (int)sqrtf((float)e);
        while (n * n > e) --n;
        while ((n + 1) * (n + 1) <= e) ++n;
        const int j = e - n * n;
        const cx<O>* x = src + s.src_off + (int64_t)n * n + n;   // (n, 0)
        const cx<O>* ph = rph + (int64_t)s.dir * (2 * prot - 1) + (prot - 1);
        cx<O> v;
        if (j == 0) {
            v = x[0];
        } else {
            const int m = j <= n ? j : j - n;
            const cx<O> xp = x[m] * ph[m], xm = x[-m] * ph[-m];
            v = j <= n ? xp + xm : xp - xm;
        }
        X0[(int64_t)sl * S + e] = cx_to<R, O>(v);
    }
}

// ------------------------------------------------------------- pass R ----
// part 0: U[slot][n^2 + mu] = E_mu (mu = 0..n); part 1: U[slot][n^2 + n + mu] = O_mu
// (mu = 1..n), from the folded inputs X0 and the R table.
template <class R>
__global__ void __launch_bounds__(STHREADS, 2) k_stg_rot(const StgTile* __restrict__ tiles,
                                                         const R* __restrict__ rf, int64_t fper,
                                                         const cx<R>* __restrict__ X0, cx<R>* __restrict__ U,
                                                         int S) {
    extern __shared__ __align__(16) unsigned char stg_smem[];
    StgSmem<R, false>& sm = *reinterpret_cast<StgSmem<R, false>*>(stg_smem);
    const StgTile tl = tiles[blockIdx.x];
    const int n = tl.n;
    const int part = tl.part;
    const int lo = part;                  // first mu (rows) and first m (K) of the block
    const int nb = n + 1 - part;          // rows = K = n + 1 (even) or n (odd)
    const int tid = threadIdx.x;
    const int64_t xoff = (int64_t)n * n + (part ? n + 1 : 0);
    if (tid < SBN) sm.col_off[tid] = tid < tl.ncol ? (int64_t)(tl.col0 + tid) * S + xoff : -1;
    __syncthreads();
    const R* A = rf + (int64_t)tl.adir * 2 * fper + fo(n) + (part ? (int64_t)(n + 1) * (n + 1) : 0) +
                 (int64_t)tl.row0 * nb;
    const int M = min(SBM, nb - tl.row0);
    auto aptr = [&](int r, int k) -> const R* { return (r < M && k < nb) ? A + (int64_t)r * nb + k : nullptr; };
    auto xptr = [&](int c, int k) -> const cx<R>* {
        const int64_t o = sm.col_off[c];
        return (o < 0 || k >= nb) ? nullptr : X0 + o + k;
    };
    cx<R> acc[4][4];
    stg_mainloop<R, false>(sm, nb, aptr, xptr, (const void*)rf, acc);
    const int ty = tid >> 4, tx = tid & 15;
    const int obase = n * n + (part ? n : 0) + lo + tl.row0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tx + 16 * j;
        if (c >= tl.ncol) continue;
        cx<R>* u = U + (int64_t)(tl.col0 + c) * S + obase;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ty * 4 + i;
            if (r < M) u[r] = acc[i][j];
        }
    }
}

// ------------------------------------------------------------- pass C ----
// E^{am}_{n'} (V[slot][n'^2 + am])      = sum_k C^{am}_{n', am+k} E^{am}_{am+k}   (even columns)
// O^{am}_{n'} (V[slot][n'^2 + n' + am]) = sum_k C^{am}_{n', am+k} O^{am}_{am+k}   (odd columns, am > 0)
// for n' = am + row (degree-major folded, as u)
// with E^{am}_n = U[slot][n^2 + am], O^{am}_n = U[slot][n^2 + n + am].
template <class R>
__global__ void __launch_bounds__(STHREADS, 2) k_stg_coax(const StgCTile* __restrict__ tiles,
                                                          const int32_t* __restrict__ cidx,
                                                          const cx<R>* __restrict__ coax, const cx<R>* __restrict__ U,
                                                          cx<R>* __restrict__ V, int S, int pout) {
    extern __shared__ __align__(16) unsigned char stg_smem[];
    StgSmem<R, true>& sm = *reinterpret_cast<StgSmem<R, true>*>(stg_smem);
    const StgCTile tl = tiles[blockIdx.x];
    const int am = tl.am;
    const int tid = threadIdx.x;
    if (tid < SBN) {
        if (tid < tl.nvc) {
            const int v = tl.vc0 + tid;
            const int slot = am == 0 ? cidx[tl.c0 + v] : cidx[tl.c0 + (v >> 1)];
            const int odd = (am != 0 && (v & 1)) ? 1 : 0;
            sm.col_off[tid] = (int64_t)slot * S;
            sm.col_aux[tid] = odd;
        } else {
            sm.col_off[tid] = -1;
            sm.col_aux[tid] = 0;
        }
    }
    __syncthreads();
    const cx<R>* A = coax + tl.a_off + (int64_t)tl.row0 * tl.pc;
    const int M = min(SBM, tl.M - tl.row0);
    const int K = tl.K, pc = tl.pc;
    auto aptr = [&](int r, int k) -> const cx<R>* { return (r < M && k < K) ? A + (int64_t)r * pc + k : nullptr; };
    auto xptr = [&](int c, int k) -> const cx<R>* {
        const int64_t o = sm.col_off[c];
        if (o < 0 || k >= K) return nullptr;
        const int nn = am + k;
        return U + o + (int64_t)nn * nn + (sm.col_aux[c] ? nn : 0) + am;
    };
    cx<R> acc[4][4];
    stg_mainloop<R, true>(sm, K, aptr, xptr, (const void*)coax, acc);
    const int ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tx + 16 * j;
        if (c >= tl.nvc) continue;
        cx<R>* v = V + sm.col_off[c] + am;
        const int odd = sm.col_aux[c];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ty * 4 + i;
            const int n1 = am + tl.row0 + r;
            if (r < M) v[(int64_t)n1 * n1 + (odd ? n1 : 0)] = acc[i][j];
        }
    }
}

// ------------------------------------------------------------- pass B ----
// part 0: Y+_{m'} (m' = 0..n) from E_mu = V[slot][n^2 + mu], mu = 0..mmax;
// part 1: Y-_{m'} (m' = 1..n) from O_mu = V[slot][n^2 + n + mu], mu = 1..mmax;
// mmax = min(n, p_in - 1).  dst[slot][n^2 + n +- m'] += e^{-+ i m' phi} (Y+ +- Y-)/2.
template <class R>
__device__ __forceinline__ void atomic_add_cx(cx<R>* d, const cx<R>& v);
template <>
__device__ __forceinline__ void atomic_add_cx<float>(cf* d, const cf& v) {
    atomicAdd(reinterpret_cast<float2*>(d), make_float2(v.re, v.im));
}
template <>
__device__ __forceinline__ void atomic_add_cx<double>(cd* d, const cd& v) {
    atomicAdd(&d->re, v.re);
    atomicAdd(&d->im, v.im);
}

template <class R, class O>
__global__ void __launch_bounds__(STHREADS, 2) k_stg_back(const StgTile* __restrict__ tiles,
                                                          const StgSlot* __restrict__ slots,
                                                          const R* __restrict__ rf, int64_t fper,
                                                          const cx<O>* __restrict__ rph, int prot,
                                                          const cx<R>* __restrict__ V, cx<O>* __restrict__ dst, int S,
                                                          int pin, int pout) {
    extern __shared__ __align__(16) unsigned char stg_smem[];
    StgSmem<R, false>& sm = *reinterpret_cast<StgSmem<R, false>*>(stg_smem);
    const StgTile tl = tiles[blockIdx.x];
    const int n = tl.n;
    const int part = tl.part;
    const int lo = part;
    const int mmax = min(n, pin - 1);
    const int nrow = n + 1 - part;          // m' = lo .. n; also the table's row stride
    const int K = mmax + 1 - part;          // mu = lo .. mmax
    const int tid = threadIdx.x;
    if (tid < SBN) {
        if (tid < tl.ncol) {
            StgSlot sl = slots[tl.col0 + tid];
            sm.col_off[tid] = sl.dst_off + (int64_t)n * n + n;   // entry (n, 0)
            sm.col_aux[tid] = sl.dir;
        } else {
            sm.col_off[tid] = -1;
            sm.col_aux[tid] = 0;
        }
    }
    __syncthreads();
    const R* A = rf + (int64_t)tl.adir * 2 * fper + fper + fo(n) + (part ? (int64_t)(n + 1) * (n + 1) : 0) +
                 (int64_t)tl.row0 * nrow;
    const int M = min(SBM, nrow - tl.row0);
    auto aptr = [&](int r, int k) -> const R* { return (r < M && k < K) ? A + (int64_t)r * nrow + k : nullptr; };
    const int64_t col_base = (int64_t)tl.col0 * S;
    auto xptr = [&](int c, int k) -> const cx<R>* {
        if (c >= tl.ncol || k >= K) return nullptr;
        const int mu = lo + k;
        return V + col_base + (int64_t)c * S + (int64_t)n * n + (part ? n : 0) + mu;
    };
    cx<R> acc[4][4];
    stg_mainloop<R, false>(sm, K, aptr, xptr, (const void*)rf, acc);
    const int ty = tid >> 4, tx = tid & 15;
    const O sgn = part ? O(-1) : O(1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tx + 16 * j;
        if (c >= tl.ncol) continue;
        const cx<O>* ph = rph + (int64_t)sm.col_aux[c] * (2 * prot - 1) + (prot - 1);
        cx<O>* d = dst + sm.col_off[c];   // entry (n, 0) of the target
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ty * 4 + i;
            if (r >= M) continue;
            const int mp = lo + tl.row0 + r;
            const cx<O> h = O(0.5) * cx_out<O, R>(acc[i][j]);
            if (mp == 0) {
                atomic_add_cx<O>(d, h);
            } else {
                atomic_add_cx<O>(d + mp, h * conjg(ph[mp]));
                atomic_add_cx<O>(d - mp, sgn * (h * ph[mp]));
            }
        }
    }
}

// ------------------------------------------------------------ host plan ----
struct StgLevel {
    int64_t src_base = 0, dst_base = 0;   // the level arrays it reads and writes
    int p_in = 0, p_out = 0, S = 0, nslot = 0;
    StgSlot* slots = nullptr;
    int32_t* cidx = nullptr;
    StgTile* rt = nullptr;
    StgCTile* ct = nullptr;
    StgTile* bt = nullptr;
    int nrt = 0, nct = 0, nbt = 0;
    // rotation passes on the tensor cores (rcr_staged_tc.cu) instead of rt / bt
    int tc = 0;
    int tcc = 0;  // ... and the coaxial pass too
    int df = 0;   // passes in double-FP32 arithmetic (FP64 expansions)
    StcTile* rtc = nullptr;
    StcTile* btc = nullptr;
    int nrtc = 0, nbtc = 0;
    // coaxial pass on the tensor cores (tc levels): tiles and the plan's
    // pre-split coaxial blocks
    StcCTile* ctc = nullptr;
    int nctc = 0;
    float* ctab = nullptr;
};

struct StgPlanImpl {
    std::vector<StgLevel> levels;
};

void free_level(StgLevel& lv) {
    dfree(lv.slots);
    dfree(lv.cidx);
    dfree(lv.rt);
    dfree(lv.ct);
    dfree(lv.bt);
    dfree(lv.rtc);
    dfree(lv.btc);
    dfree(lv.ctc);
    dfree(lv.ctab);
}

template <class T>
fb_status upload(T** d, const std::vector<T>& h) {
    if (h.empty()) return FB_OK;
    FB_CHECK(dalloc(d, h.size()));
    FB_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return FB_OK;
}

}  // namespace

bool fb_stg_staged(const RcrTask& tk) { return (tk.staged >= 1 && tk.staged <= 3) || tk.staged == 5; }

bool fb_rcr_tile_fits(int p_in, int p_out, size_t csize) {
    const size_t per = (size_t)((int64_t)p_in * p_in + std::max<int64_t>((int64_t)p_in * p_in, (int64_t)p_out * p_out));
    return per * csize <= 200 * 1024;
}
int fb_rcr_default_staged(int p_in, int p_out, size_t csize) {
    return !fb_rcr_tile_fits(p_in, p_out, csize) || std::max(p_in, p_out) >= FB_STG_PMIN;
}

// Builds the staged passes of the tasks of `pl` that fb_stg_staged selects.
// theta_slot[dir] is the polar-angle group of direction dir (the index of
// the group's folded rotation tables).
// *elems receives the complex coefficients one staging buffer needs (the
// largest level: pairs x max(p_in, p_out)^2).
fb_status fb_stg_build(const RcrPlan& pl, const std::vector<int>& theta_slot, int64_t per_dir, const cd* coax64,
                       void** out, int64_t* elems) {
    *out = nullptr;
    *elems = 0;
    // tasks by level (same source and target level arrays and orders)
    std::map<std::tuple<int64_t, int64_t, int, int>, std::vector<int>> by_level;
    for (int t = 0; t < (int)pl.h_tasks.size(); ++t) {
        const RcrTask& tk = pl.h_tasks[t];
        if (!fb_stg_staged(tk) || tk.npairs == 0) continue;
        by_level[std::make_tuple(tk.src_base, tk.dst_base, tk.p_in, tk.p_out)].push_back(t);
    }
    if (by_level.empty()) return FB_OK;
    StgPlanImpl* P = new StgPlanImpl();
    auto fail = [&](fb_status st) {
        for (auto& lv : P->levels) free_level(lv);
        delete P;
        return st;
    };
    for (auto& kv : by_level) {
        const std::vector<int>& ts = kv.second;
        const int p_in = std::get<2>(kv.first), p_out = std::get<3>(kv.first);
        StgLevel lv;
        lv.src_base = std::get<0>(kv.first);
        lv.dst_base = std::get<1>(kv.first);
        lv.p_in = p_in;
        lv.p_out = p_out;
        for (int t : ts) {
            lv.tc = lv.tc || pl.h_tasks[t].staged == 2 || pl.h_tasks[t].staged == 5;
            lv.tcc = lv.tcc || pl.h_tasks[t].staged == 5;
            lv.df = lv.df || pl.h_tasks[t].staged == 3;
        }
        lv.S = std::max(p_in * p_in, p_out * p_out);
        // polar-angle groups of the tasks, in order of first appearance
        std::map<int, std::vector<int>> groups;   // representative direction -> tasks
        std::vector<int> group_order;
        for (int t : ts) {
            int dir = (int)(pl.h_tasks[t].rot_off / per_dir);
            int rep = theta_slot.at(dir);
            if (!groups.count(rep)) group_order.push_back(rep);
            groups[rep].push_back(t);
        }
        std::vector<StgSlot> slots;
        std::vector<int> slot_task;
        std::vector<StgTile> rt, bt;
        std::vector<StcTile> rtc, btc;
        for (int rep : group_order) {
            const int g0 = (int)slots.size();
            for (int t : groups[rep]) {
                const RcrTask& tk = pl.h_tasks[t];
                std::vector<int32_t> si(tk.npairs), di(tk.npairs);
                if (cudaMemcpy(si.data(), pl.src_idx + tk.pair_off, sizeof(int32_t) * tk.npairs,
                               cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(di.data(), pl.dst_idx + tk.pair_off, sizeof(int32_t) * tk.npairs,
                               cudaMemcpyDeviceToHost) != cudaSuccess)
                    return fail(fb_fail(FB_ERR_CUDA, "staged RCR: pair index copy failed"));
                const int dir = (int)(tk.rot_off / per_dir);
                for (int j = 0; j < tk.npairs; ++j) {
                    StgSlot s;
                    s.src_off = tk.src_base + (int64_t)si[j] * p_in * p_in;
                    s.dst_off = tk.dst_base + (int64_t)di[j] * p_out * p_out;
                    s.dir = dir;
                    s.pad = 0;
                    slots.push_back(s);
                    slot_task.push_back(t);
                }
            }
            const int g1 = (int)slots.size();
            if (lv.tc) {
                fb_stc_group_tiles(rep, g0, g1, p_in, 0, p_in, rtc);
                fb_stc_group_tiles(rep, g0, g1, p_out, 1, p_in, btc);
                continue;
            }
            // folded blocks: even rows n + 1, odd rows n (none for n = 0)
            for (int n = 0; n < p_in; ++n)
                for (int part = 0; part < 2; ++part)
                    for (int r0 = 0; r0 < n + 1 - part; r0 += SBM)
                        for (int c0 = g0; c0 < g1; c0 += SBN)
                            rt.push_back(StgTile{c0, std::min(SBN, g1 - c0), n, r0, rep, part});
            for (int n = 0; n < p_out; ++n) {
                const int mmax = std::min(n, p_in - 1);
                for (int part = 0; part < 2; ++part) {
                    if (mmax + 1 - part <= 0) continue;   // no inner terms
                    for (int r0 = 0; r0 < n + 1 - part; r0 += SBM)
                        for (int c0 = g0; c0 < g1; c0 += SBN)
                            bt.push_back(StgTile{c0, std::min(SBN, g1 - c0), n, r0, rep, part});
                }
            }
        }
        // |t| groups (coaxial sets) of the slots
        std::map<int64_t, std::vector<int32_t>> sets;   // coax_off -> slots
        std::map<int64_t, int> set_pc;
        for (int s = 0; s < (int)slots.size(); ++s) {
            const RcrTask& tk = pl.h_tasks[slot_task[s]];
            sets[tk.coax_off].push_back(s);
            set_pc[tk.coax_off] = tk.pc;
        }
        std::vector<int32_t> cidx;
        std::vector<StgCTile> ct;
        std::vector<StcCTile> ctc;
        std::vector<StcCBlock> cblocks;
        int64_t ctab_floats = 0;
        const int q = std::min(p_in, p_out);
        for (auto& sv : sets) {
            const int c0 = (int)cidx.size();
            cidx.insert(cidx.end(), sv.second.begin(), sv.second.end());
            const int ns = (int)sv.second.size();
            const int pc = set_pc[sv.first];
            if (lv.tcc && coax64) {
                fb_stc_coax_set(c0, ns, sv.first, pc, p_in, p_out, ctc, cblocks, &ctab_floats);
                continue;
            }
            if (pl.csize != sizeof(cf)) {
                // FP64 / double-FP32 passes are bound by arithmetic: orders
                // outermost, full column blocks, each coefficient block
                // applied to every column block in turn
                for (int am = 0; am < q; ++am) {
                    const int nvc = am == 0 ? ns : 2 * ns;
                    const int M = p_out - am, K = p_in - am;
                    const int64_t a_off = sv.first + ((int64_t)am * pc + am) * pc + am;
                    for (int r0 = 0; r0 < M; r0 += SBM)
                        for (int v0 = 0; v0 < nvc; v0 += SBN)
                            ct.push_back(StgCTile{a_off, c0, v0, std::min(SBN, nvc - v0), am, r0, pc, M, K});
                }
                continue;
            }
            // FP32: slot blocks outermost, orders next: the tiles of
            // consecutive orders of one slot block run together, so each
            // 32-byte sector of u they gather from and of v they scatter to
            // (four orders of one degree) is read and written while in L2
            for (int sb = 0; sb < ns; sb += SBN / 2)
                for (int am = 0; am < q; ++am) {
                    const int M = p_out - am, K = p_in - am;
                    const int64_t a_off = sv.first + ((int64_t)am * pc + am) * pc + am;
                    // virtual columns: order 0 one per slot, else (slot, even / odd part)
                    const int v0 = am == 0 ? sb : 2 * sb;
                    const int nvc = am == 0 ? std::min(SBN / 2, ns - sb) : std::min(SBN, 2 * (ns - sb));
                    for (int r0 = 0; r0 < M; r0 += SBM)
                        ct.push_back(StgCTile{a_off, c0, v0, nvc, am, r0, pc, M, K});
                }
        }
        lv.nslot = (int)slots.size();
        lv.nrt = (int)rt.size();
        lv.nct = (int)ct.size();
        lv.nbt = (int)bt.size();
        // heaviest tensor-core tiles first (K chunks x columns), for the tail
        auto heavier = [&](int pass) {
            return [pass, p_in](const StcTile& x, const StcTile& y) {
                auto w = [&](const StcTile& t) {
                    int64_t c = 0;
                    for (int n = t.n0; n < t.n1; ++n) {
                        const int N = n + 1 - t.part;
                        const int K = pass == 0 ? N : std::min(n, p_in - 1) + 1 - t.part;
                        c += (int64_t)stc_pad16(N) * ((K + 15) / 16);
                    }
                    return c;
                };
                return w(x) > w(y);
            };
        };
        std::stable_sort(rtc.begin(), rtc.end(), heavier(0));
        std::stable_sort(btc.begin(), btc.end(), heavier(1));
        lv.nrtc = (int)rtc.size();
        lv.nbtc = (int)btc.size();
        lv.nctc = (int)ctc.size();
        fb_status st;
        StcCBlock* d_blocks = nullptr;
        if ((st = upload(&lv.slots, slots)) || (st = upload(&lv.cidx, cidx)) || (st = upload(&lv.rt, rt)) ||
            (st = upload(&lv.ct, ct)) || (st = upload(&lv.bt, bt)) || (st = upload(&lv.rtc, rtc)) ||
            (st = upload(&lv.btc, btc)) || (st = upload(&lv.ctc, ctc)) || (st = upload(&d_blocks, cblocks)) ||
            (ctab_floats > 0 && (st = dalloc(&lv.ctab, (size_t)ctab_floats))) ||
            (st = fb_stc_coax_tables(d_blocks, (int)cblocks.size(), coax64, lv.ctab, cudaStreamLegacy))) {
            dfree(d_blocks);
            free_level(lv);
            return fail(st);
        }
        if (d_blocks) {
            const cudaError_t e = cudaStreamSynchronize(cudaStreamLegacy);
            dfree(d_blocks);
            if (e != cudaSuccess) {
                free_level(lv);
                return fail(fb_fail(FB_ERR_CUDA, std::string("coaxial tables: ") + cudaGetErrorString(e)));
            }
        }
        *elems = std::max(*elems, (int64_t)lv.nslot * lv.S);
        P->levels.push_back(lv);
    }
    *out = P;
    return FB_OK;
}

void fb_stg_free(void*& plan) {
    StgPlanImpl* P = (StgPlanImpl*)plan;
    if (!P) return;
    for (auto& lv : P->levels) free_level(lv);
    delete P;
    plan = nullptr;
}

// Folded rotation tables of an operator (both passes, every polar-angle
// group, degrees < Prot) from the FP64 real factors, in the operator's
// precision.
fb_status fb_stg_tables(fb_op* op, const double* rotd64, cudaStream_t s) {
    const int ng = (int)op->theta_dirs.size();
    if (ng == 0 || op->Prot < 1) return FB_OK;
    const int P = op->Prot;
    op->rotf_per = fo(P);
    int* d_dirs = nullptr;
    FB_CHECK(dalloc(&d_dirs, (size_t)ng));
    FB_CUDA(cudaMemcpyAsync(d_dirs, op->theta_dirs.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, s));
    const size_t count = (size_t)ng * 2 * op->rotf_per;
    fb_status st;
    if (op->prec == FB_PREC_MIXED_FMM) {
        float* t = nullptr;
        st = dalloc(&t, count);
        if (st == FB_OK) k_fold_tables<float><<<dim3(P, ng), 256, 0, s>>>(rotd64, op->per_dir, d_dirs, P, t, op->rotf_per);
        op->rotf = t;
    } else {
        double* t = nullptr;
        st = dalloc(&t, count);
        if (st == FB_OK) k_fold_tables<double><<<dim3(P, ng), 256, 0, s>>>(rotd64, op->per_dir, d_dirs, P, t, op->rotf_per);
        op->rotf = t;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(d_dirs);
    FB_CHECK(st);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("folded rotation tables: ") + cudaGetErrorString(e));
    fb_count_launch();
    return FB_OK;
}

static __global__ void k_cd_to_df(const cd* __restrict__ in, int64_t n, cx<df>* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mk(df_from(in[i].re), df_from(in[i].im));
}

// Folded rotation tables and coaxial sets of an FP64 operator in
// double-FP32, for its staged levels in that arithmetic (built once).
fb_status fb_stg_df_tables(fb_op* op, cudaStream_t s) {
    if (op->rotf_df && op->coax_df) return FB_OK;
    if (op->prec != FB_PREC_FP64_FMM) return fb_fail(FB_ERR_ARG, "double-FP32 staged RCR applies to FP64 operators");
    const int ng = (int)op->theta_dirs.size();
    if (ng == 0 || op->Prot < 1 || !op->coax64) return fb_fail(FB_ERR_STATE, "staged RCR: no rotation groups");
    const int P = op->Prot;
    int* d_dirs = nullptr;
    FB_CHECK(dalloc(&d_dirs, (size_t)ng));
    FB_CHECK(dalloc(&op->rotf_df, (size_t)ng * 2 * op->rotf_per));
    FB_CHECK(dalloc(&op->coax_df, (size_t)op->coax_count));
    FB_CUDA(cudaMemcpyAsync(d_dirs, op->theta_dirs.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, s));
    k_fold_tables<df><<<dim3(P, ng), 256, 0, s>>>(op->rotd64, op->per_dir, d_dirs, P, op->rotf_df, op->rotf_per);
    k_cd_to_df<<<(unsigned)std::min<int64_t>((op->coax_count + 255) / 256, 4096), 256, 0, s>>>(
        op->coax64, op->coax_count, op->coax_df);
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(d_dirs);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("double-FP32 tables: ") + cudaGetErrorString(e));
    fb_count_launch(2);
    return FB_OK;
}

// Runs the staged passes of a plan for nrhs right-hand sides (set r of the
// expansions at src / dst + r * rstride), one right-hand side and one level
// at a time: pre-pass (src -> V), rotation (V -> U), coaxial (U -> V),
// back-rotation (V -> dst).
// Tensor-core rotation passes of a level (single precision only).
static fb_status stc_pass(const StgLevel& lv, int pass, const StcTabs* tc, const cf* X, cf* out, const cf* rph,
                          int prot, cudaStream_t s) {
    if (!tc || !tc->tab) return fb_fail(FB_ERR_STATE, "staged RCR: tensor-core tables missing");
    const int np = std::max(lv.p_in, lv.p_out);
    return pass == 0 ? fb_stc_run(0, lv.rtc, lv.nrtc, np, tc->off, tc->tab, tc->per, lv.slots, X, out, lv.S, lv.p_in,
                                  lv.p_out, rph, prot, tc->err, s)
                     : fb_stc_run(1, lv.btc, lv.nbtc, np, tc->off, tc->tab, tc->per, lv.slots, X, out, lv.S, lv.p_in,
                                  lv.p_out, rph, prot, tc->err, s);
}
template <class X, class Y, class Ph>
static fb_status stc_pass(const StgLevel&, int, const StcTabs*, const X*, Y*, const Ph*, int, cudaStream_t) {
    return fb_fail(FB_ERR_ARG, "tensor-core staged RCR applies to single precision");
}
// Tensor-core coaxial pass of a level (single precision only).
static fb_status stc_coax(const StgLevel& lv, const StcTabs* tc, const cf* U, cf* V, cudaStream_t s) {
    if (!tc) return fb_fail(FB_ERR_STATE, "staged RCR: tensor-core error flag missing");
    return fb_stc_coax_run(lv.ctc, lv.nctc, lv.cidx, lv.ctab, U, V, lv.S, lv.p_out, tc->err, s);
}
template <class X>
static fb_status stc_coax(const StgLevel&, const StcTabs*, const X*, X*, cudaStream_t) {
    return fb_fail(FB_ERR_ARG, "tensor-core staged RCR applies to single precision");
}


// The four passes of one level and right-hand side: arithmetic in R
// (tables rf / coax, staging buffers U, V), expansions and phases stored in
// O (R = O, or R = double-FP32 for FP64 expansions).
template <class R, class O>
static fb_status stg_level(const StgLevel& lv, int pass_mask, const R* rf, int64_t fper, const cx<O>* rph, int prot,
                           const cx<R>* coax, const cx<O>* sr, cx<O>* dr, cx<R>* U, cx<R>* V, cudaStream_t s,
                           const StcTabs* tc) {
    const size_t sm_rc = sizeof(StgSmem<R, false>), sm_c = sizeof(StgSmem<R, true>);
    FB_CHECK(fb_smem_cap((const void*)k_stg_rot<R>, sm_rc));
    FB_CHECK(fb_smem_cap((const void*)k_stg_coax<R>, sm_c));
    FB_CHECK(fb_smem_cap((const void*)k_stg_back<R, O>, sm_rc));
    if ((pass_mask & 1) && !lv.tc) {   // the tensor-core rotation pass folds its inputs itself
        const int64_t tot = (int64_t)lv.nslot * lv.p_in * lv.p_in;
        const int pb = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
        k_stg_prep<R, O><<<pb, 256, 0, s>>>(lv.slots, lv.nslot, sr, rph, prot, lv.p_in * lv.p_in, lv.S, V);
        fb_count_launch();
    }
    if (pass_mask & 2) {
        if (lv.tc) {
            FB_CHECK(stc_pass(lv, 0, tc, sr, U, rph, prot, s));
        } else if (lv.nrt) {
            k_stg_rot<R><<<lv.nrt, STHREADS, sm_rc, s>>>(lv.rt, rf, fper, V, U, lv.S);
            fb_count_launch();
        }
    }
    if ((pass_mask & 4) && lv.nctc) {
        FB_CHECK(stc_coax(lv, tc, U, V, s));
    } else if ((pass_mask & 4) && lv.nct) {
        k_stg_coax<R><<<lv.nct, STHREADS, sm_c, s>>>(lv.ct, lv.cidx, coax, U, V, lv.S, lv.p_out);
        fb_count_launch();
    }
    if (pass_mask & 8) {
        if (lv.tc) {
            FB_CHECK(stc_pass(lv, 1, tc, V, dr, rph, prot, s));
        } else if (lv.nbt) {
            k_stg_back<R, O><<<lv.nbt, STHREADS, sm_rc, s>>>(lv.bt, lv.slots, rf, fper, rph, prot, V, dr, lv.S,
                                                             lv.p_in, lv.p_out);
            fb_count_launch();
        }
    }
    FB_LAUNCH_CHECK();
    return FB_OK;
}

template <class R>
static fb_status stg_run(void* plan, const R* rf, int64_t fper, const cx<R>* rph, int prot, const cx<R>* coax,
                         const cx<R>* src, cx<R>* dst, cx<R>* U, cx<R>* V, cudaStream_t s, int nrhs, int64_t rstride,
                         const StcTabs* tc, const DfTabs* dft, int only_level, int pass_mask) {
    StgPlanImpl* P = (StgPlanImpl*)plan;
    if (!P) return FB_OK;
    if (!U || !V || !rf) return fb_fail(FB_ERR_STATE, "staged RCR: staging buffers or tables missing");
    for (int r = 0; r < nrhs; ++r) {
        const cx<R>* sr = src + r * rstride;
        cx<R>* dr = dst + r * rstride;
        for (int li = 0; li < (int)P->levels.size(); ++li) {
            if (only_level >= 0 && li != only_level) continue;
            const StgLevel& lv = P->levels[li];
            if constexpr (sizeof(R) == 8) {
                if (lv.df) {
                    if (!dft || !dft->rf || !dft->coax)
                        return fb_fail(FB_ERR_STATE, "staged RCR: double-FP32 tables missing");
                    // the staging buffers hold complex double-FP32 values (16 bytes, as FP64)
                    FB_CHECK((stg_level<df, double>(lv, pass_mask, dft->rf, fper, rph, prot, dft->coax, sr, dr,
                                                    (cx<df>*)U, (cx<df>*)V, s, nullptr)));
                    continue;
                }
            }
            FB_CHECK((stg_level<R, R>(lv, pass_mask, rf, fper, rph, prot, coax, sr, dr, U, V, s, tc)));
        }
    }
    return FB_OK;
}

fb_status fb_stg_run_f(void* plan, const float* rf, int64_t fper, const cf* rph, int prot, const cf* coax,
                       const cf* src, cf* dst, cf* U, cf* V, cudaStream_t s, int nrhs, int64_t rstride,
                       const StcTabs& tc, int only_level, int pass_mask) {
    return stg_run<float>(plan, rf, fper, rph, prot, coax, src, dst, U, V, s, nrhs, rstride, &tc, nullptr,
                          only_level, pass_mask);
}
fb_status fb_stg_run_d(void* plan, const double* rf, int64_t fper, const cd* rph, int prot, const cd* coax,
                       const cd* src, cd* dst, cd* U, cd* V, cudaStream_t s, int nrhs, int64_t rstride,
                       const DfTabs& dft, int only_level, int pass_mask) {
    return stg_run<double>(plan, rf, fper, rph, prot, coax, src, dst, U, V, s, nrhs, rstride, nullptr, &dft,
                           only_level, pass_mask);
}

int fb_stg_level_count(const void* plan) {
    const StgPlanImpl* P = (const StgPlanImpl*)plan;
    return P ? (int)P->levels.size() : 0;
}
void fb_stg_level_info(const void* plan, int li, int64_t* src_base, int64_t* dst_base, int* form) {
    const StgLevel& lv = ((const StgPlanImpl*)plan)->levels[li];
    *src_base = lv.src_base;
    *dst_base = lv.dst_base;
    *form = lv.tcc ? 5 : (lv.tc ? 2 : (lv.df ? 3 : 1));
}

bool fb_stg_uses_df(const void* plan) {
    const StgPlanImpl* P = (const StgPlanImpl*)plan;
    if (!P) return false;
    for (const StgLevel& lv : P->levels)
        if (lv.df) return true;
    return false;
}

bool fb_stg_uses_tc(const void* plan) {
    const StgPlanImpl* P = (const StgPlanImpl*)plan;
    if (!P) return false;
    for (const StgLevel& lv : P->levels)
        if (lv.tc) return true;
    return false;
}
