// FMM matrix-vector product (Sec. 3.3): P2M -> M2M -> M2L -> L2L -> L2P,
// plus the stored near field.  Templated on the arithmetic type R (double
// for the plain FP64 path, float for the mixed path); input and output
// vectors are complex128 in the caller's element order.
//
// Translations use the stacked form: all box pairs of one level that share a
// translation vector share one p^2 x p^2 matrix, so each (level, offset)
// group is one complex GEMM  Y = T X  with X gathered from the source boxes
// and Y scatter-added into the target boxes.
#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"

// ------------------------------------------------------ gather-GEMM-scatter
// Tile: 64 output rows x 32 column pairs, K chunks of 16; 256 threads, each
// 4 rows x 2 columns.  dst[dst_idx] += T * src[src_idx] (atomic adds: the
// groups of one launch may share targets).
template <class R>
__global__ void __launch_bounds__(256) k_trans(const TransTask* __restrict__ tasks,
                                               const TransTile* __restrict__ tiles,
                                               const cx<R>* __restrict__ Tbuf,
                                               const int32_t* __restrict__ src_idx,
                                               const int32_t* __restrict__ dst_idx,
                                               const cx<R>* __restrict__ src, cx<R>* __restrict__ dst) {
    constexpr int BM = 64, BN = 32, BK = 16;
    __shared__ cx<R> Ts[BK][BM];
    __shared__ cx<R> Xs[BK][BN];
    __shared__ int s_src[BN];
    __shared__ int s_dst[BN];
    TransTile tl = tiles[blockIdx.x];
    TransTask tk = tasks[tl.task];
    int tid = threadIdx.x;
    int ty = tid >> 4, tx = tid & 15;
    if (tid < BN) {
        int c = tl.col0 + tid;
        s_src[tid] = c < tk.npairs ? src_idx[tk.pair_off + c] : -1;
        s_dst[tid] = c < tk.npairs ? dst_idx[tk.pair_off + c] : -1;
    }
    __syncthreads();
    const cx<R>* T = Tbuf + tk.t_off;
    cx<R> acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = mk<R>(0, 0);
    for (int k0 = 0; k0 < tk.cols; k0 += BK) {
#pragma unroll
        for (int it = 0; it < (BM * BK) / 256; ++it) {
            int idx = tid + it * 256;
            int r = idx / BK, kk = idx % BK;
            int row = tl.row0 + r, k = k0 + kk;
            Ts[kk][r] = (row < tk.rows && k < tk.cols) ? T[(int64_t)row * tk.cols + k] : mk<R>(0, 0);
        }
#pragma unroll
        for (int it = 0; it < (BN * BK) / 256; ++it) {
            int idx = tid + it * 256;
            int c = idx / BK, kk = idx % BK;
            int k = k0 + kk;
            int sb = s_src[c];
            Xs[kk][c] = (sb >= 0 && k < tk.cols) ? src[tk.src_base + (int64_t)sb * tk.cols + k] : mk<R>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            cx<R> a[4], b[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ts[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 2; ++j) b[j] = Xs[kk][tx * 2 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) cmac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        int c = tx * 2 + j;
        int db = s_dst[c];
        if (db < 0) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int row = tl.row0 + ty * 4 + i;
            if (row >= tk.rows) continue;
            cx<R>* d = dst + tk.dst_base + (int64_t)db * tk.rows + row;
            atomicAdd(&d->re, acc[i][j].re);
            atomicAdd(&d->im, acc[i][j].im);
        }
    }
}

// ----------------------------------------------------------------- P2M ----
// mp[leaf][r] = sum_{pos in leaf} W[pos][r] x[perm[pos]]
// (blockIdx.y = right-hand side: x and mp advance by xstride / mstride)
template <class R>
__global__ void k_p2m(int P, const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ perm,
                      const cx<R>* __restrict__ W, const cd* __restrict__ x, cx<R>* __restrict__ mp,
                      int64_t xstride, int64_t mstride) {
    x += blockIdx.y * xstride;
    mp += blockIdx.y * mstride;
    int b = blockIdx.x;
    int s0 = leaf_start[b], s1 = leaf_start[b + 1];
    __shared__ cx<R> xs[256];
    for (int r0 = 0; r0 < P; r0 += blockDim.x) {
        int r = r0 + threadIdx.x;
        cx<R> acc = mk<R>(0, 0);
        for (int c0 = s0; c0 < s1; c0 += 256) {
            int cn = min(256, s1 - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < cn; i += blockDim.x) xs[i] = from_d<R>(x[perm[c0 + i]]);
            __syncthreads();
            if (r < P)
                for (int i = 0; i < cn; ++i) cmac(acc, W[(int64_t)(c0 + i) * P + r], xs[i]);
        }
        if (r < P) mp[(int64_t)b * P + r] = acc;
    }
}

// ----------------------------------------------------- near field + L2P ----
// y[perm[pos]] = sum_c A_t[row][c] x[col c] + sum_r V[pos][r] loc[leaf][r]
// for up to NB right-hand sides per CTA (blockIdx.y selects the chunk): each
// near-field and L2P entry is read once and applied to every right-hand side
// of the chunk.  x, y advance by xstride per rhs, loc by lstride.
// A near-field entry as stored: complex FP32 / FP64, or a BF16 pair (real
// part in the low, imaginary part in the high 16 bits; BF16 is the upper
// half of an FP32 word).
__device__ __forceinline__ cf nf_entry(const cf& a) { return a; }
__device__ __forceinline__ cd nf_entry(const cd& a) { return a; }
__device__ __forceinline__ cf nf_entry(uint32_t a) {
    return mk(__uint_as_float(a << 16), __uint_as_float(a & 0xFFFF0000u));
}

template <class R, int NB, class AS = cx<R>>
__global__ void k_near_l2p(int P, const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ ucnt, const int32_t* __restrict__ ulist,
                           const int64_t* __restrict__ nf_off, const int32_t* __restrict__ nf_ncol,
                           const AS* __restrict__ A, const cx<R>* __restrict__ V,
                           const cx<R>* __restrict__ loc, const cd* __restrict__ x, cd* __restrict__ y,
                           int nrhs, int64_t xstride, int64_t lstride) {
    extern __shared__ unsigned char smem_raw[];
    const int r0 = blockIdx.y * NB;
    const int nr = min(NB, nrhs - r0);
    cx<R>* xs = (cx<R>*)smem_raw;       // [nr][K]
    int t = blockIdx.x;
    int K = nf_ncol[t];
    cx<R>* ls = xs + nr * K;            // [nr][P]
    // gather the x values of the U-list leaves in column order
    int nu = ucnt[t];
    int c = 0;
    for (int i = 0; i < nu; ++i) {
        int s = ulist[(int64_t)t * FB_ULIST + i];
        int a0 = leaf_start[s], a1 = leaf_start[s + 1];
        for (int q = threadIdx.x; q < a1 - a0; q += blockDim.x) {
            int e = perm[a0 + q];
            for (int j = 0; j < nr; ++j) xs[j * K + c + q] = from_d<R>(x[(r0 + j) * xstride + e]);
        }
        c += a1 - a0;
    }
    if (loc)
        for (int j = 0; j < nr; ++j)
            for (int q = threadIdx.x; q < P; q += blockDim.x)
                ls[j * P + q] = loc[(r0 + j) * lstride + (int64_t)t * P + q];
    __syncthreads();
    int rb = leaf_start[t], nrow = leaf_start[t + 1] - rb;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const AS* At = A + nf_off[t];
    for (int r = warp; r < nrow; r += nw) {
        cx<R> acc[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = mk<R>(0, 0);
        const AS* row = At + (int64_t)r * K;
        // unrolled: several independent row loads in flight per lane
#pragma unroll 4
        for (int q = lane; q < K; q += 32) {
            const cx<R> a = nf_entry(row[q]);
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < nr) cmac(acc[j], a, xs[j * K + q]);
        }
        if (loc) {
            const cx<R>* vr = V + (int64_t)(rb + r) * P;
            for (int q = lane; q < P; q += 32) {
                cx<R> v = vr[q];
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j < nr) cmac(acc[j], v, ls[j * P + q]);
            }
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[j].re += __shfl_xor_sync(0xffffffffu, acc[j].re, o);
                acc[j].im += __shfl_xor_sync(0xffffffffu, acc[j].im, o);
            }
        }
        if (lane == 0) {
            int e = perm[rb + r];
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < nr) y[(r0 + j) * xstride + e] = mk<double>((double)acc[j].re, (double)acc[j].im);
        }
    }
}


// ------------------------------------------------------- RCR translation ----
// Rotation - coaxial translation - back-rotation (Sec. 3.3) applied per box
// pair: for a group of pairs sharing one translation vector (one direction,
// one |t|) each CTA takes nb pairs.  The rotations run folded by the
// symmetry of the real factors, d^n_{-mu,-m} = d^n_{mu,m}: with the phased
// input x_m = e^{i m phi} src_m and s_m = x_m + x_{-m}, t_m = x_m - x_{-m}
// (m > 0), s_0 = x_0,
//   E_mu = u_mu + u_{-mu} = 2 d_{mu,0} s_0 + sum_{m>0} (d_{mu,m} + d_{mu,-m}) s_m   (mu = 0..n)
//   O_mu = u_mu - u_{-mu} =                  sum_{m>0} (d_{mu,m} - d_{mu,-m}) t_m   (mu = 1..n)
// (half the multiplications of u = d x); the coaxial blocks, which depend
// on |m| only, map E to E and O to O; the back-rotation folds the same way,
//   Y+_{m'} = y_{m'} + y_{-m'} = d_{0,m'} E_0 + sum_{mu>0} (d_{mu,m'} + d_{-mu,m'}) E_mu
//   Y-_{m'} = y_{m'} - y_{-m'} =               sum_{mu>0} (d_{mu,m'} - d_{-mu,m'}) O_mu
// and y_{+-m'} = (Y+ +- Y-)/2, e^{-+ i m' phi} applied, scatter-added into the
// target (atomic adds: the groups of one launch may share targets).  Folded
// layout of degree n within a vector: [0..n] even part, [n+1..2n] odd part.
__device__ __forceinline__ void nm_of(int e, int& n, int& m) {
    n = (int)sqrtf((float)e);
    while (n * n > e) --n;
    while ((n + 1) * (n + 1) <= e) ++n;
    m = e - n * n - n;
}
// (n, j) of a folded degree-major index e = n^2 + j, j in [0, 2n]
__device__ __forceinline__ void nj_of(int e, int& n, int& j) {
    nm_of(e, n, j);
    j += n;
}
// pair index e -> (n1, m') for m' = 0..n1 (e = n1 (n1 + 1) / 2 + m')
__device__ __forceinline__ void tri_of(int e, int& n, int& m) {
    n = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (n * (n + 1) / 2 > e) --n;
    while ((n + 1) * (n + 2) / 2 <= e) ++n;
    m = e - n * (n + 1) / 2;
}

// Each thread owns one (folded) coefficient and computes it for a chunk of W
// pairs at once, so every rotation / coaxial entry it loads is used W times
// from registers; the pair operands come from shared memory, where the
// threads of a warp that share a degree read the same word (broadcast).
// Full chunks use W = RcrChunk, the remainder of a tile one pair at a time.
template <class R> struct RcrChunk { static constexpr int value = 8; };
template <> struct RcrChunk<double> { static constexpr int value = 4; };
template <> struct RcrChunk<df> { static constexpr int value = 4; };
// CTAs per SM the register budget must allow: FP64 tiles (48 KB of shared
// memory each) are latency bound and want four resident CTAs, FP32 tiles
// (96 KB) fit two.
template <class R> struct RcrMinBlocks { static constexpr int value = 2; };
template <> struct RcrMinBlocks<double> { static constexpr int value = 4; };
template <> struct RcrMinBlocks<df> { static constexpr int value = 4; };

// acc += a x for real a
template <class R>
__device__ __forceinline__ void rmac(cx<R>& acc, R a, const cx<R>& x) {
    acc.re = fma(a, x.re, acc.re);
    acc.im = fma(a, x.im, acc.im);
}

// folded rotation of degree n, output j (E_j for j <= n, O_{j-n} otherwise);
// Dc points at d_{0,0} of the degree-n block (row stride w = 2n + 1)
template <int W, class R>
__device__ __forceinline__ void rcr_rotate(const R* Dc, int n, int j, const cx<R>* xs, int Pin, int b0, int e,
                                           cx<R>* us) {
    cx<R> acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = mk<R>(0, 0);
    const int w = 2 * n + 1;
    const cx<R>* xb = xs + b0 * Pin + n * n;
    if (j <= n) {
        const R* row = Dc + (int64_t)j * w;
        {
            const R a = R(2) * row[0];
#pragma unroll
            for (int q = 0; q < W; ++q) rmac(acc[q], a, xb[q * Pin]);
        }
#pragma unroll 4
        for (int m = 1; m <= n; ++m) {
            const R a = row[m] + row[-m];
#pragma unroll
            for (int q = 0; q < W; ++q) rmac(acc[q], a, xb[q * Pin + m]);
        }
    } else {
        const R* row = Dc + (int64_t)(j - n) * w;
#pragma unroll 4
        for (int m = 1; m <= n; ++m) {
            const R a = row[m] - row[-m];
#pragma unroll
            for (int q = 0; q < W; ++q) rmac(acc[q], a, xb[q * Pin + n + m]);
        }
    }
#pragma unroll
    for (int q = 0; q < W; ++q) us[(b0 + q) * Pin + e] = acc[q];
}

// coaxial step on folded data: output (n1, j1) of order am (even or odd part)
// input of degree n at n^2 + withn * n + a: folded even part (withn = 0,
// a = am), folded odd part (1, am), or unfolded order mu (1, mu)
template <int W, class R>
__device__ __forceinline__ void rcr_coax(const cx<R>* Cr, int am, int withn, int a, int pmid, const cx<R>* us,
                                         int Pin, int Pout, int b0, int e, cx<R>* vs) {
    cx<R> acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = mk<R>(0, 0);
    const cx<R>* ub = us + b0 * Pin;
#pragma unroll 4
    for (int n = am; n < pmid; ++n) {
        cx<R> c = Cr[n];
        int o = n * n + withn * n + a;
#pragma unroll
        for (int q = 0; q < W; ++q) cmac(acc[q], c, ub[q * Pin + o]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) vs[(b0 + q) * Pout + e] = acc[q];
}

// folded back-rotation of degree n1 for the output pair +-m' (m' >= 0),
// inner range |mu| <= mmax; Dc at d_{0,0} of the degree-n1 block
template <int W, class R>
__device__ __forceinline__ void rcr_back(const R* Dc, int n1, int mp, int mmax, cx<R> ph, const cx<R>* vs,
                                         int Pout, int b0, const int64_t* dsto, cx<R>* dst) {
    cx<R> yp[W], ym[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        yp[q] = mk<R>(0, 0);
        ym[q] = mk<R>(0, 0);
    }
    const int w = 2 * n1 + 1;
    const cx<R>* vb = vs + b0 * Pout + n1 * n1;
    {
        const R a = Dc[mp];
#pragma unroll
        for (int q = 0; q < W; ++q) rmac(yp[q], a, vb[q * Pout]);
    }
#pragma unroll 4
    for (int mu = 1; mu <= mmax; ++mu) {
        const R dp = Dc[(int64_t)mu * w + mp], dm = Dc[-(int64_t)mu * w + mp];
        const R ap = dp + dm, am = dp - dm;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            rmac(yp[q], ap, vb[q * Pout + mu]);
            rmac(ym[q], am, vb[q * Pout + n1 + mu]);
        }
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
        cx<R>* d = dst + dsto[b0 + q] + n1 * n1 + n1;
        if (mp == 0) {
            const cx<R> y = R(0.5) * yp[q];
            atomicAdd(&d->re, y.re);
            atomicAdd(&d->im, y.im);
        } else {
            const cx<R> y1 = (R(0.5) * (yp[q] + ym[q])) * conjg(ph);
            const cx<R> y2 = (R(0.5) * (yp[q] - ym[q])) * ph;
            atomicAdd(&d[mp].re, y1.re);
            atomicAdd(&d[mp].im, y1.im);
            atomicAdd(&d[-mp].re, y2.re);
            atomicAdd(&d[-mp].im, y2.im);
        }
    }
}

// Unfolded forms (u = d x over all m, each output m' on its own), used by the
// FP64 tiles: they are bound by FP64 latency rather than multiplies, and the
// folded form's wider per-thread state costs them more than it saves.
template <int W, class R>
__device__ __forceinline__ void rcr_rotate_full(const R* dn, int n, const cx<R>* xs, int Pin, int b0, int e,
                                                cx<R>* us) {
    cx<R> acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = mk<R>(0, 0);
    const cx<R>* xb = xs + b0 * Pin + n * n;
#pragma unroll 4
    for (int m = 0; m <= 2 * n; ++m) {
        R d = dn[m];
#pragma unroll
        for (int q = 0; q < W; ++q) rmac(acc[q], d, xb[q * Pin + m]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) us[(b0 + q) * Pin + e] = acc[q];
}
template <int W, class R, class O>
__device__ __forceinline__ void rcr_back_full(const R* dn, int n1, cx<O> phc, const cx<R>* vs, int Pout, int b0,
                                              int e, const int64_t* dsto, cx<O>* dst) {
    cx<R> acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = mk<R>(0, 0);
    int w = 2 * n1 + 1;
    const cx<R>* vb = vs + b0 * Pout + n1 * n1;
#pragma unroll 4
    for (int mu = 0; mu < w; ++mu) {
        R d = dn[(int64_t)mu * w];
#pragma unroll
        for (int q = 0; q < W; ++q) rmac(acc[q], d, vb[q * Pout + mu]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
        cx<O> y = cx_out<O, R>(acc[q]) * phc;
        cx<O>* d = dst + dsto[b0 + q] + e;
        atomicAdd(&d->re, y.re);
        atomicAdd(&d->im, y.im);
    }
}

// R: arithmetic and tables (rotd, coax), O: expansions and phases (R = O,
// or R = double-FP32 on FP64 expansions); rot_stride: values per direction
// in rotd.
template <class R, class O>
__global__ void __launch_bounds__(256, RcrMinBlocks<R>::value) k_rcr(const RcrTask* __restrict__ tasks, const RcrTile* __restrict__ tiles,
                                             const R* __restrict__ rotd, const cx<O>* __restrict__ rph,
                                             int64_t per_dir, int64_t rot_stride, int prot,
                                             const cx<R>* __restrict__ coax,
                                             const int32_t* __restrict__ src_idx,
                                             const int32_t* __restrict__ dst_idx,
                                             const cx<O>* __restrict__ src, cx<O>* __restrict__ dst,
                                             int nrhs, int64_t rstride) {
    constexpr int BCH = RcrChunk<R>::value;
    constexpr bool kFold = sizeof(R) == 4;   // FP32: folded rotations; FP64, double-FP32: unfolded
    extern __shared__ unsigned char smem_raw[];
    __shared__ int64_t s_dst_off[16];
    RcrTile tl = tiles[blockIdx.x];
    RcrTask tk = tasks[tl.task];
    const int nb = tl.nb;
    const int Pin = tk.p_in * tk.p_in, Pout = tk.p_out * tk.p_out;
    const int pmid = tk.p_in;   // the rotated input keeps degrees n < p_in
    cx<R>* buf = (cx<R>*)smem_raw;
    cx<R>* xs = buf;                    // [nb][Pin] folded phased input, later reused for vs
    cx<R>* us = buf + nb * max(Pin, Pout);   // [nb][Pin]
    cx<R>* vs = buf;                    // [nb][Pout] (xs is dead after the rotation)
    int tid = threadIdx.x, nth = blockDim.x;
    // column b of the tile: pair (col0 + b) / nrhs, right-hand side (col0 + b) % nrhs
    for (int b = tid; b < nb; b += nth) {
        int col = tl.col0 + b;
        int pr = col / nrhs, rh = col - pr * nrhs;
        s_dst_off[b] = rh * rstride + tk.dst_base + (int64_t)dst_idx[tk.pair_off + pr] * Pout;
    }
    const int64_t dir = tk.rot_off / per_dir;
    const cx<O>* ph = rph + dir * (2 * prot - 1) + (prot - 1);   // ph[m] = e^{i m phi}
    for (int q = tid; q < nb * Pin; q += nth) {
        int b = q / Pin, e = q % Pin;
        int col = tl.col0 + b;
        int pr = col / nrhs, rh = col - pr * nrhs;
        int sb = src_idx[tk.pair_off + pr];
        int n, j;
        nj_of(e, n, j);
        const cx<O>* x = src + rh * rstride + tk.src_base + (int64_t)sb * Pin + (int64_t)n * n + n;   // (n, 0)
        cx<O> v;
        if constexpr (!kFold) {
            v = x[j - n] * ph[j - n];   // plain phased input, degree-major
        } else if (j == 0) {
            v = x[0];
        } else {
            const int m = j <= n ? j : j - n;
            const cx<O> xp = x[m] * ph[m], xm = x[-m] * ph[-m];
            v = j <= n ? xp + xm : xp - xm;
        }
        xs[q] = cx_to<R, O>(v);
    }
    __syncthreads();
    const R* D = rotd + dir * rot_stride;
    // chunk widths BCH, then 4, 2, 1 for the rest of the tile
#define RCR_CHUNKS(CALL)                                              \
    {                                                                 \
        int b0 = 0;                                                   \
        for (; b0 + BCH <= nb; b0 += BCH) CALL(BCH);                  \
        if (BCH > 4 && b0 + 4 <= nb) { CALL(4); b0 += 4; }            \
        if (b0 + 2 <= nb) { CALL(2); b0 += 2; }                       \
        if (b0 < nb) CALL(1);                                         \
    }
    // rotation: folded E_j / O_{j-n}, or u_{n,mu} = sum_m d_{mu,m} x_m unfolded
    for (int e = tid; e < Pin; e += nth) {
        int n, j;
        nj_of(e, n, j);
        const R* Dc = D + (int64_t)n * (2 * n - 1) * (2 * n + 1) / 3 + (int64_t)n * (2 * n + 1) + n;
        if constexpr (kFold) {
#define RCR_ROT(W) rcr_rotate<(W)>(Dc, n, j, xs, Pin, b0, e, us)
            RCR_CHUNKS(RCR_ROT)
#undef RCR_ROT
        } else {
            const R* Dn = Dc + (int64_t)(j - n) * (2 * n + 1) - n;   // row mu = j - n
#define RCR_ROT(W) rcr_rotate_full<(W)>(Dn, n, xs, Pin, b0, e, us)
            RCR_CHUNKS(RCR_ROT)
#undef RCR_ROT
        }
    }
    __syncthreads();
    // coaxial: v^{am}_{n'} = sum_n C^{am}_{n'n} u^{am}_n on the even and odd parts
    const cx<R>* C = coax + tk.coax_off;
    const int pc = tk.pc;
    for (int e = tid; e < Pout; e += nth) {
        int n1, j1;
        nj_of(e, n1, j1);
        // folded: even part of order j1 or odd part of order j1 - n1; unfolded:
        // order mu = j1 - n1 at offset n^2 + n + mu
        const bool odd = kFold && j1 > n1;
        const int am = kFold ? (odd ? j1 - n1 : j1) : abs(j1 - n1);
        const int withn = (kFold && !odd) ? 0 : 1;
        const int a = kFold ? am : j1 - n1;
        const cx<R>* Cr = C + ((int64_t)am * pc + n1) * pc;
        const int hi = am < pmid ? pmid : am;   // empty sum when |mu| >= p_in
#define RCR_COAX(W) rcr_coax<(W)>(Cr, am, withn, a, hi, us, Pin, Pout, b0, e, vs)
        RCR_CHUNKS(RCR_COAX)
#undef RCR_COAX
    }
    __syncthreads();
    if constexpr (!kFold) {
        // back-rotate: y_{n'}^{m'} = sum_mu d^{n'}_{mu,m'} v_{n'}^mu, e^{-i m' phi}, scatter-add
        for (int e = tid; e < Pout; e += nth) {
            int n1, m1;
            nm_of(e, n1, m1);
            const R* Dn = D + (int64_t)n1 * (2 * n1 - 1) * (2 * n1 + 1) / 3 + (m1 + n1);
            const cx<O> phc = conjg(ph[m1]);
#define RCR_BACK(W) rcr_back_full<(W)>(Dn, n1, phc, vs, Pout, b0, e, s_dst_off, dst)
            RCR_CHUNKS(RCR_BACK)
#undef RCR_BACK
        }
    } else {
        // folded back-rotation of every pair +-m' of every degree n' < p_out, then scatter-add
        const int npairs_out = tk.p_out * (tk.p_out + 1) / 2;
        for (int e = tid; e < npairs_out; e += nth) {
            int n1, mp;
            tri_of(e, n1, mp);
            const R* Dc = D + (int64_t)n1 * (2 * n1 - 1) * (2 * n1 + 1) / 3 + (int64_t)n1 * (2 * n1 + 1) + n1;
            const int mmax = min(n1, pmid - 1);
            const cx<R> phm = ph[mp];
#define RCR_BACK(W) rcr_back<(W)>(Dc, n1, mp, mmax, phm, vs, Pout, b0, s_dst_off, dst)
            RCR_CHUNKS(RCR_BACK)
#undef RCR_BACK
        }
    }
#undef RCR_CHUNKS
}

// Tiles of up to 16 columns per CTA within a shared-memory budget: 96 KB for
// FP32 (two CTAs per SM; the columns of a tile reuse each rotation / coaxial
// entry from registers, so larger tiles raise the arithmetic per load) and
// 48 KB for FP64 (bound by the FP64 pipe, it wants more resident warps).
// Tasks of large order are left to the staged passes (fb_stg_staged).
// want_df: the tiles of the tasks in double-FP32 arithmetic (staged == 4),
// else the others.
static void rcr_make_tiles(const RcrPlan& pl, int nrhs, std::vector<RcrTile>& tiles, size_t& smem,
                           bool want_df = false) {
    const size_t budget = pl.csize == sizeof(cf) ? 96 * 1024 : 48 * 1024;
    tiles.clear();
    smem = 0;
    for (int t = 0; t < (int)pl.h_tasks.size(); ++t) {
        const RcrTask& tk = pl.h_tasks[t];
        if (fb_stg_staged(tk) || (tk.staged == 4) != want_df) continue;
        int64_t elems = (int64_t)tk.p_in * tk.p_in + std::max(tk.p_in * tk.p_in, tk.p_out * tk.p_out);
        size_t per = (size_t)elems * pl.csize;
        int nb = (int)std::max<size_t>(1, std::min<size_t>(16, budget / per));
        int ncol = tk.npairs * nrhs;
        for (int c = 0; c < ncol; c += nb) {
            int k = std::min(nb, ncol - c);
            tiles.push_back(RcrTile{t, c, k, 0});
            smem = std::max(smem, per * k);
        }
    }
}

static fb_status rcr_tiles_for(RcrPlan& pl, int nrhs, RcrTileSet* out, bool want_df = false) {
    if (nrhs == 1) {
        if (want_df) {
            *out = pl.df_tiles;
            return FB_OK;
        }
        out->tiles = pl.tiles;
        out->ntiles = pl.ntiles;
        out->smem = pl.smem;
        return FB_OK;
    }
    auto it = pl.multi.find(2 * nrhs + (want_df ? 1 : 0));
    if (it == pl.multi.end()) {
        std::vector<RcrTile> h;
        RcrTileSet ts;
        rcr_make_tiles(pl, nrhs, h, ts.smem, want_df);
        ts.ntiles = (int)h.size();
        if (!h.empty()) {
            FB_CHECK(dalloc(&ts.tiles, h.size()));
            FB_CUDA(cudaMemcpy(ts.tiles, h.data(), sizeof(RcrTile) * h.size(), cudaMemcpyHostToDevice));
        }
        it = pl.multi.emplace(2 * nrhs + (want_df ? 1 : 0), ts).first;
    }
    *out = it->second;
    return FB_OK;
}

// Rotation data of an operator for the RCR kernels: real factors, phase
// tables and their strides.
template <class R>
struct RotArgs {
    const R* d;
    const cx<R>* ph;
    int64_t per_dir;
    int prot;
    cx<R>* U;   // staging buffers of the large-order passes
    cx<R>* V;
    const void* rf;   // folded rotation tables and their per-group stride
    int64_t fper;
    StcTabs tc;       // tables of the tensor-core staged passes (single precision)
    DfTabs dft;       // tables of the double-FP32 staged passes (FP64 operators)
    const df* d_df;   // real factors in double-FP32 (degrees < the tiles' largest order)
    int64_t per_dir_df;
};
template <class R>
static RotArgs<R> rot_args(const fb_op* op) {
    RotArgs<R> a;
    a.d = (const R*)(sizeof(R) == 8 ? (const void*)op->rotd64 : (const void*)op->rotd32);
    a.ph = (const cx<R>*)(sizeof(R) == 8 ? (const void*)op->rph64 : (const void*)op->rph32);
    a.per_dir = op->per_dir;
    a.prot = op->Prot;
    a.U = (cx<R>*)op->stg_u;
    a.V = (cx<R>*)op->stg_v;
    a.rf = op->rotf;
    a.fper = op->rotf_per;
    a.tc = StcTabs{op->stc_tab, op->stc_off, op->stc_per, op->stc_err};
    a.dft = DfTabs{op->rotf_df, op->coax_df};
    a.d_df = op->rotd_df;
    a.per_dir_df = op->rotd_df_per;
    return a;
}
static fb_status stg_run(void* plan, const RotArgs<float>& r, const cf* coax, const cf* src, cf* dst,
                         cudaStream_t s, int nrhs, int64_t rstride) {
    return fb_stg_run_f(plan, (const float*)r.rf, r.fper, r.ph, r.prot, coax, src, dst, r.U, r.V, s, nrhs, rstride,
                        r.tc);
}
static fb_status stg_run(void* plan, const RotArgs<double>& r, const cd* coax, const cd* src, cd* dst,
                         cudaStream_t s, int nrhs, int64_t rstride) {
    return fb_stg_run_d(plan, (const double*)r.rf, r.fper, r.ph, r.prot, coax, src, dst, r.U, r.V, s, nrhs, rstride,
                        r.dft);
}

// Device time (ms, median of 3 after one untimed run, one right-hand side)
// of each pass of every staged M2L level of an operator, on its expansion
// buffers: ms[4 l + {0..3}] = pre-pass, rotation, coaxial, back-rotation of
// level l (-1: not staged); form[l] = 1 CUDA cores, 2 rotations on the
// tensor cores, 3 double-FP32 arithmetic, 5 rotations and coaxial step on
// the tensor cores (0: not staged).
fb_status fb_stg_op_pass_times(fb_op* op, cudaStream_t s, double* ms, int* tc) {
    for (int i = 0; i < 4 * (FB_MAXLEV + 1); ++i) ms[i] = -1.0;
    for (int l = 0; l <= FB_MAXLEV; ++l) tc[l] = 0;
    const bool mixed = op->prec == FB_PREC_MIXED_FMM;
    RcrPlan& pl = (mixed && op->method == FB_TRANS_AUTO && op->tc_plan) ? op->m2l_rcr_rest : op->m2l_rcr;
    if (!pl.stg || !op->mp || !op->loc) return FB_OK;
    cudaEvent_t e0, e1;
    FB_CUDA(cudaEventCreate(&e0));
    FB_CUDA(cudaEventCreate(&e1));
    fb_status st = FB_OK;
    for (int li = 0; li < fb_stg_level_count(pl.stg) && st == FB_OK; ++li) {
        int64_t sb = 0, db = 0;
        int t = 0;
        fb_stg_level_info(pl.stg, li, &sb, &db, &t);
        int lev = -1;
        for (int l = 2; l <= op->L; ++l)
            if (op->lev_off[l] == sb) lev = l;
        if (lev < 0 || sb != db) continue;
        tc[lev] = t;
        for (int pass = 0; pass < 4 && st == FB_OK; ++pass) {
            if (pass == 0 && (t == 2 || t == 5)) continue;   // the tensor-core rotation pass folds its inputs
            auto run = [&]() {
                return mixed ? fb_stg_run_f(pl.stg, (const float*)op->rotf, op->rotf_per, (const cf*)op->rph32,
                                            op->Prot, op->coax32, (const cf*)op->mp, (cf*)op->loc, (cf*)op->stg_u,
                                            (cf*)op->stg_v, s, 1, 0, rot_args<float>(op).tc, li, 1 << pass)
                             : fb_stg_run_d(pl.stg, (const double*)op->rotf, op->rotf_per, (const cd*)op->rph64,
                                            op->Prot, op->coax64, (const cd*)op->mp, (cd*)op->loc, (cd*)op->stg_u,
                                            (cd*)op->stg_v, s, 1, 0, rot_args<double>(op).dft, li, 1 << pass);
            };
            std::vector<float> v;
            st = run();
            for (int r = 0; r < 3 && st == FB_OK; ++r) {
                cudaEventRecord(e0, s);
                st = run();
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = fb_fail(FB_ERR_CUDA, "staged pass timing failed");
                float x = 0.f;
                cudaEventElapsedTime(&x, e0, e1);
                v.push_back(x);
            }
            if (st == FB_OK) {
                std::sort(v.begin(), v.end());
                ms[4 * lev + pass] = v[1];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

template <class R>
static fb_status run_rcr(RcrPlan& pl, const RotArgs<R>& rot, const cx<R>* coax, const cx<R>* src, cx<R>* dst,
                         cudaStream_t s, int nrhs = 1, int64_t rstride = 0) {
    RcrTileSet ts;
    FB_CHECK(rcr_tiles_for(pl, nrhs, &ts));
    if (ts.ntiles > 0) {
        FB_CHECK(fb_smem_cap((const void*)k_rcr<R, R>, ts.smem));
        k_rcr<R, R><<<ts.ntiles, 256, ts.smem, s>>>(pl.tasks, ts.tiles, rot.d, rot.ph, rot.per_dir, rot.per_dir,
                                                    rot.prot, coax, pl.src_idx, pl.dst_idx, src, dst, nrhs, rstride);
        FB_LAUNCH_CHECK();
        fb_count_launch();
    }
    if constexpr (sizeof(R) == 8) {
        // tiles in double-FP32 arithmetic on the FP64 expansions
        FB_CHECK(rcr_tiles_for(pl, nrhs, &ts, true));
        if (ts.ntiles > 0) {
            if (!rot.d_df || !rot.dft.coax) return fb_fail(FB_ERR_STATE, "RCR tiles: double-FP32 tables missing");
            FB_CHECK(fb_smem_cap((const void*)k_rcr<df, double>, ts.smem));
            k_rcr<df, double><<<ts.ntiles, 256, ts.smem, s>>>(pl.tasks, ts.tiles, rot.d_df, rot.ph, rot.per_dir,
                                                              rot.per_dir_df, rot.prot, rot.dft.coax, pl.src_idx,
                                                              pl.dst_idx, src, dst, nrhs, rstride);
            FB_LAUNCH_CHECK();
            fb_count_launch();
        }
    }
    if (pl.stg) FB_CHECK(stg_run(pl.stg, rot, coax, src, dst, s, nrhs, rstride));
    return FB_OK;
}

static __global__ void k_d_to_df(const double* __restrict__ in, int64_t per_in, int64_t per_out, int ndir,
                                 df* __restrict__ out) {
    const int64_t total = (int64_t)ndir * per_out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i / per_out, e = i - d * per_out;
        out[i] = df_from(in[d * per_in + e]);
    }
}

// Real rotation factors of every direction in double-FP32, degrees < P (the
// largest order of the tiles that use them), rebuilt when a larger P is asked.
fb_status fb_rcr_df_factors(fb_op* op, int P) {
    if (op->rotd_df && op->rotd_df_P >= P) return FB_OK;
    if (!op->rotd64 || P > op->Prot) return fb_fail(FB_ERR_STATE, "RCR tiles: no FP64 rotation factors");
    const int ndir = (int)(op->rot_count / op->per_dir);
    const int64_t per = (int64_t)P * (2 * P - 1) * (2 * P + 1) / 3;   // sum_{n<P} (2n+1)^2
    FB_CUDA(cudaDeviceSynchronize());
    dfree(op->rotd_df);
    FB_CHECK(dalloc(&op->rotd_df, (size_t)ndir * per));
    k_d_to_df<<<(unsigned)std::min<int64_t>(((int64_t)ndir * per + 255) / 256, 8192), 256>>>(op->rotd64, op->per_dir,
                                                                                          per, ndir, op->rotd_df);
    FB_CUDA(cudaDeviceSynchronize());
    op->rotd_df_P = P;
    op->rotd_df_per = per;
    op->buf_gen++;   // captured graphs refer to the old factors
    fb_count_launch();
    return FB_OK;
}

// Uploads an RCR plan: per-pair tiles for the tasks of moderate order and the
// staged passes of the large-order ones, whose staging buffers (shared by
// every plan of the operator: the passes of one matvec run one after the
// other) grow to the largest level's need.
fb_status fb_rcr_upload(fb_op* op, RcrPlan& pl, const int32_t* src, const int32_t* dst, size_t csize) {
    pl.src_idx = src;
    pl.dst_idx = dst;
    pl.csize = csize;
    for (const RcrTask& tk : pl.h_tasks) {
        if ((tk.staged == 2 || tk.staged == 5) && op->prec != FB_PREC_MIXED_FMM)
            return fb_fail(FB_ERR_ARG, "tensor-core staged RCR applies to mixed operators");
        if ((tk.staged == 3 || tk.staged == 4) && op->prec != FB_PREC_FP64_FMM)
            return fb_fail(FB_ERR_ARG, "double-FP32 RCR applies to FP64 operators");
    }
    // a pair whose working set does not fit one CTA can only run staged
    for (RcrTask& tk : pl.h_tasks)
        if ((tk.staged == 0 || tk.staged == 4) && !fb_rcr_tile_fits(tk.p_in, tk.p_out, csize))
            tk.staged = tk.staged == 4 ? 3 : 1;
    rcr_make_tiles(pl, 1, pl.h_tiles, pl.smem);
    pl.ntiles = (int)pl.h_tiles.size();
    if (pl.h_tasks.empty()) return FB_OK;
    FB_CHECK(dalloc(&pl.tasks, pl.h_tasks.size()));
    FB_CUDA(cudaMemcpy(pl.tasks, pl.h_tasks.data(), sizeof(RcrTask) * pl.h_tasks.size(), cudaMemcpyHostToDevice));
    if (pl.ntiles) {
        FB_CHECK(dalloc(&pl.tiles, pl.h_tiles.size()));
        FB_CUDA(cudaMemcpy(pl.tiles, pl.h_tiles.data(), sizeof(RcrTile) * pl.h_tiles.size(), cudaMemcpyHostToDevice));
    }
    {
        std::vector<RcrTile> h;
        rcr_make_tiles(pl, 1, h, pl.df_tiles.smem, true);
        pl.df_tiles.ntiles = (int)h.size();
        if (!h.empty()) {
            int pmax = 0;
            for (const RcrTask& tk : pl.h_tasks)
                if (tk.staged == 4) pmax = std::max(pmax, std::max(tk.p_in, tk.p_out));
            FB_CHECK(fb_rcr_df_factors(op, pmax));
            FB_CHECK(fb_stg_df_tables(op, cudaStreamLegacy));   // coaxial sets in double-FP32
            FB_CHECK(dalloc(&pl.df_tiles.tiles, h.size()));
            FB_CUDA(cudaMemcpy(pl.df_tiles.tiles, h.data(), sizeof(RcrTile) * h.size(), cudaMemcpyHostToDevice));
        }
    }
    FB_CHECK(fb_stg_build(pl, op->theta_slot, op->per_dir, op->coax64, &pl.stg, &pl.stg_elems));
    if (fb_stg_uses_tc(pl.stg)) FB_CHECK(fb_stc_tables(op, cudaStreamLegacy));
    if (fb_stg_uses_df(pl.stg)) FB_CHECK(fb_stg_df_tables(op, cudaStreamLegacy));
    if (pl.stg_elems > op->stg_elems) {
        FB_CUDA(cudaDeviceSynchronize());
        dfree(op->stg_u);
        dfree(op->stg_v);
        op->stg_elems = 0;
        FB_CHECK(dalloc((unsigned char**)&op->stg_u, (size_t)pl.stg_elems * csize));
        FB_CHECK(dalloc((unsigned char**)&op->stg_v, (size_t)pl.stg_elems * csize));
        op->stg_elems = pl.stg_elems;
        op->buf_gen++;   // captured graphs refer to the old buffers
    }
    return FB_OK;
}

template <class R>
static fb_status run_plan(const TransPlan& pl, const cx<R>* T, const cx<R>* src, cx<R>* dst, cudaStream_t s) {
    if (pl.ntiles == 0) return FB_OK;
    k_trans<R><<<pl.ntiles, 256, 0, s>>>(pl.tasks, pl.tiles, T, pl.src_idx, pl.dst_idx, src, dst);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

// One FMM matvec for nrhs right-hand sides (x, y: nrhs x N, rhs-major).  The
// expansions of rhs r sit at mp / loc + r * cnt; every kernel handles all
// right-hand sides in one launch, so the near-field entries, the P2M / L2P
// operators and every translation operator are read once per matvec.
template <class R>
static fb_status fmm_apply_t(fb_op* op, const cd* x, cd* y, cudaStream_t s, const cx<R>* A,
                             const cx<R>* W, const cx<R>* V, const cx<R>* T, PhaseTimer* pt,
                             void* scratch = nullptr, int nrhs = 1) {
    auto mark = [&](int i) { if (pt) cudaEventRecord(pt->ev[i], s); };
    const fb_tree* t = op->tree;
    int L = op->L;
    int pL = op->p[L], PL = pL * pL;
    int64_t cnt = op->lev_off[L + 1];
    const int64_t n = op->n;
    const bool composed = op->method == FB_TRANS_COMPOSED;
    if (composed && nrhs > 1) {   // the composed SIMT path takes one right-hand side at a time
        for (int r = 0; r < nrhs; ++r)
            FB_CHECK(fmm_apply_t<R>(op, x + r * n, y + r * n, s, A, W, V, T, r == 0 ? pt : nullptr, scratch, 1));
        return FB_OK;
    }
    // expansions: the operator's own buffers (grown to nrhs sets), or a
    // caller-provided region holding the multipoles followed by the locals
    if (!scratch && nrhs > op->exp_nrhs) {
        cudaStreamSynchronize(s);
        dfree(op->mp);
        dfree(op->loc);
        op->mp = nullptr;
        op->loc = nullptr;
        FB_CHECK(dalloc((cx<R>**)&op->mp, cnt * nrhs));
        FB_CHECK(dalloc((cx<R>**)&op->loc, cnt * nrhs));
        op->exp_nrhs = nrhs;
        op->buf_gen++;   // captured graphs of this operator refer to the old buffers
    }
    cx<R>* mp = scratch ? (cx<R>*)scratch : (cx<R>*)op->mp;
    cx<R>* loc = scratch ? (cx<R>*)scratch + cnt * nrhs : (cx<R>*)op->loc;
    mark(0);
    FB_CUDA(cudaMemsetAsync(mp, 0, sizeof(cx<R>) * cnt * nrhs, s));
    FB_CUDA(cudaMemsetAsync(loc, 0, sizeof(cx<R>) * cnt * nrhs, s));
    int nleaf = t->nbox[L];
    k_p2m<R><<<dim3(nleaf, nrhs), 128, 0, s>>>(PL, t->leaf_start, t->perm, W, x, mp + op->lev_off[L], n, cnt);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    mark(1);
    const RotArgs<R> rot = rot_args<R>(op);
    const cx<R>* coax = (const cx<R>*)(sizeof(R) == 8 ? (const void*)op->coax64 : (const void*)op->coax32);
    const bool auto_tc = sizeof(R) == 4 && op->method == FB_TRANS_AUTO;
    for (int l = L; l >= 3; --l) {
        if (composed) FB_CHECK(run_plan<R>(op->m2m[l], T, mp, mp, s));
        else if (auto_tc && op->tc_m2m[l])
            FB_CHECK(fb_tc_run(op, op->tc_m2m[l], (const cf*)mp, (cf*)mp, s, nrhs, cnt));
        else FB_CHECK(run_rcr<R>(op->m2m_rcr[l], rot, coax, mp, mp, s, nrhs, cnt));
    }
    mark(2);
    // phase [2] is the tensor-core part of M2L: empty unless it runs below
    const bool tc_split = sizeof(R) == 4 && op->method == FB_TRANS_AUTO && op->tc_plan != nullptr;
    if (!tc_split) mark(3);
    if (composed) {
        FB_CHECK(run_plan<R>(op->m2l, T, mp, loc, s));
    } else if (op->method == FB_TRANS_RCR) {
        FB_CHECK(run_rcr<R>(op->m2l_rcr, rot, coax, mp, loc, s, nrhs, cnt));
    } else {
        if constexpr (sizeof(R) == 4) {
            if (op->method == FB_TRANS_TENSOR) {
                FB_CHECK(fb_tc_run(op, op->tc_plan_all, (const cf*)mp, (cf*)loc, s, nrhs, cnt));
            } else if (op->tc_plan) {
                FB_CHECK(fb_tc_run(op, op->tc_plan, (const cf*)mp, (cf*)loc, s, nrhs, cnt));
                mark(3);
                FB_CHECK(run_rcr<R>(op->m2l_rcr_rest, rot, coax, mp, loc, s, nrhs, cnt));
            } else {
                FB_CHECK(run_rcr<R>(op->m2l_rcr, rot, coax, mp, loc, s, nrhs, cnt));
            }
        } else {
            FB_CHECK(run_rcr<R>(op->m2l_rcr, rot, coax, mp, loc, s, nrhs, cnt));
        }
    }
    mark(4);
    for (int l = 3; l <= L; ++l) {
        if (composed) FB_CHECK(run_plan<R>(op->l2l[l], T, loc, loc, s));
        else if (auto_tc && op->tc_l2l[l])
            FB_CHECK(fb_tc_run(op, op->tc_l2l[l], (const cf*)loc, (cf*)loc, s, nrhs, cnt));
        else FB_CHECK(run_rcr<R>(op->l2l_rcr[l], rot, coax, loc, loc, s, nrhs, cnt));
    }
    mark(5);
    int maxK = 0;
    for (int v : op->h_nf_ncol) maxK = std::max(maxK, v);
    const cx<R>* locL = loc + op->lev_off[L];
    if (nrhs == 1) {
        size_t smem = sizeof(cx<R>) * (maxK + PL);
        bool done16 = false;
        if constexpr (sizeof(R) == 4) {
            if (op->near16 && op->nf16) {   // 16-bit near-field entries
                FB_CHECK(fb_smem_cap((const void*)k_near_l2p<R, 1, uint32_t>, smem));
                k_near_l2p<R, 1, uint32_t><<<nleaf, 256, smem, s>>>(PL, t->leaf_start, t->perm, t->ucnt,
                                                                    t->ulist, op->nf_off, op->nf_ncol, op->nf16, V,
                                                                    locL, x, y, 1, n, cnt);
                done16 = true;
            }
        }
        if (!done16) {
            FB_CHECK(fb_smem_cap((const void*)k_near_l2p<R, 1>, smem));
            k_near_l2p<R, 1><<<nleaf, 256, smem, s>>>(PL, t->leaf_start, t->perm, t->ucnt, t->ulist, op->nf_off,
                                                      op->nf_ncol, A, V, locL, x, y, 1, n, cnt);
        }
    } else {
        constexpr int NB = 4;
        int nr = std::min(nrhs, NB);
        size_t smem = sizeof(cx<R>) * (size_t)nr * (maxK + PL);
        if (smem > 227 * 1024) return fb_fail(FB_ERR_ARG, "near-field tile exceeds shared memory");
        bool done16 = false;
        if constexpr (sizeof(R) == 4) {
            if (op->near16 && op->nf16) {
                FB_CHECK(fb_smem_cap((const void*)k_near_l2p<R, NB, uint32_t>, smem));
                k_near_l2p<R, NB, uint32_t><<<dim3(nleaf, div_up(nrhs, NB)), 256, smem, s>>>(
                    PL, t->leaf_start, t->perm, t->ucnt, t->ulist, op->nf_off, op->nf_ncol, op->nf16, V, locL, x,
                    y, nrhs, n, cnt);
                done16 = true;
            }
        }
        if (!done16) {
            FB_CHECK(fb_smem_cap((const void*)k_near_l2p<R, NB>, smem));
            k_near_l2p<R, NB><<<dim3(nleaf, div_up(nrhs, NB)), 256, smem, s>>>(
                PL, t->leaf_start, t->perm, t->ucnt, t->ulist, op->nf_off, op->nf_ncol, A, V, locL, x, y, nrhs, n,
                cnt);
        }
    }
    FB_LAUNCH_CHECK();
    fb_count_launch();
    mark(6);
    return FB_OK;
}

// FP32 -> BF16 with round to nearest even (finite values)
__device__ __forceinline__ uint32_t bf16_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
static __global__ void k_cf_to_bf16(const cf* __restrict__ in, int64_t n, uint32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = bf16_bits(in[i].re) | (bf16_bits(in[i].im) << 16);
}

// Near-field entries of a mixed operator in BF16 (8-bit significand,
// relative rounding 2^-9 per entry) for low-accuracy operators, whose
// matvec then reads half the near-field bytes; enable = 0 returns to FP32.
fb_status fb_near_bf16(fb_op* op, int enable, cudaStream_t s) {
    if (op->prec != FB_PREC_MIXED_FMM || !op->nf32)
        return fb_fail(FB_ERR_ARG, "BF16 near field applies to mixed FMM operators");
    if (enable && !op->nf16) {
        FB_CHECK(dalloc(&op->nf16, (size_t)op->nf_count));
        k_cf_to_bf16<<<(unsigned)std::min<int64_t>(div_up(op->nf_count, 256), 8192), 256, 0, s>>>(
            op->nf32, op->nf_count, op->nf16);
        FB_LAUNCH_CHECK();
        FB_CUDA(cudaStreamSynchronize(s));
        fb_count_launch();
    }
    op->near16 = enable ? 1 : 0;
    op->buf_gen++;   // captured graphs read the other entries
    return FB_OK;
}

static size_t op_csize(const fb_op* op) { return op->prec == FB_PREC_MIXED_FMM ? sizeof(cf) : sizeof(cd); }

// Level whose RCR flag governs a task: M2L tasks read and write one level;
// M2M / L2L tasks are governed by their finer (child) level, whose
// expansions lie after the parent's in the level arrays.  Levels 0 and 1
// hold no expansions (their offsets equal level 2's), so the search starts
// at level 2.
static int task_level(const fb_op* op, const RcrTask& tk, bool* m2l) {
    *m2l = tk.src_base == tk.dst_base;
    const int64_t b = std::max(tk.src_base, tk.dst_base);
    for (int l = 2; l <= op->L; ++l)
        if (op->lev_off[l] == b) return l;
    return 2;
}

fb_status fb_rcr_restage(fb_op* op, const int* m2l, const int* pair) {
    const size_t csz = op_csize(op);
    for (int l = 2; l <= op->L; ++l) {
        // 1: staged on CUDA cores, 2: staged with the rotations on the tensor cores
        op->stg_m2l[l] = m2l[l] ? m2l[l] : (!fb_rcr_tile_fits(op->p[l], op->p[l], csz) ? 1 : 0);
        if (l >= 3) {
            const int pm = std::max(op->p[l], op->p[l - 1]);
            op->stg_pair[l] = pair[l] ? pair[l] : (!fb_rcr_tile_fits(pm, pm, csz) ? 1 : 0);
        }
    }
    FB_CUDA(cudaDeviceSynchronize());
    op->buf_gen++;   // captured graphs refer to the plans rebuilt here
    auto redo = [&](RcrPlan& pl) -> fb_status {
        if (pl.h_tasks.empty()) return FB_OK;
        bool changed = false;
        for (RcrTask& tk : pl.h_tasks) {
            bool is_m2l = false;
            const int l = task_level(op, tk, &is_m2l);
            const int want = is_m2l ? op->stg_m2l[l] : op->stg_pair[l];
            changed = changed || tk.staged != want;
            tk.staged = want;
        }
        if (!changed) return FB_OK;
        const int32_t* si = pl.src_idx;
        const int32_t* di = pl.dst_idx;
        fb_rcr_free(pl);
        return fb_rcr_upload(op, pl, si, di, csz);
    };
    FB_CHECK(redo(op->m2l_rcr));
    FB_CHECK(redo(op->m2l_rcr_rest));
    for (int l = 3; l <= op->L; ++l) {
        FB_CHECK(redo(op->m2m_rcr[l]));
        FB_CHECK(redo(op->l2l_rcr[l]));
    }
    return FB_OK;
}

// One RCR plan on the operator's expansion buffers (precision of the op).
fb_status fb_rcr_run_op(fb_op* op, RcrPlan& pl, void* src, void* dst, cudaStream_t s, int nrhs, int64_t rstride) {
    if (op->prec == FB_PREC_MIXED_FMM)
        return run_rcr<float>(pl, rot_args<float>(op), op->coax32, (const cf*)src, (cf*)dst, s, nrhs, rstride);
    return run_rcr<double>(pl, rot_args<double>(op), op->coax64, (const cd*)src, (cd*)dst, s, nrhs, rstride);
}

fb_status fb_fmm_apply(fb_op* op, const cd* x, cd* y, cudaStream_t s, PhaseTimer* pt, int nrhs) {
    if (op->prec == FB_PREC_MIXED_FMM)
        return fmm_apply_t<float>(op, x, y, s, op->nf32, op->w32, op->v32, op->T32, pt, nullptr, nrhs);
    return fmm_apply_t<double>(op, x, y, s, op->nf64, op->w64, op->v64, op->T64, pt, nullptr, nrhs);
}

static void free_plan(TransPlan& p) {
    dfree(p.tasks);
    dfree(p.tiles);
}
void fb_rcr_free(RcrPlan& p) {
    dfree(p.tasks);
    dfree(p.tiles);
    dfree(p.df_tiles.tiles);
    p.df_tiles = RcrTileSet();
    fb_stg_free(p.stg);
    p.stg_elems = 0;
    for (auto& kv : p.multi) dfree(kv.second.tiles);
    p.multi.clear();
}
static void free_plan(RcrPlan& p) { fb_rcr_free(p); }

void fb_fmm_destroy(fb_op* op) {
    dfree(op->nf_off);
    dfree(op->nf_ncol);
    dfree(op->nf64);
    dfree(op->nf32);
    dfree(op->nf16);
    dfree(op->self64);
    dfree(op->w64);
    dfree(op->w32);
    dfree(op->v64);
    dfree(op->v32);
    dfree(op->mp);
    dfree(op->loc);
    dfree(op->T64);
    dfree(op->T32);
    free_plan(op->m2l);
    free_plan(op->m2l_rcr);
    free_plan(op->m2l_rcr_rest);
    fb_tc_free(op->tc_plan);
    fb_tc_free(op->tc_plan_all);
    for (int l = 0; l <= FB_MAXLEV; ++l) {
        fb_tc_free(op->tc_m2m[l]);
        fb_tc_free(op->tc_l2l[l]);
    }
    for (int l = 0; l <= FB_MAXLEV; ++l) {
        free_plan(op->m2m[l]);
        free_plan(op->l2l[l]);
        free_plan(op->m2m_rcr[l]);
        free_plan(op->l2l_rcr[l]);
    }
    op->rot64 = nullptr;   // owned by the tree
    op->rotd64 = nullptr;
    op->rotd32 = nullptr;
    op->rph64 = nullptr;
    op->rph32 = nullptr;
    dfree(op->coax64);
    dfree(op->coax32);
    dfree(op->stg_u);
    dfree(op->stg_v);
    op->stg_elems = 0;
    if (op->rotf) cudaFree(op->rotf);
    op->rotf = nullptr;
    dfree(op->stc_tab);
    dfree(op->stc_off);
    dfree(op->stc_err);
    dfree(op->rotf_df);
    dfree(op->coax_df);
    dfree(op->rotd_df);
}

// ---------------------------------------------------------------------------
// Matvec without allocation.  Some callers cannot allocate device memory when
// they apply an operator: real-time audio callbacks that must not block in the
// driver's allocator, or hosts whose device memory is owned by a fixed arena
// that the library may not grow.  For
// them fb_operator_apply_noalloc keeps the FMM's per-call scratch (the
// multipole and local expansions of every level) in this library-wide
// static device array instead of the operator's own buffers.  Every GPU that
// loads the library holds the array until the process exits.
static __device__ __align__(256) unsigned char fb_noalloc_scratch[FB_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// Resolves the device address of the static array for the current device
// (once per device; host code only sees a stand-in for the symbol).
static fb_status noalloc_scratch_ptr(void** out) {
    int dev = 0;
    FB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fb_fail(FB_ERR_ARG, "device ordinal out of range for the static scratch");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, fb_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fb_fail(FB_ERR_CUDA, std::string("cudaGetSymbolAddress(fb_noalloc_scratch) failed: ") +
                                            cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FB_OK;
}

fb_status fb_fmm_apply_noalloc(fb_op* op, const cd* x, cd* y, cudaStream_t s) {
    if (op->prec == FB_PREC_FP64_DENSE)
        return fb_fail(FB_ERR_ARG, "fb_operator_apply_noalloc needs an FMM operator (dense ones use no scratch)");
    // the static array is resolved per device: the operator's data and the
    // scratch must be on the same GPU
    int cur = -1;
    FB_CUDA(cudaGetDevice(&cur));
    if (cur != op->dev)
        return fb_fail(FB_ERR_ARG, "fb_operator_apply_noalloc: current device " + std::to_string(cur) +
                                       " differs from the operator's device " + std::to_string(op->dev));
    size_t elem = op->prec == FB_PREC_MIXED_FMM ? sizeof(cf) : sizeof(cd);
    size_t need = 2 * (size_t)op->lev_off[op->L + 1] * elem;
    if (need > (size_t)FB_NOALLOC_SCRATCH_BYTES)
        return fb_fail(FB_ERR_ARG, "operator needs " + std::to_string(need) +
                                       " bytes of expansion scratch; the static buffer holds " +
                                       std::to_string((size_t)FB_NOALLOC_SCRATCH_BYTES));
    void* p = nullptr;
    FB_CHECK(noalloc_scratch_ptr(&p));
    if (op->prec == FB_PREC_MIXED_FMM)
        return fmm_apply_t<float>(op, x, y, s, op->nf32, op->w32, op->v32, op->T32, nullptr, p);
    return fmm_apply_t<double>(op, x, y, s, op->nf64, op->w64, op->v64, op->T64, nullptr, p);
}
