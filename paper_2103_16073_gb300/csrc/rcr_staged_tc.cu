// Rotation passes of the staged RCR translation (Sec. 3.3) on the tensor
// cores (tcgen05, 3xTF32).
//
// The rotation pass R and the back-rotation pass B of rcr_staged.cu are
// real-by-complex GEMMs per (polar-angle group, degree n, folded part): the
// folded real table block d (N x K, N = K = n + 1 or n) applied to the
// complex vectors of every slot (pair) of the group.  Here they run
// transposed, so that the short dimension of a degree block is the MMA's N:
//     D[(slot, re/im)][row] = sum_k  x[slot][k].{re, im}  d[row][k]
//   A = the slots' vectors: 64 slots per tile as 128 real rows (row 2j the
//       real parts of slot j, row 2j + 1 the imaginary parts), loaded by
//       producer warps with plain loads (pass R folds and phases the source
//       expansions on the fly; pass B reads contiguous runs of v), split
//       into TF32 hi + lo and stored in the canonical layout;
//   B = the table block, K-major as stored (row-major [row][k]), pre-split
//       into hi + lo and laid out canonically per K chunk of 16 at setup, so
//       that one bulk copy moves a chunk;
//   D = FP32 accumulators in tensor memory, one column range per degree; a
//       tile packs consecutive degrees up to 256 columns.
// 3xTF32: D += A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// Pipeline (10 warps, 3 shared-memory stages):
//   warps 0-7  A producers (each thread 4 consecutive K values of one slot
//              per chunk, the next chunk's loads in flight while the current
//              one is stored), then the epilogue;
//   warp 8     lane 0: bulk copies of the table chunks (transaction count);
//   warp 9     lane 0: MMA issuer (waits for both operands of a stage,
//              6 MMAs per chunk, commits to the stage's "empty" barrier).
//   epilogue   warps w and w + 4 read the accumulator lanes of quadrant
//              w % 4 (even / odd 16-column groups); lanes 2j and 2j + 1
//              hold the real and imaginary part of slot j and trade halves
//              (one shuffle) so that each lane writes whole complex values:
//              pass R stores u (degree-major, folded), pass B adds the
//              phased y_{+-m'} = (Y+ +- Y-)/2 into the targets (atomics).
// Every mbarrier wait is bounded; on timeout the kernel records an error
// flag, drains its own bulk copies and MMAs (bounded) and frees its tensor
// memory.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "rcr_staged.cuh"
#include "tc_common.cuh"

using namespace stg;

namespace {

using tcx::canon;
using tcx::DRAIN_LIMIT;
using tcx::KC;
using tcx::LBO;
using tcx::mbar_init;
using tcx::mbar_wait;
using tcx::mma_commit;
using tcx::mma_tf32;
using tcx::smem_u32;
using tcx::tf32_hi;
using tcx::umma_desc;

constexpr int STC_M = 2 * STC_SLOTS;         // real rows of a tile
constexpr int STC_PRODW = 8;                 // producer / epilogue warps
constexpr int STC_NPROD = STC_PRODW * 32;
constexpr int STC_THREADS = STC_NPROD + 64;  // + bulk-copy warp + MMA warp
constexpr int A_PLANE = STC_M * KC;          // floats of one (hi or lo) A block
constexpr int STC_STAGES = 3;
// at most two CTAs per SM, so that their tensor memory (2 x 256 columns)
// is always free when they start
constexpr size_t STC_SMEM_MIN = 80 * 1024;

static_assert(STC_NPROD == STC_SLOTS * (KC / 4), "one producer thread per (slot, 4 K values)");

// accumulator columns N (output rows of the table block) and summed length
// K of degree n, folded part `part`, of pass R (0) or B (1)
__host__ __device__ __forceinline__ void stc_dims(int pass, int n, int part, int p_in, int& N, int& K) {
    N = n + 1 - part;
    K = pass == 0 ? N : std::min(n, p_in - 1) + 1 - part;
}

struct StcArgs {
    const StcTile* tiles;
    const int64_t* toff;   // table block offsets [2 n + part]
    const float* tab;      // group g: R table at g * 2 tper, B table at g * 2 tper + tper
    int64_t tper;
    const StgSlot* slots;
    const cf* X;           // R: source expansions; B: v (degree-major, folded)
    cf* out;               // R: u (degree-major, folded); B: target expansions
    const cf* rph;         // phases e^{i m phi} per direction
    int* err;
    long long wait_limit;
    int S, p_in, p_out, prot;
    int stage_floats;
    int inject_stall;
};

// 4 consecutive K values (k0 .. k0 + 3) of one slot's vector of degree n.
// Pass R folds and phases the source expansion on the fly (m = part + k):
// s_0 = x_0, s_m = x_m e^{i m phi} + x_{-m} e^{-i m phi}, t_m = the
// difference; pass B reads E_mu / O_mu (mu = part + k) of v.
template <int PASS>
__device__ __forceinline__ void stc_load(const StcArgs& a, int64_t row, int dir, int n, int part, int K, int k0,
                                         float (&v)[8]) {
    const cf* ph = a.rph + (int64_t)dir * (2 * a.prot - 1) + (a.prot - 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        float2 x = make_float2(0.f, 0.f);
        if (row >= 0 && k < K) {
            if (PASS == 0) {
                const cf* xs = a.X + row + (int64_t)n * n + n;   // (n, 0)
                const int m = part + k;
                if (m == 0) {
                    x = __ldg(reinterpret_cast<const float2*>(xs));
                } else {
                    const float2 xp = __ldg(reinterpret_cast<const float2*>(xs + m));
                    const float2 xm = __ldg(reinterpret_cast<const float2*>(xs - m));
                    const float2 pp = __ldg(reinterpret_cast<const float2*>(ph + m));
                    const float2 pm = __ldg(reinterpret_cast<const float2*>(ph - m));
                    const float ar = xp.x * pp.x - xp.y * pp.y, ai = xp.x * pp.y + xp.y * pp.x;
                    const float br = xm.x * pm.x - xm.y * pm.y, bi = xm.x * pm.y + xm.y * pm.x;
                    x = part ? make_float2(ar - br, ai - bi) : make_float2(ar + br, ai + bi);
                }
            } else {
                x = __ldg(reinterpret_cast<const float2*>(a.X + row + (int64_t)n * n + (part ? n : 0) + part + k));
            }
        }
        v[2 * i] = x.x;
        v[2 * i + 1] = x.y;
    }
}

// stores them as rows 2j (real parts) and 2j + 1 (imaginary parts) of the
// hi and lo A blocks of a stage
__device__ __forceinline__ void stc_store(float* st, int j, int q, const float (&v)[8]) {
    float4 rh, rl, ih, il;
    float* prh = &rh.x;
    float* prl = &rl.x;
    float* pih = &ih.x;
    float* pil = &il.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float re = v[2 * i], im = v[2 * i + 1];
        const float hr = tf32_hi(re), hi = tf32_hi(im);
        prh[i] = hr;
        prl[i] = re - hr;
        pih[i] = hi;
        pil[i] = im - hi;
    }
    const int ore = canon(2 * j, 4 * q) >> 2, oim = canon(2 * j + 1, 4 * q) >> 2;
    *reinterpret_cast<float4*>(st + ore) = rh;
    *reinterpret_cast<float4*>(st + A_PLANE + ore) = rl;
    *reinterpret_cast<float4*>(st + oim) = ih;
    *reinterpret_cast<float4*>(st + A_PLANE + oim) = il;
}

template <int PASS>
__global__ void __launch_bounds__(STC_THREADS, 2) k_stg_tc(const StcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STC_STAGES];    // A producers' stores
    __shared__ __align__(8) uint64_t b_bar[STC_STAGES];       // the bulk copy of the table chunk
    __shared__ __align__(8) uint64_t empty_bar[STC_STAGES];   // MMAs of the stage complete
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ __align__(8) uint64_t never_bar;               // test hook: nothing arrives on it
    __shared__ uint32_t tmem_holder;
    __shared__ int64_t s_row[STC_SLOTS];   // slot * S (-1: padding row of zeros)
    __shared__ int64_t s_dst[STC_SLOTS];   // pass R: the slot's row of u; pass B: its target expansion
    __shared__ int32_t s_dir[STC_SLOTS];   // pass B: direction (phases)
    __shared__ int s_fail;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024 - (raw & 1023)) & 1023;
    float* stage0 = (float*)(smem_raw + pad);

    const StcTile tl = a.tiles[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int part = tl.part;
    if (tid < STC_SLOTS) {
        const bool ok = tid < tl.ns;
        const int sl = tl.s0 + tid;
        // pass R: the source expansion of the slot; pass B: its row of v
        s_row[tid] = ok ? (PASS == 0 ? a.slots[sl].src_off : (int64_t)sl * a.S) : -1;
        s_dst[tid] = ok ? (PASS == 0 ? (int64_t)sl * a.S : a.slots[sl].dst_off) : 0;
        s_dir[tid] = ok ? a.slots[sl].dir : 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(STC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < STC_STAGES; ++s) {
            mbar_init(&full_bar[s], STC_NPROD);
            mbar_init(&b_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        mbar_init(&never_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const float* tabg = a.tab + (int64_t)tl.g * 2 * a.tper + (PASS ? a.tper : 0);

    if (warp < STC_PRODW) {
        // ---------------- A producers ---------------------------------------
        const int j = tid >> 2, q = tid & 3;
        const int64_t row = s_row[j];
        const int dir = s_dir[j];
        int n = tl.n0, kc = 0, N, K;
        stc_dims(PASS, n, part, a.p_in, N, K);
        float cur[8], nxt[8];
        stc_load<PASS>(a, row, dir, n, part, K, 4 * q, cur);
        for (int c = 0;; ++c) {
            // the next chunk's loads go out before this one is stored
            int n2 = n, kc2 = kc + 1, K2 = K;
            if (kc2 * KC >= K) {
                ++n2;
                kc2 = 0;
                if (n2 < tl.n1) stc_dims(PASS, n2, part, a.p_in, N, K2);
            }
            const bool more = n2 < tl.n1;
            if (more) stc_load<PASS>(a, row, dir, n2, part, K2, kc2 * KC + 4 * q, nxt);
            const int s = c % STC_STAGES, u = c / STC_STAGES;
            if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (u - 1) & 1, a.wait_limit)) {
                atomicExch(&s_fail, 1);
                break;
            }
            stc_store(stage0 + (size_t)s * a.stage_floats, j, q, cur);
            // generic-proxy stores become visible to the tensor core's reads
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])));
            if (!more) break;
#pragma unroll
            for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
            n = n2;
            kc = kc2;
            K = K2;
        }
    } else if (warp == STC_PRODW) {
        // ---------------- table chunks: one bulk copy per stage --------------
        if (lane == 0) {
            int issued = 0;
            bool fail = false;
            for (int n = tl.n0, c = 0; n < tl.n1 && !fail; ++n) {
                int N, K;
                stc_dims(PASS, n, part, a.p_in, N, K);
                const int np = stc_pad16(N), nkc = (K + KC - 1) / KC;
                const float* tb = tabg + a.toff[2 * n + part];
                const uint32_t bytes = (uint32_t)(2 * np * KC * sizeof(float));
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int s = c % STC_STAGES, u = c / STC_STAGES;
                    if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (u - 1) & 1, a.wait_limit)) {
                        atomicExch(&s_fail, 1);
                        fail = true;
                        break;
                    }
                    const uint32_t bb = smem_u32(&b_bar[s]);
                    const uint32_t dB = smem_u32(stage0 + (size_t)s * a.stage_floats + 2 * A_PLANE);
                    const float* g = tb + (int64_t)kc * 2 * np * KC;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(bytes));
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            dB),
                        "l"(g), "r"(bytes), "r"(bb));
                    ++issued;
                }
            }
            // every bulk copy this CTA issued lands before the CTA may exit
            for (int c = std::max(0, issued - STC_STAGES); c < issued; ++c)
                mbar_wait(smem_u32(&b_bar[c % STC_STAGES]), (c / STC_STAGES) & 1, DRAIN_LIMIT);
        }
        __syncwarp();
    } else {
        // ---------------- MMA issuer ----------------------------------------
        if (lane == 0) {
            // test hook: a wait on a barrier nothing arrives on runs out
            const bool stalled = a.inject_stall && !mbar_wait(smem_u32(&never_bar), 0, a.wait_limit);
            bool fail = stalled;
            if (stalled) atomicExch(&s_fail, 1);
            uint32_t col = 0;
            for (int n = tl.n0, c = 0; n < tl.n1 && !fail; ++n) {
                int N, K;
                stc_dims(PASS, n, part, a.p_in, N, K);
                const int np = stc_pad16(N), nkc = (K + KC - 1) / KC;
                const uint32_t idesc = tcx::idesc_tf32(STC_M, np);
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int s = c % STC_STAGES, u = c / STC_STAGES;
                    if (!mbar_wait(smem_u32(&full_bar[s]), u & 1, a.wait_limit) ||
                        !mbar_wait(smem_u32(&b_bar[s]), u & 1, a.wait_limit)) {
                        atomicExch(&s_fail, 1);
                        fail = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const float* st = stage0 + (size_t)s * a.stage_floats;
                    const uint32_t aH = smem_u32(st), aL = smem_u32(st + A_PLANE);
                    const uint32_t bH = smem_u32(st + 2 * A_PLANE), bL = smem_u32(st + 2 * A_PLANE + np * KC);
#pragma unroll
                    for (int ks = 0; ks < KC / 8; ++ks) {
                        const uint32_t o = ks * 2 * LBO;
                        const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
                        mma_tf32(tmem + col, umma_desc(aH + o), umma_desc(bH + o), idesc, first);
                        mma_tf32(tmem + col, umma_desc(aH + o), umma_desc(bL + o), idesc, 1u);
                        mma_tf32(tmem + col, umma_desc(aL + o), umma_desc(bH + o), idesc, 1u);
                    }
                    mma_commit(&empty_bar[s]);
                }
                col += np;
            }
            // completion of every MMA issued above (also on failure)
            mma_commit(&done_bar);
        }
        __syncwarp();
    }

    // ---------------- epilogue ------------------------------------------------
    const bool done = mbar_wait(smem_u32(&done_bar), 0, DRAIN_LIMIT);
    __syncthreads();
    const bool ok = done && s_fail == 0;
    if (!ok && tid == 0) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && warp < STC_PRODW) {
        const int quad = warp & 3, half = warp >> 2;
        const int rr = quad * 32 + lane;           // accumulator lane = real row
        const int j = rr >> 1, cpt = rr & 1;       // slot, 0: real / 1: imaginary part
        const bool valid = j < tl.ns;
        const float sgn = part ? -1.f : 1.f;
        const cf* ph = a.rph + (int64_t)s_dir[j] * (2 * a.prot - 1) + (a.prot - 1);
        uint32_t col = 0;
        for (int n = tl.n0; n < tl.n1; ++n) {
            int N, K;
            stc_dims(PASS, n, part, a.p_in, N, K);
            const int np = stc_pad16(N);
            for (int g16 = half; g16 < np / 16; g16 += 2) {
                uint32_t v[16];
                tcx::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + col + (uint32_t)(g16 * 16), v);
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    // the real lane holds columns (c, c+1) of re, the imaginary
                    // lane of im: trade so that each writes one complex value
                    const float x0 = __uint_as_float(v[2 * qq]), x1 = __uint_as_float(v[2 * qq + 1]);
                    const float recv = __shfl_xor_sync(0xffffffffu, cpt ? x0 : x1, 1);
                    const float re = cpt ? recv : x0, im = cpt ? x1 : recv;
                    const int i = g16 * 16 + 2 * qq + cpt;   // row of the degree block
                    if (!valid || i >= N) continue;
                    if (PASS == 0) {
                        cf* u = a.out + s_dst[j] + (int64_t)n * n + (part ? n : 0) + part + i;
                        *reinterpret_cast<float2*>(u) = make_float2(re, im);
                    } else {
                        const int mp = part + i;
                        const float hr = 0.5f * re, hi = 0.5f * im;
                        cf* d = a.out + s_dst[j] + (int64_t)n * n + n;   // entry (n, 0) of the target
                        if (mp == 0) {
                            atomicAdd(reinterpret_cast<float2*>(d), make_float2(hr, hi));
                        } else {
                            const cf e = ph[mp];
                            atomicAdd(reinterpret_cast<float2*>(d + mp),
                                      make_float2(hr * e.re + hi * e.im, hi * e.re - hr * e.im));
                            atomicAdd(reinterpret_cast<float2*>(d - mp),
                                      make_float2(sgn * (hr * e.re - hi * e.im), sgn * (hr * e.im + hi * e.re)));
                        }
                    }
                }
            }
            col += np;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(STC_TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Coaxial pass (complex blocks): D[v][(i, re/im)] = sum_k u_v[k] C[i][k] in
// the real form with interleaved K (u as stored, complex = (re, im) pairs):
//   A[v][(k, c)] = u_v[k].c  (v: virtual column = slot x even/odd part),
//   B[(i, 0)][(k, 0)] = Re C,  B[(i, 0)][(k, 1)] = -Im C,
//   B[(i, 1)][(k, 0)] = Im C,  B[(i, 1)][(k, 1)] = Re C,
// so D[v][(i, 0)] = Re(sum u C), D[v][(i, 1)] = Im(sum u C): no zero blocks,
// and each accumulator lane holds one output vector (degrees n' at a fixed
// order), scattered into the degree-major folded v.
struct StcCArgs {
    const StcCTile* tiles;
    const int32_t* cidx;
    const float* tab;
    const cf* U;
    cf* V;
    int* err;
    long long wait_limit;
    int S, p_out;
    int stage_floats;
    int nst;            // pipeline stages (<= STC_CSTAGES)
    int inject_stall;
};

constexpr int STC_CSTAGES = 3;

__global__ void __launch_bounds__(STC_THREADS, 2) k_stc_coax(const StcCArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STC_CSTAGES];
    __shared__ __align__(8) uint64_t b_bar[STC_CSTAGES];
    __shared__ __align__(8) uint64_t empty_bar[STC_CSTAGES];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ __align__(8) uint64_t never_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ int64_t s_row[STC_M];   // slot * S (-1: padding row)
    __shared__ int32_t s_odd[STC_M];
    __shared__ int s_fail;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024 - (raw & 1023)) & 1023;
    float* stage0 = (float*)(smem_raw + pad);

    const StcCTile tl = a.tiles[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int am = tl.am;
    if (tid < STC_M) {
        const int v = tl.vc0 + tid;
        const bool ok = tid < tl.nvc;
        const int slot = ok ? (am == 0 ? a.cidx[tl.c0 + v] : a.cidx[tl.c0 + (v >> 1)]) : 0;
        s_row[tid] = ok ? (int64_t)slot * a.S : -1;
        s_odd[tid] = (ok && am != 0 && (v & 1)) ? 1 : 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(STC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < STC_CSTAGES; ++s) {
            mbar_init(&full_bar[s], STC_NPROD);
            mbar_init(&b_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        mbar_init(&never_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const int nst = a.nst;
    const int np = stc_pad16(2 * tl.nr);
    const int nkc = (2 * tl.K + KC - 1) / KC;   // K chunks of 8 complex input degrees

    if (warp < STC_PRODW) {
        // ---------------- A producers: 2 (row, 2 complex K values) units each
        auto load = [&](int kc, int unit, float (&v)[4]) {
            const int r = unit >> 2, q = unit & 3;
            const int64_t row = s_row[r];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int k = kc * (KC / 2) + 2 * q + i;
                float2 x = make_float2(0.f, 0.f);
                if (row >= 0 && k < tl.K) {
                    const int n = am + k;
                    x = __ldg(reinterpret_cast<const float2*>(a.U + row + (int64_t)n * n + (s_odd[r] ? n : 0) + am));
                }
                v[2 * i] = x.x;
                v[2 * i + 1] = x.y;
            }
        };
        float cur[2][4], nxt[2][4];
        load(0, tid, cur[0]);
        load(0, tid + STC_NPROD, cur[1]);
        for (int c = 0; c < nkc; ++c) {
            const bool more = c + 1 < nkc;
            if (more) {
                load(c + 1, tid, nxt[0]);
                load(c + 1, tid + STC_NPROD, nxt[1]);
            }
            const int s = c % nst, u = c / nst;
            if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (u - 1) & 1, a.wait_limit)) {
                atomicExch(&s_fail, 1);
                break;
            }
            float* st = stage0 + (size_t)s * a.stage_floats;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int unit = tid + h * STC_NPROD;
                const int r = unit >> 2, q = unit & 3;
                float4 hi4, lo4;
                float* ph = &hi4.x;
                float* pl = &lo4.x;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float t = tf32_hi(cur[h][i]);
                    ph[i] = t;
                    pl[i] = cur[h][i] - t;
                }
                const int o = canon(r, 4 * q) >> 2;
                *reinterpret_cast<float4*>(st + o) = hi4;
                *reinterpret_cast<float4*>(st + A_PLANE + o) = lo4;
            }
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])));
            if (!more) break;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < 4; ++i) cur[h][i] = nxt[h][i];
        }
    } else if (warp == STC_PRODW) {
        // ---------------- coaxial block chunks: one bulk copy per stage -----
        if (lane == 0) {
            int issued = 0;
            const uint32_t bytes = (uint32_t)(2 * np * KC * sizeof(float));
            for (int c = 0; c < nkc; ++c) {
                const int s = c % nst, u = c / nst;
                if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (u - 1) & 1, a.wait_limit)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                const uint32_t bb = smem_u32(&b_bar[s]);
                const uint32_t dB = smem_u32(stage0 + (size_t)s * a.stage_floats + 2 * A_PLANE);
                const float* g = a.tab + tl.toff + (int64_t)c * 2 * np * KC;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(bytes));
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dB),
                    "l"(g), "r"(bytes), "r"(bb));
                ++issued;
            }
            for (int c = std::max(0, issued - nst); c < issued; ++c)
                mbar_wait(smem_u32(&b_bar[c % nst]), (c / nst) & 1, DRAIN_LIMIT);
        }
        __syncwarp();
    } else {
        // ---------------- MMA issuer ----------------------------------------
        if (lane == 0) {
            const bool stalled = a.inject_stall && !mbar_wait(smem_u32(&never_bar), 0, a.wait_limit);
            if (stalled) atomicExch(&s_fail, 1);
            const uint32_t idesc = tcx::idesc_tf32(STC_M, np);
            for (int c = 0; c < nkc && !stalled; ++c) {
                const int s = c % nst, u = c / nst;
                if (!mbar_wait(smem_u32(&full_bar[s]), u & 1, a.wait_limit) ||
                    !mbar_wait(smem_u32(&b_bar[s]), u & 1, a.wait_limit)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const float* st = stage0 + (size_t)s * a.stage_floats;
                const uint32_t aH = smem_u32(st), aL = smem_u32(st + A_PLANE);
                const uint32_t bH = smem_u32(st + 2 * A_PLANE), bL = smem_u32(st + 2 * A_PLANE + np * KC);
#pragma unroll
                for (int ks = 0; ks < KC / 8; ++ks) {
                    const uint32_t o = ks * 2 * LBO;
                    const uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
                    mma_tf32(tmem, umma_desc(aH + o), umma_desc(bH + o), idesc, first);
                    mma_tf32(tmem, umma_desc(aH + o), umma_desc(bL + o), idesc, 1u);
                    mma_tf32(tmem, umma_desc(aL + o), umma_desc(bH + o), idesc, 1u);
                }
                mma_commit(&empty_bar[s]);
            }
            mma_commit(&done_bar);
        }
        __syncwarp();
    }

    // ---------------- epilogue: v[slot][n'^2 + (odd ? n' : 0) + am], n' = am + r0 + i
    const bool done = mbar_wait(smem_u32(&done_bar), 0, DRAIN_LIMIT);
    __syncthreads();
    const bool ok = done && s_fail == 0;
    if (!ok && tid == 0) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && warp < STC_PRODW) {
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane;
        const bool valid = r < tl.nvc;
        cf* vout = a.V + (valid ? s_row[r] : 0) + am;
        const int odd = s_odd[r];
        for (int g16 = half; g16 < np / 16; g16 += 2) {
            uint32_t v[16];
            tcx::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g16 * 16), v);
            if (!valid) continue;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int i = g16 * 8 + t;
                const int n1 = am + tl.r0 + i;
                if (i < tl.nr)
                    *reinterpret_cast<float2*>(vout + (int64_t)n1 * n1 + (odd ? n1 : 0)) =
                        make_float2(__uint_as_float(v[2 * t]), __uint_as_float(v[2 * t + 1]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(STC_TMEM_COLS));
}

// Pre-split real-form coaxial blocks (grid: one CTA per block).
__global__ void k_stc_coax_tables(const StcCBlock* __restrict__ blocks, const cd* __restrict__ coax,
                                  float* __restrict__ out) {
    const StcCBlock b = blocks[blockIdx.x];
    const int np = stc_pad16(2 * b.nr), kp = ((2 * b.K + KC - 1) / KC) * KC;
    float* T = out + b.toff;
    for (int e = threadIdx.x; e < np * kp; e += blockDim.x) {
        const int j = e / kp, k2 = e % kp;   // row (i, c'), K index (k, c)
        const int i = j >> 1, cp = j & 1, k = k2 >> 1, c = k2 & 1;
        double v = 0.0;
        if (i < b.nr && k < b.K) {
            const cd C = coax[b.cs_off + ((int64_t)b.am * b.pc + b.am + b.r0 + i) * b.pc + b.am + k];
            v = cp == 0 ? (c == 0 ? C.re : -C.im) : (c == 0 ? C.im : C.re);
        }
        const int64_t o = (int64_t)(k2 / KC) * 2 * np * KC + (canon(j, k2 % KC) >> 2);
        const float h = tf32_hi((float)v);
        T[o] = h;
        T[o + (int64_t)np * KC] = (float)(v - (double)h);
    }
}

// Pre-split canonical table blocks of every group (grid: degree n, group g)
// from the FP64 real factors d^n of the group's representative direction:
// the folded R and B tables of rcr_staged.cu, zero-padded to whole
// 16 x 16 core blocks.
__global__ void k_stc_tables(const double* __restrict__ rotd, int64_t per_dir, const int* __restrict__ rep_dirs,
                             const int64_t* __restrict__ toff, int64_t tper, float* __restrict__ out) {
    const int n = blockIdx.x, g = blockIdx.y;
    const int w = 2 * n + 1;
    const double* Dc = rotd + (int64_t)rep_dirs[g] * per_dir + rot_off(n) + (int64_t)n * w + n;   // d_{0,0}
    for (int part = 0; part < 2; ++part) {
        const int nb = n + 1 - part;
        if (nb <= 0) continue;
        const int np = stc_pad16(nb);
        float* Rt = out + (int64_t)g * 2 * tper + toff[2 * n + part];
        float* Bt = Rt + tper;
        for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
            const int r = e / np, k = e % np;   // block row, K index
            double rv = 0.0, bv = 0.0;
            if (r < nb && k < nb) {
                const int a = r + part, b = k + part;
                // R: row mu = a, column m = b;  B: row m' = a, column mu = b
                if (part == 0) {
                    rv = b == 0 ? 2.0 * Dc[(int64_t)a * w] : Dc[(int64_t)a * w + b] + Dc[(int64_t)a * w - b];
                    bv = b == 0 ? Dc[a] : Dc[(int64_t)b * w + a] + Dc[-(int64_t)b * w + a];
                } else {
                    rv = Dc[(int64_t)a * w + b] - Dc[(int64_t)a * w - b];
                    bv = Dc[(int64_t)b * w + a] - Dc[-(int64_t)b * w + a];
                }
            }
            const int64_t o = (int64_t)(k / KC) * 2 * np * KC + (canon(r, k % KC) >> 2);
            const float rh = tf32_hi((float)rv), bh = tf32_hi((float)bv);
            Rt[o] = rh;
            Rt[o + (int64_t)np * KC] = (float)(rv - (double)rh);
            Bt[o] = bh;
            Bt[o + (int64_t)np * KC] = (float)(bv - (double)bh);
        }
    }
}

}  // namespace

namespace stg {

int64_t fb_stc_layout(int P, std::vector<int64_t>& toff) {
    toff.assign((size_t)2 * std::max(P, 1), 0);
    int64_t off = 0;
    for (int n = 0; n < P; ++n)
        for (int part = 0; part < 2; ++part) {
            const int nb = n + 1 - part;
            toff[(size_t)2 * n + part] = off;
            if (nb <= 0) continue;
            const int64_t np = stc_pad16(nb);
            off += 2 * np * np;   // hi and lo planes of np rows x np K values
        }
    return off;
}

void fb_stc_group_tiles(int g, int g0, int g1, int nmax, int pass, int p_in, std::vector<StcTile>& out) {
    for (int part = 0; part < 2; ++part) {
        int n0 = -1, cols = 0;
        auto flush = [&](int n1) {
            if (n0 < 0) return;
            for (int s0 = g0; s0 < g1; s0 += STC_SLOTS)
                out.push_back(StcTile{g, part, n0, n1, s0, std::min(STC_SLOTS, g1 - s0)});
            n0 = -1;
            cols = 0;
        };
        for (int n = 0; n < nmax; ++n) {
            int N, K;
            stc_dims(pass, n, part, p_in, N, K);
            if (N <= 0 || K <= 0) {
                flush(n);
                continue;
            }
            const int np = stc_pad16(N);
            if (n0 >= 0 && cols + np > STC_TMEM_COLS) flush(n);
            if (n0 < 0) n0 = n;
            cols += np;
        }
        flush(nmax);
    }
}

void fb_stc_coax_set(int c0, int ns, int64_t cs_off, int pc, int p_in, int p_out, std::vector<StcCTile>& tiles,
                     std::vector<StcCBlock>& blocks, int64_t* tfloats) {
    const int q = std::min(p_in, p_out);
    // one pre-split block per (order, row block)
    std::vector<std::vector<int64_t>> toff(q);
    for (int am = 0; am < q; ++am) {
        const int M = p_out - am, K = p_in - am;
        for (int r0 = 0; r0 < M; r0 += STC_CROWS) {
            const int nr = std::min(STC_CROWS, M - r0);
            const int np = stc_pad16(2 * nr), kp = ((2 * K + KC - 1) / KC) * KC;
            blocks.push_back(StcCBlock{cs_off, *tfloats, pc, am, r0, nr, K, 0});
            toff[am].push_back(*tfloats);
            *tfloats += (int64_t)2 * np * kp;
        }
    }
    // slot blocks outermost, orders next (sectors of u and v shared by
    // consecutive orders are used while in L2)
    for (int sb = 0; sb < ns; sb += STC_M / 2)
        for (int am = 0; am < q; ++am) {
            const int M = p_out - am, K = p_in - am;
            const int v0 = am == 0 ? sb : 2 * sb;
            const int nvc = am == 0 ? std::min(STC_M / 2, ns - sb) : std::min(STC_M, 2 * (ns - sb));
            int b = 0;
            for (int r0 = 0; r0 < M; r0 += STC_CROWS, ++b)
                tiles.push_back(StcCTile{toff[am][b], c0, v0, nvc, am, r0, std::min(STC_CROWS, M - r0), K, 0});
        }
}

fb_status fb_stc_coax_tables(const StcCBlock* blocks, int nblocks, const cd* coax64, float* out, cudaStream_t s) {
    if (nblocks == 0) return FB_OK;
    k_stc_coax_tables<<<(unsigned)nblocks, 256, 0, s>>>(blocks, coax64, out);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

fb_status fb_stc_coax_run(const StcCTile* tiles, int ntiles, const int32_t* cidx, const float* tab, const cf* U,
                          cf* V, int S, int p_out, int* err, cudaStream_t s) {
    if (ntiles == 0) return FB_OK;
    const int npmax = stc_pad16(2 * std::min(STC_CROWS, p_out));
    StcCArgs a;
    a.tiles = tiles;
    a.cidx = cidx;
    a.tab = tab;
    a.U = U;
    a.V = V;
    a.err = err;
    a.wait_limit = fb_tc_wait_limit();
    a.S = S;
    a.p_out = p_out;
    a.stage_floats = 2 * A_PLANE + 2 * npmax * KC;
    // three stages while two CTAs still fit an SM, else two
    a.nst = (size_t)STC_CSTAGES * a.stage_floats * sizeof(float) + 1024 <= 110 * 1024 ? STC_CSTAGES : 2;
    a.inject_stall = fb_tc_inject_stall();
    const size_t smem = std::max(STC_SMEM_MIN, (size_t)a.nst * a.stage_floats * sizeof(float) + 1024);
    FB_CHECK(fb_smem_cap((const void*)k_stc_coax, smem));
    k_stc_coax<<<(unsigned)ntiles, STC_THREADS, smem, s>>>(a);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

fb_status fb_stc_run(int pass, const StcTile* tiles, int ntiles, int npmax, const int64_t* toff, const float* tab,
                     int64_t tper, const StgSlot* slots, const cf* X, cf* out, int S, int p_in, int p_out,
                     const cf* rph, int prot, int* err, cudaStream_t s) {
    if (ntiles == 0) return FB_OK;
    if (npmax > STC_TMEM_COLS) return fb_fail(FB_ERR_ARG, "tensor-core staged RCR: order above 256");
    StcArgs a;
    a.tiles = tiles;
    a.toff = toff;
    a.tab = tab;
    a.tper = tper;
    a.slots = slots;
    a.X = X;
    a.out = out;
    a.rph = rph;
    a.err = err;
    a.wait_limit = fb_tc_wait_limit();
    a.S = S;
    a.p_in = p_in;
    a.p_out = p_out;
    a.prot = prot;
    a.stage_floats = 2 * A_PLANE + 2 * stc_pad16(npmax) * KC;
    a.inject_stall = fb_tc_inject_stall();
    const size_t smem = std::max(STC_SMEM_MIN, (size_t)STC_STAGES * a.stage_floats * sizeof(float) + 1024);
    const void* fn = pass == 0 ? (const void*)k_stg_tc<0> : (const void*)k_stg_tc<1>;
    FB_CHECK(fb_smem_cap(fn, smem));
    if (pass == 0)
        k_stg_tc<0><<<(unsigned)ntiles, STC_THREADS, smem, s>>>(a);
    else
        k_stg_tc<1><<<(unsigned)ntiles, STC_THREADS, smem, s>>>(a);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

}  // namespace stg

// Pre-split canonical rotation tables of the tensor-core staged passes for
// every polar-angle group of a mixed operator (built once, on first use).
fb_status fb_stc_tables(fb_op* op, cudaStream_t s) {
    if (op->stc_tab) return FB_OK;
    if (op->prec != FB_PREC_MIXED_FMM)
        return fb_fail(FB_ERR_ARG, "tensor-core staged RCR applies to mixed operators");
    const int ng = (int)op->theta_dirs.size();
    const int P = op->Prot;
    if (ng == 0 || P < 1) return fb_fail(FB_ERR_STATE, "tensor-core staged RCR: no rotation groups");
    std::vector<int64_t> toff;
    const int64_t tper = stg::fb_stc_layout(P, toff);
    int* d_dirs = nullptr;
    FB_CHECK(dalloc(&d_dirs, (size_t)ng));
    FB_CHECK(dalloc(&op->stc_off, toff.size()));
    FB_CHECK(dalloc(&op->stc_tab, (size_t)ng * 2 * tper));
    if (!op->stc_err) {
        FB_CHECK(dalloc(&op->stc_err, 1));
        FB_CUDA(cudaMemsetAsync(op->stc_err, 0, sizeof(int), s));
    }
    FB_CUDA(cudaMemcpyAsync(d_dirs, op->theta_dirs.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemcpyAsync(op->stc_off, toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice, s));
    k_stc_tables<<<dim3(P, ng), 256, 0, s>>>(op->rotd64, op->per_dir, d_dirs, op->stc_off, tper, op->stc_tab);
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(d_dirs);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("tensor-core rotation tables: ") + cudaGetErrorString(e));
    op->stc_per = tper;
    op->stc_P = P;
    fb_count_launch();
    return FB_OK;
}
