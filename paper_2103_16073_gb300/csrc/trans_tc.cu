// Stacked M2L translations on the 5th-generation tensor cores (tcgen05).
//
// All box pairs of one level that share a translation vector share one
// composed translation matrix T (p^2 x p^2 complex, Sec. 3.3 RCR composed in
// FP64).  The complex GEMM  Y = T X  (X: gathered source multipoles, one
// column per pair) runs as a real GEMM on interleaved (re, im) rows and
// columns,
//     [Y_re(r)]   [ T_re  -T_im ] [X_re]
//     [Y_im(r)] = [ T_im   T_re ] [X_im],
// in 3xTF32: every FP32 operand is split into hi (TF32) + lo, and
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in tensor
// memory.
//
// Operands:  A = real T rows, M = 128 per tile, pre-split and stored in
// global memory already in the canonical no-swizzle K-major layout, one
// 16 KB (hi + lo) block per (row tile, K chunk of 16) -> one bulk TMA copy.
// B = gathered X columns, N <= 256 per tile, from hi/lo planes of the level
// multipoles written once per matvec by k_tc_split -> 16-byte cp.async
// pieces into the canonical layout.
//
// Pipeline (8 warps, 2 shared-memory stages of 48 KB, two CTAs per SM):
//   warps 0-5  B producers (cp.async, completion tracked by the stage's
//              "full" mbarrier), warp 6 lane 0 A producer (bulk copy with
//              transaction count), warp 7 lane 0 MMA issuer (waits "full",
//              issues 6 MMAs, commits to the stage's "empty" mbarrier);
//   epilogue   all warps: tcgen05.ld of the accumulator (warps w and w+4
//              share lane quadrant w % 4 and split the columns), atomic
//              scatter-add into the target locals.
// Every mbarrier wait is bounded; on timeout the kernel records an error
// flag, drains its own copies and MMAs (bounded) and releases tensor memory.
#include <algorithm>
#include <atomic>

#include <map>

#include "common.cuh"
#include "tc_common.cuh"

namespace {

constexpr int TC_M = 128;       // real output rows per tile
constexpr int TC_NMAX = 256;    // box pairs per tile
constexpr int TC_KC = 16;       // real K per stage
constexpr int TC_STAGES = 2;   // two 48 KB stages: two CTAs (and 2 x 256 TMEM columns) per SM
constexpr int A_BLOCK = TC_M * TC_KC;       // floats per (hi or lo) A block
constexpr int B_BLOCK = TC_NMAX * TC_KC;    // floats per (hi or lo) B block
constexpr int STAGE_FLOATS = 2 * A_BLOCK + 2 * B_BLOCK;
constexpr int NPROD = 192;                  // B producer threads (warps 0-5)
using tcx::canon;
using tcx::DRAIN_LIMIT;
using tcx::LBO;
using tcx::mbar_wait;
using tcx::mma_tf32;
using tcx::smem_u32;
using tcx::tf32_hi;
using tcx::umma_desc;
static_assert(TC_KC == tcx::KC, "one canonical block width");

}  // namespace

struct TcTask {
    int64_t a_off;          // float offset of the pre-split tiles of T
    int64_t pair_off;
    int32_t npairs, nrt, nkc, p_out2;   // p_out2 = complex rows P_out
    int32_t p_in2;                      // complex columns P_in
    int32_t stride_f;                   // floats per box vector in the hi/lo planes
    int64_t plane_base;                 // float offset of the level in the planes
    int64_t dst_base;                   // complex offset of the target level
    int32_t nbox_src;                   // boxes of the source level (planes hold nrhs sets)
    int32_t pad;
};
struct TcTile {
    int32_t task, rt, col0, ncol;
};

// Pre-split canonical tiles of the real interleaved form of a complex matrix.
__global__ void k_tc_pack(const cd* __restrict__ T, int rows, int cols, int nrt, int nkc, float* __restrict__ out) {
    int64_t total = (int64_t)nrt * nkc * A_BLOCK;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t blk = i / A_BLOCK;
        int e = (int)(i % A_BLOCK);
        int rt = (int)(blk / nkc), kc = (int)(blk % nkc);
        int ri = e / TC_KC, ki = e % TC_KC;
        int rr = rt * TC_M + ri, kk = kc * TC_KC + ki;
        int r = rr >> 1, sr = rr & 1, k = kk >> 1, sk = kk & 1;
        double v = 0.0;
        if (r < rows && k < cols) {
            cd t = T[(int64_t)r * cols + k];
            v = sr == 0 ? (sk == 0 ? t.re : -t.im) : (sk == 0 ? t.im : t.re);
        }
        float f = (float)v;
        float hi = tf32_hi(f);
        float lo = (float)(v - (double)hi);
        float* base = out + blk * 2 * A_BLOCK;
        int off = canon(ri, ki) >> 2;
        base[off] = hi;
        base[A_BLOCK + off] = lo;
    }
}

// hi/lo planes of the multipoles of the tensor-core levels: box vectors of
// 2P floats padded to stride_f (multiple of 4) with zeros.
struct SplitLevel {
    int64_t src_base;     // complex offset of the level in the multipoles
    int64_t plane_base;   // float offset in the planes
    int32_t nbox, P, stride_f, pad;
};
// With nrhs right-hand sides a level's planes hold nrhs sets of nbox vectors
// (plane_base scaled by nrhs), set r read from mp + r * rstride.
__global__ void k_tc_split(const SplitLevel* __restrict__ lv, int nlev, const cf* __restrict__ mp,
                           float* __restrict__ hi, float* __restrict__ lo, int nrhs, int64_t rstride) {
    int l = blockIdx.y;
    if (l >= nlev) return;
    SplitLevel L = lv[l];
    int64_t per = (int64_t)L.nbox * L.stride_f;
    int64_t total = per * nrhs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / per, ib = i - r * per;
        int64_t b = ib / L.stride_f;
        int k = (int)(ib % L.stride_f);
        const float* src = (const float*)(mp + r * rstride + L.src_base);
        float v = k < 2 * L.P ? src[b * 2 * L.P + k] : 0.f;
        float h = tf32_hi(v);
        hi[L.plane_base * nrhs + i] = h;
        lo[L.plane_base * nrhs + i] = v - h;
    }
}

__global__ void __launch_bounds__(256, 2) k_trans_tc(const TcTask* __restrict__ tasks, const TcTile* __restrict__ tiles,
                                                      const float* __restrict__ Abuf, const int32_t* __restrict__ src_idx,
                                                      const int32_t* __restrict__ dst_idx,
                                                      const float* __restrict__ plane_hi,
                                                      const float* __restrict__ plane_lo, cf* __restrict__ dst,
                                                      int* __restrict__ err, int nrhs, int64_t rstride,
                                                      long long wait_limit, int inject_stall) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES];    // B producers' cp.async pieces
    __shared__ __align__(8) uint64_t a_bar[TC_STAGES];       // the A producer's bulk copy
    __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ __align__(8) uint64_t never_bar;              // test hook: nothing arrives on it
    __shared__ uint32_t tmem_holder;
    __shared__ int s_src[TC_NMAX];       // source vector index in the planes (rhs * nbox + box)
    __shared__ int s_dst[TC_NMAX];
    __shared__ int s_rhs[TC_NMAX];
    __shared__ int s_fail;
    uint32_t raw = smem_u32(smem_raw);
    uint32_t pad = (1024 - (raw & 1023)) & 1023;
    float* stage0 = (float*)(smem_raw + pad);

    const TcTile tl = tiles[blockIdx.x];
    const TcTask tk = tasks[tl.task];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncol = tl.ncol;
    const int nmma = (ncol + 15) & ~15;
    const int nkc = tk.nkc;
    // column j: pair (col0 + j) / nrhs, right-hand side (col0 + j) % nrhs
    for (int j = tid; j < TC_NMAX; j += blockDim.x) {
        bool ok = j < ncol;
        int col = tl.col0 + j;
        int pr = col / nrhs, rh = col - pr * nrhs;
        s_src[j] = ok ? rh * tk.nbox_src + src_idx[tk.pair_off + pr] : -1;
        s_dst[j] = ok ? dst_idx[tk.pair_off + pr] : -1;
        s_rhs[j] = ok ? rh : 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TC_NMAX));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_bar[s])), "r"(NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&a_bar[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty_bar[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done_bar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&never_bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;

    if (warp < 6) {
        // ---------------- B producers: 16-byte cp.async pieces -------------
        const int npieces = nmma * (TC_KC / 4) * 2;   // columns x K pieces x {hi, lo}
        for (int c = 0; c < nkc; ++c) {
            const int s = c % TC_STAGES, u = c / TC_STAGES;
            if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (u - 1) & 1, wait_limit)) {
                atomicExch(&s_fail, 1);
                break;
            }
            float* sBh = stage0 + s * STAGE_FLOATS + 2 * A_BLOCK;
            for (int i = tid; i < npieces; i += NPROD) {
                int plane = i & 1;
                int q = (i >> 1) % (TC_KC / 4);
                int j = (i >> 1) / (TC_KC / 4);
                int k = c * TC_KC + 4 * q;
                int sb = s_src[j];
                const float* pl = plane ? plane_lo : plane_hi;
                const int64_t base = tk.plane_base * nrhs;
                const float* g = pl + base;   // valid address even when nothing is read
                int bytes = 0;
                if (sb >= 0 && k < tk.stride_f) {
                    g = pl + base + (int64_t)sb * tk.stride_f + k;
                    bytes = 16;
                }
                uint32_t d = smem_u32(sBh + plane * B_BLOCK) + canon(j, 4 * q);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(bytes));
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full_bar[s])));
        }
        asm volatile("cp.async.wait_all;");
    } else if (warp == 6) {
        // ---------------- A producer: one bulk copy per stage ----------------
        if (lane == 0) {
            const float* Atile = Abuf + tk.a_off + (int64_t)tl.rt * nkc * 2 * A_BLOCK;
            int issued = 0;
            for (int c = 0; c < nkc; ++c) {
                const int s = c % TC_STAGES, u = c / TC_STAGES;
                if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (u - 1) & 1, wait_limit)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                uint32_t ab = smem_u32(&a_bar[s]);
                uint32_t dA = smem_u32(stage0 + s * STAGE_FLOATS);
                const float* g = Atile + (int64_t)c * 2 * A_BLOCK;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ab), "r"(2 * A_BLOCK * 4));
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dA),
                    "l"(g), "r"(2 * A_BLOCK * 4), "r"(ab));
                ++issued;
            }
            // every bulk copy this CTA issued lands before the CTA may exit
            // (on success the MMA issuer has already waited for each of them)
            for (int c = max(0, issued - TC_STAGES); c < issued; ++c)
                mbar_wait(smem_u32(&a_bar[c % TC_STAGES]), (c / TC_STAGES) & 1, DRAIN_LIMIT);
        }
        __syncwarp();
    } else {
        // ---------------- MMA issuer ----------------------------------------
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);
            // test hook: a wait on a barrier nothing arrives on runs out
            const bool stalled = inject_stall && !mbar_wait(smem_u32(&never_bar), 0, wait_limit);
            if (stalled) atomicExch(&s_fail, 1);
            for (int c = 0; c < nkc && !stalled; ++c) {
                const int s = c % TC_STAGES, u = c / TC_STAGES;
                if (!mbar_wait(smem_u32(&full_bar[s]), u & 1, wait_limit) ||
                    !mbar_wait(smem_u32(&a_bar[s]), u & 1, wait_limit)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                float* st = stage0 + s * STAGE_FLOATS;
                uint32_t aH = smem_u32(st), aL = smem_u32(st + A_BLOCK);
                uint32_t bH = smem_u32(st + 2 * A_BLOCK), bL = smem_u32(st + 2 * A_BLOCK + B_BLOCK);
#pragma unroll
                for (int ks = 0; ks < TC_KC / 8; ++ks) {
                    uint32_t o = ks * 2 * LBO;
                    uint32_t first = (c == 0 && ks == 0) ? 0u : 1u;
                    mma_tf32(tmem, umma_desc(aH + o), umma_desc(bH + o), idesc, first);
                    mma_tf32(tmem, umma_desc(aH + o), umma_desc(bL + o), idesc, 1u);
                    mma_tf32(tmem, umma_desc(aL + o), umma_desc(bH + o), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&empty_bar[s])));
            }
            // completion of every MMA issued above (also on failure)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&done_bar)));
        }
        __syncwarp();
    }

    // ---------------- epilogue ------------------------------------------------
    bool done = mbar_wait(smem_u32(&done_bar), 0, DRAIN_LIMIT);
    __syncthreads();
    const bool ok = done && s_fail == 0;
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int quad = warp & 3;
        const int half = warp >> 2;
        const int rr = tl.rt * TC_M + quad * 32 + lane;      // real output row
        const int r = rr >> 1, part = rr & 1;
        const int cmid = ((nmma / 16 + 1) / 2) * 16;        // split on 16-column boundaries
        const int cbeg = half ? cmid : 0;
        const int cend = half ? nmma : cmid;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            uint32_t v[16];
            uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (r < tk.p_out2) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    int j = c0 + q;
                    int db = s_dst[j];
                    if (db < 0) continue;
                    float* d = (float*)(dst + s_rhs[j] * rstride + tk.dst_base + (int64_t)db * tk.p_out2 + r) +
                               part;
                    atomicAdd(d, __uint_as_float(v[q]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NMAX));
}

// ------------------------------------------------------------- host side ----
struct TcPlanImpl {
    std::vector<TcTask> h_tasks;
    std::vector<TcTile> h_tiles;
    std::vector<SplitLevel> h_split;
    TcTask* tasks = nullptr;
    TcTile* tiles = nullptr;
    SplitLevel* split = nullptr;
    float* A = nullptr;
    float* plane_hi = nullptr;
    float* plane_lo = nullptr;
    int* err = nullptr;
    const int32_t* src_idx = nullptr;
    const int32_t* dst_idx = nullptr;
    int64_t a_floats = 0, plane_floats = 0;
    int max_split = 0;
    int plane_nrhs = 1;                     // right-hand sides the planes hold
    std::map<int, std::pair<TcTile*, int>> multi;   // tiles for nrhs > 1
};

// Bound of the pipeline's device waits (mbarrier polls) and the test hook
// that makes one of them run out; library-wide, read at each launch.
static std::atomic<long long> g_wait_limit{1LL << 26};
static std::atomic<int> g_inject_stall{0};
long long fb_tc_set_wait_limit(long long limit) { return g_wait_limit.exchange(limit); }
int fb_tc_set_inject_stall(int on) { return g_inject_stall.exchange(on ? 1 : 0); }
long long fb_tc_wait_limit() { return g_wait_limit.load(); }
int fb_tc_inject_stall() { return g_inject_stall.load(); }

size_t fb_tc_smem_bytes() { return (size_t)TC_STAGES * STAGE_FLOATS * sizeof(float) + 1024; }

// Builds a tensor-core plan for groups of box pairs; each group shares one
// composed translation matrix (job) and reads the source expansions of one
// level (hi/lo planes split once per run).
fb_status fb_tc_build_groups(fb_op* op, const std::vector<TcGroup>& groups, const int32_t* src_idx,
                             const int32_t* dst_idx, void** slot, cudaStream_t s) {
    const fb_tree* t = op->tree;
    TcPlanImpl* pl = new TcPlanImpl();
    *slot = pl;
    pl->src_idx = src_idx;
    pl->dst_idx = dst_idx;
    std::vector<int> split_of(FB_MAXLEV + 1, -1);
    for (const TcGroup& g : groups) {
        int ls = g.src_level;
        if (split_of[ls] < 0) {
            int Pin = op->p[ls] * op->p[ls];
            SplitLevel sl;
            sl.src_base = op->lev_off[ls];
            sl.plane_base = pl->plane_floats;
            sl.nbox = t->nbox[ls];
            sl.P = Pin;
            sl.stride_f = (2 * Pin + TC_KC - 1) / TC_KC * TC_KC;   // whole K chunks, 16-byte pieces
            sl.pad = 0;
            split_of[ls] = (int)pl->h_split.size();
            pl->h_split.push_back(sl);
            pl->plane_floats += (int64_t)sl.nbox * sl.stride_f;
            pl->max_split = std::max<int>(pl->max_split,
                                          (int)std::min<int64_t>((int64_t)sl.nbox * sl.stride_f / 256 + 1, 4096));
        }
        const SplitLevel& sl = pl->h_split[split_of[ls]];
        const ComposeJob& jb = op->h_jobs[g.job];
        int Pout = jb.p_out * jb.p_out;
        TcTask tk;
        tk.a_off = pl->a_floats;
        tk.pair_off = g.pair_off;
        tk.npairs = g.npairs;
        tk.nrt = (2 * Pout + TC_M - 1) / TC_M;
        tk.nkc = sl.stride_f / TC_KC;
        tk.p_out2 = Pout;
        tk.p_in2 = sl.P;
        tk.stride_f = sl.stride_f;
        tk.plane_base = sl.plane_base;
        tk.dst_base = op->lev_off[g.dst_level];
        tk.nbox_src = sl.nbox;
        tk.pad = 0;
        int ti = (int)pl->h_tasks.size();
        pl->h_tasks.push_back(tk);
        for (int rt = 0; rt < tk.nrt; ++rt)
            for (int c0 = 0; c0 < tk.npairs; c0 += TC_NMAX)
                pl->h_tiles.push_back(TcTile{ti, rt, c0, std::min(TC_NMAX, tk.npairs - c0)});
        pl->a_floats += (int64_t)tk.nrt * tk.nkc * 2 * A_BLOCK;
    }
    if (pl->h_tasks.empty()) return FB_OK;
    FB_CHECK(dalloc(&pl->A, pl->a_floats));
    FB_CHECK(dalloc(&pl->plane_hi, pl->plane_floats));
    FB_CHECK(dalloc(&pl->plane_lo, pl->plane_floats));
    FB_CHECK(dalloc(&pl->tasks, pl->h_tasks.size()));
    FB_CHECK(dalloc(&pl->tiles, pl->h_tiles.size()));
    FB_CHECK(dalloc(&pl->split, pl->h_split.size()));
    FB_CHECK(dalloc(&pl->err, 1));
    FB_CUDA(cudaMemsetAsync(pl->err, 0, sizeof(int), s));
    FB_CUDA(cudaMemcpyAsync(pl->tasks, pl->h_tasks.data(), sizeof(TcTask) * pl->h_tasks.size(),
                            cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemcpyAsync(pl->tiles, pl->h_tiles.data(), sizeof(TcTile) * pl->h_tiles.size(),
                            cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemcpyAsync(pl->split, pl->h_split.data(), sizeof(SplitLevel) * pl->h_split.size(),
                            cudaMemcpyHostToDevice, s));
    for (size_t i = 0; i < groups.size(); ++i) {
        const TcTask& tk = pl->h_tasks[i];
        const ComposeJob& jb = op->h_jobs[groups[i].job];
        int64_t total = (int64_t)tk.nrt * tk.nkc * A_BLOCK;
        k_tc_pack<<<(unsigned)std::min<int64_t>(div_up(total, 256), 4096), 256, 0, s>>>(
            op->T64 + jb.t_off, tk.p_out2, jb.p_in * jb.p_in, tk.nrt, tk.nkc, pl->A + tk.a_off);
    }
    FB_LAUNCH_CHECK();
    FB_CHECK(fb_smem_cap((const void*)k_trans_tc, fb_tc_smem_bytes()));
    return FB_OK;
}

// M2L groups (every non-empty (level, offset) group) of the given levels.
fb_status fb_tc_build(fb_op* op, const std::vector<int>& levels, void** slot, cudaStream_t s) {
    const fb_tree* t = op->tree;
    std::vector<TcGroup> groups;
    for (int l : levels)
        for (int c = 0; c < FB_NOFF; ++c) {
            int64_t g0 = t->m2l_group[(size_t)l * FB_NOFF + c], g1 = t->m2l_group[(size_t)l * FB_NOFF + c + 1];
            if (g1 == g0) continue;
            int job = op->m2l_job[(size_t)l * FB_NOFF + c];
            groups.push_back(TcGroup{job, g0, (int32_t)(g1 - g0), l, l});
        }
    return fb_tc_build_groups(op, groups, t->m2l_src, t->m2l_dst, slot, s);
}

// Runs a plan on nrhs sets of expansions (set r at src/dst + r * rstride).
// The columns of a task are its (pair, rhs) combinations, so every tile of
// the translation matrix is loaded once for all right-hand sides.
fb_status fb_tc_run(fb_op* op, void* plan, const cf* src, cf* dst, cudaStream_t s, int nrhs, int64_t rstride) {
    TcPlanImpl* pl = (TcPlanImpl*)plan;
    if (!pl || pl->h_tiles.empty()) return FB_OK;
    const TcTile* tiles = pl->tiles;
    int ntiles = (int)pl->h_tiles.size();
    if (nrhs > 1) {
        if (nrhs > pl->plane_nrhs) {
            cudaStreamSynchronize(s);
            dfree(pl->plane_hi);
            dfree(pl->plane_lo);
            FB_CHECK(dalloc(&pl->plane_hi, pl->plane_floats * nrhs));
            FB_CHECK(dalloc(&pl->plane_lo, pl->plane_floats * nrhs));
            pl->plane_nrhs = nrhs;
            op->buf_gen++;   // captured graphs of this operator refer to the old planes
        }
        auto it = pl->multi.find(nrhs);
        if (it == pl->multi.end()) {
            std::vector<TcTile> h;
            for (int ti = 0; ti < (int)pl->h_tasks.size(); ++ti) {
                const TcTask& tk = pl->h_tasks[ti];
                int ncol = tk.npairs * nrhs;
                for (int rt = 0; rt < tk.nrt; ++rt)
                    for (int c0 = 0; c0 < ncol; c0 += TC_NMAX)
                        h.push_back(TcTile{ti, rt, c0, std::min(TC_NMAX, ncol - c0)});
            }
            TcTile* d = nullptr;
            FB_CHECK(dalloc(&d, h.size()));
            FB_CUDA(cudaMemcpy(d, h.data(), sizeof(TcTile) * h.size(), cudaMemcpyHostToDevice));
            it = pl->multi.emplace(nrhs, std::make_pair(d, (int)h.size())).first;
        }
        tiles = it->second.first;
        ntiles = it->second.second;
    }
    dim3 sg(pl->max_split, (unsigned)pl->h_split.size());
    k_tc_split<<<sg, 256, 0, s>>>(pl->split, (int)pl->h_split.size(), src, pl->plane_hi, pl->plane_lo, nrhs,
                                  rstride);
    k_trans_tc<<<(unsigned)ntiles, 256, fb_tc_smem_bytes(), s>>>(pl->tasks, tiles, pl->A, pl->src_idx,
                                                                 pl->dst_idx, pl->plane_hi, pl->plane_lo, dst,
                                                                 pl->err, nrhs, rstride, g_wait_limit.load(),
                                                                 g_inject_stall.load());
    FB_LAUNCH_CHECK();
    fb_count_launch(2);
    return FB_OK;
}

// Error flags of the tensor-core kernels of an operator (1 = a bounded wait
// ran out); read and cleared (the caller has synchronised the work).
fb_status fb_tc_check(const fb_op* op) {
    std::vector<void*> plans = {op->tc_plan, op->tc_plan_all};
    for (int l = 0; l <= FB_MAXLEV; ++l) {
        plans.push_back(op->tc_m2m[l]);
        plans.push_back(op->tc_l2l[l]);
    }
    if (op->stc_err) {   // tensor-core staged rotation passes
        int h = 0;
        FB_CUDA(cudaMemcpy(&h, op->stc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (h) {
            FB_CUDA(cudaMemset(op->stc_err, 0, sizeof(int)));
            return fb_fail(FB_ERR_TIMEOUT, "tensor-core staged rotation kernel: a bounded wait ran out");
        }
    }
    for (void* v : plans) {
        TcPlanImpl* pl = (TcPlanImpl*)v;
        if (!pl || !pl->err) continue;
        int h = 0;
        FB_CUDA(cudaMemcpy(&h, pl->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (h) {
            FB_CUDA(cudaMemset(pl->err, 0, sizeof(int)));
            return fb_fail(FB_ERR_TIMEOUT, "tensor-core translation kernel: a bounded wait ran out");
        }
    }
    return FB_OK;
}

void fb_tc_free(void*& plan) {
    TcPlanImpl* pl = (TcPlanImpl*)plan;
    if (!pl) return;
    dfree(pl->A);
    dfree(pl->plane_hi);
    dfree(pl->plane_lo);
    dfree(pl->tasks);
    dfree(pl->tiles);
    dfree(pl->split);
    dfree(pl->err);
    for (auto& kv : pl->multi) dfree(kv.second.first);
    delete pl;
    plan = nullptr;
}
