// Autotuner of the translation passes.  For every level it times on the
// device (median of 3 runs, or one run for the batch scheduler's quick
// pass), for a given number of right-hand sides, the forms a translation
// pass can take and keeps the fastest:
//   * rotation - coaxial - rotation (RCR, Sec. 3.3) as per-pair tiles
//     (where a pair's working set fits a CTA's shared memory),
//   * RCR as staged batched GEMM passes (pairs grouped by polar angle and by
//     |t|; rcr_staged.cu), in mixed precision also with the rotation passes
//     on the tensor cores (rcr_staged_tc.cu), in FP64 also in double-FP32
//     arithmetic (as are the FP64 per-pair tiles),
//   * mixed precision only: the stacked tensor-core GEMM of composed
//     matrices (3xTF32),
// for M2L and for the M2M / L2L passes into that level.  The tensor-core
// candidate of an M2L level is skipped when its order exceeds 20, when it
// has fewer than 16 box pairs per translation vector on average, or when
// its composed matrices would exceed a memory cap.  The result replaces the
// operator's rule-based choice.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// Median of `reps` timed runs of f (after one untimed run), in ms.
template <class F>
fb_status time_ms(F&& f, cudaStream_t s, int reps, double* out) {
    Timer t;
    FB_CHECK(f());
    std::vector<float> v;
    for (int i = 0; i < reps; ++i) {
        FB_CUDA(cudaEventRecord(t.a, s));
        FB_CHECK(f());
        FB_CUDA(cudaEventRecord(t.b, s));
        FB_CUDA(cudaEventSynchronize(t.b));
        float ms = 0.f;
        FB_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
        v.push_back(ms);
    }
    std::sort(v.begin(), v.end());
    *out = v[v.size() / 2];
    return FB_OK;
}

void free_rcr(RcrPlan& p) { fb_rcr_free(p); }

// Candidates worth timing (measured crossovers on GB300: per-pair tiles lose
// to the staged passes from order ~40 on and by ~5x at 89; the staged passes
// lose below order ~30, where a level's coefficient blocks are small).  A
// level always keeps at least one candidate.
bool rcr_tile_candidate(int p, size_t csz) { return fb_rcr_tile_fits(p, p, csz) && p < 60; }
bool rcr_staged_candidate(int p, size_t csz) { return p >= 24 || !rcr_tile_candidate(p, csz); }
// double-FP32 passes: their arithmetic runs several times faster than FP64,
// which moves the crossover with the FP64 tiles to lower orders
bool rcr_df_candidate(int p) { return p >= 16; }
// staged passes with tensor-core rotations: their degree blocks pack into
// one tile up to 256 columns, so low orders stay worth timing
bool rcr_stc_candidate(int p) { return p >= 12; }

}  // namespace

fb_status fb_install_forms(fb_op* op, const std::vector<int>& tc_m2l, cudaStream_t s);

// Times the tasks of `base` that `pick` selects, with their RCR form set to
// `staged`, as a temporary plan on the expansion buffers (-1: no task).
template <class Pick>
fb_status time_rcr(fb_op* op, const RcrPlan& base, Pick pick, int staged, void* src, void* dst, cudaStream_t s,
                   int nrhs, int64_t cnt, int reps, double* ms) {
    *ms = -1.0;
    RcrPlan pl;
    for (const RcrTask& tk : base.h_tasks)
        if (pick(tk)) {
            RcrTask t2 = tk;
            t2.staged = staged;
            pl.h_tasks.push_back(t2);
        }
    if (pl.h_tasks.empty()) return FB_OK;
    const size_t csz = op->prec == FB_PREC_MIXED_FMM ? sizeof(cf) : sizeof(cd);
    fb_status st = fb_rcr_upload(op, pl, base.src_idx, base.dst_idx, csz);
    if (st == FB_OK) st = time_ms([&]() { return fb_rcr_run_op(op, pl, src, dst, s, nrhs, cnt); }, s, reps, ms);
    cudaStreamSynchronize(s);
    free_rcr(pl);
    return st;
}

// times[14 * l + {0..11}] = M2L RCR tiles, M2L tensor, M2M+L2L RCR tiles,
// M2M+L2L tensor, M2L RCR staged, M2M+L2L RCR staged, M2L RCR staged with
// tensor-core rotations, M2M+L2L RCR staged with tensor-core rotations, M2L
// RCR staged in double-FP32, M2M+L2L RCR staged in double-FP32, M2L RCR
// tiles in double-FP32, M2M+L2L RCR tiles in double-FP32 (ms, -1 when not a
// candidate) for l = 0..L; choice[l] bit 0 = M2L on the tensor cores, bit 1
// = M2M/L2L into level l on the tensor cores, bit 2 = M2L by staged RCR,
// bit 3 = M2M/L2L into level l by staged RCR, bit 4 = the staged M2L's
// rotations on the tensor cores, bit 5 = the same for M2M/L2L, bit 6 = the
// staged M2L in double-FP32, bit 7 = the same for M2M/L2L, bit 8 = the M2L
// tiles in double-FP32, bit 9 = the same for M2M/L2L, bit 10 = the staged
// M2L's coaxial step on the tensor cores too (with bit 4), bit 11 = the same
// for M2M/L2L (with bit 5); times[14 l + 12, 13] time those forms.
fb_status fb_autotune_impl(fb_op* op, int nrhs, cudaStream_t s, double* times_out, int* choice, int reps) {
    const bool mixed = op->prec == FB_PREC_MIXED_FMM;
    double times_local[FB_TUNE_TIMES * (FB_MAXLEV + 1)];
    double* times = times_out ? times_out : times_local;   // callers may pass NULL
    const fb_tree* t = op->tree;
    const int L = op->L;
    const int64_t cnt = op->lev_off[L + 1];
    const size_t csz = mixed ? sizeof(cf) : sizeof(cd);
    reps = std::max(1, reps);
    const double cap_bytes = 8.0e9;   // composed FP64 + packed TF32 tiles of one level
    // expansion buffers for nrhs sets (contents do not matter for timing)
    if (nrhs > op->exp_nrhs) {
        cudaStreamSynchronize(s);
        dfree(op->mp);
        dfree(op->loc);
        op->mp = op->loc = nullptr;
        FB_CHECK(dalloc((unsigned char**)&op->mp, (size_t)cnt * nrhs * csz));
        FB_CHECK(dalloc((unsigned char**)&op->loc, (size_t)cnt * nrhs * csz));
        op->exp_nrhs = nrhs;
        op->buf_gen++;
    }
    void* mp = op->mp;
    void* loc = op->loc;
    FB_CUDA(cudaMemsetAsync(mp, 0, csz * cnt * nrhs, s));
    FB_CUDA(cudaMemsetAsync(loc, 0, csz * cnt * nrhs, s));
    std::vector<int> tc_m2l;
    int stg_m2l[FB_MAXLEV + 1] = {0}, stg_pair[FB_MAXLEV + 1] = {0};
    for (int l = 2; l <= L; ++l) {
        double* tl = times + FB_TUNE_TIMES * l;
        for (int q = 0; q < FB_TUNE_TIMES; ++q) tl[q] = -1.0;
        int ch = 0;
        // ---- M2L of level l: RCR tiles, RCR staged, tensor cores
        auto at_level = [&](const RcrTask& tk) { return tk.src_base == op->lev_off[l] && tk.dst_base == tk.src_base; };
        if (rcr_tile_candidate(op->p[l], csz)) {
            FB_CHECK(time_rcr(op, op->m2l_rcr, at_level, 0, mp, loc, s, nrhs, cnt, reps, &tl[0]));
            if (!mixed) FB_CHECK(time_rcr(op, op->m2l_rcr, at_level, 4, mp, loc, s, nrhs, cnt, reps, &tl[10]));
        }
        if (rcr_staged_candidate(op->p[l], csz))
            FB_CHECK(time_rcr(op, op->m2l_rcr, at_level, 1, mp, loc, s, nrhs, cnt, reps, &tl[4]));
        if (mixed && rcr_stc_candidate(op->p[l])) {
            FB_CHECK(time_rcr(op, op->m2l_rcr, at_level, 2, mp, loc, s, nrhs, cnt, reps, &tl[6]));
            FB_CHECK(time_rcr(op, op->m2l_rcr, at_level, 5, mp, loc, s, nrhs, cnt, reps, &tl[12]));
        }
        if (!mixed && rcr_df_candidate(op->p[l]))
            FB_CHECK(time_rcr(op, op->m2l_rcr, at_level, 3, mp, loc, s, nrhs, cnt, reps, &tl[8]));
        double best = -1.0;
        if (tl[0] >= 0) best = tl[0];
        for (int form = 1; form <= 5; ++form) {
            const double v = tl[2 + 2 * form];
            if (v >= 0 && (best < 0 || v < best)) {
                best = v;
                stg_m2l[l] = form;
            }
        }
        if (mixed && best >= 0) {
            int64_t p2 = (int64_t)op->p[l] * op->p[l];
            double bytes = 0;
            int64_t groups = 0, pairs = 0;
            for (int c = 0; c < FB_NOFF; ++c) {
                int64_t g = t->m2l_group[(size_t)l * FB_NOFF + c + 1] - t->m2l_group[(size_t)l * FB_NOFF + c];
                if (g > 0) {
                    bytes += (double)p2 * p2 * (16.0 + 2 * 8.0);
                    ++groups;
                    pairs += g;
                }
            }
            // the composed form costs ~p/4 times the RCR arithmetic: only dense
            // levels of moderate order are worth timing
            const bool candidate = op->p[l] <= 20 && pairs >= 16 * groups;
            if (candidate && bytes <= cap_bytes) {
                std::vector<int> need;
                for (size_t j = 0; j < op->h_jobs.size(); ++j)
                    if (op->h_job_m2l[j] && op->h_job_level[j] == l) need.push_back((int)j);
                FB_CHECK(fb_compose_jobs(op, need, s));
                void* plan = nullptr;
                fb_status st2 = fb_tc_build(op, {l}, &plan, s);
                if (st2 == FB_OK)
                    st2 = time_ms([&]() { return fb_tc_run(op, plan, (const cf*)mp, (cf*)loc, s, nrhs, cnt); }, s,
                                  reps, &tl[1]);
                cudaStreamSynchronize(s);
                fb_tc_free(plan);
                FB_CHECK(st2);
                if (tl[1] < best) {
                    ch |= 1;
                    tc_m2l.push_back(l);
                }
            }
        }
        if (stg_m2l[l] && !(ch & 1)) {
            const int f = stg_m2l[l];
            ch |= f == 4 ? 256 : (f == 5 ? 4 | 16 | 1024 : (f == 2 ? 4 | 16 : (f == 3 ? 4 | 64 : 4)));
        }
        // ---- M2M + L2L between levels l-1 and l
        if (l >= 3) {
            const int pm = std::max(op->p[l], op->p[l - 1]);
            auto all = [](const RcrTask&) { return true; };
            double rt = -1.0, rs = -1.0, rc = -1.0, rd = -1.0, rtd = -1.0, rcc = -1.0;
            if (rcr_tile_candidate(pm, csz)) {
                double a = 0, b = 0;
                FB_CHECK(time_rcr(op, op->m2m_rcr[l], all, 0, mp, mp, s, nrhs, cnt, reps, &a));
                FB_CHECK(time_rcr(op, op->l2l_rcr[l], all, 0, loc, loc, s, nrhs, cnt, reps, &b));
                rt = std::max(a, 0.0) + std::max(b, 0.0);
                if (!mixed) {
                    FB_CHECK(time_rcr(op, op->m2m_rcr[l], all, 4, mp, mp, s, nrhs, cnt, reps, &a));
                    FB_CHECK(time_rcr(op, op->l2l_rcr[l], all, 4, loc, loc, s, nrhs, cnt, reps, &b));
                    rtd = std::max(a, 0.0) + std::max(b, 0.0);
                }
            }
            if (rcr_staged_candidate(pm, csz)) {
                double a = 0, b = 0;
                FB_CHECK(time_rcr(op, op->m2m_rcr[l], all, 1, mp, mp, s, nrhs, cnt, reps, &a));
                FB_CHECK(time_rcr(op, op->l2l_rcr[l], all, 1, loc, loc, s, nrhs, cnt, reps, &b));
                rs = std::max(a, 0.0) + std::max(b, 0.0);
            }
            if (mixed && rcr_stc_candidate(pm)) {
                double a = 0, b = 0;
                FB_CHECK(time_rcr(op, op->m2m_rcr[l], all, 2, mp, mp, s, nrhs, cnt, reps, &a));
                FB_CHECK(time_rcr(op, op->l2l_rcr[l], all, 2, loc, loc, s, nrhs, cnt, reps, &b));
                rc = std::max(a, 0.0) + std::max(b, 0.0);
                FB_CHECK(time_rcr(op, op->m2m_rcr[l], all, 5, mp, mp, s, nrhs, cnt, reps, &a));
                FB_CHECK(time_rcr(op, op->l2l_rcr[l], all, 5, loc, loc, s, nrhs, cnt, reps, &b));
                rcc = std::max(a, 0.0) + std::max(b, 0.0);
            }
            if (!mixed && rcr_df_candidate(pm)) {
                double a = 0, b = 0;
                FB_CHECK(time_rcr(op, op->m2m_rcr[l], all, 3, mp, mp, s, nrhs, cnt, reps, &a));
                FB_CHECK(time_rcr(op, op->l2l_rcr[l], all, 3, loc, loc, s, nrhs, cnt, reps, &b));
                rd = std::max(a, 0.0) + std::max(b, 0.0);
            }
            tl[2] = rt;
            tl[5] = rs;
            tl[7] = rc;
            tl[9] = rd;
            tl[11] = rtd;
            tl[13] = rcc;
            double best2 = rt;
            if (rt < 0 || (rs >= 0 && rs < rt)) {
                best2 = rs;
                stg_pair[l] = 1;
            }
            if (rc >= 0 && (best2 < 0 || rc < best2)) {
                best2 = rc;
                stg_pair[l] = 2;
            }
            if (rd >= 0 && (best2 < 0 || rd < best2)) {
                best2 = rd;
                stg_pair[l] = 3;
            }
            if (rtd >= 0 && (best2 < 0 || rtd < best2)) {
                best2 = rtd;
                stg_pair[l] = 4;
            }
            if (rcc >= 0 && (best2 < 0 || rcc < best2)) {
                best2 = rcc;
                stg_pair[l] = 5;
            }
            std::vector<int> need;
            std::vector<TcGroup> up, down;
            for (int o = 0; o < 8; ++o) {
                int64_t g0 = t->oct_group[l][o], g1 = t->oct_group[l][o + 1];
                if (g1 == g0) continue;
                need.push_back(op->m2m_job[l][o]);
                need.push_back(op->l2l_job[l][o]);
                up.push_back(TcGroup{op->m2m_job[l][o], g0, (int32_t)(g1 - g0), l, l - 1});
                down.push_back(TcGroup{op->l2l_job[l][o], g0, (int32_t)(g1 - g0), l - 1, l});
            }
            if (mixed && !up.empty() && fb_composable(op, l, true)) {
                FB_CHECK(fb_compose_jobs(op, need, s));
                if (!op->tc_m2m[l])
                    FB_CHECK(fb_tc_build_groups(op, up, t->oct_child[l], t->oct_parent[l], &op->tc_m2m[l], s));
                if (!op->tc_l2l[l])
                    FB_CHECK(fb_tc_build_groups(op, down, t->oct_parent[l], t->oct_child[l], &op->tc_l2l[l], s));
                double a = 0, b = 0;
                FB_CHECK(time_ms([&]() { return fb_tc_run(op, op->tc_m2m[l], (const cf*)mp, (cf*)mp, s, nrhs, cnt); },
                                 s, reps, &a));
                FB_CHECK(time_ms([&]() { return fb_tc_run(op, op->tc_l2l[l], (const cf*)loc, (cf*)loc, s, nrhs, cnt); },
                                 s, reps, &b));
                tl[3] = a + b;
                if (tl[3] < best2) {
                    ch |= 2;
                } else {
                    cudaStreamSynchronize(s);
                    fb_tc_free(op->tc_m2m[l]);
                    fb_tc_free(op->tc_l2l[l]);
                }
            }
            if (stg_pair[l] && !(ch & 2)) {
                const int f = stg_pair[l];
                ch |= f == 4 ? 512 : (f == 5 ? 8 | 32 | 2048 : (f == 2 ? 8 | 32 : (f == 3 ? 8 | 128 : 8)));
            }
        }
        if (choice) choice[l] = ch;
    }
    FB_CUDA(cudaStreamSynchronize(s));
    FB_CHECK(fb_rcr_restage(op, stg_m2l, stg_pair));
    if (!mixed) return FB_OK;
    return fb_install_forms(op, tc_m2l, s);
}

// Installs per-level M2L forms: tensor-core plan of `tc_m2l` levels, RCR for
// the rest.
fb_status fb_install_forms(fb_op* op, const std::vector<int>& tc_m2l, cudaStream_t s) {
    const fb_tree* t = op->tree;
    const size_t csz = sizeof(cf);
    if (!tc_m2l.empty()) {
        std::vector<int> need;
        for (size_t j = 0; j < op->h_jobs.size(); ++j)
            if (op->h_job_m2l[j] && std::find(tc_m2l.begin(), tc_m2l.end(), op->h_job_level[j]) != tc_m2l.end())
                need.push_back((int)j);
        FB_CHECK(fb_compose_jobs(op, need, s));
    }
    FB_CUDA(cudaStreamSynchronize(s));
    op->buf_gen++;   // captured graphs refer to the plans replaced here
    fb_tc_free(op->tc_plan);
    free_rcr(op->m2l_rcr_rest);
    op->m2l_rcr_rest.h_tasks.clear();
    for (int l = 0; l <= FB_MAXLEV; ++l) op->tc_level[l] = 0;
    for (int l : tc_m2l) op->tc_level[l] = 1;
    for (const RcrTask& tk : op->m2l_rcr.h_tasks) {
        bool tc = false;
        for (int l : tc_m2l) tc = tc || tk.src_base == op->lev_off[l];
        if (!tc) op->m2l_rcr_rest.h_tasks.push_back(tk);
    }
    FB_CHECK(fb_rcr_upload(op, op->m2l_rcr_rest, t->m2l_src, t->m2l_dst, csz));
    if (!tc_m2l.empty()) FB_CHECK(fb_tc_build(op, tc_m2l, &op->tc_plan, s));
    FB_CUDA(cudaStreamSynchronize(s));
    op->method = FB_TRANS_AUTO;
    return FB_OK;
}

// Installs a given per-level choice (bits as returned by the autotuner);
// lets a tuned configuration be saved and restored.
fb_status fb_set_forms_impl(fb_op* op, const int* choice, cudaStream_t s) {
    const fb_tree* t = op->tree;
    const int L = op->L;
    int stg_m2l[FB_MAXLEV + 1] = {0}, stg_pair[FB_MAXLEV + 1] = {0};
    for (int l = 2; l <= L; ++l) {
        const int c = choice[l];
        if (op->prec != FB_PREC_MIXED_FMM && (c & (1 | 2 | 16 | 32 | 1024 | 2048)))
            return fb_fail(FB_ERR_ARG, "tensor-core forms apply to mixed operators");
        if (op->prec != FB_PREC_FP64_FMM && (c & (64 | 128 | 256 | 512)))
            return fb_fail(FB_ERR_ARG, "double-FP32 forms apply to FP64 operators");
        if (((c & (16 | 64)) && !(c & 4)) || ((c & (32 | 128)) && !(c & 8)))
            return fb_fail(FB_ERR_ARG, "bits 4-7 refine the staged bits 2/3");
        if (((c & 256) && (c & 4)) || ((c & 512) && (c & 8)))
            return fb_fail(FB_ERR_ARG, "bits 8/9 (tiles in double-FP32) exclude the staged bits 2/3");
        if (((c & 1024) && !(c & 16)) || ((c & 2048) && !(c & 32)))
            return fb_fail(FB_ERR_ARG, "bits 10/11 (tensor-core coaxial step) refine bits 4/5");
        stg_m2l[l] = (c & 4) ? ((c & 16) ? ((c & 1024) ? 5 : 2) : ((c & 64) ? 3 : 1)) : ((c & 256) ? 4 : 0);
        stg_pair[l] = (c & 8) ? ((c & 32) ? ((c & 2048) ? 5 : 2) : ((c & 128) ? 3 : 1)) : ((c & 512) ? 4 : 0);
    }
    FB_CHECK(fb_rcr_restage(op, stg_m2l, stg_pair));
    if (op->prec != FB_PREC_MIXED_FMM) return FB_OK;
    std::vector<int> tc_m2l;
    for (int l = 2; l <= L; ++l) {
        if ((choice[l] & 1) && !fb_composable(op, l, false))
            return fb_fail(FB_ERR_ARG, "tensor-core M2L needs order <= " + std::to_string(FB_COMPOSE_PMAX));
        if (l >= 3 && (choice[l] & 2) && !fb_composable(op, l, true))
            return fb_fail(FB_ERR_ARG, "tensor-core M2M/L2L needs order <= " + std::to_string(FB_COMPOSE_PMAX));
    }
    for (int l = 2; l <= L; ++l) {
        if (choice[l] & 1) tc_m2l.push_back(l);
        if (l < 3) continue;
        bool want = (choice[l] & 2) != 0;
        if (!want) {
            FB_CUDA(cudaStreamSynchronize(s));
            op->buf_gen++;
            fb_tc_free(op->tc_m2m[l]);
            fb_tc_free(op->tc_l2l[l]);
        } else if (!op->tc_m2m[l] || !op->tc_l2l[l]) {
            std::vector<int> need;
            std::vector<TcGroup> up, down;
            for (int o = 0; o < 8; ++o) {
                int64_t g0 = t->oct_group[l][o], g1 = t->oct_group[l][o + 1];
                if (g1 == g0) continue;
                need.push_back(op->m2m_job[l][o]);
                need.push_back(op->l2l_job[l][o]);
                up.push_back(TcGroup{op->m2m_job[l][o], g0, (int32_t)(g1 - g0), l, l - 1});
                down.push_back(TcGroup{op->l2l_job[l][o], g0, (int32_t)(g1 - g0), l - 1, l});
            }
            if (up.empty()) continue;
            FB_CHECK(fb_compose_jobs(op, need, s));
            if (!op->tc_m2m[l])
                FB_CHECK(fb_tc_build_groups(op, up, t->oct_child[l], t->oct_parent[l], &op->tc_m2m[l], s));
            if (!op->tc_l2l[l])
                FB_CHECK(fb_tc_build_groups(op, down, t->oct_parent[l], t->oct_child[l], &op->tc_l2l[l], s));
        }
    }
    return fb_install_forms(op, tc_m2l, s);
}
