// Batch scheduler: many (frequency, source-set) solves with uneven mesh
// sizes (the paper's frequency sweeps, Sec. 4, treat every frequency and
// source independently).  Per job it builds the operators once (mixed FMM
// for the Krylov matvecs, FP64 FMM for the true residual and the right-hand
// side b = L gamma), block Jacobi, optionally autotunes the translation
// forms for the job's number of right-hand sides, and solves all of the
// job's sources as one lockstep batched FGMRES (one multi-RHS matvec per
// Arnoldi step).  Jobs run largest predicted cost first; with look-ahead a
// host thread builds the next job's operators on a second stream while the
// current job solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

int fb_order_rule(double k, double delta, double d0, int pmin);

namespace {

struct JobState {
    fb_op* A32 = nullptr;
    fb_op* A64 = nullptr;
    fb_op* L64 = nullptr;
    fb_precond* pc = nullptr;
    fb_op* Alow = nullptr;        // inner-outer: low-accuracy operator,
    fb_precond* pclow = nullptr;  // its block Jacobi,
    fb_precond* inner = nullptr;  // and the preconditioner of the solve
    fb_status st = FB_OK;
    std::string msg;          // error text of a failed setup (kept per thread by the library)
    double setup_ms = 0;
    void release() {
        fb_precond_destroy(inner);
        fb_precond_destroy(pclow);
        fb_operator_destroy(Alow);
        inner = pclow = nullptr;
        Alow = nullptr;
        fb_precond_destroy(pc);
        fb_operator_destroy(A32);
        fb_operator_destroy(A64);
        fb_operator_destroy(L64);
        pc = nullptr;
        A32 = A64 = L64 = nullptr;
    }
};

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void setup_job(const fb_batch_job& jb, const fb_batch_opts& o, cudaStream_t s, JobState& js, int dev) {
    cudaSetDevice(dev);   // the current device is per host thread
    double t0 = now_ms();
    auto run = [&]() -> fb_status {
        // the FP64 true-residual operator first: the mixed operators copy its near-field entries
        if (o.fp64_judge) {
            FB_CHECK(fb_operator_create(jb.mesh, jb.tree, jb.k, FB_OP_A, FB_PREC_FP64_FMM, o.d0, o.pmin, s, &js.A64));
            FB_CHECK(fb_operator_create_like(js.A64, FB_PREC_MIXED_FMM, o.d0, o.pmin, s, &js.A32));
        } else {
            FB_CHECK(fb_operator_create(jb.mesh, jb.tree, jb.k, FB_OP_A, FB_PREC_MIXED_FMM, o.d0, o.pmin, s, &js.A32));
        }
        FB_CHECK(fb_operator_create(jb.mesh, jb.tree, jb.k, FB_OP_L, FB_PREC_FP64_FMM, o.d0, o.pmin, s, &js.L64));
        FB_CHECK(fb_precond_create(js.A32, FB_PC_BLOCK_JACOBI, s, &js.pc));
        const int nrhs = std::max(1, std::min(jb.nsrc, o.max_rhs));
        // one timed run per candidate: the setup of a sweep, not its solves,
        // bounds a batch's throughput
        if (o.autotune) FB_CHECK(fb_autotune_impl(js.A32, nrhs, s, nullptr, nullptr, 1));
        if (o.inner_iters > 0) {
            if (js.A64)
                FB_CHECK(fb_operator_create_like(js.A64, FB_PREC_MIXED_FMM, o.inner_d0, o.inner_pmin, s, &js.Alow));
            else
                FB_CHECK(fb_operator_create(jb.mesh, jb.tree, jb.k, FB_OP_A, FB_PREC_MIXED_FMM, o.inner_d0,
                                            o.inner_pmin, s, &js.Alow));
            FB_CHECK(fb_precond_create(js.Alow, FB_PC_BLOCK_JACOBI, s, &js.pclow));
            FB_CHECK(fb_operator_set_near_bf16(js.Alow, 1, s));   // low-accuracy operator: 16-bit near field
            FB_CHECK(fb_precond_create_inner(js.A32, js.Alow, js.pclow, o.inner_iters, s, &js.inner));
            FB_CHECK(fb_operator_use_graphs(js.Alow, 1));
            FB_CHECK(fb_precond_use_graphs(js.inner, 1));
        }
        FB_CUDA(cudaStreamSynchronize(s));
        return FB_OK;
    };
    js.st = run();
    if (js.st != FB_OK) {
        char buf[1024];
        fb_last_error(buf, sizeof(buf));
        js.msg = buf;
    }
    js.setup_ms = now_ms() - t0;
}

fb_status solve_job(fb_batch_job& jb, const fb_batch_opts& o, cudaStream_t s, JobState& js) {
    const int64_t n = jb.mesh->n;
    cd *G = nullptr, *B = nullptr;
    auto cleanup = [&]() { dfree(G); dfree(B); };
    fb_status st = FB_OK;
    if ((st = dalloc(&G, (size_t)n * jb.nsrc)) || (st = dalloc(&B, (size_t)n * jb.nsrc))) {
        cleanup();
        return st;
    }
    double t0 = now_ms();
    for (int q = 0; q < jb.nsrc && st == FB_OK; ++q)
        st = fb_gamma_monopole(jb.mesh, jb.k, jb.src + 3 * q, (double*)(G + q * n), FB_MEM_DEVICE, s);
    const int step = std::max(1, std::min(o.max_rhs, (int)FB_MAX_RHS));
    for (int q0 = 0; q0 < jb.nsrc && st == FB_OK; q0 += step) {
        int r = std::min(step, jb.nsrc - q0);
        st = fb_operator_apply_multi(js.L64, (const double*)(G + q0 * n), (double*)(B + q0 * n), r, FB_MEM_DEVICE, s);
        if (st != FB_OK) break;
        fb_solver_opts so{o.tol, o.restart, o.maxit, 4, 0.0, js.A64};
        fb_status sv = fb_fgmres_solve_multi(js.A32, js.inner ? js.inner : js.pc, (const double*)(B + q0 * n),
                                             jb.x + 2 * q0 * n, r, &so,
                                             jb.info ? jb.info + q0 : nullptr, FB_MEM_DEVICE, s);
        if (sv != FB_OK && jb.status == FB_OK) jb.status = sv;
        if (sv != FB_OK && sv != FB_ERR_NOCONV && sv != FB_ERR_NAN) st = sv;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == FB_OK && e != cudaSuccess) st = fb_fail(FB_ERR_CUDA, cudaGetErrorString(e));
    jb.solve_ms = now_ms() - t0;
    cleanup();
    return st;
}

}  // namespace

fb_status fb_batch_solve_impl(fb_batch_job* jobs, int njobs, const fb_batch_opts* opts) {
    fb_batch_opts o = *opts;
    if (o.max_rhs < 1) o.max_rhs = 8;
    if (o.restart < 1) o.restart = 40;
    if (o.maxit < 1) o.maxit = 3000;
    if (!(o.d0 > 0)) o.d0 = 6.0;
    if (o.pmin < 1) o.pmin = 12;
    if (o.inner_iters < 0) o.inner_iters = 0;
    if (!(o.inner_d0 > 0)) o.inner_d0 = 0.5;
    if (o.inner_pmin < 1) o.inner_pmin = 2;
    for (int i = 0; i < njobs; ++i) {
        const fb_batch_job& jb = jobs[i];
        if (!jb.mesh || !jb.tree || !jb.src || !jb.x || jb.nsrc < 1 || !(jb.k > 0))
            return fb_fail(FB_ERR_ARG, "batch job " + std::to_string(i) + ": bad arguments");
        if (jb.tree->mesh != jb.mesh) return fb_fail(FB_ERR_ARG, "batch job " + std::to_string(i) + ": tree of another mesh");
    }
    // largest predicted cost first: sources x N x (leaf order)^2
    std::vector<int> order(njobs);
    std::vector<double> cost(njobs);
    for (int i = 0; i < njobs; ++i) {
        const fb_tree* t = jobs[i].tree;
        double delta = t->side / (double)(1 << t->L);
        int p = fb_order_rule(jobs[i].k, delta, o.d0, o.pmin);
        cost[i] = (double)jobs[i].nsrc * (double)jobs[i].mesh->n * p * p;
        order[i] = i;
        jobs[i].status = FB_OK;
        jobs[i].order = -1;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    int dev = 0;
    FB_CUDA(cudaGetDevice(&dev));
    cudaStream_t s[2];
    FB_CUDA(cudaStreamCreateWithFlags(&s[0], cudaStreamNonBlocking));
    FB_CUDA(cudaStreamCreateWithFlags(&s[1], cudaStreamNonBlocking));
    std::vector<JobState> state(njobs);
    fb_status worst = FB_OK;
    std::string first_msg;
    if (njobs > 0) setup_job(jobs[order[0]], o, s[0], state[order[0]], dev);
    for (int qi = 0; qi < njobs; ++qi) {
        int i = order[qi];
        jobs[i].order = qi;
        std::thread ahead;
        if (qi + 1 < njobs) {
            int nx = order[qi + 1];
            if (o.lookahead) ahead = std::thread(setup_job, std::cref(jobs[nx]), std::cref(o), s[(qi + 1) & 1],
                                                 std::ref(state[nx]), dev);
        }
        JobState& js = state[i];
        jobs[i].setup_ms = js.setup_ms;
        fb_status st = js.st;
        if (st != FB_OK) fb_set_error(st, "batch job " + std::to_string(i) + " setup: " + js.msg);
        if (st == FB_OK) st = solve_job(jobs[i], o, s[qi & 1], js);
        if (st != FB_OK && jobs[i].status == FB_OK) jobs[i].status = st;
        if (jobs[i].status != FB_OK && first_msg.empty()) {
            char buf[1024];
            fb_last_error(buf, sizeof(buf));
            first_msg = "batch job " + std::to_string(i) + ": " + buf;
        }
        js.release();
        if (ahead.joinable()) ahead.join();
        else if (qi + 1 < njobs) setup_job(jobs[order[qi + 1]], o, s[(qi + 1) & 1], state[order[qi + 1]], dev);
        if (worst == FB_OK && jobs[i].status != FB_OK) worst = jobs[i].status;
    }
    cudaStreamDestroy(s[0]);
    cudaStreamDestroy(s[1]);
    if (worst != FB_OK) fb_set_error(worst, first_msg);
    return worst;
}

// Largest-first greedy bin-packing of independent jobs over ranks (Sec. 4:
// frequencies and sources are independent solves, so a sweep shards over
// GPUs without any exchange): jobs in order of decreasing cost (index order
// on ties), each to the rank with the least load so far (lowest rank on
// ties).  The makespan is within 4/3 of the optimum (Graham's bound for
// this rule).  Host only.
extern "C" fb_status fb_batch_partition(const double* cost, int njobs, int nranks, int* owner, double* load) {
    if (njobs < 0 || nranks < 1 || (njobs > 0 && (!cost || !owner)))
        return fb_fail(FB_ERR_ARG, "fb_batch_partition: bad arguments");
    for (int i = 0; i < njobs; ++i)
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i]))
            return fb_fail(FB_ERR_ARG, "fb_batch_partition: costs must be finite and >= 0");
    std::vector<int> order(njobs);
    for (int i = 0; i < njobs; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> ld(nranks, 0.0);
    for (int i : order) {
        int r = 0;
        for (int q = 1; q < nranks; ++q)
            if (ld[q] < ld[r]) r = q;
        owner[i] = r;
        ld[r] += cost[i];
    }
    if (load)
        for (int q = 0; q < nranks; ++q) load[q] = ld[q];
    return FB_OK;
}
