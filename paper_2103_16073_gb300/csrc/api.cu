// C ABI entry points (include/fmmbem.h): argument checks, host/device
// memory-space handling and dispatch to the CUDA implementation.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include <map>
#include <mutex>

#include "common.cuh"

// implemented in the other translation units
fb_status fb_mesh_create_impl(const double*, int64_t, const int32_t*, int64_t, cudaStream_t, fb_mesh**);
void fb_mesh_free(fb_mesh*);
fb_status fb_gamma_impl(const fb_mesh*, double, const double*, cd*, cudaStream_t);
fb_status fb_eval_impl(const fb_mesh*, double, const cd*, const cd*, const double*, const double*, int64_t,
                       cd*, cudaStream_t);
fb_status fb_tree_build_impl(const fb_mesh*, int, cudaStream_t, fb_tree**);
void fb_tree_free(fb_tree*);
fb_status fb_tree_export_impl(const fb_tree*, int, int, int64_t*, int64_t*);
fb_status fb_fgmres_impl(fb_op*, fb_precond*, const cd*, cd*, const fb_solver_opts*, fb_solve_info*, cudaStream_t);
fb_status fb_fgmres_multi_impl(fb_op*, fb_precond*, const cd*, cd*, int, const fb_solver_opts*, fb_solve_info*,
                               cudaStream_t);
fb_status fb_precond_create_impl(fb_op*, int, cudaStream_t, fb_precond**);
fb_status fb_batch_solve_impl(fb_batch_job*, int, const fb_batch_opts*);
fb_status fb_krylov_basis_impl(fb_op*, const fb_precond*, const cd*, int, cd*, cudaStream_t);
fb_status fb_ibem_gammas_impl(fb_op*, const double*, cd*, cd*, cudaStream_t);
fb_status fb_ibem_rhs_impl(fb_op*, const cd*, const cd*, cd*, cudaStream_t);
fb_status fb_ibem_field_impl(fb_op*, const cd*, const cd*, const cd*, const double*, int64_t, cd*, cudaStream_t);
fb_status fb_dbem5_rhs_impl(fb_op*, const cd*, cd*, cudaStream_t);
fb_status fb_image_field_impl(const double*, const double*, const cd*, double, const double*, int, const double*,
                              int64_t, cd*, cudaStream_t);
fb_status fb_pulse_synthesis_impl(const cd*, const double*, int, int64_t, double, double, int, double, double*,
                                  cudaStream_t);
fb_status fb_dbem5_psi_impl(fb_op*, const cd*, const cd*, cd*, cudaStream_t);
void fb_precond_free(fb_precond*);
fb_status fb_alu_peaks_impl(double*, double*, cudaStream_t);

static std::atomic<long long> g_launches{0};
void fb_count_launch(long long n) { g_launches += n; }

static thread_local fb_status g_last_code = FB_OK;
static thread_local char g_last_msg[1024] = "";

fb_status fb_smem_cap(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<const void*, size_t> cap;
    std::lock_guard<std::mutex> lk(mu);
    size_t& c = cap[func];
    if (bytes <= c) return FB_OK;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("shared-memory opt-in: ") + cudaGetErrorString(e));
    c = bytes;
    return FB_OK;
}

void fb_set_error(fb_status code, const std::string& msg) {
    g_last_code = code;
    snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg.c_str());
}
fb_status fb_fail(fb_status code, const std::string& msg) {
    fb_set_error(code, msg);
    return code;
}

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

fb_status fb_op_wait_status(const fb_op* op) {
    if (!op) return FB_OK;
    if (fb_is_composite(op)) {
        for (int q = 0; q < 4 && op->sub[q]; ++q) FB_CHECK(fb_op_wait_status(op->sub[q]));
        return FB_OK;
    }
    if (op->prec != FB_PREC_MIXED_FMM) return FB_OK;
    return fb_tc_check(op);
}


// Temporary device copy of a caller array for host memspace.
struct Staged {
    void* d = nullptr;
    ~Staged() { if (d) cudaFree(d); }
};
static fb_status stage_in(const void* src, size_t bytes, int memspace, Staged& st, const void** dev,
                          cudaStream_t s) {
    if (memspace == FB_MEM_DEVICE) {
        *dev = src;
        return FB_OK;
    }
    if (memspace != FB_MEM_HOST) return fb_fail(FB_ERR_ARG, "memspace must be FB_MEM_HOST or FB_MEM_DEVICE");
    FB_CUDA(cudaMalloc(&st.d, bytes ? bytes : 1));
    FB_CUDA(cudaMemcpyAsync(st.d, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = st.d;
    return FB_OK;
}
static fb_status stage_out_alloc(size_t bytes, int memspace, void* user, Staged& st, void** dev) {
    if (memspace == FB_MEM_DEVICE) {
        *dev = user;
        return FB_OK;
    }
    if (memspace != FB_MEM_HOST) return fb_fail(FB_ERR_ARG, "memspace must be FB_MEM_HOST or FB_MEM_DEVICE");
    FB_CUDA(cudaMalloc(&st.d, bytes ? bytes : 1));
    *dev = st.d;
    return FB_OK;
}
static fb_status stage_out_finish(size_t bytes, int memspace, void* user, const Staged& st, cudaStream_t s) {
    if (memspace == FB_MEM_HOST) {
        FB_CUDA(cudaMemcpyAsync(user, st.d, bytes, cudaMemcpyDeviceToHost, s));
        FB_CUDA(cudaStreamSynchronize(s));
    }
    return FB_OK;
}

long long fb_launch_count() { return g_launches.load(); }

fb_status fb_apply_any(fb_op* op, const cd* x, cd* y, cudaStream_t s, int nrhs) {
    if (op->kind == FB_OP_IBEM) return fb_ibem_apply(op, x, y, s, nrhs);
    if (op->kind == FB_OP_DBEM5) return fb_dbem5_apply(op, x, y, s, nrhs);
    if (op->prec == FB_PREC_FP64_DENSE) {
        for (int r = 0; r < nrhs; ++r) FB_CHECK(fb_dense_apply(op, x + r * op->n, y + r * op->n, s));
        return FB_OK;
    }
    if (op->use_graphs) {
        const int64_t e = op->n * nrhs;
        return fb_graph_run(
            op->graphs, nrhs, e, e, x, y, s,
            [op, nrhs](const cd* gx, cd* gy, cudaStream_t st) { return fb_fmm_apply(op, gx, gy, st, nullptr, nrhs); },
            &op->buf_gen);
    }
    return fb_fmm_apply(op, x, y, s, nullptr, nrhs);
}

extern "C" {

const char* fb_version(void) { return "fmmbem 0.1 (sm_103a)"; }

fb_status fb_last_error(char* buf, size_t len) {
    if (buf && len) snprintf(buf, len, "%s", g_last_msg);
    return g_last_code;
}

fb_status fb_mesh_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, void* stream,
                         fb_mesh** out) {
    return fb_mesh_create_impl(verts, nv, tris, nt, as_stream(stream), out);
}

fb_status fb_mesh_set_admittance(fb_mesh* m, const double* beta, int memspace, void* stream) {
    if (!m || !beta) return fb_fail(FB_ERR_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * m->n;
    if (memspace == FB_MEM_DEVICE) {
        FB_CUDA(cudaMemcpyAsync(m->beta, beta, bytes, cudaMemcpyDeviceToDevice, s));
    } else if (memspace == FB_MEM_HOST) {
        FB_CUDA(cudaMemcpyAsync(m->beta, beta, bytes, cudaMemcpyHostToDevice, s));
        FB_CUDA(cudaStreamSynchronize(s));
    } else {
        return fb_fail(FB_ERR_ARG, "bad memspace");
    }
    return FB_OK;
}

fb_status fb_mesh_info(const fb_mesh* m, int64_t* nt, double* rc, double* max_edge) {
    if (!m) return fb_fail(FB_ERR_ARG, "NULL mesh");
    if (nt) *nt = m->n;
    if (rc) *rc = m->rc;
    if (max_edge) *max_edge = m->max_edge;
    return FB_OK;
}

fb_status fb_mesh_geometry(const fb_mesh* m, double* centroids, double* normals) {
    if (!m) return fb_fail(FB_ERR_ARG, "NULL mesh");
    int64_t n = m->n;
    std::string tmp;
    for (int which = 0; which < 2; ++which) {
        double* out = which == 0 ? centroids : normals;
        if (!out) continue;
        const double* src = m->buf + (which == 0 ? 0 : 3 * n);
        std::vector<double> h(3 * n);
        FB_CUDA(cudaMemcpy(h.data(), src, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) out[3 * i + d] = h[d * n + i];
    }
    return FB_OK;
}

void fb_mesh_destroy(fb_mesh* m) { fb_mesh_free(m); }

fb_status fb_tree_build(const fb_mesh* mesh, int leaf_max, void* stream, fb_tree** out) {
    return fb_tree_build_impl(mesh, leaf_max, as_stream(stream), out);
}

fb_status fb_tree_info(const fb_tree* t, int* leaf_level, double* origin, double* side, int64_t* nboxes) {
    if (!t) return fb_fail(FB_ERR_ARG, "NULL tree");
    if (leaf_level) *leaf_level = t->L;
    if (origin) for (int d = 0; d < 3; ++d) origin[d] = t->origin[d];
    if (side) *side = t->side;
    if (nboxes) for (int l = 0; l <= t->L; ++l) nboxes[l] = t->nbox[l];
    return FB_OK;
}

fb_status fb_tree_export(const fb_tree* t, int which, int level, int64_t* out, int64_t* count) {
    return fb_tree_export_impl(t, which, level, out, count);
}

void fb_tree_destroy(fb_tree* t) { fb_tree_free(t); }

}  // extern "C"

fb_status fb_operator_create_impl(const fb_mesh* mesh, const fb_tree* tree, double k, int kind, int precision,
                                  double d0, int pmin, cudaStream_t s, fb_op** out, const fb_op* donor) {
    if (!mesh || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (!(k > 0.0)) return fb_fail(FB_ERR_ARG, "k must be > 0");
    if (kind < FB_OP_L || kind > FB_OP_DBEM5) return fb_fail(FB_ERR_ARG, "unknown operator kind");
    if (precision < FB_PREC_FP64_DENSE || precision > FB_PREC_MIXED_FMM)
        return fb_fail(FB_ERR_ARG, "unknown precision");
    if (precision != FB_PREC_FP64_DENSE) {
        if (!tree) return fb_fail(FB_ERR_ARG, "FMM precision needs a tree");
        if (tree->mesh != mesh) return fb_fail(FB_ERR_ARG, "tree was built from another mesh");
        if (!(d0 > 0.0) || pmin < 1) return fb_fail(FB_ERR_ARG, "need d0 > 0 and pmin >= 1");
    }
    fb_op* op = new fb_op();
    op->mesh = mesh;
    op->tree = tree;
    op->dev = mesh->dev;
    op->kind = kind;
    op->prec = precision;
    op->k = k;
    op->d0 = d0;
    op->pmin = pmin;
    op->n = mesh->n;
    op->near_donor = donor;
    fb_status st = kind == FB_OP_IBEM                  ? fb_ibem_create(op, s)
                   : kind == FB_OP_DBEM5             ? fb_dbem5_create(op, s)
                   : precision == FB_PREC_FP64_DENSE ? fb_dense_create(op, s)
                                                     : fb_fmm_create(op, d0, pmin, s);
    if (st == FB_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fb_fail(FB_ERR_CUDA, std::string("operator setup: ") + cudaGetErrorString(e));
    }
    op->near_donor = nullptr;
    if (st != FB_OK) {
        fb_operator_destroy(op);
        return st;
    }
    *out = op;
    return FB_OK;
}

extern "C" {

fb_status fb_operator_create(const fb_mesh* mesh, const fb_tree* tree, double k, int kind, int precision,
                             double d0, int pmin, void* stream, fb_op** out) {
    return fb_operator_create_impl(mesh, tree, k, kind, precision, d0, pmin, as_stream(stream), out);
}

fb_status fb_operator_create_like(const fb_op* donor, int precision, double d0, int pmin, void* stream,
                                  fb_op** out) {
    if (!donor || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (fb_is_composite(donor) || donor->prec == FB_PREC_FP64_DENSE)
        return fb_fail(FB_ERR_ARG, "the donor must be an FMM operator");
    if (precision != FB_PREC_FP64_FMM && precision != FB_PREC_MIXED_FMM)
        return fb_fail(FB_ERR_ARG, "FMM precisions only");
    return fb_operator_create_impl(donor->mesh, donor->tree, donor->k, donor->kind, precision, d0, pmin,
                                   as_stream(stream), out, donor);
}

fb_status fb_mesh_set_admittance_plus(fb_mesh* m, const double* beta, int memspace, void* stream) {
    if (!m || !beta) return fb_fail(FB_ERR_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    if (!m->beta_p) FB_CHECK(dalloc(&m->beta_p, (size_t)m->n));
    size_t bytes = sizeof(cd) * m->n;
    if (memspace == FB_MEM_DEVICE) {
        FB_CUDA(cudaMemcpyAsync(m->beta_p, beta, bytes, cudaMemcpyDeviceToDevice, s));
    } else if (memspace == FB_MEM_HOST) {
        FB_CUDA(cudaMemcpyAsync(m->beta_p, beta, bytes, cudaMemcpyHostToDevice, s));
        FB_CUDA(cudaStreamSynchronize(s));
    } else {
        return fb_fail(FB_ERR_ARG, "bad memspace");
    }
    return FB_OK;
}

fb_status fb_ibem_gammas_monopole(fb_op* op, const double* src, double* gamma_p, double* gamma_m, void* stream) {
    if (!op || !src || !gamma_p || !gamma_m) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (op->kind != FB_OP_IBEM) return fb_fail(FB_ERR_ARG, "not an indirect-system operator");
    return fb_ibem_gammas_impl(op, src, (cd*)gamma_p, (cd*)gamma_m, as_stream(stream));
}

fb_status fb_ibem_rhs(fb_op* op, const double* gamma_p, const double* gamma_m, double* b, void* stream) {
    if (!op || !gamma_p || !gamma_m || !b) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (op->kind != FB_OP_IBEM) return fb_fail(FB_ERR_ARG, "not an indirect-system operator");
    return fb_ibem_rhs_impl(op, (const cd*)gamma_p, (const cd*)gamma_m, (cd*)b, as_stream(stream));
}

fb_status fb_ibem_field(fb_op* op, const double* x, const double* gamma_p, const double* gamma_m, const double* rcv,
                        int64_t nr, double* out, void* stream) {
    if (!op || !x || !gamma_p || !gamma_m || !rcv || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (op->kind != FB_OP_IBEM) return fb_fail(FB_ERR_ARG, "not an indirect-system operator");
    if (nr < 0) return fb_fail(FB_ERR_ARG, "nr < 0");
    return fb_ibem_field_impl(op, (const cd*)x, (const cd*)gamma_p, (const cd*)gamma_m, rcv, nr, (cd*)out,
                              as_stream(stream));
}

fb_status fb_image_field(const double* room, const double* src, const double* R_walls, double a_th,
                         const double* k, int nf, const double* rcv, int64_t nr, double* out, void* stream) {
    if (!room || !src || !R_walls || !k || !rcv || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (nf < 1 || nr < 0 || !(a_th > 0.0)) return fb_fail(FB_ERR_ARG, "need nf >= 1, nr >= 0, a_th > 0");
    for (int d = 0; d < 3; ++d)
        if (!(room[d] > 0.0) || !(src[d] > 0.0 && src[d] < room[d]))
            return fb_fail(FB_ERR_ARG, "room sides must be > 0 and the source inside the room");
    return fb_image_field_impl(room, src, (const cd*)R_walls, a_th, k, nf, rcv, nr, (cd*)out, as_stream(stream));
}

fb_status fb_pulse_synthesis(const double* psi, const double* freqs, int nf, int64_t nr, double df, double dt, int nt,
                             double pulse_dt, double* out, void* stream) {
    if (!psi || !freqs || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (nf < 1 || nr < 0 || nt < 1 || !(df > 0.0) || !(dt > 0.0)) return fb_fail(FB_ERR_ARG, "bad sizes or steps");
    return fb_pulse_synthesis_impl((const cd*)psi, freqs, nf, nr, df, dt, nt, pulse_dt, out, as_stream(stream));
}

fb_status fb_dbem5_rhs(fb_op* op, const double* gamma, double* b, void* stream) {
    if (!op || !gamma || !b) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (op->kind != FB_OP_DBEM5) return fb_fail(FB_ERR_ARG, "not an FB_OP_DBEM5 operator");
    return fb_dbem5_rhs_impl(op, (const cd*)gamma, (cd*)b, as_stream(stream));
}

fb_status fb_dbem5_psi(fb_op* op, const double* q, const double* gamma, double* psi, void* stream) {
    if (!op || !q || !gamma || !psi) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (op->kind != FB_OP_DBEM5) return fb_fail(FB_ERR_ARG, "not an FB_OP_DBEM5 operator");
    return fb_dbem5_psi_impl(op, (const cd*)q, (const cd*)gamma, (cd*)psi, as_stream(stream));
}

fb_status fb_operator_apply(fb_op* op, const double* x, double* y, int memspace, void* stream) {
    if (!op || !x || !y) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (x == y) return fb_fail(FB_ERR_ARG, "x and y must not overlap");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * op->n;
    Staged sx, sy;
    const void* dx = nullptr;
    void* dy = nullptr;
    FB_CHECK(stage_in(x, bytes, memspace, sx, &dx, s));
    FB_CHECK(stage_out_alloc(bytes, memspace, y, sy, &dy));
    FB_CHECK(fb_apply_any(op, (const cd*)dx, (cd*)dy, s));
    return stage_out_finish(bytes, memspace, y, sy, s);
}

long long fb_kernel_launches(void) { return g_launches.load(); }

fb_status fb_operator_apply_multi(fb_op* op, const double* x, double* y, int nrhs, int memspace, void* stream) {
    if (!op || !x || !y) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (nrhs < 1 || nrhs > FB_MAX_RHS) return fb_fail(FB_ERR_ARG, "nrhs must be in [1, FB_MAX_RHS]");
    if (x == y) return fb_fail(FB_ERR_ARG, "x and y must not overlap");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * op->n * nrhs;
    Staged sx, sy;
    const void* dx = nullptr;
    void* dy = nullptr;
    FB_CHECK(stage_in(x, bytes, memspace, sx, &dx, s));
    FB_CHECK(stage_out_alloc(bytes, memspace, y, sy, &dy));
    FB_CHECK(fb_apply_any(op, (const cd*)dx, (cd*)dy, s, nrhs));
    return stage_out_finish(bytes, memspace, y, sy, s);
}

fb_status fb_precond_apply(const fb_precond* pc, const double* x, double* y, int memspace, void* stream) {
    if (!pc || !x || !y) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (x == y) return fb_fail(FB_ERR_ARG, "x and y must not overlap");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * pc->n;
    Staged sx, sy;
    const void* dx = nullptr;
    void* dy = nullptr;
    FB_CHECK(stage_in(x, bytes, memspace, sx, &dx, s));
    FB_CHECK(stage_out_alloc(bytes, memspace, y, sy, &dy));
    FB_CHECK(fb_pc_apply(pc, (const cd*)dx, (cd*)dy, s));
    FB_LAUNCH_CHECK();
    return stage_out_finish(bytes, memspace, y, sy, s);
}

fb_status fb_measure_alu_peaks(double* fp32_tflops, double* fp64_tflops, void* stream) {
    return fb_alu_peaks_impl(fp32_tflops, fp64_tflops, as_stream(stream));
}

fb_status fb_operator_apply_timed(fb_op* op, const double* x, double* y, void* stream, double* phase_ms) {
    if (!op || !x || !y || !phase_ms) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (fb_is_composite(op)) return fb_fail(FB_ERR_ARG, "phase timing is per FMM operator");
    cudaStream_t s = as_stream(stream);
    for (int i = 0; i < FB_NPHASE; ++i) phase_ms[i] = 0.0;
    if (op->prec == FB_PREC_FP64_DENSE) {
        cudaEvent_t a, b;
        FB_CUDA(cudaEventCreate(&a));
        FB_CUDA(cudaEventCreate(&b));
        cudaEventRecord(a, s);
        fb_status st = fb_dense_apply(op, (const cd*)x, (cd*)y, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        phase_ms[FB_NPHASE - 1] = ms;
        return st;
    }
    PhaseTimer pt;
    for (int i = 0; i <= FB_NPHASE; ++i) FB_CUDA(cudaEventCreate(&pt.ev[i]));
    fb_status st = fb_fmm_apply(op, (const cd*)x, (cd*)y, s, &pt);
    if (st == FB_OK) {
        // marks 0..6 bracket the six phases; phase_ms[6] is the total
        FB_CUDA(cudaEventSynchronize(pt.ev[FB_NPHASE - 1]));
        for (int i = 0; i < FB_NPHASE - 1; ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, pt.ev[i], pt.ev[i + 1]);
            phase_ms[i] = ms;
        }
        float tot = 0;
        cudaEventElapsedTime(&tot, pt.ev[0], pt.ev[FB_NPHASE - 1]);
        phase_ms[FB_NPHASE - 1] = tot;
    }
    for (int i = 0; i <= FB_NPHASE; ++i) cudaEventDestroy(pt.ev[i]);
    return st;
}

fb_status fb_operator_apply_noalloc(fb_op* op, const double* x, double* y, void* stream) {
    if (!op || !x || !y) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (x == y) return fb_fail(FB_ERR_ARG, "x and y must not overlap");
    if (fb_is_composite(op)) return fb_fail(FB_ERR_ARG, "composite systems keep their own work space");
    return fb_fmm_apply_noalloc(op, (const cd*)x, (cd*)y, as_stream(stream));
}

fb_status fb_operator_set_translation(fb_op* op, int method) {
    if (!op) return fb_fail(FB_ERR_ARG, "NULL operator");
    if (fb_is_composite(op)) {
        for (int q = 0; q < 4 && op->sub[q]; ++q) FB_CHECK(fb_operator_set_translation(op->sub[q], method));
        return FB_OK;
    }
    if (op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "dense operators have no translations");
    if (method < FB_TRANS_AUTO || method > FB_TRANS_TENSOR) return fb_fail(FB_ERR_ARG, "unknown translation method");
    if (method == FB_TRANS_TENSOR && op->prec != FB_PREC_MIXED_FMM)
        return fb_fail(FB_ERR_ARG, "tensor-core translations need the mixed precision");
    if (method == FB_TRANS_COMPOSED || method == FB_TRANS_TENSOR) {
        for (int l = 2; l <= op->L; ++l)
            if (!fb_composable(op, l, l >= 3))
                return fb_fail(FB_ERR_ARG, "composed and tensor-core translations need every level's order <= " +
                                               std::to_string(FB_COMPOSE_PMAX));
        FB_CHECK(fb_compose_all(op, nullptr));
    }
    if (method == FB_TRANS_TENSOR) {
        if (!op->tc_plan_all) {
            std::vector<int> all;
            for (int l = 2; l <= op->L; ++l) all.push_back(l);
            fb_status st = fb_tc_build(op, all, &op->tc_plan_all, nullptr);
            if (st != FB_OK) {
                fb_tc_free(op->tc_plan_all);
                return st;
            }
            FB_CUDA(cudaStreamSynchronize(nullptr));
        }
    }
    if (op->method != method) op->buf_gen++;   // captured graphs hold the previous method
    op->method = method;
    fb_graph_free(op->graphs);
    return FB_OK;
}

fb_status fb_operator_use_graphs(fb_op* op, int enable) {
    if (!op) return fb_fail(FB_ERR_ARG, "NULL operator");
    if (fb_is_composite(op)) {
        for (int q = 0; q < 4 && op->sub[q]; ++q) FB_CHECK(fb_operator_use_graphs(op->sub[q], enable));
        return FB_OK;
    }
    op->use_graphs = enable ? 1 : 0;
    if (!enable) fb_graph_free(op->graphs);
    return FB_OK;
}

fb_status fb_precond_use_graphs(fb_precond* pc, int enable) {
    if (!pc) return fb_fail(FB_ERR_ARG, "NULL preconditioner");
    pc->use_graphs = enable ? 1 : 0;
    if (!enable) fb_graph_free(pc->graphs);
    return FB_OK;
}

fb_status fb_operator_autotune(fb_op* op, int nrhs, void* stream, double* times, int* choice) {
    if (!op) return fb_fail(FB_ERR_ARG, "NULL operator");
    if (op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "dense operators have no translations");
    if (nrhs < 1 || nrhs > FB_MAX_RHS) return fb_fail(FB_ERR_ARG, "nrhs must be in [1, FB_MAX_RHS]");
    if (times)
        for (int i = 0; i < FB_TUNE_TIMES * (FB_MAXLEV + 1); ++i) times[i] = -1.0;
    if (choice)
        for (int i = 0; i <= FB_MAXLEV; ++i) choice[i] = 0;
    if (fb_is_composite(op)) {   // each constituent operator; times/choice of the first
        for (int q = 0; q < 4 && op->sub[q]; ++q)
            FB_CHECK(fb_operator_autotune(op->sub[q], nrhs, stream, q == 0 ? times : nullptr, q == 0 ? choice : nullptr));
        return FB_OK;
    }
    fb_graph_free(op->graphs);
    return fb_autotune_impl(op, nrhs, as_stream(stream), times, choice);
}

fb_status fb_operator_set_forms(fb_op* op, const int* choice, void* stream) {
    if (!op || !choice) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (fb_is_composite(op)) {
        for (int q = 0; q < 4 && op->sub[q]; ++q) FB_CHECK(fb_operator_set_forms(op->sub[q], choice, stream));
        return FB_OK;
    }
    fb_graph_free(op->graphs);
    fb_status st = fb_set_forms_impl(op, choice, as_stream(stream));
    if (st == FB_OK) {
        op->method = FB_TRANS_AUTO;
        op->buf_gen++;
    }
    return st;
}

fb_status fb_operator_info(const fb_op* op, int64_t* n, int* leaf_level, int* p) {
    if (!op) return fb_fail(FB_ERR_ARG, "NULL operator");
    if (fb_is_composite(op)) {
        FB_CHECK(fb_operator_info(op->sub[0], nullptr, leaf_level, p));
        if (n) *n = op->n;
        return FB_OK;
    }
    if (n) *n = op->n;
    if (leaf_level) *leaf_level = op->L;
    if (p) for (int l = 0; l <= op->L; ++l) p[l] = op->p[l];
    return FB_OK;
}

fb_status fb_operator_status(fb_op* op, void* stream) {
    if (!op) return fb_fail(FB_ERR_ARG, "NULL operator");
    FB_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return fb_op_wait_status(op);
}

fb_status fb_operator_set_near_bf16(fb_op* op, int enable, void* stream) {
    if (!op) return fb_fail(FB_ERR_ARG, "NULL operator");
    if (fb_is_composite(op)) return fb_fail(FB_ERR_ARG, "set the constituent operators instead");
    return fb_near_bf16(op, enable, as_stream(stream));
}

fb_status fb_operator_staged_pass_times(fb_op* op, void* stream, double* ms, int* tc) {
    if (!op || !ms || !tc) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (fb_is_composite(op) || op->prec == FB_PREC_FP64_DENSE)
        return fb_fail(FB_ERR_ARG, "staged pass times need an FMM operator");
    return fb_stg_op_pass_times(op, as_stream(stream), ms, tc);
}

fb_status fb_set_device_wait_limit(long long limit, long long* previous) {
    if (limit < 1) return fb_fail(FB_ERR_ARG, "wait limit must be >= 1");
    long long old = fb_tc_set_wait_limit(limit);
    if (previous) *previous = old;
    return FB_OK;
}

fb_status fb_test_stall_device_waits(int enable) {
    fb_tc_set_inject_stall(enable);
    return FB_OK;
}

fb_status fb_operator_export(const fb_op* op, int which, int level, int64_t index, double* out, int64_t* count) {
    if (!op || !count) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (fb_is_composite(op)) return fb_fail(FB_ERR_ARG, "export the constituent operators instead");
    const cd* src = nullptr;
    int64_t cnt = 0;
    if (which == 7) {
        if (op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "not an FMM operator");
        *count = op->L + 1;
        if (out)
            for (int l = 0; l <= op->L; ++l) {
                bool tc = op->prec == FB_PREC_MIXED_FMM &&
                          (op->method == FB_TRANS_TENSOR ? l >= 2 : (op->method == FB_TRANS_AUTO && op->tc_level[l]));
                out[2 * l] = tc ? 1.0 : 0.0;
                out[2 * l + 1] = 0.0;
            }
        return FB_OK;
    }
    if (which == 8) {
        // real rotation factors d^n (n = level) of the direction of M2L offset code `index`
        if (op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "not an FMM operator");
        if (index < 0 || index >= FB_NOFF || (size_t)index >= op->dir_of_code.size() || op->dir_of_code[index] < 0)
            return fb_fail(FB_ERR_ARG, "offset code is not an M2L translation direction");
        if (level < 0 || level >= op->Prot) return fb_fail(FB_ERR_ARG, "degree out of range");
        const int n = level, w = 2 * n + 1;
        *count = (int64_t)w * w;
        if (out) {
            const int64_t off = (int64_t)op->dir_of_code[index] * op->per_dir + (int64_t)n * (2 * n - 1) * (2 * n + 1) / 3;
            std::vector<double> h((size_t)w * w);
            if (op->prec == FB_PREC_MIXED_FMM) {
                std::vector<float> f((size_t)w * w);
                FB_CUDA(cudaMemcpy(f.data(), op->rotd32 + off, sizeof(float) * f.size(), cudaMemcpyDeviceToHost));
                for (size_t i = 0; i < f.size(); ++i) h[i] = f[i];
            } else {
                FB_CUDA(cudaMemcpy(h.data(), op->rotd64 + off, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
            }
            for (size_t i = 0; i < h.size(); ++i) {
                out[2 * i] = h[i];
                out[2 * i + 1] = 0.0;
            }
        }
        return FB_OK;
    }
    if (which == 6) {
        if (!op->dense) return fb_fail(FB_ERR_ARG, "not a dense operator");
        if (index < 0 || index >= op->n) return fb_fail(FB_ERR_ARG, "row out of range");
        src = op->dense + index * op->n;
        cnt = op->n;
    } else {
        if (op->prec == FB_PREC_FP64_DENSE) return fb_fail(FB_ERR_ARG, "not an FMM operator");
        const fb_tree* t = op->tree;
        int L = op->L;
        int nleaf = t->nbox[L];
        int PL = op->p[L] * op->p[L];
        if (which >= 0 && which <= 2) {
            if (index < 0 || index >= nleaf) return fb_fail(FB_ERR_ARG, "leaf out of range");
            if (!op->nf64)
                return fb_fail(FB_ERR_ARG, "mixed operators keep FP32 entries only: export from an FP64 operator");
            int r0 = t->h_leaf_start[index], nr = t->h_leaf_start[index + 1] - r0;
            if (which == 0) {
                src = op->nf64 + op->h_nf_off[index];
                cnt = (int64_t)nr * op->h_nf_ncol[index];
            } else {
                src = (which == 1 ? op->w64 : op->v64) + (int64_t)r0 * PL;
                cnt = (int64_t)nr * PL;
            }
        } else if (which == 3) {
            if (level < 2 || level > L || index < 0 || index >= FB_NOFF) return fb_fail(FB_ERR_ARG, "bad level/offset");
            if (!fb_composable(op, level, false)) return fb_fail(FB_ERR_ARG, "no composed matrix above order 32");
            FB_CHECK(fb_compose_all(const_cast<fb_op*>(op), nullptr));
            int64_t off = op->m2l_toff[(size_t)level * FB_NOFF + index];
            if (off < 0) return fb_fail(FB_ERR_ARG, "offset not used at this level");
            src = op->T64 + off;
            cnt = (int64_t)op->p[level] * op->p[level] * op->p[level] * op->p[level];
        } else if (which == 4 || which == 5) {
            if (level < 3 || level > L || index < 0 || index > 7) return fb_fail(FB_ERR_ARG, "bad level/octant");
            if (!fb_composable(op, level, true)) return fb_fail(FB_ERR_ARG, "no composed matrix above order 32");
            FB_CHECK(fb_compose_all(const_cast<fb_op*>(op), nullptr));
            int64_t off = which == 4 ? op->m2m_toff[level][index] : op->l2l_toff[level][index];
            if (off < 0) return fb_fail(FB_ERR_ARG, "octant not used at this level");
            src = op->T64 + off;
            cnt = (int64_t)op->p[level] * op->p[level] * op->p[level - 1] * op->p[level - 1];
        } else {
            return fb_fail(FB_ERR_ARG, "unknown export");
        }
    }
    *count = cnt;
    if (out) FB_CUDA(cudaMemcpy(out, src, sizeof(cd) * cnt, cudaMemcpyDeviceToHost));
    return FB_OK;
}

void fb_operator_destroy(fb_op* op) {
    if (!op) return;
    fb_krylov_free(op);
    fb_ibem_free(op);
    dfree(op->dense);
    fb_fmm_destroy(op);
    dfree(op->io_x);
    dfree(op->io_y);
    fb_graph_free(op->graphs);
    delete op;
}

fb_status fb_gamma_monopole(const fb_mesh* m, double k, const double* src, double* gamma, int memspace,
                            void* stream) {
    if (!m || !src || !gamma) return fb_fail(FB_ERR_ARG, "NULL argument");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * m->n;
    Staged so;
    void* dg = nullptr;
    FB_CHECK(stage_out_alloc(bytes, memspace, gamma, so, &dg));
    FB_CHECK(fb_gamma_impl(m, k, src, (cd*)dg, s));
    return stage_out_finish(bytes, memspace, gamma, so, s);
}

fb_status fb_precond_create(fb_op* op, int kind, void* stream, fb_precond** out) {
    if (!op || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    return fb_precond_create_impl(op, kind, as_stream(stream), out);
}

void fb_precond_destroy(fb_precond* pc) { fb_precond_free(pc); }

fb_status fb_krylov_basis(fb_op* A, const fb_precond* pc, const double* b, int k, double* V, void* stream) {
    if (!A || !b || !V) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (k < 1 || k > 200) return fb_fail(FB_ERR_ARG, "k must be in [1, 200]");
    if (pc && pc->op != A) return fb_fail(FB_ERR_ARG, "preconditioner built for another operator");
    return fb_krylov_basis_impl(A, pc, (const cd*)b, k, (cd*)V, as_stream(stream));
}

fb_status fb_precond_create_inner(fb_op* op, fb_op* inner_op, const fb_precond* inner_pc, int iters, void* stream,
                                  fb_precond** out) {
    if (!op || !inner_op || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (inner_op->n != op->n) return fb_fail(FB_ERR_ARG, "inner operator size differs");
    if (iters < 1 || iters > 200) return fb_fail(FB_ERR_ARG, "iters must be in [1, 200]");
    if (inner_pc && inner_pc->op != inner_op)
        return fb_fail(FB_ERR_ARG, "the inner preconditioner must belong to the inner operator");
    fb_precond* pc = new fb_precond();
    pc->op = op;
    pc->kind = FB_PC_INNER;
    pc->n = op->n;
    pc->inner_op = inner_op;
    pc->inner_its = iters;
    pc->base = inner_pc;
    fb_status st = fb_inner_create(pc, as_stream(stream));
    if (st != FB_OK) {
        fb_precond_free(pc);
        return st;
    }
    *out = pc;
    return FB_OK;
}

fb_status fb_precond_create_learned(fb_op* op, const fb_precond* base, uint64_t seed, void* stream,
                                    fb_precond** out) {
    if (!op || !base || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (fb_is_composite(op)) return fb_fail(FB_ERR_ARG, "the learned network serves single FMM operators");
    if ((base->kind != FB_PC_BLOCK_JACOBI && base->kind != FB_PC_INNER) || base->op != op)
        return fb_fail(FB_ERR_ARG, "the base must be a block-Jacobi or inner-outer preconditioner of the same "
                                   "operator");
    cudaStream_t s = as_stream(stream);
    fb_precond* pc = new fb_precond();
    pc->op = op;
    pc->kind = FB_PC_LEARNED;
    pc->n = op->n;
    pc->base = base;
    fb_status st = fb_learned_alloc(pc->net, op, base, s);
    if (st == FB_OK) st = fb_learned_init(pc->net, seed, s);
    if (st != FB_OK) {
        fb_precond_destroy(pc);
        return st;
    }
    *out = pc;
    return FB_OK;
}

static fb_status learned_of(fb_precond* pc) {
    if (!pc || !pc->net) return fb_fail(FB_ERR_ARG, "not a learned preconditioner");
    return FB_OK;
}

fb_status fb_learned_params(fb_precond* pc, float* host_out, const float* host_in, int64_t* count) {
    FB_CHECK(learned_of(pc));
    if (!count) return fb_fail(FB_ERR_ARG, "NULL count");
    int64_t np = fb_learned_nparam(pc->net);
    if (host_in) {
        if (*count != np) return fb_fail(FB_ERR_ARG, "parameter count mismatch");
        FB_CUDA(cudaMemcpy(fb_learned_weights(pc->net), host_in, sizeof(float) * np, cudaMemcpyHostToDevice));
        FB_CHECK(fb_learned_params_changed(pc->net, nullptr));
        FB_CUDA(cudaDeviceSynchronize());
    }
    *count = np;
    if (host_out) FB_CUDA(cudaMemcpy(host_out, fb_learned_weights(pc->net), sizeof(float) * np, cudaMemcpyDeviceToHost));
    return FB_OK;
}

fb_status fb_learned_set_objective(fb_precond* pc, int objective) {
    FB_CHECK(learned_of(pc));
    return fb_learned_set_objective(pc->net, objective);
}

fb_status fb_learned_loss_and_grad(fb_precond* pc, const double* R, const double* E, int npairs, double* loss,
                                   float* grad_host, void* stream) {
    FB_CHECK(learned_of(pc));
    if (!R || !E || npairs < 1) return fb_fail(FB_ERR_ARG, "need pairs");
    cudaStream_t s = as_stream(stream);
    FB_CHECK(fb_learned_loss_grad(pc->net, (const cd*)R, (const cd*)E, npairs, loss, s));
    if (grad_host) {
        FB_CUDA(cudaMemcpyAsync(grad_host, fb_learned_grads(pc->net), sizeof(float) * fb_learned_nparam(pc->net),
                                cudaMemcpyDeviceToHost, s));
        FB_CUDA(cudaStreamSynchronize(s));
    }
    return FB_OK;
}

fb_status fb_learned_train_step(fb_precond* pc, const double* R, const double* E, int npairs, double lr,
                                double* loss, void* stream) {
    FB_CHECK(learned_of(pc));
    if (!R || !E || npairs < 1 || !(lr > 0)) return fb_fail(FB_ERR_ARG, "need pairs and lr > 0");
    cudaStream_t s = as_stream(stream);
    FB_CHECK(fb_learned_loss_grad(pc->net, (const cd*)R, (const cd*)E, npairs, loss, s));
    return fb_learned_adam_step(pc->net, lr, s);
}

fb_status fb_fgmres_solve(fb_op* A, fb_precond* pc, const double* b, double* x, const fb_solver_opts* opts,
                          fb_solve_info* info, int memspace, void* stream) {
    if (!A || !b || !x || !opts) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (pc && pc->op != A) return fb_fail(FB_ERR_ARG, "preconditioner built for another operator");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * A->n;
    Staged sb, sx;
    const void* db = nullptr;
    void* dx = nullptr;
    FB_CHECK(stage_in(b, bytes, memspace, sb, &db, s));
    FB_CHECK(stage_out_alloc(bytes, memspace, x, sx, &dx));
    fb_status st = fb_fgmres_impl(A, pc, (const cd*)db, (cd*)dx, opts, info, s);
    if (st != FB_OK && st != FB_ERR_NOCONV && st != FB_ERR_NAN) return st;
    fb_status st2 = stage_out_finish(bytes, memspace, x, sx, s);
    return st != FB_OK ? st : st2;
}

fb_status fb_fgmres_solve_multi(fb_op* A, fb_precond* pc, const double* b, double* x, int nrhs,
                                const fb_solver_opts* opts, fb_solve_info* info, int memspace, void* stream) {
    if (!A || !b || !x || !opts) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (nrhs < 1 || nrhs > FB_MAX_RHS) return fb_fail(FB_ERR_ARG, "nrhs must be in [1, FB_MAX_RHS]");
    if (pc && pc->op != A) return fb_fail(FB_ERR_ARG, "preconditioner built for another operator");
    cudaStream_t s = as_stream(stream);
    size_t bytes = sizeof(cd) * A->n * nrhs;
    Staged sb, sx;
    const void* db = nullptr;
    void* dx = nullptr;
    FB_CHECK(stage_in(b, bytes, memspace, sb, &db, s));
    FB_CHECK(stage_out_alloc(bytes, memspace, x, sx, &dx));
    fb_status st = fb_fgmres_multi_impl(A, pc, (const cd*)db, (cd*)dx, nrhs, opts, info, s);
    if (st != FB_OK && st != FB_ERR_NOCONV && st != FB_ERR_NAN) return st;
    fb_status st2 = stage_out_finish(bytes, memspace, x, sx, s);
    return st != FB_OK ? st : st2;
}

fb_status fb_batch_solve(fb_batch_job* jobs, int njobs, const fb_batch_opts* opts) {
    if ((!jobs && njobs > 0) || njobs < 0 || !opts) return fb_fail(FB_ERR_ARG, "bad batch arguments");
    return fb_batch_solve_impl(jobs, njobs, opts);
}

fb_status fb_eval_field(const fb_mesh* m, double k, const double* psi_sc, const double* gamma, const double* src,
                        const double* rcv, int64_t nr, double* out, int memspace, void* stream) {
    if (!m || !psi_sc || !gamma || !rcv || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    if (nr < 0) return fb_fail(FB_ERR_ARG, "nr < 0");
    cudaStream_t s = as_stream(stream);
    size_t nb = sizeof(cd) * m->n;
    Staged a, b, c, d;
    const void *dp = nullptr, *dg = nullptr, *dr = nullptr;
    void* dout = nullptr;
    FB_CHECK(stage_in(psi_sc, nb, memspace, a, &dp, s));
    FB_CHECK(stage_in(gamma, nb, memspace, b, &dg, s));
    FB_CHECK(stage_in(rcv, sizeof(double) * 3 * nr, memspace, c, &dr, s));
    FB_CHECK(stage_out_alloc(sizeof(cd) * nr, memspace, out, d, &dout));
    FB_CHECK(fb_eval_impl(m, k, (const cd*)dp, (const cd*)dg, src, (const double*)dr, nr, (cd*)dout, s));
    return stage_out_finish(sizeof(cd) * nr, memspace, out, d, s);
}

}  // extern "C"
