// Internal definitions shared by the CUDA translation units of the library:
// complex arithmetic, error handling, device-memory helpers and the handle
// structures behind the opaque types of include/fmmbem.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <deque>
#include <string>
#include <map>
#include <vector>

#include "../../include/fmmbem.h"
#include "df.cuh"

// ------------------------------------------------------------- complex ----
template <class R>
struct __align__(2 * sizeof(R)) cx {
    R re, im;
};
using cd = cx<double>;
using cf = cx<float>;

template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> conjg(cx<R> a) { return mk(a.re, -a.im); }
template <class R>
__host__ __device__ __forceinline__ R abs2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// a += b * c
template <class R>
__host__ __device__ __forceinline__ void cmac(cx<R>& a, cx<R> b, cx<R> c) {
    a.re += b.re * c.re - b.im * c.im;
    a.im += b.re * c.im + b.im * c.re;
}
// a += conj(b) * c
template <class R>
__host__ __device__ __forceinline__ void cmacc(cx<R>& a, cx<R> b, cx<R> c) {
    a.re += b.re * c.re + b.im * c.im;
    a.im += b.re * c.im - b.im * c.re;
}
// double-FP32 complex multiply-accumulate (a += b c), four df FMAs
__device__ __forceinline__ void cmac(cx<df>& a, cx<df> b, cx<df> c) {
    a.re = fma(b.re, c.re, a.re);
    a.re = fma(-b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im);
    a.im = fma(b.im, c.re, a.im);
}
// conversions between the storage precision of expansions (O) and the
// arithmetic of a translation kernel (R): equal types, or FP64 <-> double-FP32
template <class R>
__host__ __device__ __forceinline__ R real_from(double v) { return (R)v; }
template <>
__host__ __device__ __forceinline__ df real_from<df>(double v) { return df_from(v); }
template <class R, class O>
__device__ __forceinline__ cx<R> cx_to(const cx<O>& a) { return mk<R>(real_from<R>(a.re), real_from<R>(a.im)); }
template <>
__device__ __forceinline__ cx<float> cx_to<float, float>(const cx<float>& a) { return a; }
template <class O, class R>
__device__ __forceinline__ cx<O> cx_out(const cx<R>& a) { return a; }
template <>
__device__ __forceinline__ cx<double> cx_out<double, df>(const cx<df>& a) { return mk(df_to(a.re), df_to(a.im)); }
__host__ __device__ __forceinline__ cf to_f(cd a) { return mk<float>((float)a.re, (float)a.im); }
__host__ __device__ __forceinline__ cd to_d(cf a) { return mk<double>((double)a.re, (double)a.im); }
template <class R> __host__ __device__ __forceinline__ cx<R> from_d(cd a);
template <> __host__ __device__ __forceinline__ cd from_d<double>(cd a) { return a; }
template <> __host__ __device__ __forceinline__ cf from_d<float>(cd a) { return to_f(a); }

// --------------------------------------------------------- error state ----
void fb_set_error(fb_status code, const std::string& msg);
// Raises a kernel's dynamic shared-memory cap to at least `bytes`, never
// lowering it, so launches from several host threads cannot race on the
// attribute (thread-safe).  Call it before every launch with dynamic shared
// memory: the default cap is 48 KB minus the kernel's static shared memory.
fb_status fb_smem_cap(const void* func, size_t bytes);
// CUDA-graph replay helpers (graphs.cu): `cache` is an opaque per-object
// cache; body(x, y, s) is the work replayed (run uncaptured once, then
// captured on x/y staging vectors of in_elems / out_elems complex entries).
#include <functional>
fb_status fb_graph_run(void*& cache, int key, int64_t in_elems, int64_t out_elems, const cd* x, cd* y,
                       cudaStream_t s, const std::function<fb_status(const cd*, cd*, cudaStream_t)>& body,
                       const long long* gen = nullptr);
void fb_graph_free(void*& cache);
fb_status fb_fail(fb_status code, const std::string& msg);

#define FB_CUDA(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            return fb_fail(e_ == cudaErrorMemoryAllocation ? FB_ERR_OOM : FB_ERR_CUDA, \
                           std::string(#call " failed at " __FILE__ ":") +           \
                               std::to_string(__LINE__) + ": " + cudaGetErrorString(e_)); \
        }                                                                           \
    } while (0)

#define FB_CHECK(st)                   \
    do {                               \
        fb_status s_ = (st);           \
        if (s_ != FB_OK) return s_;    \
    } while (0)

#define FB_LAUNCH_CHECK() FB_CUDA(cudaGetLastError())

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// A device allocation released by its owner's destroy function.
template <class T>
fb_status dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return FB_OK;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fb_fail(FB_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                       " bytes failed: " + cudaGetErrorString(e));
    }
    return FB_OK;
}
template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// --------------------------------------------------------------- mesh ----
// Element geometry, structure of arrays in FP64 on the device.
struct Geom {
    int64_t n;
    const double *cx, *cy, *cz;     // centroids (collocation points)
    const double *nx, *ny, *nz;     // unit normals (outward)
    const double* area;
    const double *ax, *ay, *az;     // vertex 0
    const double *bx, *by, *bz;     // vertex 1
    const double *qx, *qy, *qz;     // vertex 2
    const double *gx, *gy, *gz;     // 3-point Gauss points: point q of element i at 3i+q
    const cd* beta;                 // admittance
};

struct fb_mesh {
    int dev = 0;
    int64_t n = 0;
    double* buf = nullptr;          // 16 n doubles + 9 n Gauss coordinates
    cd* beta = nullptr;
    cd* beta_p = nullptr;           // admittance of the + side (indirect system; NULL = same as beta)
    double rc = 0, max_edge = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};   // bounding box of the vertices
    Geom g{};
};

// --------------------------------------------------------------- tree ----
constexpr int FB_MAXLEV = 12;
constexpr int FB_NOFF = 343;   // M2L offsets (dx,dy,dz) in [-3,3]^3 -> (dx+3)*49+(dy+3)*7+(dz+3)
constexpr int FB_ULIST = 27;
constexpr int FB_VLIST = 189;

struct fb_tree {
    const fb_mesh* mesh = nullptr;
    int dev = 0;
    int L = 0;
    double origin[3] = {0, 0, 0}, side = 0;
    int64_t n = 0;
    int32_t* perm = nullptr;                 // sorted position -> element
    int32_t* elem_pos = nullptr;             // element -> sorted position
    int32_t nbox[FB_MAXLEV + 1] = {0};
    uint32_t* keys[FB_MAXLEV + 1] = {nullptr};   // Morton keys of non-empty boxes, ascending
    int32_t* parent[FB_MAXLEV + 1] = {nullptr};  // parent box index (level l-1)
    int32_t* leaf_start = nullptr;           // nleaf + 1
    std::vector<int32_t> h_leaf_start;       // host copy
    int32_t* ucnt = nullptr;                 // per leaf
    int32_t* ulist = nullptr;                // per leaf x 27, ascending
    int32_t* vcnt[FB_MAXLEV + 1] = {nullptr};
    int32_t* vlist[FB_MAXLEV + 1] = {nullptr};   // per box x 189, ascending
    // M2L pairs grouped by (level, offset code): src box, dst box
    int32_t* m2l_src = nullptr;
    int32_t* m2l_dst = nullptr;
    std::vector<int64_t> m2l_group;          // (L+1)*343 + 1 prefix offsets
    // M2M / L2L pairs per level l (child level), grouped by octant: child, parent
    int32_t* oct_child[FB_MAXLEV + 1] = {nullptr};
    int32_t* oct_parent[FB_MAXLEV + 1] = {nullptr};
    std::vector<int64_t> oct_group[FB_MAXLEV + 1];   // 9 prefix offsets
    int64_t nlist_u = 0;
    // rotation blocks of the translation directions, one set per degree
    // bound P, shared by every operator built on this tree
    // Rotation blocks D^n of a set of directions.  D^n_{mu,m} = d^n_{mu,m}
    // e^{i m phi} with d real (Q = R_y(-theta) R_z(-phi)): d and the phase
    // table e^{i m phi} (m = -(P-1)..P-1) are kept too, so the RCR kernels
    // rotate with real multipliers after one phase per coefficient.
    struct RotSet {
        cd* r64 = nullptr;          // complex blocks, degrees < Pc (composed matrices)
        double* d64 = nullptr;      // real factors, degrees < P
        float* d32 = nullptr;
        cd* ph64 = nullptr;         // phase tables e^{i m phi}
        cf* ph32 = nullptr;
        int P = 0, Pc = 0, ndir = 0;
        int64_t per_dir = 0, per_dir_c = 0;
    };
    std::deque<RotSet> rot_sets;   // deque: references stay valid on push_back
};

// ----------------------------------------------------------- operator ----
// One translation task: dst[dst_idx[c]] += T * src[src_idx[c]] for a group
// of column pairs sharing the matrix T (rows x cols, row-major).
struct TransTask {
    int64_t t_off;       // offset of T in the matrix buffer (complex entries)
    int64_t pair_off;    // first pair in the pair arrays
    int32_t npairs;
    int32_t rows, cols;
    int64_t src_base, dst_base;   // offsets (complex entries) of the level arrays
};
struct TransTile {
    int32_t task, row0, col0, pad;
};

struct TransPlan {
    std::vector<TransTask> h_tasks;
    std::vector<TransTile> h_tiles;
    TransTask* tasks = nullptr;
    TransTile* tiles = nullptr;
    const int32_t* src_idx = nullptr;
    const int32_t* dst_idx = nullptr;
    int ntiles = 0;
};

// One RCR translation task: dst[dst_idx[c]] += D_out^H C D_in src[src_idx[c]]
// with the rotation blocks D of one direction and one coaxial set C.
struct RcrTask {
    int64_t rot_off;     // complex offset of the direction's rotation blocks
    int64_t coax_off;    // complex offset of the coaxial set [m][n'][n] (stride pc)
    int64_t pair_off;
    int32_t npairs, p_out, p_in, pc;
    int64_t src_base, dst_base;
    int32_t staged;      // 0: per-pair tiles, 1: staged GEMM passes, 2: staged with tensor-core
                         // rotations, 3: staged in double-FP32, 4: per-pair tiles in double-FP32,
                         // 5: staged with tensor-core rotations and coaxial step
    int32_t pad;
};
struct RcrTile {
    int32_t task, col0, nb, pad;
};
// Tiles of an RCR plan for a number of right-hand sides: the columns of a
// task are its (pair, rhs) combinations, pair-major.
struct RcrTileSet {
    RcrTile* tiles = nullptr;
    int ntiles = 0;
    size_t smem = 0;
};
// Large orders run as staged batched GEMM passes (rcr_staged.cu) instead of
// per-pair tiles: a pair's rotation and coaxial blocks must then be shared
// by many pairs to be read at a useful rate.  By default a level is staged
// from order FB_STG_PMIN on, and always when a pair's working set
// (p_in^2 + max(p_in, p_out)^2 coefficients) exceeds what one CTA's shared
// memory holds; the autotuner and fb_operator_set_forms choose per level.
constexpr int FB_STG_PMIN = 40;
bool fb_rcr_tile_fits(int p_in, int p_out, size_t csize);
int fb_rcr_default_staged(int p_in, int p_out, size_t csize);
struct RcrPlan {
    std::vector<RcrTask> h_tasks;
    std::vector<RcrTile> h_tiles;
    RcrTask* tasks = nullptr;
    RcrTile* tiles = nullptr;
    const int32_t* src_idx = nullptr;
    const int32_t* dst_idx = nullptr;
    int ntiles = 0;
    int nb = 1;          // box pairs per CTA
    size_t smem = 0;     // dynamic shared memory per CTA (bytes)
    size_t csize = 0;    // bytes per complex coefficient
    void* stg = nullptr;        // staged passes of the large-order tasks
    int64_t stg_elems = 0;      // staging coefficients they need per buffer
    std::map<int, RcrTileSet> multi;   // tiles for nrhs > 1 (built on first use), key 2 nrhs + df
    RcrTileSet df_tiles;        // tiles of the double-FP32 tasks (one right-hand side)
};
void fb_rcr_free(RcrPlan& p);
bool fb_stg_staged(const RcrTask& tk);
fb_status fb_stg_build(const RcrPlan& pl, const std::vector<int>& theta_slot, int64_t per_dir, const cd* coax64,
                       void** out, int64_t* elems);
void fb_stg_free(void*& plan);
// tables of the staged levels that run in double-FP32 arithmetic (FP64 operators)
struct DfTabs {
    const df* rf;        // folded rotation tables
    const cx<df>* coax;  // coaxial sets
};
// tables of the tensor-core rotation passes of the staged levels that use them
struct StcTabs {
    const float* tab;
    const int64_t* off;
    int64_t per;
    int* err;
};
// Runs the staged passes of a plan (pass_mask bits: pre-pass, rotation,
// coaxial, back-rotation; only_level >= 0: that level of the plan alone).
fb_status fb_stg_run_f(void* plan, const float* rf, int64_t fper, const cf* rph, int prot, const cf* coax,
                       const cf* src, cf* dst, cf* U, cf* V, cudaStream_t s, int nrhs, int64_t rstride,
                       const StcTabs& tc, int only_level = -1, int pass_mask = 15);
bool fb_stg_uses_tc(const void* plan);
fb_status fb_stg_run_d(void* plan, const double* rf, int64_t fper, const cd* rph, int prot, const cd* coax,
                       const cd* src, cd* dst, cd* U, cd* V, cudaStream_t s, int nrhs, int64_t rstride,
                       const DfTabs& dft, int only_level = -1, int pass_mask = 15);
bool fb_stg_uses_df(const void* plan);
int fb_stg_level_count(const void* plan);
// form: 1 CUDA cores, 2 rotations on the tensor cores, 3 double-FP32 arithmetic,
// 5 rotations and coaxial step on the tensor cores
void fb_stg_level_info(const void* plan, int li, int64_t* src_base, int64_t* dst_base, int* form);
struct fb_op;
fb_status fb_stg_op_pass_times(fb_op* op, cudaStream_t s, double* ms, int* form);
fb_status fb_stg_df_tables(fb_op* op, cudaStream_t s);
fb_status fb_rcr_df_factors(fb_op* op, int P);
fb_status fb_near_bf16(fb_op* op, int enable, cudaStream_t s);
// Creates an operator; `donor` (an FP64 FMM operator of the same mesh, tree,
// k and kind, or NULL) lends its near-field entries.
fb_status fb_operator_create_impl(const fb_mesh* mesh, const fb_tree* tree, double k, int kind, int precision,
                                  double d0, int pmin, cudaStream_t s, fb_op** out, const fb_op* donor = nullptr);
fb_status fb_stg_tables(fb_op* op, const double* rotd64, cudaStream_t s);

// A group of box pairs sharing one composed translation matrix (job) on the
// tensor cores: sources from level src_level, targets in level dst_level.
struct TcGroup {
    int job;
    int64_t pair_off;
    int32_t npairs;
    int src_level, dst_level;
};

// One composed translation matrix T = D_out^H C D_in to build.
struct ComposeJob {
    int64_t t_off;       // output offset (complex entries)
    int64_t rot_off;     // rotation blocks of the direction
    int64_t coax_off;    // coaxial set [m][n'][n] with stride pc
    int p_out, p_in, pc;
};

struct fb_op {
    const fb_mesh* mesh = nullptr;
    const fb_tree* tree = nullptr;
    int dev = 0;
    int kind = 0, prec = 0;
    double k = 0;
    double d0 = 0;           // order rule parameters (FMM)
    int pmin = 0;
    int64_t n = 0;
    // indirect system (FB_OP_IBEM): constituent M, L, M', L' and work space
    fb_op* sub[4] = {nullptr, nullptr, nullptr, nullptr};
    cd* ib_work = nullptr;                   // 6 N
    cd *ib_beta_p = nullptr, *ib_beta_m = nullptr;
    // dense
    cd* dense = nullptr;
    // FMM
    int L = 0;
    int p[FB_MAXLEV + 1] = {0};
    int64_t lev_off[FB_MAXLEV + 2] = {0};    // offsets of each level in mp/loc (complex entries)
    int64_t nf_count = 0;
    int64_t* nf_off = nullptr;               // per leaf, entries offset
    int32_t* nf_ncol = nullptr;              // per leaf, columns K_t
    std::vector<int64_t> h_nf_off;
    std::vector<int32_t> h_nf_ncol;
    cd* nf64 = nullptr;                      // FP64 operators only
    cf* nf32 = nullptr;
    cd* self64 = nullptr;                    // mixed: FP64 leaf self-blocks (nr x nr, leaf-major)
    cd* w64 = nullptr; cf* w32 = nullptr;    // P2M, [N sorted][P_L]
    cd* v64 = nullptr; cf* v32 = nullptr;    // L2P, [N sorted][P_L]
    void* mp = nullptr;                      // multipoles (all levels; exp_nrhs sets)
    void* loc = nullptr;                     // locals (all levels; exp_nrhs sets)
    int exp_nrhs = 1;                        // right-hand sides the expansion buffers hold
    cd* T64 = nullptr; cf* T32 = nullptr;    // translation matrices
    int64_t T_count = 0;
    std::vector<int64_t> m2l_toff;           // (L+1)*343: offset of T or -1
    int64_t m2m_toff[FB_MAXLEV + 1][8];      // child level l, octant
    int64_t l2l_toff[FB_MAXLEV + 1][8];
    TransPlan m2l, m2m[FB_MAXLEV + 1], l2l[FB_MAXLEV + 1];
    // RCR form: rotation blocks per direction, coaxial sets, plans
    int Prot = 0;
    int64_t per_dir = 0;
    cd* rot64 = nullptr;                     // complex rotation blocks, degrees < FB_COMPOSE_PMAX
    double* rotd64 = nullptr; float* rotd32 = nullptr;   // real parts d (owned by the tree)
    cd* rph64 = nullptr; cf* rph32 = nullptr;            // phase tables (owned by the tree)
    cd* coax64 = nullptr; cf* coax32 = nullptr;
    int64_t coax_count = 0, rot_count = 0;
    // per direction: a direction with the same polar angle (shares d^n)
    std::vector<int> theta_rep;
    std::vector<int> theta_slot;             // direction -> its polar-angle group
    std::vector<int> theta_dirs;             // group -> its representative direction
    void* rotf = nullptr;                    // folded rotation tables (staged RCR), per group
    int64_t rotf_per = 0;                    // values per group and table
    float* stc_tab = nullptr;                // pre-split canonical tables of the tensor-core staged passes
    int64_t* stc_off = nullptr;              // their block offsets per (degree, part)
    int64_t stc_per = 0;                     // floats per group and table
    int stc_P = 0;
    int* stc_err = nullptr;                  // error flag of the tensor-core staged passes
    const fb_op* near_donor = nullptr;       // during creation: an FP64 FMM operator of the same
                                             // mesh, tree, k and kind whose near-field entries are copied
    uint32_t* nf16 = nullptr;                // near-field entries as BF16 pairs (re low, im high half)
    int near16 = 0;                          // 1: the matvec reads nf16 instead of nf32
    df* rotf_df = nullptr;                   // FP64 operators: folded tables and coaxial sets in
    cx<df>* coax_df = nullptr;               // double-FP32 for the staged levels that use it
    df* rotd_df = nullptr;                   // ... and the real factors of degrees < rotd_df_P
    int rotd_df_P = 0;                       // (per-pair tiles in double-FP32)
    int64_t rotd_df_per = 0;                 // values per direction
    std::vector<int> dir_of_code;            // M2L offset code -> direction (-1: near)
    // RCR form per level: 1 = staged passes, 0 = per-pair tiles (M2L of
    // level l; M2M and L2L between levels l-1 and l)
    int stg_m2l[FB_MAXLEV + 1] = {0};
    int stg_pair[FB_MAXLEV + 1] = {0};
    // staging buffers of the large-order RCR passes (U, V: stg_elems
    // complex values each, in the operator's precision)
    void* stg_u = nullptr;
    void* stg_v = nullptr;
    int64_t stg_elems = 0;
    RcrPlan m2l_rcr, m2m_rcr[FB_MAXLEV + 1], l2l_rcr[FB_MAXLEV + 1];
    // tensor-core (3xTF32) stacked M2L: dense levels (auto) / every level
    void* tc_plan = nullptr;
    void* tc_plan_all = nullptr;
    int tc_level[FB_MAXLEV + 1] = {0};      // 1: M2L of this level on tensor cores (auto)
    RcrPlan m2l_rcr_rest;                   // RCR M2L of the other levels
    void* tc_m2m[FB_MAXLEV + 1] = {nullptr};   // tensor-core M2M / L2L per child level
    void* tc_l2l[FB_MAXLEV + 1] = {nullptr};
    std::vector<int> m2l_job;               // (level, offset) -> compose job
    int m2m_job[FB_MAXLEV + 1][8];
    int l2l_job[FB_MAXLEV + 1][8];
    int method = 0;                         // FB_TRANS_*
    std::vector<ComposeJob> h_jobs;         // composed matrices (built on demand)
    std::vector<int> h_job_level, h_job_m2l;
    std::vector<char> job_done;
    // translation method per level: 0 = composed stacked GEMM, 1 = RCR
    int mode_m2l[FB_MAXLEV + 1] = {0};
    int mode_m2m[FB_MAXLEV + 1] = {0};
    int mode_l2l[FB_MAXLEV + 1] = {0};
    // device vectors for host-memspace calls
    cd* io_x = nullptr;
    cd* io_y = nullptr;
    // FGMRES workspaces of solves with this operator as A, kept between
    // solves so that a steady-state solve allocates nothing (krylov.cu)
    void* fg_work = nullptr;
    void* fg_bwork = nullptr;
    // CUDA-graph replay of the FMM matvec (fb_operator_use_graphs)
    int use_graphs = 0;
    void* graphs = nullptr;
    long long buf_gen = 0;                   // bumped when a buffer a graph may capture is reallocated
};

struct LearnedNet;
struct fb_precond {
    fb_op* op = nullptr;
    int kind = 0;
    int64_t n = 0;
    int64_t* blk_off = nullptr;    // per leaf, offset of its inverse block
    cd* inv64 = nullptr;
    cf* inv32 = nullptr;
    LearnedNet* net = nullptr;     // learned preconditioner (refines `base`)
    const fb_precond* base = nullptr;
    int use_graphs = 0;            // CUDA-graph replay of the apply (fb_precond_use_graphs)
    int ibem = 0;                  // block Jacobi of the indirect system: 2 x 2 leaf blocks
    void* graphs = nullptr;
    // inner-outer preconditioner: `inner_its` GMRES steps on `inner_op`
    // (right-preconditioned by `base`), work buffers in `inner`
    fb_op* inner_op = nullptr;
    int inner_its = 0;
    void* inner = nullptr;
};
fb_status fb_inner_create(fb_precond* pc, cudaStream_t s);
// Releases the FGMRES workspaces cached on an operator.
void fb_krylov_free(fb_op* op);
void fb_inner_free(void*& inner);

// ------------------------------------------------------ launch counting ----
// Running total of kernel launches issued by the library (tracing aid,
// reported by fb_kernel_launches()).
void fb_count_launch(long long n = 1);

// Per-phase CUDA-event timing of one FMM matvec (tracing aid).
constexpr int FB_NPHASE = 7;   // P2M, M2M, M2L tensor part, M2L rest, L2L, near+L2P, total
struct PhaseTimer {
    cudaEvent_t ev[FB_NPHASE + 1];
};

// --------------------------------------------------- internal interface ----
fb_status fb_dense_create(fb_op* op, cudaStream_t s);
fb_status fb_dense_apply(const fb_op* op, const cd* x, cd* y, cudaStream_t s);
fb_status fb_fmm_create(fb_op* op, double d0, int pmin, cudaStream_t s);
fb_status fb_fmm_apply(fb_op* op, const cd* x, cd* y, cudaStream_t s, PhaseTimer* pt = nullptr,
                       int nrhs = 1);
fb_status fb_fmm_apply_noalloc(fb_op* op, const cd* x, cd* y, cudaStream_t s);
fb_status fb_rcr_upload(fb_op* op, RcrPlan& pl, const int32_t* src, const int32_t* dst, size_t csize);
fb_status fb_tree_rotations(fb_tree* t, int P, const std::vector<double>& dirs, cudaStream_t s,
                            const fb_tree::RotSet** out);
fb_status fb_compose_jobs(fb_op* op, const std::vector<int>& which, cudaStream_t s);
fb_status fb_rcr_run_op(fb_op* op, RcrPlan& pl, void* src, void* dst, cudaStream_t s, int nrhs, int64_t rstride);
// Installs per-level RCR forms (m2l[l], pair[l]: 1 = staged; levels whose
// per-pair working set does not fit a CTA are staged regardless) and
// rebuilds the affected plans.
fb_status fb_rcr_restage(fb_op* op, const int* m2l, const int* pair);
// reps: timed runs per candidate (median), after one untimed run
fb_status fb_autotune_impl(fb_op* op, int nrhs, cudaStream_t s, double* times, int* choice, int reps = 3);
fb_status fb_set_forms_impl(fb_op* op, const int* choice, cudaStream_t s);
fb_status fb_compose_all(fb_op* op, cudaStream_t s);
// Leaf self-blocks of the FP64 near-field entries (leaf t at d_off[t], nr x nr).
fb_status fb_self_blocks(const fb_op* op, const int64_t* d_off, cd* out, cudaStream_t s);
// Composed p^2 x p^2 translation matrices exist only for orders up to this
// bound: above it one matrix outgrows the RCR arithmetic it replaces (the
// dense form costs ~p/4 times RCR) and a level's set reaches tens of GB.
constexpr int FB_COMPOSE_PMAX = 32;
// Largest expansion order the rotation setup supports.
constexpr int FB_ROT_PMAX = 256;
// M2L of level l (pair = false) or M2M/L2L between levels l-1 and l (pair = true)
// has composed matrices.
inline bool fb_composable(const fb_op* op, int l, bool pair) {
    return op->p[l] <= FB_COMPOSE_PMAX && (!pair || op->p[l - 1] <= FB_COMPOSE_PMAX);
}
fb_status fb_learned_alloc(LearnedNet*& net, const fb_op* op, const fb_precond* bj, cudaStream_t s);
void fb_learned_free(LearnedNet*& net);
fb_status fb_learned_forward(LearnedNet* net, const cd* v, cd* z, cudaStream_t s);
fb_status fb_learned_apply(LearnedNet* net, const cd* v, cd* z, cudaStream_t s);
fb_status fb_learned_loss_grad(LearnedNet* net, const cd* R, const cd* E, int npairs, double* loss, cudaStream_t s);
fb_status fb_learned_adam_step(LearnedNet* net, double lr, cudaStream_t s);
fb_status fb_learned_init(LearnedNet* net, uint64_t seed, cudaStream_t s);
fb_status fb_learned_adjoint_ops(LearnedNet* net, cudaStream_t s);
fb_status fb_learned_set_objective(LearnedNet* net, int objective);
fb_status fb_learned_params_changed(LearnedNet* net, cudaStream_t s);
int64_t fb_learned_nparam(const LearnedNet* net);
float* fb_learned_weights(LearnedNet* net);
float* fb_learned_grads(LearnedNet* net);
fb_status fb_tc_build(fb_op* op, const std::vector<int>& levels, void** slot, cudaStream_t s);
fb_status fb_tc_build_groups(fb_op* op, const std::vector<TcGroup>& groups, const int32_t* src_idx,
                             const int32_t* dst_idx, void** slot, cudaStream_t s);
fb_status fb_tc_run(fb_op* op, void* plan, const cf* src, cf* dst, cudaStream_t s, int nrhs = 1,
                    int64_t rstride = 0);
fb_status fb_tc_check(const fb_op* op);
long long fb_tc_set_wait_limit(long long limit);
long long fb_tc_wait_limit();
int fb_tc_inject_stall();
fb_status fb_stc_tables(fb_op* op, cudaStream_t s);
int fb_tc_set_inject_stall(int on);
// Error status of the bounded device waits of an operator (and of the
// constituents of a composite); reads and clears the flags.
fb_status fb_op_wait_status(const fb_op* op);
void fb_tc_free(void*& plan);
void fb_fmm_destroy(fb_op* op);
fb_status fb_apply_any(fb_op* op, const cd* x, cd* y, cudaStream_t s, int nrhs = 1);
fb_status fb_ibem_create(fb_op* op, cudaStream_t s);
void fb_ibem_free(fb_op* op);
fb_status fb_ibem_apply(fb_op* op, const cd* x, cd* y, cudaStream_t s, int nrhs);
fb_status fb_dbem5_create(fb_op* op, cudaStream_t s);
fb_status fb_dbem5_apply(fb_op* op, const cd* x, cd* y, cudaStream_t s, int nrhs);
// operators composed of other operators (no near field or tree data of their own)
inline bool fb_is_composite(const fb_op* op) { return op->kind == FB_OP_IBEM || op->kind == FB_OP_DBEM5; }
extern "C" void fb_operator_destroy(fb_op* op);
fb_status fb_pc_apply(const fb_precond* pc, const cd* x, cd* y, cudaStream_t s, int nrhs = 1);
int fb_order_rule(double k, double delta, double d0, int pmin);
