/*
 * fmmbem.h -- C ABI of the GB300 (sm_103a) FMM-accelerated Helmholtz BEM.
 *
 * The library computes the matrix-vector product at the heart of the
 * room-acoustics boundary element method of Gumerov & Duraiswami, "Fast
 * multipole accelerated boundary element methods for room acoustics", and
 * solves the direct-BEM system with flexible GMRES on one GPU.
 *
 * Problem (Sec. 2): Helmholtz equation (Eq. sp2) in a room bounded by flat
 * triangles, impedance wall condition (Eq. sp3) with the normal pointing out
 * of the room, monopole source (Eq. sp6), time factor e^{-i omega t},
 * G = e^{ikR}/(4 pi R).  With the admittance beta = 1/zeta the direct BEM
 * (Eq. dbem4) reads
 *      A psi = L gamma,   A = 1/2 I + M - i k L diag(beta),
 *      gamma = -(dpsi_in/dn - i k beta psi_in)                 (Eq. sp7)
 * with the operators L, M (Eq. dbem2) and L' (Eq. ibem3).  Piecewise-constant
 * collocation at element centroids.
 *
 * Conventions of every call:
 *   - every function returns fb_status (FB_OK == 0); on error
 *     fb_last_error() returns a message for the calling thread;
 *   - complex arrays are interleaved (re, im) doubles: element i is
 *     (a[2i], a[2i+1]);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default);
 *     calls enqueue work on it and synchronise it only where documented;
 *   - host input arrays are copied; the caller keeps ownership of every
 *     pointer it passes; handles are owned by the library and released by
 *     the matching *_destroy (NULL is accepted and ignored);
 *   - `memspace` says where caller arrays live: FB_MEM_HOST (plain or
 *     pinned host memory; the call copies and synchronises the stream) or
 *     FB_MEM_DEVICE (device pointers on the current device, no sync);
 *   - all state of a handle lives on the device that was current when it
 *     was created; no call is thread-safe on the same handle;
 *   - no C++ exception crosses this boundary; a CUDA error is reported as
 *     FB_ERR_CUDA and leaves the handle in an unspecified state (destroy it).
 */
#ifndef FMMBEM_H
#define FMMBEM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FB_API __attribute__((visibility("default")))
#else
#define FB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int fb_status;
#define FB_OK 0
#define FB_ERR_ARG 1       /* invalid argument or unsupported combination  */
#define FB_ERR_CUDA 2      /* a CUDA runtime call failed                   */
#define FB_ERR_NOCONV 3    /* FGMRES hit maxit before the tolerance        */
#define FB_ERR_BREAKDOWN 4 /* FGMRES breakdown (zero Hessenberg pivot)     */
#define FB_ERR_NAN 5       /* NaN/Inf met in a residual                    */
#define FB_ERR_TIMEOUT 6   /* a bounded device wait ran out                */
#define FB_ERR_OOM 7       /* device allocation failed                     */
#define FB_ERR_STATE 8     /* handle in a state that does not allow this   */

/* Operators (Eqs. dbem2, ibem3, dbem4). */
#define FB_OP_L 0  /* single layer          L[s](x) = int s G dS_y           */
#define FB_OP_M 1  /* double layer          M[s](x) = int s dG/dn_y dS_y     */
#define FB_OP_LP 2 /* adjoint double layer L'[s](x) = int s dG/dn_x dS_y     */
#define FB_OP_A 3  /* direct-BEM system     A = 1/2 I + M - ik L diag(beta)  */
#define FB_OP_MP 4 /* hypersingular        M'[s](x) = d/dn_x int s dG/dn_y dS_y
                      (Eq. ibem3, finite part; near/self entries by the flat-element
                      form (n_x.n)[k^2 S + sum_e int_e grad_y G.m dl]
                      + sum_e int_e (n.grad_x G)(t.m) dl, far by the 3-point rule
                      of d2G/dn_x dn_y; FMM: dipole P2M and normal-gradient L2P) */
#define FB_OP_IBEM 5 /* indirect-BEM system of Eq. ibem5 with two unknowns per
                      element, x = [psi+ (N), psi- (N)] (scattered field on the
                      side the normal points to, and on the other side), 2N x 2N:
                        row 1: (psi- + psi+)/2 - M[psi+ - psi-] + L[a- psi- + a+ psi+]
                        row 2: -M'[psi+ - psi-] + (a+ psi+ - a- psi-)/2
                               + L'[a- psi- + a+ psi+]
                      with a = k/(i zeta) = -i k beta per side (beta- = the mesh
                      admittance, beta+ = fb_mesh_set_admittance_plus, default
                      beta-), both copied at creation.  Composed of the L, M, L',
                      M' operators of the given precision on the same tree.
                      fb_precond_create builds its block Jacobi from 2n x 2n leaf
                      blocks (FMM precisions); the learned network does not
                      apply to it. */
#define FB_OP_DBEM5 6 /* direct-BEM system of Eq. dbem5 for the unknown
                      q = d psi_sc/dn (N x N): 1/2 q + (1/zeta) M[zeta q]
                      + (k/(i zeta)) L[q], i.e. 1/2 q + beta M[q/beta]
                      - i k beta L[q]; needs beta != 0 on every element
                      (FB_ERR_ARG otherwise).  Composed of M and L; right-hand
                      side and psi_sc by fb_dbem5_rhs / fb_dbem5_psi; block
                      Jacobi from the leaf blocks 1/2 + beta_i M_ij / beta_j
                      - i k beta_i L_ij (FMM precisions). */

/* How an operator is applied. */
#define FB_PREC_FP64_DENSE 0 /* stored dense N x N complex128 matrix        */
#define FB_PREC_FP64_FMM 1   /* FMM, all arithmetic in FP64                 */
#define FB_PREC_MIXED_FMM 2  /* FMM: FP32 near field, P2M/L2P and
                                translations; FP64 setup and I/O            */

#define FB_MEM_HOST 0
#define FB_MEM_DEVICE 1

#define FB_PC_NONE 0
#define FB_PC_BLOCK_JACOBI 1 /* inverse of each leaf's self near-field block */
#define FB_PC_LEARNED 2      /* learned octree network refining block Jacobi */

typedef struct fb_mesh fb_mesh;
typedef struct fb_tree fb_tree;
typedef struct fb_op fb_op;
typedef struct fb_precond fb_precond;

/* Version string of the library (static storage). */
FB_API const char* fb_version(void);

/* Copies the last error message of the calling thread into buf (always
 * NUL-terminated when len > 0).  Returns the last error code. */
FB_API fb_status fb_last_error(char* buf, size_t len);

/* ---------------------------------------------------------------- mesh -- */

/* Flat-triangle surface mesh (Sec. 4).  verts: nv x 3 doubles (host), tris:
 * nt x 3 int32 vertex indices (host), counter-clockwise seen from outside the
 * room so that (v1-v0) x (v2-v0) is the outward normal (Eq. sp3).  Computes on
 * the device: centroids (collocation points), unit normals, areas, the
 * 3-point Gauss points of every element, the longest edge and the near-field
 * cutoff r_c = 1.5 x longest edge (Sec. 3.3: entries of elements closer than
 * r_c use closed-form integrals).  Admittance is initialised to 0 (rigid).
 * Errors: FB_ERR_ARG for nv < 3, nt < 1, an index out of range or a
 * degenerate (zero-area) triangle. */
FB_API fb_status fb_mesh_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                         void* stream, fb_mesh** out);

/* Per-element complex admittance beta = 1/zeta (Eq. sp4; beta = 0 is the
 * rigid wall of Eq. sp5), nt interleaved complex values in `memspace`. */
FB_API fb_status fb_mesh_set_admittance(fb_mesh* mesh, const double* beta, int memspace, void* stream);

/* Admittance of the + side of every element for the indirect system
 * (FB_OP_IBEM; Eq. ibem4: the side the normal points to), nt interleaved
 * complex values in `memspace`.  Until set, the + side takes the admittance
 * of fb_mesh_set_admittance. */
FB_API fb_status fb_mesh_set_admittance_plus(fb_mesh* mesh, const double* beta, int memspace, void* stream);

/* Element count, near-field cutoff r_c and longest edge. */
FB_API fb_status fb_mesh_info(const fb_mesh* mesh, int64_t* nt, double* rc, double* max_edge);

/* Copies centroids and unit normals (nt x 3 each, host; either may be NULL). */
FB_API fb_status fb_mesh_geometry(const fb_mesh* mesh, double* centroids, double* normals);

FB_API void fb_mesh_destroy(fb_mesh* mesh);

/* ---------------------------------------------------------------- tree -- */

/* Uniform octree over the element centroids (Sec. 3.3), built on the device:
 * root = bounding cube of the vertices (side x (1 + 1e-6)), an element
 * belongs to the leaf containing its centroid, leaf level = first level >= 2
 * whose fullest leaf holds <= leaf_max elements, capped at the deepest level
 * whose box side exceeds r_c (the paper's delta > r_c).  Builds the U-lists
 * (touching leaves) and V-lists (M2L interaction lists) of every level.
 * Errors: FB_ERR_ARG if leaf_max < 1 or the mesh allows no level >= 2 with
 * box side > r_c (use FB_PREC_FP64_DENSE for such meshes). */
FB_API fb_status fb_tree_build(const fb_mesh* mesh, int leaf_max, void* stream, fb_tree** out);

/* Leaf level, root origin (3 doubles), root side, and box counts per level
 * (array of leaf_level + 1 int64, may be NULL). */
FB_API fb_status fb_tree_info(const fb_tree* tree, int* leaf_level, double* origin, double* side,
                       int64_t* nboxes);

/* Host copies for inspection.  which: 0 = element order (nt int64: sorted
 * position -> element index), 1 = leaf start offsets (nleaf+1 int64),
 * 2 = box Morton keys of level `level` (nboxes int64), 3 = U-list as
 * (target, source) leaf-index pairs (2*count int64), 4 = V-list of `level`
 * as (target, source) box-index pairs.  *count receives the number of
 * entries (pairs for 3/4); pass out = NULL to query it. */
FB_API fb_status fb_tree_export(const fb_tree* tree, int which, int level, int64_t* out, int64_t* count);

FB_API void fb_tree_destroy(fb_tree* tree);

/* ------------------------------------------------------------ operator -- */

/* Operator `kind` (FB_OP_*) at wavenumber k > 0, applied as `precision`
 * (FB_PREC_*).  FMM precisions need `tree` (built from the same mesh); dense
 * ignores it (may be NULL).  Truncation per level (the paper defers it to
 * another reference): p_l = max(pmin, ceil(k r_l + 1.8 d0^(2/3) (k r_l)^(1/3))),
 * r_l = sqrt(3)/2 x box side.  Setup runs on the device in FP64: near-field
 * entries (closed-form singular parts, Sec. 3.3), per-leaf P2M/L2P operators,
 * coaxial coefficients by the recursions of Sec. 3.3.1 (original scheme for
 * k tau < 1, stabilised scheme otherwise), rotation blocks and the composed
 * translation matrices.  The admittance of `mesh` at creation time is used.
 * Errors: FB_ERR_ARG (k <= 0, kind/precision out of range, missing tree,
 * dense N > 60000), FB_ERR_OOM. */
FB_API fb_status fb_operator_create(const fb_mesh* mesh, const fb_tree* tree, double k, int kind,
                             int precision, double d0, int pmin, void* stream, fb_op** out);

/* An FMM operator of the donor's mesh, tree, wavenumber and kind, at another
 * precision or order rule (d0, p_min): the near-field entries (Sec. 3.3),
 * which depend on neither, are copied from the donor when it is an FP64 FMM
 * operator (which keeps its FP64 entries) instead of being integrated
 * again; otherwise they are computed as by fb_operator_create.  Meant for
 * the FP64 true-residual operator, the mixed operator and the low-accuracy inner operator of
 * one solve.  Errors: FB_ERR_ARG (NULL, dense or composite donor, dense
 * precision). */
FB_API fb_status fb_operator_create_like(const fb_op* donor, int precision, double d0, int pmin, void* stream,
                                         fb_op** out);

/* y = Op x.  x, y: N interleaved complex doubles in `memspace`; they must not
 * overlap.  Device memspace: enqueued on `stream`, no sync. */
FB_API fb_status fb_operator_apply(fb_op* op, const double* x, double* y, int memspace, void* stream);

/* N, number of FMM levels used (0 for dense) and p per level (array of
 * leaf_level + 1 ints, entries below level 2 are 0; may be NULL). */
FB_API fb_status fb_operator_info(const fb_op* op, int64_t* n, int* leaf_level, int* p_per_level);

/* Host copies of FP64 setup data for inspection.  which: 0 = near-field
 * entries of leaf `index` (rows x cols complex, row-major; rows = the leaf's
 * elements in tree order, cols = the elements of its U-list leaves in
 * ascending leaf order), 1 = P2M operator of leaf `index` (n_leaf x p_L^2
 * complex, row per element), 2 = L2P operator of leaf `index` (n_leaf x p_L^2),
 * 3 = M2L translation matrix of level `level`, offset code `index`
 * (p_l^2 x p_l^2; offset (dx,dy,dz) in box units, code = (dx+3)*49 +
 * (dy+3)*7 + (dz+3)), 4 = M2M matrix child->parent at child level `level`,
 * octant `index` (p_{l-1}^2 x p_l^2), 5 = L2L matrix parent->child at child
 * level `level`, octant `index` (p_l^2 x p_{l-1}^2), 6 = dense matrix row
 * `index` (N complex), 7 = per level 1 + 0i if its M2L runs on the tensor
 * cores under the current translation method, else 0 (leaf_level + 1
 * values), 8 = real rotation factors d^n of degree n = `level` for the
 * direction of M2L offset code `index` ((2n+1) x (2n+1), row mu, column m,
 * returned as complex with zero imaginary part; the rotation block of that
 * direction is D^n_{mu,m} = d^n_{mu,m} e^{i m phi}, phi its azimuth).
 * *count receives the number of complex values. */
FB_API fb_status fb_operator_export(const fb_op* op, int which, int level, int64_t index, double* out,
                             int64_t* count);

FB_API void fb_operator_destroy(fb_op* op);

/* Tracing: y = Op x on device pointers (enqueued on `stream`, then the stream
 * is synchronised) with CUDA-event times in milliseconds per phase:
 * phase_ms[0] = zeroing + P2M, [1] = M2M, [2] = M2L on the tensor cores
 * (0 when none), [3] = rest of M2L, [4] = L2L, [5] = near field + L2P,
 * [6] = total (dense operators fill only [6]).  phase_ms must hold 7
 * doubles. */
FB_API fb_status fb_operator_apply_timed(fb_op* op, const double* x, double* y, void* stream,
                                         double* phase_ms);

/* How an FMM operator applies its M2M / M2L / L2L translations. */
#define FB_TRANS_AUTO 0     /* library's choice per level (default)                 */
#define FB_TRANS_COMPOSED 1 /* stacked GEMM with the composed p^2 x p^2 matrix of
                               each (level, translation vector), Sec. 3.3           */
#define FB_TRANS_RCR 2      /* rotation - coaxial - back-rotation per box pair
                               (Sec. 3.3, Sec. 3.3.1): (10/3) p^3 complex MACs      */
#define FB_TRANS_TENSOR 3   /* mixed precision only: every M2L level as stacked
                               composed GEMMs on the tensor cores (3xTF32)          */

/* Selects the translation method of an FMM operator; results agree to
 * rounding.  FB_TRANS_AUTO: FP64 operators use RCR everywhere; mixed operators
 * run the M2L of levels with >= 48 box pairs per translation vector as
 * tensor-core GEMMs (3xTF32) and the rest, M2M and L2L by RCR.
 * FB_TRANS_TENSOR builds its tensor-core tiles on first selection
 * (allocates; synchronises the legacy stream).  Errors: FB_ERR_ARG for a
 * dense operator, an unknown method or FB_TRANS_TENSOR on an FP64 operator. */
FB_API fb_status fb_operator_set_translation(fb_op* op, int method);

/* Size of the library-wide static device buffer used by
 * fb_operator_apply_noalloc (32 MiB, held by every GPU that loads the
 * library until the process exits). */
#define FB_NOALLOC_SCRATCH_BYTES (32u << 20)

/* y = Op x for an FMM operator without allocating anything.
 *
 * (The paper has no counterpart: this is a deployment variant.)  Some callers
 * cannot allocate device memory at the moment they apply an operator:
 * real-time audio callbacks that must not block in the driver's allocator,
 * or hosts whose device memory is owned by a fixed arena that the library
 * may not grow.  This call runs the same FMM
 * matvec as fb_operator_apply, but keeps its per-call scratch (the multipole
 * and local expansions of every level) in a file-scope static device buffer
 * of FB_NOALLOC_SCRATCH_BYTES instead of the operator's own buffers; it calls
 * no cudaMalloc, cudaFree or allocating library routine.
 *   x, y:  N interleaved complex doubles, DEVICE pointers, not overlapping.
 *   The operator's device must be current (FB_ERR_ARG otherwise).  The
 *   first call on a device resolves the buffer's device address
 *   (cudaGetSymbolAddress) for that device; make that first call before any
 *   stream capture.
 *   All calls share the one buffer: the expansions are cleared at the start
 *   of every call, and calls that overlap on the GPU (other streams, other
 *   threads) race on it and give wrong results.
 * Errors: FB_ERR_ARG for a dense operator, a current device other than the
 * operator's, or when the operator's expansions
 * (2 x sum over levels of boxes x p^2 complex values, FP32 for the mixed
 * precision, FP64 otherwise) exceed FB_NOALLOC_SCRATCH_BYTES; FB_ERR_CUDA if
 * the buffer's address cannot be resolved. */
FB_API fb_status fb_operator_apply_noalloc(fb_op* op, const double* x, double* y, void* stream);

/* Failure detection of the device waits.  The tensor-core translation
 * kernels poll mbarriers in bounded loops; when a bound runs out the kernel
 * records an error flag, waits for the copies and tensor-core operations it
 * has already issued (they always complete), releases its tensor memory and
 * returns, so the context stays usable.
 * fb_operator_status: synchronises `stream` and returns FB_ERR_TIMEOUT if a
 *   bounded wait of the operator's kernels ran out since the last check
 *   (clearing the flag), else FB_OK.  fb_fgmres_solve and
 *   fb_fgmres_solve_multi check their operators the same way when they end
 *   and report FB_ERR_TIMEOUT as the solve's status.
 * fb_set_device_wait_limit: polls per wait before giving up (library-wide,
 *   default 2^26, >= 1; *previous receives the old value if not NULL).
 * fb_test_stall_device_waits: test hook; while enabled, every tensor-core
 *   translation kernel first waits on a barrier nothing signals, so that
 *   wait runs out and the kernel takes the error path above (no fault, no
 *   hang: every wait is bounded).
 * Errors: FB_ERR_ARG (NULL operator, limit < 1). */
FB_API fb_status fb_operator_status(fb_op* op, void* stream);

/* Near-field entries (Sec. 3.3, the singular and near-singular part of a
 * mixed FMM operator) stored as BF16 pairs instead of complex FP32: 8-bit
 * significand, relative rounding of 2^-9 per entry, half the bytes the
 * matvec's near-field pass reads (an HBM-bound pass).  Meant for the
 * low-accuracy operator of an inner-outer preconditioner (Sec. 4), whose own
 * truncation error is far larger; enable = 0 returns to the FP32 entries
 * (both copies are kept).  Synchronises `stream` when it builds the copy.
 * Errors: FB_ERR_ARG (NULL, dense, FP64 or composite operator). */
FB_API fb_status fb_operator_set_near_bf16(fb_op* op, int enable, void* stream);

/* Profiling: device time of each pass of the staged RCR M2L (Sec. 3.3) of
 * every staged level of an FMM operator, one right-hand side, on the
 * operator's own expansion and staging buffers (their contents are
 * overwritten; apply the operator again before using its result).  Each
 * pass is launched alone between CUDA events on `stream`, once untimed and
 * three times timed (median).  ms: 4*13 doubles, ms[4l + 0..3] = pre-pass
 * (folded phased inputs; -1 where the tensor-core rotation pass folds them
 * itself), rotation, coaxial, back-rotation of level l (-1: level not
 * staged); form: 13 ints, 1 = passes on CUDA cores, 2 = rotation
 * passes on the tensor cores, 3 = passes in double-FP32 arithmetic, 5 =
 * rotation and coaxial passes on the tensor cores (0: not staged).  Synchronises the device.
 * Errors: FB_ERR_ARG (NULL argument, dense or composite operator). */
FB_API fb_status fb_operator_staged_pass_times(fb_op* op, void* stream, double* ms, int* form);
FB_API fb_status fb_set_device_wait_limit(long long limit, long long* previous);
FB_API fb_status fb_test_stall_device_waits(int enable);

/* Measured FMA throughput of the current device (TFLOP/s, 2 flops per FMA)
 * for FP32 and FP64 (either pointer may be NULL): the ALU ceilings of the
 * CUDA-core kernels.  Launches two short kernels per type and synchronises
 * the stream. */
FB_API fb_status fb_measure_alu_peaks(double* fp32_tflops, double* fp64_tflops, void* stream);

/* CUDA-graph replay: when enabled, every application of the FMM operator
 * (or of the learned preconditioner) inside the library replays a captured
 * graph of its kernels (one per number of right-hand sides) on staging
 * vectors, with one copy in and one copy out per call.  Captured graphs are
 * dropped when the translation method or autotuned forms change.  Kernels
 * that apply the operator through a graph must not be changed concurrently.
 * Errors: FB_ERR_ARG for NULL handles. */
FB_API fb_status fb_operator_use_graphs(fb_op* op, int enable);
FB_API fb_status fb_precond_use_graphs(fb_precond* pc, int enable);

/* Operator applied to nrhs right-hand sides at once (Y = Op X; X, Y:
 * nrhs x N complex, rhs-major, in memspace, distinct).  The FMM kernels take
 * every right-hand side in one launch (near-field, P2M/L2P and translation
 * operators read once per matvec; the stacked translation GEMMs are nrhs
 * times wider), which is how several source positions of one frequency share
 * a matvec.  1 <= nrhs <= FB_MAX_RHS.  The operator's expansion buffers grow
 * to nrhs sets on first use.  Errors: FB_ERR_ARG. */
#define FB_MAX_RHS 64

/* Autotuner of the translation passes of an FMM operator: for every level
 * it times on the device (median of 3, nrhs right-hand sides) the forms a
 * pass can take and installs the fastest per level (translation method
 * FB_TRANS_AUTO), for M2L and for the M2M/L2L passes into the level:
 *   - rotation-coaxial-rotation (Sec. 3.3) as per-pair tiles (orders whose
 *     per-pair working set fits one CTA's shared memory),
 *   - rotation-coaxial-rotation as staged batched GEMMs (the pairs of a
 *     level grouped by the polar angle of their translation direction for
 *     the rotations and by |t| for the coaxial step),
 *   - mixed precision only: the staged passes with their two rotation
 *     passes on the tensor cores (3xTF32 GEMMs of the folded real rotation
 *     blocks, one polar-angle group and degree at a time), and optionally
 *     the coaxial step too (complex blocks in real form per |t| and order),
 *   - FP64 only: the staged passes in double-FP32 arithmetic (each value
 *     an unevaluated sum of two FP32 numbers, a 48-bit significand, on the
 *     FP32 pipe), from order 16 on, and the per-pair tiles in the same
 *     arithmetic,
 *   - mixed precision only: the stacked tensor-core GEMM of composed
 *     matrices (3xTF32).
 * Tiles are timed below order 60, the staged passes from order 24 on (the
 * measured crossover lies between), with tensor-core rotations from order
 * 12 on, in double-FP32 from order 16 on; a level keeps at least one
 * candidate.
 * times: FB_TUNE_TIMES*13 doubles or NULL, times[FB_TUNE_TIMES l + 0..13] =
 * M2L RCR tiles, M2L tensor, M2M+L2L RCR tiles, M2M+L2L tensor, M2L RCR
 * staged, M2M+L2L RCR staged, M2L RCR staged with tensor-core rotations,
 * M2M+L2L RCR staged with tensor-core rotations, M2L RCR staged in
 * double-FP32, M2M+L2L RCR staged in double-FP32, M2L RCR tiles in
 * double-FP32, M2M+L2L RCR tiles in double-FP32, M2L RCR staged with
 * rotations and coaxial step on the tensor cores, the same for M2M+L2L, in
 * ms (-1: not a candidate); choice: 13 ints or NULL, bit 0 = M2L of level l on the tensor
 * cores, bit 1 = M2M/L2L into level l on the tensor cores, bit 2 = M2L of
 * level l by staged RCR, bit 3 = M2M/L2L into level l by staged RCR, bit 4 =
 * the staged M2L's rotations on the tensor cores (with bit 2), bit 5 = the
 * staged M2M/L2L's rotations on the tensor cores (with bit 3), bit 6 = the
 * staged M2L in double-FP32 (with bit 2), bit 7 = the staged M2M/L2L in
 * double-FP32 (with bit 3), bit 8 = the M2L tiles in double-FP32 (without
 * bit 2), bit 9 = the M2M/L2L tiles in double-FP32 (without bit 3), bit 10
 * = the staged M2L's coaxial step on the tensor cores too (with bit 4),
 * bit 11 = the same for M2M/L2L (with bit 5).
 * Rebuilds the operator's translation plans (synchronises the device).
 * Errors: FB_ERR_ARG. */
#define FB_TUNE_TIMES 14
FB_API fb_status fb_operator_autotune(fb_op* op, int nrhs, void* stream, double* times, int* choice);

/* Installs a per-level choice in the format the autotuner returns (13 ints,
 * bits as above), so that a tuned configuration can be saved and restored
 * without timing.  Levels whose per-pair RCR working set does not fit one
 * CTA run staged whatever bit 2/3 says.  Tensor-core bits (0, 1, 4, 5) need
 * a mixed-precision operator (so do 10, 11), double-FP32 bits (6-9) an FP64
 * FMM operator; bits 4 and 6 need bit 2, bits 5 and 7 need bit 3, bit 8
 * excludes bit 2 and bit 9 bit 3, bit 10 needs bit 4 and bit 11 bit 5.
 * Errors: FB_ERR_ARG. */
FB_API fb_status fb_operator_set_forms(fb_op* op, const int* choice, void* stream);
FB_API fb_status fb_operator_apply_multi(fb_op* op, const double* x, double* y, int nrhs, int memspace,
                                         void* stream);

/* Tracing: running total of kernel launches issued by the library in this
 * process (setup and apply); differences bracket a region of interest. */
FB_API long long fb_kernel_launches(void);

/* ------------------------------------------------------ right-hand side -- */

/* gamma_j = -(dpsi_in/dn - i k beta_j psi_in) at the centroids for a unit
 * monopole at src (Eq. sp7).  gamma: N complex in memspace. */
FB_API fb_status fb_gamma_monopole(const fb_mesh* mesh, double k, const double* src, double* gamma,
                            int memspace, void* stream);

/* ------------------------------------------------------- preconditioner -- */

/* Block-Jacobi right preconditioner for an FMM operator: the inverse of each
 * leaf's self block of the near-field matrix, factorised in FP64 on the
 * device (Gauss-Jordan with partial pivoting) and applied in the operator's
 * precision.  Errors: FB_ERR_ARG for dense operators, FB_ERR_BREAKDOWN for a
 * singular block. */
FB_API fb_status fb_precond_create(fb_op* op, int kind, void* stream, fb_precond** out);
FB_API void fb_precond_destroy(fb_precond* pc);

/* y = P x for a preconditioner handle (block Jacobi, or a learned network
 * over its block-Jacobi base).  x, y: N complex in memspace, distinct.
 * Errors: FB_ERR_ARG for NULL or overlapping arrays. */
FB_API fb_status fb_precond_apply(const fb_precond* pc, const double* x, double* y, int memspace, void* stream);

/* Inner-outer preconditioner (Sec. 4: flexible GMRES preconditioned by a few
 * GMRES iterations of a low-accuracy FMM): P(v) = d_k, the k-step GMRES
 * approximation (zero initial guess, one cycle, no restart) of
 * inner_op d = v, right-preconditioned by inner_pc (e.g. block Jacobi of
 * inner_op; may be NULL).  op is the outer operator the preconditioner is
 * used with (its size must match inner_op's); inner_op and inner_pc must
 * outlive it.  The inner steps run without host synchronisation.  P is not a
 * fixed linear map, which flexible GMRES admits.  Errors: FB_ERR_ARG. */
#define FB_PC_INNER 3

/* Indirect system (FB_OP_IBEM) helpers, device pointers, enqueued on `stream`.
 * fb_ibem_gammas_monopole: boundary data of Eq. (ibem4) for a monopole at
 *   src (3 doubles, host): gamma+ = d psi_in/dn - a+ psi_in and
 *   gamma- = -d psi_in/dn - a- psi_in at the centroids (N complex each).
 * fb_ibem_rhs: right-hand side of Eq. (ibem5), b = [L(gamma- + gamma+),
 *   (gamma+ - gamma-)/2 + L'(gamma- + gamma+)] (2N complex).
 * fb_ibem_field: scattered field off the surface, psi_sc = L[sigma] + M[mu]
 *   (Eq. ibem1) with mu = psi+ - psi- and sigma = gamma- + gamma+ - a- psi-
 *   - a+ psi+ (Eq. ibem4), from a solution x (2N) at nr receivers rcv
 *   (nr x 3 doubles, device), by direct summation into out (nr complex).
 *   The mesh admittance must still be the one the operator was built with.
 * Errors: FB_ERR_ARG if op is not FB_OP_IBEM. */
FB_API fb_status fb_ibem_gammas_monopole(fb_op* op, const double* src, double* gamma_p, double* gamma_m,
                                         void* stream);
FB_API fb_status fb_ibem_rhs(fb_op* op, const double* gamma_p, const double* gamma_m, double* b, void* stream);
FB_API fb_status fb_ibem_field(fb_op* op, const double* x, const double* gamma_p, const double* gamma_m,
                               const double* rcv, int64_t nr, double* out, void* stream);

/* Eq. dbem5 helpers (FB_OP_DBEM5), device pointers, N complex each:
 * fb_dbem5_rhs: b = 1/2 gamma + (1/zeta) M[zeta gamma];
 * fb_dbem5_psi: psi_sc = (q - gamma) / (i k beta) (the boundary condition).
 * Errors: FB_ERR_ARG if op is not FB_OP_DBEM5. */
FB_API fb_status fb_dbem5_rhs(fb_op* op, const double* gamma, double* b, void* stream);
FB_API fb_status fb_dbem5_psi(fb_op* op, const double* q, const double* gamma, double* psi, void* stream);

/* ------------------------------------------------------- broadband -- */

/* Image-source field of a shoebox room (Sec. 4, Eq. an2; images of Allen
 * and Berkley): out[m][r] = sum_j A_j e^{i k_m R_j}/(4 pi R_j) over the
 * source and its images, A_j the product of the wall reflection
 * coefficients met (R_walls: 6 complex, walls x=0, x=lx, y=0, y=ly, z=0,
 * z=lz), images with |A_j| < a_th dropped (Sec. 4 uses 1e-7; refused with
 * FB_ERR_ARG when that needs more than 64 image orders per axis; with
 * |R| >= 1, 20 orders per axis are kept).  room, src:
 * 3 doubles (host); k: nf wavenumbers (host); rcv: nr x 3 doubles and out:
 * nf x nr complex (device).  Synchronous.  Errors: FB_ERR_ARG. */
FB_API fb_status fb_image_field(const double* room, const double* src, const double* R_walls, double a_th,
                                const double* k, int nf, const double* rcv, int64_t nr, double* out, void* stream);

/* Time-domain response to the pulse of Eq. (an3), f(t) = delta(t - Dt) -
 * delta(t + Dt), from frequency-domain solutions psi (nf x nr complex,
 * device; unit monopole, time convention e^{-i omega t}) at frequencies
 * freqs (nf Hz, host, spacing df):
 *   out[n][r] = 2 df Re sum_m psi[m][r] 2 i sin(2 pi f_m Dt) e^{-i 2 pi f_m n dt},
 * n = 0..nt-1 (device, nt x nr doubles).  Synchronous.  Errors: FB_ERR_ARG. */
FB_API fb_status fb_pulse_synthesis(const double* psi, const double* freqs, int nf, int64_t nr, double df, double dt,
                                    int nt, double pulse_dt, double* out, void* stream);

/* Training-data helper for learned preconditioners: the first k+1 Arnoldi
 * vectors of the right-preconditioned Krylov space of A from start vector b
 * (the vectors a preconditioner receives in the first k iterations of
 * flexible GMRES), computed by k GMRES steps with CGS2.  b: N complex,
 * V: (k+1) x N complex, both device.  Errors: FB_ERR_ARG. */
FB_API fb_status fb_krylov_basis(fb_op* A, const fb_precond* pc, const double* b, int k, double* V, void* stream);
FB_API fb_status fb_precond_create_inner(fb_op* op, fb_op* inner_op, const fb_precond* inner_pc, int iters,
                                         void* stream, fb_precond** out);

/* Learned octree preconditioner (the variable preconditioner that flexible
 * GMRES admits, Sec. 3.1 / Sec. 4): z = BJ(v) + s ph N(conj(ph) v / s,
 * conj(ph) BJ(v) / s), where BJ is the block-Jacobi `base` of the same FMM
 * operator (which must outlive it), s = rms(v), ph the unit phase of sum v
 * (so z(a v) = a z(v) for complex a), and N a hierarchical network over the
 * octree (element encoder, leaf pooling, 3 coarser pooling levels, down-sweep
 * back to the leaves, element decoder; 64-wide features, SiLU).  Per element
 * it sees the two normalised inputs, the normal, the admittance and k times
 * the leaf side, so one parameter set can serve several frequencies and
 * wall materials (fb_learned_params moves it between operators).  Its matrix products run
 * on the tensor cores in BF16 with FP32 accumulation; parameters, gradients
 * and Adam moments are FP32.  Parameters start from a deterministic seeded
 * initialisation with a small output layer (close to block Jacobi).
 * The base may also be an inner-outer preconditioner of op (FB_PC_INNER);
 * the network then refines its output the same way.
 * Errors: FB_ERR_ARG if base is neither block Jacobi nor inner-outer of op. */
FB_API fb_status fb_precond_create_learned(fb_op* op, const fb_precond* base, uint64_t seed, void* stream,
                                           fb_precond** out);

/* Parameters of a learned preconditioner as FP32 host arrays: if host_in is
 * given they are replaced (*count must equal the parameter count); if
 * host_out is given they are copied out; *count receives the count. */
FB_API fb_status fb_learned_params(fb_precond* pc, float* host_out, const float* host_in, int64_t* count);

/* Training objectives for a pair (r, e) with A e = r:
 *   FB_LOSS_ERROR:    ||z(r) - e||^2 / ||e||^2
 *   FB_LOSS_RESIDUAL: ||A z(r) - r||^2 / ||r||^2   (default)
 * The residual objective is the quantity right-preconditioned GMRES reduces.
 * Its reverse pass through A uses a matrix-free stand-in for A^H: with one
 * collocation point per flat element the far-field kernels of M and L' (and
 * of L and its transpose) are the same function of the centroid pair, so
 *   A^H ~ I/2 + D conj(L') D^-1 + i k conj(beta) D conj(L) D^-1,  D = diag(area),
 * applied with single- and adjoint-double-layer FMM operators (mixed
 * precision, same tree and order rule) that the preconditioner builds on
 * first use.  The returned gradient is the pull-back through that stand-in. */
#define FB_LOSS_ERROR 0
#define FB_LOSS_RESIDUAL 1
FB_API fb_status fb_learned_set_objective(fb_precond* pc, int objective);

/* Training objective on a batch of residual/error pairs (R, E: npairs x N
 * complex, device, element order, pair q at offset q*N):
 *   loss = mean_q of the selected objective,  z(r) = BJ(r) + s ph N(...),
 * and its gradient w.r.t. the parameters (FP32, host, may be NULL). */
FB_API fb_status fb_learned_loss_and_grad(fb_precond* pc, const double* R, const double* E, int npairs,
                                          double* loss, float* grad_host, void* stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the batch; *loss (may be
 * NULL) receives the loss before the step. */
FB_API fb_status fb_learned_train_step(fb_precond* pc, const double* R, const double* E, int npairs, double lr,
                                       double* loss, void* stream);

/* ---------------------------------------------------------------- solve -- */

typedef struct {
    double tol;            /* target true relative residual ||b-Ax||/||b||     */
    int restart;           /* Krylov dimension m (>= 1)                        */
    int maxit;             /* max total inner iterations                       */
    int max_refine;        /* max outer refinement sweeps (>= 1)               */
    double inner_tol;      /* tolerance of each inner FGMRES (<= 0: tol)       */
    const fb_op* true_op;  /* operator of the true residual (NULL: A itself)   */
} fb_solver_opts;

typedef struct {
    int iters;             /* inner FGMRES iterations (= preconditioned matvecs) */
    int refinements;       /* outer sweeps run                                  */
    int true_matvecs;      /* applications of true_op                            */
    double est_relres;     /* last Arnoldi residual estimate                     */
    double true_relres;    /* ||b - true_op x|| / ||b|| at exit                  */
    int status;            /* FB_OK, FB_ERR_NOCONV, FB_ERR_BREAKDOWN, FB_ERR_NAN */
    int pc_fallbacks;      /* refinement sweeps in which a learned preconditioner
                              was replaced by its block-Jacobi base (see below)  */
} fb_solve_info;

/* Solves A x = b by flexible GMRES (right preconditioned, restarted, FP64
 * Arnoldi with classical Gram-Schmidt applied twice, Givens least squares),
 * wrapped in iterative refinement on the true residual of opts->true_op:
 *   r = b - T x;  stop if ||r||/||b|| <= tol;  solve A d = r to inner_tol;  x += d.
 * x0 = 0.  b, x: N complex in memspace.  The host reads one scalar per
 * Arnoldi step (the residual estimate).  Returns info->status as the status.
 * A learned preconditioner (fb_precond_create_learned) falls back to its
 * block-Jacobi base for the remaining sweeps when a sweep under it produced
 * a non-finite estimate (its correction is then discarded) or failed to halve
 * the true residual; info->pc_fallbacks counts such switches. */
FB_API fb_status fb_fgmres_solve(fb_op* A, fb_precond* pc, const double* b, double* x,
                          const fb_solver_opts* opts, fb_solve_info* info, int memspace,
                          void* stream);

/* nrhs systems A x_r = b_r with one operator (several source positions of
 * one frequency) solved by flexible GMRES in lockstep: each Arnoldi step
 * applies the preconditioner and the operator to the nrhs basis vectors in
 * one batched call (see fb_operator_apply_multi); every system keeps its own
 * Hessenberg matrix, restart cycles, convergence test and true-residual
 * refinement as in fb_fgmres_solve (no learned-to-block-Jacobi fallback
 * here).  b, x: nrhs x N complex, rhs-major, in memspace; info: nrhs entries
 * (may be NULL).  Returns FB_OK when every system converged, otherwise the
 * first failing system's status. */
FB_API fb_status fb_fgmres_solve_multi(fb_op* A, fb_precond* pc, const double* b, double* x, int nrhs,
                                       const fb_solver_opts* opts, fb_solve_info* info, int memspace,
                                       void* stream);

/* ------------------------------------------------------- batch scheduler -- */

/* One job of a batch: a mesh (admittance set) with its tree at one
 * wavenumber, and nsrc monopole sources (Eq. sp6).  Outputs: x (device,
 * nsrc x N complex, the surface field psi_sc of each source, Eq. dbem4),
 * info (host, nsrc entries, may be NULL), times and status. */
typedef struct fb_batch_job {
    const fb_mesh* mesh;
    const fb_tree* tree;
    double k;
    int nsrc;
    const double* src;        /* host, nsrc x 3                               */
    double* x;                /* device, nsrc x N complex                     */
    fb_solve_info* info;      /* host, nsrc entries, or NULL                  */
    double setup_ms;          /* out: operator + preconditioner (+ tuning)    */
    double solve_ms;          /* out: right-hand sides + batched solves       */
    int status;               /* out: FB_OK or the first failure              */
    int order;                /* out: position in the execution order         */
} fb_batch_job;

typedef struct fb_batch_opts {
    double tol;               /* true relative residual (FP64 judge)          */
    int restart, maxit;       /* FGMRES; <= 0 selects 40 / 3000               */
    double d0;                /* order rule (<= 0: 6)                         */
    int pmin;                 /* order rule (<= 0: 12)                        */
    int autotune;             /* 1: autotune the mixed operator per job (one
                                 timed run per candidate form)              */
    int max_rhs;              /* sources per batched solve (<= 0: 8)          */
    int fp64_judge;           /* 1: true residual by the FP64 FMM operator    */
    int lookahead;            /* 1: build job i+1 while job i solves          */
    int inner_iters;          /* > 0: inner-outer preconditioner (Sec. 4) with
                                 this many GMRES steps on a low-accuracy mixed
                                 FMM (all sources of a batch in lockstep,
                                 replayed as captured graphs); 0: block Jacobi */
    double inner_d0;          /* order rule of the inner operator (<= 0: 0.5) */
    int inner_pmin;           /* (<= 0: 2)                                    */
} fb_batch_opts;

/* Runs a batch (a frequency sweep with several sources per frequency, as in
 * the paper's experiments, Sec. 4): jobs in order of decreasing predicted
 * cost (sources x N x p_leaf^2); per job the mixed FMM operator, block
 * Jacobi (or the inner-outer preconditioner on a low-accuracy FMM), the FP64
 * operators (b = L gamma, true residual) and, if asked, the autotuned
 * translation forms are built once, then the job's sources are solved
 * max_rhs at a time by fb_fgmres_solve_multi.  With lookahead a host
 * thread builds the next job on a second stream while the current one
 * solves.  Operators are released after each job.  Returns FB_OK when every
 * solve converged, else the first failing status (per-job status set). */
FB_API fb_status fb_batch_solve(fb_batch_job* jobs, int njobs, const fb_batch_opts* opts);

/* Partition of independent jobs (the (frequency, source) solves of a sweep,
 * Sec. 4: every frequency and source is solved on its own, so a sweep
 * shards over GPUs without any exchange) across nranks ranks: largest cost
 * first, each job to the least loaded rank so far (ties: lower job index
 * first, lower rank).  cost: njobs finite values >= 0 (host; e.g. the
 * predicted time, N x iterations); owner: njobs ints (host, out); load:
 * nranks doubles (host, out, may be NULL).  Host only: launches nothing and
 * needs no GPU.  Errors: FB_ERR_ARG. */
FB_API fb_status fb_batch_partition(const double* cost, int njobs, int nranks, int* owner, double* load);

/* ------------------------------------------------------------ receivers -- */

/* Field at interior points by Green's identity (Eq. dbem1):
 *   psi(r) = psi_in(r) + L[gamma + i k beta psi_sc](r) - M[psi_sc](r)
 * with the same element rule as the operators (direct sum over elements).
 * src: 3 doubles on the host, or NULL (no incident field added).
 * psi_sc, gamma: N complex; rcv: nr x 3 doubles; out: nr complex; these
 * four in memspace. */
FB_API fb_status fb_eval_field(const fb_mesh* mesh, double k, const double* psi_sc, const double* gamma,
                        const double* src, const double* rcv, int64_t nr, double* out,
                        int memspace, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FMMBEM_H */
