// Mesh geometry, the dense FP64 collocation operator, the monopole boundary
// data (Eq. sp7) and direct receiver evaluation (Eq. dbem1).
#include <cstring>

#include "quad.cuh"

// Order-preserving map of doubles onto unsigned 64-bit integers (for
// atomicMin/atomicMax over doubles).
__device__ __forceinline__ unsigned long long ord_key(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
static double ord_val(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
    double d;
    memcpy(&d, &b, 8);
    return d;
}

__device__ __forceinline__ double len_rn(double dx, double dy, double dz) {
    // sqrt((dx*dx + dy*dy) + dz*dz) with no fused operations
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__global__ void k_mesh_geom(int64_t n, const double* __restrict__ V, const int32_t* __restrict__ T,
                            double* buf, unsigned long long* stats, int* bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double* cx = buf;
    double* cy = buf + n;
    double* cz = buf + 2 * n;
    double* nx = buf + 3 * n;
    double* ny = buf + 4 * n;
    double* nz = buf + 5 * n;
    double* ar = buf + 6 * n;
    double* A = buf + 7 * n;   // ax ay az bx by bz qx qy qz : 9 arrays
    double* G = buf + 16 * n;  // gx gy gz : 3 arrays of 3n
    int i0 = T[3 * i], i1 = T[3 * i + 1], i2 = T[3 * i + 2];
    double a[3], b[3], c[3];
    for (int d = 0; d < 3; ++d) {
        a[d] = V[3 * i0 + d];
        b[d] = V[3 * i1 + d];
        c[d] = V[3 * i2 + d];
    }
    // centroid ((a + b) + c) / 3, rounded exactly as written
    cx[i] = __ddiv_rn(__dadd_rn(__dadd_rn(a[0], b[0]), c[0]), 3.0);
    cy[i] = __ddiv_rn(__dadd_rn(__dadd_rn(a[1], b[1]), c[1]), 3.0);
    cz[i] = __ddiv_rn(__dadd_rn(__dadd_rn(a[2], b[2]), c[2]), 3.0);
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    double dbl = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(dbl > 0.0)) {
        atomicExch(bad, 1);
        dbl = 1.0;
    }
    nx[i] = cr[0] / dbl;
    ny[i] = cr[1] / dbl;
    nz[i] = cr[2] / dbl;
    ar[i] = 0.5 * dbl;
    for (int d = 0; d < 3; ++d) {
        A[d * n + i] = a[d];
        A[(3 + d) * n + i] = b[d];
        A[(6 + d) * n + i] = c[d];
    }
    // 3-point degree-2 rule: barycentric (2/3,1/6,1/6) and permutations
    const double hi = 2.0 / 3.0, lo = 1.0 / 6.0;
    for (int q = 0; q < 3; ++q) {
        double w0 = (q == 0) ? hi : lo, w1 = (q == 1) ? hi : lo, w2 = (q == 2) ? hi : lo;
        for (int d = 0; d < 3; ++d) G[d * 3 * n + 3 * i + q] = w0 * a[d] + w1 * b[d] + w2 * c[d];
    }
    double l0 = len_rn(b[0] - a[0], b[1] - a[1], b[2] - a[2]);
    double l1 = len_rn(c[0] - b[0], c[1] - b[1], c[2] - b[2]);
    double l2 = len_rn(a[0] - c[0], a[1] - c[1], a[2] - c[2]);
    double me = fmax(fmax(l0, l1), l2);
    atomicMax(&stats[0], ord_key(me));
    for (int d = 0; d < 3; ++d) {
        double mn = fmin(fmin(a[d], b[d]), c[d]);
        double mx = fmax(fmax(a[d], b[d]), c[d]);
        atomicMin(&stats[1 + d], ord_key(mn));
        atomicMax(&stats[4 + d], ord_key(mx));
    }
}

static void set_geom_ptrs(fb_mesh* m) {
    int64_t n = m->n;
    double* b = m->buf;
    Geom& g = m->g;
    g.n = n;
    g.cx = b; g.cy = b + n; g.cz = b + 2 * n;
    g.nx = b + 3 * n; g.ny = b + 4 * n; g.nz = b + 5 * n;
    g.area = b + 6 * n;
    g.ax = b + 7 * n; g.ay = b + 8 * n; g.az = b + 9 * n;
    g.bx = b + 10 * n; g.by = b + 11 * n; g.bz = b + 12 * n;
    g.qx = b + 13 * n; g.qy = b + 14 * n; g.qz = b + 15 * n;
    g.gx = b + 16 * n; g.gy = b + 19 * n; g.gz = b + 22 * n;
    g.beta = m->beta;
}

fb_status fb_mesh_create_impl(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                              cudaStream_t s, fb_mesh** out) {
    if (!out) return fb_fail(FB_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!verts || !tris || nv < 3 || nt < 1) return fb_fail(FB_ERR_ARG, "empty mesh");
    if (nt > (int64_t)1 << 30) return fb_fail(FB_ERR_ARG, "too many elements");
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (tris[i] < 0 || tris[i] >= nv) return fb_fail(FB_ERR_ARG, "triangle index out of range");
    fb_mesh* m = new fb_mesh();
    cudaGetDevice(&m->dev);
    m->n = nt;
    double* dV = nullptr;
    int32_t* dT = nullptr;
    unsigned long long* dstat = nullptr;
    int* dbad = nullptr;
    auto cleanup = [&]() { dfree(dV); dfree(dT); dfree(dstat); dfree(dbad); };
    fb_status st = FB_OK;
    if ((st = dalloc(&m->buf, (size_t)25 * nt)) || (st = dalloc(&m->beta, (size_t)nt)) ||
        (st = dalloc(&dV, (size_t)3 * nv)) || (st = dalloc(&dT, (size_t)3 * nt)) ||
        (st = dalloc(&dstat, 7)) || (st = dalloc(&dbad, 1))) {
        cleanup();
        fb_mesh_destroy(m);
        return st;
    }
    set_geom_ptrs(m);
    unsigned long long init[7];
    init[0] = 0ULL;
    for (int d = 0; d < 3; ++d) { init[1 + d] = ~0ULL; init[4 + d] = 0ULL; }
    cudaMemcpyAsync(dV, verts, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dT, tris, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dstat, init, sizeof(init), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(dbad, 0, sizeof(int), s);
    cudaMemsetAsync(m->beta, 0, sizeof(cd) * nt, s);
    k_mesh_geom<<<div_up(nt, 256), 256, 0, s>>>(nt, dV, dT, m->buf, dstat, dbad);
    unsigned long long hs[7];
    int hbad = 0;
    cudaMemcpyAsync(hs, dstat, sizeof(hs), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        fb_mesh_destroy(m);
        return fb_fail(FB_ERR_CUDA, std::string("mesh geometry: ") + cudaGetErrorString(e));
    }
    if (hbad) {
        fb_mesh_destroy(m);
        return fb_fail(FB_ERR_ARG, "degenerate (zero-area) triangle");
    }
    m->max_edge = ord_val(hs[0]);
    m->rc = 1.5 * m->max_edge;
    for (int d = 0; d < 3; ++d) {
        m->lo[d] = ord_val(hs[1 + d]);
        m->hi[d] = ord_val(hs[4 + d]);
    }
    *out = m;
    return FB_OK;
}

// ------------------------------------------------------------- dense ----
__global__ void k_dense_fill(Geom g, int kind, double k, double rc, cd* __restrict__ A) {
    int64_t n = g.n;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    if (j >= n) return;
    A[i * n + j] = op_entry(g, kind, i, j, k, rc);
}

// y = A x, one warp per row, complex128.
__global__ void k_dense_gemv(int64_t n, const cd* __restrict__ A, const cd* __restrict__ x,
                             cd* __restrict__ y) {
    int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    const cd* a = A + row * n;
    cd acc = mk(0.0, 0.0);
    for (int64_t j = lane; j < n; j += 32) cmac(acc, a[j], x[j]);
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) y[row] = acc;
}

fb_status fb_dense_create(fb_op* op, cudaStream_t s) {
    int64_t n = op->n;
    if (n > 60000) return fb_fail(FB_ERR_ARG, "dense operator limited to N <= 60000");
    FB_CHECK(dalloc(&op->dense, (size_t)n * n));
    dim3 grid(div_up(n, 128), (unsigned)n);
    k_dense_fill<<<grid, 128, 0, s>>>(op->mesh->g, op->kind, op->k, op->mesh->rc, op->dense);
    FB_LAUNCH_CHECK();
    return FB_OK;
}

fb_status fb_dense_apply(const fb_op* op, const cd* x, cd* y, cudaStream_t s) {
    int64_t n = op->n;
    k_dense_gemv<<<div_up(n * 32, 256), 256, 0, s>>>(n, op->dense, x, y);
    FB_LAUNCH_CHECK();
    fb_count_launch();
    return FB_OK;
}

// ------------------------------------------------------ boundary data ----
__global__ void k_gamma_monopole(Geom g, double k, double sx, double sy, double sz, cd* gam) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    V3 r = v3(g.cx[i] - sx, g.cy[i] - sy, g.cz[i] - sz);
    double R = norm(r);
    double s, c;
    sincos(k * R, &s, &c);
    cd E = mk(c, s);
    cd psi = (FB_INV4PI / R) * E;
    cd dfac = (FB_INV4PI / (R * R * R)) * (E * mk(-1.0, k * R));
    double rn = r.x * g.nx[i] + r.y * g.ny[i] + r.z * g.nz[i];
    cd dn = rn * dfac;
    cd b = g.beta[i];
    cd ikb = mk(-k * b.im, k * b.re);
    cd v = dn - ikb * psi;
    gam[i] = mk(-v.re, -v.im);
}

fb_status fb_gamma_impl(const fb_mesh* m, double k, const double* src, cd* gam, cudaStream_t s) {
    k_gamma_monopole<<<div_up(m->n, 256), 256, 0, s>>>(m->g, k, src[0], src[1], src[2], gam);
    FB_LAUNCH_CHECK();
    return FB_OK;
}

// ----------------------------------------------------------- receivers ----
__global__ void k_eval_field(Geom g, double k, double rc, const cd* __restrict__ psi,
                             const cd* __restrict__ gam, const double* __restrict__ rcv,
                             int has_src, double sx, double sy, double sz, cd* out) {
    int64_t r = blockIdx.x;
    V3 x = v3(rcv[3 * r], rcv[3 * r + 1], rcv[3 * r + 2]);
    V3 zero = v3(0, 0, 0);
    cd acc = mk(0.0, 0.0);
    for (int64_t j = threadIdx.x; j < g.n; j += blockDim.x) {
        Entry e = pair_entry(g, j, x, zero, false, k, rc);
        cd b = g.beta[j];
        cd ikb = mk(-k * b.im, k * b.re);
        cd q = gam[j] + ikb * psi[j];
        acc = acc + e.L * q - e.M * psi[j];
    }
    __shared__ double sre[32], sim[32];
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sre[w] = acc.re; sim[w] = acc.im; }
    __syncthreads();
    if (threadIdx.x == 0) {
        cd t = mk(0.0, 0.0);
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = t + mk(sre[i], sim[i]);
        if (has_src) {
            V3 d = x - v3(sx, sy, sz);
            double R = norm(d);
            double sn, cs;
            sincos(k * R, &sn, &cs);
            t = t + (FB_INV4PI / R) * mk(cs, sn);
        }
        out[r] = t;
    }
}

fb_status fb_eval_impl(const fb_mesh* m, double k, const cd* psi, const cd* gam, const double* src,
                       const double* rcv, int64_t nr, cd* out, cudaStream_t s) {
    if (nr <= 0) return FB_OK;
    k_eval_field<<<(unsigned)nr, 256, 0, s>>>(m->g, k, m->rc, psi, gam, rcv, src ? 1 : 0,
                                             src ? src[0] : 0.0, src ? src[1] : 0.0,
                                             src ? src[2] : 0.0, out);
    FB_LAUNCH_CHECK();
    return FB_OK;
}

void fb_mesh_free(fb_mesh* m) {
    if (!m) return;
    dfree(m->buf);
    dfree(m->beta);
    dfree(m->beta_p);
    delete m;
}
