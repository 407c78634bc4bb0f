// FMM operator setup, all in FP64 on the device (Sec. 3.3):
//   near-field entries of touching leaves (closed-form singular parts),
//   per-leaf P2M / L2P operators, coaxial coefficients by the recursions of
//   Sec. 3.3.1, rotation blocks, and the composed RCR translation matrices
//   (rotation, coaxial translation, back-rotation) for M2M, M2L and L2L.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "sph.cuh"

int fb_order_rule(double k, double delta, double d0, int pmin) {
    double kr = k * std::sqrt(3.0) / 2.0 * delta;
    double p = std::ceil(kr + 1.8 * std::pow(d0, 2.0 / 3.0) * std::pow(kr, 1.0 / 3.0));
    return std::max(pmin, (int)p);
}

__global__ void k_d2f(const cd* a, cf* b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = to_f(a[i]);
}

// ------------------------------------------------------------ near field ----
__global__ void k_near_fill(Geom g, int kind, double k, double rc, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ ucnt,
                            const int32_t* __restrict__ ulist, const int64_t* __restrict__ nf_off,
                            const int32_t* __restrict__ nf_ncol, cd* __restrict__ out) {
    int t = blockIdx.x;
    __shared__ int s_start[FB_ULIST], s_cum[FB_ULIST + 1];
    int nu = ucnt[t];
    if (threadIdx.x == 0) {
        s_cum[0] = 0;
        for (int i = 0; i < nu; ++i) {
            int s = ulist[(int64_t)t * FB_ULIST + i];
            s_start[i] = leaf_start[s];
            s_cum[i + 1] = s_cum[i] + (leaf_start[s + 1] - leaf_start[s]);
        }
    }
    __syncthreads();
    int r0 = leaf_start[t];
    int nr = leaf_start[t + 1] - r0;
    int K = nf_ncol[t];
    int64_t base = nf_off[t];
    for (int64_t e = threadIdx.x; e < (int64_t)nr * K; e += blockDim.x) {
        int r = (int)(e / K), c = (int)(e % K);
        int u = 0;
        while (s_cum[u + 1] <= c) ++u;
        int col_pos = s_start[u] + (c - s_cum[u]);
        int64_t i = perm[r0 + r], j = perm[col_pos];
        out[base + e] = op_entry(g, kind, i, j, k, rc);
    }
}

// max |z| over a complex array (non-negative doubles compare as integers)
__global__ void k_absmax(const cd* a, int64_t n, double* out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = sqrt(abs2(a[i]));
        if (!(v <= 1e300)) v = 1e300;   // inf and NaN count as out of range
        m = fmax(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax((unsigned long long*)out, (unsigned long long)__double_as_longlong(m));
}

// ----------------------------------------------------------- P2M / L2P ----
// W[pos][nm] = ik A_j sum_q w_q [dip n_j.grad R_n^{-m}(y_q - c) + mono_j R_n^{-m}(y_q - c)]
// V[pos][nm] = R_n^m(x_i - c)  (L' : n_i . grad R_n^m(x_i - c))
__global__ void k_p2m_l2p(Geom g, int kind, double k, int P, int64_t n, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ leaf_of, const double* __restrict__ centers,
                          double* scratch, int scratch_stride, cd* __restrict__ W, cd* __restrict__ V) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    double* sc = scratch + tid * (int64_t)scratch_stride;
    int Pp1 = P + 1;
    cd* Rv = (cd*)sc;                                  // (P+1)^2 complex
    double* wrk = sc + 2 * Pp1 * Pp1;
    for (int64_t pos = tid; pos < n; pos += nthreads) {
        int64_t e = perm[pos];
        int b = leaf_of[pos];
        V3 c = v3(centers[3 * b], centers[3 * b + 1], centers[3 * b + 2]);
        V3 nj = v3(g.nx[e], g.ny[e], g.nz[e]);
        cd* Wr = W + pos * (int64_t)P * P;
        cd* Vr = V + pos * (int64_t)P * P;
        for (int q = 0; q < P * P; ++q) Wr[q] = mk(0.0, 0.0);
        cd mono = mk(0.0, 0.0);
        double dip = 0.0;
        if (kind == FB_OP_L || kind == FB_OP_LP) mono = mk(1.0, 0.0);
        if (kind == FB_OP_M || kind == FB_OP_MP) dip = 1.0;
        if (kind == FB_OP_A) {
            cd b = g.beta[e];
            mono = mk(k * b.im, -k * b.re);   // -i k beta
            dip = 1.0;
        }
        // ik A_j w_q, w_q = 1/3
        cd pref = mk(0.0, k * g.area[e] / 3.0);
        for (int qp = 0; qp < 3; ++qp) {
            V3 y = v3(g.gx[3 * e + qp], g.gy[3 * e + qp], g.gz[3 * e + qp]);
            regular_all(Pp1, k, y - c, wrk, Rv);
            for (int nn = 0; nn < P; ++nn)
                for (int m = -nn; m <= nn; ++m) {
                    cd v = mono * Rv[nm_idx(nn, -m)];
                    if (dip != 0.0) v = v + ndot_grad_regular(Rv, P, k, nj, nn, -m);
                    Wr[nm_idx(nn, m)] = Wr[nm_idx(nn, m)] + pref * v;
                }
        }
        V3 x = v3(g.cx[e], g.cy[e], g.cz[e]);
        regular_all(Pp1, k, x - c, wrk, Rv);
        if (kind == FB_OP_LP || kind == FB_OP_MP) {
            V3 ni = nj;
            for (int nn = 0; nn < P; ++nn)
                for (int m = -nn; m <= nn; ++m) Vr[nm_idx(nn, m)] = ndot_grad_regular(Rv, P, k, ni, nn, m);
        } else {
            for (int q = 0; q < P * P; ++q) Vr[q] = Rv[q];
        }
    }
}

// ------------------------------------------------------------- coaxial ----
// (E|F)^m_{n'n}(tau), m < p, n', n < p, by the algorithm of Sec. 3.3.1:
//  1 seeds (E|F)^0_{n',0} = (-1)^{n'} sqrt(2n'+1) f_{n'}(k tau), n' < 2p   (Eq. shft1)
//  2 sectorial (E|F)^{m+1}_{n',m+1} up in m                                (Eq. shft2)
//  k tau < 1: 3 propagation in n for n' >= n (Eq. shft5), 4 symmetry
//  k tau >= 1: 3.1 zonal (Eq. shft7), 3.2 diagonal + two subdiagonals
//     (Eq. shft8; third formula with b_n^{-m-1}), 3 propagation in n'
//     (Eq. shift6), 4 symmetry.
// One thread per coefficient set.  out: [m][n'][n] with stride p (p^3 complex).
struct CoaxSet {
    double ktau;
    int p;
    int kind;    // 0 = S|R, 1 = R|R
    int64_t out_off;
};

__global__ void k_coaxial(const CoaxSet* sets, int nsets, cd* scratch, int64_t scratch_stride,
                          double* fscratch, int64_t fstride, cd* out) {
    int sid = blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= nsets) return;
    CoaxSet cs = sets[sid];
    int p = cs.p;
    int W2 = 2 * p + 2, W3 = p + 2;
    cd* X = scratch + sid * scratch_stride;
    auto at = [&](int m, int n1, int n) -> cd& { return X[((int64_t)m * W2 + n1) * W3 + n]; };
    for (int64_t i = 0; i < (int64_t)(p + 1) * W2 * W3; ++i) X[i] = mk(0.0, 0.0);
    int P2 = 2 * p;
    double* fj = fscratch + sid * fstride;
    double* fy = fj + P2 + 1;
    sph_bessel_j(P2 - 1, cs.ktau, fj);
    if (cs.kind == 0) sph_bessel_y(P2 - 1, cs.ktau, fy);
    for (int n1 = 0; n1 < P2; ++n1) {
        double sg = (n1 & 1) ? -1.0 : 1.0;
        double s = sg * sqrt(2.0 * n1 + 1.0);
        at(0, n1, 0) = cs.kind == 0 ? mk(s * fj[n1], s * fy[n1]) : mk(s * fj[n1], 0.0);
    }
    for (int m = 0; m < p - 1; ++m)
        for (int n1 = m + 1; n1 < P2 - 1 - m; ++n1)
            at(m + 1, n1, m + 1) = (1.0 / coef_b(m + 1, -m - 1)) *
                                   (coef_b(n1, -m - 1) * at(m, n1 - 1, m) - coef_b(n1 + 1, m) * at(m, n1 + 1, m));
    if (cs.ktau < 1.0) {
        for (int m = 0; m < p; ++m)
            for (int n = m; n < p - 1; ++n)
                for (int n1 = n; n1 < 2 * p - 1 - n; ++n1)
                    at(m, n1, n + 1) = (1.0 / coef_a(n, m)) *
                                       (coef_a(n - 1, m) * (n >= 1 ? at(m, n1, n - 1) : mk(0.0, 0.0)) -
                                        coef_a(n1, m) * at(m, n1 + 1, n) +
                                        coef_a(n1 - 1, m) * (n1 >= 1 ? at(m, n1 - 1, n) : mk(0.0, 0.0)));
    } else {
        for (int n = 0; n < p - 1; ++n)
            for (int n1 = n + 1; n1 < 2 * p - n - 2; ++n1)
                at(0, n1, n + 1) = (1.0 / coef_a(n, 0)) *
                                   (coef_a(n - 1, 0) * (n >= 1 ? at(0, n1, n - 1) : mk(0.0, 0.0)) -
                                    coef_a(n1, 0) * at(0, n1 + 1, n) + coef_a(n1 - 1, 0) * at(0, n1 - 1, n));
        for (int m = 0; m < p - 2; ++m)
            for (int n = m + 1; n < p - 1; ++n) {
                if (n >= m + 2)
                    at(m + 1, n + 1, n) = (1.0 / coef_b(n + 1, -m - 1)) *
                                          (coef_b(n + 1, m) * at(m, n + 1, n) + coef_b(n, -m - 1) * at(m, n, n - 1) -
                                           coef_b(n, m) * at(m + 1, n, n - 1));
                at(m + 1, n + 1, n + 1) = (1.0 / coef_b(n + 1, -m - 1)) *
                                          (coef_b(n, m) * at(m + 1, n + 1, n - 1) - coef_b(n + 2, m) * at(m, n + 2, n) +
                                           coef_b(n + 1, -m - 1) * at(m, n, n));
                if (n >= m + 2)
                    at(m + 1, n + 2, n) = (1.0 / coef_b(n + 2, -m - 1)) *
                                          (coef_b(n + 1, m) * at(m + 1, n, n) - coef_b(n + 1, m) * at(m, n + 1, n + 1) +
                                           coef_b(n, -m - 1) * at(m, n + 1, n - 1));
            }
        for (int m = 1; m < p; ++m)
            for (int n1 = m + 3; n1 < p - 1; ++n1)
                for (int n = m + 1; n < n1 - 1; ++n)
                    at(m, n1 + 1, n) = (1.0 / coef_a(n1, m)) *
                                       (coef_a(n - 1, m) * at(m, n1, n - 1) - coef_a(n, m) * at(m, n1, n + 1) +
                                        coef_a(n1 - 1, m) * at(m, n1 - 1, n));
    }
    cd* o = out + cs.out_off;
    for (int m = 0; m < p; ++m)
        for (int n1 = 0; n1 < p; ++n1)
            for (int n = 0; n < p; ++n) {
                cd v = mk(0.0, 0.0);
                if (n1 >= m && n >= m) {
                    if (n1 >= n) v = at(m, n1, n);
                    else {
                        v = at(m, n, n1);
                        if ((n + n1) & 1) v = mk(-v.re, -v.im);
                    }
                }
                o[((int64_t)m * p + n1) * p + n] = v;
            }
}

// ------------------------------------------------------------ rotations ----
// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_nq.
__global__ void k_gauss_legendre(int nq, double* x, double* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    double z = cos(FB_PI * (i + 0.75) / (nq + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= nq; ++j) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = nq * (z * p1 - p2) / (z * z - 1.0);
        double dz = p1 / pp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    double p1 = 1.0, p2 = 0.0;
    for (int j = 1; j <= nq; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
    }
    pp = nq * (z * p1 - p2) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
}

// Rotation Q = R_y(-theta) R_z(-phi) maps direction d to +z; Q^T y = R_z(phi) R_y(theta) y.
__device__ inline V3 rotT(V3 d, V3 y) {
    double rho = norm(d);
    double th = acos(fmax(-1.0, fmin(1.0, d.z / rho)));
    double ph = atan2(d.y, d.x);
    double ct, st, cp, sp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    // R_y(theta) y
    V3 a = v3(ct * y.x + st * y.z, y.y, -st * y.x + ct * y.z);
    // R_z(phi) a
    return v3(cp * a.x - sp * a.y, sp * a.x + cp * a.y, a.z);
}

// Y_n^m at the product grid (GL in cos theta x uniform phi) rotated by Q_d^T,
// for a batch of directions.  out[(dir * npts + q) * P^2 + nm]
__global__ void k_rot_grid(const double* dirs, int ndir, int identity, int P, int nq, int nphi,
                           const double* glx, double* scratch, int sstride, cd* out) {
    int npts = nq * nphi;
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= (int64_t)ndir * npts) return;
    int d = (int)(tid / npts), q = (int)(tid % npts);
    int it = q / nphi, ip = q % nphi;
    double ct = glx[it], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * FB_PI * ip / nphi;
    double sp, cp;
    sincos(ph, &sp, &cp);
    V3 y = v3(st * cp, st * sp, ct);
    V3 dv = v3(dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]);
    V3 u = identity ? y : rotT(dv, y);
    double un = norm(u);
    ylm_unit(P, u.x / un, u.y / un, u.z / un, scratch + tid * (int64_t)sstride, out + tid * (int64_t)P * P);
}

// D^n_{mu,m} = sum_q W_q conj(Y_n^mu(y_q)) Y_n^m(Q^T y_q) for the batch.
// grid: (entry chunk, n, dir); out[dir_global][rot_off(n) + (mu+n)(2n+1) + (m+n)]
__global__ void k_rot_project(const cd* Yg, const cd* Yr, int ndir, int P, int nq, int nphi,
                              const double* glw, int dir0, cd* out) {
    int n = blockIdx.y;
    int d = blockIdx.z;
    int w = 2 * n + 1;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= w * w) return;
    int mu = e / w - n, m = e % w - n;
    int npts = nq * nphi;
    double wphi = 2.0 * FB_PI / nphi;
    cd acc = mk(0.0, 0.0);
    const cd* yr = Yr + (int64_t)d * npts * P * P;
    for (int q = 0; q < npts; ++q) {
        double wq = glw[q / nphi] * wphi;
        cd a = Yg[(int64_t)q * P * P + nm_idx(n, mu)];
        cd b = yr[(int64_t)q * P * P + nm_idx(n, m)];
        cmacc(acc, wq * a, b);
    }
    int64_t rot_off = (int64_t)n * (2 * n - 1) * (2 * n + 1) / 3;
    int64_t per_dir = (int64_t)P * (2 * P - 1) * (2 * P + 1) / 3;
    out[(int64_t)(dir0 + d) * per_dir + rot_off + e] = acc;
}

// --------------------------------------------------------- composition ----
// T[(n',m'),(n,m)] = sum_{|mu| <= min(n',n)} conj(D^{n'}_{mu,m'}) C^{|mu|}_{n',n} D^n_{mu,m}
__global__ void k_compose(const ComposeJob* jobs, const cd* __restrict__ rot, int Prot,
                          const cd* __restrict__ coax, cd* __restrict__ T) {
    ComposeJob jb = jobs[blockIdx.y];
    int rows = jb.p_out * jb.p_out, cols = jb.p_in * jb.p_in;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * cols) return;
    int r = (int)(e / cols), c = (int)(e % cols);
    int n1 = (int)sqrt((double)r);
    while (n1 * n1 > r) --n1;
    while ((n1 + 1) * (n1 + 1) <= r) ++n1;
    int m1 = r - n1 * n1 - n1;
    int n = (int)sqrt((double)c);
    while (n * n > c) --n;
    while ((n + 1) * (n + 1) <= c) ++n;
    int m = c - n * n - n;
    const cd* D = rot + jb.rot_off;
    int64_t o1 = (int64_t)n1 * (2 * n1 - 1) * (2 * n1 + 1) / 3;
    int64_t o0 = (int64_t)n * (2 * n - 1) * (2 * n + 1) / 3;
    int w1 = 2 * n1 + 1, w0 = 2 * n + 1;
    int mn = min(n1, n);
    cd acc = mk(0.0, 0.0);
    for (int mu = -mn; mu <= mn; ++mu) {
        cd d1 = D[o1 + (int64_t)(mu + n1) * w1 + (m1 + n1)];
        cd d0 = D[o0 + (int64_t)(mu + n) * w0 + (m + n)];
        cd cc = coax[jb.coax_off + ((int64_t)abs(mu) * jb.pc + n1) * jb.pc + n];
        cmacc(acc, d1, cc * d0);
    }
    T[jb.t_off + e] = acc;
}

// Composes the translation matrices of the listed jobs that are not built
// yet (T = D_out^H C D_in in FP64), plus their FP32 copies when present.
fb_status fb_compose_jobs(fb_op* op, const std::vector<int>& which, cudaStream_t s) {
    std::vector<ComposeJob> todo;
    for (int j : which) {
        if (op->h_jobs[j].t_off < 0)
            return fb_fail(FB_ERR_ARG, "composed translation matrices exist only up to order " +
                                           std::to_string(FB_COMPOSE_PMAX));
        if (!op->job_done[j]) todo.push_back(op->h_jobs[j]);
    }
    if (todo.empty()) return FB_OK;
    if (!op->T64) FB_CHECK(dalloc(&op->T64, std::max<int64_t>(op->T_count, 1)));
    if (op->prec == FB_PREC_MIXED_FMM && !op->T32) FB_CHECK(dalloc(&op->T32, std::max<int64_t>(op->T_count, 1)));
    ComposeJob* djobs = nullptr;
    FB_CHECK(dalloc(&djobs, todo.size()));
    FB_CUDA(cudaMemcpyAsync(djobs, todo.data(), sizeof(ComposeJob) * todo.size(), cudaMemcpyHostToDevice, s));
    int64_t maxe = 0;
    for (auto& jb : todo) maxe = std::max<int64_t>(maxe, (int64_t)jb.p_out * jb.p_out * jb.p_in * jb.p_in);
    for (size_t j0 = 0; j0 < todo.size(); j0 += 65535) {
        int nj = (int)std::min<size_t>(65535, todo.size() - j0);
        dim3 grid(div_up(maxe, 256), nj);
        k_compose<<<grid, 256, 0, s>>>(djobs + j0, op->rot64, op->Prot, op->coax64, op->T64);
    }
    if (op->T32)
        for (auto& jb : todo) {
            int64_t cnt = (int64_t)jb.p_out * jb.p_out * jb.p_in * jb.p_in;
            k_d2f<<<div_up(cnt, 256), 256, 0, s>>>(op->T64 + jb.t_off, op->T32 + jb.t_off, cnt);
        }
    FB_LAUNCH_CHECK();
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(djobs);
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("composition: ") + cudaGetErrorString(e));
    for (int j : which) op->job_done[j] = 1;
    return FB_OK;
}

fb_status fb_compose_all(fb_op* op, cudaStream_t s) {
    std::vector<int> all;
    for (size_t j = 0; j < op->h_jobs.size(); ++j)
        if (op->h_jobs[j].t_off >= 0) all.push_back((int)j);
    return fb_compose_jobs(op, all, s);
}

// ------------------------------------------------------------ host side ----
__global__ void k_leaf_of(const int32_t* leaf_start, int nleaf, int32_t* leaf_of) {
    int b = blockIdx.x;
    if (b >= nleaf) return;
    for (int i = leaf_start[b] + threadIdx.x; i < leaf_start[b + 1]; i += blockDim.x) leaf_of[i] = b;
}
__global__ void k_box_centers(const uint32_t* keys, int n, int level, double ox, double oy, double oz,
                              double delta, double* c) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    uint32_t k = keys[b];
    int x = 0, y = 0, z = 0;
    for (int i = 0; i < level; ++i) {
        x |= ((k >> (3 * i)) & 1u) << i;
        y |= ((k >> (3 * i + 1)) & 1u) << i;
        z |= ((k >> (3 * i + 2)) & 1u) << i;
    }
    c[3 * b] = ox + (x + 0.5) * delta;
    c[3 * b + 1] = oy + (y + 0.5) * delta;
    c[3 * b + 2] = oz + (z + 0.5) * delta;
}

// Real factors d^n(theta) of the rotation blocks of every direction from the
// single matrix Delta^n = d^n(pi/2):
//   d^n_{mu,m}(theta) = sum_k Delta^n_{mu,k} Delta^n_{m,k} cos(k theta + (mu - m) pi/2),
// the rotation about y written as a rotation about z between two quarter
// turns (the identity holds for the real factors of this harmonic
// convention; checked against the projection of the definition to 1e-13 up
// to degree 40, and against the exponential of the rotation generator J_y to
// 1e-12 up to degree 318).  Also writes the phase tables ph[m + P - 1] = e^{i m phi}
// and, for degrees n < Pc, the complex blocks D = d e^{i m phi} the
// composed matrices use.  grid: (entry chunk, n, dir)
__global__ void k_rot_delta(const cd* delta, const double* dirs, int ndir, int P, int Pc, double* d64, float* d32,
                            cd* ph64, cf* ph32, cd* r64) {
    __shared__ double cs[FB_ROT_PMAX], sn[FB_ROT_PMAX];
    int n = blockIdx.y, dd = blockIdx.z;
    int w = 2 * n + 1;
    double x = dirs[3 * dd], y = dirs[3 * dd + 1], z = dirs[3 * dd + 2];
    double th = acos(fmax(-1.0, fmin(1.0, z / sqrt(x * x + y * y + z * z))));
    double phi = atan2(y, x);
    for (int k = threadIdx.x; k <= n; k += blockDim.x) sincos((double)k * th, &sn[k], &cs[k]);
    __syncthreads();
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && n == 0)
        for (int q = threadIdx.x; q < 2 * P - 1; q += blockDim.x) {
            double sp, cp;
            sincos((double)(q - (P - 1)) * phi, &sp, &cp);
            ph64[(int64_t)dd * (2 * P - 1) + q] = mk(cp, sp);
            ph32[(int64_t)dd * (2 * P - 1) + q] = mk((float)cp, (float)sp);
        }
    if (e >= w * w) return;
    int mu = e / w - n, m = e % w - n;
    int64_t off = (int64_t)n * (2 * n - 1) * (2 * n + 1) / 3;
    const cd* Dm = delta + off + (int64_t)(mu + n) * w;
    const cd* Dn = delta + off + (int64_t)(m + n) * w;
    // cos(k th + j pi/2) for j = (mu - m) mod 4: cos, -sin, -cos, sin
    int j = ((mu - m) % 4 + 4) % 4;
    double acc = 0.0;
    for (int k = -n; k <= n; ++k) {
        int ak = k < 0 ? -k : k;
        double c = cs[ak], sg = k < 0 ? -sn[ak] : sn[ak];
        double f = j == 0 ? c : (j == 1 ? -sg : (j == 2 ? -c : sg));
        acc = fma(Dm[k + n].re * Dn[k + n].re, f, acc);
    }
    int64_t per_dir = (int64_t)P * (2 * P - 1) * (2 * P + 1) / 3;
    int64_t o = (int64_t)dd * per_dir + off + e;
    d64[o] = acc;
    d32[o] = (float)acc;
    if (n < Pc) {
        double sp, cp;
        sincos((double)m * phi, &sp, &cp);
        int64_t per_c = (int64_t)Pc * (2 * Pc - 1) * (2 * Pc + 1) / 3;
        r64[(int64_t)dd * per_c + off + e] = mk(acc * cp, acc * sp);
    }
}

// Rotation data of every direction up to degree P, cached in the tree and
// recomputed only when a larger P is needed.  Delta^n = d^n(pi/2) comes from
// the definition of the rotation coefficients, evaluated by projection
// quadrature (exact for the band limit) for the direction +x; every
// direction's real factors then follow from it (k_rot_delta).
fb_status fb_tree_rotations(fb_tree* t, int P, const std::vector<double>& dirs, cudaStream_t s,
                            const fb_tree::RotSet** out) {
    int ndir = (int)dirs.size() / 3;
    for (const auto& rs : t->rot_sets)
        if (rs.P == P && rs.ndir == ndir) {
            *out = &rs;
            return FB_OK;
        }
    if (P > FB_ROT_PMAX) return fb_fail(FB_ERR_ARG, "expansion order above " + std::to_string(FB_ROT_PMAX));
    const int Prot = P;
    const int Pc = std::min(P, FB_COMPOSE_PMAX);
    const int64_t per_dir = (int64_t)Prot * (2 * Prot - 1) * (2 * Prot + 1) / 3;
    const int64_t per_c = (int64_t)Pc * (2 * Pc - 1) * (2 * Pc + 1) / 3;
    const int nq = Prot + 1, nphi = 2 * Prot + 1, npts = nq * nphi;
    const int ystride = Prot * (Prot + 1) / 2 + 8;
    double *glx = nullptr, *glw = nullptr, *ddirs = nullptr, *dx = nullptr, *yscr = nullptr;
    cd *Yg = nullptr, *Yr = nullptr, *delta = nullptr;
    auto free_tmp = [&]() { dfree(glx); dfree(glw); dfree(ddirs); dfree(dx); dfree(yscr); dfree(Yg); dfree(Yr); dfree(delta); };
    fb_status st;
    if ((st = dalloc(&glx, nq)) || (st = dalloc(&glw, nq)) || (st = dalloc(&ddirs, dirs.size())) ||
        (st = dalloc(&dx, 3)) || (st = dalloc(&yscr, (size_t)npts * ystride)) ||
        (st = dalloc(&Yg, (size_t)npts * Prot * Prot)) || (st = dalloc(&Yr, (size_t)npts * Prot * Prot)) ||
        (st = dalloc(&delta, per_dir))) {
        free_tmp();
        return st;
    }
    const double xdir[3] = {1.0, 0.0, 0.0};
    FB_CUDA(cudaMemcpyAsync(ddirs, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemcpyAsync(dx, xdir, sizeof(xdir), cudaMemcpyHostToDevice, s));
    k_gauss_legendre<<<div_up(nq, 64), 64, 0, s>>>(nq, glx, glw);
    // Y_n^m on the grid, unrotated and rotated for the direction +x
    k_rot_grid<<<div_up(npts, 128), 128, 0, s>>>(dx, 1, 1, Prot, nq, nphi, glx, yscr, ystride, Yg);
    k_rot_grid<<<div_up(npts, 128), 128, 0, s>>>(dx, 1, 0, Prot, nq, nphi, glx, yscr, ystride, Yr);
    {
        dim3 grid(div_up((2 * Prot - 1) * (2 * Prot - 1), 128), Prot, 1);
        k_rot_project<<<grid, 128, 0, s>>>(Yg, Yr, 1, Prot, nq, nphi, glw, 0, delta);
    }
    FB_LAUNCH_CHECK();
    fb_tree::RotSet rs;
    rs.P = Prot;
    rs.Pc = Pc;
    rs.per_dir = per_dir;
    rs.per_dir_c = per_c;
    rs.ndir = ndir;
    auto free_rs = [&]() { dfree(rs.r64); dfree(rs.d64); dfree(rs.d32); dfree(rs.ph64); dfree(rs.ph32); };
    if ((st = dalloc(&rs.r64, (size_t)ndir * per_c)) || (st = dalloc(&rs.d64, (size_t)ndir * per_dir)) ||
        (st = dalloc(&rs.d32, (size_t)ndir * per_dir)) || (st = dalloc(&rs.ph64, (size_t)ndir * (2 * Prot - 1))) ||
        (st = dalloc(&rs.ph32, (size_t)ndir * (2 * Prot - 1)))) {
        free_tmp();
        free_rs();
        return st;
    }
    {
        dim3 grid(div_up((2 * Prot - 1) * (2 * Prot - 1), 128), Prot, ndir);
        k_rot_delta<<<grid, 128, 0, s>>>(delta, ddirs, ndir, Prot, Pc, rs.d64, rs.d32, rs.ph64, rs.ph32, rs.r64);
    }
    FB_LAUNCH_CHECK();
    cudaError_t e = cudaStreamSynchronize(s);
    free_tmp();
    if (e != cudaSuccess) {
        free_rs();
        return fb_fail(FB_ERR_CUDA, std::string("rotation setup: ") + cudaGetErrorString(e));
    }
    t->rot_sets.push_back(rs);
    *out = &t->rot_sets.back();
    return FB_OK;
}

static int igcd(int a, int b) {
    a = std::abs(a);
    b = std::abs(b);
    while (b) { int t = a % b; a = b; b = t; }
    return a;
}

static void build_tiles(TransPlan& pl) {
    const int BM = 64, BN = 32;
    pl.h_tiles.clear();
    for (int t = 0; t < (int)pl.h_tasks.size(); ++t) {
        const TransTask& tk = pl.h_tasks[t];
        for (int r = 0; r < tk.rows; r += BM)
            for (int c = 0; c < tk.npairs; c += BN) pl.h_tiles.push_back(TransTile{t, r, c, 0});
    }
    pl.ntiles = (int)pl.h_tiles.size();
}

static fb_status upload_plan(TransPlan& pl, const int32_t* src, const int32_t* dst) {
    pl.src_idx = src;
    pl.dst_idx = dst;
    build_tiles(pl);
    if (pl.h_tasks.empty()) return FB_OK;
    FB_CHECK(dalloc(&pl.tasks, pl.h_tasks.size()));
    FB_CHECK(dalloc(&pl.tiles, pl.h_tiles.size()));
    FB_CUDA(cudaMemcpy(pl.tasks, pl.h_tasks.data(), sizeof(TransTask) * pl.h_tasks.size(), cudaMemcpyHostToDevice));
    FB_CUDA(cudaMemcpy(pl.tiles, pl.h_tiles.data(), sizeof(TransTile) * pl.h_tiles.size(), cudaMemcpyHostToDevice));
    return FB_OK;
}

fb_status fb_fmm_create(fb_op* op, double d0, int pmin, cudaStream_t s) {
    const fb_tree* t = op->tree;
    const fb_mesh* m = op->mesh;
    int L = t->L;
    op->L = L;
    int64_t n = op->n;
    double k = op->k;
    for (int l = 2; l <= L; ++l) op->p[l] = fb_order_rule(k, t->side / (double)(1 << l), d0, pmin);
    int pL = op->p[L], PL = pL * pL;
    op->lev_off[0] = 0;
    for (int l = 0; l <= L; ++l) {
        int P = l >= 2 ? op->p[l] * op->p[l] : 0;
        op->lev_off[l + 1] = op->lev_off[l] + (int64_t)t->nbox[l] * P;
    }
    int64_t mp_count = op->lev_off[L + 1];
    // ---- near field
    int nleaf = t->nbox[L];
    std::vector<int32_t> ucnt(nleaf), ulist((size_t)nleaf * FB_ULIST);
    FB_CUDA(cudaMemcpyAsync(ucnt.data(), t->ucnt, sizeof(int32_t) * nleaf, cudaMemcpyDeviceToHost, s));
    FB_CUDA(cudaMemcpyAsync(ulist.data(), t->ulist, sizeof(int32_t) * ulist.size(), cudaMemcpyDeviceToHost, s));
    FB_CUDA(cudaStreamSynchronize(s));
    const std::vector<int32_t>& ls = t->h_leaf_start;
    op->h_nf_off.assign(nleaf + 1, 0);
    op->h_nf_ncol.assign(nleaf, 0);
    for (int b = 0; b < nleaf; ++b) {
        int K = 0;
        for (int i = 0; i < ucnt[b]; ++i) {
            int sl = ulist[(size_t)b * FB_ULIST + i];
            K += ls[sl + 1] - ls[sl];
        }
        op->h_nf_ncol[b] = K;
        op->h_nf_off[b + 1] = op->h_nf_off[b] + (int64_t)(ls[b + 1] - ls[b]) * K;
    }
    op->nf_count = op->h_nf_off[nleaf];
    FB_CHECK(dalloc(&op->nf_off, nleaf + 1));
    FB_CHECK(dalloc(&op->nf_ncol, nleaf));
    FB_CHECK(dalloc(&op->nf64, op->nf_count));
    FB_CUDA(cudaMemcpyAsync(op->nf_off, op->h_nf_off.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, s));
    FB_CUDA(cudaMemcpyAsync(op->nf_ncol, op->h_nf_ncol.data(), sizeof(int32_t) * nleaf, cudaMemcpyHostToDevice, s));
    const fb_op* dn = op->near_donor;
    if (dn && dn->nf64 && dn->kind == op->kind && dn->k == k && dn->mesh == m && dn->tree == t &&
        dn->nf_count == op->nf_count) {
        // the same entries: copy them instead of integrating again
        FB_CUDA(cudaMemcpyAsync(op->nf64, dn->nf64, sizeof(cd) * op->nf_count, cudaMemcpyDeviceToDevice, s));
    } else {
        k_near_fill<<<nleaf, 256, 0, s>>>(m->g, op->kind, k, m->rc, t->perm, t->leaf_start, t->ucnt, t->ulist,
                                          op->nf_off, op->nf_ncol, op->nf64);
        FB_LAUNCH_CHECK();
    }
    // ---- box centres of every level
    std::vector<double*> centers(L + 1, nullptr);
    auto free_centers = [&]() { for (auto& c : centers) dfree(c); };
    for (int l = 0; l <= L; ++l) {
        fb_status st = dalloc(&centers[l], (size_t)3 * t->nbox[l]);
        if (st) { free_centers(); return st; }
        k_box_centers<<<div_up(t->nbox[l], 128), 128, 0, s>>>(t->keys[l], t->nbox[l], l, t->origin[0],
                                                              t->origin[1], t->origin[2],
                                                              t->side / (double)(1 << l), centers[l]);
    }
    // ---- P2M / L2P operators
    {
        int32_t* leaf_of = nullptr;
        double* scratch = nullptr;
        int nthreads = 152 * 256;
        int Pp1 = pL + 1;
        // even stride: each thread's slice starts with complex values (16-byte aligned)
        int sstride = (2 * Pp1 * Pp1 + Pp1 * (Pp1 + 1) / 2 + Pp1 + 32 + 1) & ~1;
        fb_status st;
        if ((st = dalloc(&leaf_of, n)) || (st = dalloc(&scratch, (size_t)nthreads * sstride)) ||
            (st = dalloc(&op->w64, (size_t)n * PL)) || (st = dalloc(&op->v64, (size_t)n * PL))) {
            dfree(leaf_of); dfree(scratch); free_centers();
            return st;
        }
        k_leaf_of<<<nleaf, 64, 0, s>>>(t->leaf_start, nleaf, leaf_of);
        k_p2m_l2p<<<nthreads / 128, 128, 0, s>>>(m->g, op->kind, k, pL, n, t->perm, leaf_of, centers[L],
                                                  scratch, sstride, op->w64, op->v64);
        cudaError_t e = cudaStreamSynchronize(s);
        dfree(leaf_of);
        dfree(scratch);
        if (e != cudaSuccess) { free_centers(); return fb_fail(FB_ERR_CUDA, std::string("P2M/L2P setup: ") + cudaGetErrorString(e)); }
    }
    free_centers();
    // ---- translation inventory: directions, coaxial sets, matrices
    int pmax = 0;
    for (int l = 2; l <= L; ++l) pmax = std::max(pmax, op->p[l]);
    std::vector<int> dir_of_code(FB_NOFF, -1);
    std::vector<double> dirs;    // unit-free integer directions
    std::map<std::tuple<int, int, int>, int> dir_index;
    auto get_dir = [&](int dx, int dy, int dz) {
        int g = igcd(igcd(dx, dy), dz);
        auto key = std::make_tuple(dx / g, dy / g, dz / g);
        auto it = dir_index.find(key);
        if (it != dir_index.end()) return it->second;
        int id = (int)dirs.size() / 3;
        dirs.push_back(dx / g);
        dirs.push_back(dy / g);
        dirs.push_back(dz / g);
        dir_index[key] = id;
        return id;
    };
    for (int c = 0; c < FB_NOFF; ++c) {
        int dx = c / 49 - 3, dy = (c / 7) % 7 - 3, dz = c % 7 - 3;
        if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) <= 1) continue;
        dir_of_code[c] = get_dir(dx, dy, dz);
    }
    int oct_dir_m2m[8], oct_dir_l2l[8];
    for (int o = 0; o < 8; ++o) {
        int sx = 1 - 2 * (o & 1), sy = 1 - 2 * ((o >> 1) & 1), sz = 1 - 2 * ((o >> 2) & 1);
        oct_dir_m2m[o] = get_dir(sx, sy, sz);     // parent - child = (1/2 - b) delta
        oct_dir_l2l[o] = get_dir(-sx, -sy, -sz);  // child - parent
    }
    int ndir = (int)dirs.size() / 3;
    op->dir_of_code = dir_of_code;
    // directions sharing a polar angle share their real rotation factors d^n
    // (D^n_{mu,m} = d^n_{mu,m}(theta) e^{i m phi}): representative of each
    // direction = the first direction with the same cos(theta) = dz / |d|,
    // compared exactly on the integer vectors (dz^2 |d'|^2 = dz'^2 |d|^2,
    // same sign of dz)
    op->theta_rep.assign(ndir, -1);
    for (int a = 0; a < ndir; ++a) {
        const int64_t za = (int64_t)dirs[3 * a + 2];
        const int64_t na = (int64_t)(dirs[3 * a] * dirs[3 * a] + dirs[3 * a + 1] * dirs[3 * a + 1] + za * za);
        for (int b = 0; b <= a; ++b) {
            const int64_t zb = (int64_t)dirs[3 * b + 2];
            const int64_t nb = (int64_t)(dirs[3 * b] * dirs[3 * b] + dirs[3 * b + 1] * dirs[3 * b + 1] + zb * zb);
            if ((za > 0) == (zb > 0) && (za < 0) == (zb < 0) && za * za * nb == zb * zb * na) {
                op->theta_rep[a] = b;
                break;
            }
        }
    }
    // polar-angle groups: one folded rotation table each (staged RCR)
    op->theta_slot.assign(ndir, -1);
    op->theta_dirs.clear();
    for (int a = 0; a < ndir; ++a) {
        const int rep = op->theta_rep[a];
        if (rep == a) {
            op->theta_slot[a] = (int)op->theta_dirs.size();
            op->theta_dirs.push_back(a);
        } else {
            op->theta_slot[a] = op->theta_slot[rep];
        }
    }
    // coaxial sets
    std::vector<CoaxSet> sets;
    std::map<std::tuple<int, int, int64_t>, int> set_index;   // (kind, p, ktau bits)
    auto get_set = [&](int kind, int p, double ktau) {
        int64_t bits;
        memcpy(&bits, &ktau, 8);
        auto key = std::make_tuple(kind, p, bits);
        auto it = set_index.find(key);
        if (it != set_index.end()) return it->second;
        int id = (int)sets.size();
        sets.push_back(CoaxSet{ktau, p, kind, 0});
        set_index[key] = id;
        return id;
    };
    struct MatReq { int level, which, code, pout, pin, dir, set; };
    std::vector<MatReq> reqs;
    op->m2l_toff.assign((size_t)(L + 1) * FB_NOFF, -1);
    for (int l = 2; l <= L; ++l) {
        double delta = t->side / (double)(1 << l);
        for (int c = 0; c < FB_NOFF; ++c) {
            int64_t cnt = t->m2l_group[(size_t)l * FB_NOFF + c + 1] - t->m2l_group[(size_t)l * FB_NOFF + c];
            if (cnt == 0) continue;
            int dx = c / 49 - 3, dy = (c / 7) % 7 - 3, dz = c % 7 - 3;
            double tau = std::sqrt((double)(dx * dx + dy * dy + dz * dz)) * delta;
            reqs.push_back(MatReq{l, 0, c, op->p[l], op->p[l], dir_of_code[c], get_set(0, op->p[l], k * tau)});
        }
    }
    for (int l = 3; l <= L; ++l) {
        double tau = std::sqrt(3.0) * 0.5 * (t->side / (double)(1 << l));
        int pc = std::max(op->p[l], op->p[l - 1]);
        int sidx = get_set(1, pc, k * tau);
        for (int o = 0; o < 8; ++o) {
            op->m2m_toff[l][o] = -1;
            op->l2l_toff[l][o] = -1;
            if (t->oct_group[l][o + 1] == t->oct_group[l][o]) continue;
            reqs.push_back(MatReq{l, 1, o, op->p[l - 1], op->p[l], oct_dir_m2m[o], sidx});
            reqs.push_back(MatReq{l, 2, o, op->p[l], op->p[l - 1], oct_dir_l2l[o], sidx});
        }
    }
    // coaxial coefficients
    int64_t coax_total = 0, scr_stride = 0, f_stride = 0;
    for (auto& cs : sets) {
        cs.out_off = coax_total;
        coax_total += (int64_t)cs.p * cs.p * cs.p;
        scr_stride = std::max<int64_t>(scr_stride, (int64_t)(cs.p + 1) * (2 * cs.p + 2) * (cs.p + 2));
        f_stride = std::max<int64_t>(f_stride, 4 * cs.p + 4);
    }
    cd* coax = nullptr;
    cd* cscr = nullptr;
    double* fscr = nullptr;
    CoaxSet* dsets = nullptr;
    auto free_coax = [&]() { dfree(coax); dfree(cscr); dfree(fscr); dfree(dsets); };
    fb_status st;
    if ((st = dalloc(&coax, std::max<int64_t>(coax_total, 1))) ||
        (st = dalloc(&cscr, std::max<int64_t>(scr_stride * (int64_t)sets.size(), 1))) ||
        (st = dalloc(&fscr, std::max<int64_t>(f_stride * (int64_t)sets.size(), 1))) ||
        (st = dalloc(&dsets, std::max<size_t>(sets.size(), 1)))) {
        free_coax();
        return st;
    }
    if (!sets.empty()) {
        FB_CUDA(cudaMemcpyAsync(dsets, sets.data(), sizeof(CoaxSet) * sets.size(), cudaMemcpyHostToDevice, s));
        k_coaxial<<<div_up((int64_t)sets.size(), 32), 32, 0, s>>>(dsets, (int)sets.size(), cscr, scr_stride,
                                                                  fscr, f_stride, coax);
        FB_LAUNCH_CHECK();
    }
    // rotation blocks of every direction up to pmax (cached in the tree: they
    // depend only on the directions, not on k or the operator)
    const fb_tree::RotSet* rset = nullptr;
    FB_CHECK(fb_tree_rotations(const_cast<fb_tree*>(t), pmax, dirs, s, &rset));
    int Prot = rset->P;
    int64_t per_dir = rset->per_dir;
    cd* rot = rset->r64;
    const int64_t per_dir_c = rset->per_dir_c;
    // composed translation matrices
    std::vector<ComposeJob> jobs;
    int64_t T_total = 0;
    for (auto& r : reqs) {
        ComposeJob jb;
        const bool fits = r.pout <= FB_COMPOSE_PMAX && r.pin <= FB_COMPOSE_PMAX;
        jb.t_off = fits ? T_total : -1;
        jb.rot_off = (int64_t)r.dir * per_dir_c;   // complex blocks: degrees < FB_COMPOSE_PMAX
        jb.coax_off = sets[r.set].out_off;
        jb.p_out = r.pout;
        jb.p_in = r.pin;
        jb.pc = sets[r.set].p;
        jobs.push_back(jb);
        if (r.which == 0) op->m2l_toff[(size_t)r.level * FB_NOFF + r.code] = jb.t_off;
        else if (r.which == 1) op->m2m_toff[r.level][r.code] = jb.t_off;
        else op->l2l_toff[r.level][r.code] = jb.t_off;
        if (fits) T_total += (int64_t)r.pout * r.pout * r.pin * r.pin;
    }
    // the matrix buffers are allocated by the first composition
    op->T_count = T_total;
    cudaError_t e = cudaStreamSynchronize(s);
    // the rotation blocks and coaxial sets stay with the operator (RCR form)
    op->coax64 = coax;
    op->coax_count = std::max<int64_t>(coax_total, 1);
    coax = nullptr;
    op->rot64 = rot;
    op->rotd64 = rset->d64;
    op->rotd32 = rset->d32;
    op->rph64 = rset->ph64;
    op->rph32 = rset->ph32;
    op->rot_count = (int64_t)ndir * per_dir;
    op->Prot = Prot;
    op->per_dir = per_dir;
    free_coax();
    FB_CHECK(fb_stg_tables(op, rset->d64, s));
    // composed matrices are built on demand (tensor-core levels below,
    // everything for the composed method or for inspection)
    op->h_jobs = jobs;
    op->h_job_level.clear();
    op->h_job_m2l.clear();
    for (auto& r : reqs) {
        op->h_job_level.push_back(r.level);
        op->h_job_m2l.push_back(r.which == 0 ? 1 : 0);
    }
    op->job_done.assign(jobs.size(), 0);
    op->m2l_job.assign((size_t)(L + 1) * FB_NOFF, -1);
    for (int l = 0; l <= FB_MAXLEV; ++l)
        for (int o = 0; o < 8; ++o) op->m2m_job[l][o] = op->l2l_job[l][o] = -1;
    for (size_t j = 0; j < reqs.size(); ++j) {
        const MatReq& r = reqs[j];
        if (r.which == 0) op->m2l_job[(size_t)r.level * FB_NOFF + r.code] = (int)j;
        else if (r.which == 1) op->m2m_job[r.level][r.code] = (int)j;
        else op->l2l_job[r.level][r.code] = (int)j;
    }
    if (e != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("translation setup: ") + cudaGetErrorString(e));
    // RCR plans: one task per (level, offset) / (level, octant) group
    {
        auto rcr_task = [&](const MatReq& r, int64_t g0, int64_t g1, int64_t src_base, int64_t dst_base) {
            RcrTask tk;
            tk.rot_off = (int64_t)r.dir * per_dir;
            tk.coax_off = sets[r.set].out_off;
            tk.pair_off = g0;
            tk.npairs = (int32_t)(g1 - g0);
            tk.p_out = r.pout;
            tk.p_in = r.pin;
            tk.pc = sets[r.set].p;
            tk.src_base = src_base;
            tk.dst_base = dst_base;
            tk.staged = r.which == 0 ? op->stg_m2l[r.level] : op->stg_pair[r.level];
            tk.pad = 0;
            return tk;
        };
        {
            const size_t cs = op->prec == FB_PREC_MIXED_FMM ? sizeof(cf) : sizeof(cd);
            for (int l = 2; l <= L; ++l) {
                op->stg_m2l[l] = fb_rcr_default_staged(op->p[l], op->p[l], cs);
                if (l >= 3) {
                    const int pm = std::max(op->p[l], op->p[l - 1]);
                    op->stg_pair[l] = fb_rcr_default_staged(pm, pm, cs);
                }
            }
        }
        // levels whose M2L groups are dense enough for the tensor-core form
        // (mixed precision): on average >= 48 box pairs per translation vector
        std::vector<int> tc_levels;
        if (op->prec == FB_PREC_MIXED_FMM) {
            for (int l = 2; l <= L; ++l) {
                int64_t pairs = 0, groups = 0;
                for (int c = 0; c < FB_NOFF; ++c) {
                    int64_t cnt = t->m2l_group[(size_t)l * FB_NOFF + c + 1] - t->m2l_group[(size_t)l * FB_NOFF + c];
                    if (cnt) { pairs += cnt; ++groups; }
                }
                if (groups && pairs >= 48 * groups && fb_composable(op, l, false)) {
                    tc_levels.push_back(l);
                    op->tc_level[l] = 1;
                }
            }
        }
        for (auto& r : reqs) {
            if (r.which == 0) {
                int64_t g0 = t->m2l_group[(size_t)r.level * FB_NOFF + r.code];
                int64_t g1 = t->m2l_group[(size_t)r.level * FB_NOFF + r.code + 1];
                RcrTask tk = rcr_task(r, g0, g1, op->lev_off[r.level], op->lev_off[r.level]);
                op->m2l_rcr.h_tasks.push_back(tk);
                if (!op->tc_level[r.level]) op->m2l_rcr_rest.h_tasks.push_back(tk);
            } else {
                int64_t g0 = t->oct_group[r.level][r.code], g1 = t->oct_group[r.level][r.code + 1];
                if (r.which == 1)
                    op->m2m_rcr[r.level].h_tasks.push_back(
                        rcr_task(r, g0, g1, op->lev_off[r.level], op->lev_off[r.level - 1]));
                else
                    op->l2l_rcr[r.level].h_tasks.push_back(
                        rcr_task(r, g0, g1, op->lev_off[r.level - 1], op->lev_off[r.level]));
            }
        }
        size_t csz = op->prec == FB_PREC_MIXED_FMM ? sizeof(cf) : sizeof(cd);
        FB_CHECK(fb_rcr_upload(op, op->m2l_rcr, t->m2l_src, t->m2l_dst, csz));
        FB_CHECK(fb_rcr_upload(op, op->m2l_rcr_rest, t->m2l_src, t->m2l_dst, csz));
        if (!tc_levels.empty()) {
            std::vector<int> need;
            for (size_t j = 0; j < op->h_jobs.size(); ++j)
                if (op->h_job_m2l[j] && op->tc_level[op->h_job_level[j]]) need.push_back((int)j);
            FB_CHECK(fb_compose_jobs(op, need, s));
            FB_CHECK(fb_tc_build(op, tc_levels, &op->tc_plan, s));
        }
        // M2M / L2L of child levels with >= 48 boxes per octant on average
        if (op->prec == FB_PREC_MIXED_FMM) {
            for (int l = 3; l <= L; ++l) {
                if (t->nbox[l] < 48 * 8 || !fb_composable(op, l, true)) continue;
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
                FB_CHECK(fb_compose_jobs(op, need, s));
                FB_CHECK(fb_tc_build_groups(op, up, t->oct_child[l], t->oct_parent[l], &op->tc_m2m[l], s));
                FB_CHECK(fb_tc_build_groups(op, down, t->oct_parent[l], t->oct_child[l], &op->tc_l2l[l], s));
            }
        }
        for (int l = 3; l <= L; ++l) {
            FB_CHECK(fb_rcr_upload(op, op->m2m_rcr[l], t->oct_child[l], t->oct_parent[l], csz));
            FB_CHECK(fb_rcr_upload(op, op->l2l_rcr[l], t->oct_parent[l], t->oct_child[l], csz));
        }
        op->method = FB_TRANS_AUTO;
    }
    // ---- FP32 copies for the mixed path.  High orders at small k tau give
    // coaxial coefficients (spherical Hankel functions of high order) beyond
    // the FP32 range; the mixed form is refused for such operators instead of
    // producing overflowed translations (the FP64 form handles them).
    if (op->prec == FB_PREC_MIXED_FMM) {
        double* dmax = nullptr;
        FB_CHECK(dalloc(&dmax, 1));
        FB_CUDA(cudaMemsetAsync(dmax, 0, sizeof(double), s));
        k_absmax<<<std::min(div_up(op->coax_count, 256), 1024), 256, 0, s>>>(op->coax64, op->coax_count, dmax);
        double hmax = 0.0;
        cudaError_t ce = cudaMemcpyAsync(&hmax, dmax, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        dfree(dmax);
        if (ce != cudaSuccess) return fb_fail(FB_ERR_CUDA, cudaGetErrorString(ce));
        if (!(hmax < 1e37))
            return fb_fail(FB_ERR_ARG, "mixed precision: translation coefficients reach " + std::to_string(hmax) +
                                           ", beyond the FP32 range at this order and wavenumber; use "
                                           "FB_PREC_FP64_FMM or a lower p_min");
    }
    if (op->prec == FB_PREC_MIXED_FMM) {
        FB_CHECK(dalloc(&op->nf32, op->nf_count));
        FB_CHECK(dalloc(&op->w32, (size_t)n * PL));
        FB_CHECK(dalloc(&op->v32, (size_t)n * PL));
        k_d2f<<<div_up(op->nf_count, 256), 256, 0, s>>>(op->nf64, op->nf32, op->nf_count);
        k_d2f<<<div_up(n * PL, 256), 256, 0, s>>>(op->w64, op->w32, n * PL);
        k_d2f<<<div_up(n * PL, 256), 256, 0, s>>>(op->v64, op->v32, n * PL);
        FB_CHECK(dalloc(&op->coax32, op->coax_count));
        k_d2f<<<div_up(op->coax_count, 256), 256, 0, s>>>(op->coax64, op->coax32, op->coax_count);
        FB_LAUNCH_CHECK();
        FB_CHECK(dalloc((cf**)&op->mp, mp_count));
        FB_CHECK(dalloc((cf**)&op->loc, mp_count));
        // of the FP64 entries only the leaf self-blocks stay (block-Jacobi
        // factorisation); the rest are dropped once the FP32 copies exist
        {
            int nleaf = t->nbox[L];
            std::vector<int64_t> off(nleaf + 1, 0);
            for (int b = 0; b < nleaf; ++b) {
                int64_t nb = t->h_leaf_start[b + 1] - t->h_leaf_start[b];
                off[b + 1] = off[b] + nb * nb;
            }
            int64_t* d_off = nullptr;
            FB_CHECK(dalloc(&d_off, nleaf + 1));
            fb_status st2 = dalloc(&op->self64, std::max<int64_t>(off[nleaf], 1));
            if (st2 == FB_OK) {
                cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (nleaf + 1), cudaMemcpyHostToDevice, s);
                st2 = fb_self_blocks(op, d_off, op->self64, s);
            }
            cudaError_t e2 = cudaStreamSynchronize(s);
            dfree(d_off);
            FB_CHECK(st2);
            if (e2 != cudaSuccess) return fb_fail(FB_ERR_CUDA, std::string("self blocks: ") + cudaGetErrorString(e2));
            dfree(op->nf64);
            dfree(op->w64);
            dfree(op->v64);
        }
    } else {
        FB_CHECK(dalloc((cd**)&op->mp, mp_count));
        FB_CHECK(dalloc((cd**)&op->loc, mp_count));
    }
    // ---- translation plans
    for (int l = 2; l <= L; ++l)
        for (int c = 0; c < FB_NOFF; ++c) {
            int64_t g0 = t->m2l_group[(size_t)l * FB_NOFF + c], g1 = t->m2l_group[(size_t)l * FB_NOFF + c + 1];
            if (g1 == g0) continue;
            TransTask tk;
            tk.t_off = op->m2l_toff[(size_t)l * FB_NOFF + c];
            tk.pair_off = g0;
            tk.npairs = (int32_t)(g1 - g0);
            tk.rows = tk.cols = op->p[l] * op->p[l];
            tk.src_base = op->lev_off[l];
            tk.dst_base = op->lev_off[l];
            op->m2l.h_tasks.push_back(tk);
        }
    FB_CHECK(upload_plan(op->m2l, t->m2l_src, t->m2l_dst));
    for (int l = 3; l <= L; ++l) {
        for (int o = 0; o < 8; ++o) {
            int64_t g0 = t->oct_group[l][o], g1 = t->oct_group[l][o + 1];
            if (g1 == g0) continue;
            TransTask up;
            up.t_off = op->m2m_toff[l][o];
            up.pair_off = g0;
            up.npairs = (int32_t)(g1 - g0);
            up.rows = op->p[l - 1] * op->p[l - 1];
            up.cols = op->p[l] * op->p[l];
            up.src_base = op->lev_off[l];
            up.dst_base = op->lev_off[l - 1];
            op->m2m[l].h_tasks.push_back(up);
            TransTask dn;
            dn.t_off = op->l2l_toff[l][o];
            dn.pair_off = g0;
            dn.npairs = (int32_t)(g1 - g0);
            dn.rows = op->p[l] * op->p[l];
            dn.cols = op->p[l - 1] * op->p[l - 1];
            dn.src_base = op->lev_off[l - 1];
            dn.dst_base = op->lev_off[l];
            op->l2l[l].h_tasks.push_back(dn);
        }
        // M2M: src child -> dst parent; L2L: src parent -> dst child
        FB_CHECK(upload_plan(op->m2m[l], t->oct_child[l], t->oct_parent[l]));
        FB_CHECK(upload_plan(op->l2l[l], t->oct_parent[l], t->oct_child[l]));
    }
    FB_CUDA(cudaStreamSynchronize(s));
    return FB_OK;
}
