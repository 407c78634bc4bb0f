// Uniform octree over the element centroids, built on the device (Sec. 3.3:
// the smallest box delta must exceed the near-field cutoff r_c).
//
//   root      bounding cube of the vertices, side = largest extent x (1+1e-6)
//   leaf      the box containing the centroid: floor((c - origin)/delta),
//             clamped; FP64 rounding identical to plain IEEE evaluation
//   level     first level >= 2 whose fullest leaf holds <= leaf_max elements,
//             capped at the deepest level with delta > r_c
//   order     elements sorted by (leaf Morton key, element index)
//   U-list    touching non-empty leaves (itself included), ascending
//   V-list    boxes of the same level not touching, parents touching, ascending
// Morton keys interleave x (lowest bit), y, z.
#include <algorithm>

#include "common.cuh"

// ------------------------------------------------------- bitonic sort ----
__global__ void k_bitonic_global(uint64_t* a, int64_t n, int64_t j, int64_t k) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t p = i ^ j;
    if (p > i) {
        uint64_t x = a[i], y = a[p];
        bool up = (i & k) == 0;
        if ((x > y) == up) { a[i] = y; a[p] = x; }
    }
}

// All stages j <= jmax (< 2048) of step k inside blocks of 2048 elements.
__global__ void k_bitonic_shared(uint64_t* a, int64_t k, int64_t jmax) {
    __shared__ uint64_t s[2048];
    int64_t base = (int64_t)blockIdx.x * 2048;
    s[threadIdx.x] = a[base + threadIdx.x];
    s[threadIdx.x + 1024] = a[base + threadIdx.x + 1024];
    __syncthreads();
    for (int64_t j = jmax; j > 0; j >>= 1) {
        int t = threadIdx.x;
        int lo = (int)((t / j) * 2 * j + (t % j));
        int hi = lo + (int)j;
        int64_t gi = base + lo;
        bool up = (gi & k) == 0;
        uint64_t x = s[lo], y = s[hi];
        if ((x > y) == up) { s[lo] = y; s[hi] = x; }
        __syncthreads();
    }
    a[base + threadIdx.x] = s[threadIdx.x];
    a[base + threadIdx.x + 1024] = s[threadIdx.x + 1024];
}

__global__ void k_fill_u64(uint64_t* a, int64_t from, int64_t to, uint64_t v) {
    int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < to) a[i] = v;
}

// Sorts a[0..n) ascending; `a` must hold npad = max(2048, pow2 >= n) entries.
static fb_status bitonic_sort(uint64_t* a, int64_t n, int64_t npad, cudaStream_t s) {
    if (npad > n) k_fill_u64<<<div_up(npad - n, 256), 256, 0, s>>>(a, n, npad, ~0ULL);
    for (int64_t k = 2; k <= npad; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            if (j < 2048 && j <= 1024) {
                k_bitonic_shared<<<(unsigned)(npad / 2048), 1024, 0, s>>>(a, k, j);
                break;
            }
            k_bitonic_global<<<div_up(npad, 256), 256, 0, s>>>(a, npad, j, k);
        }
    }
    FB_LAUNCH_CHECK();
    return FB_OK;
}

static int64_t pad_pow2(int64_t n) {
    int64_t p = 2048;
    while (p < n) p <<= 1;
    return p;
}

// ------------------------------------------------------------- helpers ----
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z, int level) {
    uint32_t k = 0;
    for (int b = 0; b < level; ++b) {
        k |= ((x >> b) & 1u) << (3 * b);
        k |= ((y >> b) & 1u) << (3 * b + 1);
        k |= ((z >> b) & 1u) << (3 * b + 2);
    }
    return k;
}
__device__ __forceinline__ void demorton3(uint32_t k, int level, int& x, int& y, int& z) {
    x = y = z = 0;
    for (int b = 0; b < level; ++b) {
        x |= ((k >> (3 * b)) & 1u) << b;
        y |= ((k >> (3 * b + 1)) & 1u) << b;
        z |= ((k >> (3 * b + 2)) & 1u) << b;
    }
}
__device__ __forceinline__ int lower_bound_u32(const uint32_t* a, int n, uint32_t v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int find_box(const uint32_t* a, int n, uint32_t v) {
    int p = lower_bound_u32(a, n, v);
    return (p < n && a[p] == v) ? p : -1;
}

// key at `level` combined with the element index for sorting
__global__ void k_elem_keys(Geom g, double ox, double oy, double oz, double delta, int level,
                            uint64_t* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    int nb = 1 << level;
    double c[3] = {g.cx[i], g.cy[i], g.cz[i]};
    double o[3] = {ox, oy, oz};
    uint32_t ic[3];
    for (int d = 0; d < 3; ++d) {
        double f = floor(__ddiv_rn(__dsub_rn(c[d], o[d]), delta));
        int v = (int)f;
        v = v < 0 ? 0 : (v > nb - 1 ? nb - 1 : v);
        ic[d] = (uint32_t)v;
    }
    uint32_t key = morton3(ic[0], ic[1], ic[2], level);
    out[i] = ((uint64_t)key << 32) | (uint64_t)i;
}

// run length of identical (key >> shift) starting at each head; max into *mx
__global__ void k_max_run(const uint64_t* a, int64_t n, int shift, int* mx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = (uint32_t)(a[i] >> 32) >> shift;
    if (i > 0 && ((uint32_t)(a[i - 1] >> 32) >> shift) == key) return;
    int64_t lo = i, hi = n;   // first position with a different key
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (((uint32_t)(a[mid] >> 32) >> shift) == key) lo = mid + 1; else hi = mid;
    }
    atomicMax(mx, (int)(lo - i));
}

// heads of runs of (key >> shift): appended (unordered) as (key<<32 | pos)
__global__ void k_heads(const uint64_t* a, int64_t n, int shift, uint64_t* heads, int* cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = (uint32_t)(a[i] >> 32) >> shift;
    if (i > 0 && ((uint32_t)(a[i - 1] >> 32) >> shift) == key) return;
    int p = atomicAdd(cnt, 1);
    heads[p] = ((uint64_t)key << 32) | (uint64_t)i;
}

__global__ void k_split_perm(const uint64_t* a, int64_t n, int32_t* perm, int32_t* pos) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t e = (int32_t)(a[i] & 0xffffffffu);
    perm[i] = e;
    pos[e] = (int32_t)i;
}

__global__ void k_split_heads(const uint64_t* h, int nh, uint32_t* keys, int32_t* start, int64_t n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nh) {
        keys[i] = (uint32_t)(h[i] >> 32);
        if (start) start[i] = (int32_t)(h[i] & 0xffffffffu);
    }
    if (start && i == nh) start[nh] = (int32_t)n;
}

__global__ void k_parents(const uint32_t* keys, int n, const uint32_t* pkeys, int np, int32_t* par) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    par[i] = find_box(pkeys, np, keys[i] >> 3);
}

__global__ void k_ulist(const uint32_t* keys, int n, int level, int32_t* cnt, int32_t* list) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int x, y, z;
    demorton3(keys[b], level, x, y, z);
    int nb = 1 << level;
    int loc[FB_ULIST];
    int c = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int X = x + dx, Y = y + dy, Z = z + dz;
                if (X < 0 || Y < 0 || Z < 0 || X >= nb || Y >= nb || Z >= nb) continue;
                int f = find_box(keys, n, morton3(X, Y, Z, level));
                if (f >= 0) loc[c++] = f;
            }
    for (int i = 1; i < c; ++i) {   // ascending
        int v = loc[i], j = i - 1;
        while (j >= 0 && loc[j] > v) { loc[j + 1] = loc[j]; --j; }
        loc[j + 1] = v;
    }
    cnt[b] = c;
    for (int i = 0; i < c; ++i) list[(int64_t)b * FB_ULIST + i] = loc[i];
}

__global__ void k_vlist(const uint32_t* keys, int n, int level, int32_t* cnt, int32_t* list,
                        int* m2l_count /* [343] for this level */) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int x, y, z;
    demorton3(keys[b], level, x, y, z);
    int nb = 1 << level;
    int px = x >> 1, py = y >> 1, pz = z >> 1;
    int npar = nb >> 1;
    int32_t* out = list + (int64_t)b * FB_VLIST;
    int c = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int PX = px + dx, PY = py + dy, PZ = pz + dz;
                if (PX < 0 || PY < 0 || PZ < 0 || PX >= npar || PY >= npar || PZ >= npar) continue;
                for (int o = 0; o < 8; ++o) {
                    int X = 2 * PX + (o & 1), Y = 2 * PY + ((o >> 1) & 1), Z = 2 * PZ + ((o >> 2) & 1);
                    int ax = abs(X - x), ay = abs(Y - y), az = abs(Z - z);
                    if (max(ax, max(ay, az)) <= 1) continue;
                    int f = find_box(keys, n, morton3(X, Y, Z, level));
                    if (f < 0) continue;
                    out[c++] = f;
                    // offset t = target - source, in box units
                    int code = (x - X + 3) * 49 + (y - Y + 3) * 7 + (z - Z + 3);
                    atomicAdd(&m2l_count[code], 1);
                }
            }
    for (int i = 1; i < c; ++i) {
        int v = out[i], j = i - 1;
        while (j >= 0 && out[j] > v) { out[j + 1] = out[j]; --j; }
        out[j + 1] = v;
    }
    cnt[b] = c;
}

__global__ void k_m2l_fill(const uint32_t* keys, int n, int level, const int32_t* cnt,
                           const int32_t* list, int64_t* cursor /* [343] */, int32_t* src,
                           int32_t* dst) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int x, y, z;
    demorton3(keys[b], level, x, y, z);
    for (int i = 0; i < cnt[b]; ++i) {
        int s = list[(int64_t)b * FB_VLIST + i];
        int X, Y, Z;
        demorton3(keys[s], level, X, Y, Z);
        int code = (x - X + 3) * 49 + (y - Y + 3) * 7 + (z - Z + 3);
        int64_t p = atomicAdd((unsigned long long*)&cursor[code], 1ULL);
        src[p] = s;
        dst[p] = b;
    }
}

__global__ void k_oct_count(const uint32_t* keys, int n, int* cnt8) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    atomicAdd(&cnt8[keys[b] & 7u], 1);
}
__global__ void k_oct_fill(const uint32_t* keys, const int32_t* par, int n, int64_t* cursor8,
                           int32_t* child, int32_t* parent) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int64_t p = atomicAdd((unsigned long long*)&cursor8[keys[b] & 7u], 1ULL);
    child[p] = b;
    parent[p] = par[b];
}

// --------------------------------------------------------------- build ----
fb_status fb_tree_build_impl(const fb_mesh* m, int leaf_max, cudaStream_t s, fb_tree** out) {
    if (!m || !out) return fb_fail(FB_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (leaf_max < 1) return fb_fail(FB_ERR_ARG, "leaf_max must be >= 1");
    int64_t n = m->n;
    fb_tree* t = new fb_tree();
    t->mesh = m;
    t->dev = m->dev;
    t->n = n;
    double side = 0.0;
    double ctr[3];
    for (int d = 0; d < 3; ++d) side = std::max(side, m->hi[d] - m->lo[d]);
    side = side * (1.0 + 1e-6);
    for (int d = 0; d < 3; ++d) {
        ctr[d] = 0.5 * (m->lo[d] + m->hi[d]);
        t->origin[d] = ctr[d] - 0.5 * side;
    }
    t->side = side;
    int lrc = 0;
    while (side / (double)(1 << (lrc + 1)) > m->rc && lrc + 1 <= 10) ++lrc;
    if (lrc < 2) {
        delete t;
        return fb_fail(FB_ERR_ARG, "mesh too coarse for the FMM: no level >= 2 has box side > r_c");
    }
    int64_t npad = pad_pow2(n);
    uint64_t* a = nullptr;
    uint64_t* heads = nullptr;
    int* dint = nullptr;
    auto cleanup = [&]() { dfree(a); dfree(heads); dfree(dint); };
    fb_status st;
    if ((st = dalloc(&a, npad)) || (st = dalloc(&heads, npad)) || (st = dalloc(&dint, 4 * FB_NOFF + 16))) {
        cleanup();
        delete t;
        return st;
    }
    // keys at level lrc, sorted; occupancy of every coarser level by shifting
    k_elem_keys<<<div_up(n, 256), 256, 0, s>>>(m->g, t->origin[0], t->origin[1], t->origin[2],
                                                side / (double)(1 << lrc), lrc, a);
    if ((st = bitonic_sort(a, n, npad, s))) { cleanup(); delete t; return st; }
    int L = lrc;
    for (int lev = 2; lev <= lrc; ++lev) {
        int hmx = 0;
        cudaMemsetAsync(dint, 0, sizeof(int), s);
        k_max_run<<<div_up(n, 256), 256, 0, s>>>(a, n, 3 * (lrc - lev), dint);
        cudaMemcpyAsync(&hmx, dint, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (hmx <= leaf_max) { L = lev; break; }
    }
    t->L = L;
    // final order: (leaf key, element index)
    k_elem_keys<<<div_up(n, 256), 256, 0, s>>>(m->g, t->origin[0], t->origin[1], t->origin[2],
                                                side / (double)(1 << L), L, a);
    if ((st = bitonic_sort(a, n, npad, s))) { cleanup(); delete t; return st; }
    if ((st = dalloc(&t->perm, n)) || (st = dalloc(&t->elem_pos, n))) { cleanup(); fb_tree_destroy(t); return st; }
    k_split_perm<<<div_up(n, 256), 256, 0, s>>>(a, n, t->perm, t->elem_pos);
    // boxes of every level: heads of runs of (leaf key >> 3(L-l))
    for (int lev = L; lev >= 0; --lev) {
        int nh = 0;
        cudaMemsetAsync(dint, 0, sizeof(int), s);
        k_heads<<<div_up(n, 256), 256, 0, s>>>(a, n, 3 * (L - lev), heads, dint);
        cudaMemcpyAsync(&nh, dint, sizeof(int), cudaMemcpyDeviceToHost, s);
        FB_CUDA(cudaStreamSynchronize(s));
        int64_t hp = pad_pow2(nh);
        if ((st = bitonic_sort(heads, nh, hp, s))) { cleanup(); fb_tree_destroy(t); return st; }
        t->nbox[lev] = nh;
        if ((st = dalloc(&t->keys[lev], nh))) { cleanup(); fb_tree_destroy(t); return st; }
        if (lev == L && (st = dalloc(&t->leaf_start, nh + 1))) { cleanup(); fb_tree_destroy(t); return st; }
        k_split_heads<<<div_up(nh + 1, 256), 256, 0, s>>>(heads, nh, t->keys[lev],
                                                          lev == L ? t->leaf_start : nullptr, n);
    }
    for (int lev = 1; lev <= L; ++lev) {
        if ((st = dalloc(&t->parent[lev], t->nbox[lev]))) { cleanup(); fb_tree_destroy(t); return st; }
        k_parents<<<div_up(t->nbox[lev], 256), 256, 0, s>>>(t->keys[lev], t->nbox[lev], t->keys[lev - 1],
                                                            t->nbox[lev - 1], t->parent[lev]);
    }
    int nleaf = t->nbox[L];
    t->h_leaf_start.resize(nleaf + 1);
    cudaMemcpyAsync(t->h_leaf_start.data(), t->leaf_start, sizeof(int32_t) * (nleaf + 1),
                    cudaMemcpyDeviceToHost, s);
    if ((st = dalloc(&t->ucnt, nleaf)) || (st = dalloc(&t->ulist, (size_t)nleaf * FB_ULIST))) {
        cleanup(); fb_tree_destroy(t); return st;
    }
    k_ulist<<<div_up(nleaf, 128), 128, 0, s>>>(t->keys[L], nleaf, L, t->ucnt, t->ulist);
    // V-lists and M2L groups
    std::vector<int> cnt((size_t)(L + 1) * FB_NOFF, 0);
    int* dcnt = nullptr;
    if ((st = dalloc(&dcnt, (size_t)(L + 1) * FB_NOFF))) { cleanup(); fb_tree_destroy(t); return st; }
    cudaMemsetAsync(dcnt, 0, sizeof(int) * (L + 1) * FB_NOFF, s);
    for (int lev = 2; lev <= L; ++lev) {
        int nb = t->nbox[lev];
        if ((st = dalloc(&t->vcnt[lev], nb)) || (st = dalloc(&t->vlist[lev], (size_t)nb * FB_VLIST))) {
            dfree(dcnt); cleanup(); fb_tree_destroy(t); return st;
        }
        k_vlist<<<div_up(nb, 64), 64, 0, s>>>(t->keys[lev], nb, lev, t->vcnt[lev], t->vlist[lev],
                                              dcnt + lev * FB_NOFF);
    }
    cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, s);
    FB_CUDA(cudaStreamSynchronize(s));
    t->m2l_group.assign(cnt.size() + 1, 0);
    for (size_t i = 0; i < cnt.size(); ++i) t->m2l_group[i + 1] = t->m2l_group[i] + cnt[i];
    int64_t npair = t->m2l_group.back();
    int64_t* dcur = nullptr;
    if ((st = dalloc(&t->m2l_src, npair ? npair : 1)) || (st = dalloc(&t->m2l_dst, npair ? npair : 1)) ||
        (st = dalloc(&dcur, cnt.size()))) {
        dfree(dcnt); dfree(dcur); cleanup(); fb_tree_destroy(t); return st;
    }
    cudaMemcpyAsync(dcur, t->m2l_group.data(), sizeof(int64_t) * cnt.size(), cudaMemcpyHostToDevice, s);
    for (int lev = 2; lev <= L; ++lev) {
        int nb = t->nbox[lev];
        k_m2l_fill<<<div_up(nb, 128), 128, 0, s>>>(t->keys[lev], nb, lev, t->vcnt[lev], t->vlist[lev],
                                                   dcur + lev * FB_NOFF, t->m2l_src, t->m2l_dst);
    }
    // octant groups (child level lev -> parent lev-1), levels 3..L
    for (int lev = 3; lev <= L; ++lev) {
        int nb = t->nbox[lev];
        int h8[8];
        cudaMemsetAsync(dcnt, 0, sizeof(int) * 8, s);
        k_oct_count<<<div_up(nb, 256), 256, 0, s>>>(t->keys[lev], nb, dcnt);
        cudaMemcpyAsync(h8, dcnt, sizeof(h8), cudaMemcpyDeviceToHost, s);
        FB_CUDA(cudaStreamSynchronize(s));
        t->oct_group[lev].assign(9, 0);
        for (int o = 0; o < 8; ++o) t->oct_group[lev][o + 1] = t->oct_group[lev][o] + h8[o];
        cudaMemcpyAsync(dcur, t->oct_group[lev].data(), sizeof(int64_t) * 8, cudaMemcpyHostToDevice, s);
        if ((st = dalloc(&t->oct_child[lev], nb)) || (st = dalloc(&t->oct_parent[lev], nb))) {
            dfree(dcnt); dfree(dcur); cleanup(); fb_tree_destroy(t); return st;
        }
        k_oct_fill<<<div_up(nb, 256), 256, 0, s>>>(t->keys[lev], t->parent[lev], nb, dcur,
                                                   t->oct_child[lev], t->oct_parent[lev]);
        FB_CUDA(cudaStreamSynchronize(s));
    }
    cudaError_t e = cudaStreamSynchronize(s);
    dfree(dcnt);
    dfree(dcur);
    cleanup();
    if (e != cudaSuccess) {
        fb_tree_destroy(t);
        return fb_fail(FB_ERR_CUDA, std::string("tree build: ") + cudaGetErrorString(e));
    }
    *out = t;
    return FB_OK;
}

void fb_tree_free(fb_tree* t) {
    if (!t) return;
    dfree(t->perm);
    dfree(t->elem_pos);
    for (int l = 0; l <= FB_MAXLEV; ++l) {
        dfree(t->keys[l]);
        dfree(t->parent[l]);
        dfree(t->vcnt[l]);
        dfree(t->vlist[l]);
        dfree(t->oct_child[l]);
        dfree(t->oct_parent[l]);
    }
    dfree(t->leaf_start);
    dfree(t->ucnt);
    dfree(t->ulist);
    dfree(t->m2l_src);
    dfree(t->m2l_dst);
    for (auto& rs : t->rot_sets) {
        dfree(rs.r64);
        dfree(rs.d64);
        dfree(rs.d32);
        dfree(rs.ph64);
        dfree(rs.ph32);
    }
    delete t;
}

fb_status fb_tree_export_impl(const fb_tree* t, int which, int level, int64_t* out, int64_t* count) {
    if (!t || !count) return fb_fail(FB_ERR_ARG, "NULL argument");
    std::vector<int64_t> v;
    auto dl = [&](const void* src, size_t nbytes, void* dst) -> fb_status {
        FB_CUDA(cudaMemcpy(dst, src, nbytes, cudaMemcpyDeviceToHost));
        return FB_OK;
    };
    if (which == 0) {
        std::vector<int32_t> p(t->n);
        FB_CHECK(dl(t->perm, sizeof(int32_t) * t->n, p.data()));
        v.assign(p.begin(), p.end());
    } else if (which == 1) {
        v.assign(t->h_leaf_start.begin(), t->h_leaf_start.end());
    } else if (which == 2) {
        if (level < 0 || level > t->L) return fb_fail(FB_ERR_ARG, "level out of range");
        std::vector<uint32_t> k(t->nbox[level]);
        FB_CHECK(dl(t->keys[level], sizeof(uint32_t) * k.size(), k.data()));
        v.assign(k.begin(), k.end());
    } else if (which == 3 || which == 4) {
        int lev = which == 3 ? t->L : level;
        if (which == 4 && (lev < 2 || lev > t->L)) return fb_fail(FB_ERR_ARG, "level out of range");
        int nb = t->nbox[lev];
        int width = which == 3 ? FB_ULIST : FB_VLIST;
        std::vector<int32_t> c(nb), l((size_t)nb * width);
        FB_CHECK(dl(which == 3 ? t->ucnt : t->vcnt[lev], sizeof(int32_t) * nb, c.data()));
        FB_CHECK(dl(which == 3 ? t->ulist : t->vlist[lev], sizeof(int32_t) * l.size(), l.data()));
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < c[b]; ++i) {
                v.push_back(b);
                v.push_back(l[(size_t)b * width + i]);
            }
        *count = (int64_t)v.size() / 2;
        if (out) std::copy(v.begin(), v.end(), out);
        return FB_OK;
    } else {
        return fb_fail(FB_ERR_ARG, "unknown export");
    }
    *count = (int64_t)v.size();
    if (out) std::copy(v.begin(), v.end(), out);
    return FB_OK;
}
