// Leaf decomposition on the GPU: chaining mesh or recursive coordinate bisection
// (Sec. 3.1 names the RCB tree; Sec. 5.3 runs the kernels over leaf pairs),
// then the periodic leaf-pair image lists used by every pair kernel.
//
// RCB without per-node sorts: every particle is ranked once per axis by a
// stable radix sort of (coordinate, index).  Each level keeps three index
// lists, each sorted along its axis inside every node.  A node's tight box is
// read off the ends of its three segments; the split takes the first
// floor(n/2) of the chosen axis' segment, and the two other lists are
// stably partitioned by a prefix sum of the side flags.  The shape of the
// tree depends on n alone, so the host precomputes every level's segments.
#include <algorithm>
#include <cstring>

#include "crk_internal.cuh"

namespace {

constexpr int kMaxLeafCap = 1024;

__device__ __forceinline__ uint32_t coord_key(float x) {
    // x >= 0 after validation: the IEEE bits of non-negative floats are ordered like the values
    return x == 0.0f ? 0u : __float_as_uint(x);
}

__global__ void validate_kernel(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                                const uint8_t *__restrict__ sp, const float *__restrict__ h, int64_t n, float box,
                                int32_t *__restrict__ flags /* [0] bad pos, [1] bad h, [2] n_gas */,
                                unsigned *__restrict__ hmax_bits) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c[3] = {x[i], y[i], z[i]};
    bool bad = false;
    for (int a = 0; a < 3; ++a) bad |= !(c[a] >= 0.0f && c[a] < box);
    if (bad) atomicAdd(&flags[0], 1);
    if (sp[i] == 0) {
        float hi = h[i];
        if (!(hi > 0.0f) || !isfinite(hi)) atomicAdd(&flags[1], 1);
        else atomicMax(hmax_bits, __float_as_uint(hi));
        atomicAdd(&flags[2], 1);
    }
}

__global__ void init_axis_keys_kernel(const float *__restrict__ c, int64_t n, uint32_t *__restrict__ keys,
                                      int32_t *__restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = coord_key(c[i]);
    vals[i] = (int32_t)i;
}

// chaining mesh cell: c = min(nc-1, floor(x nc / L)) per axis in FP64, id = (cx nc + cy) nc + cz
__global__ void mesh_keys_kernel(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                                 int64_t n, int nc, double L, uint32_t *__restrict__ keys, int32_t *__restrict__ vals,
                                 int32_t *__restrict__ counts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c3[3] = {x[i], y[i], z[i]};
    int c[3];
    for (int a = 0; a < 3; ++a) {
        double f = floor(__ddiv_rn(__dmul_rn((double)c3[a], (double)nc), L));
        int ci = (int)f;
        c[a] = ci > nc - 1 ? nc - 1 : (ci < 0 ? 0 : ci);
    }
    uint32_t id = (uint32_t)((c[0] * nc + c[1]) * nc + c[2]);
    keys[i] = id;
    vals[i] = (int32_t)i;
    atomicAdd(&counts[id], 1);
}

// --- RCB level kernels ------------------------------------------------------
struct LevelDev {
    const int32_t *lo, *hi, *k, *child, *node;
    int32_t *axis;
};

__global__ void rcb_axis_kernel(int nseg, LevelDev lv, const int32_t *__restrict__ L0, const int32_t *__restrict__ L1,
                                const int32_t *__restrict__ L2, const float *__restrict__ x,
                                const float *__restrict__ y, const float *__restrict__ z, float *__restrict__ node_box) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int k = lv.k[s];
    if (k <= 0) return;
    int lo = lv.lo[s], hi = lv.hi[s];
    const int32_t *Ls[3] = {L0, L1, L2};
    const float *cs[3] = {x, y, z};
    float blo[3], bhi[3];
    double ext[3];
    for (int a = 0; a < 3; ++a) {
        blo[a] = cs[a][Ls[a][lo]];
        bhi[a] = cs[a][Ls[a][hi - 1]];
        ext[a] = __dsub_rn((double)bhi[a], (double)blo[a]);
    }
    int axis = 0;
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    lv.axis[s] = axis;
    float *nb = node_box + 6 * (int64_t)lv.node[s];
    for (int a = 0; a < 3; ++a) {
        nb[a] = blo[a];
        nb[3 + a] = bhi[a];
    }
}

__global__ void rcb_side_kernel(int64_t n, LevelDev lv, const int32_t *__restrict__ node_of,
                                const int32_t *__restrict__ L0, const int32_t *__restrict__ L1,
                                const int32_t *__restrict__ L2, uint8_t *__restrict__ side,
                                int32_t *__restrict__ node_of_next) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int s = node_of[p];
    int k = lv.k[s];
    int lo = lv.lo[s];
    int right = (k > 0 && (int)p - lo >= k) ? 1 : 0;
    if (k > 0) {
        int ax = lv.axis[s];
        const int32_t *L = ax == 0 ? L0 : (ax == 1 ? L1 : L2);
        side[L[p]] = (uint8_t)right;
    }
    node_of_next[p] = lv.child[s] + right;
}

__global__ void rcb_flag_kernel(int64_t n, LevelDev lv, const int32_t *__restrict__ node_of,
                                const int32_t *__restrict__ Lb, const uint8_t *__restrict__ side,
                                int32_t *__restrict__ flag) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int s = node_of[p];
    flag[p] = (lv.k[s] > 0 && side[Lb[p]] == 0) ? 1 : 0;
}

__global__ void rcb_scatter_kernel(int64_t n, LevelDev lv, const int32_t *__restrict__ node_of,
                                   const int32_t *__restrict__ Lb, const uint8_t *__restrict__ side,
                                   const int32_t *__restrict__ scan, int32_t *__restrict__ out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int s = node_of[p];
    int k = lv.k[s];
    int32_t id = Lb[p];
    if (k <= 0) {
        out[p] = id;
        return;
    }
    int lo = lv.lo[s];
    int lb = scan[p] - scan[lo];
    int np = side[id] == 0 ? lo + lb : lo + k + ((int)p - lo - lb);
    out[np] = id;
}

// --- per-leaf data ------------------------------------------------------------
// One block per leaf: canonical order (gas first, then dark matter, each by
// index), tight box, gas count, largest gas h, leaf-relative positions.
__global__ void leaf_data_kernel(int64_t n_leaves, const int32_t *__restrict__ leaf_start,
                                 const int32_t *__restrict__ members, const float *__restrict__ x,
                                 const float *__restrict__ y, const float *__restrict__ z,
                                 const uint8_t *__restrict__ sp, const float *__restrict__ h,
                                 int32_t *__restrict__ perm, int32_t *__restrict__ kperm,
                                 int32_t *__restrict__ leaf_ngas, float *__restrict__ bbox,
                                 float *__restrict__ hmax, float4 *__restrict__ pos, int32_t *__restrict__ err) {
    __shared__ uint64_t key[kMaxLeafCap];
    __shared__ float red[6][32];
    __shared__ int ngs[32];
    __shared__ float hms[32];
    const int64_t a = blockIdx.x;
    if (a >= n_leaves) return;
    const int lo = leaf_start[a], hi = leaf_start[a + 1], cnt = hi - lo;
    if (cnt > kMaxLeafCap) {
        if (threadIdx.x == 0) atomicAdd(err, 1);
        return;
    }
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int32_t id = members[lo + t];
        key[t] = ((uint64_t)(sp[id] != 0) << 32) | (uint32_t)id;
    }
    __syncthreads();
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int ng = 0;
    float hm = 0.0f;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        uint64_t kt = key[t];
        int r = 0;
        for (int u = 0; u < cnt; ++u) r += key[u] < kt;
        int32_t id = (int32_t)(uint32_t)kt;
        perm[lo + r] = id;
        kperm[lo + r] = id;
        float c[3] = {x[id], y[id], z[id]};
        for (int q = 0; q < 3; ++q) {
            mn[q] = fminf(mn[q], c[q]);
            mx[q] = fmaxf(mx[q], c[q]);
        }
        if (sp[id] == 0) {
            ++ng;
            hm = fmaxf(hm, h[id]);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        for (int q = 0; q < 3; ++q) {
            mn[q] = fminf(mn[q], __shfl_xor_sync(CRK_FULL_MASK, mn[q], o));
            mx[q] = fmaxf(mx[q], __shfl_xor_sync(CRK_FULL_MASK, mx[q], o));
        }
        ng += __shfl_xor_sync(CRK_FULL_MASK, ng, o);
        hm = fmaxf(hm, __shfl_xor_sync(CRK_FULL_MASK, hm, o));
    }
    if (lane == 0) {
        for (int q = 0; q < 3; ++q) {
            red[q][w] = mn[q];
            red[3 + q][w] = mx[q];
        }
        ngs[w] = ng;
        hms[w] = hm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 1; v < nw; ++v) {
            for (int q = 0; q < 3; ++q) {
                red[q][0] = fminf(red[q][0], red[q][v]);
                red[3 + q][0] = fmaxf(red[3 + q][0], red[3 + q][v]);
            }
            ngs[0] += ngs[v];
            hms[0] = fmaxf(hms[0], hms[v]);
        }
        for (int q = 0; q < 6; ++q) bbox[6 * a + q] = red[q][0];
        leaf_ngas[a] = ngs[0];
        hmax[a] = hms[0];
    }
    __syncthreads();
    const float ox = red[0][0], oy = red[1][0], oz = red[2][0];
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int32_t id = kperm[lo + t];
        pos[lo + t] = make_float4(x[id] - ox, y[id] - oy, z[id] - oz, sp[id] == 0 ? h[id] : 0.0f);
    }
}

// --- leaf-pair images ------------------------------------------------------------
struct TreeDev {
    const float *node_box;       // [nodes][6]
    const int32_t *node_left;    // child ids, -1 for leaves
    const int32_t *node_right;
    const int32_t *node_leaf;    // leaf id for leaves, -1 otherwise
    int32_t root;
};

__device__ __forceinline__ double axis_gap_shift(double loa, double hia, double lob, double hib, double s) {
    double t1 = __dsub_rn(__dadd_rn(lob, s), hia);
    double t2 = __dsub_rn(__dsub_rn(loa, hib), s);
    double g = t1 > t2 ? t1 : t2;
    return g < 0.0 ? 0.0 : g;
}

__device__ __forceinline__ double axis_gap(double loa, double hia, double lob, double hib, double L) {
    double g0 = axis_gap_shift(loa, hia, lob, hib, -L);
    double g1 = axis_gap_shift(loa, hia, lob, hib, 0.0);
    double g2 = axis_gap_shift(loa, hia, lob, hib, L);
    double g = g0 < g1 ? g0 : g1;
    return g < g2 ? g : g2;
}

__device__ __forceinline__ double sum_sq(double gx, double gy, double gz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
}

// Emits the images of leaf b that lie within `cut` of leaf a; returns how many.
template <bool kFill>
__device__ int leaf_images(const float *__restrict__ bbox, int64_t a, int64_t b, double L, double cut2,
                           crk_image *__restrict__ out) {
    const float *A = bbox + 6 * a, *B = bbox + 6 * b;
    double g[3][3];
    for (int q = 0; q < 3; ++q) {
        g[q][0] = axis_gap_shift(A[q], A[3 + q], B[q], B[3 + q], -L);
        g[q][1] = axis_gap_shift(A[q], A[3 + q], B[q], B[3 + q], 0.0);
        g[q][2] = axis_gap_shift(A[q], A[3 + q], B[q], B[3 + q], L);
    }
    int cnt = 0;
    for (int ix = 0; ix < 3; ++ix)
        for (int iy = 0; iy < 3; ++iy)
            for (int iz = 0; iz < 3; ++iz) {
                double d2 = sum_sq(g[0][ix], g[1][iy], g[2][iz]);
                if (d2 < cut2) {
                    if (kFill) {
                        crk_image im;
                        im.b = (int32_t)b;
                        double sx = (ix - 1) * L, sy = (iy - 1) * L, sz = (iz - 1) * L;
                        im.sx = (float)__dsub_rn(__dadd_rn((double)B[0], sx), (double)A[0]);
                        im.sy = (float)__dsub_rn(__dadd_rn((double)B[1], sy), (double)A[1]);
                        im.sz = (float)__dsub_rn(__dadd_rn((double)B[2], sz), (double)A[2]);
                        out[cnt] = im;
                    }
                    ++cnt;
                }
            }
    return cnt;
}

template <bool kFill>
__global__ void pairs_kernel(int64_t n_leaves, const int32_t *__restrict__ leaf_start,
                             const int32_t *__restrict__ leaf_ngas, const float *__restrict__ bbox,
                             const float *__restrict__ hmax, TreeDev tree, int brute, int hydro, double L,
                             double rc, double hmax_all, int32_t *__restrict__ img_cnt, int32_t *__restrict__ pair_cnt,
                             const int32_t *__restrict__ img_ptr, crk_image *__restrict__ img,
                             const int32_t *__restrict__ pair_ptr, int32_t *__restrict__ pair_list) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_leaves) return;
    int ni = 0, np = 0;
    crk_image *io = kFill ? img + img_ptr[a] : nullptr;
    int32_t *po = kFill ? pair_list + pair_ptr[a] : nullptr;
    const bool a_ok = leaf_start[a + 1] > leaf_start[a] && (!hydro || leaf_ngas[a] > 0);
    if (a_ok) {
        const float *A = bbox + 6 * a;
        const double ha = hydro ? (double)hmax[a] : 0.0;
        auto visit_leaf = [&](int64_t b) {
            if (leaf_start[b + 1] == leaf_start[b]) return;
            if (hydro && leaf_ngas[b] == 0) return;
            double cut = rc;
            if (hydro) {
                double hb = (double)hmax[b];
                cut = __dmul_rn(2.0, ha > hb ? ha : hb);
            }
            int c = leaf_images<kFill>(bbox, a, b, L, __dmul_rn(cut, cut), kFill ? io + ni : nullptr);
            if (c > 0) {
                if (kFill) po[np] = (int32_t)b;
                ni += c;
                np += 1;
            }
        };
        if (brute) {
            for (int64_t b = 0; b < n_leaves; ++b) visit_leaf(b);
        } else {
            double cutn = hydro ? 2.0 * (ha > hmax_all ? ha : hmax_all) : rc;
            double cutn2 = cutn * cutn * (1.0 + 1e-12);
            int32_t stack[64];
            int top = 0;
            stack[top++] = tree.root;
            while (top > 0) {
                int32_t nd = stack[--top];
                const float *Nb = tree.node_box + 6 * (int64_t)nd;
                double gx = axis_gap(A[0], A[3], Nb[0], Nb[3], L);
                double gy = axis_gap(A[1], A[4], Nb[1], Nb[4], L);
                double gz = axis_gap(A[2], A[5], Nb[2], Nb[5], L);
                if (!(sum_sq(gx, gy, gz) < cutn2)) continue;
                int32_t lf = tree.node_leaf[nd];
                if (lf >= 0) {
                    visit_leaf(lf);
                } else if (top + 2 <= 64) {
                    stack[top++] = tree.node_right[nd];
                    stack[top++] = tree.node_left[nd];
                }
            }
        }
    }
    if (!kFill) {
        img_cnt[a] = ni;
        pair_cnt[a] = np;
    }
}

__global__ void leaf_box_to_node_kernel(int64_t n_leaves, const float *__restrict__ bbox,
                                        const int32_t *__restrict__ leaf_node, float *__restrict__ node_box) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_leaves) return;
    for (int q = 0; q < 6; ++q) node_box[6 * (int64_t)leaf_node[a] + q] = bbox[6 * a + q];
}

struct HostSeg {
    int32_t lo, hi, k, child, node;
};

}  // namespace

// ---------------------------------------------------------------------------------
static int upload(crk_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return CRK_OK;
    CRK_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return CRK_OK;
}

int crk_build_leaves(crk_ctx *ctx, const crk_particles *p, const float *h, const crk_leaf_params *lp,
                     crk_leaves **out) {
    if (!ctx) return CRK_EINVAL;
    if (!p || !lp || !out) return crk_fail(ctx, CRK_EINVAL, "null argument");
    *out = nullptr;
    const int64_t n = p->n;
    if (n < 0 || n > 2000000000LL) return crk_fail(ctx, CRK_EINVAL, "particle count out of range");
    if (n > 0 && (!p->x || !p->y || !p->z || !p->species || !h)) return crk_fail(ctx, CRK_EINVAL, "null array");
    if (!(p->box > 0.0f)) return crk_fail(ctx, CRK_EINVAL, "box must be positive");
    if (lp->mode != 0 && lp->mode != 1) return crk_fail(ctx, CRK_EINVAL, "leaf mode must be 0 or 1");
    if (lp->mode == 0 && (lp->cells_per_side < 1 || lp->cells_per_side > 40))
        return crk_fail(ctx, CRK_EINVAL, "cells_per_side must be in [1, 40]");
    if (lp->mode == 1 && (lp->max_leaf < 1 || lp->max_leaf > kMaxLeafCap))
        return crk_fail(ctx, CRK_EINVAL, "max_leaf must be in [1, 1024]");
    if (!(lp->r_cut_grav > 0.0f) || !((double)lp->r_cut_grav < 0.5 * (double)p->box))
        return crk_fail(ctx, CRK_EBOX, "r_cut_grav must be positive and below box/2");

    crk_leaves *lv = new crk_leaves();
    lv->n = n;
    lv->box = p->box;
    lv->mode = lp->mode;
    lv->r_cut_grav = lp->r_cut_grav;
    cudaStream_t st = ctx->stream;
    int rc = CRK_OK;
#define TRY(expr)                          \
    do {                                   \
        rc = (expr);                       \
        if (rc != CRK_OK) goto fail;       \
    } while (0)
#define ALLOC(ptr, type, count)                                                          \
    do {                                                                                 \
        ptr = (type *)crk_leaves_alloc(ctx, lv, sizeof(type) * (size_t)((count) > 0 ? (count) : 1)); \
        if (!ptr) { rc = crk_fail(ctx, CRK_ENOMEM, "leaf allocation"); goto fail; }      \
    } while (0)
    {
        // ---- validation flags
        int32_t *flags = (int32_t *)crk_scratch(ctx, 0, 64);
        if (!flags) { rc = crk_fail(ctx, CRK_ENOMEM, "scratch"); goto fail; }
        if (cudaMemsetAsync(flags, 0, 64, st) != cudaSuccess) { rc = crk_fail(ctx, CRK_ECUDA, "memset"); goto fail; }
        unsigned *hbits = (unsigned *)(flags + 8);
        if (n > 0)
            validate_kernel<<<crk_grid(n, 256), 256, 0, st>>>(p->x, p->y, p->z, p->species, h, n, p->box, flags, hbits);
        ctx->launches += n > 0;

        std::vector<int32_t> h_leaf_start;  // host copy of leaf boundaries (RCB known from the shape)
        int32_t *members = nullptr;         // device: particle ids grouped by leaf
        int64_t nl = 0;
        // tree for traversal (RCB)
        std::vector<int32_t> n_left, n_right, n_leaf, leaf_node;
        float *node_box = nullptr;
        int32_t root = 0;

        if (lp->mode == 0) {
            int nc = lp->cells_per_side;
            nl = (int64_t)nc * nc * nc;
            uint32_t *keys = (uint32_t *)crk_scratch(ctx, 1, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
            int32_t *vals = (int32_t *)crk_scratch(ctx, 2, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            int32_t *cnts = (int32_t *)crk_scratch(ctx, 3, sizeof(int32_t) * (size_t)(nl + 1));
            if (!keys || !vals || !cnts) { rc = crk_fail(ctx, CRK_ENOMEM, "scratch"); goto fail; }
            ALLOC(lv->leaf_start, int32_t, nl + 1);
            if (cudaMemsetAsync(cnts, 0, sizeof(int32_t) * (size_t)(nl + 1), st) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "memset");
                goto fail;
            }
            if (n > 0)
                mesh_keys_kernel<<<crk_grid(n, 256), 256, 0, st>>>(p->x, p->y, p->z, n, nc, (double)p->box, keys,
                                                                   vals, cnts);
            ctx->launches += n > 0;
            int bits = 1;
            while ((1LL << bits) < nl) ++bits;
            TRY(crk_radix_sort_u32(ctx, keys, vals, n, bits));
            TRY(crk_exclusive_scan_i32(ctx, cnts, lv->leaf_start, nl + 1, nullptr));
            members = vals;
        } else {
            // host: tree shape from n alone
            const int ml = lp->max_leaf;
            std::vector<std::vector<HostSeg>> levels;
            std::vector<HostSeg> cur;
            int32_t next_node = 0;
            if (n > 0) cur.push_back({0, (int32_t)n, 0, 0, next_node++});
            n_left.assign(1, -1);
            n_right.assign(1, -1);
            bool any = true;
            while (any && !cur.empty()) {
                any = false;
                for (auto &s : cur)
                    if (s.hi - s.lo > ml) { s.k = (s.hi - s.lo) / 2; any = true; }
                if (!any) break;
                std::vector<HostSeg> nxt;
                nxt.reserve(cur.size() * 2);
                for (auto &s : cur) {
                    s.child = (int32_t)nxt.size();
                    if (s.k > 0) {
                        int32_t l = next_node++, r = next_node++;
                        n_left.resize(next_node, -1);
                        n_right.resize(next_node, -1);
                        n_left[s.node] = l;
                        n_right[s.node] = r;
                        nxt.push_back({s.lo, s.lo + s.k, 0, 0, l});
                        nxt.push_back({s.lo + s.k, s.hi, 0, 0, r});
                    } else {
                        nxt.push_back({s.lo, s.hi, 0, 0, s.node});
                    }
                }
                levels.push_back(cur);
                cur.swap(nxt);
            }
            // cur now lists the leaves in position (= depth-first) order
            nl = (int64_t)cur.size();
            n_leaf.assign(next_node, -1);
            h_leaf_start.resize(nl + 1);
            leaf_node.resize(nl);
            for (int64_t a = 0; a < nl; ++a) {
                h_leaf_start[a] = cur[a].lo;
                n_leaf[cur[a].node] = (int32_t)a;
                leaf_node[a] = cur[a].node;
            }
            h_leaf_start[nl] = (int32_t)n;
            ALLOC(lv->leaf_start, int32_t, nl + 1);
            TRY(upload(ctx, lv->leaf_start, h_leaf_start.data(), sizeof(int32_t) * (size_t)(nl + 1)));
            ALLOC(node_box, float, 6 * (int64_t)next_node);
            // three presorted lists
            int32_t *Lc[3], *Ln[3];
            uint32_t *keys = (uint32_t *)crk_scratch(ctx, 1, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
            for (int a = 0; a < 3; ++a) {
                Lc[a] = (int32_t *)crk_scratch(ctx, 2 + a, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
                Ln[a] = (int32_t *)crk_scratch(ctx, 5 + a, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            }
            int32_t *node_of = (int32_t *)crk_scratch(ctx, 8, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            int32_t *node_nx = (int32_t *)crk_scratch(ctx, 9, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            uint8_t *side = (uint8_t *)crk_scratch(ctx, 10, (size_t)(n > 0 ? n : 1));
            int32_t *flag = (int32_t *)crk_scratch(ctx, 11, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            if (!keys || !node_of || !node_nx || !side || !flag || !Lc[0] || !Lc[1] || !Lc[2] || !Ln[0] || !Ln[1] ||
                !Ln[2]) {
                rc = crk_fail(ctx, CRK_ENOMEM, "scratch");
                goto fail;
            }
            const float *cs[3] = {p->x, p->y, p->z};
            for (int a = 0; a < 3 && n > 0; ++a) {
                init_axis_keys_kernel<<<crk_grid(n, 256), 256, 0, st>>>(cs[a], n, keys, Lc[a]);
                ++ctx->launches;
                TRY(crk_radix_sort_u32(ctx, keys, Lc[a], n, 32));
            }
            if (n > 0 && cudaMemsetAsync(node_of, 0, sizeof(int32_t) * (size_t)n, st) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "memset");
                goto fail;
            }
            // device copies of the level tables (one buffer for all levels)
            size_t tot = 0;
            for (auto &L : levels) tot += L.size();
            std::vector<int32_t> packed(6 * (tot > 0 ? tot : 1));
            int32_t *dtab;
            ALLOC(dtab, int32_t, 6 * (int64_t)(tot > 0 ? tot : 1));
            {
                size_t off = 0;
                for (auto &L : levels) {
                    size_t m = L.size();
                    for (size_t s = 0; s < m; ++s) {
                        packed[off + s] = L[s].lo;
                        packed[off + m + s] = L[s].hi;
                        packed[off + 2 * m + s] = L[s].k;
                        packed[off + 3 * m + s] = L[s].child;
                        packed[off + 4 * m + s] = L[s].node;
                        packed[off + 5 * m + s] = 0;
                    }
                    off += 6 * m;
                }
                TRY(upload(ctx, dtab, packed.data(), sizeof(int32_t) * 6 * tot));
            }
            size_t off = 0;
            for (auto &L : levels) {
                int m = (int)L.size();
                LevelDev d;
                d.lo = dtab + off;
                d.hi = dtab + off + m;
                d.k = dtab + off + 2 * m;
                d.child = dtab + off + 3 * m;
                d.node = dtab + off + 4 * m;
                d.axis = dtab + off + 5 * m;
                off += 6 * (size_t)m;
                rcb_axis_kernel<<<crk_grid(m, 128), 128, 0, st>>>(m, d, Lc[0], Lc[1], Lc[2], p->x, p->y, p->z,
                                                                  node_box);
                rcb_side_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, d, node_of, Lc[0], Lc[1], Lc[2], side, node_nx);
                ctx->launches += 2 + 2 * 3;
                for (int b = 0; b < 3; ++b) {
                    rcb_flag_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, d, node_of, Lc[b], side, flag);
                    TRY(crk_exclusive_scan_i32(ctx, flag, flag, n, nullptr));
                    rcb_scatter_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, d, node_of, Lc[b], side, flag, Ln[b]);
                }
                for (int b = 0; b < 3; ++b) std::swap(Lc[b], Ln[b]);
                std::swap(node_of, node_nx);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) { rc = crk_check_cuda(ctx, e, "rcb level"); goto fail; }
            }
            members = Lc[0];
            root = 0;
        }
        lv->n_leaves = nl;
        ALLOC(lv->perm, int32_t, n);
        ALLOC(lv->kperm, int32_t, n);
        ALLOC(lv->leaf_ngas, int32_t, nl);
        ALLOC(lv->bbox, float, 6 * nl);
        ALLOC(lv->hmax, float, nl);
        ALLOC(lv->pos, float4, n);
        int32_t *err_flag = flags + 4;
        if (nl > 0)
            leaf_data_kernel<<<(unsigned)nl, 128, 0, st>>>(nl, lv->leaf_start, members, p->x, p->y, p->z,
                                                           p->species, h, lv->perm, lv->kperm, lv->leaf_ngas,
                                                           lv->bbox, lv->hmax, lv->pos, err_flag);
        ctx->launches += nl > 0;
        {
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { rc = crk_check_cuda(ctx, e, "leaf data"); goto fail; }
        }
        // ---- host checks (one synchronisation)
        int32_t hflags[16];
        if (cudaMemcpyAsync(hflags, flags, 64, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = crk_fail(ctx, CRK_ECUDA, "leaf build: %s", cudaGetErrorString(cudaGetLastError()));
            goto fail;
        }
        if (hflags[0] > 0) { rc = crk_fail(ctx, CRK_EBOX, "%d particle positions outside [0, box)", hflags[0]); goto fail; }
        if (hflags[1] > 0) { rc = crk_fail(ctx, CRK_EINVAL, "%d gas particles with h <= 0 or not finite", hflags[1]); goto fail; }
        if (hflags[4] > 0) { rc = crk_fail(ctx, CRK_EINVAL, "a leaf holds more than %d particles", kMaxLeafCap); goto fail; }
        lv->n_gas = hflags[2];
        float hmax_all;
        std::memcpy(&hmax_all, &hflags[8], sizeof(float));
        lv->hmax_all = hmax_all;
        if (!(2.0 * (double)hmax_all < 0.5 * (double)p->box)) {
            rc = crk_fail(ctx, CRK_EBOX, "2 h_max = %g is not below box/2", 2.0 * hmax_all);
            goto fail;
        }
        if (lp->mode == 0) {
            std::vector<int32_t> ls(nl + 1);
            if (cudaMemcpy(ls.data(), lv->leaf_start, sizeof(int32_t) * (nl + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "leaf starts");
                goto fail;
            }
            int mx = 0;
            for (int64_t a = 0; a < nl; ++a) mx = std::max(mx, ls[a + 1] - ls[a]);
            lv->max_leaf_size = mx;
            if (mx > kMaxLeafCap) { rc = crk_fail(ctx, CRK_EINVAL, "a chaining-mesh cell holds more than %d particles", kMaxLeafCap); goto fail; }
        } else {
            int mx = 0;
            for (int64_t a = 0; a < nl; ++a) mx = std::max(mx, h_leaf_start[a + 1] - h_leaf_start[a]);
            lv->max_leaf_size = mx;
        }

        // ---- tree arrays for traversal
        TreeDev tree{};
        int brute = lp->mode == 0 ? 1 : 0;
        if (!brute && nl > 0) {
            int32_t *dl, *dr, *dlf, *dln;
            int64_t nn = (int64_t)n_left.size();
            ALLOC(dl, int32_t, nn);
            ALLOC(dr, int32_t, nn);
            ALLOC(dlf, int32_t, nn);
            ALLOC(dln, int32_t, nl);
            TRY(upload(ctx, dl, n_left.data(), sizeof(int32_t) * nn));
            TRY(upload(ctx, dr, n_right.data(), sizeof(int32_t) * nn));
            TRY(upload(ctx, dlf, n_leaf.data(), sizeof(int32_t) * nn));
            TRY(upload(ctx, dln, leaf_node.data(), sizeof(int32_t) * nl));
            leaf_box_to_node_kernel<<<crk_grid(nl, 128), 128, 0, st>>>(nl, lv->bbox, dln, node_box);
            ++ctx->launches;
            tree.node_box = node_box;
            tree.node_left = dl;
            tree.node_right = dr;
            tree.node_leaf = dlf;
            tree.root = root;
        }
        // ---- image lists: count, scan, fill (gravity then hydro)
        for (int hyd = 0; hyd < 2; ++hyd) {
            int32_t *icnt = (int32_t *)crk_scratch(ctx, 1, sizeof(int32_t) * (size_t)(nl + 1));
            int32_t *pcnt = (int32_t *)crk_scratch(ctx, 2, sizeof(int32_t) * (size_t)(nl + 1));
            int32_t *tot2 = (int32_t *)crk_scratch(ctx, 3, 64);
            if (!icnt || !pcnt || !tot2) { rc = crk_fail(ctx, CRK_ENOMEM, "scratch"); goto fail; }
            int32_t *iptr, *pptr;
            ALLOC(iptr, int32_t, nl + 1);
            ALLOC(pptr, int32_t, nl + 1);
            if (nl > 0)
                pairs_kernel<false><<<crk_grid(nl, 128), 128, 0, st>>>(nl, lv->leaf_start, lv->leaf_ngas, lv->bbox,
                                                                     lv->hmax, tree, brute, hyd, (double)p->box,
                                                                     (double)lp->r_cut_grav, (double)hmax_all, icnt,
                                                                     pcnt, nullptr, nullptr, nullptr, nullptr);
            else {
                if (cudaMemsetAsync(icnt, 0, sizeof(int32_t), st) != cudaSuccess) { rc = crk_fail(ctx, CRK_ECUDA, "memset"); goto fail; }
                if (cudaMemsetAsync(pcnt, 0, sizeof(int32_t), st) != cudaSuccess) { rc = crk_fail(ctx, CRK_ECUDA, "memset"); goto fail; }
            }
            ctx->launches += nl > 0;
            TRY(crk_exclusive_scan_i32(ctx, icnt, iptr, nl + 1, tot2));
            TRY(crk_exclusive_scan_i32(ctx, pcnt, pptr, nl + 1, tot2 + 1));
            int32_t tots[2];
            if (cudaMemcpyAsync(tots, tot2, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "pair counts: %s", cudaGetErrorString(cudaGetLastError()));
                goto fail;
            }
            // scan of nl+1 entries where the last count is garbage: recompute totals from ptr[nl]
            int32_t ni = 0, np = 0;
            if (nl > 0) {
                if (cudaMemcpy(&ni, iptr + nl, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(&np, pptr + nl, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
                    rc = crk_fail(ctx, CRK_ECUDA, "pair totals");
                    goto fail;
                }
            }
            crk_image *img;
            int32_t *plist;
            ALLOC(img, crk_image, ni);
            ALLOC(plist, int32_t, np);
            if (nl > 0)
                pairs_kernel<true><<<crk_grid(nl, 128), 128, 0, st>>>(nl, lv->leaf_start, lv->leaf_ngas, lv->bbox,
                                                                    lv->hmax, tree, brute, hyd, (double)p->box,
                                                                    (double)lp->r_cut_grav, (double)hmax_all, nullptr,
                                                                    nullptr, iptr, img, pptr, plist);
            ctx->launches += nl > 0;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { rc = crk_check_cuda(ctx, e, "pair lists"); goto fail; }
            if (hyd == 0) {
                lv->gimg_ptr = iptr; lv->gimg = img; lv->n_gimg = ni;
                lv->gpair_ptr = pptr; lv->gpair_list = plist; lv->n_gpairs = np;
            } else {
                lv->himg_ptr = iptr; lv->himg = img; lv->n_himg = ni;
                lv->hpair_ptr = pptr; lv->hpair_list = plist; lv->n_hpairs = np;
            }
        }
    }
#undef TRY
#undef ALLOC
    *out = lv;
    return CRK_OK;
fail:
    crk_leaves_free(ctx, lv);
    return rc;
}

int crk_leaves_info(const crk_leaves *lv, int64_t info[6]) {
    if (!lv || !info) return CRK_EINVAL;
    info[0] = lv->n;
    info[1] = lv->n_leaves;
    info[2] = lv->n_gpairs;
    info[3] = lv->n_hpairs;
    info[4] = lv->n_gimg;
    info[5] = lv->n_himg;
    return CRK_OK;
}

int crk_leaves_export(crk_ctx *ctx, const crk_leaves *lv, int32_t *perm, int32_t *leaf_start, int32_t *grav_ptr,
                      int32_t *grav_list, int32_t *hydro_ptr, int32_t *hydro_list) {
    if (!ctx) return CRK_EINVAL;
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null leaves");
    CRK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    struct {
        void *dst;
        const void *src;
        size_t bytes;
    } cp[6] = {{perm, lv->perm, sizeof(int32_t) * (size_t)lv->n},
               {leaf_start, lv->leaf_start, sizeof(int32_t) * (size_t)(lv->n_leaves + 1)},
               {grav_ptr, lv->gpair_ptr, sizeof(int32_t) * (size_t)(lv->n_leaves + 1)},
               {grav_list, lv->gpair_list, sizeof(int32_t) * (size_t)lv->n_gpairs},
               {hydro_ptr, lv->hpair_ptr, sizeof(int32_t) * (size_t)(lv->n_leaves + 1)},
               {hydro_list, lv->hpair_list, sizeof(int32_t) * (size_t)lv->n_hpairs}};
    for (auto &c : cp)
        if (c.dst && c.bytes && c.src) CRK_CUDA(ctx, cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost));
    return CRK_OK;
}

void crk_leaves_free(crk_ctx *ctx, crk_leaves *lv) {
    (void)ctx;
    if (!lv) return;
    for (void *q : lv->allocs) cudaFree(q);
    delete lv;
}
