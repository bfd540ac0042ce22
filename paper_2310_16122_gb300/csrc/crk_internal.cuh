// Internal declarations of libcrk (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/crk.h"

#define CRK_WARP 32
#define CRK_FULL_MASK 0xffffffffu

// One periodic image of a j-leaf as seen from an i-leaf: adding (sx, sy, sz)
// to the j-leaf's leaf-relative coordinates expresses them in the i-leaf frame.
struct crk_image {
    int32_t b;
    float sx, sy, sz;
};

// Shape of an RCB tree: with the left child taking floor(n/2) it depends on
// the particle count and the leaf capacity only, so it is computed once on
// the host and cached (with its device copies) in the context.
struct crk_rcb_shape {
    int64_t n = -1;
    int max_leaf = 0;
    std::vector<int64_t> box_start;             // the boxes this shape was built for
    std::vector<int32_t> box_root;              // root node of each box (-1 for an empty box)
    std::vector<int32_t> leaf_box;              // box of each leaf (host copy)
    int64_t n_leaves = 0, n_nodes = 0;
    int max_leaf_size = 0;
    std::vector<size_t> level_off, level_size;  // segment tables, 7 int32 columns per level
    std::vector<int32_t> level_max;             // largest segment of each level
    int32_t *dtab = nullptr;                    // device: lo, hi, k, child, node, axis, leftbase per segment
    int32_t *leaf_start = nullptr;              // device [n_leaves + 1]
    int32_t *left = nullptr, *right = nullptr;  // device [n_nodes], -1 for leaves
    int32_t *leaf_of = nullptr;                 // device [n_nodes], leaf id or -1
    int32_t *leaf_node = nullptr;               // device [n_leaves]
    int32_t *d_leaf_box = nullptr;              // device [n_leaves]
    int32_t *d_box_root = nullptr;              // device [nbox]
};

struct crk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    // growable scratch arena: one buffer per slot
    static const int kSlots = 38;  // leaf build 0-16 and 19-31, radix sort 12-14, scan 15, queue 17, step 18,
                                   // integrator 32, corrections adjoint 33, adjoint chain 34, half-warp force 35,
                                   // tuner 36, split-sweep candidates 37
    void *slot[kSlots] = {};
    size_t slot_bytes[kSlots] = {};
    int64_t launches = 0;  // kernels this context has launched
    // device blocks released by crk_leaves_free, reused by later leaf builds
    // on this context (stream order makes the reuse safe)
    std::vector<std::pair<void *, size_t>> block_cache;
    crk_rcb_shape *rcb = nullptr;
    bool trace = false;  // CRK_TRACE=1: synchronise and print phase times of the leaf build
    // launch shape of each pair kernel (autotuner choices), indexed by CRK_K_*: persistent grid +
    // atomic work queue, and the j-tile depth of the gravity tiles sweeps
    int persist[CRK_N_KERNELS] = {};
    int depth[CRK_N_KERNELS] = {32, 32, 32, 32, 32, 32, 32, 32, 32};
    int warps[CRK_N_KERNELS] = {4, 4, 4, 4, 4, 4, 4, 4, 4};  // warps per i-leaf of the packed gravity tiles
    // crk_step profiling: 8 events per step (start, after each of the 6 stages, end)
    std::vector<cudaEvent_t> prof_ev;
    int prof_max = 0, prof_used = 0;
    // kernel variants (autotuner choices), indexed by CRK_K_*; 0 = default
    int variant[CRK_N_KERNELS] = {};
};

struct crk_nlist {
    int32_t *gstart = nullptr;  // [n_leaves + 1] first group of each leaf
    int32_t *gleaf = nullptr;   // [groups] leaf of each group
    int32_t *goff = nullptr;    // [groups + 1] list row offsets, units of 32 entries
    int32_t *cnt = nullptr;     // [n] list length per kernel-order position
    uint16_t *list = nullptr;   // per-lane indices into the group's j table, k-major rows of 32
    int32_t *uoff = nullptr;    // [groups + 1] first j-table entry of each group
    int32_t *unum = nullptr;    // [groups] j-table size of each group
    uint32_t *ucode = nullptr;  // j-table entries: image << 10 | j inside the j-leaf
    int64_t groups = 0, entries = 0, table = 0;  // groups: the capacity of the group arrays
    int32_t *dgroups = nullptr;  // device: groups of the last build (at most `groups`)
    bool onepass = false;        // fixed capacities per group (a rebuild can reuse them)
};

struct crk_leaves {
    int64_t n = 0;
    int64_t n_gas = 0;
    int64_t n_leaves = 0;
    float box = 0.f;  // largest box side
    int nbox = 1;
    int mode = 1;
    float r_cut_grav = 0.f;
    float hmax_all = 0.f;
    int max_leaf_size = 0;  // largest leaf population
    // device arrays
    int32_t *perm = nullptr;        // canonical order -> original index
    int32_t *kperm = nullptr;       // kernel order -> original index
    int32_t *leaf_start = nullptr;  // [n_leaves + 1]
    int32_t *leaf_ngas = nullptr;   // [n_leaves]
    float *bbox = nullptr;          // [n_leaves][6]: lo xyz, hi xyz
    float *hmax = nullptr;          // [n_leaves]
    float4 *pos = nullptr;          // [n] kernel order: leaf-relative x, y, z and h (gas) or 0
    int32_t *kperm_g = nullptr;     // gravity kernel order (species mixed) -> original index
    int32_t *kinv = nullptr;        // original index -> kernel order position (inverse of kperm)
    int32_t *kinv_g = nullptr;      // original index -> gravity kernel order position
    float4 *pos_g = nullptr;        // [n] gravity kernel order: leaf-relative x, y, z and h or 0
    // leaf-pair lists: per i-leaf a, entries [start[a], start[a] + count[a]) in
    // ascending j-leaf order (leaves may be laid out in any order)
    int32_t *gimg_start = nullptr, *gimg_cnt = nullptr;  // gravity images
    crk_image *gimg = nullptr;
    int32_t *himg_start = nullptr, *himg_cnt = nullptr;  // hydro images
    crk_image *himg = nullptr;
    int32_t *gpair_start = nullptr, *gpair_cnt = nullptr, *gpair_list = nullptr;  // canonical gravity pairs
    int32_t *hpair_start = nullptr, *hpair_cnt = nullptr, *hpair_list = nullptr;  // canonical hydro pairs
    int64_t n_gimg = 0, n_himg = 0, n_gpairs = 0, n_hpairs = 0;
    // exact neighbour lists (decided in FP32 exactly as the kernels decide the
    // range): gas pairs r < h_i + h_j, and gravity pairs r < r_cut.  One block
    // per group of 32 consecutive particles of a leaf in kernel order (gas
    // prefix only for the gas lists), stored k-major (entry k of lane l at
    // k*32 + l); an entry is (image index in the leaf's image list << 10) |
    // index of j inside its leaf
    crk_nlist gas_lists, grav_lists;
    std::vector<std::pair<void *, size_t>> allocs;
    // what a capture-safe rebuild (crk_leaves_rebuild) reuses
    int max_leaf = 0, cells = 0;
    bool cells8 = false;  // gravity order bisected down to RCB cells of 8 (split gravity sweeps)
    std::vector<int64_t> box_start;
    std::vector<float> box_side;
    float *node_box = nullptr, *node_hmax = nullptr;  // RCB traversal tree: node boxes and h_max
    int64_t img_cap[4] = {0, 0, 0, 0};               // capacities of gimg, gpair, himg, hpair
    unsigned char *boxtab = nullptr;                  // device copy of the build's box-table block
    size_t boxtab_bytes = 0;
    // device: [0] status bits, [1] gas groups, [2] gravity groups; [16..27] the six list cursors (u64)
    int32_t *dev = nullptr;
};

// ---- host helpers (api.cu) ----
int crk_fail(crk_ctx *ctx, int code, const char *fmt, ...);
int crk_check_cuda(crk_ctx *ctx, cudaError_t e, const char *what);
void *crk_scratch(crk_ctx *ctx, int slot, size_t bytes);
void *crk_leaves_alloc(crk_ctx *ctx, crk_leaves *lv, size_t bytes);
void crk_rcb_shape_free(crk_ctx *ctx);
// neighbour lists of the leaves; reuse: a rebuild into the buffers of the first build (no host
// synchronisation; a capacity overflow sets a bit of the leaves' status word)
int crk_build_lists(crk_ctx *ctx, crk_leaves *lv, bool gas, bool reuse);
int crk_step_fused(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
                   const crk_step_io *io);
// One stage of crk_advance in the library's kernel orders.  The work array
// holds crk_stage_cols::count columns of n floats: the state permuted into
// the gas kernel order (m, v, u), m in the gravity order, the chain's
// intermediates, the accelerations dv (gas order) and ag (gravity order), du
// and v* (gas order).
namespace crk_stage_cols {
enum : int {
    m = 0, v = 1, u = 4, mg = 5, V = 6, rho = 7, A = 8, B = 9, gA = 12, gB = 15, rhoR = 24, dvdx = 25, dv = 34,
    du = 37, ag = 38, vs = 41, count = 44
};
}
// geometry, corrections, (Extras), Acceleration with the signal-velocity max and (gravity)
int crk_stage_forces(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
                     int limited, int gravity, float sig_beta, const float *m, const float *v3, const float *u,
                     uint32_t *vsig_h, int32_t *n_singular, float *work);
// Energy on v* (caller order; NULL: v* = v) with the intermediates of the last crk_stage_forces
int crk_stage_energy(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, int limited,
                     const float *vstar3, float *work, double *conservation);
// records event k (0..7) of the current profiled step, if profiling is on
void crk_step_mark(crk_ctx *ctx, int k);

#define CRK_CUDA(ctx, call)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return crk_check_cuda(ctx, e_, #call); \
    } while (0)

#define CRK_LAUNCH_CHECK(ctx, what)                                           \
    do {                                                                      \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) return crk_check_cuda(ctx, e_, what);          \
    } while (0)

// ---- scan / sort primitives (scan.cu) ----
// exclusive prefix sum of n int32 values (in may equal out); total (device int32) optional
int crk_exclusive_scan_i32(crk_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *total);
// stable LSD radix sort of (key, value) pairs by all 32 key bits
int crk_radix_sort_u32(crk_ctx *ctx, uint32_t *keys, int32_t *vals, int64_t n, int key_bits);

static inline int crk_grid(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 2147483647LL) g = 2147483647LL;
    return (int)g;
}

// Block-wide exclusive scan of one int32 per thread (all threads must call);
// warp_tot needs blockDim/32 entries.  Returns the thread's exclusive prefix.
__device__ __forceinline__ int32_t crk_block_scan(int32_t v, int32_t *warp_tot, int32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(CRK_FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(CRK_FULL_MASK, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    int32_t r = (warp > 0 ? warp_tot[warp - 1] : 0) + x - v;
    __syncthreads();
    return r;
}
