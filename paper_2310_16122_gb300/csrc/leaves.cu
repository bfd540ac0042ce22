// Leaf decomposition on the GPU: chaining mesh or recursive coordinate bisection
// (Sec. 3.1 names the RCB tree; Sec. 5.3 runs the kernels over leaf pairs),
// then the periodic leaf-pair image lists used by every pair kernel.
//
// RCB without per-node sorts: every particle is ranked once per axis by a
// stable radix sort of (coordinate, index).  Each level keeps three lists,
// each sorted along its axis inside every node, whose entries carry the
// particle's ranks along the two other axes.  A node's tight box is read off
// the ends of its three segments; the split takes the first floor(n/2) of the
// chosen axis' segment, which is a threshold on the rank along that axis, so
// the two other lists are stably partitioned by comparing the ranks they
// carry (a prefix sum of the left flags orders the output).  The shape of the
// tree depends on n alone, so the host precomputes every level's segments.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>

#include "crk_internal.cuh"

namespace {

constexpr int kMaxLeafCap = 1024;

__device__ __forceinline__ uint32_t coord_key(float x) {
    // x >= 0 after validation: the IEEE bits of non-negative floats are ordered like the values
    return x == 0.0f ? 0u : __float_as_uint(x);
}

// Positions in [0, L_box), gas h > 0 and finite; largest gas h per box.
// Each block takes kValItems rows of 256 consecutive particles and combines
// its counts (and, when its range lies in one box, its h maximum) in shared
// memory, so the global atomics are a few per block: same-address atomics
// from every warp of a 33M-particle launch serialise at L2 (about 1.7 ms).
constexpr int kValItems = 16;
constexpr int kValTile = 256 * kValItems;

__global__ void __launch_bounds__(256) validate_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                       const float *__restrict__ z, const uint8_t *__restrict__ sp,
                                                       const float *__restrict__ h, int64_t n,
                                                       const int32_t *__restrict__ box_of,
                                                       const float *__restrict__ box_L,
                                                       int32_t *__restrict__ flags /* [0] bad pos, [1] bad h, [2] n_gas */,
                                                       unsigned *__restrict__ hmax_bits /* per box */) {
    __shared__ unsigned part[4][8];
    const int64_t base = (int64_t)blockIdx.x * kValTile;
    const int64_t last = (base + kValTile < n ? base + kValTile : n) - 1;
    const int bfirst = box_of ? box_of[base] : 0;
    const bool one_box = !box_of || box_of[last] == bfirst;  // boxes are contiguous ranges
    unsigned nbad = 0, nbadh = 0, ngas = 0, hb_blk = 0;
    for (int k = 0; k < kValItems; ++k) {
        const int64_t i = base + (int64_t)k * 256 + threadIdx.x;
        if (i >= n) break;
        const int b = box_of ? box_of[i] : 0;
        const float L = box_L[b];
        const float c[3] = {x[i], y[i], z[i]};
        bool bad = false;
        for (int a = 0; a < 3; ++a) bad |= !(c[a] >= 0.0f && c[a] < L);
        nbad += bad;
        if (sp[i] == 0) {
            ++ngas;
            const float hi = h[i];
            if (!(hi > 0.0f) || !isfinite(hi)) {
                ++nbadh;
            } else {
                const unsigned hb = __float_as_uint(hi);  // positive floats order like their bits
                if (one_box) hb_blk = hb > hb_blk ? hb : hb_blk;
                else atomicMax(&hmax_bits[b], hb);
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    nbad = __reduce_add_sync(CRK_FULL_MASK, nbad);
    nbadh = __reduce_add_sync(CRK_FULL_MASK, nbadh);
    ngas = __reduce_add_sync(CRK_FULL_MASK, ngas);
    hb_blk = __reduce_max_sync(CRK_FULL_MASK, hb_blk);
    if (lane == 0) {
        part[0][w] = nbad;
        part[1][w] = nbadh;
        part[2][w] = ngas;
        part[3][w] = hb_blk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 1; v < 8; ++v) {
            for (int q = 0; q < 3; ++q) part[q][0] += part[q][v];
            part[3][0] = part[3][v] > part[3][0] ? part[3][v] : part[3][0];
        }
        for (int q = 0; q < 3; ++q)
            if (part[q][0]) atomicAdd(&flags[q], (int)part[q][0]);
        if (part[3][0]) atomicMax(&hmax_bits[bfirst], part[3][0]);
    }
}

// box of each particle from the box starts (binary search)
__global__ void box_of_kernel(int64_t n, const int64_t *__restrict__ box_start, int nbox, int32_t *__restrict__ box_of) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (box_start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    box_of[i] = lo;
}

// keys for the stable re-sort of an axis list by box
__global__ void box_keys_kernel(int64_t n, const int32_t *__restrict__ list, const int32_t *__restrict__ box_of,
                                uint32_t *__restrict__ keys) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) keys[p] = (uint32_t)box_of[list[p]];
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
    const int32_t *leftbase;  // sum of k over the earlier segments of the level
};

// everything the partition needs about one segment, in one 32-byte record
struct __align__(16) SegRec {
    int32_t lo, hi, k, child;
    int32_t axis, leftbase, thr, pad;  // thr: rank along the split axis of the first right-going particle
};

// The three axis lists carry ranks, not particle ids.  S[t] is the stable
// (coordinate, index) order along axis t (box-major for batches) and R[t] its
// inverse (the rank of each particle along t).  Entry p of list a holds the
// ranks of its particle along the two other axes:
// A[a][c][p] = rank along axis (a + 1 + c) % 3.  Inside a node, list a is
// sorted by rank along a, so the node's split is a rank threshold: an entry of
// another list goes left iff its rank along the split axis is below the rank
// of the first right-going entry of the split axis' own list.  A level is then
// pure streaming (no per-particle side flag is scattered or gathered).
struct RankLists {
    const int32_t *A[3][2];
};
struct RankListsOut {
    int32_t *A[3][2];
};
struct AxisOrder {
    const int32_t *S[3];
    const int32_t *R[3];
};

__device__ __forceinline__ unsigned lanemask_lt_u() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int rank_comp(int a, int t) { return (t - a + 2) % 3; }  // component of list a holding t

// particle id of entry p of list a
__device__ __forceinline__ int32_t rank_entry_id(const RankLists &L, const AxisOrder &o, int a, int64_t p) {
    const int32_t r = L.A[a][0][p];
    return a == 0 ? o.S[1][r] : (a == 1 ? o.S[2][r] : o.S[0][r]);
}

// R[S[p]] = p: the inverse of one axis order (one axis per launch, so the
// randomly written array, n ints, stays about the size of L2)
__global__ void rank_of_kernel(int64_t n, const int32_t *__restrict__ S, int32_t *__restrict__ R) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) R[S[p]] = (int32_t)p;
}

// dst[p] = R[S[p]]: one rank column of one axis list (one source array per launch, as above)
__global__ void rank_column_kernel(int64_t n, const int32_t *__restrict__ S, const int32_t *__restrict__ R,
                                   int32_t *__restrict__ dst) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = __ldg(R + S[p]);
}

// final member order (list 0) as particle ids
__global__ void rank_members_kernel(int64_t n, RankLists L, AxisOrder o, int32_t *__restrict__ members) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) members[p] = rank_entry_id(L, o, 0, p);
}

// per split node: tight box from the ends of its three list segments, split
// axis (longest extent, ties to the lower axis), rank threshold
__global__ void rcb_axis_kernel(int nseg, LevelDev lv, RankLists L, AxisOrder o, const float *__restrict__ x,
                                const float *__restrict__ y, const float *__restrict__ z, float *__restrict__ node_box,
                                SegRec *__restrict__ seg) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int k = lv.k[s];
    int lo = lv.lo[s], hi = lv.hi[s];
    SegRec r{lo, hi, k, lv.child[s], 0, lv.leftbase[s], 0, 0};
    if (k <= 0) {
        seg[s] = r;
        return;
    }
    const float *cs[3] = {x, y, z};
    float blo[3], bhi[3];
    double ext[3];
    for (int a = 0; a < 3; ++a) {
        blo[a] = cs[a][rank_entry_id(L, o, a, lo)];
        bhi[a] = cs[a][rank_entry_id(L, o, a, hi - 1)];
        ext[a] = __dsub_rn((double)bhi[a], (double)blo[a]);
    }
    int axis = 0;
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    lv.axis[s] = axis;
    r.axis = axis;
    r.thr = o.R[axis][rank_entry_id(L, o, axis, lo + k)];
    seg[s] = r;
    float *nb = node_box + 6 * (int64_t)lv.node[s];
    for (int a = 0; a < 3; ++a) {
        nb[a] = blo[a];
        nb[3 + a] = bhi[a];
    }
}

// Stable partition of the three lists, one level at a time.  The prefix count
// of left-going entries at a segment's start equals the sum of k over the
// earlier split segments (every split segment sends exactly k entries left in
// every list), so the prefix is never materialised: tiles count, a 3-column
// scan orders the tiles, and the scatter re-derives the tile-local prefixes.
constexpr int kPartThreads = 256;
constexpr int kPartItems = 8;
constexpr int kPartTile = kPartThreads * kPartItems;

// left flags of entry p (bit b: list b), or 0 for entries of unsplit segments
__device__ __forceinline__ unsigned rcb_left3(const SegRec &sr, const RankLists &L, int64_t p) {
    const int ks = sr.k;
    if (ks <= 0) return 0u;
    const int ax = sr.axis, lo = sr.lo;
    const int32_t th = sr.thr;
    unsigned f = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        bool left;
        if (b == ax) {
            left = (int)p - lo < ks;
        } else {
            const int32_t *col = rank_comp(b, ax) == 0 ? L.A[b][0] : L.A[b][1];  // no dynamic index into the parameter
            left = col[p] < th;
        }
        f |= (unsigned)left << b;
    }
    return f;
}

__global__ void __launch_bounds__(kPartThreads) rcb_count3_kernel(int64_t n, const SegRec *__restrict__ segs,
                                                                   const int32_t *__restrict__ node_of, RankLists L,
                                                                   int32_t *__restrict__ bsum, int64_t nb) {
    __shared__ int32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
    int32_t seg[kPartItems];
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
        int64_t p = base + (int64_t)k * kPartThreads + threadIdx.x;
        seg[k] = p < n ? node_of[p] : -1;
    }
    int32_t c[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
        int64_t p = base + (int64_t)k * kPartThreads + threadIdx.x;
        unsigned f = 0u;
        if (seg[k] >= 0) {
            const SegRec sr = segs[seg[k]];
            f = rcb_left3(sr, L, p);
        }
        c[0] += f & 1u;
        c[1] += (f >> 1) & 1u;
        c[2] += (f >> 2) & 1u;
    }
    for (int b = 0; b < 3; ++b) {
        int32_t tot;
        crk_block_scan(c[b], wt, tot);
        if (threadIdx.x == 0) bsum[(int64_t)b * nb + blockIdx.x] = tot;
    }
}

// single block: exclusive scan of the three columns of tile sums, in place
__global__ void rcb_scan3_kernel(int32_t *__restrict__ bsum, int64_t nb) {
    __shared__ int32_t wt[32];
    for (int b = 0; b < 3; ++b) {
        int32_t carry = 0;
        int32_t *col = bsum + (int64_t)b * nb;
        for (int64_t s0 = 0; s0 < nb; s0 += blockDim.x) {
            int64_t i = s0 + threadIdx.x;
            int32_t v = i < nb ? col[i] : 0;
            int32_t tot;
            int32_t e = crk_block_scan(v, wt, tot);
            if (i < nb) col[i] = carry + e;
            carry += tot;
        }
    }
}

// Entries are taken in rows of kPartThreads consecutive positions (entry k of
// thread t is position base + k kPartThreads + t), so the left-going (and the
// right-going) entries of one warp row land in consecutive output positions:
// coalesced stores.  The tile-local prefix of an entry is the count over
// earlier (row, warp) pairs plus the ballot rank inside its warp.  The kernel
// waits on its loads (segment record, rank columns): compiled for six
// resident blocks per SM (40 registers) it ran the 14 streamed levels of the
// 33.5M-particle build 2.0 ms faster than at four.
constexpr int kPartWarps = kPartThreads / 32;

__global__ void __launch_bounds__(kPartThreads, 6) rcb_scatter3_kernel(int64_t n, const SegRec *__restrict__ segs,
                                                                      const int32_t *__restrict__ node_of, RankLists L,
                                                                      const int32_t *__restrict__ bsum, int64_t nb,
                                                                      RankListsOut O, int32_t *__restrict__ node_of_next,
                                                                      int32_t *__restrict__ err) {
    static_assert(kPartItems * kPartWarps == 64, "prefix table: two entries per lane of one warp");
    __shared__ int32_t wc[3][kPartItems * kPartWarps];  // left count per (list, row, warp), then its prefix
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned below = lanemask_lt_u();
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
    int32_t seg[kPartItems];
    unsigned f[kPartItems];
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
        int64_t p = base + (int64_t)k * kPartThreads + threadIdx.x;
        seg[k] = p < n ? node_of[p] : -1;
    }
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
        int64_t p = base + (int64_t)k * kPartThreads + threadIdx.x;
        f[k] = 0u;
        if (seg[k] >= 0) {
            const SegRec sr = segs[seg[k]];
            f[k] = rcb_left3(sr, L, p);
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const unsigned m = __ballot_sync(0xffffffffu, (f[k] >> b) & 1u);
            if (lane == 0) wc[b][k * kPartWarps + warp] = __popc(m);
        }
    }
    __syncthreads();
    if (warp == 0) {
        for (int b = 0; b < 3; ++b) {
            const int32_t e0 = wc[b][2 * lane], e1 = wc[b][2 * lane + 1];
            int32_t v = e0 + e1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            const int32_t ex = v - e0 - e1;
            wc[b][2 * lane] = ex;
            wc[b][2 * lane + 1] = ex + e0;
        }
    }
    __syncthreads();
    int32_t tile0[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) tile0[b] = bsum[(int64_t)b * nb + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
        const int64_t p = base + (int64_t)k * kPartThreads + threadIdx.x;
        const bool valid = seg[k] >= 0;
        SegRec sr{0, 0, 0, 0, 0, 0, 0, 0};
        if (valid) sr = segs[seg[k]];
        const int ks = sr.k, lo = sr.lo;
        if (valid) node_of_next[p] = sr.child + ((ks > 0 && (int)p - lo >= ks) ? 1 : 0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const bool left = (f[k] >> b) & 1u;
            const unsigned m = __ballot_sync(0xffffffffu, left);
            if (!valid) continue;
            const int32_t r0 = L.A[b][0][p], r1 = L.A[b][1][p];
            int64_t np = p;
            if (ks > 0) {
                // left-going entries before p in this segment
                const int lb = tile0[b] + wc[b][k * kPartWarps + warp] + __popc(m & below) - sr.leftbase;
                np = left ? lo + lb : lo + ks + ((int)p - lo - lb);
                if (!(np >= lo && np < sr.hi)) {
                    atomicAdd(err, 1);  // inconsistent partition: reported, never written out of the segment
                    continue;
                }
            }
            O.A[b][0][np] = r0;
            O.A[b][1][np] = r1;
        }
    }
}

// --- RCB bottom levels in shared memory --------------------------------------
// Once every segment of a level holds at most kLocalCap entries, one block
// takes one segment and runs all the remaining levels on it in shared memory:
// the same boxes, axes, rank thresholds and stable partitions as the level
// kernels above (so the same tree, bit for bit), but a level costs a few
// shared-memory passes instead of three DRAM passes over the six rank
// columns.  The block ends by writing the final member order of its range.
constexpr int kLocalCap = 2048;
constexpr int kLocalThreads = 512;
constexpr int kLocalBlocks = 2;                         // resident blocks per SM (shared memory: ~113 KB each)
constexpr int kLocalItems = kLocalCap / kLocalThreads;  // consecutive positions per thread
constexpr int kLocalLevels = 7;                         // levels one block may run
constexpr int kLocalSegs = 1 << kLocalLevels;           // segments per block at its deepest level
constexpr size_t kLocalSmem = sizeof(int32_t) * 2 * 6 * kLocalCap + sizeof(int16_t) * 2 * kLocalCap;
static_assert(kLocalItems == 4, "positions are moved as int4");

// the level tables a block walks: tab[l] = 7 columns of m[l] segments (lo, hi, k, child, node, axis, leftbase)
struct LocalShape {
    int32_t *tab[kLocalLevels];
    int32_t m[kLocalLevels];
    int nlev;
};

struct __align__(16) LocalSeg {
    int32_t lo, hi, k, child;  // lo, hi relative to the block's range; child relative to the next level's first
    int32_t axis, thr, lb, pad;  // lb: left entries of the block's earlier segments (every list alike)
};

// three 21-bit counters in one word (at most kLocalCap per counter)
__device__ __forceinline__ uint64_t pack3(unsigned f) {
    return (uint64_t)(f & 1u) | ((uint64_t)((f >> 1) & 1u) << 21) | ((uint64_t)((f >> 2) & 1u) << 42);
}
__device__ __forceinline__ int field3(uint64_t v, int b) { return (int)((v >> (21 * b)) & 0x1fffffu); }

__global__ void __launch_bounds__(kLocalThreads, kLocalBlocks) rcb_local_kernel(int64_t n, LocalShape sh, RankLists L, AxisOrder o,
                                                                       const float *__restrict__ x,
                                                                       const float *__restrict__ y,
                                                                       const float *__restrict__ z,
                                                                       float *__restrict__ node_box,
                                                                       int32_t *__restrict__ members,
                                                                       int32_t *__restrict__ err) {
    extern __shared__ int4 local_smem[];
    int32_t *cur = reinterpret_cast<int32_t *>(local_smem);  // [6][kLocalCap]: column 2b + c of list b
    int32_t *nxt = cur + 6 * kLocalCap;
    int16_t *sc = reinterpret_cast<int16_t *>(nxt + 6 * kLocalCap);  // segment of each position
    int16_t *sn = sc + kLocalCap;
    __shared__ LocalSeg seg[kLocalSegs];
    __shared__ uint64_t wsum[kLocalThreads / 32];
    __shared__ int bad;
    const int s0 = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int m0 = sh.m[0];
    const int lo = sh.tab[0][s0], cnt = sh.tab[0][m0 + s0] - lo;
    if (t == 0) bad = 0;
    if (cnt > kLocalCap) {
        if (t == 0) atomicAdd(err, 1);
        return;
    }
    for (int q = t; q < cnt; q += kLocalThreads) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cur[(2 * b) * kLocalCap + q] = L.A[b][0][lo + q];
            cur[(2 * b + 1) * kLocalCap + q] = L.A[b][1][lo + q];
        }
        sc[q] = 0;
    }
    const float *cs[3] = {x, y, z};
    // a rank used as an index; a partition found inconsistent (reported through err) may leave
    // positions unwritten, whose values then never index out of the arrays
    auto rk = [n](int32_t r) -> int64_t { return (uint64_t)r < (uint64_t)n ? r : 0; };
    int f = s0, e = s0 + 1;  // this block's segments at the current level
    for (int lev = 0; lev < sh.nlev; ++lev) {
        int32_t *tab = sh.tab[lev];
        const int m = sh.m[lev];
        const int ns = e - f;
        __syncthreads();  // the previous level is done with seg[], cur and sc
        if (ns > kLocalSegs) {  // excluded by the host's choice of levels
            if (t == 0) atomicAdd(err, 1);
            return;
        }
        for (int u = t; u < ns; u += kLocalThreads) {
            const int s = f + u;
            LocalSeg r{tab[s] - lo, tab[m + s] - lo, tab[2 * m + s], 0, 0, 0, tab[6 * m + s] - tab[6 * m + f], 0};
            const int k = r.k;
            if (k > 0) {
                // tight box from the ends of the three list segments (entry p of list a: rank
                // along axis (a + 1) % 3 in column 0)
                float blo[3], bhi[3];
                double ext[3];
                for (int a = 0; a < 3; ++a) {
                    const int32_t *S = o.S[(a + 1) % 3];
                    blo[a] = cs[a][S[rk(cur[(2 * a) * kLocalCap + r.lo])]];
                    bhi[a] = cs[a][S[rk(cur[(2 * a) * kLocalCap + r.hi - 1])]];
                    ext[a] = __dsub_rn((double)bhi[a], (double)blo[a]);
                }
                int axis = 0;
                if (ext[1] > ext[axis]) axis = 1;
                if (ext[2] > ext[axis]) axis = 2;
                r.axis = axis;
                r.thr = o.R[axis][o.S[(axis + 1) % 3][rk(cur[(2 * axis) * kLocalCap + r.lo + k])]];
                tab[5 * m + s] = axis;
                float *nb = node_box + 6 * (int64_t)tab[4 * m + s];
                for (int a = 0; a < 3; ++a) {
                    nb[a] = blo[a];
                    nb[3 + a] = bhi[a];
                }
            }
            seg[u] = r;
        }
        // the next level's range of this block's segments
        const int fn = tab[3 * m + f];
        const int en = tab[3 * m + e - 1] + (tab[2 * m + e - 1] > 0 ? 2 : 1);
        for (int u = t; u < ns; u += kLocalThreads) seg[u].child = tab[3 * m + f + u] - fn;
        __syncthreads();
        // left flags of this thread's kLocalItems consecutive positions (bit b: list b)
        const int q0 = t * kLocalItems;
        unsigned fl[kLocalItems];
        int sg[kLocalItems];
        uint64_t mine = 0;
#pragma unroll
        for (int i = 0; i < kLocalItems; ++i) {
            const int q = q0 + i;
            fl[i] = 0u;
            sg[i] = 0;
            if (q < cnt) {
                sg[i] = sc[q];
                const LocalSeg &r = seg[sg[i]];
                if (r.k > 0) {
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        bool left;
                        if (b == r.axis) {
                            left = q - r.lo < r.k;
                        } else {
                            const int c = (r.axis - b + 2) % 3;  // column of list b holding ranks along the axis
                            left = cur[(2 * b + c) * kLocalCap + q] < r.thr;
                        }
                        fl[i] |= (unsigned)left << b;
                    }
                }
                mine += pack3(fl[i]);
            }
        }
        // block exclusive scan of the three counters
        uint64_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t v = __shfl_up_sync(CRK_FULL_MASK, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            constexpr int kW = kLocalThreads / 32;
            uint64_t v = lane < kW ? wsum[lane] : 0, iv = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t u = __shfl_up_sync(CRK_FULL_MASK, iv, d);
                if (lane >= d) iv += u;
            }
            if (lane < kW) wsum[lane] = iv - v;
        }
        __syncthreads();
        uint64_t run = wsum[w] + incl - mine;
        // stable partition into nxt; the segment of each new position
#pragma unroll
        for (int i = 0; i < kLocalItems; ++i) {
            const int q = q0 + i;
            if (q >= cnt) break;
            const LocalSeg &r = seg[sg[i]];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                int np = q;
                if (r.k > 0) {
                    const int lb = field3(run, b) - r.lb;  // left entries before q in its segment
                    np = (fl[i] >> b) & 1u ? r.lo + lb : r.lo + r.k + (q - r.lo - lb);
                    if (!(np >= r.lo && np < r.hi)) {
                        bad = 1;  // inconsistent partition: reported, never written out of the segment
                        continue;
                    }
                }
                nxt[(2 * b) * kLocalCap + np] = cur[(2 * b) * kLocalCap + q];
                nxt[(2 * b + 1) * kLocalCap + np] = cur[(2 * b + 1) * kLocalCap + q];
            }
            sn[q] = (int16_t)(r.child + ((r.k > 0 && q - r.lo >= r.k) ? 1 : 0));
            run += pack3(fl[i]);
        }
        int32_t *tp = cur;
        cur = nxt;
        nxt = tp;
        int16_t *ts = sc;
        sc = sn;
        sn = ts;
        f = fn;
        e = en;
    }
    __syncthreads();
    if (t == 0 && bad) atomicAdd(err, 1);
    for (int q = t; q < cnt; q += kLocalThreads) members[lo + q] = o.S[1][rk(cur[q])];  // list 0, column 0
}

// --- per-leaf data ------------------------------------------------------------
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Shared state of bisect32 (one per block) for leaves of at most kCap members
// (parts of 8 for leaves of at most 256, parts of 32 above).
template <int kCap>
struct Bisect32 {
    static constexpr int kMaxSeg = kCap <= 256 ? kCap / 8 : kCap / 32;
    int16_t a[kCap], b[kCap];  // orders (member slots), double-buffered
    float cax[kCap];           // coordinate of the member at each position on its part's axis
    uint32_t cid[kCap];        // its particle index (ties)
    int lo[kMaxSeg], hi[kMaxSeg], ax[kMaxSeg];
    int nseg, more;
};

// Bisects positions [0, m) of the order src (bs.a or bs.b; member slots; m <= kCap)
// into groups of U: each part above U is ranked along the longest extent of
// its members in (coordinate, index) order and split with U ceil(g/2) of its
// g groups of U on the left, until every part holds at most U; then every run
// of U positions starting at a multiple of U is an RCB cell.  The parts start
// as the runs of `start` positions (start = m: the whole range; start = 32
// with U = 8: the RCB cells of 32, each bisected into cells of 8).  At most
// ceil(m/U) <= 32 parts, one per lane of warp 0.  All threads call it; returns
// the array (bs.a or bs.b) holding the result in [0, m).
template <int kCap, int U = 32>
__device__ int16_t *bisect32(Bisect32<kCap> &bs, int m, const float4 *pm, const uint64_t *key,
                             int16_t *src_in = nullptr, int start = 0) {
    static_assert(kCap / U <= Bisect32<kCap>::kMaxSeg && kCap / U <= 32, "parts per leaf");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int16_t *src = src_in ? src_in : bs.a, *dst = src == bs.a ? bs.b : bs.a;
    if (start <= 0 || start > m) start = m;
    if (threadIdx.x == 0) {
        bs.nseg = 0;
        bs.more = 0;
        for (int l = 0; l < m; l += start) {
            bs.lo[bs.nseg] = l;
            bs.hi[bs.nseg] = l + start < m ? l + start : m;
            bs.more |= bs.hi[bs.nseg] - l > U;
            ++bs.nseg;
        }
        if (m == 0) {
            bs.nseg = 1;
            bs.lo[0] = bs.hi[0] = 0;
        }
    }
    __syncthreads();
    while (bs.more) {
        // axis of the longest extent of every part above 32 (one warp per part)
        for (int sg = w; sg < bs.nseg; sg += nw) {
            const int l = bs.lo[sg], hh = bs.hi[sg];
            if (hh - l <= U) {
                if (lane == 0) bs.ax[sg] = -1;
                continue;
            }
            float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int u = l + lane; u < hh; u += 32) {
                const float4 c = pm[src[u]];
                mn[0] = fminf(mn[0], c.x); mx[0] = fmaxf(mx[0], c.x);
                mn[1] = fminf(mn[1], c.y); mx[1] = fmaxf(mx[1], c.y);
                mn[2] = fminf(mn[2], c.z); mx[2] = fmaxf(mx[2], c.z);
            }
            for (int o = 16; o > 0; o >>= 1)
                for (int q = 0; q < 3; ++q) {
                    mn[q] = fminf(mn[q], __shfl_xor_sync(CRK_FULL_MASK, mn[q], o));
                    mx[q] = fmaxf(mx[q], __shfl_xor_sync(CRK_FULL_MASK, mx[q], o));
                }
            const float e0 = mx[0] - mn[0], e1 = mx[1] - mn[1], e2 = mx[2] - mn[2];
            if (lane == 0) bs.ax[sg] = (e0 >= e1 && e0 >= e2) ? 0 : (e1 >= e2 ? 1 : 2);
        }
        __syncthreads();
        // each position's key on its part's axis, so the ranking reads two flat arrays
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            int sg = 0;
            while (bs.hi[sg] <= q) ++sg;
            const int ax = bs.ax[sg], t = src[q];
            const float4 c = pm[t];
            bs.cax[q] = ax == 0 ? c.x : (ax == 1 ? c.y : c.z);
            bs.cid[q] = (uint32_t)key[t];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            int sg = 0;
            while (bs.hi[sg] <= q) ++sg;
            if (bs.ax[sg] < 0) {
                dst[q] = src[q];
                continue;
            }
            const float cv = bs.cax[q];
            const uint32_t iv = bs.cid[q];
            const int l = bs.lo[sg], hh = bs.hi[sg];
            int r = 0;
            for (int u = l; u < hh; ++u) {
                const float cu = bs.cax[u];
                r += (cu < cv) || (cu == cv && bs.cid[u] < iv);
            }
            dst[l + r] = src[q];
        }
        __syncthreads();
        if (w == 0) {
            // the children of every part, in order (one part per lane)
            const bool have = lane < bs.nseg;
            const int l = have ? bs.lo[lane] : 0, hh = have ? bs.hi[lane] : 0;
            const bool split = have && bs.ax[lane] >= 0;
            const int nch = have ? (split ? 2 : 1) : 0;
            int off = nch;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(CRK_FULL_MASK, off, o);
                if (lane >= o) off += v;
            }
            const int total = __shfl_sync(CRK_FULL_MASK, off, 31);
            off -= nch;
            const int g = (hh - l + U - 1) / U;
            const int left = split ? U * ((g + 1) / 2) : hh - l;
            __syncwarp();
            if (have) {
                bs.lo[off] = l;
                bs.hi[off] = l + left;
                if (split) {
                    bs.lo[off + 1] = l + left;
                    bs.hi[off + 1] = hh;
                }
            }
            const bool open = have && (left > U || (split && hh - l - left > U));
            const bool any = __any_sync(CRK_FULL_MASK, open);
            if (lane == 0) {
                bs.nseg = total;
                bs.more = any;
            }
        }
        __syncthreads();
        int16_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    return src;
}

// One block per leaf: tight box, gas count, largest gas h; the canonical
// order (gas first, then dark matter, each by index) for export; the gas
// kernel order (gas first, then dark matter along a Z-order curve of the leaf
// box, ties by index; the gas part bisected into groups of 32 as below); the
// gravity kernel order (species mixed): the leaf bisected into groups of 32,
// each split along the longest extent of its part in (coordinate, index)
// order with a multiple of 32 particles on the left, so that every group of 32
// consecutive particles is an RCB cell (the gravity tiles sweep the
// candidates within r_c of a group's box: at r_c = 3 such cells cut the
// candidates per in-range pair from ~4.0 to ~3.3 against Z-order groups); and
// the leaf-relative positions in both kernel orders.
// kCap: the largest leaf the launch may meet (1024 with blocks of 128 threads; 128 with one
// warp per block for RCB leaves of at most 128, whose shared arrays then fit 32 blocks per SM).
template <int kCap>
__global__ void leaf_data_kernel(int64_t n_leaves, const int32_t *__restrict__ leaf_start,
                                 const int32_t *__restrict__ members, const float *__restrict__ x,
                                 const float *__restrict__ y, const float *__restrict__ z,
                                 const uint8_t *__restrict__ sp, const float *__restrict__ h,
                                 int32_t *__restrict__ perm, int32_t *__restrict__ kperm,
                                 int32_t *__restrict__ leaf_ngas, float *__restrict__ bbox,
                                 float *__restrict__ hmax, float4 *__restrict__ pos, int32_t *__restrict__ kperm_g,
                                 float4 *__restrict__ pos_g, int32_t *__restrict__ kinv, int32_t *__restrict__ kinv_g,
                                 int32_t *__restrict__ err, int cells8) {
    __shared__ uint64_t key[kCap], zkey[kCap];
    __shared__ Bisect32<kCap> bs;
    __shared__ float4 pm[kCap];  // member position and h (0 for dark matter), gathered once
    __shared__ float red[6][32];
    __shared__ int ngs[32];
    __shared__ float hms[32];
    const int64_t a = blockIdx.x;
    if (a >= n_leaves) return;
    const int lo = leaf_start[a], hi = leaf_start[a + 1], cnt = hi - lo;
    if (cnt > kCap) {
        if (threadIdx.x == 0) atomicAdd(err, 1);
        return;
    }
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int ng = 0;
    float hm = 0.0f;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int32_t id = members[lo + t];
        const bool gas = sp[id] == 0;
        key[t] = ((uint64_t)!gas << 32) | (uint32_t)id;
        float c[3] = {x[id], y[id], z[id]};
        const float hh = gas ? h[id] : 0.0f;
        pm[t] = make_float4(c[0], c[1], c[2], hh);
        for (int q = 0; q < 3; ++q) {
            mn[q] = fminf(mn[q], c[q]);
            mx[q] = fmaxf(mx[q], c[q]);
        }
        if (gas) {
            ++ng;
            hm = fmaxf(hm, hh);
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
    const float ext = fmaxf(fmaxf(red[3][0] - ox, red[4][0] - oy), fmaxf(red[5][0] - oz, 1e-30f));
    const float sc = 1023.0f / ext;
    // canonical ranks, and the Z-order keys of each member: zkey with the
    // species on top (gas first), gkey without (gravity order)
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        uint64_t kt = key[t];
        int r = 0;
        for (int u = 0; u < cnt; ++u) r += key[u] < kt;
        int32_t id = (int32_t)(uint32_t)kt;
        perm[lo + r] = id;
        const float4 c = pm[t];
        uint32_t mx3 = spread10((uint32_t)fminf((c.x - ox) * sc, 1023.0f)) |
                       (spread10((uint32_t)fminf((c.y - oy) * sc, 1023.0f)) << 1) |
                       (spread10((uint32_t)fminf((c.z - oz) * sc, 1023.0f)) << 2);
        zkey[t] = ((kt >> 32) << 62) | ((uint64_t)mx3 << 32) | (uint32_t)id;
    }
    __syncthreads();
    // gas order: gas first, then dark matter, each along the Z curve; then the gas part
    // bisected into groups of 32 (dark matter keeps the Z order)
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        uint64_t kt = zkey[t];
        int r = 0;
        for (int u = 0; u < cnt; ++u) r += zkey[u] < kt;
        bs.a[r] = (int16_t)t;
        bs.b[r] = (int16_t)t;
    }
    const int16_t *gsrc = bisect32(bs, ngs[0], pm, key);
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int t = gsrc[q];
        const float4 c = pm[t];
        const int32_t id = (int32_t)(uint32_t)key[t];
        kperm[lo + q] = id;
        kinv[id] = lo + q;  // the inverse permutations, written here rather than by a pass of their own
        pos[lo + q] = make_float4(c.x - ox, c.y - oy, c.z - oz, c.w);
    }
    __syncthreads();
    // gravity order: the whole leaf bisected into groups of 32, and (cells8, leaves of at most 256)
    // each group of 32 into groups of 8 (the sub-cells of the split gravity sweeps)
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) bs.a[t] = (int16_t)t;
    int16_t *src = bisect32(bs, cnt, pm, key);
    if constexpr (kCap <= 256) {
        if (cells8) src = bisect32<kCap, 8>(bs, cnt, pm, key, src, 32);
    }
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int t = src[q];
        const float4 c = pm[t];
        const int32_t id = (int32_t)(uint32_t)key[t];
        kperm_g[lo + q] = id;
        kinv_g[id] = lo + q;
        pos_g[lo + q] = make_float4(c.x - ox, c.y - oy, c.z - oz, c.w);
    }
}

// --- leaf-pair images ------------------------------------------------------------
struct TreeDev {
    const float *node_box;       // [nodes][6]
    const float *node_hmax;      // [nodes] largest gas h below the node
    const int32_t *node_left;    // child ids, -1 for leaves
    const int32_t *node_right;
    const int32_t *node_leaf;    // leaf id for leaves, -1 otherwise
    int32_t root;
};

// FP32 periodic box gap, used only to discard candidates that are clearly out
// of range (the caller adds a margin far above the FP32 rounding of the sums)
__device__ __forceinline__ float axis_gap32(float loa, float hia, float lob, float hib, float L) {
    float best = INFINITY;
#pragma unroll
    for (int k = -1; k <= 1; ++k) {
        float s = (float)k * L;
        float g = fmaxf(fmaxf((lob + s) - hia, (loa - hib) - s), 0.0f);
        best = fminf(best, g);
    }
    return best;
}

__device__ __forceinline__ bool clearly_apart(const float *A, const float *B, float L, float cut) {
    float gx = axis_gap32(A[0], A[3], B[0], B[3], L);
    float gy = axis_gap32(A[1], A[4], B[1], B[4], L);
    float gz = axis_gap32(A[2], A[5], B[2], B[5], L);
    float c = cut + 1e-5f * L + 1e-6f;
    return gx * gx + gy * gy + gz * gz > c * c;
}

__device__ __forceinline__ double axis_gap_shift(double loa, double hia, double lob, double hib, double s) {
    double t1 = __dsub_rn(__dadd_rn(lob, s), hia);
    double t2 = __dsub_rn(__dsub_rn(loa, hib), s);
    double g = t1 > t2 ? t1 : t2;
    return g < 0.0 ? 0.0 : g;
}

__device__ __forceinline__ double sum_sq(double gx, double gy, double gz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
}

// Emits the images of leaf b that lie within `cut` of leaf a; returns how many.
template <bool kFill>
__device__ int leaf_images(const float *__restrict__ bbox, int64_t a, int64_t b, double L, double cut2,
                           crk_image *__restrict__ out) {
    const float *A = bbox + 6 * a, *B = bbox + 6 * b;
    const float Lf = (float)L, cutf = (float)sqrt(cut2) + 1e-5f * Lf + 1e-6f;
    if (clearly_apart(A, B, Lf, (float)sqrt(cut2))) return 0;
    // Per axis, only the shifts whose own gap is inside the cut can give an image: the FP64
    // sum of squares is never below one of its (non-negative) terms.  An FP32 gap with a margin
    // above its rounding skips the FP64 work for the far shifts (FP64 is slow on this GPU).
    double g[3][3];
    int keep[3][3], nk[3] = {0, 0, 0};
    for (int q = 0; q < 3; ++q)
        for (int k = 0; k < 3; ++k) {
            const float sf = (float)(k - 1) * Lf;
            const float g32 = fmaxf(fmaxf((B[q] + sf) - A[3 + q], (A[q] - B[3 + q]) - sf), 0.0f);
            if (g32 > cutf) continue;
            const double gd = axis_gap_shift(A[q], A[3 + q], B[q], B[3 + q], (double)(k - 1) * L);
            if (!(__dmul_rn(gd, gd) < cut2)) continue;
            g[q][nk[q]] = gd;
            keep[q][nk[q]++] = k;
        }
    int cnt = 0;
    for (int jx = 0; jx < nk[0]; ++jx)
        for (int jy = 0; jy < nk[1]; ++jy)
            for (int jz = 0; jz < nk[2]; ++jz) {
                const int ix = keep[0][jx], iy = keep[1][jy], iz = keep[2][jz];
                double d2 = sum_sq(g[0][jx], g[1][jy], g[2][jz]);
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
            (void)hmax_all;
            int32_t stack[64];
            int top = 0;
            stack[top++] = tree.root;
            while (top > 0) {
                int32_t nd = stack[--top];
                const float *Nb = tree.node_box + 6 * (int64_t)nd;
                float cutn = hydro ? 2.0f * fmaxf((float)ha, tree.node_hmax[nd]) : (float)rc;
                if (clearly_apart(A, Nb, (float)L, cutn)) continue;
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


// --- warp-cooperative leaf-pair finder ---------------------------------------------
// One warp per i-leaf.  The warp pops up to 32 tree nodes at a time from a
// shared-memory stack, tests them in parallel (FP32, with margin, against the
// larger of the gravity cut and the hydro cut bound), pushes the children of
// the survivors and collects surviving leaves.  The candidates are sorted,
// tested exactly (FP64 per periodic image, leaf_images) for both lists, and
// the leaf's images are written with one atomic reservation per list, so each
// leaf's lists stay in ascending j-leaf order.
constexpr int kTravWarps = 4;
constexpr int kStackCap = 512;
constexpr int kCandCap = 1024;

struct PairOut {
    int32_t *start[4];  // gravity images, gravity pairs, hydro images, hydro pairs
    int32_t *count[4];
    crk_image *gimg, *himg;
    int32_t *gpair, *hpair;
    int64_t cap[4];
    unsigned long long *cursor;  // [4]
    int32_t *err;                // [0] traversal overflow, [1] output overflow
};

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int &total) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(CRK_FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(CRK_FULL_MASK, x, 31);
    return x - v;
}

template <bool kBrute>
__global__ void __launch_bounds__(kTravWarps * 32) leaf_pairs_warp_kernel(
    int64_t n_leaves, const int32_t *__restrict__ leaf_start, const int32_t *__restrict__ leaf_ngas,
    const float *__restrict__ bbox, const float *__restrict__ hmax, TreeDev tree, double L0, double rc, PairOut o,
    const int32_t *__restrict__ leaf_box, const int32_t *__restrict__ box_root, const float *__restrict__ box_L) {
    // two per-warp buffers, each reused by a later phase (32 KB a block, five blocks per SM):
    // the traversal stack, then the sorted candidates; the candidates, then the image counts
    static_assert(kStackCap <= kCandCap, "stack inside the sorted-candidate buffer");
    __shared__ int32_t buf_a[kTravWarps][kCandCap];
    __shared__ int32_t buf_b[kTravWarps][kCandCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *const stack = buf_a[warp], *const sorted = buf_a[warp];
    int32_t *const cand = buf_b[warp];
    uint8_t *const ng = reinterpret_cast<uint8_t *>(buf_b[warp]), *const nh = ng + kCandCap;
    const unsigned below = (1u << lane) - 1u;
    const int64_t a = (int64_t)blockIdx.x * kTravWarps + warp;
    if (a >= n_leaves) return;  // whole warp leaves together; no block barrier below
    const bool a_any = leaf_start[a + 1] > leaf_start[a];
    const bool a_gas = leaf_ngas[a] > 0;
    const float *A = bbox + 6 * a;
    const float ha = hmax[a];
    const int bx = leaf_box ? leaf_box[a] : 0;
    const double L = leaf_box ? (double)box_L[bx] : L0;
    const int32_t root = leaf_box ? box_root[bx] : tree.root;
    const float Lf = (float)L;
    int nc = 0;
    bool bad = false;
    if (a_any) {
        if (kBrute) {
            for (int64_t b0 = 0; b0 < n_leaves; b0 += 32) {
                int64_t b = b0 + lane;
                bool keep = false;
                if (b < n_leaves && leaf_start[b + 1] > leaf_start[b]) {
                    float cut = fmaxf((float)rc, a_gas && leaf_ngas[b] > 0 ? 2.0f * fmaxf(ha, hmax[b]) : 0.0f);
                    keep = !clearly_apart(A, bbox + 6 * b, Lf, cut);
                }
                unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
                int pos = nc + __popc(m & below);
                if (keep && pos < kCandCap) cand[pos] = (int32_t)b;
                nc += __popc(m);
            }
        } else {
            int top = 1;
            if (lane == 0) stack[0] = root;
            __syncwarp();
            while (top > 0) {
                const int take = top < 32 ? top : 32;
                const int32_t nd = lane < take ? stack[top - 1 - lane] : -1;
                top -= take;
                __syncwarp();
                bool pass = false;
                int32_t lf = -1;
                if (nd >= 0) {
                    float cut = fmaxf((float)rc, a_gas ? 2.0f * fmaxf(ha, tree.node_hmax[nd]) : 0.0f);
                    pass = !clearly_apart(A, tree.node_box + 6 * (int64_t)nd, Lf, cut);
                    lf = tree.node_leaf[nd];
                }
                const bool is_leaf = pass && lf >= 0, inner = pass && lf < 0;
                unsigned m = __ballot_sync(CRK_FULL_MASK, is_leaf);
                int pos = nc + __popc(m & below);
                if (is_leaf && pos < kCandCap) cand[pos] = lf;
                nc += __popc(m);
                unsigned m2 = __ballot_sync(CRK_FULL_MASK, inner);
                int sp = top + 2 * __popc(m2 & below);
                if (inner && sp + 1 < kStackCap) {
                    stack[sp] = tree.node_right[nd];
                    stack[sp + 1] = tree.node_left[nd];
                }
                top += 2 * __popc(m2);
                if (top > kStackCap || nc > kCandCap) {
                    bad = true;
                    break;
                }
                __syncwarp();
            }
        }
        if (nc > kCandCap) bad = true;
    }
    __syncwarp();
    if (bad) {
        if (lane == 0) atomicAdd(&o.err[0], 1);
        return;
    }
    // ascending j-leaf order (rank sort; leaf ids are unique)
    for (int t = lane; t < nc; t += 32) {
        int32_t v = cand[t];
        int r = 0;
        for (int u = 0; u < nc; ++u) r += cand[u] < v;
        sorted[r] = v;
    }
    __syncwarp();
    // exact image counts of both lists
    const double rc2 = __dmul_rn(rc, rc);
    for (int t = lane; t < nc; t += 32) {
        int32_t b = sorted[t];
        int cg = leaf_images<false>(bbox, a, b, L, rc2, nullptr);
        int ch = 0;
        if (a_gas && leaf_ngas[b] > 0) {
            double hb = (double)hmax[b], hA = (double)ha;
            double cut = __dmul_rn(2.0, hA > hb ? hA : hb);
            ch = leaf_images<false>(bbox, a, b, L, __dmul_rn(cut, cut), nullptr);
        }
        ng[t] = (uint8_t)cg;
        nh[t] = (uint8_t)ch;
    }
    __syncwarp();
    int tot[4] = {0, 0, 0, 0};
    for (int t0 = 0; t0 < nc; t0 += 32) {
        int t = t0 + lane;
        int cg = t < nc ? ng[t] : 0, ch = t < nc ? nh[t] : 0;
        int v[4] = {cg, cg > 0, ch, ch > 0};
        for (int k = 0; k < 4; ++k) {
            int s;
            warp_excl_scan(v[k], lane, s);
            tot[k] += s;
        }
    }
    unsigned long long base[4] = {0, 0, 0, 0};
    if (lane == 0)
        for (int k = 0; k < 4; ++k) base[k] = tot[k] ? atomicAdd(&o.cursor[k], (unsigned long long)tot[k]) : 0ull;
    bool over = false;
    for (int k = 0; k < 4; ++k) {
        base[k] = __shfl_sync(CRK_FULL_MASK, base[k], 0);
        over |= base[k] + (unsigned long long)tot[k] > (unsigned long long)o.cap[k];
    }
    if (over) {
        if (lane == 0) atomicAdd(&o.err[1], 1);
        return;
    }
    if (lane == 0)
        for (int k = 0; k < 4; ++k) {
            o.start[k][a] = (int32_t)base[k];
            o.count[k][a] = tot[k];
        }
    int run[4] = {0, 0, 0, 0};
    for (int t0 = 0; t0 < nc; t0 += 32) {
        int t = t0 + lane;
        int cg = t < nc ? ng[t] : 0, ch = t < nc ? nh[t] : 0;
        int v[4] = {cg, cg > 0, ch, ch > 0};
        int off[4];
        for (int k = 0; k < 4; ++k) {
            int s;
            off[k] = run[k] + warp_excl_scan(v[k], lane, s);
            run[k] += s;
        }
        if (t < nc) {
            int32_t b = sorted[t];
            if (cg > 0) {
                o.gpair[base[1] + off[1]] = b;
                leaf_images<true>(bbox, a, b, L, rc2, o.gimg + base[0] + off[0]);
            }
            if (ch > 0) {
                double hb = (double)hmax[b], hA = (double)ha;
                double cut = __dmul_rn(2.0, hA > hb ? hA : hb);
                o.hpair[base[3] + off[3]] = b;
                leaf_images<true>(bbox, a, b, L, __dmul_rn(cut, cut), o.himg + base[2] + off[2]);
            }
        }
    }
}

__global__ void leaf_box_to_node_kernel(int64_t n_leaves, const float *__restrict__ bbox,
                                        const float *__restrict__ hmax, const int32_t *__restrict__ leaf_node,
                                        float *__restrict__ node_box, float *__restrict__ node_hmax) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_leaves) return;
    int64_t nd = leaf_node[a];
    for (int q = 0; q < 6; ++q) node_box[6 * nd + q] = bbox[6 * a + q];
    node_hmax[nd] = hmax[a];
}

// one level of split nodes, deepest level first: node h_max = max of the children
__global__ void node_hmax_kernel(int nseg, LevelDev lv, const int32_t *__restrict__ left,
                                 const int32_t *__restrict__ right, float *__restrict__ node_hmax) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg || lv.k[s] <= 0) return;
    int nd = lv.node[s];
    node_hmax[nd] = fmaxf(node_hmax[left[nd]], node_hmax[right[nd]]);
}

struct HostSeg {
    int32_t lo, hi, k, child, node;
};

}  // namespace

// ---------------------------------------------------------------------------------
void crk_rcb_shape_free(crk_ctx *ctx) {
    if (!ctx || !ctx->rcb) return;
    crk_rcb_shape *r = ctx->rcb;
    cudaFree(r->dtab);
    cudaFree(r->leaf_start);
    cudaFree(r->left);
    cudaFree(r->right);
    cudaFree(r->leaf_of);
    cudaFree(r->leaf_node);
    cudaFree(r->d_leaf_box);
    cudaFree(r->d_box_root);
    delete r;
    ctx->rcb = nullptr;
}

// The RCB tree shape for the boxes [box_start[b], box_start[b+1]) and
// max_leaf: level segment tables, leaf starts, children (one root per box).
static int rcb_shape(crk_ctx *ctx, const std::vector<int64_t> &box_start, int ml, const crk_rcb_shape **out) {
    const int64_t n = box_start.back();
    if (ctx->rcb && ctx->rcb->box_start == box_start && ctx->rcb->max_leaf == ml) {
        *out = ctx->rcb;
        return CRK_OK;
    }
    CRK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the old shape may still be in use
    crk_rcb_shape_free(ctx);
    crk_rcb_shape *r = new crk_rcb_shape();
    r->n = n;
    r->max_leaf = ml;
    r->box_start = box_start;
    const int nbox = (int)box_start.size() - 1;
    std::vector<std::vector<HostSeg>> levels;
    std::vector<HostSeg> cur;
    std::vector<int32_t> left, right;
    int32_t next_node = 0;
    r->box_root.assign(nbox, -1);
    for (int b = 0; b < nbox; ++b)
        if (box_start[b + 1] > box_start[b]) {
            r->box_root[b] = next_node;
            cur.push_back({(int32_t)box_start[b], (int32_t)box_start[b + 1], 0, 0, next_node++});
        }
    left.assign(next_node > 0 ? next_node : 1, -1);
    right.assign(next_node > 0 ? next_node : 1, -1);
    while (!cur.empty()) {
        bool any = false;
        for (auto &sg : cur)
            if (sg.hi - sg.lo > ml) {
                sg.k = (sg.hi - sg.lo) / 2;
                any = true;
            }
        if (!any) break;
        std::vector<HostSeg> nxt;
        nxt.reserve(cur.size() * 2);
        for (auto &sg : cur) {
            sg.child = (int32_t)nxt.size();
            if (sg.k > 0) {
                int32_t l = next_node++, rr = next_node++;
                left.resize(next_node, -1);
                right.resize(next_node, -1);
                left[sg.node] = l;
                right[sg.node] = rr;
                nxt.push_back({sg.lo, sg.lo + sg.k, 0, 0, l});
                nxt.push_back({sg.lo + sg.k, sg.hi, 0, 0, rr});
            } else {
                nxt.push_back({sg.lo, sg.hi, 0, 0, sg.node});
            }
        }
        levels.push_back(cur);
        cur.swap(nxt);
    }
    const int64_t nl = (int64_t)cur.size();
    r->n_leaves = nl;
    r->n_nodes = next_node;
    std::vector<int32_t> leaf_start(nl + 1), leaf_of(next_node > 0 ? next_node : 1, -1), leaf_node(nl > 0 ? nl : 1);
    r->leaf_box.assign(nl > 0 ? nl : 1, 0);
    for (int64_t a = 0, b = 0; a < nl; ++a) {
        leaf_start[a] = cur[a].lo;
        leaf_of[cur[a].node] = (int32_t)a;
        leaf_node[a] = cur[a].node;
        while (b + 1 < nbox && box_start[b + 1] <= cur[a].lo) ++b;
        r->leaf_box[a] = (int32_t)b;
        r->max_leaf_size = std::max(r->max_leaf_size, cur[a].hi - cur[a].lo);
    }
    leaf_start[nl] = (int32_t)n;
    size_t tot = 0;
    for (auto &L : levels) {
        r->level_off.push_back(tot);
        r->level_size.push_back(L.size());
        int32_t mx = 0;
        for (auto &sg : L) mx = std::max(mx, sg.hi - sg.lo);
        r->level_max.push_back(mx);
        tot += 7 * L.size();
    }
    std::vector<int32_t> packed(tot > 0 ? tot : 1);
    for (size_t d = 0; d < levels.size(); ++d) {
        const auto &L = levels[d];
        size_t m = L.size(), off = r->level_off[d];
        int64_t leftbase = 0;
        for (size_t q = 0; q < m; ++q) {
            packed[off + q] = L[q].lo;
            packed[off + m + q] = L[q].hi;
            packed[off + 2 * m + q] = L[q].k;
            packed[off + 3 * m + q] = L[q].child;
            packed[off + 4 * m + q] = L[q].node;
            packed[off + 5 * m + q] = 0;
            packed[off + 6 * m + q] = (int32_t)leftbase;
            leftbase += L[q].k;
        }
    }
    auto dev = [&](int32_t **p, const std::vector<int32_t> &v) -> int {
        if (cudaMalloc(p, sizeof(int32_t) * (v.size() > 0 ? v.size() : 1)) != cudaSuccess) {
            cudaGetLastError();
            return CRK_ENOMEM;
        }
        return cudaMemcpy(*p, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice) == cudaSuccess
                   ? CRK_OK
                   : CRK_ECUDA;
    };
    int rc = CRK_OK;
    if (!rc) rc = dev(&r->dtab, packed);
    if (!rc) rc = dev(&r->leaf_start, leaf_start);
    if (!rc) rc = dev(&r->left, left);
    if (!rc) rc = dev(&r->right, right);
    if (!rc) rc = dev(&r->leaf_of, leaf_of);
    if (!rc) rc = dev(&r->leaf_node, leaf_node);
    if (!rc) rc = dev(&r->d_leaf_box, r->leaf_box);
    if (!rc) rc = dev(&r->d_box_root, r->box_root);
    ctx->rcb = r;
    if (rc) {
        crk_rcb_shape_free(ctx);
        return crk_fail(ctx, rc, "RCB shape tables");
    }
    *out = r;
    return CRK_OK;
}

namespace {
struct Tracer {
    crk_ctx *ctx;
    bool on;  // never during a rebuild (it may be captured)
    std::chrono::steady_clock::time_point t;
    Tracer(crk_ctx *c, bool allowed) : ctx(c), on(allowed && c->trace), t(std::chrono::steady_clock::now()) {}
    void mark(const char *what) {
        if (!on) return;
        cudaStreamSynchronize(ctx->stream);
        auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[crk] %-18s %8.3f ms\n", what, std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};
}  // namespace

__global__ void init_node_of_kernel(int64_t n, const int32_t *__restrict__ box_of, const int32_t *__restrict__ seg_of_box,
                                    int32_t *__restrict__ node_of) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) node_of[p] = seg_of_box[box_of[p]];
}

// The host checks of a build as bits of the leaves' status word (rebuilds, which do not synchronise).
__global__ void leaf_status_kernel(const int32_t *__restrict__ flags, const unsigned *__restrict__ hbits,
                                   const float *__restrict__ box_L, int nbox, int32_t n_gas, int32_t *__restrict__ status) {
    int32_t s = 0;
    if (threadIdx.x == 0) {
        if (flags[0] > 0) s |= CRK_LEAVES_BAD_POSITION;
        if (flags[1] > 0) s |= CRK_LEAVES_BAD_H;
        if (flags[2] != n_gas) s |= CRK_LEAVES_GAS_COUNT;
        if (flags[4] > 0) s |= CRK_LEAVES_LEAF_SIZE;
        if (flags[5] > 0) s |= CRK_LEAVES_INTERNAL;
    }
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
        const float hm = __uint_as_float(hbits[b]);
        if (!(2.0 * (double)hm < 0.5 * (double)box_L[b])) s |= CRK_LEAVES_HMAX;
    }
    if (s) atomicOr(status, s);
}

__global__ void pairs_status_kernel(const int32_t *__restrict__ err, int32_t *__restrict__ status) {
    int32_t s = 0;
    if (err[0] > 0) s |= CRK_LEAVES_CANDIDATES;
    if (err[1] > 0) s |= CRK_LEAVES_IMAGE_CAP;
    if (s) atomicOr(status, s);
}

// Leaves of one box (nbox = 1) or of several independent periodic boxes whose
// particles are the consecutive ranges box_start[b] .. box_start[b+1].
// re != NULL: rebuild those leaves in place (crk_leaves_rebuild): no host synchronisation and no
// allocation; the host checks become bits of the leaves' device status word.
static int build_leaves_impl(crk_ctx *ctx, const crk_particles *p, const float *h, const crk_leaf_params *lp,
                             const std::vector<int64_t> &box_start, const std::vector<float> &box_side,
                             crk_leaves **out, crk_leaves *re = nullptr) {
    if (!p || !lp || !out) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (!re) *out = nullptr;
    const int64_t n = p->n;
    const int nbox = (int)box_side.size();
    if (n < 0 || n > 2000000000LL) return crk_fail(ctx, CRK_EINVAL, "particle count out of range");
    if (n > 0 && (!p->x || !p->y || !p->z || !p->species || !h)) return crk_fail(ctx, CRK_EINVAL, "null array");
    if (lp->mode != 0 && lp->mode != 1) return crk_fail(ctx, CRK_EINVAL, "leaf mode must be 0 or 1");
    if (lp->mode == 0 && nbox != 1) return crk_fail(ctx, CRK_EINVAL, "chaining-mesh leaves take one box");
    if (lp->mode == 0 && (lp->cells_per_side < 1 || lp->cells_per_side > 40))
        return crk_fail(ctx, CRK_EINVAL, "cells_per_side must be in [1, 40]");
    if (lp->mode == 1 && (lp->max_leaf < 1 || lp->max_leaf > kMaxLeafCap))
        return crk_fail(ctx, CRK_EINVAL, "max_leaf must be in [1, 1024]");
    float box_max = 0.0f;
    for (int b = 0; b < nbox; ++b) {
        if (!(box_side[b] > 0.0f)) return crk_fail(ctx, CRK_EINVAL, "box %d: side must be positive", b);
        if (box_start[b + 1] < box_start[b]) return crk_fail(ctx, CRK_EINVAL, "box starts must not decrease");
        if (box_start[b + 1] > box_start[b] && (!(lp->r_cut_grav > 0.0f) ||
                                                !((double)lp->r_cut_grav < 0.5 * (double)box_side[b])))
            return crk_fail(ctx, CRK_EBOX, "box %d: r_cut_grav must be positive and below box/2", b);
        box_max = std::max(box_max, box_side[b]);
    }
    if (box_start[0] != 0 || box_start[nbox] != n) return crk_fail(ctx, CRK_EINVAL, "box starts must span [0, n]");
    if (re) {
        if (re->n != n || re->box_start != box_start || re->box_side != box_side || re->mode != lp->mode ||
            re->max_leaf != lp->max_leaf || re->cells != lp->cells_per_side || re->r_cut_grav != lp->r_cut_grav)
            return crk_fail(ctx, CRK_ESTATE, "rebuild: particles, boxes or leaf parameters differ from the leaves'");
        if (re->grav_lists.list) return crk_fail(ctx, CRK_ESTATE, "rebuild: leaves with gravity lists");
        if (re->gas_lists.list && !re->gas_lists.onepass)
            return crk_fail(ctx, CRK_ESTATE, "rebuild: gas lists of the exact two-pass build");
        if (!re->dev || !re->boxtab) return crk_fail(ctx, CRK_ESTATE, "rebuild: leaves without rebuild state");
        if (n > 0 && lp->mode == 1 && !(ctx->rcb && ctx->rcb->box_start == box_start && ctx->rcb->max_leaf == lp->max_leaf)) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            cudaStreamIsCapturing(ctx->stream, &cs);
            if (cs != cudaStreamCaptureStatusNone)
                return crk_fail(ctx, CRK_ESTATE, "rebuild under capture: the context holds another RCB shape");
        }
    }

    Tracer tr(ctx, re == nullptr);
    crk_leaves *lv = re ? re : new crk_leaves();
    lv->n = n;
    lv->box = box_max;
    lv->nbox = nbox;
    lv->mode = lp->mode;
    lv->r_cut_grav = lp->r_cut_grav;
    lv->max_leaf = lp->max_leaf;
    lv->cells = lp->cells_per_side;
    lv->box_start = box_start;
    lv->box_side = box_side;
    if (!re)  // the split gravity sweeps want RCB cells of 8 in the gravity order (kept by rebuilds)
        lv->cells8 = ctx->variant[CRK_K_GRAVITY] == CRK_VARIANT_SPLIT8 ||
                     ctx->variant[CRK_K_GRAVITY_ADJOINT] == CRK_VARIANT_SPLIT8;
    cudaStream_t st = ctx->stream;
    int rc = CRK_OK;
#define TRY(expr)                          \
    do {                                   \
        rc = (expr);                       \
        if (rc != CRK_OK) goto fail;       \
    } while (0)
#define ALLOC(ptr, type, count)                                                                          \
    do {                                                                                                 \
        if (!re) { /* a rebuild keeps the buffers of the first build */                                \
            ptr = (type *)crk_leaves_alloc(ctx, lv, sizeof(type) * (size_t)((count) > 0 ? (count) : 1)); \
            if (!ptr) {                                                                                  \
                rc = crk_fail(ctx, CRK_ENOMEM, "leaf allocation");                                       \
                goto fail;                                                                               \
            }                                                                                            \
        }                                                                                                \
    } while (0)
#define KCHECK(what)                                       \
    do {                                                   \
        cudaError_t e_ = cudaGetLastError();               \
        if (e_ != cudaSuccess) {                           \
            rc = crk_check_cuda(ctx, e_, what);            \
            goto fail;                                     \
        }                                                  \
    } while (0)
    {
        // flags[0..15]; then per box: hmax bits, side, start (int64), segment index
        const size_t fbytes = 64 + 4 * (size_t)nbox + 4 * (size_t)nbox + 8 * (size_t)(nbox + 1) + 4 * (size_t)nbox;
        int32_t *flags = (int32_t *)crk_scratch(ctx, 0, fbytes + 64);
        if (!flags) { rc = crk_fail(ctx, CRK_ENOMEM, "scratch"); goto fail; }
        unsigned *hbits = (unsigned *)(flags + 16);
        float *box_L = (float *)(flags + 16 + nbox);
        int64_t *d_box_start = (int64_t *)(((uintptr_t)(flags + 16 + 2 * nbox) + 7) & ~(uintptr_t)7);
        int32_t *seg_of_box = (int32_t *)(d_box_start + nbox + 1);
        std::vector<int32_t> h_seg(nbox, 0);
        for (int b = 0, q = 0; b < nbox; ++b) {
            h_seg[b] = q;
            if (box_start[b + 1] > box_start[b]) ++q;
        }
        if (!re) {
            if (cudaMemcpyAsync(box_L, box_side.data(), 4 * (size_t)nbox, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(d_box_start, box_start.data(), 8 * (size_t)(nbox + 1), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(seg_of_box, h_seg.data(), 4 * (size_t)nbox, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "leaf build set-up copies");
                goto fail;
            }
            // the rebuild state: a device copy of the box tables, the status word, group counts and cursors
            lv->boxtab_bytes = fbytes + 64;
            lv->boxtab = (unsigned char *)crk_leaves_alloc(ctx, lv, lv->boxtab_bytes);
            lv->dev = (int32_t *)crk_leaves_alloc(ctx, lv, 256);
            if (!lv->boxtab || !lv->dev) { rc = crk_fail(ctx, CRK_ENOMEM, "leaf allocation"); goto fail; }
            if (cudaMemcpyAsync(lv->boxtab, flags, lv->boxtab_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "leaf build set-up copies");
                goto fail;
            }
        } else if (cudaMemcpyAsync(flags, lv->boxtab, lv->boxtab_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            rc = crk_fail(ctx, CRK_ECUDA, "leaf build set-up copies");
            goto fail;
        }
        if (cudaMemsetAsync(flags, 0, 64 + 4 * (size_t)nbox, st) != cudaSuccess ||
            cudaMemsetAsync(lv->dev, 0, 256, st) != cudaSuccess) {
            rc = crk_fail(ctx, CRK_ECUDA, "memset");
            goto fail;
        }
        int32_t *box_of = nullptr;
        if (nbox > 1 && n > 0) {
            box_of = (int32_t *)crk_scratch(ctx, 16, sizeof(int32_t) * (size_t)n);
            if (!box_of) { rc = crk_fail(ctx, CRK_ENOMEM, "scratch"); goto fail; }
            box_of_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, d_box_start, nbox, box_of);
            ++ctx->launches;
        }
        if (n > 0) {
            validate_kernel<<<(unsigned)((n + kValTile - 1) / kValTile), 256, 0, st>>>(
                p->x, p->y, p->z, p->species, h, n, box_of, box_L, flags, hbits);
            ++ctx->launches;
        }
        int32_t *members = nullptr;  // particle ids grouped by leaf
        int64_t nl = 0;
        const crk_rcb_shape *shape = nullptr;
        float *node_box = nullptr, *node_hmax = nullptr;

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
            if (n > 0) {
                mesh_keys_kernel<<<crk_grid(n, 256), 256, 0, st>>>(p->x, p->y, p->z, n, nc, (double)box_side[0], keys,
                                                                   vals, cnts);
                ++ctx->launches;
            }
            int bits = 1;
            while ((1LL << bits) < nl) ++bits;
            TRY(crk_radix_sort_u32(ctx, keys, vals, n, bits));
            TRY(crk_exclusive_scan_i32(ctx, cnts, lv->leaf_start, nl + 1, nullptr));
            members = vals;
        } else {
            TRY(rcb_shape(ctx, box_start, lp->max_leaf, &shape));
            nl = shape->n_leaves;
            ALLOC(lv->leaf_start, int32_t, nl + 1);
            if (cudaMemcpyAsync(lv->leaf_start, shape->leaf_start, sizeof(int32_t) * (size_t)(nl + 1),
                                cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                rc = crk_fail(ctx, CRK_ECUDA, "leaf starts");
                goto fail;
            }
            ALLOC(lv->node_box, float, 6 * shape->n_nodes);
            ALLOC(lv->node_hmax, float, shape->n_nodes);
            node_box = lv->node_box;
            node_hmax = lv->node_hmax;
            tr.mark("shape");
            int32_t *Lc[3];
            size_t nb = sizeof(int32_t) * (size_t)(n > 0 ? n : 1);
            uint32_t *keys = (uint32_t *)crk_scratch(ctx, 1, nb);
            int32_t *R[3], *Ac[3][2], *An[3][2];
            for (int a = 0; a < 3; ++a) {
                Lc[a] = (int32_t *)crk_scratch(ctx, 2 + a, nb);
                R[a] = (int32_t *)crk_scratch(ctx, 5 + a, nb);
                for (int c = 0; c < 2; ++c) {
                    Ac[a][c] = (int32_t *)crk_scratch(ctx, 19 + 2 * a + c, nb);
                    An[a][c] = (int32_t *)crk_scratch(ctx, 25 + 2 * a + c, nb);
                }
            }
            int32_t *node_of = (int32_t *)crk_scratch(ctx, 8, nb);
            int32_t *node_nx = (int32_t *)crk_scratch(ctx, 9, nb);
            int32_t *mem = (int32_t *)crk_scratch(ctx, 10, nb);
            int32_t *flag = (int32_t *)crk_scratch(ctx, 11, nb + 3 * sizeof(int32_t) * (size_t)(n / 2048 + 2));
            size_t max_seg = 1;
            for (size_t m : shape->level_size) max_seg = std::max(max_seg, m);
            SegRec *segs = (SegRec *)crk_scratch(ctx, 31, sizeof(SegRec) * max_seg);
            bool ok = keys && node_of && node_nx && mem && flag && segs;
            for (int a = 0; a < 3; ++a) ok = ok && Lc[a] && R[a] && Ac[a][0] && Ac[a][1] && An[a][0] && An[a][1];
            if (!ok) {
                rc = crk_fail(ctx, CRK_ENOMEM, "scratch");
                goto fail;
            }
            const float *cs[3] = {p->x, p->y, p->z};
            for (int a = 0; a < 3 && n > 0; ++a) {
                init_axis_keys_kernel<<<crk_grid(n, 256), 256, 0, st>>>(cs[a], n, keys, Lc[a]);
                ++ctx->launches;
                TRY(crk_radix_sort_u32(ctx, keys, Lc[a], n, 32));
                if (box_of) {  // stable by box: (box, coordinate, index) order
                    box_keys_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, Lc[a], box_of, keys);
                    ++ctx->launches;
                    int bits = 1;
                    while ((1 << bits) < nbox) ++bits;
                    TRY(crk_radix_sort_u32(ctx, keys, Lc[a], n, bits));
                }
            }
            tr.mark("axis sorts");
            const AxisOrder ord{{Lc[0], Lc[1], Lc[2]}, {R[0], R[1], R[2]}};
            if (n > 0) {
                for (int t = 0; t < 3; ++t) rank_of_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, Lc[t], R[t]);
                // list a, column c holds the rank along axis (a + 1 + c) % 3
                for (int t = 0; t < 3; ++t) {
                    const int a0 = (t + 2) % 3, a1 = (t + 1) % 3;
                    rank_column_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, Lc[a0], R[t], Ac[a0][0]);
                    rank_column_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, Lc[a1], R[t], Ac[a1][1]);
                }
                ctx->launches += 9;
                if (box_of) {
                    init_node_of_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, box_of, seg_of_box, node_of);
                    ++ctx->launches;
                } else if (cudaMemsetAsync(node_of, 0, sizeof(int32_t) * (size_t)n, st) != cudaSuccess) {
                    rc = crk_fail(ctx, CRK_ECUDA, "memset");
                    goto fail;
                }
            }
            // levels [0, d_local) stream through DRAM; the rest run in shared memory, one block per
            // segment of level d_local (every segment there holds at most kLocalCap entries)
            const int n_lev = (int)shape->level_size.size();
            int d_local = n_lev;
            for (int d = 0; d < n_lev; ++d)
                if (shape->level_max[d] <= kLocalCap) {
                    d_local = d;
                    break;
                }
            if (n_lev - d_local > kLocalLevels) d_local = n_lev - kLocalLevels;
            for (int d = 0; d < d_local; ++d) {
                int m = (int)shape->level_size[d];
                int32_t *tab = shape->dtab + shape->level_off[d];
                LevelDev dv{tab, tab + m, tab + 2 * m, tab + 3 * m, tab + 4 * m, tab + 5 * m, tab + 6 * m};
                const RankLists Lr{{{Ac[0][0], Ac[0][1]}, {Ac[1][0], Ac[1][1]}, {Ac[2][0], Ac[2][1]}}};
                const RankListsOut Lo{{{An[0][0], An[0][1]}, {An[1][0], An[1][1]}, {An[2][0], An[2][1]}}};
                rcb_axis_kernel<<<crk_grid(m, 128), 128, 0, st>>>(m, dv, Lr, ord, p->x, p->y, p->z, node_box, segs);
                const int64_t nbt = (n + kPartTile - 1) / kPartTile;
                rcb_count3_kernel<<<(unsigned)nbt, kPartThreads, 0, st>>>(n, segs, node_of, Lr, flag, nbt);
                rcb_scan3_kernel<<<1, 1024, 0, st>>>(flag, nbt);
                rcb_scatter3_kernel<<<(unsigned)nbt, kPartThreads, 0, st>>>(n, segs, node_of, Lr, flag, nbt, Lo, node_nx,
                                                                            flags + 5);
                ctx->launches += 4;
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 2; ++c) std::swap(Ac[a][c], An[a][c]);
                std::swap(node_of, node_nx);
                KCHECK("rcb level");
            }
            const RankLists Lfin{{{Ac[0][0], Ac[0][1]}, {Ac[1][0], Ac[1][1]}, {Ac[2][0], Ac[2][1]}}};
            if (n > 0 && d_local < n_lev) {
                static bool smem_set = false;  // opt-in above 48 KB, once (never inside a capture: a
                if (!smem_set) {               // rebuild always follows a fresh build)
                    cudaFuncSetAttribute(rcb_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLocalSmem);
                    smem_set = true;
                }
                LocalShape ls{};
                ls.nlev = n_lev - d_local;
                for (int l = 0; l < ls.nlev; ++l) {
                    ls.tab[l] = shape->dtab + shape->level_off[d_local + l];
                    ls.m[l] = (int32_t)shape->level_size[d_local + l];
                }
                rcb_local_kernel<<<(unsigned)shape->level_size[d_local], kLocalThreads, kLocalSmem, st>>>(
                    n, ls, Lfin, ord, p->x, p->y, p->z, node_box, mem, flags + 5);
                ++ctx->launches;
                KCHECK("rcb local levels");
            } else if (n > 0) {
                rank_members_kernel<<<crk_grid(n, 256), 256, 0, st>>>(n, Lfin, ord, mem);
                ++ctx->launches;
            }
            tr.mark("rcb levels");
            members = mem;
        }
        lv->n_leaves = nl;
        ALLOC(lv->perm, int32_t, n);
        ALLOC(lv->kperm, int32_t, n);
        ALLOC(lv->leaf_ngas, int32_t, nl);
        ALLOC(lv->bbox, float, 6 * nl);
        ALLOC(lv->hmax, float, nl);
        ALLOC(lv->pos, float4, n);
        ALLOC(lv->kperm_g, int32_t, n);
        ALLOC(lv->pos_g, float4, n);
        ALLOC(lv->kinv, int32_t, n);
        ALLOC(lv->kinv_g, int32_t, n);
        if (nl > 0) {
            if (lp->mode == 1 && shape && shape->max_leaf_size <= 128)
                leaf_data_kernel<128><<<(unsigned)nl, 32, 0, st>>>(nl, lv->leaf_start, members, p->x, p->y, p->z,
                                                                   p->species, h, lv->perm, lv->kperm, lv->leaf_ngas,
                                                                   lv->bbox, lv->hmax, lv->pos, lv->kperm_g,
                                                                   lv->pos_g, lv->kinv, lv->kinv_g, flags + 4,
                                                                   lv->cells8 ? 1 : 0);
            else
                leaf_data_kernel<kMaxLeafCap><<<(unsigned)nl, 128, 0, st>>>(
                    nl, lv->leaf_start, members, p->x, p->y, p->z, p->species, h, lv->perm, lv->kperm, lv->leaf_ngas,
                    lv->bbox, lv->hmax, lv->pos, lv->kperm_g, lv->pos_g, lv->kinv, lv->kinv_g, flags + 4, 0);
            ++ctx->launches;
        }
        KCHECK("leaf data");
        if (re) {  // the checks below, on the device
            leaf_status_kernel<<<1, 256, 0, st>>>(flags, hbits, box_L, nbox, (int32_t)lv->n_gas, lv->dev);
            ++ctx->launches;
        }
        // ---- host checks (one synchronisation)
        int32_t hflags[16];
        std::vector<unsigned> hb(nbox);
        if (re) {
        } else if (cudaMemcpyAsync(hflags, flags, 64, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hb.data(), hbits, 4 * (size_t)nbox, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = crk_fail(ctx, CRK_ECUDA, "leaf build: %s", cudaGetErrorString(cudaGetLastError()));
            goto fail;
        }
        tr.mark("leaf data");
        if (!re) {
        if (hflags[0] > 0) { rc = crk_fail(ctx, CRK_EBOX, "%d particle positions outside [0, box)", hflags[0]); goto fail; }
        if (hflags[1] > 0) { rc = crk_fail(ctx, CRK_EINVAL, "%d gas particles with h <= 0 or not finite", hflags[1]); goto fail; }
        if (hflags[4] > 0) { rc = crk_fail(ctx, CRK_EINVAL, "a leaf holds more than %d particles", kMaxLeafCap); goto fail; }
        if (hflags[5] > 0) { rc = crk_fail(ctx, CRK_ESTATE, "internal error: inconsistent RCB partition"); goto fail; }
        lv->n_gas = hflags[2];
        float hmax_all = 0.0f;
        for (int b = 0; b < nbox; ++b) {
            float hm;
            std::memcpy(&hm, &hb[b], sizeof(float));
            hmax_all = std::max(hmax_all, hm);
            if (!(2.0 * (double)hm < 0.5 * (double)box_side[b])) {
                rc = crk_fail(ctx, CRK_EBOX, "box %d: 2 h_max = %g is not below box/2", b, 2.0 * hm);
                goto fail;
            }
        }
        lv->hmax_all = hmax_all;
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
            lv->max_leaf_size = shape->max_leaf_size;
        }
        }
        // ---- tree for traversal (RCB): leaf boxes and h_max into the nodes, then bottom-up h_max
        TreeDev tree{};
        const int brute = lp->mode == 0 ? 1 : 0;
        if (!brute && nl > 0) {
            leaf_box_to_node_kernel<<<crk_grid(nl, 128), 128, 0, st>>>(nl, lv->bbox, lv->hmax, shape->leaf_node,
                                                                       node_box, node_hmax);
            ++ctx->launches;
            for (size_t d = shape->level_size.size(); d-- > 0;) {
                int m = (int)shape->level_size[d];
                int32_t *tab = shape->dtab + shape->level_off[d];
                LevelDev dv{tab, tab + m, tab + 2 * m, tab + 3 * m, tab + 4 * m, tab + 5 * m, tab + 6 * m};
                node_hmax_kernel<<<crk_grid(m, 128), 128, 0, st>>>(m, dv, shape->left, shape->right, node_hmax);
                ++ctx->launches;
            }
            KCHECK("node h_max");
            tree.node_box = node_box;
            tree.node_hmax = node_hmax;
            tree.node_left = shape->left;
            tree.node_right = shape->right;
            tree.node_leaf = shape->leaf_of;
            tree.root = 0;
        }
        // ---- leaf-pair image lists, one warp per leaf; retried once with exact
        // capacities if the first estimate is too small
        {
            int32_t *se[8] = {lv->gimg_start, lv->gimg_cnt, lv->gpair_start, lv->gpair_cnt,
                              lv->himg_start, lv->himg_cnt, lv->hpair_start, lv->hpair_cnt};
            for (int q = 0; q < 8; ++q) ALLOC(se[q], int32_t, nl);
            // the list cursors live with the leaves (a rebuild refreshes the counts from them later)
            unsigned long long *cur = (unsigned long long *)(lv->dev + 16);
            int64_t cap[4] = {48 * nl + 64, 32 * nl + 64, 48 * nl + 64, 32 * nl + 64};
            if (re)
                for (int k = 0; k < 4; ++k) cap[k] = lv->img_cap[k];
            crk_image *gimg = lv->gimg, *himg = lv->himg;
            int32_t *gpair = lv->gpair_list, *hpair = lv->hpair_list;
            unsigned long long hcur[6] = {(unsigned long long)lv->n_gimg, (unsigned long long)lv->n_gpairs,
                                          (unsigned long long)lv->n_himg, (unsigned long long)lv->n_hpairs, 0, 0};
            for (int attempt = 0; attempt < 2; ++attempt) {
                // capacity blocks come from the leaves' own allocations; a retry leaves the
                // first (too small) blocks unused until the leaves are freed
                ALLOC(gimg, crk_image, cap[0]);
                ALLOC(gpair, int32_t, cap[1]);
                ALLOC(himg, crk_image, cap[2]);
                ALLOC(hpair, int32_t, cap[3]);
                if (cudaMemsetAsync(cur, 0, 64, st) != cudaSuccess) { rc = crk_fail(ctx, CRK_ECUDA, "memset"); goto fail; }
                PairOut po;
                for (int k = 0; k < 4; ++k) {
                    po.start[k] = se[2 * k];
                    po.count[k] = se[2 * k + 1];
                    po.cap[k] = cap[k];
                }
                po.gimg = gimg; po.gpair = gpair; po.himg = himg; po.hpair = hpair;
                po.cursor = cur;
                po.err = (int32_t *)(cur + 4);
                if (nl > 0) {
                    unsigned grid = (unsigned)((nl + kTravWarps - 1) / kTravWarps);
                    if (brute)
                        leaf_pairs_warp_kernel<true><<<grid, kTravWarps * 32, 0, st>>>(
                            nl, lv->leaf_start, lv->leaf_ngas, lv->bbox, lv->hmax, tree, (double)box_side[0],
                            (double)lp->r_cut_grav, po, nullptr, nullptr, nullptr);
                    else
                        leaf_pairs_warp_kernel<false><<<grid, kTravWarps * 32, 0, st>>>(
                            nl, lv->leaf_start, lv->leaf_ngas, lv->bbox, lv->hmax, tree, (double)box_side[0],
                            (double)lp->r_cut_grav, po, shape->d_leaf_box, shape->d_box_root, box_L);
                    ++ctx->launches;
                }
                KCHECK("pair lists");
                if (re) {  // one attempt at the first build's capacities; overflows go to the status word
                    pairs_status_kernel<<<1, 1, 0, st>>>(po.err, lv->dev);
                    ++ctx->launches;
                    break;
                }
                if (cudaMemcpyAsync(hcur, cur, 48, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = crk_fail(ctx, CRK_ECUDA, "pair lists: %s", cudaGetErrorString(cudaGetLastError()));
                    goto fail;
                }
                const int32_t *herr = (const int32_t *)(hcur + 4);
                if (herr[0] > 0) {
                    rc = crk_fail(ctx, CRK_EINVAL,
                                  "%d leaves have more than %d candidate leaves within the cut (leaves too small "
                                  "for r_cut or h)", herr[0], kCandCap);
                    goto fail;
                }
                if (herr[1] == 0) break;
                // exact counts plus an eighth (room for the rebuilds of moved particles)
                for (int k = 0; k < 4; ++k) cap[k] = (int64_t)hcur[k] + (int64_t)(hcur[k] / 8) + 64;
                if (attempt == 1) { rc = crk_fail(ctx, CRK_ESTATE, "pair list capacity"); goto fail; }
            }
            lv->gimg_start = se[0]; lv->gimg_cnt = se[1]; lv->gimg = gimg; lv->n_gimg = (int64_t)hcur[0];
            lv->gpair_start = se[2]; lv->gpair_cnt = se[3]; lv->gpair_list = gpair; lv->n_gpairs = (int64_t)hcur[1];
            lv->himg_start = se[4]; lv->himg_cnt = se[5]; lv->himg = himg; lv->n_himg = (int64_t)hcur[2];
            lv->hpair_start = se[6]; lv->hpair_cnt = se[7]; lv->hpair_list = hpair; lv->n_hpairs = (int64_t)hcur[3];
            for (int k = 0; k < 4; ++k) lv->img_cap[k] = cap[k];
        }
        tr.mark("pair lists");
        bool gas_lists = false;  // every gas-pair kernel may walk the gas lists
        for (int k : {CRK_K_GEOMETRY, CRK_K_CORRECTIONS, CRK_K_HYDRO, CRK_K_GEOMETRY_ADJOINT, CRK_K_EXTRAS, CRK_K_ACCEL,
                      CRK_K_ENERGY})
            gas_lists = gas_lists || ctx->variant[k] == CRK_VARIANT_LISTS;
        if (re ? lv->gas_lists.list != nullptr : gas_lists) TRY(crk_build_lists(ctx, lv, true, re != nullptr));
        tr.mark("gas lists");
        if (!re && (ctx->variant[CRK_K_GRAVITY] == CRK_VARIANT_LISTS ||
                    ctx->variant[CRK_K_GRAVITY_ADJOINT] == CRK_VARIANT_LISTS))
            TRY(crk_build_lists(ctx, lv, false, false));
        tr.mark("gravity lists");
    }
#undef TRY
#undef ALLOC
#undef KCHECK
    *out = lv;
    return CRK_OK;
fail:
    if (!re) crk_leaves_free(ctx, lv);
    return rc;
}

int crk_build_leaves(crk_ctx *ctx, const crk_particles *p, const float *h, const crk_leaf_params *lp,
                     crk_leaves **out) {
    if (!ctx) return CRK_EINVAL;
    if (!p) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (p->n < 0) return crk_fail(ctx, CRK_EINVAL, "particle count out of range");
    std::vector<int64_t> bs = {0, p->n};
    std::vector<float> side = {p->box};
    return build_leaves_impl(ctx, p, h, lp, bs, side, out);
}

int crk_build_leaves_batch(crk_ctx *ctx, const crk_batch *bt, const float *h, const crk_leaf_params *lp,
                           crk_leaves **out) {
    if (!ctx) return CRK_EINVAL;
    if (!bt || !bt->box_start || !bt->box_side || bt->nbox < 1) return crk_fail(ctx, CRK_EINVAL, "bad batch");
    std::vector<int64_t> bs(bt->box_start, bt->box_start + bt->nbox + 1);
    std::vector<float> side(bt->box_side, bt->box_side + bt->nbox);
    crk_particles p{bt->x, bt->y, bt->z, bt->species, bt->n, 0.0f};
    for (float s : side) p.box = std::max(p.box, s);
    return build_leaves_impl(ctx, &p, h, lp, bs, side, out);
}

int crk_leaves_rebuild(crk_ctx *ctx, crk_leaves *lv, const crk_particles *p, const float *h) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !p) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->nbox != 1) return crk_fail(ctx, CRK_ESTATE, "rebuild: the leaves hold several boxes");
    std::vector<int64_t> bs = {0, p->n};
    std::vector<float> side = {p->box};
    crk_leaf_params lp{lv->mode, lv->cells, lv->max_leaf, lv->r_cut_grav};
    crk_leaves *out = lv;
    return build_leaves_impl(ctx, p, h, &lp, bs, side, &out, lv);
}

int crk_leaves_rebuild_batch(crk_ctx *ctx, crk_leaves *lv, const crk_batch *bt, const float *h) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !bt || !bt->box_start || !bt->box_side || bt->nbox < 1) return crk_fail(ctx, CRK_EINVAL, "bad batch");
    std::vector<int64_t> bs(bt->box_start, bt->box_start + bt->nbox + 1);
    std::vector<float> side(bt->box_side, bt->box_side + bt->nbox);
    crk_particles p{bt->x, bt->y, bt->z, bt->species, bt->n, 0.0f};
    for (float s : side) p.box = std::max(p.box, s);
    crk_leaf_params lp{lv->mode, lv->cells, lv->max_leaf, lv->r_cut_grav};
    crk_leaves *out = lv;
    return build_leaves_impl(ctx, &p, h, &lp, bs, side, &out, lv);
}

int crk_leaves_status(crk_ctx *ctx, crk_leaves *lv, int32_t *status) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !status) return crk_fail(ctx, CRK_EINVAL, "null argument");
    *status = 0;
    if (!lv->dev) return CRK_OK;  // an empty box
    int32_t head[4];
    unsigned long long cur[6];
    CRK_CUDA(ctx, cudaMemcpyAsync(head, lv->dev, sizeof(head), cudaMemcpyDeviceToHost, ctx->stream));
    CRK_CUDA(ctx, cudaMemcpyAsync(cur, lv->dev + 16, sizeof(cur), cudaMemcpyDeviceToHost, ctx->stream));
    CRK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *status = head[0];
    lv->n_gimg = (int64_t)cur[0];
    lv->n_gpairs = (int64_t)cur[1];
    lv->n_himg = (int64_t)cur[2];
    lv->n_hpairs = (int64_t)cur[3];
    return CRK_OK;
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
    const int64_t n = lv->n, nl = lv->n_leaves;
    if (perm && n) CRK_CUDA(ctx, cudaMemcpy(perm, lv->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (leaf_start) CRK_CUDA(ctx, cudaMemcpy(leaf_start, lv->leaf_start, sizeof(int32_t) * (nl + 1), cudaMemcpyDeviceToHost));
    struct {
        int32_t *ptr, *list;
        const int32_t *start, *cnt, *data;
        int64_t total;
    } L[2] = {{grav_ptr, grav_list, lv->gpair_start, lv->gpair_cnt, lv->gpair_list, lv->n_gpairs},
              {hydro_ptr, hydro_list, lv->hpair_start, lv->hpair_cnt, lv->hpair_list, lv->n_hpairs}};
    for (auto &l : L) {
        if (!l.ptr && !l.list) continue;
        std::vector<int32_t> st(nl), ct(nl), data(l.total);
        if (nl) {
            CRK_CUDA(ctx, cudaMemcpy(st.data(), l.start, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost));
            CRK_CUDA(ctx, cudaMemcpy(ct.data(), l.cnt, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost));
        }
        if (l.total) CRK_CUDA(ctx, cudaMemcpy(data.data(), l.data, sizeof(int32_t) * l.total, cudaMemcpyDeviceToHost));
        int64_t k = 0;
        for (int64_t a = 0; a < nl; ++a) {
            if (l.ptr) l.ptr[a] = (int32_t)k;
            for (int32_t q = 0; q < ct[a]; ++q, ++k)
                if (l.list) l.list[k] = data[st[a] + q];
        }
        if (l.ptr) l.ptr[nl] = (int32_t)k;
    }
    return CRK_OK;
}

void crk_leaves_free(crk_ctx *ctx, crk_leaves *lv) {
    if (!lv) return;
    for (auto &b : lv->allocs) {
        if (ctx && ctx->block_cache.size() < 256) ctx->block_cache.push_back(b);
        else cudaFree(b.first);
    }
    delete lv;
}
