// Device-wide exclusive scan and stable LSD radix sort used by the leaf build.
#include "crk_internal.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one int32 per thread; returns the block total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_tot, int32_t &total) {
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
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    int32_t base = warp > 0 ? warp_tot[warp - 1] : 0;
    int32_t r = base + x - v;
    __syncthreads();
    return r;
}

__global__ void scan_reduce_kernel(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ sums) {
    __shared__ int32_t wt[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    int32_t tot;
    block_exclusive_scan(s, wt, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block: exclusive scan of nb block sums in place; writes the grand total
__global__ void scan_sums_kernel(int32_t *sums, int64_t nb, int32_t *total) {
    __shared__ int32_t wt[32];
    int32_t carry = 0;
    for (int64_t s0 = 0; s0 < nb; s0 += blockDim.x) {
        int64_t i = s0 + threadIdx.x;
        int32_t v = i < nb ? sums[i] : 0;
        int32_t tot;
        int32_t e = block_exclusive_scan(v, wt, tot);
        if (i < nb) sums[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_tile_kernel(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                                 const int32_t *__restrict__ sums) {
    __shared__ int32_t wt[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;  // blocked
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t e = block_exclusive_scan(s, wt, tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = e;
        e += v[k];
    }
}

// ---------------------------------------------------------------- radix sort
// LSD radix sort with 8-bit digits: a histogram pass per tile, one exclusive
// scan of the digit-major counts, and a scatter pass that ranks each tile
// stably by digit and writes every digit's run to consecutive positions.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadix = 256;  // 8-bit digits
static_assert(kRadix == kSortThreads, "one digit per thread in the scatter's digit scan");

__device__ __forceinline__ unsigned lanemask_below() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// per tile: the count of each digit (lanes with equal digits add once per warp step)
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                                  int shift, int32_t *__restrict__ counts, int64_t nb) {
    __shared__ int32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        const int d = i < n ? (int)((keys[i] >> shift) & (kRadix - 1)) : kRadix;
        const unsigned peers = __match_any_sync(CRK_FULL_MASK, d);
        if (d < kRadix && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// One LSD pass over a tile.  Warp w takes the tile's items w*256 .. w*256 + 255
// in 8 coalesced steps of 32 (8 items per thread keep the kernel at 48
// registers, five blocks per SM; 16 items took 80 registers and 0.4 ms more
// per 33.5M-particle leaf build); the lanes of a step with equal digits are found
// by __match_any_sync, so each item's rank among the earlier items of its warp
// with the same digit is a running per-warp count plus its rank among its
// peers.  The per-warp counts then give each warp's offset inside the digit,
// a scan over the 256 digits gives each digit's start in the tile, the tile is
// sorted in shared memory, and every digit's run is written to consecutive
// global positions (coalesced stores).  Stable: the tile order is item order.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint32_t *__restrict__ kin,
                                                                     const int32_t *__restrict__ vin,
                                                                     uint32_t *__restrict__ kout,
                                                                     int32_t *__restrict__ vout, int64_t n, int shift,
                                                                     const int32_t *__restrict__ offsets, int64_t nb) {
    __shared__ int32_t whist[kSortWarps][kRadix];  // per-warp digit counts, then the warp's offset in the digit
    __shared__ int32_t dstart[kRadix];
    __shared__ int32_t goff[kRadix];
    __shared__ uint32_t skey[kSortTile];
    __shared__ int32_t sval[kSortTile];
    __shared__ int32_t wt[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    goff[t] = offsets[(int64_t)t * nb + blockIdx.x];
#pragma unroll
    for (int v = 0; v < kSortWarps; ++v) whist[v][t] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const unsigned below = lanemask_below();
    uint32_t key[kSortItems];
    int32_t val[kSortItems];
    int dig[kSortItems], rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = tile0 + (int64_t)w * (32 * kSortItems) + 32 * r + lane;
        const bool ok = i < n;
        key[r] = ok ? kin[i] : 0u;
        val[r] = ok ? vin[i] : 0;
        const int d = ok ? (int)((key[r] >> shift) & (kRadix - 1)) : kRadix;
        dig[r] = d;
        const unsigned peers = __match_any_sync(CRK_FULL_MASK, d);
        const int leader = __ffs(peers) - 1;
        int before = 0;
        if (lane == leader && d < kRadix) {
            before = whist[w][d];
            whist[w][d] = before + __popc(peers);
        }
        before = __shfl_sync(CRK_FULL_MASK, before, leader);
        rank[r] = before + __popc(peers & below);
        __syncwarp();
    }
    __syncthreads();
    // thread t = digit t: the warps' offsets inside the digit, then the digits' starts in the tile
    int32_t tot = 0;
#pragma unroll
    for (int v = 0; v < kSortWarps; ++v) {
        const int32_t c = whist[v][t];
        whist[v][t] = tot;
        tot += c;
    }
    int32_t all;
    dstart[t] = block_exclusive_scan(tot, wt, all);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int d = dig[r];
        if (d < kRadix) {
            const int pos = dstart[d] + whist[w][d] + rank[r];
            skey[pos] = key[r];
            sval[pos] = val[r];
        }
    }
    __syncthreads();
    const int m = (int)(n - tile0 < kSortTile ? n - tile0 : kSortTile);
    for (int i = t; i < m; i += kSortThreads) {
        const uint32_t kk = skey[i];
        const int d = (int)((kk >> shift) & (kRadix - 1));
        const int64_t pos = (int64_t)goff[d] + (i - dstart[d]);
        kout[pos] = kk;
        vout[pos] = sval[i];
    }
}

}  // namespace

int crk_exclusive_scan_i32(crk_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *total) {
    if (n <= 0) {
        if (total) CRK_CUDA(ctx, cudaMemsetAsync(total, 0, sizeof(int32_t), ctx->stream));
        return CRK_OK;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    int32_t *sums = (int32_t *)crk_scratch(ctx, 15, sizeof(int32_t) * (size_t)nb);
    if (!sums) return crk_fail(ctx, CRK_ENOMEM, "scan scratch");
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, n, sums);
    scan_sums_kernel<<<1, 1024, 0, ctx->stream>>>(sums, nb, total);
    scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, out, n, sums);
    ctx->launches += 3;
    CRK_LAUNCH_CHECK(ctx, "exclusive scan");
    return CRK_OK;
}

int crk_radix_sort_u32(crk_ctx *ctx, uint32_t *keys, int32_t *vals, int64_t n, int key_bits) {
    if (n <= 1) return CRK_OK;
    if (n > 2147483647LL) return crk_fail(ctx, CRK_EINVAL, "radix sort: n too large");
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    int passes = (key_bits + 7) / 8;
    uint32_t *k2 = (uint32_t *)crk_scratch(ctx, 13, sizeof(uint32_t) * (size_t)n);
    int32_t *v2 = (int32_t *)crk_scratch(ctx, 14, sizeof(int32_t) * (size_t)n);
    int32_t *counts = (int32_t *)crk_scratch(ctx, 12, sizeof(int32_t) * (size_t)(nb * kRadix));
    if (!k2 || !v2 || !counts) return crk_fail(ctx, CRK_ENOMEM, "radix sort scratch");
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        radix_hist_kernel<<<(unsigned)nb, kSortThreads, 0, ctx->stream>>>(ka, n, shift, counts, nb);
        CRK_LAUNCH_CHECK(ctx, "radix hist");
        int rc = crk_exclusive_scan_i32(ctx, counts, counts, nb * kRadix, nullptr);
        if (rc) return rc;
        radix_scatter_kernel<<<(unsigned)nb, kSortThreads, 0, ctx->stream>>>(ka, va, kb, vb, n, shift, counts, nb);
        ctx->launches += 2;
        CRK_LAUNCH_CHECK(ctx, "radix scatter");
        uint32_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        CRK_CUDA(ctx, cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
        CRK_CUDA(ctx, cudaMemcpyAsync(vals, va, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return CRK_OK;
}
