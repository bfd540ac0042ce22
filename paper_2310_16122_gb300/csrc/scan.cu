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
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 16;  // 4-bit digits

__global__ void radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ counts,
                                  int64_t nb) {
    __shared__ int32_t h[kRadix];
    if (threadIdx.x < kRadix) h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kRadix) counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// One LSD pass over a tile: stable tile-local ranks by digit (per-thread
// counts in digit-major, thread-minor order, scanned), the tile sorted by
// digit in shared memory, then written out in order so that each digit's run
// goes to consecutive global positions (coalesced stores).
__global__ void radix_scatter_kernel(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                     uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int shift,
                                     const int32_t *__restrict__ offsets, int64_t nb) {
    static_assert(kRadix * kSortThreads <= 2 * kSortTile, "counters fit the staging buffer");
    __shared__ int32_t sm[2 * kSortTile];  // first the counters, then the digit-sorted tile (keys, values)
    int32_t *cnt = sm;                     // digit-major, thread-minor
    __shared__ int32_t wt[32];
    __shared__ int32_t goff[kRadix];
    __shared__ int32_t dstart[kRadix];
    const int t = threadIdx.x;
    if (t < kRadix) goff[t] = offsets[(int64_t)t * nb + blockIdx.x];
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)t * kSortItems;  // blocked: thread-contiguous
    uint32_t key[kSortItems];
    int32_t val[kSortItems];
    int dig[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + k;
        bool ok = i < n;
        key[k] = ok ? kin[i] : 0u;
        val[k] = ok ? vin[i] : 0;
        dig[k] = ok ? (int)((key[k] >> shift) & (kRadix - 1)) : -1;
    }
#pragma unroll
    for (int d = 0; d < kRadix; ++d) {
        int c = 0;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) c += dig[k] == d;
        cnt[d * kSortThreads + t] = c;
    }
    __syncthreads();
    // exclusive scan of the kRadix*kSortThreads counters (each thread owns 16 consecutive ones)
    int32_t loc[kSortItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        loc[k] = cnt[t * kSortItems + k];
        s += loc[k];
    }
    int32_t tot;
    int32_t e = block_exclusive_scan(s, wt, tot);
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        cnt[t * kSortItems + k] = e;
        e += loc[k];
    }
    __syncthreads();
    // cnt now holds prefixes in digit-major order (they include the counts of all smaller
    // digits in this tile); dstart[d] is the tile-local start of digit d
    if (t < kRadix) dstart[t] = cnt[t * kSortThreads];
    __syncthreads();     // dstart read before thread 0 advances its counters
    int rr[kSortItems];  // tile-local sorted position of each item
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int d = dig[k];
        rr[k] = -1;
        if (d < 0) continue;
        rr[k] = cnt[d * kSortThreads + t];
        cnt[d * kSortThreads + t] = rr[k] + 1;  // only this thread touches its own counter
    }
    __syncthreads();  // counters read: the buffer now takes the sorted tile
    uint32_t *skey = reinterpret_cast<uint32_t *>(sm);
    int32_t *sval = sm + kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (rr[k] >= 0) {
            skey[rr[k]] = key[k];
            sval[rr[k]] = val[k];
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
    int passes = (key_bits + 3) / 4;
    uint32_t *k2 = (uint32_t *)crk_scratch(ctx, 13, sizeof(uint32_t) * (size_t)n);
    int32_t *v2 = (int32_t *)crk_scratch(ctx, 14, sizeof(int32_t) * (size_t)n);
    int32_t *counts = (int32_t *)crk_scratch(ctx, 12, sizeof(int32_t) * (size_t)(nb * kRadix));
    if (!k2 || !v2 || !counts) return crk_fail(ctx, CRK_ENOMEM, "radix sort scratch");
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes; ++p) {
        int shift = 4 * p;
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
