// Context, errors and device memory of libcrk.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>

#include "crk_internal.cuh"

int crk_fail(crk_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int crk_check_cuda(crk_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return CRK_OK;
    if (e == cudaErrorMemoryAllocation) return crk_fail(ctx, CRK_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return crk_fail(ctx, CRK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Growable per-slot scratch.  Growing frees the old buffer: cudaFree waits for
// the device, so work still using it on the context stream has finished.
void *crk_scratch(crk_ctx *ctx, int slot, size_t bytes) {
    if (slot < 0 || slot >= crk_ctx::kSlots) return nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->slot_bytes[slot] >= bytes) return ctx->slot[slot];
    if (ctx->slot[slot]) cudaFree(ctx->slot[slot]);
    ctx->slot[slot] = nullptr;
    ctx->slot_bytes[slot] = 0;
    size_t want = bytes + bytes / 8;  // headroom for slowly growing inputs
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        want = bytes;
    }
    ctx->slot[slot] = p;
    ctx->slot_bytes[slot] = want;
    return p;
}

void *crk_leaves_alloc(crk_ctx *ctx, crk_leaves *lv, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    // best fit among cached blocks no more than twice as large
    int best = -1;
    for (size_t k = 0; k < ctx->block_cache.size(); ++k) {
        size_t sz = ctx->block_cache[k].second;
        if (sz >= bytes && sz <= 2 * bytes + (1 << 16) && (best < 0 || sz < ctx->block_cache[best].second))
            best = (int)k;
    }
    if (best >= 0) {
        auto blk = ctx->block_cache[best];
        ctx->block_cache.erase(ctx->block_cache.begin() + best);
        lv->allocs.push_back(blk);
        return blk.first;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        // drop the cache and retry once
        for (auto &b : ctx->block_cache) cudaFree(b.first);
        ctx->block_cache.clear();
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    }
    lv->allocs.push_back({p, bytes});
    return p;
}

extern "C" {

int crk_create(crk_ctx **out, int device, void *cuda_stream) {
    if (!out) return CRK_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CRK_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return CRK_ECUDA;
    crk_ctx *ctx = new crk_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    const char *tr = getenv("CRK_TRACE");
    ctx->trace = tr && tr[0] && tr[0] != '0';
    // gravity: the tiles beat the lists on GB300 (the lists make the gravity
    // pair loop gather-bound and cost a build pass of their own)
    ctx->variant[CRK_K_GRAVITY] = CRK_VARIANT_TILES;
    ctx->variant[CRK_K_GRAVITY_ADJOINT] = CRK_VARIANT_TILES;

    *out = ctx;
    return CRK_OK;
}

void crk_destroy(crk_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (int s = 0; s < crk_ctx::kSlots; ++s)
        if (ctx->slot[s]) cudaFree(ctx->slot[s]);
    for (auto &b : ctx->block_cache) cudaFree(b.first);
    crk_rcb_shape_free(ctx);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    delete ctx;
}

int crk_set_stream(crk_ctx *ctx, void *cuda_stream) {
    if (!ctx) return CRK_EINVAL;
    ctx->stream = (cudaStream_t)cuda_stream;
    return CRK_OK;
}

const char *crk_last_error(const crk_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char *crk_version(void) { return "libcrk 1 sm_103a"; }

int crk_set_variant(crk_ctx *ctx, int kernel, int variant) {
    if (!ctx) return CRK_EINVAL;
    if (kernel < 0 || kernel >= CRK_N_KERNELS) return crk_fail(ctx, CRK_EINVAL, "unknown kernel %d", kernel);
    if (variant < CRK_VARIANT_LISTS || variant >= CRK_N_VARIANTS)
        return crk_fail(ctx, CRK_EINVAL, "variant %d not available for kernel %d", variant, kernel);
    ctx->variant[kernel] = variant;
    return CRK_OK;
}

int crk_get_variant(const crk_ctx *ctx, int kernel, int *variant) {
    if (!ctx || !variant || kernel < 0 || kernel >= CRK_N_KERNELS) return CRK_EINVAL;
    *variant = ctx->variant[kernel];
    return CRK_OK;
}

int crk_set_persistent(crk_ctx *ctx, int on) {
    if (!ctx) return CRK_EINVAL;
    for (int k = 0; k < CRK_N_KERNELS; ++k) ctx->persist[k] = on != 0;
    return CRK_OK;
}

int crk_set_launch(crk_ctx *ctx, int kernel, int persistent, int depth, int warps) {
    if (!ctx) return CRK_EINVAL;
    if (kernel < 0 || kernel >= CRK_N_KERNELS) return crk_fail(ctx, CRK_EINVAL, "unknown kernel %d", kernel);
    if (depth != 32 && depth != 64 && depth != 96) return crk_fail(ctx, CRK_EINVAL, "depth must be 32, 64 or 96");
    if (warps != 2 && warps != 4) return crk_fail(ctx, CRK_EINVAL, "warps per leaf must be 2 or 4");
    ctx->persist[kernel] = persistent != 0;
    ctx->depth[kernel] = depth;
    ctx->warps[kernel] = warps;
    return CRK_OK;
}

int crk_get_launch(const crk_ctx *ctx, int kernel, int *persistent, int *depth, int *warps) {
    if (!ctx || kernel < 0 || kernel >= CRK_N_KERNELS) return CRK_EINVAL;
    if (persistent) *persistent = ctx->persist[kernel];
    if (depth) *depth = ctx->depth[kernel];
    if (warps) *warps = ctx->warps[kernel];
    return CRK_OK;
}

int crk_set_trace(crk_ctx *ctx, int on) {
    if (!ctx) return CRK_EINVAL;
    ctx->trace = on != 0;
    return CRK_OK;
}

int crk_launch_count(const crk_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return CRK_EINVAL;
    *out = ctx->launches;
    return CRK_OK;
}

}  // extern "C"
