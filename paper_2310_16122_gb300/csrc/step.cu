// One whole step of the pair path on a set of leaves (geometry, corrections,
// hydro, gravity, gravity adjoint, geometry adjoint), its CUDA-graph capture
// and replay, and the kernel-variant autotuner.
#include <cstdio>
#include <vector>

#include "crk_internal.cuh"

struct crk_graph {
    crk_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void crk_step_mark(crk_ctx *ctx, int k) {
    if (ctx->prof_max <= 0 || ctx->prof_used >= ctx->prof_max) return;
    cudaEventRecord(ctx->prof_ev[8 * (size_t)ctx->prof_used + k], ctx->stream);
}

int crk_step(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
             const crk_step_io *io) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !gp || !hp || !io) return crk_fail(ctx, CRK_EINVAL, "null argument");
    int rc = crk_step_fused(ctx, lv, gp, hp, io);
    if (rc == CRK_OK && lv->n > 0 && ctx->prof_max > 0 && ctx->prof_used < ctx->prof_max) ++ctx->prof_used;
    return rc;
}

int crk_step_profile(crk_ctx *ctx, int max_steps) {
    if (!ctx || max_steps < 0) return CRK_EINVAL;
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    ctx->prof_max = 0;
    ctx->prof_used = 0;
    for (int k = 0; k < 8 * max_steps; ++k) {
        cudaEvent_t e;
        CRK_CUDA(ctx, cudaEventCreate(&e));
        ctx->prof_ev.push_back(e);
    }
    ctx->prof_max = max_steps;
    return CRK_OK;
}

int crk_step_profile_read(crk_ctx *ctx, float ms[7], int *steps) {
    if (!ctx || !ms || !steps) return CRK_EINVAL;
    for (int k = 0; k < 7; ++k) ms[k] = 0.0f;
    *steps = ctx->prof_used;
    if (ctx->prof_used == 0) return CRK_OK;
    CRK_CUDA(ctx, cudaEventSynchronize(ctx->prof_ev[8 * (size_t)ctx->prof_used - 1]));
    for (int s = 0; s < ctx->prof_used; ++s)
        for (int k = 0; k < 7; ++k) {
            float t = 0.0f;
            CRK_CUDA(ctx, cudaEventElapsedTime(&t, ctx->prof_ev[8 * (size_t)s + k], ctx->prof_ev[8 * (size_t)s + k + 1]));
            ms[k] += t / ctx->prof_used;
        }
    ctx->prof_used = 0;
    return CRK_OK;
}

int crk_step_graph_create(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
                          const crk_step_io *io, crk_graph **out) {
    if (!ctx) return CRK_EINVAL;
    if (!out) return crk_fail(ctx, CRK_EINVAL, "null argument");
    *out = nullptr;
    if (!ctx->stream) return crk_fail(ctx, CRK_EINVAL, "graph capture needs a non-default context stream");
    // one uncaptured step sizes every scratch buffer, so the captured step allocates nothing
    int rc = crk_step(ctx, lv, gp, hp, io);
    if (rc) return rc;
    CRK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    crk_graph *g = new crk_graph();
    g->ctx = ctx;
    const int prof = ctx->prof_max;  // no profiling events inside the graph
    ctx->prof_max = 0;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        return crk_check_cuda(ctx, e, "begin capture");
    }
    rc = crk_step(ctx, lv, gp, hp, io);
    e = cudaStreamEndCapture(ctx->stream, &g->graph);
    ctx->prof_max = prof;
    if (rc || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        cudaGetLastError();
        return rc ? rc : crk_check_cuda(ctx, e, "end capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return crk_check_cuda(ctx, e, "graph instantiate");
    }
    *out = g;
    return CRK_OK;
}

// The batched driver's graph: the capture-safe leaf rebuild followed by the whole step.
int crk_rebuild_step_graph_create(crk_ctx *ctx, crk_leaves *lv, const crk_batch *bt, const float *h,
                                  const crk_grav_params *gp, const crk_hydro_params *hp, const crk_step_io *io,
                                  crk_graph **out) {
    if (!ctx) return CRK_EINVAL;
    if (!out || !lv || !bt || !gp || !hp || !io) return crk_fail(ctx, CRK_EINVAL, "null argument");
    *out = nullptr;
    if (!ctx->stream) return crk_fail(ctx, CRK_EINVAL, "graph capture needs a non-default context stream");
    // one uncaptured rebuild and step size every scratch buffer, so the captured ones allocate nothing
    int rc = crk_leaves_rebuild_batch(ctx, lv, bt, h);
    if (rc) return rc;
    if ((rc = crk_step(ctx, lv, gp, hp, io))) return rc;
    int32_t status = 0;
    if ((rc = crk_leaves_status(ctx, lv, &status))) return rc;
    if (status) return crk_fail(ctx, CRK_ESTATE, "rebuild status 0x%x: the leaves need a fresh build", status);
    crk_graph *g = new crk_graph();
    g->ctx = ctx;
    const int prof = ctx->prof_max;  // no profiling events inside the graph
    ctx->prof_max = 0;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        ctx->prof_max = prof;
        delete g;
        return crk_check_cuda(ctx, e, "begin capture");
    }
    rc = crk_leaves_rebuild_batch(ctx, lv, bt, h);
    if (!rc) rc = crk_step(ctx, lv, gp, hp, io);
    e = cudaStreamEndCapture(ctx->stream, &g->graph);
    ctx->prof_max = prof;
    if (rc || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        cudaGetLastError();
        return rc ? rc : crk_check_cuda(ctx, e, "end capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return crk_check_cuda(ctx, e, "graph instantiate");
    }
    *out = g;
    return CRK_OK;
}

int crk_graph_launch(crk_graph *g) {
    if (!g || !g->exec) return CRK_EINVAL;
    cudaError_t e = cudaGraphLaunch(g->exec, g->ctx->stream);
    return e == cudaSuccess ? CRK_OK : crk_check_cuda(g->ctx, e, "graph launch");
}

void crk_graph_destroy(crk_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

// ---------------------------------------------------------------------------
// Autotuner (Sec. 5.2 tunes register use and sub-group size per kernel and
// device; here: the sweep variant, the launch mode and the j-tile depth).
// Every kernel is timed on these leaves with CUDA events on the context stream
// (best of `reps` after one warm-up).  Coordinate descent: first the variant
// (non-persistent, depth 32), then the launch mode of the fastest variant,
// then (gravity kernels on tiles) the depth.  Variants that need neighbour
// lists the leaves do not hold, and variants a kernel does not implement (it
// would run another one), are skipped.  ms_out / best_out: see crk.h.
namespace {
// variants each kernel implements (the others fall back to tiles)
bool tune_variant_available(int k, int v, bool have_lists) {
    if (v == CRK_VARIANT_LISTS) return have_lists;
    if (v == CRK_VARIANT_TILES) return true;
    if (v == CRK_VARIANT_SPLIT8) return k == CRK_K_GRAVITY || k == CRK_K_GRAVITY_ADJOINT;
    const bool halfwarp = k == CRK_K_GRAVITY || k == CRK_K_GRAVITY_ADJOINT || k == CRK_K_HYDRO || k == CRK_K_ACCEL ||
                          k == CRK_K_ENERGY;
    if (v >= CRK_VARIANT_HALFWARP_SHFL && v <= CRK_VARIANT_HALFWARP_LOAD) return halfwarp;
    if (k == CRK_K_ACCEL || k == CRK_K_ENERGY) return false;        // lists, tiles and half-warp only
    if (v == CRK_VARIANT_RING16 && k == CRK_K_HYDRO) return false;  // hydro has no ring arm
    return true;
}
}  // namespace

int crk_tune(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
             const crk_step_io *io, int reps, float *ms_out, int *best_out) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !gp || !hp || !io) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (reps < 1) reps = 1;
    if (!io->V || !io->rho || !io->A || !io->B || !io->gradA || !io->gradB || !io->dvdt3 || !io->dudt || !io->a3 ||
        !io->gx3_grav || !io->gm_grav || !io->gx3_geom || !io->gm_geom)
        return crk_fail(ctx, CRK_EINVAL, "crk_tune needs every output array of the step");
    if (io->extras && (!io->rho_r || !io->dvdx)) return crk_fail(ctx, CRK_EINVAL, "extras needs rho_r and dvdx");
    const int nvar = CRK_N_VARIANTS, cols = CRK_TUNE_COLS;
    int keep_v[CRK_N_KERNELS], keep_p[CRK_N_KERNELS], keep_d[CRK_N_KERNELS], keep_w[CRK_N_KERNELS];
    for (int k = 0; k < CRK_N_KERNELS; ++k) {
        keep_v[k] = ctx->variant[k];
        keep_p[k] = ctx->persist[k];
        keep_d[k] = ctx->depth[k];
        keep_w[k] = ctx->warps[k];
    }
    if (ms_out)
        for (int q = 0; q < CRK_N_KERNELS * cols; ++q) ms_out[q] = -1.0f;
    // inputs of the later kernels come from one full step
    int rc = crk_step(ctx, lv, gp, hp, io);
    if (rc) return rc;
    uint32_t *vsig = (uint32_t *)crk_scratch(ctx, 36, 64);
    if (!vsig) return crk_fail(ctx, CRK_ENOMEM, "tune scratch");
    cudaEvent_t e0, e1;
    CRK_CUDA(ctx, cudaEventCreate(&e0));
    CRK_CUDA(ctx, cudaEventCreate(&e1));
    // timing only: any arrays of the right size serve as cotangents
    const float *abar = io->abar3 ? io->abar3 : io->a3;
    const float *rhob = io->rhobar ? io->rhobar : io->rho;
    const float *dvdx = io->extras ? io->dvdx : nullptr;
    auto run = [&](int k) -> int {
        switch (k) {
            case CRK_K_GEOMETRY: return crk_geometry(ctx, lv, io->m, io->V, io->rho, nullptr);
            case CRK_K_CORRECTIONS: return crk_corrections(ctx, lv, io->V, io->A, io->B, io->gradA, io->gradB, nullptr);
            case CRK_K_HYDRO:
                return crk_hydro(ctx, lv, hp, io->m, io->v3, io->u, io->V, io->rho, io->A, io->B, io->gradA,
                                 io->gradB, io->dvdt3, io->dudt, io->conservation, nullptr);
            case CRK_K_GRAVITY: return grav_short(ctx, lv, gp, io->m, io->a3, nullptr);
            case CRK_K_GRAVITY_ADJOINT: return grav_short_adjoint(ctx, lv, gp, io->m, abar, io->gx3_grav, io->gm_grav);
            case CRK_K_GEOMETRY_ADJOINT:
                return crk_geometry_adjoint(ctx, lv, io->m, io->V, rhob, io->Vbar, io->gx3_geom, io->gm_geom);
            case CRK_K_EXTRAS:
                return crk_extras(ctx, lv, io->m, io->v3, io->V, io->A, io->B, io->gradA, io->gradB, io->rho_r,
                                  io->dvdx, nullptr);
            case CRK_K_ACCEL:
                return crk_hydro_accel(ctx, lv, hp, io->m, io->v3, io->u, io->V, io->rho, io->A, io->B, io->gradA,
                                       io->gradB, dvdx, 3.0f, io->dvdt3, vsig, io->conservation, nullptr);
            default:
                return crk_hydro_energy(ctx, lv, hp, io->m, io->v3, io->u, io->V, io->rho, io->A, io->B, io->gradA,
                                        io->gradB, dvdx, io->v3, io->dudt, io->conservation, nullptr);
        }
    };
    // best of reps after a warm-up; sets rc on failure.  A candidate whose warm-up already takes
    // more than three times the best time so far is not timed further (its warm-up time is kept).
    auto timed = [&](int k, float best_so_far) -> float {
        float tmin = 1e30f;
        for (int r = 0; r <= reps; ++r) {
            cudaEventRecord(e0, ctx->stream);
            if ((rc = run(k)) != CRK_OK) return -1.0f;
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r == 0 && ms > 3.0f * best_so_far) return ms;
            if (r > 0 && ms < tmin) tmin = ms;  // r = 0 is the warm-up
        }
        return tmin;
    };
    for (int k = 0; k < CRK_N_KERNELS && rc == CRK_OK; ++k) {
        int bv = keep_v[k], bp = keep_p[k], bd = keep_d[k], bw = keep_w[k];
        if (k == CRK_K_EXTRAS && !io->extras) {
            if (best_out) {
                best_out[4 * k] = bv; best_out[4 * k + 1] = bp; best_out[4 * k + 2] = bd; best_out[4 * k + 3] = bw;
            }
            continue;
        }
        const bool gas = k != CRK_K_GRAVITY && k != CRK_K_GRAVITY_ADJOINT;
        const bool have_lists = gas ? lv->gas_lists.list != nullptr : lv->grav_lists.list != nullptr;
        float *row = ms_out ? ms_out + (size_t)k * cols : nullptr;
        // 1. the variant
        float best = 1e30f;
        ctx->persist[k] = 0;
        ctx->depth[k] = 32;
        ctx->warps[k] = 4;
        for (int v = 0; v < nvar && rc == CRK_OK; ++v) {
            if (!tune_variant_available(k, v, have_lists)) continue;
            ctx->variant[k] = v;
            const float t = timed(k, best);
            if (rc) break;
            if (row) row[v] = t;
            if (t < best) { best = t; bv = v; }
        }
        if (rc) break;
        ctx->variant[k] = bv;
        // 2. the launch mode of that variant
        best = 1e30f;
        for (int pm = 0; pm < 2 && rc == CRK_OK; ++pm) {
            ctx->persist[k] = pm;
            const float t = timed(k, best);
            if (rc) break;
            if (row) row[nvar + pm] = t;
            if (t < best) { best = t; bp = pm; }
        }
        if (rc) break;
        ctx->persist[k] = bp;
        // 3. the j-tile depth of the packed gravity sweeps
        bd = 32;
        if ((k == CRK_K_GRAVITY || k == CRK_K_GRAVITY_ADJOINT) && bv == CRK_VARIANT_TILES) {
            best = 1e30f;
            for (int q = 0; q < 3 && rc == CRK_OK; ++q) {
                ctx->depth[k] = 32 * (q + 1);
                const float t = timed(k, best);
                if (rc) break;
                if (row) row[nvar + 2 + q] = t;
                if (t < best) { best = t; bd = 32 * (q + 1); }
            }
            if (rc) break;
        }
        ctx->depth[k] = bd;
        // 4. the warps per leaf of the packed gravity tiles
        bw = 4;
        if ((k == CRK_K_GRAVITY || k == CRK_K_GRAVITY_ADJOINT) && bv == CRK_VARIANT_TILES) {
            best = 1e30f;
            for (int q = 0; q < 2 && rc == CRK_OK; ++q) {
                ctx->warps[k] = q ? 2 : 4;
                const float t = timed(k, best);
                if (rc) break;
                if (row) row[nvar + 5 + q] = t;
                if (t < best) { best = t; bw = q ? 2 : 4; }
            }
            if (rc) break;
        }
        ctx->warps[k] = bw;
        if (best_out) {
            best_out[4 * k] = bv; best_out[4 * k + 1] = bp; best_out[4 * k + 2] = bd; best_out[4 * k + 3] = bw;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        for (int k = 0; k < CRK_N_KERNELS; ++k) {
            ctx->variant[k] = keep_v[k];
            ctx->persist[k] = keep_p[k];
            ctx->depth[k] = keep_d[k];
            ctx->warps[k] = keep_w[k];
        }
        return rc;
    }
    return CRK_OK;
}
