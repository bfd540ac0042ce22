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
// Autotuner: time every variant of every kernel on these leaves (CUDA events
// on the context stream, best of `reps` after one warm-up) and keep the
// fastest.  Variants that need neighbour lists the leaves do not hold are
// skipped.  ms_out (host, 6 x CRK_N_VARIANTS, may be NULL) receives the timings (-1 when
// skipped), best_out (host, 6, may be NULL) the chosen variants.
int crk_tune(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
             const crk_step_io *io, int reps, float *ms_out, int *best_out) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !gp || !hp || !io) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (reps < 1) reps = 1;
    const int nvar = CRK_N_VARIANTS;
    int keep[6];
    for (int k = 0; k < 6; ++k) keep[k] = ctx->variant[k];
    // inputs of the later kernels come from one full step
    int rc = crk_step(ctx, lv, gp, hp, io);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CRK_CUDA(ctx, cudaEventCreate(&e0));
    CRK_CUDA(ctx, cudaEventCreate(&e1));
    if (!io->V || !io->rho || !io->A || !io->B || !io->gradA || !io->gradB || !io->dvdt3 || !io->dudt || !io->a3 ||
        !io->gx3_grav || !io->gm_grav || !io->gx3_geom || !io->gm_geom)
        return crk_fail(ctx, CRK_EINVAL, "crk_tune needs every output array of the step");
    // timing only: any arrays of the right size serve as cotangents
    const float *abar = io->abar3 ? io->abar3 : io->a3;
    const float *rhob = io->rhobar ? io->rhobar : io->rho;
    for (int k = 0; k < 6; ++k) {
        float best = 1e30f;
        int bv = keep[k];
        const bool gas = k != CRK_K_GRAVITY && k != CRK_K_GRAVITY_ADJOINT;
        const bool have_lists = gas ? lv->gas_lists.list != nullptr : lv->grav_lists.list != nullptr;
        for (int v = 0; v < nvar; ++v) {
            if (ms_out) ms_out[k * nvar + v] = -1.0f;
            if (v == CRK_VARIANT_LISTS && !have_lists) continue;
            if (v >= CRK_VARIANT_HALFWARP_SHFL && gas) continue;  // half-warp arms: gravity kernels only
            ctx->variant[k] = v;
            float tmin = 1e30f;
            for (int r = 0; r <= reps; ++r) {
                cudaEventRecord(e0, ctx->stream);
                switch (k) {
                    case CRK_K_GEOMETRY: rc = crk_geometry(ctx, lv, io->m, io->V, io->rho, nullptr); break;
                    case CRK_K_CORRECTIONS:
                        rc = crk_corrections(ctx, lv, io->V, io->A, io->B, io->gradA, io->gradB, nullptr);
                        break;
                    case CRK_K_HYDRO:
                        rc = crk_hydro(ctx, lv, hp, io->m, io->v3, io->u, io->V, io->rho, io->A, io->B, io->gradA,
                                       io->gradB, io->dvdt3, io->dudt, io->conservation, nullptr);
                        break;
                    case CRK_K_GRAVITY: rc = grav_short(ctx, lv, gp, io->m, io->a3, nullptr); break;
                    case CRK_K_GRAVITY_ADJOINT:
                        rc = grav_short_adjoint(ctx, lv, gp, io->m, abar, io->gx3_grav, io->gm_grav);
                        break;
                    default:
                        rc = crk_geometry_adjoint(ctx, lv, io->m, io->V, rhob, io->Vbar, io->gx3_geom, io->gm_geom);
                        break;
                }
                if (rc) break;
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0 && ms < tmin) tmin = ms;  // r = 0 is the warm-up
            }
            if (rc) break;
            if (ms_out) ms_out[k * nvar + v] = tmin;
            if (tmin < best) {
                best = tmin;
                bv = v;
            }
        }
        if (rc) break;
        ctx->variant[k] = bv;
        if (best_out) best_out[k] = bv;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        for (int k = 0; k < 6; ++k) ctx->variant[k] = keep[k];
        return rc;
    }
    return CRK_OK;
}
