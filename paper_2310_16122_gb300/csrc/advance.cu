// The time step around the pair kernels: the Courant timestep from the
// signal-velocity atomic max (Sec. 5.1), and a two-stage kick-drift step that
// calls Acceleration and Energy twice (Sec. 5.4) with the compatible energy
// update.  The elementwise kernels read dt from device memory, so a step
// issues no host round trip beyond the two leaf builds.
#include "crk_internal.cuh"

namespace {

// x + d wrapped into [0, L) (|d| < L); a value that rounds onto L maps to 0
__device__ __forceinline__ float wrap_add(float x, float d, float L) {
    float y = x + d;
    if (y >= L) y -= L;
    else if (y < 0.0f) y += L;
    return (y >= 0.0f && y < L) ? y : 0.0f;
}

__global__ void timestep_kernel(const uint32_t *__restrict__ vsig_h_max, float cfl, float dt_max, float dt_fixed,
                                float *__restrict__ dt) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float d = dt_max;
    if (dt_fixed > 0.0f) {
        d = dt_fixed;
    } else if (vsig_h_max) {
        const float q = __uint_as_float(*vsig_h_max);  // max_i vsig_i / h_i
        if (q > 0.0f) d = fminf(dt_max, cfl / q);
    }
    *dt = d;
}

// The accelerations and du come from the stage in the library's kernel orders:
// hydro dv and du in the gas order (position kinv[o] for particle o), gravity
// in the gravity order (kinv_g[o]).
struct StageOut {
    const float *dv, *ag, *du;
    const int32_t *kinv, *kinv_g;
    int64_t n;
    __device__ float acc(int c, int64_t o) const {
        float a = dv[c * n + kinv[o]];
        if (ag) a += ag[c * n + kinv_g[o]];
        return a;
    }
    __device__ float dudt(int64_t o) const { return du[kinv[o]]; }
};

// predictor: v_p = v + dt/2 a, u_p = u + dt/2 du, x_p = x + dt/2 v_p (a = hydro + gravity)
__global__ void predict_kernel(int64_t n, float L, const float *__restrict__ dtp, const float *__restrict__ x,
                               const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ v3,
                               const float *__restrict__ u, StageOut so, float *__restrict__ xp,
                               float *__restrict__ yp, float *__restrict__ zp, float *__restrict__ vp3,
                               float *__restrict__ up) {
    const float h = 0.5f * *dtp;
    const float *pos[3] = {x, y, z};
    float *posp[3] = {xp, yp, zp};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = fmaf(h, so.acc(c, i), v3[c * n + i]);
            vp3[c * n + i] = v;
            posp[c][i] = wrap_add(pos[c][i], h * v, L);
        }
        up[i] = fmaf(h, so.dudt(i), u[i]);
    }
}

// kick: v1 = v + dt a_p (in place), v* = (v + v1)/2
__global__ void kick_kernel(int64_t n, const float *__restrict__ dtp, float *__restrict__ v3, StageOut so,
                            float *__restrict__ vs3) {
    const float dt = *dtp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v0 = v3[c * n + i];
            const float v1 = fmaf(dt, so.acc(c, i), v0);
            v3[c * n + i] = v1;
            vs3[c * n + i] = 0.5f * (v0 + v1);
        }
    }
}

// final update: u1 = u + dt du, x1 = x + dt v* (wrapped)
__global__ void drift_kernel(int64_t n, float L, const float *__restrict__ dtp, float *__restrict__ x,
                             float *__restrict__ y, float *__restrict__ z, const float *__restrict__ vs3,
                             float *__restrict__ u, StageOut so) {
    const float dt = *dtp;
    float *pos[3] = {x, y, z};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) pos[c][i] = wrap_add(pos[c][i], dt * vs3[c * n + i], L);
        u[i] = fmaf(dt, so.dudt(i), u[i]);
    }
}

// n_singular of the step: both stages' counts
__global__ void sum_counts_kernel(const int32_t *__restrict__ c, int32_t *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = c[0] + c[1];
}

int elementwise_grid(const crk_ctx *ctx, int64_t n) {
    const int g = crk_grid(n, 256);
    const int cap = ctx->num_sms > 0 ? 8 * ctx->num_sms : 1216;  // 8 resident blocks of 256 per SM
    return g < cap ? g : cap;
}

// the stage's kernel-order columns, then the caller-order predicted state and v*
enum Col : int {
    kXp = crk_stage_cols::count, kVp = kXp + 3, kUp = kVp + 3, kVs = kUp + 1, kCols = kVs + 3
};

StageOut stage_out(const crk_leaves *lv, const float *w, int gravity) {
    namespace K = crk_stage_cols;
    const int64_t n = lv->n;
    return StageOut{w + (size_t)K::dv * n, gravity ? w + (size_t)K::ag * n : nullptr, w + (size_t)K::du * n,
                    lv->kinv, lv->kinv_g, n};
}

}  // namespace

int crk_timestep(crk_ctx *ctx, const uint32_t *vsig_h_max, float cfl, float dt_max, float *dt) {
    if (!ctx) return CRK_EINVAL;
    if (!vsig_h_max || !dt) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (!(cfl > 0.0f) || !(dt_max > 0.0f)) return crk_fail(ctx, CRK_EINVAL, "cfl and dt_max must be > 0");
    timestep_kernel<<<1, 32, 0, ctx->stream>>>(vsig_h_max, cfl, dt_max, 0.0f, dt);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "timestep");
    return CRK_OK;
}

int crk_advance(crk_ctx *ctx, int64_t n, float box, float *x, float *y, float *z, const uint8_t *species,
                const float *h, const float *m, float *v3, float *u, const crk_leaf_params *lp,
                const crk_hydro_params *hp, const crk_grav_params *gp, const crk_advance_params *ap, float *dt,
                double *conservation, int32_t *n_singular) {
    if (!ctx) return CRK_EINVAL;
    if (!lp || !hp || !ap || !dt) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (n < 0) return crk_fail(ctx, CRK_EINVAL, "particle count out of range");
    if (n > 0 && (!x || !y || !z || !species || !h || !m || !v3 || !u)) return crk_fail(ctx, CRK_EINVAL, "null array");
    if (!(ap->cfl > 0.0f) || !(ap->dt_max > 0.0f) || !(ap->sig_beta >= 0.0f) || !(ap->dt_fixed >= 0.0f))
        return crk_fail(ctx, CRK_EINVAL, "bad step parameters");
    if (ap->gravity) {
        if (!gp) return crk_fail(ctx, CRK_EINVAL, "gravity needs its parameters");
        if (gp->r_cut != lp->r_cut_grav) return crk_fail(ctx, CRK_ESTATE, "r_cut differs from the leaves' r_cut_grav");
    }
    // the state columns and, past them, the signal-velocity max and the singular counts
    const size_t cols = (size_t)kCols * (size_t)(n > 0 ? n : 1);
    char *base = (char *)crk_scratch(ctx, 32, cols * sizeof(float) + 256);
    if (!base) return crk_fail(ctx, CRK_ENOMEM, "step state");
    float *col = (float *)base;
    uint32_t *vsig = (uint32_t *)(base + ((cols * sizeof(float) + 127) & ~(size_t)127));
    int32_t *nsing = (int32_t *)(vsig + 4);
    CRK_CUDA(ctx, cudaMemsetAsync(vsig, 0, 4 * sizeof(uint32_t) + 2 * sizeof(int32_t), ctx->stream));
    if (conservation) CRK_CUDA(ctx, cudaMemsetAsync(conservation, 0, 4 * sizeof(double), ctx->stream));
    if (n == 0) {
        if (n_singular) CRK_CUDA(ctx, cudaMemsetAsync(n_singular, 0, sizeof(int32_t), ctx->stream));
        timestep_kernel<<<1, 32, 0, ctx->stream>>>(nullptr, ap->cfl, ap->dt_max, ap->dt_fixed, dt);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "timestep");
        return CRK_OK;
    }
    const int grid = elementwise_grid(ctx, n);
    auto C = [&](int k) { return col + (size_t)k * n; };
    int rc;
    // ---- stage 1 at t^n: Acceleration (with the signal velocity) and Energy on v* = v
    crk_leaves *lv = nullptr;
    {
        crk_particles pt{x, y, z, species, n, box};
        if ((rc = crk_build_leaves(ctx, &pt, h, lp, &lv))) return rc;
        rc = crk_stage_forces(ctx, lv, gp, hp, ap->limited, ap->gravity, ap->sig_beta, m, v3, u, vsig, nsing, col);
        if (!rc) rc = crk_stage_energy(ctx, lv, hp, ap->limited, nullptr, col, nullptr);
        if (!rc) {
            timestep_kernel<<<1, 32, 0, ctx->stream>>>(vsig, ap->cfl, ap->dt_max, ap->dt_fixed, dt);
            predict_kernel<<<grid, 256, 0, ctx->stream>>>(n, box, dt, x, y, z, v3, u, stage_out(lv, col, ap->gravity),
                                                          C(kXp), C(kXp + 1), C(kXp + 2), C(kVp), C(kUp));
            ctx->launches += 2;
            rc = crk_check_cuda(ctx, cudaGetLastError(), "predictor");
        }
        crk_leaves_free(ctx, lv);
        if (rc) return rc;
    }
    // ---- stage 2 at the predicted state: Acceleration, kick, Energy on v* = (v + v1)/2, drift
    {
        crk_particles pt{C(kXp), C(kXp + 1), C(kXp + 2), species, n, box};
        if ((rc = crk_build_leaves(ctx, &pt, h, lp, &lv))) return rc;
        rc = crk_stage_forces(ctx, lv, gp, hp, ap->limited, ap->gravity, ap->sig_beta, m, C(kVp), C(kUp), nullptr,
                              nsing + 1, col);
        if (!rc) {
            kick_kernel<<<grid, 256, 0, ctx->stream>>>(n, dt, v3, stage_out(lv, col, ap->gravity), C(kVs));
            ++ctx->launches;
            rc = crk_check_cuda(ctx, cudaGetLastError(), "kick");
        }
        if (!rc) rc = crk_stage_energy(ctx, lv, hp, ap->limited, C(kVs), col, conservation);
        if (!rc) {
            drift_kernel<<<grid, 256, 0, ctx->stream>>>(n, box, dt, x, y, z, C(kVs), u, stage_out(lv, col, ap->gravity));
            ++ctx->launches;
            rc = crk_check_cuda(ctx, cudaGetLastError(), "drift");
        }
        crk_leaves_free(ctx, lv);
        if (rc) return rc;
    }
    if (n_singular) {
        sum_counts_kernel<<<1, 32, 0, ctx->stream>>>(nsing, n_singular);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "singular counts");
    }
    return CRK_OK;
}
