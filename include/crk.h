/*
 * crk.h -- C ABI of libcrk, the GB300 (sm_103a) library of CRK-HACC's
 * short-range particle-pair kernels.
 *
 * The paper (arXiv 2310.16122) names the hot kernels of CRK-HACC's adiabatic
 * solver and what each computes in one sentence (Sec. 5, opening paragraph):
 * Geometry (gas-particle volumes), Corrections (reproducing-kernel
 * coefficients), Acceleration (momentum derivative) and Energy (internal-
 * energy derivative); Sec. 3.1 adds the short-range gravity solver (direct
 * particle-particle force under a particle-mesh force split, polynomial order
 * 5 per the appendix's HACC_CUDA_POLY_ORDER), the two species, and the RCB
 * tree; Sec. 5.3 states that the kernels run over pairs of tree leaves.  The
 * paper prints no equation for any of them; each entry point below states the
 * reading it implements (conservative reproducing-kernel SPH, linear
 * corrections, Wendland C4 kernel with support 2h, symmetric h_ij = (h_i+h_j)/2,
 * periodic minimum image).
 *
 * Conventions for every call
 *  - All particle arrays are DEVICE pointers owned by the caller, FP32
 *    structure-of-arrays in the caller's original particle order, length n.
 *    Vectors are packed component-major: v3[c*n + i], c = 0,1,2.
 *  - Gas-only quantities (h, V, rho, u, A, B, ...) also have length n; their
 *    dark-matter entries are ignored on input and written as 0 on output.
 *  - Every compute call is asynchronous on the context's stream and does not
 *    synchronise.  crk_build_leaves synchronises once (it reads back sizes).
 *  - Every call returns CRK_OK (0) or a negative status; crk_last_error()
 *    gives a message.  Device-side results that the host cannot see without a
 *    synchronisation (singular moment matrices, pair counts) are written to
 *    optional device outputs instead.
 *  - Calls on one context must not run concurrently from several host threads.
 */
#ifndef CRK_H
#define CRK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRK_OK 0
#define CRK_EINVAL (-1)    /* bad argument (null pointer, negative size, bad mode) */
#define CRK_ENOMEM (-2)    /* device allocation failed */
#define CRK_ECUDA (-3)     /* a CUDA runtime call failed */
#define CRK_EBOX (-4)      /* a cut (r_c or 2 h_max) is not below half the box, or positions outside [0, box) */
#define CRK_ESTATE (-5)    /* leaves and arrays do not belong together */
#define CRK_ETIMEOUT (-6)  /* a bounded device wait expired (batched work queue) */
#define CRK_ETOOLARGE (-7) /* more particles than an allocation-free entry point can hold */

typedef struct crk_ctx crk_ctx;       /* opaque: device, stream, scratch arena, autotuner table */
typedef struct crk_leaves crk_leaves; /* opaque: library-owned device buffers of one leaf build */

/* One periodic box.  x, y, z in [0, box); species 0 = gas, 1 = dark matter. */
typedef struct {
    const float *x, *y, *z;
    const uint8_t *species;
    int64_t n;
    float box;
} crk_particles;

/* Leaf decomposition (Sec. 3.1 RCB tree; Sec. 5.3 leaf pairs).
 *  mode 0: fixed chaining mesh of cells_per_side^3 cells (a cell may hold at
 *          most 1024 particles);
 *  mode 1: recursive coordinate bisection down to leaves of <= max_leaf
 *          particles (1 <= max_leaf <= 1024).
 * r_cut_grav is the gravity cutoff used for the gravity leaf-pair list. */
typedef struct {
    int mode;
    int cells_per_side;
    int max_leaf;
    float r_cut_grav;
} crk_leaf_params;

/* Short-range gravity: g(s) = (s + eps^2)^-3/2 - sum_k poly[k] s^k, s = r^2,
 * zero for r >= r_cut (which must equal the leaves' r_cut_grav). */
typedef struct {
    float eps;
    float r_cut;
    float poly[6];
} crk_grav_params;

/* Ideal-gas index and Monaghan viscosity constants (alpha, beta, eta^2). */
typedef struct {
    float gamma;
    float alpha;
    float beta;
    float eta2;
} crk_hydro_params;

/* Create a context on `device` that issues all work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The context owns a
 * growable device scratch arena. */
int crk_create(crk_ctx **out, int device, void *cuda_stream);
void crk_destroy(crk_ctx *ctx);
int crk_set_stream(crk_ctx *ctx, void *cuda_stream);
const char *crk_last_error(const crk_ctx *ctx);
/* Library version and build info, e.g. "libcrk 1 sm_103a". */
const char *crk_version(void);
/* Tracing: when on (or when the environment variable CRK_TRACE is set at
 * crk_create), crk_build_leaves synchronises after each phase and prints the
 * phase times to stderr.  Off by default; it serialises the build. */
int crk_set_trace(crk_ctx *ctx, int on);
/* Kernel variants: the execution scheme of one pair kernel (the results agree
 * within FP32 rounding).  CRK_VARIANT_LISTS walks exact per-particle neighbour
 * lists (gas pairs for geometry, corrections, hydro and the geometry adjoint;
 * gravity pairs for gravity and its adjoint) that crk_build_leaves builds when
 * a kernel that uses them is set to LISTS at build time; CRK_VARIANT_TILES
 * sweeps ballot-compacted j-leaf tiles and needs no lists.  A kernel set to
 * LISTS on leaves built without its lists runs as TILES.  Defaults: LISTS for
 * the gas-pair kernels, TILES for the gravity kernels. */
#define CRK_K_GEOMETRY 0
#define CRK_K_CORRECTIONS 1
#define CRK_K_HYDRO 2
#define CRK_K_GRAVITY 3
#define CRK_K_GRAVITY_ADJOINT 4
#define CRK_K_GEOMETRY_ADJOINT 5
#define CRK_K_EXTRAS 6
#define CRK_K_ACCEL 7  /* the Acceleration pass (crk_hydro_accel, and inside crk_advance) */
#define CRK_K_ENERGY 8 /* the Energy pass (crk_hydro_energy, and inside crk_advance) */
#define CRK_N_KERNELS 9
#define CRK_VARIANT_LISTS 0
#define CRK_VARIANT_TILES 1
#define CRK_VARIANT_TILES16 2 /* tiles with two 16-particle i-groups per warp */
#define CRK_VARIANT_TILES8 3  /* tiles with four 8-particle i-groups per warp */
#define CRK_VARIANT_RING16 4  /* two 16-particle i-groups per warp, balanced ring-buffer sweeps
                                 (every kernel but hydro, which falls back to TILES) */
/* the paper's half-warp leaf-pair scheme (Sec. 5.3), for the gravity kernels and the hydro
 * passes (crk_hydro, Acceleration, Energy): lanes 0-15 hold 16 particles of leaf A, lanes 16-31
 * 16 of leaf B, and the pair is evaluated in both directions in one step; partial sums are
 * added atomically (the hydro passes then take their conservation sums from the finished
 * outputs).  The partner's particle arrives by register shuffle (Sec. 5.3.1), through shared
 * memory (Sec. 5.3.2), or by a second load.  The other gas kernels run tiles instead. */
#define CRK_VARIANT_HALFWARP_SHFL 5
#define CRK_VARIANT_HALFWARP_SMEM 6
#define CRK_VARIANT_HALFWARP_LOAD 7
/* gravity kernels: the candidates of each 32-particle group compacted once, then swept once per
 * 8-particle sub-cell (only those within the cut of its box) by 4 lanes per particle; the leaf
 * build makes the sub-cells RCB cells of 8 when a gravity kernel is set to it at build time */
#define CRK_VARIANT_SPLIT8 8
#define CRK_N_VARIANTS 9
int crk_set_variant(crk_ctx *ctx, int kernel, int variant);
/* Launch mode of every pair kernel: 0 (default) one block per i-leaf (one warp
 * per group for the list kernels); 1 persistent: a grid of resident blocks on
 * every SM (list kernels: as many as the kernel's registers and shared memory
 * allow; tiles kernels: 4) whose blocks (warps) take i-leaves (groups) from an
 * atomic work queue (no block ever waits on another).  Same results. */
int crk_set_persistent(crk_ctx *ctx, int on);
/* Launch shape of one pair kernel (CRK_K_*), as the autotuner sets it:
 * persistent as above; the j-tile depth of the packed tiles sweeps of the
 * gravity kernels (candidates compacted before each sweep: 32, 64 or 96); and
 * their warps per i-leaf block (4: one warp per 32-particle group of a
 * 128-leaf; 2: blocks of two warps, each taking two groups).  The other
 * kernels and variants sweep at depth 32 with 4 warps and ignore both.  The
 * results agree up to the order of FP32 additions.  CRK_EINVAL for an unknown
 * kernel, a depth other than 32, 64, 96 or warps other than 2, 4. */
int crk_set_launch(crk_ctx *ctx, int kernel, int persistent, int depth, int warps);
int crk_get_launch(const crk_ctx *ctx, int kernel, int *persistent, int *depth, int *warps);
int crk_get_variant(const crk_ctx *ctx, int kernel, int *variant);
/* Number of CUDA kernels this context has launched so far (host counter). */
int crk_launch_count(const crk_ctx *ctx, int64_t *out);

/* Build leaves (Sec. 3.1, 5.3).  Reads the positions and species, and the gas
 * smoothing lengths h (device, length n; dark-matter entries ignored), which
 * the leaves keep: every later call on these leaves uses this h.  Produces
 * the leaf permutation and two lists of leaf pairs: gravity (periodic box
 * gap < r_cut_grav) and hydro (both leaves hold gas, gap < 2 max h of the
 * two leaves).  The box gap of two leaves is, per axis, the smallest over
 * the periodic shifts {-box, 0, box} of the distance between their tight
 * FP32 boxes, summed in squares in FP64.  Errors: CRK_EBOX if r_cut_grav or
 * 2 max h is not below box/2 or a position lies outside [0, box).
 * Synchronises the context stream once. */
int crk_build_leaves(crk_ctx *ctx, const crk_particles *p, const float *h, const crk_leaf_params *lp,
                     crk_leaves **out);

/* Leaves of many independent periodic boxes in one build (the batched form):
 * the particles of box b are the consecutive range box_start[b] ..
 * box_start[b+1] - 1 of the device arrays, in [0, box_side[b]) (host arrays
 * box_start[nbox + 1], box_side[nbox]).  RCB leaves only (mode 1); every box
 * gets its own tree, leaves are numbered box by box, and leaf pairs never
 * cross boxes.  Every kernel then runs over all boxes in one launch.  Cuts
 * are checked per box (CRK_EBOX). */
typedef struct {
    const float *x, *y, *z;
    const uint8_t *species;
    int64_t n;
    int nbox;
    const int64_t *box_start;
    const float *box_side;
} crk_batch;
int crk_build_leaves_batch(crk_ctx *ctx, const crk_batch *b, const float *h, const crk_leaf_params *lp,
                           crk_leaves **out);

/* info[0] = n, info[1] = number of leaves, info[2] = gravity leaf pairs,
 * info[3] = hydro leaf pairs, info[4] = gravity image entries, info[5] = hydro
 * image entries (a leaf pair with several periodic images near each other
 * has one image entry per image). */
int crk_leaves_info(const crk_leaves *lv, int64_t info[6]);

/* Copy the canonical leaf structure to HOST arrays (synchronous; for checks):
 * perm[n] (original index of the particle at leaf-order position p; inside a
 * leaf gas comes first, then dark matter, each by original index),
 * leaf_start[n_leaves + 1], and the two CSR lists (ptr[n_leaves + 1],
 * list[pairs], j-leaves ascending, a = b included).  Any pointer may be NULL. */
int crk_leaves_export(crk_ctx *ctx, const crk_leaves *lv, int32_t *perm, int32_t *leaf_start, int32_t *grav_ptr,
                      int32_t *grav_list, int32_t *hydro_ptr, int32_t *hydro_list);
void crk_leaves_free(crk_ctx *ctx, crk_leaves *lv);

/* Capture-safe rebuild (the batched driver's CUDA graph holds the leaf build;
 * Sec. 5.3 runs every kernel over the leaf pairs of the current positions).
 * Recomputes leaves lv in place for new positions and h of the same particles
 * (same count, species, boxes and leaf parameters as the build that made lv),
 * with no host synchronisation and no allocation, so the call can be captured
 * in a CUDA graph together with the kernels that use the leaves.  Every
 * buffer keeps the size the first build gave it (the leaf-pair image lists
 * their first capacities, the gas neighbour lists 1/8 more groups than the
 * first build held).  What a build checks on the host becomes a bit of the
 * leaves' device status word instead: positions outside the box, gas h <= 0,
 * 2 h_max >= box/2, a changed gas count, a capacity overflow.  After a
 * nonzero status the leaves and every result computed from them are invalid:
 * build new leaves with crk_build_leaves.  The particle arrays are device
 * pointers laid out as for crk_build_leaves (crk_leaves_rebuild) or
 * crk_build_leaves_batch (crk_leaves_rebuild_batch).  Returns CRK_ESTATE
 * (before launching anything) if the inputs do not match the leaves, if the
 * leaves hold gravity neighbour lists (their sizes vary), or if the gas lists
 * were built by the exact two-pass path; the RCB tree shape of the context
 * must still be the one of lv (a context caches one shape: a build of other
 * boxes in between makes the next rebuild recompute it, which synchronises
 * and fails under stream capture). */
#define CRK_LEAVES_BAD_POSITION 1   /* a position outside [0, box) */
#define CRK_LEAVES_BAD_H 2          /* a gas h <= 0 or not finite */
#define CRK_LEAVES_GAS_COUNT 4      /* the number of gas particles changed */
#define CRK_LEAVES_LEAF_SIZE 8      /* a leaf above the largest leaf size */
#define CRK_LEAVES_HMAX 16          /* 2 h_max >= box/2 in some box */
#define CRK_LEAVES_CANDIDATES 32    /* a leaf with too many candidate leaves within the cut */
#define CRK_LEAVES_IMAGE_CAP 64     /* a leaf-pair image list above its capacity */
#define CRK_LEAVES_GROUP_CAP 128    /* more gas groups than the gas lists hold */
#define CRK_LEAVES_LIST_CAP 256     /* a gas neighbour list or group table above its capacity */
#define CRK_LEAVES_INTERNAL 512     /* an inconsistent RCB partition */
int crk_leaves_rebuild(crk_ctx *ctx, crk_leaves *lv, const crk_particles *p, const float *h);
int crk_leaves_rebuild_batch(crk_ctx *ctx, crk_leaves *lv, const crk_batch *b, const float *h);
/* Synchronises the context stream, then writes the status word of the last
 * build or rebuild of lv to *status (host; 0 = valid) and refreshes the pair
 * and image counts that crk_leaves_info reports. */
int crk_leaves_status(crk_ctx *ctx, crk_leaves *lv, int32_t *status);

/* Geometry (Sec. 5: volumes of gas particles).
 *   V_i = 1 / sum_{gas j, r_ij < 2 h_ij} W(r_ij, h_ij)  (j = i included),  rho_i = m_i / V_i.
 * Inputs m[n]; outputs V[n], rho[n].  pair_count (device int64, may be NULL)
 * receives the number of ordered in-range gas pairs with i != j. */
int crk_geometry(crk_ctx *ctx, const crk_leaves *lv, const float *m, float *V, float *rho, int64_t *pair_count);

/* Corrections (Sec. 5: reproducing-kernel coefficients), linear CRK.  With
 * w = V_j W_ij and x = x_ij the moments m0, m1, m2 and their gradients in the
 * evaluation point give B = -m2^-1 m1, A = 1/(m0 + B.m1),
 * dA = -A^2 (dm0 + 2 B.dm1 + B^T dm2 B), dB = -m2^-1 (dm1 + dm2 B).
 * Moment sums in FP32 (compensated for m0, m1, m2); the 3x3 inverse in FP64.
 * Outputs A[n], B[3n], gradA[3n], gradB[9n] with gradB[(3g+a)n + i] =
 * d B^a / d x^g.  A particle with det(m2) <= 1e-12 tr(m2)^3 gets NaN outputs
 * and is counted in n_singular (device int32, may be NULL). */
int crk_corrections(crk_ctx *ctx, const crk_leaves *lv, const float *V, float *A, float *B, float *gradA,
                    float *gradB, int32_t *n_singular);

/* Acceleration + Energy (Sec. 5: momentum and internal-energy derivatives),
 * CRKSPH with an unlimited Monaghan viscosity and an equal energy split:
 *   f_ij = -1/2 V_i V_j (P_i + P_j + Q_ij)(grad_i W^R_ij - grad_j W^R_ji),
 *   m_i dv_i/dt = sum_j f_ij,  m_i du_i/dt = -1/2 sum_j (v_i - v_j).f_ij,
 * P = (gamma-1) rho u, W^R_ij = A_i (1 + B_i.x_ij) W_ij.  Inputs m, v3, u, V,
 * rho, A, B, gradA, gradB; outputs dvdt3[3n], dudt[n].  conservation (device
 * double[4], may be NULL) receives sum m_i dv_i (3) and
 * sum m_i (v_i.dv_i + du_i) accumulated in FP64. */
int crk_hydro(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
              const float *u, const float *V, const float *rho, const float *A, const float *B, const float *gradA,
              const float *gradB, float *dvdt3, float *dudt, double *conservation, int64_t *pair_count);

/* Extras (Sec. 5: "evaluates the density and state gradients").  The paper
 * prints no formula; CRKSPH reading, over gas j including j = i, with the
 * corrected kernel W^R_ij = A_i (1 + B_i.x_ij) W_ij and its evaluation-point
 * gradient (as in crk_hydro):
 *   rho_r_i = sum_j m_j W^R_ij                        (corrected-kernel density)
 *   dvdx_i[3a+b] = sum_j V_j (v_j^a - v_i^a) (grad_i W^R_ij)^b   (d v^a / d x^b)
 * Inputs m, v3, V and the corrections A, B, gradA, gradB (caller order);
 * outputs rho_r[n], dvdx[9n] with dvdx[(3a+b)n + i]; dark matter gets 0.
 * pair_count as for crk_geometry. */
int crk_extras(crk_ctx *ctx, const crk_leaves *lv, const float *m, const float *v3, const float *V, const float *A,
               const float *B, const float *gradA, const float *gradB, float *rho_r, float *dvdx,
               int64_t *pair_count);

/* crk_hydro with the limited viscosity (the paper prints no formula; CRKSPH
 * reading fed by crk_extras): the viscosity sees both velocities
 * reconstructed linearly to the pair midpoint, v*_ij = v_ij - phi/2 (s_i + s_j)
 * with s = dvdx x_ij, and the van Leer limiter phi = 4r/(1+r)^2 for
 * r = (x.s_i)/(x.s_j) > 0, else 0.  Q_ij stays symmetric, so momentum and
 * energy are conserved as before; the work term keeps the true v_ij.  dvdx is
 * the crk_extras output layout; rho is the density the equation of state uses
 * (crk_extras' rho_r in the Extras chain). */
int crk_hydro_limited(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m,
                      const float *v3, const float *u, const float *V, const float *rho, const float *A,
                      const float *B, const float *gradA, const float *gradB, const float *dvdx, float *dvdt3,
                      float *dudt, double *conservation, int64_t *pair_count);

/* Acceleration pass of a timestep (Sec. 5: the momentum derivative; Sec. 5.4:
 * Acceleration and Energy each run twice per timestep).  The pair force of
 * crk_hydro (dvdx NULL: Monaghan viscosity) or crk_hydro_limited (dvdx given)
 * summed into dvdt3[3n] only, plus the signal velocity (the paper prints no
 * formula; Monaghan's pair signal speed, over gas j in range incl. j = i):
 *   vsig_i = max_j (c_i + c_j - sig_beta min(0, v_ij.x_ij / r_ij)),
 * folded into *vsig_h_max = max(*vsig_h_max, max_i vsig_i / h_i) by an atomic
 * max on the FP32 bit pattern (Sec. 5.1: floating-point atomic max; a
 * non-negative FP32 value orders like its bits).  vsig_h_max: device uint32
 * holding FP32 bits, may be NULL; the pass only raises it, so the caller
 * zeroes it once per step.  conservation (device double[4], may be NULL):
 * sum m_i dv_i (3) and sum m_i v_i.dv_i.  sig_beta >= 0, else CRK_EINVAL. */
int crk_hydro_accel(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
                    const float *u, const float *V, const float *rho, const float *A, const float *B,
                    const float *gradA, const float *gradB, const float *dvdx, float sig_beta, float *dvdt3,
                    uint32_t *vsig_h_max, double *conservation, int64_t *pair_count);

/* Energy pass (Sec. 5: the internal-energy derivative) with the compatible
 * split (the paper prints no formula; compatible differencing of the pair
 * work): the pair force f_ij as in crk_hydro_accel (same v3, u, dvdx), its
 * work on the time-centred velocities vstar3[3n] returned as heat,
 *   dE_ij = -f_ij.(v*_i - v*_j),
 * of which i takes the share
 *   w_ij = 1/2 (1 + sgn(dE_ij) (u_j - u_i) / (|u_j - u_i| + (u_i + u_j)/2))
 * (1/2 for u_i = u_j: heating favours the colder particle, cooling the
 * hotter), m_i du_i/dt = sum_j w_ij dE_ij into dudt[n].  w_ij + w_ji = 1, so
 * sum m_i du_i = -sum m_i v*_i.dv_i: a step with v* = (v + v1)/2 conserves
 * kinetic plus thermal energy.  conservation (device double[4], may be
 * NULL): sum m_i dv_i (3) and sum m_i (v*_i.dv_i + du_i) (zero up to
 * rounding).  With equal u and vstar3 = v3 this is crk_hydro's dudt. */
int crk_hydro_energy(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
                     const float *u, const float *V, const float *rho, const float *A, const float *B,
                     const float *gradA, const float *gradB, const float *dvdx, const float *vstar3, float *dudt,
                     double *conservation, int64_t *pair_count);

/* Courant timestep from the signal-velocity max of crk_hydro_accel:
 * *dt = min(dt_max, cfl / q) with q = max_i vsig_i / h_i read from
 * *vsig_h_max (dt_max when q = 0).  Device in, device out (no host sync);
 * cfl > 0 and dt_max > 0, else CRK_EINVAL. */
int crk_timestep(crk_ctx *ctx, const uint32_t *vsig_h_max, float cfl, float dt_max, float *dt);

/* Parameters of crk_advance.  cfl, dt_max: the Courant step; dt_fixed > 0
 * replaces it; sig_beta as in crk_hydro_accel; limited != 0: Extras and the
 * limited viscosity with rho_r as the equation-of-state density (else the
 * Monaghan viscosity on the geometry density); gravity != 0: grav_short is
 * added to the kicks of every species (dark matter feels gravity only). */
typedef struct {
    float cfl;
    float dt_max;
    float dt_fixed;
    float sig_beta;
    int limited;
    int gravity;
} crk_advance_params;

/* One two-stage kick-drift timestep with the compatible energy update (the
 * paper prints no integrator; Sec. 5.4 calls Acceleration and Energy twice
 * per step).  Stage 1 at t^n: leaves, geometry, corrections (Extras),
 * Acceleration (with the signal velocity), Energy on v* = v, gravity; the
 * Courant dt; the predictor v_p = v + dt/2 a, u_p = u + dt/2 du,
 * x_p = x + dt/2 v_p.  Stage 2 at the predicted state: leaves, the same chain,
 * Acceleration a_p; the kick v1 = v + dt a_p; Energy on v* = (v + v1)/2;
 * u1 = u + dt du; the drift x1 = x + dt v* wrapped into [0, box).
 * Device arrays in the caller's order: x, y, z, v3[3n], u updated in place;
 * species, h, m held fixed.  dt: device float (out).  conservation (device
 * double[4], may be NULL): the final Energy pass' balance.  n_singular
 * (device int32, may be NULL): singular corrections over both stages.  The
 * two leaf builds read back their sizes (host syncs); everything else stays
 * on the context stream.  Errors as crk_build_leaves and the single calls;
 * CRK_ESTATE when gravity is on and gp->r_cut != lp->r_cut_grav. */
int crk_advance(crk_ctx *ctx, int64_t n, float box, float *x, float *y, float *z, const uint8_t *species,
                const float *h, const float *m, float *v3, float *u, const crk_leaf_params *lp,
                const crk_hydro_params *hp, const crk_grav_params *gp, const crk_advance_params *ap, float *dt,
                double *conservation, int32_t *n_singular);

/* Short-range gravity (Sec. 3.1), G = 1, all species:
 *   a_i = sum_{j != i, r < r_c} m_j (x_j - x_i) g(r^2).
 * Input m[n]; output a3[3n]. */
int grav_short(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const float *m, float *a3,
               int64_t *pair_count);

/* Reverse mode of grav_short for a cotangent abar3 = dL/da (not in the paper):
 *   gm_k = -sum_j abar_j . d_kj g(s_kj),
 *   gx_k =  sum_j J(d_kj) (m_k abar_j - m_j abar_k),  J(d) = g I + 2 g'(s) d d^T,
 * with d_kj = x_j - x_k; pair terms are recomputed, nothing per pair is stored.
 * Outputs gx3[3n], gm[n] (overwritten). */
int grav_short_adjoint(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const float *m,
                       const float *abar3, float *gx3, float *gm);

/* Reverse mode of crk_geometry at fixed h (not in the paper).  With
 * S_i = 1/V_i and cotangents rhobar (and Vbar, may be NULL):
 *   Sbar_i = rhobar_i m_i - Vbar_i V_i^2,  gm_i = rhobar_i S_i,
 *   gx_k = sum_j (Sbar_k + Sbar_j) grad_k W_kj.
 * V is the forward output.  Outputs gx3[3n], gm[n] (overwritten; dark matter 0). */
int crk_geometry_adjoint(crk_ctx *ctx, const crk_leaves *lv, const float *m, const float *V, const float *rhobar,
                         const float *Vbar, float *gx3, float *gm);

/* Reverse mode of crk_corrections (not in the paper; extends the gravity and
 * geometry adjoints to the corrections).  For cotangents Abar[n], Bbar[3n],
 * gradAbar[3n], gradBbar[9n] (the layouts of crk_corrections' outputs) it
 * returns the gradient of
 *   L = sum_i Abar_i A_i + Bbar_i.B_i + gradAbar_i.gradA_i + gradBbar_i:gradB_i
 * in the positions, xbar3[3n], and in the volumes, Vbar[n] (h held fixed; the
 * leaves are constant).  Pair (i, j) enters i's moments as V_j t(x_ij); each
 * particle's moment cotangents come from the closed-form reverse of its FP64
 * 3x3 step (a first sweep recomputes the moments), then
 *   xbar_i = sum_j V_j grad T_i(x_ij) - V_i grad T_j(x_ji),  Vbar_i = sum_j T_j(x_ji)
 * with T_i the moment terms weighted by i's cotangents (a second sweep; nothing
 * per pair is stored).  A singular particle contributes nothing and is
 * counted in n_singular (device int32, may be NULL).  Outputs overwritten;
 * dark matter gets 0. */
int crk_corrections_adjoint(crk_ctx *ctx, const crk_leaves *lv, const float *V, const float *Abar,
                            const float *Bbar, const float *gradAbar, const float *gradBbar, float *xbar3,
                            float *Vbar, int32_t *n_singular);

/* Reverse mode of crk_hydro (Monaghan viscosity, equal split; not in the
 * paper) for cotangents dvbar3[3n] of dvdt3 and dubar[n] of dudt, every input
 * of the pair force held independent: the gradients in the positions
 * (xbar3[3n]), velocities (vbar3[3n]), u, m, V, rho (ubar, mbar, Vbar, rhobar
 * [n]) and the corrections (Abar[n], Bbar3[3n], gradAbar3[3n], gradBbar9[9n],
 * crk_corrections' layouts).  With a_i = dvbar_i/m_i and b_i = dubar_i/m_i the
 * loss is a sum over unordered pairs of (a_i - a_j).f_ij + (b_i + b_j) e_ij;
 * each particle gathers the derivative of its pairs' terms in its own inputs
 * (pair terms recomputed, no atomics).  Chained with crk_corrections_adjoint
 * and crk_geometry_adjoint it gives the gradient of a loss of dv/dt, du/dt in
 * the positions and masses through the whole forward chain.  Outputs
 * overwritten; dark matter gets 0. */
int crk_hydro_adjoint(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
                      const float *u, const float *V, const float *rho, const float *A, const float *B,
                      const float *gradA, const float *gradB, const float *dvbar3, const float *dubar, float *xbar3,
                      float *vbar3, float *ubar, float *mbar, float *Vbar, float *rhobar, float *Abar, float *Bbar3,
                      float *gradAbar3, float *gradBbar9);

/* Forward and reverse pass of the hydro chain on one set of leaves, with
 * every intermediate in the library's kernel order (as crk_step): geometry,
 * corrections, hydro (its outputs only when dvdt3 or dudt is given), then
 * crk_hydro_adjoint, crk_corrections_adjoint and crk_geometry_adjoint chained,
 * for the cotangents dvbar3[3n], dubar[n] of dv/dt and du/dt.  Returns the
 * gradient of L = sum dvbar.dv/dt + dubar du/dt in the positions (xbar3[3n])
 * and masses (mbar[n]) through V, rho and the corrections, and in the
 * velocities (vbar3[3n]) and u (ubar[n]); every output may be NULL; caller
 * order and layouts; h held fixed.  n_singular as for crk_corrections. */
typedef struct {
    const float *m, *v3, *u;       /* inputs */
    const float *dvbar3, *dubar;   /* cotangents */
    float *dvdt3, *dudt;           /* forward outputs, may be NULL */
    float *xbar3, *mbar, *vbar3, *ubar;  /* gradients, may be NULL */
    int32_t *n_singular;           /* may be NULL */
} crk_chain_adjoint_io;

int crk_hydro_chain_adjoint(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp,
                            const crk_chain_adjoint_io *io);

/* One whole step of the path on one set of leaves, in this order: geometry,
 * corrections, hydro, gravity, gravity adjoint, geometry adjoint.  Inputs m,
 * v3, u (caller order, as for the single calls).  The intermediates stay in
 * the library's kernel order (coalesced, no scatter/gather round trips);
 * every output pointer may be NULL, and those given receive the values in the
 * caller's order and layout.  The adjoint cotangents default to the loss
 * sum |a|^2 + sum_gas rho (abar3 = NULL: 2a; rhobar = NULL: 1 on gas); Vbar
 * may be NULL.  pair_count (device int64[3], may be NULL) receives the
 * geometry, hydro and gravity pair counts, and swept_count (read only with
 * pair_count) the candidate pair evaluations of the same kernels (tiles: every
 * active lane of a group times every swept candidate; lists: the list
 * entries), so pair_count/swept_count is the useful fraction of the pair work;
 * n_singular and conservation as for
 * the single calls.  With extras != 0 the step runs crk_extras after the
 * corrections and crk_hydro_limited in place of crk_hydro, with rho_r as the
 * equation-of-state density (rho then still receives the geometry density). */
typedef struct {
    const float *m, *v3, *u;                /* inputs */
    float *V, *rho, *A, *B, *gradA, *gradB; /* geometry, corrections */
    float *dvdt3, *dudt;                    /* hydro */
    double *conservation;                   /* double[4], may be NULL */
    float *a3;                              /* gravity */
    const float *abar3;                     /* gravity cotangent, NULL = 2 a */
    float *gx3_grav, *gm_grav;              /* gravity adjoint */
    const float *rhobar, *Vbar;             /* geometry cotangents; rhobar NULL = 1 on gas; Vbar may be NULL */
    float *gx3_geom, *gm_geom;              /* geometry adjoint */
    int32_t *n_singular;                    /* may be NULL */
    int64_t *pair_count;                    /* int64[3], may be NULL */
    int extras;                             /* nonzero: Extras chain (see below) */
    float *rho_r, *dvdx;                    /* Extras outputs, may be NULL */
    int64_t *swept_count;                   /* int64[3], may be NULL: candidate pair evaluations */
} crk_step_io;

int crk_step(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
             const crk_step_io *io);

/* Per-stage timing of crk_step.  crk_step_profile(ctx, k) creates 8 CUDA
 * events for each of the next k steps (0 turns profiling off); those steps
 * record them on the context stream: start, after geometry, corrections,
 * hydro, gravity, gravity adjoint, geometry adjoint, and after the outputs.
 * crk_step_profile_read waits for the last recorded event, returns the mean
 * ms of the 7 intervals over the recorded steps (the first interval includes
 * the input permutation, the sixth the cotangent kernel) and starts over. */
int crk_step_profile(crk_ctx *ctx, int max_steps);
int crk_step_profile_read(crk_ctx *ctx, float ms[7], int *steps);

/* CUDA graph of crk_step (the batched form: one graph launch replays every
 * kernel of the step).  Creation runs one uncaptured step (sizing the scratch
 * arena) and then captures one step on the context stream, which must not be
 * the legacy default stream.  The graph bakes in the leaves, the arrays and
 * the kernel variants current at creation; replay it only while they are
 * alive and unchanged in shape (their contents may change). */
typedef struct crk_graph crk_graph;
int crk_step_graph_create(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
                          const crk_step_io *io, crk_graph **out);
/* The batched driver as one CUDA graph: crk_leaves_rebuild_batch of lv (for the
 * positions and h the arrays of b and h hold when the graph is launched) and
 * then crk_step, every pair kernel in its context launch shape (persistent
 * where crk_set_persistent or the autotuner chose it).  The creating call runs
 * one rebuild and step uncaptured first (sizing the scratch), and fails with
 * CRK_ESTATE if that rebuild's status is nonzero.  After each launch the
 * caller reads crk_leaves_status when it needs to know the leaves were valid
 * (a nonzero status invalidates that step's outputs). */
int crk_rebuild_step_graph_create(crk_ctx *ctx, crk_leaves *lv, const crk_batch *b, const float *h,
                                  const crk_grav_params *gp, const crk_hydro_params *hp, const crk_step_io *io,
                                  crk_graph **out);
int crk_graph_launch(crk_graph *g);
void crk_graph_destroy(crk_graph *g);

/* Autotuner (Sec. 5.2 tunes register use and sub-group size per kernel and
 * device; here the dimensions are the sweep variant, the launch mode, the
 * j-tile depth and the warps per leaf).  For every kernel CRK_K_* it times each variant on these
 * leaves (best of reps after a warm-up, CUDA events on the context stream;
 * a candidate whose warm-up takes more than three times the best time so far
 * is not timed further and reports its warm-up time) and keeps the fastest,
 * then times the fastest variant non-persistent and
 * persistent, then (gravity kernels on tiles) at depths 32, 64 and 96 and with
 * 2 and 4 warps per leaf, and keeps the fastest shape in the context.
 * ms_out[CRK_N_KERNELS * CRK_TUNE_COLS] (kernel-major: CRK_N_VARIANTS variant
 * timings, 2 launch-mode timings, 3 depth timings, 2 warps timings; -1 = not
 * timed) and best_out[4 * CRK_N_KERNELS] (variant, persistent, depth, warps
 * per kernel) are host arrays and may be NULL.  Runs one
 * crk_step first; every output array of io must be given (they are
 * overwritten while timing).  Extras is timed when io->extras is set, the
 * Acceleration and Energy passes always (with io->dvdx as the limiter's
 * velocity gradient when io->extras is set). */
#define CRK_TUNE_COLS (CRK_N_VARIANTS + 7)
int crk_tune(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
             const crk_step_io *io, int reps, float *ms_out, int *best_out);

/* Allocation-free short-range gravity.  The paper has no counterpart: this is
 * for callers that cannot let a library allocate device memory, such as an
 * application whose own memory pool already owns the GPU, or a step loop that
 * must never pay the device synchronisation cudaMalloc/cudaFree can imply.
 * It computes what grav_short computes, with grav_short's tiles kernel, or
 * its lists kernel when the context's gravity variant is CRK_VARIANT_LISTS
 * and the leaves hold gravity lists (no pair count).  The other sweep
 * variants and the persistent launch mode are not used here: after crk_tune
 * or crk_set_variant selects one of them, the two calls agree within FP32
 * rounding instead of bit for bit.  It calls no cudaMalloc, cudaFree or other
 * allocating routine: its only
 * scratch, 16 bytes per particle, is a file-scope device array of
 * CRK_NOALLOC_MAX_PARTICLES entries (32 MiB) that every GPU which loads the
 * library holds until the process exits.  The caller passes the inputs (leaves
 * built earlier, m) and the output a3 as for grav_short.
 *  - n > CRK_NOALLOC_MAX_PARTICLES: returns CRK_ETOOLARGE and does nothing.
 *  - The context's device must be the current device (else CRK_ESTATE).
 *  - The first call on a device looks up the array's device address (a
 *    runtime query, no allocation); make that first call before any stream
 *    capture begins.
 *  - All calls share the one array: calls whose work overlaps on the GPU
 *    (other streams, other host threads) race and give wrong results; issue
 *    them in one stream order.  Nothing in the array needs clearing: every
 *    call rewrites the entries it reads.
 * Errors are reported by the status code only (crk_last_error is not set). */
#define CRK_NOALLOC_MAX_PARTICLES (1 << 21)
int grav_short_noalloc(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const float *m, float *a3);

#ifdef __cplusplus
}
#endif
#endif /* CRK_H */
