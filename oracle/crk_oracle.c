/*
 * crk_oracle.c -- plain, slow FP64 CPU oracle of the CRK-HACC short-range pair
 * kernels.  TEST INFRASTRUCTURE ONLY: nothing in the product path links,
 * loads or calls this file; it shares no code, header or table with the CUDA
 * library.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it (through oracle/oracle.py).
 *
 * What the paper fixes, and what it leaves open.
 *   The paper (Sec. 5, opening paragraph) names the hot kernels and what each
 *   computes in one sentence: Geometry (gas-particle volumes), Corrections
 *   (reproducing-kernel coefficients), Extras (density and state gradients),
 *   Acceleration (momentum derivative) and Energy (internal-energy
 *   derivative).  Sec. 3.1 adds the short-range
 *   gravity solver (direct particle-particle force under a particle-mesh force
 *   split), the two species (dark matter: gravity only; gas: gravity + hydro)
 *   and the RCB tree; Sec. 5.3 adds that kernels run over pairs of leaves; the
 *   appendix fixes the gravity polynomial order (HACC_CUDA_POLY_ORDER=5).
 *   The paper prints no equation for any kernel.  Every formula below is the
 *   standard reading of linear conservative reproducing-kernel SPH (CRKSPH)
 *   and is marked "paper silent"; each has invariant pins in tests/.
 *
 * Conventions (all "paper silent" readings):
 *   - periodic cube of side L, minimum image: d <- d - L*rint(d/L);
 *   - x_ij = x_i - x_j; symmetric smoothing length h_ij = (h_i + h_j)/2;
 *   - Wendland C4 kernel in 3-D with support 2h;
 *   - hydro sums run over gas j including j = i; gravity sums over all j != i;
 *   - a pair is "in range" iff r^2 < cut^2 with cut = 2 h_ij (hydro) or r_c.
 *   Positions, masses etc. are FP64 here; the tests promote the FP32 inputs
 *   exactly.  Compile with -ffp-contract=off so that the integer decisions
 *   (leaves, leaf pairs) are the exact IEEE results of the stated operations.
 *
 * Neighbour search: brute force over all particles, or a periodic cell list
 * with cells no smaller than the largest cut (27 neighbouring cells).  Both
 * visit every j with r < cut; tests check that they agree.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EBOX (-4)

static const double PI = 3.14159265358979323846;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Wendland C4 (3-D), support 2h.  Paper silent; standard form:              */
/*   W(r,h) = 495/(256 pi h^3) (1 - q/2)^6 (1 + 3q + 35q^2/12),  q = r/h < 2 */
/*   (dW/dr)/r = 495/(256 pi h^5) (1 - q/2)^5 (-14/3)(1 + 5q/2)             */
/* The second form is dW/dr divided by r, so grad_i W_ij = that * x_ij.      */
/* ------------------------------------------------------------------------ */
static void wendland(double r, double h, double *W, double *dWr) {
    double q = r / h;
    if (q >= 2.0) { *W = 0.0; *dWr = 0.0; return; }
    double s = 495.0 / (256.0 * PI);
    double t = 1.0 - 0.5 * q;
    double t5 = t * t * t * t * t;
    double h3 = h * h * h;
    *W = s / h3 * t5 * t * (1.0 + 3.0 * q + 35.0 * q * q / 12.0);
    *dWr = s / (h3 * h * h) * t5 * (-14.0 / 3.0) * (1.0 + 2.5 * q);
}

void orc_wendland(int64_t n, const double *r, const double *h, double *W, double *dWr) {
    for (int64_t i = 0; i < n; ++i) wendland(r[i], h[i], &W[i], &dWr[i]);
}

/* ------------------------------------------------------------------------ */
/* Short-range gravity pair function (Sec. 3.1: softened Newtonian pair      */
/* force minus a polynomial fit of the mesh force; order 5 from the          */
/* appendix).  Paper silent on the exact form; reading:                      */
/*   g(s) = (s + eps^2)^(-3/2) - sum_k c_k s^k,  s = r^2,  zero for r >= r_c */
/*   g'(s) = -3/2 (s + eps^2)^(-5/2) - sum_k k c_k s^(k-1)                  */
/* ------------------------------------------------------------------------ */
static double grav_g(double s, double eps, const double *c) {
    double p = 0.0, sk = 1.0;
    for (int k = 0; k <= 5; ++k) { p += c[k] * sk; sk *= s; }
    return pow(s + eps * eps, -1.5) - p;
}

static double grav_dg(double s, double eps, const double *c) {
    double p = 0.0, sk = 1.0;
    for (int k = 1; k <= 5; ++k) { p += (double)k * c[k] * sk; sk *= s; }
    return -1.5 * pow(s + eps * eps, -2.5) - p;
}

void orc_grav_g(int64_t n, const double *s, double eps, const double *c, double *g, double *dg) {
    for (int64_t i = 0; i < n; ++i) { g[i] = grav_g(s[i], eps, c); dg[i] = grav_dg(s[i], eps, c); }
}

/* ------------------------------------------------------------------------ */
/* neighbour search                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t count;       /* particles indexed */
    int64_t *items;      /* particle ids, grouped by cell */
    int64_t *start;      /* nc^3 + 1 offsets (NULL when brute force) */
    int nc;              /* cells per side; 0 = brute force */
    double cs;           /* cell side */
    int64_t max_cell;
} CellList;

static void min_image(const double *pi, const double *pj, double L, double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double t = pi[a] - pj[a];
        d[a] = t - L * rint(t / L);
    }
}

static int cell_coord(double x, double cs, int nc) {
    int c = (int)floor(x / cs);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

/* mask: NULL = all particles; else only particles with mask[i] != 0 */
static int cells_build(CellList *cl, int64_t n, const double *pos, const uint8_t *mask, double L, double cut,
                       int brute) {
    memset(cl, 0, sizeof(*cl));
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) if (!mask || mask[i]) ++cnt;
    cl->count = cnt;
    cl->items = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!cl->items) return ORC_ENOMEM;
    int nc = brute ? 0 : (int)floor(L / cut);
    if (nc < 3) nc = 0;
    if (nc > 512) nc = 512;
    cl->nc = nc;
    if (nc == 0) {
        int64_t k = 0;
        for (int64_t i = 0; i < n; ++i) if (!mask || mask[i]) cl->items[k++] = i;
        cl->max_cell = cnt;
        return ORC_OK;
    }
    cl->cs = L / nc;
    int64_t ncell = (int64_t)nc * nc * nc;
    cl->start = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    if (!cl->start || !fill) { free(fill); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        int64_t c = ((int64_t)cell_coord(pos[3 * i], cl->cs, nc) * nc + cell_coord(pos[3 * i + 1], cl->cs, nc)) * nc +
                    cell_coord(pos[3 * i + 2], cl->cs, nc);
        cl->start[c + 1]++;
    }
    cl->max_cell = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        if (cl->start[c + 1] > cl->max_cell) cl->max_cell = cl->start[c + 1];
        cl->start[c + 1] += cl->start[c];
    }
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        int64_t c = ((int64_t)cell_coord(pos[3 * i], cl->cs, nc) * nc + cell_coord(pos[3 * i + 1], cl->cs, nc)) * nc +
                    cell_coord(pos[3 * i + 2], cl->cs, nc);
        cl->items[cl->start[c] + fill[c]++] = i;
    }
    free(fill);
    return ORC_OK;
}

static void cells_free(CellList *cl) {
    free(cl->items);
    free(cl->start);
}

static int64_t cells_buffer_size(const CellList *cl) {
    return cl->nc == 0 ? (cl->count > 0 ? cl->count : 1) : 27 * (cl->max_cell > 0 ? cl->max_cell : 1);
}

/* every indexed particle in the 27 cells around p (all of them when brute) */
static int64_t cells_candidates(const CellList *cl, const double *p, int64_t *buf) {
    if (cl->nc == 0) {
        memcpy(buf, cl->items, sizeof(int64_t) * (size_t)cl->count);
        return cl->count;
    }
    int nc = cl->nc;
    int cx = cell_coord(p[0], cl->cs, nc), cy = cell_coord(p[1], cl->cs, nc), cz = cell_coord(p[2], cl->cs, nc);
    int64_t k = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
                int64_t c = ((int64_t)x * nc + y) * nc + z;
                for (int64_t t = cl->start[c]; t < cl->start[c + 1]; ++t) buf[k++] = cl->items[t];
            }
    return k;
}

/* the i-loop: either every particle, or only the listed subset */
#define FOR_EACH_I(sub, nsub, n, ...)                                                     \
    do {                                                                                  \
        int64_t nI = (sub) ? (nsub) : (n);                                                \
        _Pragma("omp parallel") {                                                         \
            int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cells_buffer_size(&cl)); \
            _Pragma("omp for schedule(dynamic, 64) reduction(+ : pairs)")                 \
            for (int64_t ii = 0; ii < nI; ++ii) {                                         \
                int64_t i = (sub) ? (sub)[ii] : ii;                                       \
                __VA_ARGS__                                                               \
            }                                                                             \
            free(buf);                                                                    \
        }                                                                                 \
    } while (0)

static double max_h_gas(int64_t n, const uint8_t *species, const double *h) {
    double hm = 0.0;
    for (int64_t i = 0; i < n; ++i) if (species[i] == 0 && h[i] > hm) hm = h[i];
    return hm;
}

static uint8_t *gas_mask(int64_t n, const uint8_t *species) {
    uint8_t *m = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) m[i] = species[i] == 0;
    return m;
}

/* ------------------------------------------------------------------------ */
/* short-range gravity:  a_i = sum_{j != i, r < r_c} m_j (x_j - x_i) g(r^2)   */
/* (G = 1).  npairs counts ordered in-range pairs (i, j != i) for i in the    */
/* i-set.                                                                     */
/* ------------------------------------------------------------------------ */
int orc_gravity(int64_t n, const double *pos, const double *m, double L, double rc, double eps, const double *poly,
                const int64_t *sub, int64_t nsub, int brute, double *acc, int64_t *npairs) {
    if (n < 0 || L <= 0 || rc <= 0 || !(rc < 0.5 * L)) return ORC_EBOX;
    CellList cl;
    if (cells_build(&cl, n, pos, NULL, L, rc, brute)) return ORC_ENOMEM;
    int64_t pairs = 0;
    double rc2 = rc * rc;
    FOR_EACH_I(sub, nsub, n, {
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            if (j == i) continue;
            double d[3];
            min_image(&pos[3 * j], &pos[3 * i], L, d); /* d = x_j - x_i */
            double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(s < rc2)) continue;
            ++pairs;
            double g = grav_g(s, eps, poly);
            for (int c = 0; c < 3; ++c) a[c] += m[j] * d[c] * g;
        }
        for (int c = 0; c < 3; ++c) acc[3 * i + c] = a[c];
    });
    cells_free(&cl);
    if (npairs) *npairs = pairs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* gravity adjoint (reverse mode of orc_gravity, h-free).  With d = x_j-x_i, */
/* F(d) = d g(|d|^2) and J(d) = g I + 2 g'(s) d d^T, for a cotangent abar:   */
/*   dL/dm_k = - sum_j abar_j . d_kj g(s_kj)                                  */
/*   dL/dx_k =   sum_j J(d_kj) (m_k abar_j - m_j abar_k)                      */
/* (paper silent: the adjoint is not part of the paper).                      */
/* ------------------------------------------------------------------------ */
int orc_gravity_adjoint(int64_t n, const double *pos, const double *m, double L, double rc, double eps,
                        const double *poly, const double *abar, const int64_t *sub, int64_t nsub, int brute,
                        double *gx, double *gm, int64_t *npairs) {
    if (n < 0 || L <= 0 || rc <= 0 || !(rc < 0.5 * L)) return ORC_EBOX;
    CellList cl;
    if (cells_build(&cl, n, pos, NULL, L, rc, brute)) return ORC_ENOMEM;
    int64_t pairs = 0;
    double rc2 = rc * rc;
    FOR_EACH_I(sub, nsub, n, {
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double gxi[3] = {0.0, 0.0, 0.0}, gmi = 0.0;
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            if (j == i) continue;
            double d[3];
            min_image(&pos[3 * j], &pos[3 * i], L, d); /* d_ij = x_j - x_i */
            double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(s < rc2)) continue;
            ++pairs;
            double g = grav_g(s, eps, poly), dg = grav_dg(s, eps, poly);
            double w[3];
            for (int c = 0; c < 3; ++c) w[c] = m[i] * abar[3 * j + c] - m[j] * abar[3 * i + c];
            double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            for (int c = 0; c < 3; ++c) gxi[c] += g * w[c] + 2.0 * dg * d[c] * dw;
            gmi -= (abar[3 * j] * d[0] + abar[3 * j + 1] * d[1] + abar[3 * j + 2] * d[2]) * g;
        }
        for (int c = 0; c < 3; ++c) gx[3 * i + c] = gxi[c];
        gm[i] = gmi;
    });
    cells_free(&cl);
    if (npairs) *npairs = pairs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 5: "measures the volumes of gas particles").  Paper silent */
/* on the formula; CRKSPH reading:                                           */
/*   V_i = 1 / sum_{j gas, r_ij < 2h_ij} W(r_ij, h_ij)   (j = i included)    */
/*   rho_i = m_i / V_i                                                        */
/* Dark-matter entries of V and rho are left at 0.                           */
/* ------------------------------------------------------------------------ */
int orc_geometry(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m, double L,
                 const int64_t *sub, int64_t nsub, int brute, double *V, double *rho, int64_t *npairs) {
    double hmax = max_h_gas(n, species, h);
    if (n < 0 || L <= 0 || !(2.0 * hmax < 0.5 * L)) return ORC_EBOX;
    uint8_t *gm = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gm, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, brute)) { free(gm); return ORC_ENOMEM; }
    int64_t pairs = 0;
    FOR_EACH_I(sub, nsub, n, {
        if (species[i] != 0) { V[i] = 0.0; rho[i] = 0.0; continue; }
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double S = 0.0;
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double d[3];
            min_image(&pos[3 * i], &pos[3 * j], L, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            if (j != i) ++pairs;
            double W, dWr;
            wendland(sqrt(r2), hij, &W, &dWr);
            S += W;
        }
        V[i] = 1.0 / S;
        rho[i] = m[i] / V[i];
    });
    cells_free(&cl);
    free(gm);
    if (npairs) *npairs = pairs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Corrections (Sec. 5: "computes the reproducing kernel coefficients").     */
/* Paper silent; linear CRK reading with w_j = V_j W_ij and x = x_ij:        */
/*   m0 = sum w, m1^a = sum w x^a, m2^ab = sum w x^a x^b                     */
/*   d_g m0    = sum V_j d_g W                                               */
/*   d_g m1^a  = sum V_j (delta_ag W + x^a d_g W)                            */
/*   d_g m2^ab = sum V_j (delta_ag x^b W + delta_bg x^a W + x^a x^b d_g W)   */
/*   B = -M^-1 m1,  A = 1/(m0 + B.m1)      (M = m2)                          */
/*   d_g A = -A^2 (d_g m0 + 2 B.d_g m1 + B^T (d_g M) B)                      */
/*   d_g B = -M^-1 (d_g m1 + (d_g M) B)                                      */
/* with d_g = d/dx_i^g at fixed h and V: the derivative in the evaluation    */
/* point x_i with every particle (i included) held in place, so              */
/* d x_ij/d x_i = I in every term, the self term too (the CRKSPH convention  */
/* under which sum_j V_j grad_i W^R_ij = 0 holds exactly).                   */
/* Output layout: B[i][a], gA[i][g],                                         */
/* gB[i][g][a] = d_g B^a.  M^-1 = adj(M)/det(M); a particle with             */
/* det(M) <= 1e-12 tr(M)^3 is singular: its outputs are NaN.                 */
/* ------------------------------------------------------------------------ */
static double det3(const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

static void inv3(const double M[3][3], double det, double R[3][3]) {
    R[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
    R[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
    R[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
    R[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
    R[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
    R[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
    R[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
    R[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
    R[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
}

int orc_corrections(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *V, double L,
                    const int64_t *sub, int64_t nsub, int brute, double *A, double *B, double *gA, double *gB,
                    int64_t *nsing, int64_t *npairs) {
    double hmax = max_h_gas(n, species, h);
    if (n < 0 || L <= 0 || !(2.0 * hmax < 0.5 * L)) return ORC_EBOX;
    uint8_t *gmask = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gmask, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, brute)) { free(gmask); return ORC_ENOMEM; }
    int64_t pairs = 0; /* in-range pairs with i != j */
    int64_t singular = 0;
    FOR_EACH_I(sub, nsub, n, {
        if (species[i] != 0) {
            A[i] = 0.0;
            for (int c = 0; c < 3; ++c) { B[3 * i + c] = 0.0; gA[3 * i + c] = 0.0; }
            for (int c = 0; c < 9; ++c) gB[9 * i + c] = 0.0;
            continue;
        }
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double m0 = 0.0, m1[3] = {0}, m2[3][3] = {{0}};
        double dm0[3] = {0}, dm1[3][3] = {{0}}, dm2[3][3][3] = {{{0}}}; /* dm1[g][a], dm2[g][a][b] */
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double x[3];
            min_image(&pos[3 * i], &pos[3 * j], L, x); /* x = x_ij */
            double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            if (j != i) ++pairs;
            double W, dWr;
            wendland(sqrt(r2), hij, &W, &dWr);
            double dW[3] = {dWr * x[0], dWr * x[1], dWr * x[2]};
            double Vj = V[j];
            m0 += Vj * W;
            for (int a = 0; a < 3; ++a) {
                m1[a] += Vj * W * x[a];
                for (int b = 0; b < 3; ++b) m2[a][b] += Vj * W * x[a] * x[b];
            }
            for (int g = 0; g < 3; ++g) {
                dm0[g] += Vj * dW[g];
                for (int a = 0; a < 3; ++a) {
                    dm1[g][a] += Vj * ((a == g ? W : 0.0) + x[a] * dW[g]);
                    for (int b = 0; b < 3; ++b)
                        dm2[g][a][b] += Vj * ((a == g ? x[b] * W : 0.0) + (b == g ? x[a] * W : 0.0) + x[a] * x[b] * dW[g]);
                }
            }
        }
        double det = det3(m2);
        double tr = m2[0][0] + m2[1][1] + m2[2][2];
        if (!(det > 1e-12 * tr * tr * tr)) {
            _Pragma("omp atomic") ++singular;
            A[i] = NAN;
            for (int c = 0; c < 3; ++c) { B[3 * i + c] = NAN; gA[3 * i + c] = NAN; }
            for (int c = 0; c < 9; ++c) gB[9 * i + c] = NAN;
            continue;
        }
        double Mi[3][3];
        inv3(m2, det, Mi);
        double Bv[3];
        for (int a = 0; a < 3; ++a) Bv[a] = -(Mi[a][0] * m1[0] + Mi[a][1] * m1[1] + Mi[a][2] * m1[2]);
        double Av = 1.0 / (m0 + Bv[0] * m1[0] + Bv[1] * m1[1] + Bv[2] * m1[2]);
        A[i] = Av;
        for (int a = 0; a < 3; ++a) B[3 * i + a] = Bv[a];
        for (int g = 0; g < 3; ++g) {
            /* t = d_g m1 + (d_g M) B */
            double tv[3];
            double BdmB = 0.0, Bdm1 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double dMB = dm2[g][a][0] * Bv[0] + dm2[g][a][1] * Bv[1] + dm2[g][a][2] * Bv[2];
                tv[a] = dm1[g][a] + dMB;
                BdmB += Bv[a] * dMB;
                Bdm1 += Bv[a] * dm1[g][a];
            }
            gA[3 * i + g] = -Av * Av * (dm0[g] + 2.0 * Bdm1 + BdmB);
            for (int a = 0; a < 3; ++a)
                gB[9 * i + 3 * g + a] = -(Mi[a][0] * tv[0] + Mi[a][1] * tv[1] + Mi[a][2] * tv[2]);
        }
    });
    cells_free(&cl);
    free(gmask);
    if (nsing) *nsing = singular;
    if (npairs) *npairs = pairs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Acceleration + Energy (Sec. 5: "calculates the momentum derivative" and   */
/* "solves the derivative of the internal energy").  Paper silent; CRKSPH    */
/* reading with an unlimited Monaghan viscosity and an equal energy split:   */
/*   P = (gamma-1) rho u,  c = sqrt(gamma (gamma-1) u)                       */
/*   grad_i W^R_ij = gA_i (1 + B_i.x) W + A_i (gB_i.x + B_i) W               */
/*                   + A_i (1 + B_i.x) grad_i W,       x = x_ij              */
/*   (gB_i.x)_g = sum_a d_g B_i^a x^a                                         */
/*   grad_j W^R_ji: the same with i <-> j and x -> x_ji = -x_ij               */
/*   mu = h_ij (v_ij.x)/(r^2 + eta2 h_ij^2) if v_ij.x < 0 else 0             */
/*   Q  = rhobar (-alpha cbar mu + beta mu^2)   (arithmetic means)           */
/*   f_ij = -1/2 V_i V_j (P_i + P_j + Q)(grad_i W^R_ij - grad_j W^R_ji)       */
/*   m_i dv_i/dt = sum_j f_ij,   m_i du_i/dt = -1/2 sum_j (v_i - v_j).f_ij    */
/* f_ij = -f_ji, so momentum and total energy are conserved pair by pair.    */
/*                                                                          */
/* Limited viscosity (dvg != NULL; the Extras velocity gradients feed it,   */
/* paper silent on the form).  Both velocities are reconstructed linearly to */
/* the pair midpoint before mu is formed, with a van Leer limiter on the     */
/* gradients projected on the pair direction:                               */
/*   s_i = (dv_i) x,  s_j = (dv_j) x   ((dv)[a][b] = d v^a / d x^b)          */
/*   r = (x.s_i)/(x.s_j)  (0 if x.s_j = 0),  phi = 4r/(1+r)^2 if r > 0 else 0 */
/*   v*_ij = v_ij - phi/2 (s_i + s_j)  replaces v_ij in mu                   */
/* phi and v*_ij.x are unchanged under i <-> j, so Q_ij = Q_ji and the       */
/* conservation is kept; a linear velocity field with its exact gradient     */
/* gives v*_ij = 0 (no viscosity in a smooth shear or compression).  The     */
/* work term keeps the true v_ij.                                            */
/* ------------------------------------------------------------------------ */
static void grad_WR(const double x[3], double W, double dWr, double A, const double *B, const double *gA,
                    const double *gB, double out[3]) {
    double Bx = B[0] * x[0] + B[1] * x[1] + B[2] * x[2];
    for (int g = 0; g < 3; ++g) {
        double gBx = gB[3 * g] * x[0] + gB[3 * g + 1] * x[1] + gB[3 * g + 2] * x[2];
        out[g] = gA[g] * (1.0 + Bx) * W + A * (gBx + B[g]) * W + A * (1.0 + Bx) * dWr * x[g];
    }
}

/* ------------------------------------------------------------------------ */
/* Compatible energy split (Sec. 5: Acceleration and Energy are separate    */
/* kernels; Sec. 5.4: each is called twice per timestep).  Paper silent; the */
/* reading is the compatible differencing of the thermal energy: the work a */
/* pair's force does on the time-centred velocities v* is returned to the   */
/* pair as heat,                                                             */
/*   dE_ij = -f_ij.(v*_i - v*_j)   (= dE_ji, since f_ji = -f_ij),            */
/* and is shared asymmetrically so that it drives the two particles toward  */
/* thermal equilibrium (heating favours the colder one, cooling the hotter): */
/*   w_ij = 1/2 (1 + sgn(dE_ij) (u_j - u_i) / (|u_j - u_i| + (u_i + u_j)/2)) */
/*   with w_ij = 1/2 when u_i = u_j;  w_ij + w_ji = 1,  0 < w_ij < 1,       */
/*   m_i du_i/dt = sum_j w_ij dE_ij.                                         */
/* Summed over particles: sum_i m_i du_i = -sum_i m_i v*_i.dv_i, so a step  */
/* v1 = v + dt dv/dt with v* = (v + v1)/2 conserves kinetic plus thermal    */
/* energy exactly.  With u_i = u_j and v* = v it is the equal split.        */
/*                                                                          */
/* Signal velocity (the Courant timestep; Sec. 5.1: floating-point atomic    */
/* max).  Paper silent; Monaghan's pair signal speed over gas j in range,   */
/* including j = i:                                                          */
/*   vsig_i = max_j (c_i + c_j - sig_beta min(0, v_ij.x_ij / r_ij))          */
/*   (the j = i term is 2 c_i).                                              */
/* ------------------------------------------------------------------------ */
static double energy_share(double ui, double uj, double dE) {
    if (ui == uj) return 0.5;
    double t = (uj - ui) / (fabs(uj - ui) + 0.5 * (ui + uj));
    return 0.5 * (1.0 + (dE > 0.0 ? t : (dE < 0.0 ? -t : 0.0)));
}

double orc_energy_share(double ui, double uj, double dE) { return energy_share(ui, uj, dE); }

static int hydro_impl(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m,
                      const double *v, const double *u, const double *V, const double *rho, const double *A,
                      const double *B, const double *gA, const double *gB, const double *dvg, const double *vstar,
                      double sig_beta, double L, double gamma, double alpha, double beta, double eta2,
                      const int64_t *sub, int64_t nsub, int brute, double *dvdt, double *dudt, double *vsig,
                      int64_t *npairs) {
    double hmax = max_h_gas(n, species, h);
    if (n < 0 || L <= 0 || !(2.0 * hmax < 0.5 * L)) return ORC_EBOX;
    uint8_t *gmask = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gmask, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, brute)) { free(gmask); return ORC_ENOMEM; }
    int64_t pairs = 0;
    FOR_EACH_I(sub, nsub, n, {
        if (species[i] != 0) {
            for (int c = 0; c < 3; ++c) dvdt[3 * i + c] = 0.0;
            dudt[i] = 0.0;
            if (vsig) vsig[i] = 0.0;
            continue;
        }
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double Pi = (gamma - 1.0) * rho[i] * u[i];
        double ci = sqrt(gamma * (gamma - 1.0) * u[i]);
        double F[3] = {0.0, 0.0, 0.0}, E = 0.0, S = 0.0;
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double x[3];
            min_image(&pos[3 * i], &pos[3 * j], L, x); /* x_ij */
            double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            if (j != i) ++pairs;
            double W, dWr;
            wendland(sqrt(r2), hij, &W, &dWr);
            double xm[3] = {-x[0], -x[1], -x[2]};
            double gi[3], gj[3];
            grad_WR(x, W, dWr, A[i], &B[3 * i], &gA[3 * i], &gB[9 * i], gi);
            grad_WR(xm, W, dWr, A[j], &B[3 * j], &gA[3 * j], &gB[9 * j], gj);
            double Pj = (gamma - 1.0) * rho[j] * u[j];
            double cj = sqrt(gamma * (gamma - 1.0) * u[j]);
            double vij[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
            double vs[3] = {vij[0], vij[1], vij[2]}; /* velocity difference seen by the viscosity */
            if (dvg) {
                double si[3], sj[3];
                for (int a = 0; a < 3; ++a) {
                    si[a] = dvg[9 * i + 3 * a] * x[0] + dvg[9 * i + 3 * a + 1] * x[1] + dvg[9 * i + 3 * a + 2] * x[2];
                    sj[a] = dvg[9 * j + 3 * a] * x[0] + dvg[9 * j + 3 * a + 1] * x[1] + dvg[9 * j + 3 * a + 2] * x[2];
                }
                double ai = x[0] * si[0] + x[1] * si[1] + x[2] * si[2];
                double aj = x[0] * sj[0] + x[1] * sj[1] + x[2] * sj[2];
                double rr = aj != 0.0 ? ai / aj : 0.0;
                double phi = rr > 0.0 ? 4.0 * rr / ((1.0 + rr) * (1.0 + rr)) : 0.0;
                for (int a = 0; a < 3; ++a) vs[a] = vij[a] - 0.5 * phi * (si[a] + sj[a]);
            }
            double vx = vs[0] * x[0] + vs[1] * x[1] + vs[2] * x[2];
            double mu = vx < 0.0 ? hij * vx / (r2 + eta2 * hij * hij) : 0.0;
            double Q = 0.5 * (rho[i] + rho[j]) * (-alpha * 0.5 * (ci + cj) * mu + beta * mu * mu);
            double pre = -0.5 * V[i] * V[j] * (Pi + Pj + Q);
            double f[3];
            for (int c = 0; c < 3; ++c) f[c] = pre * (gi[c] - gj[c]);
            for (int c = 0; c < 3; ++c) F[c] += f[c];
            if (vstar) {
                double dE = -((vstar[3 * i] - vstar[3 * j]) * f[0] + (vstar[3 * i + 1] - vstar[3 * j + 1]) * f[1] +
                              (vstar[3 * i + 2] - vstar[3 * j + 2]) * f[2]);
                E += energy_share(u[i], u[j], dE) * dE;
            } else {
                E += -0.5 * (vij[0] * f[0] + vij[1] * f[1] + vij[2] * f[2]);
            }
            if (vsig) {
                double w = r2 > 0.0 ? (vij[0] * x[0] + vij[1] * x[1] + vij[2] * x[2]) / sqrt(r2) : 0.0;
                double sij = ci + cj - sig_beta * (w < 0.0 ? w : 0.0);
                if (sij > S) S = sij;
            }
        }
        for (int c = 0; c < 3; ++c) dvdt[3 * i + c] = F[c] / m[i];
        dudt[i] = E / m[i];
        if (vsig) vsig[i] = S;
    });
    cells_free(&cl);
    free(gmask);
    if (npairs) *npairs = pairs;
    return ORC_OK;
}

int orc_hydro(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m, const double *v,
              const double *u, const double *V, const double *rho, const double *A, const double *B, const double *gA,
              const double *gB, const double *dvg, double L, double gamma, double alpha, double beta, double eta2,
              const int64_t *sub, int64_t nsub, int brute, double *dvdt, double *dudt, int64_t *npairs) {
    return hydro_impl(n, pos, species, h, m, v, u, V, rho, A, B, gA, gB, dvg, NULL, 0.0, L, gamma, alpha, beta, eta2,
                      sub, nsub, brute, dvdt, dudt, NULL, npairs);
}

/* the same pair force with the compatible energy split on v* (vstar, NULL:   */
/* the equal split on v) and the signal velocity (vsig, may be NULL)          */
int orc_hydro_compatible(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m,
                         const double *v, const double *u, const double *V, const double *rho, const double *A,
                         const double *B, const double *gA, const double *gB, const double *dvg, const double *vstar,
                         double sig_beta, double L, double gamma, double alpha, double beta, double eta2,
                         const int64_t *sub, int64_t nsub, int brute, double *dvdt, double *dudt, double *vsig,
                         int64_t *npairs) {
    return hydro_impl(n, pos, species, h, m, v, u, V, rho, A, B, gA, gB, dvg, vstar, sig_beta, L, gamma, alpha, beta,
                      eta2, sub, nsub, brute, dvdt, dudt, vsig, npairs);
}

/* ------------------------------------------------------------------------ */
/* Extras (Sec. 5: "evaluates the density and state gradients").  Paper      */
/* silent; CRKSPH reading, over gas j including j = i, with the corrected    */
/* kernel W^R_ij = A_i (1 + B_i.x_ij) W_ij and its evaluation-point gradient */
/* grad_i W^R_ij (as in orc_hydro):                                          */
/*   rhoR_i = sum_j m_j W^R_ij                     (corrected-kernel density) */
/*   dv_i[3a + b] = sum_j V_j (v_j^a - v_i^a) (grad_i W^R_ij)^b  = dv^a/dx^b */
/* The first reproduces a density rho0 exactly when m_j = rho0 V_j; the      */
/* second is exact for a linear velocity field.  Dark matter gets zeros.    */
/* ------------------------------------------------------------------------ */
int orc_extras(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m, const double *v,
               const double *V, const double *A, const double *B, const double *gA, const double *gB, double L,
               const int64_t *sub, int64_t nsub, int brute, double *rhoR, double *dvg, int64_t *npairs) {
    double hmax = max_h_gas(n, species, h);
    if (n < 0 || L <= 0 || !(2.0 * hmax < 0.5 * L)) return ORC_EBOX;
    uint8_t *gmask = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gmask, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, brute)) { free(gmask); return ORC_ENOMEM; }
    int64_t pairs = 0;
    FOR_EACH_I(sub, nsub, n, {
        if (species[i] != 0) {
            rhoR[i] = 0.0;
            for (int c = 0; c < 9; ++c) dvg[9 * i + c] = 0.0;
            continue;
        }
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double rho = 0.0, G[9] = {0.0};
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double x[3];
            min_image(&pos[3 * i], &pos[3 * j], L, x); /* x_ij */
            double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            if (j != i) ++pairs;
            double W, dWr;
            wendland(sqrt(r2), hij, &W, &dWr);
            double Bx = B[3 * i] * x[0] + B[3 * i + 1] * x[1] + B[3 * i + 2] * x[2];
            rho += m[j] * A[i] * (1.0 + Bx) * W;
            double g[3];
            grad_WR(x, W, dWr, A[i], &B[3 * i], &gA[3 * i], &gB[9 * i], g);
            for (int a = 0; a < 3; ++a) {
                double dva = v[3 * j + a] - v[3 * i + a];
                for (int b = 0; b < 3; ++b) G[3 * a + b] += V[j] * dva * g[b];
            }
        }
        rhoR[i] = rho;
        for (int c = 0; c < 9; ++c) dvg[9 * i + c] = G[c];
    });
    cells_free(&cl);
    free(gmask);
    if (npairs) *npairs = pairs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Geometry adjoint (reverse mode of orc_geometry at fixed h; not in the     */
/* paper).  With S_i = sum_j W_ij, V_i = 1/S_i, rho_i = m_i S_i and          */
/* cotangents rhobar, Vbar (gas only):                                       */
/*   Sbar_i  = rhobar_i m_i - Vbar_i / S_i^2                                  */
/*   dL/dm_i = rhobar_i S_i                                                   */
/*   dL/dx_k = sum_j (Sbar_k + Sbar_j) grad_k W_kj                            */
/* Vbar may be NULL (zero).  Dark-matter entries get 0.                      */
/* ------------------------------------------------------------------------ */
int orc_geometry_adjoint(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m,
                         const double *rhobar, const double *Vbar, double L, const int64_t *sub, int64_t nsub,
                         int brute, double *gx, double *gm) {
    double *V = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *Sbar = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!V || !rho || !Sbar) { free(V); free(rho); free(Sbar); return ORC_ENOMEM; }
    int rc = orc_geometry(n, pos, species, h, m, L, NULL, 0, brute, V, rho, NULL);
    if (rc) { free(V); free(rho); free(Sbar); return rc; }
    for (int64_t i = 0; i < n; ++i) {
        if (species[i] != 0) continue;
        double S = 1.0 / V[i];
        Sbar[i] = rhobar[i] * m[i] - (Vbar ? Vbar[i] / (S * S) : 0.0);
    }
    double hmax = max_h_gas(n, species, h);
    uint8_t *gmask = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gmask, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, brute)) {
        free(gmask); free(V); free(rho); free(Sbar);
        return ORC_ENOMEM;
    }
    int64_t pairs = 0; /* unused here; the loop macro reduces into it */
    (void)pairs;
    FOR_EACH_I(sub, nsub, n, {
        if (species[i] != 0) {
            for (int c = 0; c < 3; ++c) gx[3 * i + c] = 0.0;
            gm[i] = 0.0;
            continue;
        }
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        double g[3] = {0.0, 0.0, 0.0};
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double x[3];
            min_image(&pos[3 * i], &pos[3 * j], L, x);
            double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            double W, dWr;
            wendland(sqrt(r2), hij, &W, &dWr);
            for (int c = 0; c < 3; ++c) g[c] += (Sbar[i] + Sbar[j]) * dWr * x[c];
        }
        for (int c = 0; c < 3; ++c) gx[3 * i + c] = g[c];
        gm[i] = rhobar[i] / V[i];
    });
    cells_free(&cl);
    free(gmask); free(V); free(rho); free(Sbar);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Leaves.  Sec. 3.1 names the RCB tree; Sec. 5.3 runs kernels over leaf     */
/* pairs.  The paper fixes none of the tie rules; this reading makes every   */
/* integer result unique:                                                    */
/*  chaining mesh: cell c = min(nc-1, floor(x nc / L)) per axis, leaf id      */
/*    (cx nc + cy) nc + cz (empty cells are empty leaves);                    */
/*  RCB: split the longest extent hi - lo of the node's tight box (ties       */
/*    prefer x, then y), order members by (coordinate, original index), the   */
/*    left child takes the first floor(n/2); recurse while n > max_leaf;      */
/*    leaves numbered depth first, left before right;                         */
/*  inside each leaf: gas first, then dark matter, each by original index.    */
/* perm[p] = original index of the particle at leaf-order position p.        */
/* ------------------------------------------------------------------------ */
static const double *g_sort_pos;
static int g_sort_axis;
static const uint8_t *g_sort_species;

static int cmp_axis(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double xa = g_sort_pos[3 * a + g_sort_axis], xb = g_sort_pos[3 * b + g_sort_axis];
    if (xa < xb) return -1;
    if (xa > xb) return 1;
    return (a > b) - (a < b);
}

static int cmp_species_index(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    int sa = g_sort_species[a] != 0, sb = g_sort_species[b] != 0;
    if (sa != sb) return sa - sb;
    return (a > b) - (a < b);
}

int orc_leaves_mesh(int64_t n, const double *pos, const uint8_t *species, double L, int nc, int32_t *perm,
                    int32_t *leaf_start) {
    if (nc <= 0 || n < 0) return ORC_EINVAL;
    int64_t ncell = (int64_t)nc * nc * nc;
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!cell || !cnt) { free(cell); free(cnt); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double f = floor(pos[3 * i + a] * (double)nc / L);
            int ci = (int)f;
            if (ci > nc - 1) ci = nc - 1;
            if (ci < 0) ci = 0;
            c[a] = ci;
        }
        cell[i] = (int32_t)(((int64_t)c[0] * nc + c[1]) * nc + c[2]);
        cnt[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    for (int64_t c = 0; c <= ncell; ++c) leaf_start[c] = (int32_t)cnt[c];
    for (int64_t i = 0; i < n; ++i) perm[cnt[cell[i]]++] = (int32_t)i; /* index order within a cell */
    g_sort_species = species;
    for (int64_t c = 0; c < ncell; ++c)
        qsort(perm + leaf_start[c], (size_t)(leaf_start[c + 1] - leaf_start[c]), sizeof(int32_t), cmp_species_index);
    free(cell);
    free(cnt);
    return ORC_OK;
}

typedef struct {
    const double *pos;
    int max_leaf;
    int32_t *idx;
    int32_t *leaf_start;
    int64_t cap, nleaf;
} RcbState;

static void rcb_node(RcbState *st, int64_t lo, int64_t hi) {
    int64_t cnt = hi - lo;
    if (cnt <= st->max_leaf) {
        if (st->nleaf < st->cap) st->leaf_start[st->nleaf] = (int32_t)lo;
        st->nleaf++;
        qsort(st->idx + lo, (size_t)cnt, sizeof(int32_t), cmp_species_index);
        return;
    }
    double bl[3], bh[3];
    for (int a = 0; a < 3; ++a) { bl[a] = st->pos[3 * st->idx[lo] + a]; bh[a] = bl[a]; }
    for (int64_t t = lo; t < hi; ++t)
        for (int a = 0; a < 3; ++a) {
            double x = st->pos[3 * st->idx[t] + a];
            if (x < bl[a]) bl[a] = x;
            if (x > bh[a]) bh[a] = x;
        }
    int axis = 0;
    double ext[3] = {bh[0] - bl[0], bh[1] - bl[1], bh[2] - bl[2]};
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    g_sort_axis = axis;
    qsort(st->idx + lo, (size_t)cnt, sizeof(int32_t), cmp_axis);
    int64_t mid = lo + cnt / 2;
    rcb_node(st, lo, mid);
    rcb_node(st, mid, hi);
}

/* leaf_start needs room for cap + 1 entries; *n_leaves gets the true count */
int orc_leaves_rcb(int64_t n, const double *pos, const uint8_t *species, int max_leaf, int32_t *perm,
                   int32_t *leaf_start, int64_t cap, int64_t *n_leaves) {
    if (max_leaf < 1 || n < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    *n_leaves = 0;
    if (n == 0) { leaf_start[0] = 0; return ORC_OK; }
    RcbState st = {pos, max_leaf, perm, leaf_start, cap, 0};
    g_sort_pos = pos;
    g_sort_species = species;
    rcb_node(&st, 0, n);
    *n_leaves = st.nleaf;
    if (st.nleaf <= cap) leaf_start[st.nleaf] = (int32_t)n;
    return st.nleaf <= cap ? ORC_OK : ORC_ENOMEM;
}

/* ------------------------------------------------------------------------ */
/* Leaf-pair lists (Sec. 5.3: work runs over pairs of leaves).  Reading:     */
/* per axis, the periodic gap between the leaves' tight boxes is             */
/*   min over s in {-L, 0, L} of max(0, (lo_b + s) - hi_a, (lo_a - hi_b) - s) */
/* and (a, b) is listed iff (gx^2 + gy^2) + gz^2 < cut^2, all in FP64.        */
/* Gravity: cut = r_c, both leaves non-empty.  Hydro: both leaves hold gas   */
/* and cut = 2 max(hmax_a, hmax_b) with hmax the largest gas h of a leaf.    */
/* Lists run over a (all leaves, or the subset asub) and b ascending,        */
/* a = b included.                                                           */
/* ------------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3], hmax; int64_t cnt, ngas; } LeafBox;

static double axis_gap(double loa, double hia, double lob, double hib, double L) {
    double best = INFINITY;
    const double sh[3] = {-L, 0.0, L};
    for (int k = 0; k < 3; ++k) {
        double s = sh[k];
        double t1 = (lob + s) - hia;
        double t2 = (loa - hib) - s;
        double g = t1 > t2 ? t1 : t2;
        if (g < 0.0) g = 0.0;
        if (g < best) best = g;
    }
    return best;
}

int orc_leaf_pairs(int64_t n_leaves, const int32_t *leaf_start, const int32_t *perm, const double *pos,
                   const uint8_t *species, const double *h, double L, int hydro, double rc, const int32_t *asub,
                   int64_t nasub, int32_t *ptr, int32_t *list, int64_t cap, int64_t *total) {
    LeafBox *bx = (LeafBox *)calloc((size_t)(n_leaves > 0 ? n_leaves : 1), sizeof(LeafBox));
    if (!bx) return ORC_ENOMEM;
    for (int64_t a = 0; a < n_leaves; ++a) {
        LeafBox *b = &bx[a];
        b->cnt = leaf_start[a + 1] - leaf_start[a];
        for (int c = 0; c < 3; ++c) { b->lo[c] = INFINITY; b->hi[c] = -INFINITY; }
        for (int32_t p = leaf_start[a]; p < leaf_start[a + 1]; ++p) {
            int32_t i = perm[p];
            for (int c = 0; c < 3; ++c) {
                if (pos[3 * i + c] < b->lo[c]) b->lo[c] = pos[3 * i + c];
                if (pos[3 * i + c] > b->hi[c]) b->hi[c] = pos[3 * i + c];
            }
            if (species[i] == 0) {
                b->ngas++;
                if (h[i] > b->hmax) b->hmax = h[i];
            }
        }
    }
    int64_t na = asub ? nasub : n_leaves;
    int64_t k = 0;
    for (int64_t ia = 0; ia < na; ++ia) {
        int64_t a = asub ? asub[ia] : ia;
        ptr[ia] = (int32_t)(k < cap ? k : cap);
        const LeafBox *A = &bx[a];
        if (A->cnt == 0 || (hydro && A->ngas == 0)) continue;
        for (int64_t b = 0; b < n_leaves; ++b) {
            const LeafBox *Bb = &bx[b];
            if (Bb->cnt == 0 || (hydro && Bb->ngas == 0)) continue;
            double cut = rc;
            if (hydro) cut = 2.0 * (A->hmax > Bb->hmax ? A->hmax : Bb->hmax);
            double gx = axis_gap(A->lo[0], A->hi[0], Bb->lo[0], Bb->hi[0], L);
            double gy = axis_gap(A->lo[1], A->hi[1], Bb->lo[1], Bb->hi[1], L);
            double gz = axis_gap(A->lo[2], A->hi[2], Bb->lo[2], Bb->hi[2], L);
            double d2 = (gx * gx + gy * gy) + gz * gz;
            if (d2 < cut * cut) {
                if (k < cap) list[k] = (int32_t)b;
                ++k;
            }
        }
    }
    ptr[na] = (int32_t)(k < cap ? k : cap);
    *total = k;
    free(bx);
    return k <= cap ? ORC_OK : ORC_ENOMEM;
}

/* ------------------------------------------------------------------------ */
/* Neighbour closure (test/benchmark helper): mark[j] = 1 for every j that is */
/* in range of some i with mark_in[i] != 0, and for those i themselves.       */
/* hydro != 0: gas pairs with r < h_i + h_j; else all pairs with r < rc.      */
/* ------------------------------------------------------------------------ */
int orc_mark_neighbours(int64_t n, const double *pos, const uint8_t *species, const double *h, double L, double rc,
                        int hydro, const uint8_t *mark_in, uint8_t *mark_out) {
    double hmax = max_h_gas(n, species, h);
    double cut = hydro ? 2.0 * hmax : rc;
    if (!(cut > 0.0) || !(cut < 0.5 * L)) return ORC_EBOX;
    uint8_t *gm = hydro ? gas_mask(n, species) : NULL;
    CellList cl;
    if (cells_build(&cl, n, pos, gm, L, cut, 0)) { free(gm); return ORC_ENOMEM; }
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cells_buffer_size(&cl));
    for (int64_t i = 0; i < n; ++i) mark_out[i] = mark_in[i];
    for (int64_t i = 0; i < n; ++i) {
        if (!mark_in[i] || (hydro && species[i] != 0)) continue;
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double d[3];
            min_image(&pos[3 * i], &pos[3 * j], L, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double c = hydro ? h[i] + h[j] : rc;
            if (r2 < c * c) mark_out[j] = 1;
        }
    }
    free(buf);
    cells_free(&cl);
    free(gm);
    return ORC_OK;
}

/* ======================================================================== */
/* Reverse mode of Corrections and of the hydro pair force (not in the     */
/* paper; the adjoints extend the gravity and geometry ones to the rest of  */
/* the forward chain).  Hand-written FP64 reverse mode of the forward       */
/* formulas above, pinned by central differences in tests/.                 */
/* ======================================================================== */

/* W, (dW/dr)/r and (d[(dW/dr)/r]/dr)/r of the Wendland C4 kernel:          */
/*   ddWr = 495/(256 pi h^7) 35 (1 - q/2)^4, so that grad (dWr) = ddWr x.   */
static void wendland2(double r, double h, double *W, double *dWr, double *ddWr) {
    double q = r / h;
    if (q >= 2.0) { *W = 0.0; *dWr = 0.0; *ddWr = 0.0; return; }
    wendland(r, h, W, dWr);
    double t = 1.0 - 0.5 * q;
    double h7 = h * h * h * h * h * h * h;
    *ddWr = 495.0 / (256.0 * PI) / h7 * 35.0 * t * t * t * t;
}

void orc_wendland2(int64_t n, const double *r, const double *h, double *W, double *dWr, double *ddWr) {
    for (int64_t i = 0; i < n; ++i) wendland2(r[i], h[i], &W[i], &dWr[i], &ddWr[i]);
}

/* moments of particle i (the sums of orc_corrections) */
typedef struct {
    double m0, m1[3], m2[3][3], dm0[3], dm1[3][3], dm2[3][3][3]; /* dm1[g][a], dm2[g][a][b] */
} Moments;

/* Cotangents of the moments from those of A, B, gA, gB (closed-form        */
/* reverse of orc_corrections' per-particle step; M = m2 is symmetric, so   */
/* M^-1 is too).                                                             */
static int moments_bar(const Moments *mo, double Abar, const double *Bbar_in, const double *gAbar,
                       const double *gBbar, Moments *mb) {
    memset(mb, 0, sizeof(*mb));
    double det = det3(mo->m2);
    double tr = mo->m2[0][0] + mo->m2[1][1] + mo->m2[2][2];
    if (!(det > 1e-12 * tr * tr * tr)) return 1;
    double Mi[3][3];
    inv3(mo->m2, det, Mi);
    double B[3], Bbar[3], Mibar[3][3] = {{0}};
    for (int a = 0; a < 3; ++a) B[a] = -(Mi[a][0] * mo->m1[0] + Mi[a][1] * mo->m1[1] + Mi[a][2] * mo->m1[2]);
    double A = 1.0 / (mo->m0 + B[0] * mo->m1[0] + B[1] * mo->m1[1] + B[2] * mo->m1[2]);
    for (int a = 0; a < 3; ++a) Bbar[a] = Bbar_in[a];
    double Atot = Abar;
    for (int g = 0; g < 3; ++g) {
        /* gB[g][a] = -(Mi t_g)_a with t_g = dm1[g] + dm2[g] B */
        double t[3], tb[3], K = mo->dm0[g];
        for (int a = 0; a < 3; ++a) {
            t[a] = mo->dm1[g][a];
            for (int b = 0; b < 3; ++b) t[a] += mo->dm2[g][a][b] * B[b];
            K += 2.0 * B[a] * mo->dm1[g][a];
            for (int b = 0; b < 3; ++b) K += B[a] * mo->dm2[g][a][b] * B[b];
        }
        const double *gb = &gBbar[3 * g];
        for (int a = 0; a < 3; ++a) tb[a] = -(Mi[a][0] * gb[0] + Mi[a][1] * gb[1] + Mi[a][2] * gb[2]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Mibar[a][b] += -gb[a] * t[b];
        for (int a = 0; a < 3; ++a) {
            mb->dm1[g][a] += tb[a];
            for (int b = 0; b < 3; ++b) {
                mb->dm2[g][a][b] += tb[a] * B[b];
                Bbar[b] += tb[a] * mo->dm2[g][a][b];
            }
        }
        /* gA[g] = -A^2 K_g, K_g = dm0[g] + 2 B.dm1[g] + B^T dm2[g] B */
        double Kb = -A * A * gAbar[g];
        Atot += -2.0 * A * K * gAbar[g];
        mb->dm0[g] += Kb;
        for (int a = 0; a < 3; ++a) {
            mb->dm1[g][a] += 2.0 * B[a] * Kb;
            Bbar[a] += 2.0 * mo->dm1[g][a] * Kb;
            for (int b = 0; b < 3; ++b) {
                Bbar[a] += (mo->dm2[g][a][b] + mo->dm2[g][b][a]) * B[b] * Kb;
                mb->dm2[g][a][b] += B[a] * B[b] * Kb;
            }
        }
    }
    /* A = 1/(m0 + B.m1) */
    double denb = -A * A * Atot;
    mb->m0 += denb;
    for (int a = 0; a < 3; ++a) {
        Bbar[a] += mo->m1[a] * denb;
        mb->m1[a] += B[a] * denb;
    }
    /* B = -Mi m1 */
    for (int a = 0; a < 3; ++a) {
        mb->m1[a] += -(Mi[0][a] * Bbar[0] + Mi[1][a] * Bbar[1] + Mi[2][a] * Bbar[2]);
        for (int b = 0; b < 3; ++b) Mibar[a][b] += -Bbar[a] * mo->m1[b];
    }
    /* Mi = M^-1: Mbar = -Mi^T Mibar Mi^T */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) s += Mi[c][a] * Mibar[c][d] * Mi[b][d];
            mb->m2[a][b] = -s;
        }
    return 0;
}

/* One pair's moment terms weighted by the moment cotangents mb, and their   */
/* gradient in the separation x = x_i - x_j, written out term by term from    */
/* the definitions in orc_corrections (per unit V_j):                          */
/*   m0: W    m1^a: W x^a    m2^ab: W x^a x^b    dm0_g: dW_g                   */
/*   dm1_g^a: d_ag W + x^a dW_g                                                */
/*   dm2_g^ab: d_ag x^b W + d_bg x^a W + x^a x^b dW_g                          */
/* with dW_g = (dW/dr/r) x_g, so dW/dx_c = dWr x_c and                        */
/* d(dW_g)/dx_c = ddWr x_c x_g + d_gc dWr, ddWr = (d[(dW/dr)/r]/dr)/r.          */
static double moment_term(const Moments *mb, const double x[3], double W, double dWr, double ddWr, double grad[3]) {
    double dW[3], gW[3], gdW[3][3];
    for (int g = 0; g < 3; ++g) {
        dW[g] = dWr * x[g];
        gW[g] = dWr * x[g];
        for (int c = 0; c < 3; ++c) gdW[g][c] = ddWr * x[c] * x[g] + (g == c ? dWr : 0.0);
    }
    double T = 0.0;
    for (int c = 0; c < 3; ++c) grad[c] = 0.0;
    /* m0 */
    T += mb->m0 * W;
    for (int c = 0; c < 3; ++c) grad[c] += mb->m0 * gW[c];
    for (int a = 0; a < 3; ++a) {
        /* m1^a */
        T += mb->m1[a] * W * x[a];
        for (int c = 0; c < 3; ++c) grad[c] += mb->m1[a] * (gW[c] * x[a] + (a == c ? W : 0.0));
        for (int b = 0; b < 3; ++b) {
            /* m2^ab */
            T += mb->m2[a][b] * W * x[a] * x[b];
            for (int c = 0; c < 3; ++c)
                grad[c] += mb->m2[a][b] *
                           (gW[c] * x[a] * x[b] + W * ((a == c ? x[b] : 0.0) + (b == c ? x[a] : 0.0)));
        }
    }
    for (int g = 0; g < 3; ++g) {
        /* dm0_g */
        T += mb->dm0[g] * dW[g];
        for (int c = 0; c < 3; ++c) grad[c] += mb->dm0[g] * gdW[g][c];
        for (int a = 0; a < 3; ++a) {
            /* dm1_g^a */
            T += mb->dm1[g][a] * ((a == g ? W : 0.0) + x[a] * dW[g]);
            for (int c = 0; c < 3; ++c)
                grad[c] += mb->dm1[g][a] *
                           ((a == g ? gW[c] : 0.0) + (a == c ? dW[g] : 0.0) + x[a] * gdW[g][c]);
            for (int b = 0; b < 3; ++b) {
                /* dm2_g^ab */
                const double w = mb->dm2[g][a][b];
                T += w * ((a == g ? x[b] * W : 0.0) + (b == g ? x[a] * W : 0.0) + x[a] * x[b] * dW[g]);
                for (int c = 0; c < 3; ++c)
                    grad[c] += w * ((a == g ? (b == c ? W : 0.0) + x[b] * gW[c] : 0.0) +
                                    (b == g ? (a == c ? W : 0.0) + x[a] * gW[c] : 0.0) +
                                    ((a == c ? x[b] : 0.0) + (b == c ? x[a] : 0.0)) * dW[g] + x[a] * x[b] * gdW[g][c]);
            }
        }
    }
    return T;
}

/* Reverse mode of orc_corrections for the cotangents Abar[n], Bbar[3n],     */
/* gAbar[3n], gBbar[9n] (layouts of its outputs): the gradient of            */
/*   L = sum_i Abar_i A_i + Bbar_i.B_i + gAbar_i.gA_i + gBbar_i:gB_i          */
/* in the positions (xbar[3n]) and volumes (Vbar[n]).  Pair (i, j) enters i's */
/* moments as V_j t(x_ij), so                                                 */
/*   xbar_k = sum_j V_j grad T_k(x_kj) - V_k grad T_j(x_jk),                  */
/*   Vbar_k = sum_j T_j(x_jk)   (j = k included),                            */
/* with T_i the moment terms weighted by i's moment cotangents.  A singular  */
/* particle contributes nothing and is counted.                              */
int orc_corrections_adjoint(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *V,
                            double L, const double *Abar, const double *Bbar, const double *gAbar, const double *gBbar,
                            double *xbar, double *Vbar, int64_t *nsing) {
    double hmax = max_h_gas(n, species, h);
    if (n < 0 || L <= 0 || !(2.0 * hmax < 0.5 * L)) return ORC_EBOX;
    uint8_t *gmask = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gmask, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, 0)) { free(gmask); return ORC_ENOMEM; }
    Moments *mb = (Moments *)calloc((size_t)(n > 0 ? n : 1), sizeof(Moments));
    const int64_t *nosub = NULL;
    int64_t pairs = 0, singular = 0;
    /* pass 1: every particle's moments and their cotangents */
    FOR_EACH_I(nosub, 0, n, {
        if (species[i] != 0) continue;
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        Moments mo;
        memset(&mo, 0, sizeof(mo));
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double x[3];
            min_image(&pos[3 * i], &pos[3 * j], L, x);
            double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            double W, dWr;
            wendland(sqrt(r2), hij, &W, &dWr);
            double Vj = V[j];
            mo.m0 += Vj * W;
            for (int a = 0; a < 3; ++a) {
                mo.m1[a] += Vj * W * x[a];
                for (int b = 0; b < 3; ++b) mo.m2[a][b] += Vj * W * x[a] * x[b];
            }
            for (int g = 0; g < 3; ++g) {
                mo.dm0[g] += Vj * dWr * x[g];
                for (int a = 0; a < 3; ++a) {
                    mo.dm1[g][a] += Vj * ((a == g ? W : 0.0) + x[a] * dWr * x[g]);
                    for (int b = 0; b < 3; ++b)
                        mo.dm2[g][a][b] +=
                            Vj * ((a == g ? x[b] * W : 0.0) + (b == g ? x[a] * W : 0.0) + x[a] * x[b] * dWr * x[g]);
                }
            }
        }
        if (moments_bar(&mo, Abar[i], &Bbar[3 * i], &gAbar[3 * i], &gBbar[9 * i], &mb[i])) {
            _Pragma("omp atomic") ++singular;
        }
    });
    /* pass 2: gather over pairs */
    FOR_EACH_I(nosub, 0, n, {
        for (int c = 0; c < 3; ++c) xbar[3 * i + c] = 0.0;
        Vbar[i] = 0.0;
        if (species[i] != 0) continue;
        int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
        for (int64_t t = 0; t < nc; ++t) {
            int64_t j = buf[t];
            double x[3], xm[3];
            min_image(&pos[3 * i], &pos[3 * j], L, x); /* x_ij */
            double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
            double hij = 0.5 * (h[i] + h[j]);
            if (!(r2 < 4.0 * hij * hij)) continue;
            double W, dWr, ddWr;
            wendland2(sqrt(r2), hij, &W, &dWr, &ddWr);
            for (int c = 0; c < 3; ++c) xm[c] = -x[c];
            double gi[3], gj[3];
            moment_term(&mb[i], x, W, dWr, ddWr, gi);
            double Tj = moment_term(&mb[j], xm, W, dWr, ddWr, gj);
            for (int c = 0; c < 3; ++c) xbar[3 * i + c] += V[j] * gi[c] - V[i] * gj[c];
            Vbar[i] += Tj;
        }
    });
    (void)pairs;
    cells_free(&cl);
    free(gmask);
    free(mb);
    if (nsing) *nsing = singular;
    return ORC_OK;
}

/* d G / d y contracted with c, for G_q(y) = gA_q (1 + B.y) W + A ((gB y)_q +  */
/* B_q) W + A (1 + B.y) dWr y_q (the corrected-kernel gradient of orc_hydro, */
/* (gB y)_q = sum_a gB[3q+a] y_a, W and dWr taken at |y|): out_p =           */
/* sum_q c_q dG_q/dy_p; and the cotangents of G's parameters, added to       */
/* Ab, Bb[3], gAb[3], gBb[9] (any of them may be NULL).                      */
static void grad_WR_vjp(const double y[3], double W, double dWr, double ddWr, double A, const double *B,
                        const double *gA, const double *gB, const double c[3], double out[3], double *Ab, double *Bb,
                        double *gAb, double *gBb) {
    double By = B[0] * y[0] + B[1] * y[1] + B[2] * y[2];
    double cy = c[0] * y[0] + c[1] * y[1] + c[2] * y[2];
    double cgA = c[0] * gA[0] + c[1] * gA[1] + c[2] * gA[2];
    double gBy[3], cgBy = 0.0, cB = c[0] * B[0] + c[1] * B[1] + c[2] * B[2];
    for (int q = 0; q < 3; ++q) {
        gBy[q] = gB[3 * q] * y[0] + gB[3 * q + 1] * y[1] + gB[3 * q + 2] * y[2];
        cgBy += c[q] * gBy[q];
    }
    for (int p = 0; p < 3; ++p) {
        double gBtc = c[0] * gB[p] + c[1] * gB[3 + p] + c[2] * gB[6 + p];
        out[p] = B[p] * (W * cgA + A * dWr * cy) + y[p] * (cgA * (1.0 + By) * dWr + A * dWr * (cgBy + cB) +
                                                         A * (1.0 + By) * ddWr * cy) +
                 A * W * gBtc + A * (1.0 + By) * dWr * c[p];
    }
    if (gAb)
        for (int q = 0; q < 3; ++q) gAb[q] += c[q] * (1.0 + By) * W;
    if (Ab) *Ab += W * (cgBy + cB) + (1.0 + By) * dWr * cy;
    if (Bb)
        for (int a = 0; a < 3; ++a) Bb[a] += y[a] * (W * cgA + A * dWr * cy) + A * W * c[a];
    if (gBb)
        for (int q = 0; q < 3; ++q)
            for (int a = 0; a < 3; ++a) gBb[3 * q + a] += c[q] * A * W * y[a];
}

/* Reverse mode of orc_hydro (Monaghan viscosity, equal split) for the        */
/* cotangents dvbar[3n], dubar[n] of dv/dt and du/dt, with every input of the */
/* pair force independent: out xbar[3n], vbar[3n], ubar[n], mbar[n],          */
/* Vbar[n], rhobar[n], Abar[n], Bbar[3n], gAbar[3n], gBbar[9n].  With        */
/* a_i = dvbar_i/m_i and b_i = dubar_i/m_i the loss is a sum over unordered   */
/* pairs i != j of l_ij = (a_i - a_j).f_ij + (b_i + b_j) e_ij,               */
/* e_ij = -1/2 v_ij.f_ij (f_ji = -f_ij, e_ji = e_ij; the self pair has        */
/* f_ii = 0 for every value of i's inputs), so particle k's cotangents are   */
/* the sums over its neighbours of dl_kj/d(k's inputs), plus                  */
/* mbar_k = -(a_k.F_k + b_k E_k)/m_k from dv = F/m and du = E/m.             */
int orc_hydro_adjoint(int64_t n, const double *pos, const uint8_t *species, const double *h, const double *m,
                      const double *v, const double *u, const double *V, const double *rho, const double *A,
                      const double *B, const double *gA, const double *gB, double L, double gamma, double alpha,
                      double beta, double eta2, const double *dvbar, const double *dubar, double *xbar, double *vbar,
                      double *ubar, double *mbar, double *Vbar, double *rhobar, double *Abar, double *Bbar,
                      double *gAbar, double *gBbar) {
    double hmax = max_h_gas(n, species, h);
    if (n < 0 || L <= 0 || !(2.0 * hmax < 0.5 * L)) return ORC_EBOX;
    uint8_t *gmask = gas_mask(n, species);
    CellList cl;
    if (cells_build(&cl, n, pos, gmask, L, 2.0 * hmax > 0 ? 2.0 * hmax : L, 0)) { free(gmask); return ORC_ENOMEM; }
    const int64_t *nosub = NULL;
    int64_t pairs = 0;
    FOR_EACH_I(nosub, 0, n, {
        double xb[3] = {0, 0, 0}, vb[3] = {0, 0, 0}, Vb = 0.0, Pb = 0.0, cb = 0.0, rb = 0.0;
        double Ab = 0.0, Bb[3] = {0, 0, 0}, gAb[3] = {0, 0, 0}, gBb[9] = {0};
        double F[3] = {0, 0, 0}, E = 0.0;
        if (species[i] == 0) {
            int64_t nc = cells_candidates(&cl, &pos[3 * i], buf);
            double Pi = (gamma - 1.0) * rho[i] * u[i];
            double ci = sqrt(gamma * (gamma - 1.0) * u[i]);
            double ai[3] = {dvbar[3 * i] / m[i], dvbar[3 * i + 1] / m[i], dvbar[3 * i + 2] / m[i]};
            double bi = dubar[i] / m[i];
            for (int64_t t = 0; t < nc; ++t) {
                int64_t j = buf[t];
                if (j == i) continue;
                double x[3], xm[3];
                min_image(&pos[3 * i], &pos[3 * j], L, x);
                double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                double hij = 0.5 * (h[i] + h[j]);
                if (!(r2 < 4.0 * hij * hij)) continue;
                double W, dWr, ddWr;
                wendland2(sqrt(r2), hij, &W, &dWr, &ddWr);
                for (int c = 0; c < 3; ++c) xm[c] = -x[c];
                double gi[3], gj[3];
                grad_WR(x, W, dWr, A[i], &B[3 * i], &gA[3 * i], &gB[9 * i], gi);
                grad_WR(xm, W, dWr, A[j], &B[3 * j], &gA[3 * j], &gB[9 * j], gj);
                double Pj = (gamma - 1.0) * rho[j] * u[j];
                double cj = sqrt(gamma * (gamma - 1.0) * u[j]);
                double vij[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
                double vx = vij[0] * x[0] + vij[1] * x[1] + vij[2] * x[2];
                double den = r2 + eta2 * hij * hij;
                double mu = vx < 0.0 ? hij * vx / den : 0.0;
                double rbar = 0.5 * (rho[i] + rho[j]), cbar = 0.5 * (ci + cj);
                double Q = rbar * (-alpha * cbar * mu + beta * mu * mu);
                double Pi_ = Pi + Pj + Q;
                double pre = -0.5 * V[i] * V[j] * Pi_;
                double d[3] = {gi[0] - gj[0], gi[1] - gj[1], gi[2] - gj[2]};
                double aj[3] = {dvbar[3 * j] / m[j], dvbar[3 * j + 1] / m[j], dvbar[3 * j + 2] / m[j]};
                double s = bi + dubar[j] / m[j];
                double z[3], D = 0.0;
                for (int c = 0; c < 3; ++c) {
                    z[c] = ai[c] - aj[c] - 0.5 * s * vij[c];
                    D += z[c] * d[c];
                    F[c] += pre * d[c];
                }
                E += -0.5 * pre * (vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2]);
                double Pib = -0.5 * V[i] * V[j] * D;
                Vb += -0.5 * V[j] * Pi_ * D;
                Pb += Pib;
                if (vx < 0.0) {
                    double mub = Pib * rbar * (-alpha * cbar + 2.0 * beta * mu);
                    rb += Pib * 0.5 * mu * (-alpha * cbar + beta * mu);
                    cb += Pib * rbar * mu * (-0.5 * alpha);
                    double vxb = mub * hij / den;
                    double r2b = -mub * hij * vx / (den * den);
                    for (int c = 0; c < 3; ++c) {
                        xb[c] += vxb * vij[c] + 2.0 * r2b * x[c];
                        vb[c] += vxb * x[c];
                    }
                }
                double dbar[3] = {pre * z[0], pre * z[1], pre * z[2]};
                for (int c = 0; c < 3; ++c) vb[c] += -0.5 * s * pre * d[c];
                double o1[3], o2[3];
                grad_WR_vjp(x, W, dWr, ddWr, A[i], &B[3 * i], &gA[3 * i], &gB[9 * i], dbar, o1, &Ab, Bb, gAb, gBb);
                grad_WR_vjp(xm, W, dWr, ddWr, A[j], &B[3 * j], &gA[3 * j], &gB[9 * j], dbar, o2, NULL, NULL, NULL,
                            NULL);
                for (int c = 0; c < 3; ++c) xb[c] += o1[c] + o2[c];
            }
            rb += Pb * (gamma - 1.0) * u[i];
            double ub = Pb * (gamma - 1.0) * rho[i] + (ci > 0.0 ? cb * gamma * (gamma - 1.0) / (2.0 * ci) : 0.0);
            ubar[i] = ub;
            mbar[i] = -(ai[0] * F[0] + ai[1] * F[1] + ai[2] * F[2] + bi * E) / m[i];
        } else {
            ubar[i] = 0.0;
            mbar[i] = 0.0;
        }
        for (int c = 0; c < 3; ++c) {
            xbar[3 * i + c] = xb[c];
            vbar[3 * i + c] = vb[c];
            Bbar[3 * i + c] = Bb[c];
            gAbar[3 * i + c] = gAb[c];
        }
        for (int c = 0; c < 9; ++c) gBbar[9 * i + c] = gBb[c];
        Vbar[i] = Vb;
        rhobar[i] = rb;
        Abar[i] = Ab;
    });
    (void)pairs;
    cells_free(&cl);
    free(gmask);
    return ORC_OK;
}
