// Short-range pair kernels of CRK-HACC (Sec. 5: Geometry, Corrections,
// Acceleration/Energy; Sec. 3.1: short-range gravity) and the two adjoints.
//
// Work decomposition (Sec. 5.3 runs the kernels over leaf pairs; the paper's
// "half-warp" lane split is prior art, not reused): one block per i-leaf, one
// warp per group of 32 consecutive i-particles of that leaf.  The warp walks
// the leaf's periodic images of j-leaves; every j-particle whose distance to
// the warp's i-box is below the cut is appended, already shifted into the
// i-leaf frame, to a per-warp buffer in shared memory (ballot compaction).
// Each full buffer is then swept by all 32 lanes, every lane accumulating the
// pair terms of its own i-particle (one-sided: no atomics, deterministic).
// Positions are FP32 relative to the i-leaf origin; sums are FP32 (Kahan-
// compensated for the moment sums); the CRK 3x3 inverse and the conservation
// reductions are FP64.
#include <cmath>
#include <mutex>

#include <type_traits>

#include "crk_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kCap = 64;                     // per-warp candidate buffer
constexpr int kCapPair = 128;                // per-warp candidate buffer of the packed sweeps (depth <= 96)
constexpr int kGroupImgCap = 128;            // image table of one i-leaf staged per warp in shared memory
// capacities of the one-pass gas lists (adaptive h keeps a gas particle near 58 neighbours;
// the largest lane list and group table seen in the clustered workloads are ~95 and ~360)
constexpr int kGasListCapRows = 128;
constexpr int kGasTableCap = 512;
constexpr float kSigmaW = 0.61548156588532f;  // 495 / (256 pi), Wendland C4 3-D normalisation

struct LeafView {
    const int32_t *leaf_start;
    const int32_t *leaf_ngas;
    const float *bbox;
    const float *hmax;
    const float4 *pos;
    const int32_t *kperm;
    const int32_t *img_start;
    const int32_t *img_cnt;
    const crk_image *img;
    int64_t n_leaves;
    int32_t *queue;  // persistent mode: next leaf to take (zeroed before launch); NULL = one block per leaf
    int korder;      // 1: the stage's per-particle arrays are in kernel order (no permutation)
    int depth;       // packed tiles sweeps: candidates compacted before each sweep (32, 64 or 96)
};

// Next i-leaf of this block: the grid-stride successor, or (persistent mode)
// the next unclaimed leaf of the work queue.  Block-uniform; every thread calls it.
__device__ __forceinline__ int64_t next_leaf(const LeafView &lv, int64_t cur, int64_t *slot) {
    if (!lv.queue) return cur < 0 ? (int64_t)blockIdx.x : cur + gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(lv.queue, 1);
    __syncthreads();
    return *slot;
}

// Next group of this warp (warp-granular work: one warp per group of 32
// consecutive kernel-order particles of one leaf): the grid-stride successor,
// or (persistent mode) the next unclaimed group of the work queue.  Warp-uniform.
__device__ __forceinline__ int64_t next_group(const LeafView &lv, int64_t cur, int lane) {
    if (!lv.queue) return cur < 0 ? (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5) : cur + (int64_t)gridDim.x * kWarps;
    int g = 0;
    if (lane == 0) g = atomicAdd(lv.queue, 1);
    return __shfl_sync(CRK_FULL_MASK, g, 0);
}

// index of kernel-order position q in the stage's per-particle arrays
__device__ __forceinline__ int32_t stage_index(const LeafView &lv, int q) { return lv.korder ? q : lv.kperm[q]; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Wendland C4 with support 2h: W and (dW/dr)/r at distance^2 r2, h = hij.
__device__ __forceinline__ void wendland(float r2, float hij, float &W, float &dWr) {
    float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    float ih = __fdividef(1.0f, hij);
    float q = r * ih;
    float t = fmaxf(1.0f - 0.5f * q, 0.0f);
    float t2 = t * t;
    float t5 = t2 * t2 * t;
    float ih2 = ih * ih;
    float ih3 = ih2 * ih;
    float n3 = kSigmaW * ih3;
    W = n3 * t5 * t * (1.0f + q * (3.0f + q * (35.0f / 12.0f)));
    dWr = n3 * ih2 * t5 * (-14.0f / 3.0f) * (1.0f + 2.5f * q);
}

// W, (dW/dr)/r and (d[(dW/dr)/r]/dr)/r = 495/(256 pi h^7) 35 (1 - q/2)^4 (zero beyond 2h)
__device__ __forceinline__ void wendland2(float r2, float hij, float &W, float &dWr, float &ddWr) {
    float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    float ih = __fdividef(1.0f, hij);
    float q = r * ih;
    float t = fmaxf(1.0f - 0.5f * q, 0.0f);
    float t2 = t * t;
    float t4 = t2 * t2;
    float ih2 = ih * ih;
    float n3 = kSigmaW * ih2 * ih;
    W = n3 * t4 * t2 * (1.0f + q * (3.0f + q * (35.0f / 12.0f)));
    dWr = n3 * ih2 * t4 * t * (-14.0f / 3.0f) * (1.0f + 2.5f * q);
    ddWr = n3 * ih2 * ih2 * 35.0f * t4;
}

// ------------------------------------------------------------------ stages
// Each stage defines Rec (one kernel-order record, also the shared-memory
// entry), gather (build Rec of particle p), box_cut (pruning radius of a
// candidate against the i-group box), I (per-lane state), init, interact and
// finish.

struct GravP {
    const float *m;
    float *a3;
    float rc2, eps2;
    float c[6];
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

struct GravStage {
    static constexpr bool kHalfWarp = true;
    static constexpr bool kGasOnly = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = true;
    using P = GravP;
    struct Rec {
        float x, y, z, m;
    };
    struct I {
        float ax, ay, az;
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t orig, float4 ps) { return {ps.x, ps.y, ps.z, p.m[orig]}; }
    static constexpr bool kCons = false;
    __device__ static float box_cut(const P &p, float, const Rec &) { return sqrtf(p.rc2); }
    __device__ static float leaf_cut(const P &p, float, float) { return sqrtf(p.rc2); }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) { s.ax = s.ay = s.az = 0.f; s.cnt = 0; }
    template <bool kCount>
    __device__ static void interact(const P &p, I &s, const Rec &ri, const Rec &rj) {
        float dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float rinv = rsqrtf(r2 + p.eps2);
        float r3 = rinv * rinv * rinv;
        float poly = fmaf(fmaf(fmaf(fmaf(fmaf(p.c[5], r2, p.c[4]), r2, p.c[3]), r2, p.c[2]), r2, p.c[1]), r2, p.c[0]);
        bool in = r2 < p.rc2;
        float f = in ? rj.m * (r3 - poly) : 0.0f;
        s.ax = fmaf(f, dx, s.ax);
        s.ay = fmaf(f, dy, s.ay);
        s.az = fmaf(f, dz, s.az);
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t orig, int64_t) {
        p.a3[orig] = s.ax;
        p.a3[p.n + orig] = s.ay;
        p.a3[2 * p.n + orig] = s.az;
    }
    __device__ static void finish_other(const P &, int32_t) {}

    // Two candidates per lane step with packed FP32 (f32x2) arithmetic: the
    // same operations and roundings per pair as interact, half the
    // instructions.  Rec2 holds two candidates field-interleaved, so each
    // field pair is one register pair.
    static constexpr bool kPair = true;
    struct __align__(16) Rec2 {
        float2 x, y, z, m;
    };
    struct I2 {
        float2 nx, ny, nz;  // -x_i, broadcast
        float2 ax, ay, az;
        int cnt;
    };
    __device__ static void put2(Rec2 *b, int c, const Rec &r) {
        float *d = reinterpret_cast<float *>(b + (c >> 1)) + (c & 1);
        d[0] = r.x; d[2] = r.y; d[4] = r.z; d[6] = r.m;
    }
    __device__ static Rec far_dummy(float fx, float fy, float fz) { return {fx, fy, fz, 0.0f}; }
    __device__ static void init2(const P &, I2 &s, const Rec &ri) {
        s.nx = make_float2(-ri.x, -ri.x);
        s.ny = make_float2(-ri.y, -ri.y);
        s.nz = make_float2(-ri.z, -ri.z);
        s.ax = s.ay = s.az = make_float2(0.f, 0.f);
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact2(const P &p, I2 &s, const Rec2 &rj) {
        const float2 dx = __fadd2_rn(rj.x, s.nx), dy = __fadd2_rn(rj.y, s.ny), dz = __fadd2_rn(rj.z, s.nz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const float2 t = __fadd2_rn(r2, make_float2(p.eps2, p.eps2));
        const float2 rinv = make_float2(rsqrtf(t.x), rsqrtf(t.y));
        const float2 r3 = __fmul2_rn(__fmul2_rn(rinv, rinv), rinv);
        // -P5(r^2) by Horner with negated coefficients (negation is exact)
        float2 np = __ffma2_rn(make_float2(-p.c[5], -p.c[5]), r2, make_float2(-p.c[4], -p.c[4]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[3], -p.c[3]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[2], -p.c[2]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[1], -p.c[1]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[0], -p.c[0]));
        const float2 g = __fmul2_rn(rj.m, __fadd2_rn(r3, np));
        const bool in0 = r2.x < p.rc2, in1 = r2.y < p.rc2;
        const float2 f = make_float2(in0 ? g.x : 0.0f, in1 ? g.y : 0.0f);
        s.ax = __ffma2_rn(f, dx, s.ax);
        s.ay = __ffma2_rn(f, dy, s.ay);
        s.az = __ffma2_rn(f, dz, s.az);
        if (kCount) s.cnt += (int)in0 + (int)in1;
    }
    // partial sums of one i from one leaf-pair tile (half-warp arms): added atomically
    __device__ static void flush(const P &p, const I &s, const Rec &, int32_t o) {
        atomicAdd(&p.a3[o], s.ax);
        atomicAdd(&p.a3[p.n + o], s.ay);
        atomicAdd(&p.a3[2 * p.n + o], s.az);
    }
    static void zero_outputs(const P &p, cudaStream_t st) { cudaMemsetAsync(p.a3, 0, sizeof(float) * 3 * p.n, st); }
    // adds the accumulators of lane ^ x (split sweeps: the lanes sharing one i)
    __device__ static void combine2(I2 &s, int x) {
        s.ax.x += __shfl_xor_sync(CRK_FULL_MASK, s.ax.x, x);
        s.ax.y += __shfl_xor_sync(CRK_FULL_MASK, s.ax.y, x);
        s.ay.x += __shfl_xor_sync(CRK_FULL_MASK, s.ay.x, x);
        s.ay.y += __shfl_xor_sync(CRK_FULL_MASK, s.ay.y, x);
        s.az.x += __shfl_xor_sync(CRK_FULL_MASK, s.az.x, x);
        s.az.y += __shfl_xor_sync(CRK_FULL_MASK, s.az.y, x);
        s.cnt += __shfl_xor_sync(CRK_FULL_MASK, s.cnt, x);
    }
    __device__ static void finish2(const P &p, I2 &s, int32_t orig) {
        p.a3[orig] = s.ax.x + s.ax.y;
        p.a3[p.n + orig] = s.ay.x + s.ay.y;
        p.a3[2 * p.n + orig] = s.az.x + s.az.y;
    }
};

struct GravAdjP {
    const float *m, *abar;
    float *gx3, *gm;
    float rc2, eps2;
    float c[6];
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

struct GravAdjStage {
    static constexpr bool kHalfWarp = true;
    static constexpr bool kGasOnly = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = true;
    using P = GravAdjP;
    struct __align__(16) Rec {
        float x, y, z, m;
        float bx, by, bz, pad;
    };
    struct I {
        float gx, gy, gz, gm;
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) {
        return {ps.x, ps.y, ps.z, p.m[o], p.abar[o], p.abar[p.n + o], p.abar[2 * p.n + o], 0.f};
    }
    static constexpr bool kCons = false;
    __device__ static float box_cut(const P &p, float, const Rec &) { return sqrtf(p.rc2); }
    __device__ static float leaf_cut(const P &p, float, float) { return sqrtf(p.rc2); }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) { s.gx = s.gy = s.gz = s.gm = 0.f; s.cnt = 0; }
    template <bool kCount>
    __device__ static void interact(const P &p, I &s, const Rec &ri, const Rec &rj) {
        float dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;  // d_ij = x_j - x_i
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float rinv = rsqrtf(r2 + p.eps2);
        float ri2 = rinv * rinv;
        float r3 = ri2 * rinv;
        float poly = fmaf(fmaf(fmaf(fmaf(fmaf(p.c[5], r2, p.c[4]), r2, p.c[3]), r2, p.c[2]), r2, p.c[1]), r2, p.c[0]);
        float dpoly = fmaf(fmaf(fmaf(fmaf(5.0f * p.c[5], r2, 4.0f * p.c[4]), r2, 3.0f * p.c[3]), r2, 2.0f * p.c[2]),
                           r2, p.c[1]);
        bool in = r2 < p.rc2;
        float g = in ? r3 - poly : 0.0f;
        float dg2 = in ? 2.0f * fmaf(-1.5f * r3, ri2, -dpoly) : 0.0f;
        float wx = ri.m * rj.bx - rj.m * ri.bx;
        float wy = ri.m * rj.by - rj.m * ri.by;
        float wz = ri.m * rj.bz - rj.m * ri.bz;
        float dw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
        float k = dg2 * dw;
        s.gx = fmaf(g, wx, fmaf(k, dx, s.gx));
        s.gy = fmaf(g, wy, fmaf(k, dy, s.gy));
        s.gz = fmaf(g, wz, fmaf(k, dz, s.gz));
        s.gm = fmaf(-g, fmaf(rj.bx, dx, fmaf(rj.by, dy, rj.bz * dz)), s.gm);
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        p.gx3[o] = s.gx;
        p.gx3[p.n + o] = s.gy;
        p.gx3[2 * p.n + o] = s.gz;
        p.gm[o] = s.gm;
    }
    __device__ static void finish_other(const P &, int32_t) {}

    // Two candidates per lane step with packed FP32 (f32x2) arithmetic (see GravStage).
    static constexpr bool kPair = true;
    struct __align__(16) Rec2 {
        float2 x, y, z, m;
        float2 bx, by, bz, pad;
    };
    struct I2 {
        float2 nx, ny, nz;         // -x_i, broadcast
        float2 mi, nbx, nby, nbz;  // m_i, -abar_i, broadcast
        // sum_j g w_j = m_i sum_j g abar_j - abar_i sum_j g m_j (w = m_i abar_j - m_j abar_i), so the
        // pair loop accumulates the two sums and k d; sg accumulates g (abar_j . d) (gm = -sg)
        float2 kx, ky, kz, s1x, s1y, s1z, s2, sg;
        int cnt;
    };
    __device__ static void put2(Rec2 *b, int c, const Rec &r) {
        float *d = reinterpret_cast<float *>(b + (c >> 1)) + (c & 1);
        d[0] = r.x; d[2] = r.y; d[4] = r.z; d[6] = r.m;
        d[8] = r.bx; d[10] = r.by; d[12] = r.bz; d[14] = 0.0f;
    }
    __device__ static Rec far_dummy(float fx, float fy, float fz) { return {fx, fy, fz, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}; }
    __device__ static void init2(const P &, I2 &s, const Rec &ri) {
        s.nx = make_float2(-ri.x, -ri.x);
        s.ny = make_float2(-ri.y, -ri.y);
        s.nz = make_float2(-ri.z, -ri.z);
        s.mi = make_float2(ri.m, ri.m);
        s.nbx = make_float2(-ri.bx, -ri.bx);
        s.nby = make_float2(-ri.by, -ri.by);
        s.nbz = make_float2(-ri.bz, -ri.bz);
        s.kx = s.ky = s.kz = s.s1x = s.s1y = s.s1z = s.s2 = s.sg = make_float2(0.f, 0.f);
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact2(const P &p, I2 &s, const Rec2 &rj) {
        const float2 dx = __fadd2_rn(rj.x, s.nx), dy = __fadd2_rn(rj.y, s.ny), dz = __fadd2_rn(rj.z, s.nz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const float2 t = __fadd2_rn(r2, make_float2(p.eps2, p.eps2));
        const float2 rinv = make_float2(rsqrtf(t.x), rsqrtf(t.y));
        const float2 ri2 = __fmul2_rn(rinv, rinv);
        const float2 r3 = __fmul2_rn(ri2, rinv);
        float2 np = __ffma2_rn(make_float2(-p.c[5], -p.c[5]), r2, make_float2(-p.c[4], -p.c[4]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[3], -p.c[3]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[2], -p.c[2]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[1], -p.c[1]));
        np = __ffma2_rn(np, r2, make_float2(-p.c[0], -p.c[0]));  // -P5
        // -2 P5' with doubled coefficients (scaling by 2 is exact)
        const float c5 = -10.0f * p.c[5], c4 = -8.0f * p.c[4], c3 = -6.0f * p.c[3], c2 = -4.0f * p.c[2];
        float2 ndp = __ffma2_rn(make_float2(c5, c5), r2, make_float2(c4, c4));
        ndp = __ffma2_rn(ndp, r2, make_float2(c3, c3));
        ndp = __ffma2_rn(ndp, r2, make_float2(c2, c2));
        ndp = __ffma2_rn(ndp, r2, make_float2(-2.0f * p.c[1], -2.0f * p.c[1]));
        const bool in0 = r2.x < p.rc2, in1 = r2.y < p.rc2;
        const float2 gv = __fadd2_rn(r3, np);
        // 2 g'(s) = 2 (-1.5 r^-5 - P5')
        const float2 dv = __ffma2_rn(__fmul2_rn(make_float2(-3.0f, -3.0f), r3), ri2, ndp);
        const float2 g = make_float2(in0 ? gv.x : 0.0f, in1 ? gv.y : 0.0f);
        const float2 dg2 = make_float2(in0 ? dv.x : 0.0f, in1 ? dv.y : 0.0f);
        // abar_j . d and -abar_i . d, then d . w = m_i (abar_j . d) - m_j (abar_i . d)
        const float2 dbj = __ffma2_rn(rj.bx, dx, __ffma2_rn(rj.by, dy, __fmul2_rn(rj.bz, dz)));
        const float2 ndbi = __ffma2_rn(s.nbx, dx, __ffma2_rn(s.nby, dy, __fmul2_rn(s.nbz, dz)));
        const float2 dw = __ffma2_rn(s.mi, dbj, __fmul2_rn(rj.m, ndbi));
        const float2 k = __fmul2_rn(dg2, dw);
        s.kx = __ffma2_rn(k, dx, s.kx);
        s.ky = __ffma2_rn(k, dy, s.ky);
        s.kz = __ffma2_rn(k, dz, s.kz);
        s.s1x = __ffma2_rn(g, rj.bx, s.s1x);
        s.s1y = __ffma2_rn(g, rj.by, s.s1y);
        s.s1z = __ffma2_rn(g, rj.bz, s.s1z);
        s.s2 = __ffma2_rn(g, rj.m, s.s2);
        s.sg = __ffma2_rn(g, dbj, s.sg);
        if (kCount) s.cnt += (int)in0 + (int)in1;
    }
    // partial sums of one i from one leaf-pair tile (half-warp arms): added atomically
    __device__ static void flush(const P &p, const I &s, const Rec &, int32_t o) {
        atomicAdd(&p.gx3[o], s.gx);
        atomicAdd(&p.gx3[p.n + o], s.gy);
        atomicAdd(&p.gx3[2 * p.n + o], s.gz);
        atomicAdd(&p.gm[o], s.gm);
    }
    static void zero_outputs(const P &p, cudaStream_t st) {
        cudaMemsetAsync(p.gx3, 0, sizeof(float) * 3 * p.n, st);
        cudaMemsetAsync(p.gm, 0, sizeof(float) * p.n, st);
    }
    // adds the accumulators of lane ^ x (split sweeps: the lanes sharing one i)
    __device__ static void combine2(I2 &s, int x) {
        float2 *acc[8] = {&s.kx, &s.ky, &s.kz, &s.s1x, &s.s1y, &s.s1z, &s.s2, &s.sg};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[q]->x += __shfl_xor_sync(CRK_FULL_MASK, acc[q]->x, x);
            acc[q]->y += __shfl_xor_sync(CRK_FULL_MASK, acc[q]->y, x);
        }
        s.cnt += __shfl_xor_sync(CRK_FULL_MASK, s.cnt, x);
    }
    __device__ static void finish2(const P &p, I2 &s, int32_t o) {
        const float mi = s.mi.x, nbx = s.nbx.x, nby = s.nby.x, nbz = s.nbz.x;
        const float s2 = s.s2.x + s.s2.y;
        p.gx3[o] = fmaf(mi, s.s1x.x + s.s1x.y, fmaf(nbx, s2, s.kx.x + s.kx.y));
        p.gx3[p.n + o] = fmaf(mi, s.s1y.x + s.s1y.y, fmaf(nby, s2, s.ky.x + s.ky.y));
        p.gx3[2 * p.n + o] = fmaf(mi, s.s1z.x + s.s1z.y, fmaf(nbz, s2, s.kz.x + s.kz.y));
        p.gm[o] = -(s.sg.x + s.sg.y);
    }
};

struct GeomP {
    const float *m;
    float *V, *rho;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

struct GeomStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = true;
    using P = GeomP;
    struct Rec {
        float x, y, z, h;
    };
    struct I {
        float s, c;
        int cnt;
    };
    __device__ static Rec gather(const P &, int32_t, float4 ps) { return {ps.x, ps.y, ps.z, ps.w}; }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) { s.s = s.c = 0.f; s.cnt = 0; }
    template <bool kCount>
    __device__ static void interact(const P &, I &s, const Rec &ri, const Rec &rj) {
        float dx = ri.x - rj.x, dy = ri.y - rj.y, dz = ri.z - rj.z;
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float W, dWr;
        wendland(r2, 0.5f * hs, W, dWr);
        kahan_add(s.s, s.c, in ? W : 0.0f);
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        float sum = s.s - s.c;
        float V = 1.0f / sum;
        p.V[o] = V;
        p.rho[o] = p.m[o] * sum;
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        p.V[o] = 0.f;
        p.rho[o] = 0.f;
    }
};

struct GeomAdjP {
    const float *m, *V, *rhobar, *Vbar;
    float *gx3, *gm;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

struct GeomAdjStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = true;
    using P = GeomAdjP;
    struct __align__(16) Rec {
        float x, y, z, h;
        float sbar, pad0, pad1, pad2;
    };
    struct I {
        float gx, gy, gz;
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) {
        float V = p.V[o];
        float sb = p.rhobar[o] * p.m[o] - (p.Vbar ? p.Vbar[o] * V * V : 0.0f);
        return {ps.x, ps.y, ps.z, ps.w, sb, 0.f, 0.f, 0.f};
    }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) { s.gx = s.gy = s.gz = 0.f; s.cnt = 0; }
    template <bool kCount>
    __device__ static void interact(const P &, I &s, const Rec &ri, const Rec &rj) {
        float dx = ri.x - rj.x, dy = ri.y - rj.y, dz = ri.z - rj.z;  // x_kj
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float W, dWr;
        wendland(r2, 0.5f * hs, W, dWr);
        float k = in ? (ri.sbar + rj.sbar) * dWr : 0.0f;
        s.gx = fmaf(k, dx, s.gx);
        s.gy = fmaf(k, dy, s.gy);
        s.gz = fmaf(k, dz, s.gz);
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        p.gx3[o] = s.gx;
        p.gx3[p.n + o] = s.gy;
        p.gx3[2 * p.n + o] = s.gz;
        p.gm[o] = p.rhobar[o] / p.V[o];
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        p.gx3[o] = 0.f;
        p.gx3[p.n + o] = 0.f;
        p.gx3[2 * p.n + o] = 0.f;
        p.gm[o] = 0.f;
    }
};

struct CorrP {
    const float *V;
    float *A, *B, *gA, *gB;
    int32_t *n_singular;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

struct CorrStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = true;
    using P = CorrP;
    struct __align__(16) Rec {
        float x, y, z, h;
        float V, pad0, pad1, pad2;
    };
    struct I {
        float m0, c0;
        float m1[3], c1[3];
        float m2[6], c2[6];  // xx xy xz yy yz zz
        // Gradient moments.  With w = V_j W and d_g(V_j W) = V_j dWr x_g, the g-derivatives of
        // m1_a and m2_ab are delta_ag m0 + V_j dWr x_a x_g and delta_ag m1_b + delta_bg m1_a +
        // V_j dWr x_a x_b x_g: only the symmetric dWr sums s2 (second order) and s3 (third
        // order) are accumulated, the delta terms come from m0 and m1 in finish.
        float dm0[3];
        float s2[6];   // xx xy xz yy yz zz
        float s3[10];  // xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
        int cnt;
    };
    // packed index of (a <= b) among xx xy xz yy yz zz
    __host__ __device__ static constexpr int idx2(int a, int b) { return a * (5 - a) / 2 + b; }
    // packed index of (a <= b <= c) among xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    __host__ __device__ static constexpr int idx3(int a, int b, int c) {
        return a == 0 ? (b == 0 ? c : (b == 1 ? 2 + c : 5)) : (a == 1 ? (b == 1 ? 5 + c : 8) : 9);
    }
    // the full gradient moments dm1[g][a] and dm2[g][ab] (ab packed) from m0, m1, s2, s3
    __device__ static void grad_moments(const I &s, double m0, const double m1[3], double dm1[3][3],
                                        double dm2[3][6]) {
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int g = 0; g < 3; ++g) {
            for (int a = 0; a < 3; ++a)
                dm1[g][a] = (a == g ? m0 : 0.0) + (double)s.s2[a < g ? idx2(a, g) : idx2(g, a)];
            for (int q = 0; q < 6; ++q) {
                int t0 = ia[q], t1 = ib[q], t2 = g;  // sort (a, b, g); a <= b already
                if (t2 < t1) { t2 = t1; t1 = g; }
                if (t1 < t0) { int u = t0; t0 = t1; t1 = u; }
                dm2[g][q] = (ia[q] == g ? m1[ib[q]] : 0.0) + (ib[q] == g ? m1[ia[q]] : 0.0) +
                            (double)s.s3[idx3(t0, t1, t2)];
            }
        }
    }
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) { return {ps.x, ps.y, ps.z, ps.w, p.V[o], 0, 0, 0}; }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) {
        s.m0 = s.c0 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) s.m1[a] = s.c1[a] = s.dm0[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) s.m2[a] = s.c2[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) s.s2[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 10; ++a) s.s3[a] = 0.f;
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact(const P &, I &s, const Rec &ri, const Rec &rj) {
        float x[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};  // x_ij
        float r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float W, dWr;
        wendland(r2, 0.5f * hs, W, dWr);
        float w = in ? rj.V * W : 0.0f;
        float vd = in ? rj.V * dWr : 0.0f;
        float wx[3] = {w * x[0], w * x[1], w * x[2]};
        float dW[3] = {vd * x[0], vd * x[1], vd * x[2]};  // V_j d_g W
        kahan_add(s.m0, s.c0, w);
#pragma unroll
        for (int a = 0; a < 3; ++a) kahan_add(s.m1[a], s.c1[a], wx[a]);
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        float xx[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            xx[q] = x[ia[q]] * x[ib[q]];
            kahan_add(s.m2[q], s.c2[q], wx[ia[q]] * x[ib[q]]);
            s.s2[q] = fmaf(xx[q], vd, s.s2[q]);
        }
#pragma unroll
        for (int g = 0; g < 3; ++g) s.dm0[g] += dW[g];
        // s3[abc] += x_a x_b (V_j dWr x_c) for a <= b <= c
        const int k3q[10] = {0, 0, 0, 1, 1, 2, 3, 3, 4, 5}, k3c[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
#pragma unroll
        for (int k = 0; k < 10; ++k) s.s3[k] = fmaf(xx[k3q[k]], dW[k3c[k]], s.s3[k]);
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        double m0 = (double)s.m0 - (double)s.c0;
        double m1[3], M[3][3];
        for (int a = 0; a < 3; ++a) m1[a] = (double)s.m1[a] - (double)s.c1[a];
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int q = 0; q < 6; ++q) {
            double v = (double)s.m2[q] - (double)s.c2[q];
            M[ia[q]][ib[q]] = v;
            M[ib[q]][ia[q]] = v;
        }
        double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        double tr = M[0][0] + M[1][1] + M[2][2];
        const int64_t n = p.n;
        if (!(det > 1e-12 * tr * tr * tr)) {
            const float nan = __int_as_float(0x7fc00000);
            p.A[o] = nan;
            for (int a = 0; a < 3; ++a) { p.B[a * n + o] = nan; p.gA[a * n + o] = nan; }
            for (int a = 0; a < 9; ++a) p.gB[a * n + o] = nan;
            if (p.n_singular) atomicAdd(p.n_singular, 1);
            return;
        }
        double Mi[3][3];
        double id = 1.0 / det;
        Mi[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) * id;
        Mi[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * id;
        Mi[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * id;
        Mi[1][0] = Mi[0][1];
        Mi[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * id;
        Mi[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * id;
        Mi[2][0] = Mi[0][2];
        Mi[2][1] = Mi[1][2];
        Mi[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * id;
        double B[3];
        for (int a = 0; a < 3; ++a) B[a] = -(Mi[a][0] * m1[0] + Mi[a][1] * m1[1] + Mi[a][2] * m1[2]);
        double A = 1.0 / (m0 + B[0] * m1[0] + B[1] * m1[1] + B[2] * m1[2]);
        p.A[o] = (float)A;
        for (int a = 0; a < 3; ++a) p.B[a * n + o] = (float)B[a];
        double dm1[3][3], dm2[3][6];
        grad_moments(s, m0, m1, dm1, dm2);
        for (int g = 0; g < 3; ++g) {
            double dM[3][3];
            for (int q = 0; q < 6; ++q) {
                dM[ia[q]][ib[q]] = dm2[g][q];
                dM[ib[q]][ia[q]] = dm2[g][q];
            }
            double t[3], BdMB = 0.0, Bdm1 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double dMB = dM[a][0] * B[0] + dM[a][1] * B[1] + dM[a][2] * B[2];
                t[a] = dm1[g][a] + dMB;
                BdMB += B[a] * dMB;
                Bdm1 += B[a] * dm1[g][a];
            }
            p.gA[g * n + o] = (float)(-A * A * ((double)s.dm0[g] + 2.0 * Bdm1 + BdMB));
            for (int a = 0; a < 3; ++a)
                p.gB[(3 * g + a) * n + o] = (float)(-(Mi[a][0] * t[0] + Mi[a][1] * t[1] + Mi[a][2] * t[2]));
        }
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        const int64_t n = p.n;
        p.A[o] = 0.f;
        for (int a = 0; a < 3; ++a) { p.B[a * n + o] = 0.f; p.gA[a * n + o] = 0.f; }
        for (int a = 0; a < 9; ++a) p.gB[a * n + o] = 0.f;
    }
};

// Reverse mode of Corrections (not in the paper).  Pair (i, j) enters i's
// moments as V_j t(x_ij); with i's moment cotangents (from those of A, B, dA,
// dB by the closed-form reverse of the per-particle step) the weighted terms
// are T_i(x) = S0_i(x) W + S1_i(x) dWr, S0 a quadratic and S1 a cubic
// polynomial in x.  The preparation sweep recomputes the moments and writes
// each particle's 29 polynomial coefficients
//   [c0, l0 (3), q0 (6: xx xy xz yy yz zz), l1 (3), q1 (6), k (10: xxx xxy xxz
//    xyy xyz xzz yyy yyz yzz zzz)],
// S0 = c0 + l0.x + q0(x), S1 = l1.x + q1(x) + k(x); the gradient sweep gathers
//   xbar_i = sum_j V_j grad T_i(x_ij) - V_i grad T_j(x_ji),
//   Vbar_i = sum_j T_j(x_ji)          (j = i included).
constexpr int kCorrCoef = 29;

struct CorrAdjP : CorrP {
    const float *Abar, *Bbar, *gAbar, *gBbar;  // cotangents: A [n], B [3][n], dA [3][n], dB [9][n] (3g+a)
    float *coef;                               // out: [29][n] (kernel order when korder, else caller)
};

struct CorrAdjPrepStage : CorrStage {
    static constexpr bool kAllVariants = false;
    using P = CorrAdjP;
    // The preparation sweep accumulates the gradient moments in full (30 sums, not the forward's
    // symmetric s2/s3): with its FP64 finish the symmetric form measured slower here.
    struct I {
        float m0, c0;
        float m1[3], c1[3];
        float m2[6], c2[6];  // xx xy xz yy yz zz
        float dm0[3];
        float dm1[9];   // [g][a]
        float dm2[18];  // [g][ab]
        int cnt;
    };
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) {
        s.m0 = s.c0 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) s.m1[a] = s.c1[a] = s.dm0[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 6; ++a) s.m2[a] = s.c2[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 9; ++a) s.dm1[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 18; ++a) s.dm2[a] = 0.f;
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact(const P &, I &s, const Rec &ri, const Rec &rj) {
        float x[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};  // x_ij
        float r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float W, dWr;
        wendland(r2, 0.5f * hs, W, dWr);
        float w = in ? rj.V * W : 0.0f;
        float vd = in ? rj.V * dWr : 0.0f;
        float wx[3] = {w * x[0], w * x[1], w * x[2]};
        float dW[3] = {vd * x[0], vd * x[1], vd * x[2]};  // V_j d_g W
        kahan_add(s.m0, s.c0, w);
#pragma unroll
        for (int a = 0; a < 3; ++a) kahan_add(s.m1[a], s.c1[a], wx[a]);
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        float xx[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            xx[q] = x[ia[q]] * x[ib[q]];
            kahan_add(s.m2[q], s.c2[q], wx[ia[q]] * x[ib[q]]);
        }
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            s.dm0[g] += dW[g];
#pragma unroll
            for (int a = 0; a < 3; ++a) s.dm1[3 * g + a] = fmaf(x[a], dW[g], s.dm1[3 * g + a] + (a == g ? w : 0.0f));
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                float t = (ia[q] == g ? wx[ib[q]] : 0.0f) + (ib[q] == g ? wx[ia[q]] : 0.0f);
                s.dm2[6 * g + q] = fmaf(xx[q], dW[g], s.dm2[6 * g + q] + t);
            }
        }
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        const int64_t n = p.n;
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        double m0 = (double)s.m0 - (double)s.c0, m1[3], M[3][3];
        for (int a = 0; a < 3; ++a) m1[a] = (double)s.m1[a] - (double)s.c1[a];
        for (int q = 0; q < 6; ++q) {
            double v = (double)s.m2[q] - (double)s.c2[q];
            M[ia[q]][ib[q]] = v;
            M[ib[q]][ia[q]] = v;
        }
        double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        double tr = M[0][0] + M[1][1] + M[2][2];
        if (!(det > 1e-12 * tr * tr * tr)) {  // singular: contributes nothing
            for (int k = 0; k < kCorrCoef; ++k) p.coef[k * n + o] = 0.f;
            if (p.n_singular) atomicAdd(p.n_singular, 1);
            return;
        }
        double Mi[3][3];
        double id = 1.0 / det;
        Mi[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) * id;
        Mi[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * id;
        Mi[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * id;
        Mi[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * id;
        Mi[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * id;
        Mi[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * id;
        Mi[1][0] = Mi[0][1];
        Mi[2][0] = Mi[0][2];
        Mi[2][1] = Mi[1][2];
        double B[3], Bb[3], Mib[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < 3; ++a) B[a] = -(Mi[a][0] * m1[0] + Mi[a][1] * m1[1] + Mi[a][2] * m1[2]);
        double A = 1.0 / (m0 + B[0] * m1[0] + B[1] * m1[1] + B[2] * m1[2]);
        for (int a = 0; a < 3; ++a) Bb[a] = (double)p.Bbar[a * n + o];
        double Ab = (double)p.Abar[o];
        // moment cotangents: dm1b[g][a], dm2b[g][ab] (symmetric in ab, packed as ia/ib)
        double m0b = 0.0, m1b[3] = {0, 0, 0}, dm0b[3], dm1b[3][3], dm2b[3][6];
        double dm1[3][3], dm2[3][6];
        for (int g = 0; g < 3; ++g) {
            for (int a = 0; a < 3; ++a) dm1[g][a] = (double)s.dm1[3 * g + a];
            for (int q = 0; q < 6; ++q) dm2[g][q] = (double)s.dm2[6 * g + q];
        }
        for (int g = 0; g < 3; ++g) {
            double dM[3][3], t[3], tb[3], K = (double)s.dm0[g];
            for (int q = 0; q < 6; ++q) {
                dM[ia[q]][ib[q]] = dm2[g][q];
                dM[ib[q]][ia[q]] = dm2[g][q];
            }
            for (int a = 0; a < 3; ++a) {
                t[a] = dm1[g][a] + dM[a][0] * B[0] + dM[a][1] * B[1] + dM[a][2] * B[2];
                K += 2.0 * B[a] * dm1[g][a] + B[a] * (dM[a][0] * B[0] + dM[a][1] * B[1] + dM[a][2] * B[2]);
            }
            double gb[3];
            for (int a = 0; a < 3; ++a) gb[a] = (double)p.gBbar[(3 * g + a) * n + o];
            for (int a = 0; a < 3; ++a) tb[a] = -(Mi[a][0] * gb[0] + Mi[a][1] * gb[1] + Mi[a][2] * gb[2]);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) Mib[a][b] -= gb[a] * t[b];
            const double gAb = (double)p.gAbar[g * n + o];
            const double Kb = -A * A * gAb;
            Ab += -2.0 * A * K * gAb;
            dm0b[g] = Kb;
            for (int a = 0; a < 3; ++a) {
                dm1b[g][a] = tb[a] + 2.0 * B[a] * Kb;
                Bb[a] += tb[0] * dM[0][a] + tb[1] * dM[1][a] + tb[2] * dM[2][a];  // dM symmetric
                Bb[a] += 2.0 * dm1[g][a] * Kb + 2.0 * (dM[a][0] * B[0] + dM[a][1] * B[1] + dM[a][2] * B[2]) * Kb;
            }
            // dm2b[g][a][b] = tb_a B_b + B_a B_b Kb, summed over (a, b) and (b, a) for a packed
            // off-diagonal entry (the moment sums are symmetric in ab)
            for (int q = 0; q < 6; ++q) {
                const int a = ia[q], b = ib[q];
                double v = tb[a] * B[b] + B[a] * B[b] * Kb;
                if (a != b) v += tb[b] * B[a] + B[b] * B[a] * Kb;
                dm2b[g][q] = v;
            }
        }
        const double denb = -A * A * Ab;
        m0b += denb;
        for (int a = 0; a < 3; ++a) {
            Bb[a] += m1[a] * denb;
            m1b[a] += B[a] * denb;
        }
        for (int a = 0; a < 3; ++a) {
            m1b[a] -= Mi[0][a] * Bb[0] + Mi[1][a] * Bb[1] + Mi[2][a] * Bb[2];
            for (int b = 0; b < 3; ++b) Mib[a][b] -= Bb[a] * m1[b];
        }
        // m2b = -Mi^T Mib Mi^T = -Mi (Mib Mi) (Mi symmetric): two 3x3 products (FP64 is 1/64 rate)
        double T[3][3], m2b[3][3];
        for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 3; ++b) T[c][b] = Mib[c][0] * Mi[0][b] + Mib[c][1] * Mi[1][b] + Mib[c][2] * Mi[2][b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) m2b[a][b] = -(Mi[a][0] * T[0][b] + Mi[a][1] * T[1][b] + Mi[a][2] * T[2][b]);
        // polynomial coefficients.  dm2b enters as sum_{g,ab} dm2b[g][ab] (delta_ag x_b W +
        // delta_bg x_a W + x_a x_b x_g dWr) with the packed (a <= b) entries carrying both orders.
        double c[kCorrCoef];
        c[0] = m0b + dm1b[0][0] + dm1b[1][1] + dm1b[2][2];
        for (int e = 0; e < 3; ++e) c[1 + e] = m1b[e];
        for (int g = 0; g < 3; ++g)
            for (int q = 0; q < 6; ++q) {
                const int a = ia[q], b = ib[q];
                // delta_ag x_b + delta_bg x_a (for a = b = g: 2 x_a)
                if (a == g) c[1 + b] += dm2b[g][q];
                if (b == g) c[1 + a] += dm2b[g][q];
            }
        // q0: x^T m2b x as monomials
        c[4] = m2b[0][0];
        c[5] = m2b[0][1] + m2b[1][0];
        c[6] = m2b[0][2] + m2b[2][0];
        c[7] = m2b[1][1];
        c[8] = m2b[1][2] + m2b[2][1];
        c[9] = m2b[2][2];
        for (int e = 0; e < 3; ++e) c[10 + e] = dm0b[e];
        // q1: sum_ga dm1b[g][a] x_a x_g
        c[13] = dm1b[0][0];
        c[14] = dm1b[0][1] + dm1b[1][0];
        c[15] = dm1b[0][2] + dm1b[2][0];
        c[16] = dm1b[1][1];
        c[17] = dm1b[1][2] + dm1b[2][1];
        c[18] = dm1b[2][2];
        // k: sum_{g,ab} dm2b[g][ab] x_g x_a x_b (packed entries already hold both ab orders)
        for (int e = 0; e < 10; ++e) c[19 + e] = 0.0;
        for (int g = 0; g < 3; ++g)
            for (int q = 0; q < 6; ++q) {
                int t[3] = {g, ia[q], ib[q]};
                // sort the three axes to find the monomial
                if (t[0] > t[1]) { int u = t[0]; t[0] = t[1]; t[1] = u; }
                if (t[1] > t[2]) { int u = t[1]; t[1] = t[2]; t[2] = u; }
                if (t[0] > t[1]) { int u = t[0]; t[0] = t[1]; t[1] = u; }
                // index of (t0 <= t1 <= t2) among xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
                const int idx = t[0] == 0 ? (t[1] == 0 ? t[2] : (t[1] == 1 ? 2 + t[2] : 5))
                                          : (t[0] == 1 ? (t[1] == 1 ? 6 + (t[2] - 1) : 8) : 9);
                c[19 + idx] += dm2b[g][q];
            }
        for (int k = 0; k < kCorrCoef; ++k) p.coef[k * n + o] = (float)c[k];
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        for (int k = 0; k < kCorrCoef; ++k) p.coef[k * p.n + o] = 0.f;
    }
};

struct CorrAdjSweepP {
    const float *V, *coef;
    float *xbar3, *Vbar;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;
};

// value and gradient of T(x) = S0 W + S1 dWr for coefficients c (layout above)
__device__ __forceinline__ float corr_term(const float *c, const float x[3], float W, float dWr, float ddWr,
                                           float g[3]) {
    const float X = x[0], Y = x[1], Z = x[2];
    const float q0 = fmaf(c[4] * X, X, fmaf(c[5] * X, Y, fmaf(c[6] * X, Z, fmaf(c[7] * Y, Y, fmaf(c[8] * Y, Z, c[9] * Z * Z)))));
    const float S0 = c[0] + fmaf(c[1], X, fmaf(c[2], Y, c[3] * Z)) + q0;
    const float g0x = c[1] + fmaf(2.0f * c[4], X, fmaf(c[5], Y, c[6] * Z));
    const float g0y = c[2] + fmaf(c[5], X, fmaf(2.0f * c[7], Y, c[8] * Z));
    const float g0z = c[3] + fmaf(c[6], X, fmaf(c[8], Y, 2.0f * c[9] * Z));
    const float *k = c + 19;
    const float XX = X * X, XY = X * Y, XZ = X * Z, YY = Y * Y, YZ = Y * Z, ZZ = Z * Z;
    const float q1 = fmaf(c[13], XX, fmaf(c[14], XY, fmaf(c[15], XZ, fmaf(c[16], YY, fmaf(c[17], YZ, c[18] * ZZ)))));
    const float cub = fmaf(k[0] * XX, X, fmaf(k[1] * XX, Y, fmaf(k[2] * XX, Z, fmaf(k[3] * YY, X, fmaf(k[4] * XY, Z,
                      fmaf(k[5] * ZZ, X, fmaf(k[6] * YY, Y, fmaf(k[7] * YY, Z, fmaf(k[8] * ZZ, Y, k[9] * ZZ * Z)))))))));
    const float S1 = fmaf(c[10], X, fmaf(c[11], Y, c[12] * Z)) + q1 + cub;
    const float g1x = c[10] + fmaf(2.0f * c[13], X, fmaf(c[14], Y, c[15] * Z)) +
                      fmaf(3.0f * k[0], XX, fmaf(2.0f * k[1], XY, fmaf(2.0f * k[2], XZ, fmaf(k[3], YY, fmaf(k[4], YZ, k[5] * ZZ)))));
    const float g1y = c[11] + fmaf(c[14], X, fmaf(2.0f * c[16], Y, c[17] * Z)) +
                      fmaf(k[1], XX, fmaf(2.0f * k[3], XY, fmaf(k[4], XZ, fmaf(3.0f * k[6], YY, fmaf(2.0f * k[7], YZ, k[8] * ZZ)))));
    const float g1z = c[12] + fmaf(c[15], X, fmaf(c[17], Y, 2.0f * c[18] * Z)) +
                      fmaf(k[2], XX, fmaf(k[4], XY, fmaf(2.0f * k[5], XZ, fmaf(k[7], YY, fmaf(2.0f * k[8], YZ, 3.0f * k[9] * ZZ)))));
    const float a = fmaf(S0, dWr, S1 * ddWr);
    g[0] = fmaf(g0x, W, fmaf(g1x, dWr, a * X));
    g[1] = fmaf(g0y, W, fmaf(g1y, dWr, a * Y));
    g[2] = fmaf(g0z, W, fmaf(g1z, dWr, a * Z));
    return fmaf(S0, W, S1 * dWr);
}

struct CorrAdjStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = false;
    using P = CorrAdjSweepP;
    struct __align__(16) Rec {
        float x, y, z, h;
        float V, c[kCorrCoef], pad[2];
    };
    struct I {
        float gx, gy, gz, Vb;
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) {
        Rec r;
        r.x = ps.x; r.y = ps.y; r.z = ps.z; r.h = ps.w;
        r.V = p.V[o];
#pragma unroll
        for (int k = 0; k < kCorrCoef; ++k) r.c[k] = p.coef[k * p.n + o];
        r.pad[0] = r.pad[1] = 0.f;
        return r;
    }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) {
        s.gx = s.gy = s.gz = s.Vb = 0.f;
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact(const P &, I &s, const Rec &ri, const Rec &rj) {
        float x[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};  // x_ij
        float r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float W, dWr, ddWr;
        wendland2(r2, 0.5f * hs, W, dWr, ddWr);
        W = in ? W : 0.0f;
        dWr = in ? dWr : 0.0f;
        ddWr = in ? ddWr : 0.0f;
        float gi[3], gj[3];
        const float xm[3] = {-x[0], -x[1], -x[2]};
        corr_term(ri.c, x, W, dWr, ddWr, gi);
        const float Tj = corr_term(rj.c, xm, W, dWr, ddWr, gj);
        s.gx += rj.V * gi[0] - ri.V * gj[0];
        s.gy += rj.V * gi[1] - ri.V * gj[1];
        s.gz += rj.V * gi[2] - ri.V * gj[2];
        s.Vb += Tj;
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        p.xbar3[o] = s.gx;
        p.xbar3[p.n + o] = s.gy;
        p.xbar3[2 * p.n + o] = s.gz;
        p.Vbar[o] = s.Vb;
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        p.xbar3[o] = 0.f;
        p.xbar3[p.n + o] = 0.f;
        p.xbar3[2 * p.n + o] = 0.f;
        p.Vbar[o] = 0.f;
    }
};

struct HydroP {
    const float *m, *v3, *u, *V, *rho, *A, *B, *gA, *gB;
    float *dv3, *du;
    double *cons;
    float gamma, alpha, beta, eta2;
    int64_t n;
    unsigned long long *count;
    const float *dvg;  // limited viscosity: velocity gradient [9][n], dv^a/dx^b at 3a+b
    unsigned long long *swept;  // counting runs: candidate pair evaluations, may be NULL
    const float *vstar;         // Energy pass: time-centred velocities [3][n]
    unsigned int *vsig_h;       // Acceleration pass: atomic max of vsig_i / h_i (FP32 bits), may be NULL
    float sig_beta;             // Acceleration pass: vsig_ij = c_i + c_j - sig_beta min(0, v_ij.x_ij / r)
};

struct HydroRec {
    float x, y, z, h;
    float vx, vy, vz, P;
    float c, rho, V, A;
    float B[3], gA0;
    float gA1, gA2, gB0, gB1;
    float gB[7];  // gB[2..8]
    float pad;
};
struct HydroRecLim : HydroRec {
    float G[9];  // velocity gradient, dv^a/dx^b at 3a+b
    float pad2[3];
};
template <class Base>
struct HydroRecVstar : Base {
    float wx, wy, wz, u;  // time-centred velocity v* and specific internal energy
};

// kLim: the viscosity sees both velocities reconstructed linearly to the pair
// midpoint, s = (dv) x, with the van Leer limiter
// phi = 4 r/(1+r)^2, r = (x.s_i)/(x.s_j), written 4 a_i a_j/(a_i + a_j)^2 for
// a_i a_j > 0 (else 0): the same value without a division by a_j alone.
//
// kPass (Sec. 5: Acceleration and Energy; Sec. 5.4: each runs twice a step):
//   kHydroBoth    dv/dt and du/dt with the equal split of the pair work on v;
//   kHydroAccel   dv/dt only, plus the signal velocity
//                 vsig_i = max_j (c_i + c_j - sig_beta min(0, v_ij.x_ij / r))
//                 (j = i gives 2 c_i), folded into one FP32 atomic max of
//                 vsig_i / h_i (Sec. 5.1: floating-point atomic max);
//   kHydroEnergy  du/dt with the compatible split: the pair heat
//                 dE_ij = -f_ij.(v*_i - v*_j) goes to i with the share
//                 w_ij = 1/2 (1 + sgn(dE) (u_j - u_i) / (|u_j - u_i| + (u_i + u_j)/2))
//                 (1/2 when u_i = u_j), so that sum_i m_i du_i = -sum_i f_i.v*_i.
constexpr int kHydroBoth = 0, kHydroAccel = 1, kHydroEnergy = 2;

template <bool kLim, int kPass = kHydroBoth>
struct HydroStageT {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = true;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = kPass == kHydroBoth;  // the step passes: lists and tiles only
    using P = HydroP;
    using Base = std::conditional_t<kLim, HydroRecLim, HydroRec>;
    struct __align__(16) Rec : std::conditional_t<kPass == kHydroEnergy, HydroRecVstar<Base>, Base> {};
    struct I {
        float fx, fy, fz, e;
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) {
        const int64_t n = p.n;
        Rec r;
        r.x = ps.x; r.y = ps.y; r.z = ps.z; r.h = ps.w;
        r.vx = p.v3[o]; r.vy = p.v3[n + o]; r.vz = p.v3[2 * n + o];
        float rho = p.rho[o], u = p.u[o];
        r.P = (p.gamma - 1.0f) * rho * u;
        r.c = sqrtf(p.gamma * (p.gamma - 1.0f) * u);
        r.rho = rho;
        r.V = p.V[o];
        r.A = p.A[o];
        r.B[0] = p.B[o]; r.B[1] = p.B[n + o]; r.B[2] = p.B[2 * n + o];
        r.gA0 = p.gA[o]; r.gA1 = p.gA[n + o]; r.gA2 = p.gA[2 * n + o];
        r.gB0 = p.gB[o]; r.gB1 = p.gB[n + o];
        for (int k = 0; k < 7; ++k) r.gB[k] = p.gB[(2 + k) * n + o];
        r.pad = 0.f;
        if constexpr (kLim) {
            for (int k = 0; k < 9; ++k) r.G[k] = p.dvg[k * n + o];
            r.pad2[0] = r.pad2[1] = r.pad2[2] = 0.f;
        }
        if constexpr (kPass == kHydroEnergy) {
            r.wx = p.vstar[o]; r.wy = p.vstar[n + o]; r.wz = p.vstar[2 * n + o];
            r.u = u;
        }
        return r;
    }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) { s.fx = s.fy = s.fz = s.e = 0.f; s.cnt = 0; }
    // grad W^R of record r at separation x (x = x_r - x_other): gA (1 + B.x) W + A (gB.x + B) W + A (1 + B.x) dWr x
    template <class R>
    __device__ static void grad_wr(const R &r, const float x[3], float W, float dWr, float g[3]) {
        float Bx = fmaf(r.B[0], x[0], fmaf(r.B[1], x[1], r.B[2] * x[2]));
        float gb[9] = {r.gB0, r.gB1, r.gB[0], r.gB[1], r.gB[2], r.gB[3], r.gB[4], r.gB[5], r.gB[6]};
        float gA[3] = {r.gA0, r.gA1, r.gA2};
        float k1 = (1.0f + Bx) * W;
        float k3 = r.A * (1.0f + Bx) * dWr;
        float AW = r.A * W;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float gBx = fmaf(gb[3 * q], x[0], fmaf(gb[3 * q + 1], x[1], gb[3 * q + 2] * x[2]));
            g[q] = fmaf(gA[q], k1, fmaf(AW, gBx + r.B[q], k3 * x[q]));
        }
    }
    template <bool kCount>
    __device__ static void interact(const P &p, I &s, const Rec &ri, const Rec &rj) {
        float x[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};  // x_ij
        float r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float hij = 0.5f * hs;
        float W, dWr;
        wendland(r2, hij, W, dWr);
        float gi[3], gj[3];
        grad_wr(ri, x, W, dWr, gi);
        float xm[3] = {-x[0], -x[1], -x[2]};
        grad_wr(rj, xm, W, dWr, gj);
        float vij[3] = {ri.vx - rj.vx, ri.vy - rj.vy, ri.vz - rj.vz};
        float vx;
        if constexpr (kLim) {
            float si[3], sj[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                si[a] = fmaf(ri.G[3 * a], x[0], fmaf(ri.G[3 * a + 1], x[1], ri.G[3 * a + 2] * x[2]));
                sj[a] = fmaf(rj.G[3 * a], x[0], fmaf(rj.G[3 * a + 1], x[1], rj.G[3 * a + 2] * x[2]));
            }
            const float ai = fmaf(x[0], si[0], fmaf(x[1], si[1], x[2] * si[2]));
            const float aj = fmaf(x[0], sj[0], fmaf(x[1], sj[1], x[2] * sj[2]));
            const float aa = ai * aj, as = ai + aj;
            const float phi = aa > 0.0f ? __fdividef(4.0f * aa, as * as) : 0.0f;
            const float hp = 0.5f * phi;
            float vs[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) vs[a] = fmaf(-hp, si[a] + sj[a], vij[a]);
            vx = fmaf(vs[0], x[0], fmaf(vs[1], x[1], vs[2] * x[2]));
        } else {
            vx = fmaf(vij[0], x[0], fmaf(vij[1], x[1], vij[2] * x[2]));
        }
        float mu = vx < 0.0f ? __fdividef(hij * vx, fmaf(p.eta2 * hij, hij, r2)) : 0.0f;
        float Q = 0.5f * (ri.rho + rj.rho) * mu * fmaf(-p.alpha * 0.5f, ri.c + rj.c, p.beta * mu);
        float pre = in ? -0.5f * ri.V * rj.V * (ri.P + rj.P + Q) : 0.0f;
        float f[3] = {pre * (gi[0] - gj[0]), pre * (gi[1] - gj[1]), pre * (gi[2] - gj[2])};
        s.fx += f[0];
        s.fy += f[1];
        s.fz += f[2];
        if constexpr (kPass == kHydroBoth) {
            s.e = fmaf(-0.5f, fmaf(vij[0], f[0], fmaf(vij[1], f[1], vij[2] * f[2])), s.e);
        } else if constexpr (kPass == kHydroAccel) {
            // approach speed on the true velocities (the limiter shapes only the viscosity)
            const float w = fmaf(vij[0], x[0], fmaf(vij[1], x[1], vij[2] * x[2])) * (r2 > 0.0f ? rsqrtf(r2) : 0.0f);
            const float vs = fmaf(-p.sig_beta, fminf(w, 0.0f), ri.c + rj.c);
            s.e = in ? fmaxf(s.e, vs) : s.e;
        } else {
            const float dE = -fmaf(ri.wx - rj.wx, f[0], fmaf(ri.wy - rj.wy, f[1], (ri.wz - rj.wz) * f[2]));
            const float du = rj.u - ri.u;
            // (u_j - u_i) / (|u_j - u_i| + (u_i + u_j)/2): the same magnitude for i and j, opposite sign
            const float t = du != 0.0f ? __fdividef(du, fabsf(du) + 0.5f * (ri.u + rj.u)) : 0.0f;
            const float w = 0.5f + 0.5f * (dE > 0.0f ? t : -t);
            s.e = fmaf(w, dE, s.e);
        }
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &ri, int32_t o, int64_t) {
        float mi = p.m[o];
        if constexpr (kPass != kHydroEnergy) {
            p.dv3[o] = s.fx / mi;
            p.dv3[p.n + o] = s.fy / mi;
            p.dv3[2 * p.n + o] = s.fz / mi;
        }
        if constexpr (kPass != kHydroAccel) p.du[o] = s.e / mi;
        if constexpr (kPass == kHydroAccel) {
            if (p.vsig_h) {
                // vsig / h >= 0: its FP32 bit pattern orders like the value; one atomic per
                // converged set of lanes
                const unsigned q = __float_as_uint(__fdividef(s.e, ri.h));
                const unsigned mask = __activemask();
                const unsigned qm = __reduce_max_sync(mask, q);
                if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicMax(p.vsig_h, qm);
            }
        }
    }
    // FP64 conservation terms of one gas particle: m dv (3) and m (v.dv + du), with
    // v = v* in the Energy pass (the compatible balance) and du = 0 in the Acceleration pass
    __device__ static void cons_terms(const P &p, const I &s, const Rec &ri, int32_t o, double c[4]) {
        double mi = (double)p.m[o];
        double dvx = (double)(s.fx / p.m[o]), dvy = (double)(s.fy / p.m[o]), dvz = (double)(s.fz / p.m[o]);
        double du = kPass == kHydroAccel ? 0.0 : (double)(s.e / p.m[o]);
        double wx = ri.vx, wy = ri.vy, wz = ri.vz;
        if constexpr (kPass == kHydroEnergy) { wx = ri.wx; wy = ri.wy; wz = ri.wz; }
        c[0] = mi * dvx;
        c[1] = mi * dvy;
        c[2] = mi * dvz;
        c[3] = mi * (wx * dvx + wy * dvy + wz * dvz + du);
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        if constexpr (kPass != kHydroEnergy) {
            p.dv3[o] = 0.f;
            p.dv3[p.n + o] = 0.f;
            p.dv3[2 * p.n + o] = 0.f;
        }
        if constexpr (kPass != kHydroAccel) p.du[o] = 0.f;
    }

    // Half-warp arms (Sec. 5.3): partial sums of one i from one leaf-pair tile are added
    // to the zeroed outputs with atomics (the Energy pass also adds its recomputed force
    // to p.dv3 when given, for the conservation sums); the signal-velocity maximum goes
    // straight to the one atomic max of vsig_i / h_i (a max of partial maxima).
    static constexpr bool kHalfWarp = true;
    __device__ static void flush(const P &p, const I &s, const Rec &ri, int32_t o) {
        const float mi = p.m[o];
        if (p.dv3) {
            atomicAdd(&p.dv3[o], s.fx / mi);
            atomicAdd(&p.dv3[p.n + o], s.fy / mi);
            atomicAdd(&p.dv3[2 * p.n + o], s.fz / mi);
        }
        if constexpr (kPass != kHydroAccel) atomicAdd(&p.du[o], s.e / mi);
        if constexpr (kPass == kHydroAccel) {
            if (p.vsig_h) atomicMax(p.vsig_h, __float_as_uint(__fdividef(s.e, ri.h)));
        }
    }
    // outside every cut (r^2 ~ 1e30 against (h_i + h_j)^2) with zero fields: exact zeros
    __device__ static Rec far_dummy(float fx, float fy, float fz) {
        Rec r{};
        r.x = fx; r.y = fy; r.z = fz; r.h = 1.0f;
        return r;
    }
    static void zero_outputs(const P &p, cudaStream_t st) {
        if (p.dv3) cudaMemsetAsync(p.dv3, 0, sizeof(float) * 3 * p.n, st);
        if (kPass != kHydroAccel && p.du) cudaMemsetAsync(p.du, 0, sizeof(float) * p.n, st);
    }
    // the conservation terms of cons_terms from the finished outputs of gas particle o
    __device__ static void cons_of(const P &p, int32_t o, double c[4]) {
        const int64_t n = p.n;
        const double mi = (double)p.m[o];
        const double dvx = p.dv3[o], dvy = p.dv3[n + o], dvz = p.dv3[2 * n + o];
        const double du = kPass == kHydroAccel ? 0.0 : (double)p.du[o];
        const float *w = kPass == kHydroEnergy ? p.vstar : p.v3;
        c[0] = mi * dvx;
        c[1] = mi * dvy;
        c[2] = mi * dvz;
        c[3] = mi * ((double)w[o] * dvx + (double)w[n + o] * dvy + (double)w[2 * n + o] * dvz + du);
    }
};


using HydroStage = HydroStageT<false>;
using HydroLimStage = HydroStageT<true>;
// Reverse mode of the hydro pair force (Monaghan viscosity, equal split; not
// in the paper) for cotangents dvbar, dubar, with every input independent.
// With a_i = dvbar_i/m_i, b_i = dubar_i/m_i the loss is a sum over unordered
// pairs i != j of l_ij = z.f_ij, z = (a_i - a_j) - (b_i + b_j) v_ij / 2
// (f_ji = -f_ij, e_ji = e_ij; the self pair has f_ii = 0 for all of i's
// inputs), so each i gathers dl_ij/d(i's inputs) over its neighbours: one-sided,
// nothing per pair stored, no atomics.  m enters through a and b only:
// mbar_i = -(a_i.F_i + b_i E_i)/m_i with the recomputed sums F, E.
struct HydroAdjP {
    const float *m, *v3, *u, *V, *rho, *A, *B, *gA, *gB, *dvbar3, *dubar;
    float *xbar3, *vbar3, *ubar, *mbar, *Vbar, *rhobar, *Abar, *Bbar3, *gAbar3, *gBbar9;
    float gamma, alpha, beta, eta2;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;
};

// sum_q c_q dG_q/dy_p for the corrected-kernel gradient G(y) of a record (see grad_wr), and the
// cotangents of its A, B, dA, dB when kParams
template <bool kParams, class R>
__device__ __forceinline__ void grad_wr_vjp(const R &r, const float y[3], float W, float dWr, float ddWr,
                                            const float c[3], float out[3], float *Ab, float *Bb, float *gAb,
                                            float *gBb) {
    const float gb[9] = {r.gB0, r.gB1, r.gB[0], r.gB[1], r.gB[2], r.gB[3], r.gB[4], r.gB[5], r.gB[6]};
    const float gA[3] = {r.gA0, r.gA1, r.gA2};
    const float By = fmaf(r.B[0], y[0], fmaf(r.B[1], y[1], r.B[2] * y[2]));
    const float cy = fmaf(c[0], y[0], fmaf(c[1], y[1], c[2] * y[2]));
    const float cgA = fmaf(c[0], gA[0], fmaf(c[1], gA[1], c[2] * gA[2]));
    const float cB = fmaf(c[0], r.B[0], fmaf(c[1], r.B[1], c[2] * r.B[2]));
    float cgBy = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q) cgBy = fmaf(c[q], fmaf(gb[3 * q], y[0], fmaf(gb[3 * q + 1], y[1], gb[3 * q + 2] * y[2])), cgBy);
    const float opB = 1.0f + By;
    const float kB = fmaf(W, cgA, r.A * dWr * cy);
    const float ky = fmaf(cgA * opB, dWr, r.A * fmaf(dWr, cgBy + cB, opB * ddWr * cy));
    const float AW = r.A * W, kc = r.A * opB * dWr;
#pragma unroll
    for (int pp = 0; pp < 3; ++pp) {
        const float gBtc = fmaf(c[0], gb[pp], fmaf(c[1], gb[3 + pp], c[2] * gb[6 + pp]));
        out[pp] = fmaf(r.B[pp], kB, fmaf(y[pp], ky, fmaf(AW, gBtc, kc * c[pp])));
    }
    if constexpr (kParams) {
        *Ab += fmaf(W, cgBy + cB, opB * dWr * cy);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            gAb[q] = fmaf(c[q] * opB, W, gAb[q]);
            Bb[q] = fmaf(y[q], kB, fmaf(AW, c[q], Bb[q]));
#pragma unroll
            for (int a = 0; a < 3; ++a) gBb[3 * q + a] = fmaf(c[q] * AW, y[a], gBb[3 * q + a]);
        }
    }
}

struct HydroAdjStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = false;
    using P = HydroAdjP;
    struct __align__(16) Rec : HydroRec {
        float ax, ay, az, b;  // dvbar/m, dubar/m
    };
    struct I {
        float xb[3], vb[3], Vb, Pb, cb, rb, Ab, Bb[3], gAb[3], gBb[9], F[3], E;
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) {
        const int64_t n = p.n;
        Rec r;
        r.x = ps.x; r.y = ps.y; r.z = ps.z; r.h = ps.w;
        r.vx = p.v3[o]; r.vy = p.v3[n + o]; r.vz = p.v3[2 * n + o];
        const float rho = p.rho[o], u = p.u[o];
        r.P = (p.gamma - 1.0f) * rho * u;
        r.c = sqrtf(p.gamma * (p.gamma - 1.0f) * u);
        r.rho = rho;
        r.V = p.V[o];
        r.A = p.A[o];
        r.B[0] = p.B[o]; r.B[1] = p.B[n + o]; r.B[2] = p.B[2 * n + o];
        r.gA0 = p.gA[o]; r.gA1 = p.gA[n + o]; r.gA2 = p.gA[2 * n + o];
        r.gB0 = p.gB[o]; r.gB1 = p.gB[n + o];
        for (int k = 0; k < 7; ++k) r.gB[k] = p.gB[(2 + k) * n + o];
        r.pad = __int_as_float(o);  // particle identity: the self pair is skipped
        const float im = __fdividef(1.0f, p.m[o]);
        r.ax = p.dvbar3[o] * im; r.ay = p.dvbar3[n + o] * im; r.az = p.dvbar3[2 * n + o] * im;
        r.b = p.dubar[o] * im;
        return r;
    }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &, I &s, const Rec &, int64_t, int, int, int32_t) {
#pragma unroll
        for (int a = 0; a < 3; ++a) s.xb[a] = s.vb[a] = s.Bb[a] = s.gAb[a] = s.F[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 9; ++a) s.gBb[a] = 0.f;
        s.Vb = s.Pb = s.cb = s.rb = s.Ab = s.E = 0.f;
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact(const P &p, I &s, const Rec &ri, const Rec &rj) {
        float x[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};  // x_ij
        float r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
        float hs = ri.h + rj.h;
        const bool in = r2 < hs * hs && __float_as_int(ri.pad) != __float_as_int(rj.pad);
        float hij = 0.5f * hs;
        float W, dWr, ddWr;
        wendland2(r2, hij, W, dWr, ddWr);
        W = in ? W : 0.0f;  // every term below is then zero
        dWr = in ? dWr : 0.0f;
        ddWr = in ? ddWr : 0.0f;
        float gi[3], gj[3];
        HydroStage::grad_wr(ri, x, W, dWr, gi);
        const float xm[3] = {-x[0], -x[1], -x[2]};
        HydroStage::grad_wr(rj, xm, W, dWr, gj);
        const float vij[3] = {ri.vx - rj.vx, ri.vy - rj.vy, ri.vz - rj.vz};
        const float vx = fmaf(vij[0], x[0], fmaf(vij[1], x[1], vij[2] * x[2]));
        const float den = fmaf(p.eta2 * hij, hij, r2);
        const bool visc = vx < 0.0f && in;
        const float mu = visc ? __fdividef(hij * vx, den) : 0.0f;
        const float rbar = 0.5f * (ri.rho + rj.rho), cbar = 0.5f * (ri.c + rj.c);
        const float Q = rbar * mu * fmaf(-p.alpha, cbar, p.beta * mu);
        const float Pi = ri.P + rj.P + Q;
        const float VV = ri.V * rj.V;
        const float pre = -0.5f * VV * Pi;
        const float d[3] = {gi[0] - gj[0], gi[1] - gj[1], gi[2] - gj[2]};
        const float sb = ri.b + rj.b;
        const float z[3] = {fmaf(-0.5f * sb, vij[0], ri.ax - rj.ax), fmaf(-0.5f * sb, vij[1], ri.ay - rj.ay),
                            fmaf(-0.5f * sb, vij[2], ri.az - rj.az)};
        const float D = fmaf(z[0], d[0], fmaf(z[1], d[1], z[2] * d[2]));
#pragma unroll
        for (int c = 0; c < 3; ++c) s.F[c] = fmaf(pre, d[c], s.F[c]);
        s.E = fmaf(-0.5f * pre, fmaf(vij[0], d[0], fmaf(vij[1], d[1], vij[2] * d[2])), s.E);
        const float Pib = -0.5f * VV * D;
        s.Vb = fmaf(-0.5f * rj.V * Pi, D, s.Vb);
        s.Pb += Pib;
        if (visc) {
            const float mub = Pib * rbar * fmaf(-p.alpha, cbar, 2.0f * p.beta * mu);
            s.rb = fmaf(Pib * 0.5f * mu, fmaf(-p.alpha, cbar, p.beta * mu), s.rb);
            s.cb = fmaf(Pib * rbar * mu, -0.5f * p.alpha, s.cb);
            const float vxb = __fdividef(mub * hij, den);
            const float r2b2 = -2.0f * vxb * __fdividef(vx, den);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                s.xb[c] = fmaf(vxb, vij[c], fmaf(r2b2, x[c], s.xb[c]));
                s.vb[c] = fmaf(vxb, x[c], s.vb[c]);
            }
        }
        const float dbar[3] = {pre * z[0], pre * z[1], pre * z[2]};
#pragma unroll
        for (int c = 0; c < 3; ++c) s.vb[c] = fmaf(-0.5f * sb * pre, d[c], s.vb[c]);
        float o1[3], o2[3];
        grad_wr_vjp<true>(ri, x, W, dWr, ddWr, dbar, o1, &s.Ab, s.Bb, s.gAb, s.gBb);
        grad_wr_vjp<false>(rj, xm, W, dWr, ddWr, dbar, o2, nullptr, nullptr, nullptr, nullptr);
#pragma unroll
        for (int c = 0; c < 3; ++c) s.xb[c] += o1[c] + o2[c];
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &ri, int32_t o, int64_t) {
        const int64_t n = p.n;
        const float u = p.u[o], rho = p.rho[o], g1 = p.gamma - 1.0f;
        const float ub = fmaf(s.Pb * g1, rho, ri.c > 0.0f ? __fdividef(s.cb * p.gamma * g1, 2.0f * ri.c) : 0.0f);
        const float rb = fmaf(s.Pb * g1, u, s.rb);
        const float mb = -__fdividef(fmaf(ri.ax, s.F[0], fmaf(ri.ay, s.F[1], fmaf(ri.az, s.F[2], ri.b * s.E))), p.m[o]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p.xbar3[c * n + o] = s.xb[c];
            p.vbar3[c * n + o] = s.vb[c];
            p.Bbar3[c * n + o] = s.Bb[c];
            p.gAbar3[c * n + o] = s.gAb[c];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) p.gBbar9[c * n + o] = s.gBb[c];
        p.ubar[o] = ub;
        p.mbar[o] = mb;
        p.Vbar[o] = s.Vb;
        p.rhobar[o] = rb;
        p.Abar[o] = s.Ab;
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        const int64_t n = p.n;
        for (int c = 0; c < 3; ++c) {
            p.xbar3[c * n + o] = 0.f;
            p.vbar3[c * n + o] = 0.f;
            p.Bbar3[c * n + o] = 0.f;
            p.gAbar3[c * n + o] = 0.f;
        }
        for (int c = 0; c < 9; ++c) p.gBbar9[c * n + o] = 0.f;
        p.ubar[o] = p.mbar[o] = p.Vbar[o] = p.rhobar[o] = p.Abar[o] = 0.f;
    }
};

template <bool kLim>
using HydroAccelStage = HydroStageT<kLim, kHydroAccel>;
template <bool kLim>
using HydroEnergyStage = HydroStageT<kLim, kHydroEnergy>;

// Extras (Sec. 5: the density and state gradients), over gas j including j = i:
//   rhoR_i = sum_j m_j W^R_ij,   dv_i[3a+b] = sum_j V_j (v_j^a - v_i^a) (grad_i W^R_ij)^b
// with W^R_ij = A_i (1 + B_i.x_ij) W_ij and grad_i W^R_ij as in the hydro stage.
struct ExtrasP {
    const float *m, *v3, *V, *A, *B, *gA, *gB;
    float *rhoR, *dvg;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

struct ExtrasStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = true;
    static constexpr bool kCons = false;
    static constexpr bool kTag = false;
    static constexpr bool kAllVariants = true;
    using P = ExtrasP;
    struct __align__(16) Rec {
        float x, y, z, h;
        float V, m, vx, vy;
        float vz, pad0, pad1, pad2;
    };
    struct I {
        float A, B[3], gA[3], gB[9];  // the i particle's corrections (gB[3g+a] = d_g B^a)
        float rho, crho;              // compensated sum
        float G[9];
        int cnt;
    };
    __device__ static Rec gather(const P &p, int32_t o, float4 ps) {
        const int64_t n = p.n;
        return {ps.x, ps.y, ps.z, ps.w, p.V[o], p.m[o], p.v3[o], p.v3[n + o], p.v3[2 * n + o], 0.f, 0.f, 0.f};
    }
    __device__ static float box_cut(const P &, float hmax_i, const Rec &rj) { return hmax_i + rj.h; }
    __device__ static float leaf_cut(const P &, float hmax_i, float hmax_j) { return hmax_i + hmax_j; }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void init(const P &p, I &s, const Rec &, int64_t, int, int, int32_t o) {
        const int64_t n = p.n;
        s.A = p.A[o];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s.B[a] = p.B[a * n + o];
            s.gA[a] = p.gA[a * n + o];
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            s.gB[a] = p.gB[a * n + o];
            s.G[a] = 0.f;
        }
        s.rho = s.crho = 0.f;
        s.cnt = 0;
    }
    template <bool kCount>
    __device__ static void interact(const P &, I &s, const Rec &ri, const Rec &rj) {
        float x[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};  // x_ij
        float r2 = fmaf(x[0], x[0], fmaf(x[1], x[1], x[2] * x[2]));
        float hs = ri.h + rj.h;
        bool in = r2 < hs * hs;
        float W, dWr;
        wendland(r2, 0.5f * hs, W, dWr);
        W = in ? W : 0.0f;
        dWr = in ? dWr : 0.0f;
        const float Bx = fmaf(s.B[0], x[0], fmaf(s.B[1], x[1], s.B[2] * x[2]));
        const float k1 = (1.0f + Bx) * W;
        kahan_add(s.rho, s.crho, rj.m * (s.A * k1));
        // grad_i W^R_ij = gA (1 + B.x) W + A (gB.x + B) W + A (1 + B.x) dWr x
        const float AW = s.A * W, k3 = s.A * (1.0f + Bx) * dWr;
        float g[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float gBx = fmaf(s.gB[3 * q], x[0], fmaf(s.gB[3 * q + 1], x[1], s.gB[3 * q + 2] * x[2]));
            g[q] = fmaf(s.gA[q], k1, fmaf(AW, gBx + s.B[q], k3 * x[q]));
        }
        const float dv[3] = {rj.V * (rj.vx - ri.vx), rj.V * (rj.vy - ri.vy), rj.V * (rj.vz - ri.vz)};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) s.G[3 * a + b] = fmaf(dv[a], g[b], s.G[3 * a + b]);
        if (kCount) s.cnt += in;
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t o, int64_t) {
        p.rhoR[o] = s.rho;
#pragma unroll
        for (int k = 0; k < 9; ++k) p.dvg[k * p.n + o] = s.G[k];
    }
    __device__ static void finish_other(const P &p, int32_t o) {
        p.rhoR[o] = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) p.dvg[k * p.n + o] = 0.f;
    }
};

// Builds the exact neighbour lists of every i-group (count pass, then fill
// pass): gas pairs (r < h_i + h_j) or gravity pairs (r < r_cut).  A group's
// lists index a table of the distinct j the group needs (the union over its
// lanes, in the order the sweep meets them), so that a pair kernel stages each
// j of the group once and every lane reads its j from that table.
struct ListP {
    uint16_t *list;                    // per-lane table indices, k-major rows of 32 (written when non-null)
    uint32_t *ucode;                   // table entries (written when non-null)
    const int32_t *gstart, *goff, *uoff;
    int32_t *cnt;                      // list length per kernel-order position (written when non-null)
    int32_t *ucnt;                     // table size per group (written when non-null)
    int32_t *umax;                     // largest table (atomicMax), may be null
    int32_t *overflow;                 // set when a list or a table exceeds its capacity, may be null
    int cap_rows, cap_table;           // capacity of one lane's list and of one group's table
    float rc2;
    int64_t n;
    unsigned long long *count;
    unsigned long long *swept;  // counting runs: candidate pair evaluations (tiles and lists), may be NULL
};

template <bool kGas>
struct ListStage {
    static constexpr bool kPair = false;
    static constexpr bool kGasOnly = kGas;
    static constexpr bool kCons = false;
    static constexpr bool kTag = true;
    using P = ListP;
    struct __align__(16) Rec {
        float x, y, z, h;
        uint32_t code, pad0, pad1, pad2;
    };
    struct I {
        uint16_t *out;
        uint32_t *uout;
        int64_t grp;
        int c;    // this lane's list length
        int u;    // table size (warp-uniform)
        int cnt;
    };

    __device__ static Rec gather(const P &, int32_t, float4 ps) { return {ps.x, ps.y, ps.z, ps.w, 0u, 0u, 0u, 0u}; }
    __device__ static float box_cut(const P &p, float hmax_i, const Rec &rj) {
        return kGas ? hmax_i + rj.h : sqrtf(p.rc2);
    }
    __device__ static float leaf_cut(const P &p, float hmax_i, float hmax_j) {
        return kGas ? hmax_i + hmax_j : sqrtf(p.rc2);
    }
    __device__ static void shift(Rec &r, float sx, float sy, float sz) { r.x += sx; r.y += sy; r.z += sz; }
    __device__ static void tag(Rec &r, int img_local, int j_local) {
        r.code = ((uint32_t)img_local << 10) | (uint32_t)j_local;
    }
    __device__ static void init(const P &p, I &s, const Rec &, int64_t a, int q, int lane, int32_t) {
        s.c = 0;
        s.u = 0;
        s.cnt = 0;
        s.grp = p.gstart[a] + q;
        s.out = p.list ? p.list + (size_t)p.goff[s.grp] * 32 + lane : nullptr;
        s.uout = p.ucode ? p.ucode + p.uoff[s.grp] : nullptr;
    }
    // called by all 32 lanes together (the sweep is warp-uniform)
    template <bool kCount>
    __device__ static void interact(const P &p, I &s, const Rec &ri, const Rec &rj) {
        bool in;
        if (kGas) {
            float dx = ri.x - rj.x, dy = ri.y - rj.y, dz = ri.z - rj.z;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float hs = ri.h + rj.h;
            in = r2 < hs * hs;
        } else {  // the gravity kernels take d = x_j - x_i
            float dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            in = r2 < p.rc2;
        }
        const unsigned m = __ballot_sync(CRK_FULL_MASK, in);
        if (m) {
            if (in) {
                if (s.out && s.c < p.cap_rows && s.u < p.cap_table) s.out[(size_t)s.c * 32] = (uint16_t)s.u;
                ++s.c;
            }
            if (s.uout && (int)(threadIdx.x & 31) == __ffs(m) - 1 && s.u < p.cap_table) s.uout[s.u] = rj.code;
            ++s.u;
        }
    }
    __device__ static void finish(const P &p, I &s, const Rec &, int32_t, int64_t i) {
        if (p.cnt) p.cnt[i] = s.c;
        if (p.overflow && (s.c > p.cap_rows || s.u > p.cap_table)) atomicOr(p.overflow, 1);
        if ((threadIdx.x & 31) == 0) {  // lane 0 is always active
            if (p.ucnt) p.ucnt[s.grp] = s.u;
            if (p.umax) atomicMax(p.umax, s.u);
        }
    }
    __device__ static void finish_other(const P &, int32_t) {}
};

// --------------------------------------------------------------- framework
template <class S>
__global__ void gather_kernel(int64_t n, const float4 *__restrict__ pos, const int32_t *__restrict__ kperm,
                              typename S::P p, typename S::Rec *__restrict__ rec, int korder) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float4 ps = pos[q];
    const int32_t o = korder ? (int32_t)q : kperm[q];
    if (S::kGasOnly && ps.w == 0.0f) {  // dark matter (h = 0): never read by gas-pair stages
        S::finish_other(p, o);           // its gas-only outputs are zero
        return;
    }
    rec[q] = S::gather(p, o, ps);
}

// Work of one warp on one i-group (tiles): the kernel-order particles
// g0 .. min(g0 + 32, hi) - 1 of i-leaf a (first particle lo) against every j
// of the leaf's images.  Each j within the cut of the group's box is
// ballot-compacted into the warp's shared-memory buffer; all lanes sweep the
// buffer (broadcast reads), each accumulating its own i.
template <class S, bool kCount>
__device__ __forceinline__ void tile_group(const LeafView &lv, const typename S::P &p,
                                           const typename S::Rec *__restrict__ rec, typename S::Rec *buf,
                                           int64_t a, int lo, int g0, int hi, int lane, double cons_acc[4]) {
    using Rec = typename S::Rec;
    const unsigned below = lanemask_lt();
    const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
    const int i = g0 + lane;
    const bool act = i < hi;
    const Rec ri = rec[act ? i : g0];
    typename S::I st;
    S::init(p, st, ri, a, (g0 - lo) >> 5, lane, stage_index(lv, act ? i : g0));
    // i-group box and largest h (inactive lanes repeat lane 0's particle)
    float bl0 = ri.x, bl1 = ri.y, bl2 = ri.z, bh0 = ri.x, bh1 = ri.y, bh2 = ri.z;
    float hm = lv.pos[act ? i : g0].w;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bl0 = fminf(bl0, __shfl_xor_sync(CRK_FULL_MASK, bl0, o));
        bl1 = fminf(bl1, __shfl_xor_sync(CRK_FULL_MASK, bl1, o));
        bl2 = fminf(bl2, __shfl_xor_sync(CRK_FULL_MASK, bl2, o));
        bh0 = fmaxf(bh0, __shfl_xor_sync(CRK_FULL_MASK, bh0, o));
        bh1 = fmaxf(bh1, __shfl_xor_sync(CRK_FULL_MASK, bh1, o));
        bh2 = fmaxf(bh2, __shfl_xor_sync(CRK_FULL_MASK, bh2, o));
        hm = fmaxf(hm, __shfl_xor_sync(CRK_FULL_MASK, hm, o));
    }
    int cnt = 0;
    unsigned long long swept = 0;  // counting runs: candidates swept
    for (int e = ib; e < ie; ++e) {
        const crk_image im = lv.img[e];
        const int jlo = lv.leaf_start[im.b];
        const int jhi = S::kGasOnly ? jlo + lv.leaf_ngas[im.b] : lv.leaf_start[im.b + 1];
        // whole j-leaf against the i-group box (warp-uniform)
        {
            const float *bb = lv.bbox + 6 * (int64_t)im.b;
            float gx = fmaxf(fmaxf(im.sx - bh0, bl0 - (im.sx + (bb[3] - bb[0]))), 0.f);
            float gy = fmaxf(fmaxf(im.sy - bh1, bl1 - (im.sy + (bb[4] - bb[1]))), 0.f);
            float gz = fmaxf(fmaxf(im.sz - bh2, bl2 - (im.sz + (bb[5] - bb[2]))), 0.f);
            float cut = S::leaf_cut(p, hm, lv.hmax[im.b]);
            if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut * cut * 1.0001f + 1e-6f)) continue;
        }
        for (int j0 = jlo; j0 < jhi; j0 += 32) {
            const int j = j0 + lane;
            const bool jv = j < jhi;
            Rec rj;
            bool keep = false;
            if (jv) {
                rj = rec[j];
                S::shift(rj, im.sx, im.sy, im.sz);
                if constexpr (S::kTag) S::tag(rj, e - ib, j - jlo);
                float dx = fmaxf(fmaxf(bl0 - rj.x, rj.x - bh0), 0.f);
                float dy = fmaxf(fmaxf(bl1 - rj.y, rj.y - bh1), 0.f);
                float dz = fmaxf(fmaxf(bl2 - rj.z, rj.z - bh2), 0.f);
                float cut = S::box_cut(p, hm, rj);
                keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut * cut * 1.0001f + 1e-6f;
            }
            const unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
            if (keep) buf[cnt + __popc(m & below)] = rj;
            cnt += __popc(m);
            if (cnt >= 32) {
                __syncwarp();
                for (int k = 0; k < cnt; ++k) S::template interact<kCount>(p, st, ri, buf[k]);
                if (kCount) swept += cnt;
                cnt = 0;
                __syncwarp();
            }
        }
    }
    __syncwarp();
    for (int k = 0; k < cnt; ++k) S::template interact<kCount>(p, st, ri, buf[k]);
    if (kCount) swept += cnt;
    __syncwarp();
    if (act) S::finish(p, st, ri, lv.korder ? i : lv.kperm[i], i);
    if constexpr (S::kCons) {
        double c[4] = {0.0, 0.0, 0.0, 0.0};
        if (act) S::cons_terms(p, st, ri, lv.korder ? i : lv.kperm[i], c);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(CRK_FULL_MASK, c[k], o);
            cons_acc[k] += c[k];
        }
    }
    if (kCount) {
        int c = act ? st.cnt - 1 : 0;  // the self pair (r = 0) is always in range
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(CRK_FULL_MASK, c, o);
        if (lane == 0 && c) atomicAdd(p.count, (unsigned long long)c);
        // candidate evaluations: every active lane evaluated every swept candidate
        const unsigned long long na = __popc(__ballot_sync(CRK_FULL_MASK, act));
        if (lane == 0 && p.swept) atomicAdd(p.swept, swept * na);
    }
}

// tile_group for stages with packed two-candidate interactions (kPair): the
// candidate buffer holds field-interleaved candidate pairs; an odd tail is
// padded with a massless dummy outside every i's cut, which adds exact zeros.
template <class S, bool kCount>
__device__ __forceinline__ void tile_group_pair(const LeafView &lv, const typename S::P &p,
                                                const typename S::Rec *__restrict__ rec, typename S::Rec2 *buf,
                                                int64_t a, int lo, int g0, int hi, int lane) {
    using Rec = typename S::Rec;
    static_assert(!S::kCons && !S::kGasOnly && !S::kTag, "packed sweep: gravity-type stages only");
    const unsigned below = lanemask_lt();
    const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
    const int i = g0 + lane;
    const bool act = i < hi;
    const Rec ri = rec[act ? i : g0];
    typename S::I2 st;
    S::init2(p, st, ri);
    float bl0 = ri.x, bl1 = ri.y, bl2 = ri.z, bh0 = ri.x, bh1 = ri.y, bh2 = ri.z;
    float hm = lv.pos[act ? i : g0].w;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bl0 = fminf(bl0, __shfl_xor_sync(CRK_FULL_MASK, bl0, o));
        bl1 = fminf(bl1, __shfl_xor_sync(CRK_FULL_MASK, bl1, o));
        bl2 = fminf(bl2, __shfl_xor_sync(CRK_FULL_MASK, bl2, o));
        bh0 = fmaxf(bh0, __shfl_xor_sync(CRK_FULL_MASK, bh0, o));
        bh1 = fmaxf(bh1, __shfl_xor_sync(CRK_FULL_MASK, bh1, o));
        bh2 = fmaxf(bh2, __shfl_xor_sync(CRK_FULL_MASK, bh2, o));
        hm = fmaxf(hm, __shfl_xor_sync(CRK_FULL_MASK, hm, o));
    }
    const float far = 2.0f * S::leaf_cut(p, hm, hm) + 1.0f;
    const Rec dummy = S::far_dummy(bh0 + far, bh1 + far, bh2 + far);
    // sweep once at least `depth` candidates are compacted (the buffer holds depth + 31 + 1 dummy)
    const int depth = lv.depth >= 64 ? (lv.depth >= 96 ? 96 : 64) : 32;
    auto sweep = [&](int cnt) {
        if (cnt & 1) {
            if (lane == 0) S::put2(buf, cnt, dummy);
            ++cnt;
        }
        __syncwarp();
        // unrolled: independent packed pairs interleave their dependent chains (Horner, rsqrt);
        // on the 2x256^3 box gravity and its adjoint took 28.2 and 48.8 ms rolled, 26.6 and
        // 46.9 ms unrolled by 4, 26.4 and 46.4 ms by 8
#pragma unroll 8
        for (int k = 0; k < (cnt >> 1); ++k) S::template interact2<kCount>(p, st, buf[k]);
        __syncwarp();
    };
    int cnt = 0;
    unsigned long long swept = 0;  // counting runs: candidates swept
    for (int e = ib; e < ie; ++e) {
        const crk_image im = lv.img[e];
        const int jlo = lv.leaf_start[im.b];
        const int jhi = lv.leaf_start[im.b + 1];
        {
            const float *bb = lv.bbox + 6 * (int64_t)im.b;
            float gx = fmaxf(fmaxf(im.sx - bh0, bl0 - (im.sx + (bb[3] - bb[0]))), 0.f);
            float gy = fmaxf(fmaxf(im.sy - bh1, bl1 - (im.sy + (bb[4] - bb[1]))), 0.f);
            float gz = fmaxf(fmaxf(im.sz - bh2, bl2 - (im.sz + (bb[5] - bb[2]))), 0.f);
            float cut = S::leaf_cut(p, hm, lv.hmax[im.b]);
            if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut * cut * 1.0001f + 1e-6f)) continue;
        }
        for (int j0 = jlo; j0 < jhi; j0 += 32) {
            const int j = j0 + lane;
            const bool jv = j < jhi;
            Rec rj;
            bool keep = false;
            if (jv) {
                rj = rec[j];
                S::shift(rj, im.sx, im.sy, im.sz);
                float dx = fmaxf(fmaxf(bl0 - rj.x, rj.x - bh0), 0.f);
                float dy = fmaxf(fmaxf(bl1 - rj.y, rj.y - bh1), 0.f);
                float dz = fmaxf(fmaxf(bl2 - rj.z, rj.z - bh2), 0.f);
                float cut = S::box_cut(p, hm, rj);
                keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut * cut * 1.0001f + 1e-6f;
            }
            const unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
            if (keep) S::put2(buf, cnt + __popc(m & below), rj);
            cnt += __popc(m);
            if (cnt >= depth) {
                sweep(cnt);
                if (kCount) swept += cnt;
                cnt = 0;
            }
        }
    }
    sweep(cnt);
    if (kCount) swept += cnt;
    if (act) S::finish2(p, st, lv.korder ? i : lv.kperm[i]);
    if (kCount) {
        int c = act ? st.cnt - 1 : 0;  // the self pair (r = 0) is always in range
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(CRK_FULL_MASK, c, o);
        if (lane == 0 && c) atomicAdd(p.count, (unsigned long long)c);
        const unsigned long long na = __popc(__ballot_sync(CRK_FULL_MASK, act));
        if (lane == 0 && p.swept) atomicAdd(p.swept, swept * na);
    }
}

// Split tiles for the packed gravity sweeps (CRK_VARIANT_SPLIT8).  The warp
// compacts the candidates within the cut of its 32-particle group (an RCB cell
// of the leaf) once, into a per-warp buffer in global memory (its working set
// stays in L2), then sweeps that buffer once for each of the group's four
// 8-particle RCB sub-cells: only the candidates within the cut of the
// sub-cell's box are kept (compacted into shared memory), and the 4 lanes of
// each of the sub-cell's 8 i-particles take every 4th packed candidate pair,
// so the lanes stay balanced; their partial sums are added by shuffles at the
// end.  A sub-cell box is about a quarter of the group's volume, so a larger
// share of the evaluated pairs lies within r_c.  A group whose candidates
// overflow the buffer (gcap) is swept as plain tiles.
template <class S, bool kCount>
__global__ void __launch_bounds__(kThreads) pair_kernel_split(LeafView lv, typename S::P p,
                                                              const typename S::Rec *__restrict__ rec,
                                                              typename S::Rec *__restrict__ gbuf, int gcap) {
    using Rec = typename S::Rec;
    using Rec2 = typename S::Rec2;
    static_assert(S::kPair && !S::kCons && !S::kGasOnly, "split sweeps: packed gravity-type stages only");
    __shared__ __align__(16) Rec sbuf[kWarps][kCapPair];
    __shared__ int64_t leaf_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Rec2 *buf = reinterpret_cast<Rec2 *>(sbuf[warp]);
    Rec *gb = gbuf + ((size_t)blockIdx.x * kWarps + warp) * (size_t)gcap;
    const unsigned below = lanemask_lt();
    const int depth = lv.depth >= 64 ? (lv.depth >= 96 ? 96 : 64) : 64;  // at least 64: 8 pairs per split lane
    for (int64_t a = next_leaf(lv, -1, &leaf_slot); a < lv.n_leaves; a = next_leaf(lv, a, &leaf_slot)) {
        const int lo = lv.leaf_start[a], hi = lv.leaf_start[a + 1];
        const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
        for (int g0 = lo + warp * 32; g0 < hi; g0 += kWarps * 32) {
            // ---- the group's candidates into the per-warp buffer
            const int i = g0 + lane;
            const Rec ri = rec[i < hi ? i : g0];
            float bl0 = ri.x, bl1 = ri.y, bl2 = ri.z, bh0 = ri.x, bh1 = ri.y, bh2 = ri.z;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                bl0 = fminf(bl0, __shfl_xor_sync(CRK_FULL_MASK, bl0, o));
                bl1 = fminf(bl1, __shfl_xor_sync(CRK_FULL_MASK, bl1, o));
                bl2 = fminf(bl2, __shfl_xor_sync(CRK_FULL_MASK, bl2, o));
                bh0 = fmaxf(bh0, __shfl_xor_sync(CRK_FULL_MASK, bh0, o));
                bh1 = fmaxf(bh1, __shfl_xor_sync(CRK_FULL_MASK, bh1, o));
                bh2 = fmaxf(bh2, __shfl_xor_sync(CRK_FULL_MASK, bh2, o));
            }
            const float cut = S::leaf_cut(p, 0.f, 0.f);
            const float cut2 = cut * cut * 1.0001f + 1e-6f;
            int cnt = 0;
            bool ovf = false;
            for (int e = ib; e < ie && !ovf; ++e) {
                const crk_image im = lv.img[e];
                const int jlo = lv.leaf_start[im.b], jhi = lv.leaf_start[im.b + 1];
                {
                    const float *bb = lv.bbox + 6 * (int64_t)im.b;
                    float gx = fmaxf(fmaxf(im.sx - bh0, bl0 - (im.sx + (bb[3] - bb[0]))), 0.f);
                    float gy = fmaxf(fmaxf(im.sy - bh1, bl1 - (im.sy + (bb[4] - bb[1]))), 0.f);
                    float gz = fmaxf(fmaxf(im.sz - bh2, bl2 - (im.sz + (bb[5] - bb[2]))), 0.f);
                    if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut2)) continue;
                }
                for (int j0 = jlo; j0 < jhi; j0 += 32) {
                    const int j = j0 + lane;
                    Rec rj;
                    bool keep = false;
                    if (j < jhi) {
                        rj = rec[j];
                        S::shift(rj, im.sx, im.sy, im.sz);
                        float dx = fmaxf(fmaxf(bl0 - rj.x, rj.x - bh0), 0.f);
                        float dy = fmaxf(fmaxf(bl1 - rj.y, rj.y - bh1), 0.f);
                        float dz = fmaxf(fmaxf(bl2 - rj.z, rj.z - bh2), 0.f);
                        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut2;
                    }
                    const unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
                    if (cnt + __popc(m) > gcap) {
                        ovf = true;
                        break;
                    }
                    if (keep) gb[cnt + __popc(m & below)] = rj;
                    cnt += __popc(m);
                }
            }
            if (ovf) {  // a dense group: plain tiles
                tile_group_pair<S, kCount>(lv, p, rec, buf, a, lo, g0, hi, lane);
                __syncwarp();
                continue;
            }
            __syncwarp();  // the buffer's stores are visible to the whole warp
            // ---- the four sub-cells of 8: 4 lanes per i, each taking every 4th packed pair
            const int il = lane >> 2, sp = lane & 3;
            for (int c0 = g0; c0 < g0 + 32 && c0 < hi; c0 += 8) {
                const int ii = c0 + il;
                const bool iact = ii < hi;
                const Rec rs = rec[iact ? ii : c0];
                float sl0 = rs.x, sl1 = rs.y, sl2 = rs.z, sh0 = rs.x, sh1 = rs.y, sh2 = rs.z;
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {  // over the 8 i of the sub-cell
                    sl0 = fminf(sl0, __shfl_xor_sync(CRK_FULL_MASK, sl0, o));
                    sl1 = fminf(sl1, __shfl_xor_sync(CRK_FULL_MASK, sl1, o));
                    sl2 = fminf(sl2, __shfl_xor_sync(CRK_FULL_MASK, sl2, o));
                    sh0 = fmaxf(sh0, __shfl_xor_sync(CRK_FULL_MASK, sh0, o));
                    sh1 = fmaxf(sh1, __shfl_xor_sync(CRK_FULL_MASK, sh1, o));
                    sh2 = fmaxf(sh2, __shfl_xor_sync(CRK_FULL_MASK, sh2, o));
                }
                const float far = 2.0f * cut + 1.0f;
                const Rec dummy = S::far_dummy(sh0 + far, sh1 + far, sh2 + far);
                typename S::I2 st;
                S::init2(p, st, rs);
                unsigned long long swept = 0;
                int bc = 0;
                auto sweep = [&](int n) {
                    if (n & 1) {
                        if (lane == 0) S::put2(buf, n, dummy);
                        ++n;
                    }
                    __syncwarp();
                    for (int k = sp; k < (n >> 1); k += 4) S::template interact2<kCount>(p, st, buf[k]);
                    __syncwarp();
                };
                for (int q0 = 0; q0 < cnt; q0 += 32) {
                    const int q = q0 + lane;
                    Rec rj;
                    bool keep = false;
                    if (q < cnt) {
                        rj = gb[q];
                        float dx = fmaxf(fmaxf(sl0 - rj.x, rj.x - sh0), 0.f);
                        float dy = fmaxf(fmaxf(sl1 - rj.y, rj.y - sh1), 0.f);
                        float dz = fmaxf(fmaxf(sl2 - rj.z, rj.z - sh2), 0.f);
                        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut2;
                    }
                    const unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
                    if (keep) S::put2(buf, bc + __popc(m & below), rj);
                    bc += __popc(m);
                    if (bc >= depth) {
                        sweep(bc);
                        if (kCount) swept += bc;
                        bc = 0;
                    }
                }
                sweep(bc);
                if (kCount) swept += bc;
                S::combine2(st, 1);
                S::combine2(st, 2);
                if (sp == 0 && iact) S::finish2(p, st, lv.korder ? ii : lv.kperm[ii]);
                if (kCount) {
                    int c = (sp == 0 && iact) ? st.cnt - 1 : 0;  // the self pair (r = 0) is always in range
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(CRK_FULL_MASK, c, o);
                    if (lane == 0 && c) atomicAdd(p.count, (unsigned long long)c);
                    const unsigned long long na = __popc(__ballot_sync(CRK_FULL_MASK, sp == 0 && iact));
                    if (lane == 0 && p.swept) atomicAdd(p.swept, swept * na);
                }
            }
            __syncwarp();  // the buffer is reused by the next group
        }
    }
}

// The paper's "half-warp" leaf-pair scheme (Sec. 5.3), as autotuner arms for
// the gravity stages.  Lanes 0-15 hold 16 particles of leaf A, lanes 16-31 16
// particles of leaf B (shifted into A's frame); in step s lane l and lane
// 16 + (l ^ s) exchange their particles and each evaluates the interaction on
// its own particle, so every A-B pair is evaluated once in each direction in
// the same step.  Each unordered leaf-pair image is visited once (entries with
// b > a, or b = a with a positive shift, and the leaf with itself); the
// partial sums of each tile are added to the outputs atomically, so the
// result is exact up to the order of the FP32 additions.  kEx selects how the
// partner's particle reaches a lane: 0 register shuffle, 1 shared memory,
// 2 a second load of the partner's record.
template <class Rec>
__device__ __forceinline__ Rec shfl_rec(const Rec &r, int src) {
    Rec o;
    const float *a = reinterpret_cast<const float *>(&r);
    float *b = reinterpret_cast<float *>(&o);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(Rec) / sizeof(float)); ++k) b[k] = __shfl_sync(CRK_FULL_MASK, a[k], src);
    return o;
}

__device__ __forceinline__ bool positive_shift(float sx, float sy, float sz) {
    return sx > 0.f || (sx == 0.f && (sy > 0.f || (sy == 0.f && sz > 0.f)));
}

// Gas stages (the Acceleration and Energy passes) use the gas prefix of each
// leaf and the tile cut h_max(A slice) + h_max(B slice); their conservation
// sums are taken afterwards from the finished outputs (halfwarp_cons_kernel).
template <class S, bool kCount, int kEx>
__global__ void __launch_bounds__(kThreads) pair_kernel_halfwarp(LeafView lv, typename S::P p,
                                                                 const typename S::Rec *__restrict__ rec,
                                                                 double *__restrict__) {
    using Rec = typename S::Rec;
    static_assert(S::kHalfWarp, "half-warp arms: stages with atomic partial sums");
    __shared__ __align__(16) Rec xbuf[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const float rc = S::leaf_cut(p, 0.f, 0.f);
    __shared__ int64_t leaf_slot;
    for (int64_t a = next_leaf(lv, -1, &leaf_slot); a < lv.n_leaves; a = next_leaf(lv, a, &leaf_slot)) {
        const int alo = lv.leaf_start[a];
        const int ahi = S::kGasOnly ? alo + lv.leaf_ngas[a] : lv.leaf_start[a + 1];
        const int nsa = (ahi - alo + 15) >> 4;
        const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
        int t0 = warp;  // tiles are dealt to the block's warps in turn across the leaf's entries
        for (int e = ib; e < ie; ++e) {
            const crk_image im = lv.img[e];
            const int b = im.b;
            const bool self = b == a && im.sx == 0.f && im.sy == 0.f && im.sz == 0.f;
            if (b < a || (b == a && !self && !positive_shift(im.sx, im.sy, im.sz))) continue;
            const int blo = lv.leaf_start[b];
            const int bhi = S::kGasOnly ? blo + lv.leaf_ngas[b] : lv.leaf_start[b + 1];
            const int nsb = (bhi - blo + 15) >> 4;
            const int ntile = nsa * nsb;
            int t = t0;
            for (; t < ntile; t += kWarps) {
                const int u = t / nsb, v = t - u * nsb;
                if (self && v < u) continue;
                const bool diag = self && u == v;  // the same 16 particles in both halves: only A accumulates
                const int idx = half ? blo + 16 * v + hl : alo + 16 * u + hl;
                const bool valid = idx < (half ? bhi : ahi);
                Rec r = rec[valid ? idx : (half ? blo : alo)];
                if (half) S::shift(r, im.sx, im.sy, im.sz);
                // slice boxes (valid lanes only), then the whole tile against the cut (warp-uniform)
                float l0 = valid ? r.x : INFINITY, l1 = valid ? r.y : INFINITY, l2 = valid ? r.z : INFINITY;
                float h0 = valid ? r.x : -INFINITY, h1 = valid ? r.y : -INFINITY, h2 = valid ? r.z : -INFINITY;
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    l0 = fminf(l0, __shfl_xor_sync(CRK_FULL_MASK, l0, o));
                    l1 = fminf(l1, __shfl_xor_sync(CRK_FULL_MASK, l1, o));
                    l2 = fminf(l2, __shfl_xor_sync(CRK_FULL_MASK, l2, o));
                    h0 = fmaxf(h0, __shfl_xor_sync(CRK_FULL_MASK, h0, o));
                    h1 = fmaxf(h1, __shfl_xor_sync(CRK_FULL_MASK, h1, o));
                    h2 = fmaxf(h2, __shfl_xor_sync(CRK_FULL_MASK, h2, o));
                }
                float cut = rc;
                if constexpr (S::kGasOnly) {  // h_max of each slice: the cut is their sum
                    float hs = valid ? lv.pos[idx].w : 0.0f;
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) hs = fmaxf(hs, __shfl_xor_sync(CRK_FULL_MASK, hs, o));
                    cut = S::leaf_cut(p, hs, __shfl_xor_sync(CRK_FULL_MASK, hs, 16));
                }
                const float ol0 = __shfl_xor_sync(CRK_FULL_MASK, l0, 16), ol1 = __shfl_xor_sync(CRK_FULL_MASK, l1, 16),
                            ol2 = __shfl_xor_sync(CRK_FULL_MASK, l2, 16), oh0 = __shfl_xor_sync(CRK_FULL_MASK, h0, 16),
                            oh1 = __shfl_xor_sync(CRK_FULL_MASK, h1, 16), oh2 = __shfl_xor_sync(CRK_FULL_MASK, h2, 16);
                const float gx = fmaxf(fmaxf(ol0 - h0, l0 - oh0), 0.f), gy = fmaxf(fmaxf(ol1 - h1, l1 - oh1), 0.f),
                            gz = fmaxf(fmaxf(ol2 - h2, l2 - oh2), 0.f);
                // empty halves give NaN/inf gaps: those tiles are skipped too
                if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut * cut * 1.0001f + 1e-6f)) continue;
                if (!valid) {  // a particle outside every cut that contributes exact zeros
                    r = S::far_dummy(1e15f, 1e15f, 1e15f);
                }
                if constexpr (kEx == 1) {
                    __syncwarp();
                    xbuf[warp][lane] = r;
                    __syncwarp();
                }
                typename S::I st;
                S::init(p, st, r, a, 0, lane, 0);
                const bool acc = valid && !(diag && half);
#pragma unroll 2
                for (int s = 0; s < 16; ++s) {
                    const int pl = half ? (hl ^ s) : 16 + (hl ^ s);
                    Rec q;
                    if constexpr (kEx == 0) {
                        q = shfl_rec(r, pl);
                    } else if constexpr (kEx == 1) {
                        q = xbuf[warp][pl];
                    } else {
                        const int pi = pl < 16 ? alo + 16 * u + pl : (diag ? alo + 16 * u : blo + 16 * v) + (pl - 16);
                        const bool pv = pi < (pl < 16 || diag ? ahi : bhi);
                        if (pv) {
                            q = rec[pi];
                            if (pl >= 16 && !diag) S::shift(q, im.sx, im.sy, im.sz);
                        } else {
                            q = S::far_dummy(1e15f, 1e15f, 1e15f);
                        }
                    }
                    if (acc) S::template interact<kCount>(p, st, r, q);
                }
                if (acc) S::flush(p, st, r, stage_index(lv, idx));
                if (kCount) {
                    int c = acc ? st.cnt - (diag ? 1 : 0) : 0;  // the self pair of a diagonal tile
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(CRK_FULL_MASK, c, o);
                    if (lane == 0 && c) atomicAdd(p.count, (unsigned long long)c);
                }
            }
            t0 = t - ntile;  // continue the round robin in the next entry
        }
    }
}

// one i-group, tiles (packed sweep where the stage has one)
template <class S, bool kCount>
__device__ __forceinline__ void tile_group_any(const LeafView &lv, const typename S::P &p,
                                               const typename S::Rec *__restrict__ rec, typename S::Rec *buf,
                                               int64_t a, int lo, int g0, int hi, int lane, double cons_acc[4]) {
    if constexpr (S::kPair) {
        static_assert(sizeof(typename S::Rec2) == 2 * sizeof(typename S::Rec), "pair record layout");
        tile_group_pair<S, kCount>(lv, p, rec, reinterpret_cast<typename S::Rec2 *>(buf), a, lo, g0, hi, lane);
    } else {
        tile_group<S, kCount>(lv, p, rec, buf, a, lo, g0, hi, lane, cons_acc);
    }
}

// Per-block partial of the FP64 conservation sums in a fixed order (reduced by
// cons_reduce_kernel: deterministic for a fixed assignment of work to blocks).
__device__ __forceinline__ void cons_block_partial(double (*cons_sh)[4], const double cons_acc[4],
                                                   double *__restrict__ cons_part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) cons_sh[warp][k] = cons_acc[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += cons_sh[w][k];
            cons_part[4 * (int64_t)blockIdx.x + k] = t;
        }
}

// Tiles, one block per i-leaf (or leaves from the persistent queue); the
// block's kW warps take the leaf's groups in turn (kW = 2: the packed gravity
// sweeps' narrow launch shape, two groups of a 128-leaf per warp).
template <class S, bool kCount, int kW = kWarps>
__global__ void __launch_bounds__(32 * kW) pair_kernel(LeafView lv, typename S::P p,
                                                       const typename S::Rec *__restrict__ rec,
                                                       double *__restrict__ cons_part) {
    using Rec = typename S::Rec;
    static_assert(kW == kWarps || !S::kCons, "conservation partials assume kWarps warps per block");
    __shared__ __align__(16) Rec buf[kW][S::kPair ? kCapPair : kCap];
    __shared__ double cons_sh[kWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double cons_acc[4] = {0.0, 0.0, 0.0, 0.0};
    __shared__ int64_t leaf_slot;
    for (int64_t a = next_leaf(lv, -1, &leaf_slot); a < lv.n_leaves; a = next_leaf(lv, a, &leaf_slot)) {
        const int lo = lv.leaf_start[a];
        const int hi = S::kGasOnly ? lo + lv.leaf_ngas[a] : lv.leaf_start[a + 1];
        for (int g0 = lo + warp * 32; g0 < hi; g0 += kW * 32)
            tile_group_any<S, kCount>(lv, p, rec, buf[warp], a, lo, g0, hi, lane, cons_acc);
    }
    if constexpr (S::kCons) {
        if (cons_part) cons_block_partial(cons_sh, cons_acc, cons_part);
    }
}

// Group table of one set of leaves: groups of 32 consecutive kernel-order
// particles (gas only for gas stages), numbered leaf by leaf.
struct GroupTable {
    const int32_t *gstart;   // [n_leaves + 1] first group of each leaf
    const int32_t *gleaf;    // [groups] leaf of each group
    int64_t groups;          // capacity of the group arrays
    const int32_t *dgroups;  // device: the groups of this build (<= groups), or NULL for all
};

// groups of a build: the device count when the arrays have room for more
__device__ __forceinline__ int64_t group_count(int64_t cap, const int32_t *dgroups) {
    if (!dgroups) return cap;
    const int64_t g = *dgroups;
    return g < cap ? g : cap;
}

// Tiles, one warp per i-group: every warp works even where a leaf holds fewer
// groups than a block has warps (gas stages: a leaf of 128 holds about 64 gas).
template <class S, bool kCount>
__global__ void __launch_bounds__(kThreads) pair_group_kernel(LeafView lv, typename S::P p,
                                                              const typename S::Rec *__restrict__ rec,
                                                              GroupTable gt, double *__restrict__ cons_part) {
    using Rec = typename S::Rec;
    __shared__ __align__(16) Rec buf[kWarps][kCap];
    __shared__ double cons_sh[kWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double cons_acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t ngroups = group_count(gt.groups, gt.dgroups);
    for (int64_t grp = next_group(lv, -1, lane); grp < ngroups; grp = next_group(lv, grp, lane)) {
        const int64_t a = gt.gleaf[grp];
        const int lo = lv.leaf_start[a];
        const int hi = S::kGasOnly ? lo + lv.leaf_ngas[a] : lv.leaf_start[a + 1];
        const int g0 = lo + 32 * (int)(grp - gt.gstart[a]);
        tile_group_any<S, kCount>(lv, p, rec, buf[warp], a, lo, g0, hi, lane, cons_acc);
    }
    if constexpr (S::kCons) {
        if (cons_part) cons_block_partial(cons_sh, cons_acc, cons_part);
    }
}


// Tiles with sub-warp i-groups: the warp's 32 i-particles form 32/G groups of
// G consecutive (Z-ordered) particles, each with its own box and its own
// compacted candidate buffer; lane l sweeps the buffer of group l/G.  Smaller
// groups have smaller boxes, so a larger share of the swept pairs is in range.
// Within one 8-lane phase of a shared-memory load every lane reads the same
// record (G >= 8), so the sweep stays a broadcast.
template <class S, int G, bool kCount>
__global__ void __launch_bounds__(kThreads) pair_kernel_sub(LeafView lv, typename S::P p,
                                                            const typename S::Rec *__restrict__ rec,
                                                            double *__restrict__ cons_part) {
    using Rec = typename S::Rec;
    constexpr int NS = 32 / G;
    __shared__ Rec buf[kWarps][NS][kCap];
    __shared__ double cons_sh[kWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sg = lane / G;
    const unsigned below = lanemask_lt();
    double cons_acc[4] = {0.0, 0.0, 0.0, 0.0};
    __shared__ int64_t leaf_slot;
    for (int64_t a = next_leaf(lv, -1, &leaf_slot); a < lv.n_leaves; a = next_leaf(lv, a, &leaf_slot)) {
        const int lo = lv.leaf_start[a];
        const int hi = S::kGasOnly ? lo + lv.leaf_ngas[a] : lv.leaf_start[a + 1];
        const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
        for (int g0 = lo + warp * 32; g0 < hi; g0 += kWarps * 32) {
            const int i = g0 + lane;
            const bool act = i < hi;
            const Rec ri = rec[act ? i : g0];
            typename S::I st;
            S::init(p, st, ri, a, (g0 - lo) >> 5, lane, stage_index(lv, act ? i : g0));
            // group boxes (empty for groups without active lanes) and largest h
            float l0 = act ? ri.x : INFINITY, l1 = act ? ri.y : INFINITY, l2 = act ? ri.z : INFINITY;
            float h0 = act ? ri.x : -INFINITY, h1 = act ? ri.y : -INFINITY, h2 = act ? ri.z : -INFINITY;
            float hm = act ? lv.pos[i].w : 0.0f;
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                l0 = fminf(l0, __shfl_xor_sync(CRK_FULL_MASK, l0, o));
                l1 = fminf(l1, __shfl_xor_sync(CRK_FULL_MASK, l1, o));
                l2 = fminf(l2, __shfl_xor_sync(CRK_FULL_MASK, l2, o));
                h0 = fmaxf(h0, __shfl_xor_sync(CRK_FULL_MASK, h0, o));
                h1 = fmaxf(h1, __shfl_xor_sync(CRK_FULL_MASK, h1, o));
                h2 = fmaxf(h2, __shfl_xor_sync(CRK_FULL_MASK, h2, o));
                hm = fmaxf(hm, __shfl_xor_sync(CRK_FULL_MASK, hm, o));
            }
            float bl[NS][3], bh[NS][3], bhm[NS];
            float ul0 = INFINITY, ul1 = INFINITY, ul2 = INFINITY, uh0 = -INFINITY, uh1 = -INFINITY, uh2 = -INFINITY,
                  uhm = 0.0f;
#pragma unroll
            for (int t = 0; t < NS; ++t) {
                bl[t][0] = __shfl_sync(CRK_FULL_MASK, l0, t * G);
                bl[t][1] = __shfl_sync(CRK_FULL_MASK, l1, t * G);
                bl[t][2] = __shfl_sync(CRK_FULL_MASK, l2, t * G);
                bh[t][0] = __shfl_sync(CRK_FULL_MASK, h0, t * G);
                bh[t][1] = __shfl_sync(CRK_FULL_MASK, h1, t * G);
                bh[t][2] = __shfl_sync(CRK_FULL_MASK, h2, t * G);
                bhm[t] = __shfl_sync(CRK_FULL_MASK, hm, t * G);
                ul0 = fminf(ul0, bl[t][0]); ul1 = fminf(ul1, bl[t][1]); ul2 = fminf(ul2, bl[t][2]);
                uh0 = fmaxf(uh0, bh[t][0]); uh1 = fmaxf(uh1, bh[t][1]); uh2 = fmaxf(uh2, bh[t][2]);
                uhm = fmaxf(uhm, bhm[t]);
            }
            int cnt[NS];
#pragma unroll
            for (int t = 0; t < NS; ++t) cnt[t] = 0;
            auto sweep = [&]() {
                __syncwarp();
                int kmax = 0, mine = 0;
#pragma unroll
                for (int t = 0; t < NS; ++t) {
                    kmax = max(kmax, cnt[t]);
                    if (t == sg) mine = cnt[t];
                }
                for (int k = 0; k < kmax; ++k)
                    if (k < mine) S::template interact<kCount>(p, st, ri, buf[warp][sg][k]);
#pragma unroll
                for (int t = 0; t < NS; ++t) cnt[t] = 0;
                __syncwarp();
            };
            for (int e = ib; e < ie; ++e) {
                const crk_image im = lv.img[e];
                const int jlo = lv.leaf_start[im.b];
                const int jhi = S::kGasOnly ? jlo + lv.leaf_ngas[im.b] : lv.leaf_start[im.b + 1];
                {
                    const float *bb = lv.bbox + 6 * (int64_t)im.b;
                    float gx = fmaxf(fmaxf(im.sx - uh0, ul0 - (im.sx + (bb[3] - bb[0]))), 0.f);
                    float gy = fmaxf(fmaxf(im.sy - uh1, ul1 - (im.sy + (bb[4] - bb[1]))), 0.f);
                    float gz = fmaxf(fmaxf(im.sz - uh2, ul2 - (im.sz + (bb[5] - bb[2]))), 0.f);
                    float cut = S::leaf_cut(p, uhm, lv.hmax[im.b]);
                    if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut * cut * 1.0001f + 1e-6f)) continue;
                }
                for (int j0 = jlo; j0 < jhi; j0 += 32) {
                    const int j = j0 + lane;
                    const bool jv = j < jhi;
                    Rec rj;
                    if (jv) {
                        rj = rec[j];
                        S::shift(rj, im.sx, im.sy, im.sz);
                        if constexpr (S::kTag) S::tag(rj, e - ib, j - jlo);
                    }
                    bool full = false;
#pragma unroll
                    for (int t = 0; t < NS; ++t) {
                        bool keep = false;
                        if (jv) {
                            float dx = fmaxf(fmaxf(bl[t][0] - rj.x, rj.x - bh[t][0]), 0.f);
                            float dy = fmaxf(fmaxf(bl[t][1] - rj.y, rj.y - bh[t][1]), 0.f);
                            float dz = fmaxf(fmaxf(bl[t][2] - rj.z, rj.z - bh[t][2]), 0.f);
                            float cut = S::box_cut(p, bhm[t], rj);
                            keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut * cut * 1.0001f + 1e-6f;
                        }
                        const unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
                        if (keep) buf[warp][t][cnt[t] + __popc(m & below)] = rj;
                        cnt[t] += __popc(m);
                        full |= cnt[t] >= 32;
                    }
                    if (full) sweep();
                }
            }
            sweep();
            if (act) S::finish(p, st, ri, lv.korder ? i : lv.kperm[i], i);
            if constexpr (S::kCons) {
                double cc[4] = {0.0, 0.0, 0.0, 0.0};
                if (act) S::cons_terms(p, st, ri, lv.korder ? i : lv.kperm[i], cc);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cc[k] += __shfl_xor_sync(CRK_FULL_MASK, cc[k], o);
                    cons_acc[k] += cc[k];
                }
            }
            if (kCount) {
                int cn = act ? st.cnt - 1 : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(CRK_FULL_MASK, cn, o);
                if (lane == 0 && cn) atomicAdd(p.count, (unsigned long long)cn);
            }
        }
    }
    if constexpr (S::kCons) {
        if (cons_part) {
            if (lane == 0)
                for (int k = 0; k < 4; ++k) cons_sh[warp][k] = cons_acc[k];
            __syncthreads();
            if (threadIdx.x == 0)
                for (int k = 0; k < 4; ++k) {
                    double t = 0.0;
                    for (int w = 0; w < kWarps; ++w) t += cons_sh[w][k];
                    cons_part[4 * (int64_t)blockIdx.x + k] = t;
                }
        }
    }
}


// Tiles with two 16-particle i-groups per warp for the packed gravity stages
// (kPair): each half-warp's group (an RCB cell of its leaf) has its own box
// and its own buffer of field-interleaved candidate pairs, swept two
// candidates per lane step with f32x2 arithmetic; an odd tail is padded with
// a massless dummy outside every cut.  A 16-particle cell prunes ~22% more of
// the candidates than its 32-particle parent at r_c = 3.
template <class S, bool kCount>
__global__ void __launch_bounds__(kThreads) pair_kernel_sub_pair(LeafView lv, typename S::P p,
                                                                 const typename S::Rec *__restrict__ rec,
                                                                 double *__restrict__ cons_part) {
    using Rec = typename S::Rec;
    using Rec2 = typename S::Rec2;
    constexpr int G = 16, NS = 2;
    __shared__ __align__(16) Rec2 buf[kWarps][NS][kCap / 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sg = lane / G;
    const unsigned below = lanemask_lt();
    (void)cons_part;
    __shared__ int64_t leaf_slot;
    for (int64_t a = next_leaf(lv, -1, &leaf_slot); a < lv.n_leaves; a = next_leaf(lv, a, &leaf_slot)) {
        const int lo = lv.leaf_start[a];
        const int hi = lv.leaf_start[a + 1];
        const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
        for (int g0 = lo + warp * 32; g0 < hi; g0 += kWarps * 32) {
            const int i = g0 + lane;
            const bool act = i < hi;
            const Rec ri = rec[act ? i : g0];
            typename S::I2 st;
            S::init2(p, st, ri);
            // group boxes (empty for groups without active lanes)
            float l0 = act ? ri.x : INFINITY, l1 = act ? ri.y : INFINITY, l2 = act ? ri.z : INFINITY;
            float h0 = act ? ri.x : -INFINITY, h1 = act ? ri.y : -INFINITY, h2 = act ? ri.z : -INFINITY;
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                l0 = fminf(l0, __shfl_xor_sync(CRK_FULL_MASK, l0, o));
                l1 = fminf(l1, __shfl_xor_sync(CRK_FULL_MASK, l1, o));
                l2 = fminf(l2, __shfl_xor_sync(CRK_FULL_MASK, l2, o));
                h0 = fmaxf(h0, __shfl_xor_sync(CRK_FULL_MASK, h0, o));
                h1 = fmaxf(h1, __shfl_xor_sync(CRK_FULL_MASK, h1, o));
                h2 = fmaxf(h2, __shfl_xor_sync(CRK_FULL_MASK, h2, o));
            }
            float bl[NS][3], bh[NS][3];
            float ul0 = INFINITY, ul1 = INFINITY, ul2 = INFINITY, uh0 = -INFINITY, uh1 = -INFINITY, uh2 = -INFINITY;
#pragma unroll
            for (int t = 0; t < NS; ++t) {
                bl[t][0] = __shfl_sync(CRK_FULL_MASK, l0, t * G);
                bl[t][1] = __shfl_sync(CRK_FULL_MASK, l1, t * G);
                bl[t][2] = __shfl_sync(CRK_FULL_MASK, l2, t * G);
                bh[t][0] = __shfl_sync(CRK_FULL_MASK, h0, t * G);
                bh[t][1] = __shfl_sync(CRK_FULL_MASK, h1, t * G);
                bh[t][2] = __shfl_sync(CRK_FULL_MASK, h2, t * G);
                ul0 = fminf(ul0, bl[t][0]); ul1 = fminf(ul1, bl[t][1]); ul2 = fminf(ul2, bl[t][2]);
                uh0 = fmaxf(uh0, bh[t][0]); uh1 = fmaxf(uh1, bh[t][1]); uh2 = fmaxf(uh2, bh[t][2]);
            }
            const float cut = S::leaf_cut(p, 0.0f, 0.0f);
            const float far = 2.0f * cut + 1.0f;
            const Rec dummy = S::far_dummy(uh0 + far, uh1 + far, uh2 + far);
            int cnt[NS] = {0, 0};
            unsigned long long swept = 0;  // counting runs: candidate evaluations of this lane's group
            auto sweep = [&]() {
                // pad odd counts, then every half-warp sweeps its own buffer in pairs
                if (kCount) swept += (unsigned long long)(sg ? cnt[1] : cnt[0]);
                if (lane == 0 && (cnt[0] & 1)) S::put2(buf[warp][0], cnt[0], dummy);
                if (lane == 1 && (cnt[1] & 1)) S::put2(buf[warp][1], cnt[1], dummy);
#pragma unroll
                for (int t = 0; t < NS; ++t) cnt[t] = (cnt[t] + 1) & ~1;
                __syncwarp();
                const int kmax = max(cnt[0], cnt[1]) >> 1, mine = (sg ? cnt[1] : cnt[0]) >> 1;
                for (int k = 0; k < kmax; ++k)
                    if (k < mine) S::template interact2<kCount>(p, st, buf[warp][sg][k]);
#pragma unroll
                for (int t = 0; t < NS; ++t) cnt[t] = 0;
                __syncwarp();
            };
            for (int e = ib; e < ie; ++e) {
                const crk_image im = lv.img[e];
                const int jlo = lv.leaf_start[im.b];
                const int jhi = lv.leaf_start[im.b + 1];
                {
                    const float *bb = lv.bbox + 6 * (int64_t)im.b;
                    float gx = fmaxf(fmaxf(im.sx - uh0, ul0 - (im.sx + (bb[3] - bb[0]))), 0.f);
                    float gy = fmaxf(fmaxf(im.sy - uh1, ul1 - (im.sy + (bb[4] - bb[1]))), 0.f);
                    float gz = fmaxf(fmaxf(im.sz - uh2, ul2 - (im.sz + (bb[5] - bb[2]))), 0.f);
                    if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut * cut * 1.0001f + 1e-6f)) continue;
                }
                for (int j0 = jlo; j0 < jhi; j0 += 32) {
                    const int j = j0 + lane;
                    const bool jv = j < jhi;
                    Rec rj;
                    if (jv) {
                        rj = rec[j];
                        S::shift(rj, im.sx, im.sy, im.sz);
                    }
                    bool full = false;
#pragma unroll
                    for (int t = 0; t < NS; ++t) {
                        bool keep = false;
                        if (jv) {
                            float dx = fmaxf(fmaxf(bl[t][0] - rj.x, rj.x - bh[t][0]), 0.f);
                            float dy = fmaxf(fmaxf(bl[t][1] - rj.y, rj.y - bh[t][1]), 0.f);
                            float dz = fmaxf(fmaxf(bl[t][2] - rj.z, rj.z - bh[t][2]), 0.f);
                            keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut * cut * 1.0001f + 1e-6f;
                        }
                        const unsigned m = __ballot_sync(CRK_FULL_MASK, keep);
                        if (keep) S::put2(buf[warp][t], cnt[t] + __popc(m & below), rj);
                        cnt[t] += __popc(m);
                        full |= cnt[t] >= 32;
                    }
                    if (full) sweep();
                }
            }
            sweep();
            if (act) S::finish2(p, st, lv.korder ? i : lv.kperm[i]);
            if (kCount) {
                int cn = act ? st.cnt - 1 : 0;  // the self pair (r = 0) is always in range
                unsigned long long sw = act ? swept : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    cn += __shfl_xor_sync(CRK_FULL_MASK, cn, o);
                    sw += __shfl_xor_sync(CRK_FULL_MASK, sw, o);
                }
                if (lane == 0 && cn) atomicAdd(p.count, (unsigned long long)cn);
                if (lane == 0 && p.swept) atomicAdd(p.swept, sw);
            }
        }
    }
}

// Two 16-particle i-groups per warp with balanced sweeps: each half-warp has
// a ring buffer of candidates; a sweep consumes the same number of entries
// from both rings (as many as both have ready), so neither half idles while
// the other works.  Only when a ring is about to overflow, and at the end,
// is a sweep unbalanced.
constexpr int kRing = 128;  // entries per ring (power of two)

template <class S, bool kCount>
__global__ void __launch_bounds__(kThreads) pair_kernel_ring(LeafView lv, typename S::P p,
                                                             const typename S::Rec *__restrict__ rec,
                                                             double *__restrict__ cons_part) {
    using Rec = typename S::Rec;
    static_assert(!S::kCons, "the balanced sub-warp sweep has no conservation sums");
    __shared__ Rec ring[kWarps][2][kRing];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sg = lane >> 4;
    const unsigned below = lanemask_lt();
    __shared__ int64_t leaf_slot;
    for (int64_t a = next_leaf(lv, -1, &leaf_slot); a < lv.n_leaves; a = next_leaf(lv, a, &leaf_slot)) {
        const int lo = lv.leaf_start[a];
        const int hi = S::kGasOnly ? lo + lv.leaf_ngas[a] : lv.leaf_start[a + 1];
        const int ib = lv.img_start[a], ie = ib + lv.img_cnt[a];
        for (int g0 = lo + warp * 32; g0 < hi; g0 += kWarps * 32) {
            const int i = g0 + lane;
            const bool act = i < hi;
            const Rec ri = rec[act ? i : g0];
            typename S::I st;
            S::init(p, st, ri, a, (g0 - lo) >> 5, lane, stage_index(lv, act ? i : g0));
            float l0 = act ? ri.x : INFINITY, l1 = act ? ri.y : INFINITY, l2 = act ? ri.z : INFINITY;
            float h0 = act ? ri.x : -INFINITY, h1 = act ? ri.y : -INFINITY, h2 = act ? ri.z : -INFINITY;
            float hm = act ? lv.pos[i].w : 0.0f;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                l0 = fminf(l0, __shfl_xor_sync(CRK_FULL_MASK, l0, o));
                l1 = fminf(l1, __shfl_xor_sync(CRK_FULL_MASK, l1, o));
                l2 = fminf(l2, __shfl_xor_sync(CRK_FULL_MASK, l2, o));
                h0 = fmaxf(h0, __shfl_xor_sync(CRK_FULL_MASK, h0, o));
                h1 = fmaxf(h1, __shfl_xor_sync(CRK_FULL_MASK, h1, o));
                h2 = fmaxf(h2, __shfl_xor_sync(CRK_FULL_MASK, h2, o));
                hm = fmaxf(hm, __shfl_xor_sync(CRK_FULL_MASK, hm, o));
            }
            float bl[2][3], bh[2][3], bhm[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                bl[t][0] = __shfl_sync(CRK_FULL_MASK, l0, 16 * t);
                bl[t][1] = __shfl_sync(CRK_FULL_MASK, l1, 16 * t);
                bl[t][2] = __shfl_sync(CRK_FULL_MASK, l2, 16 * t);
                bh[t][0] = __shfl_sync(CRK_FULL_MASK, h0, 16 * t);
                bh[t][1] = __shfl_sync(CRK_FULL_MASK, h1, 16 * t);
                bh[t][2] = __shfl_sync(CRK_FULL_MASK, h2, 16 * t);
                bhm[t] = __shfl_sync(CRK_FULL_MASK, hm, 16 * t);
            }
            const float ul0 = fminf(bl[0][0], bl[1][0]), ul1 = fminf(bl[0][1], bl[1][1]), ul2 = fminf(bl[0][2], bl[1][2]);
            const float uh0 = fmaxf(bh[0][0], bh[1][0]), uh1 = fmaxf(bh[0][1], bh[1][1]), uh2 = fmaxf(bh[0][2], bh[1][2]);
            const float uhm = fmaxf(bhm[0], bhm[1]);
            unsigned head0 = 0, head1 = 0, tail0 = 0, tail1 = 0;  // warp-uniform ring counters
            // consume k0 entries of ring 0 (lanes 0-15) and k1 of ring 1 (lanes 16-31)
            auto sweep = [&](unsigned k0, unsigned k1) {
                __syncwarp();
                const unsigned kmax = k0 > k1 ? k0 : k1, mine = sg ? k1 : k0, h = sg ? head1 : head0;
                for (unsigned k = 0; k < kmax; ++k)
                    if (k < mine) S::template interact<kCount>(p, st, ri, ring[warp][sg][(h + k) & (kRing - 1)]);
                head0 += k0;
                head1 += k1;
                __syncwarp();
            };
            for (int e = ib; e < ie; ++e) {
                const crk_image im = lv.img[e];
                const int jlo = lv.leaf_start[im.b];
                const int jhi = S::kGasOnly ? jlo + lv.leaf_ngas[im.b] : lv.leaf_start[im.b + 1];
                {
                    const float *bb = lv.bbox + 6 * (int64_t)im.b;
                    float gx = fmaxf(fmaxf(im.sx - uh0, ul0 - (im.sx + (bb[3] - bb[0]))), 0.f);
                    float gy = fmaxf(fmaxf(im.sy - uh1, ul1 - (im.sy + (bb[4] - bb[1]))), 0.f);
                    float gz = fmaxf(fmaxf(im.sz - uh2, ul2 - (im.sz + (bb[5] - bb[2]))), 0.f);
                    float cut = S::leaf_cut(p, uhm, lv.hmax[im.b]);
                    if (!(fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= cut * cut * 1.0001f + 1e-6f)) continue;
                }
                for (int j0 = jlo; j0 < jhi; j0 += 32) {
                    const int j = j0 + lane;
                    const bool jv = j < jhi;
                    Rec rj;
                    bool keep[2] = {false, false};
                    if (jv) {
                        rj = rec[j];
                        S::shift(rj, im.sx, im.sy, im.sz);
                        if constexpr (S::kTag) S::tag(rj, e - ib, j - jlo);
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            float dx = fmaxf(fmaxf(bl[t][0] - rj.x, rj.x - bh[t][0]), 0.f);
                            float dy = fmaxf(fmaxf(bl[t][1] - rj.y, rj.y - bh[t][1]), 0.f);
                            float dz = fmaxf(fmaxf(bl[t][2] - rj.z, rj.z - bh[t][2]), 0.f);
                            float cut = S::box_cut(p, bhm[t], rj);
                            keep[t] = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= cut * cut * 1.0001f + 1e-6f;
                        }
                    }
                    const unsigned m0 = __ballot_sync(CRK_FULL_MASK, keep[0]);
                    const unsigned m1 = __ballot_sync(CRK_FULL_MASK, keep[1]);
                    if (keep[0]) ring[warp][0][(tail0 + __popc(m0 & below)) & (kRing - 1)] = rj;
                    if (keep[1]) ring[warp][1][(tail1 + __popc(m1 & below)) & (kRing - 1)] = rj;
                    tail0 += __popc(m0);
                    tail1 += __popc(m1);
                    const unsigned r0 = tail0 - head0, r1 = tail1 - head1;
                    const unsigned both = r0 < r1 ? r0 : r1;
                    if (r0 > kRing - 32 || r1 > kRing - 32) sweep(r0, r1);  // a ring is nearly full
                    else if (both >= 32) sweep(both, both);                // balanced
                }
            }
            sweep(tail0 - head0, tail1 - head1);
            if (act) S::finish(p, st, ri, lv.korder ? i : lv.kperm[i], i);
            if (kCount) {
                int cn = act ? st.cnt - 1 : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(CRK_FULL_MASK, cn, o);
                if (lane == 0 && cn) atomicAdd(p.count, (unsigned long long)cn);
            }
        }
    }
}

// stages with half-warp arms (kHalfWarp): partial sums flushed with atomics
template <class S, class = void>
struct has_halfwarp : std::false_type {};
template <class S>
struct has_halfwarp<S, std::void_t<decltype(S::kHalfWarp)>> : std::bool_constant<S::kHalfWarp> {};

// Conservation sums of a half-warp arm, from the finished outputs: per-block
// FP64 partials over the gas particles in kernel order (fixed assignment of
// particles to blocks and a fixed reduction order: deterministic).
template <class S>
__global__ void __launch_bounds__(256) halfwarp_cons_kernel(int64_t n, const float4 *__restrict__ pos,
                                                            const int32_t *__restrict__ kperm, int korder,
                                                            typename S::P p, double *__restrict__ part) {
    __shared__ double sh[8][4];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        if (!(pos[q].w > 0.0f)) continue;  // dark matter
        double c[4];
        S::cons_of(p, korder ? (int32_t)q : kperm[q], c);
        for (int k = 0; k < 4; ++k) acc[k] += c[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(CRK_FULL_MASK, acc[k], o);
        if (lane == 0) sh[w][k] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int v = 0; v < (int)(blockDim.x >> 5); ++v) t += sh[v][threadIdx.x];
        part[4 * blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void cons_reduce_kernel(const double *__restrict__ part, int64_t nb, double *__restrict__ out) {
    __shared__ double sh[256];
    for (int k = 0; k < 4; ++k) {
        double t = 0.0;
        for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) t += part[4 * b + k];
        sh[threadIdx.x] = t;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}


// Gas-pair stages driven by the exact neighbour lists: each lane walks its own
// list (k-major, so entry k of the 32 lanes is one coalesced row); inactive
// lanes (k beyond their length) idle.
struct GasLists {
    const int32_t *gstart, *goff, *cnt;
    const uint16_t *list;
    const int32_t *uoff, *unum;
    const uint32_t *ucode;
    const int32_t *gleaf;
    int64_t groups;          // capacity of the group arrays
    const int32_t *dgroups;  // device: the groups of this build, or NULL for all
};

// j-table entries staged per warp in shared memory (records of at most 48
// bytes; the hydro record is too large to stage, its lanes gather directly)
template <class S>
__host__ __device__ constexpr int table_cap() {
    // corrections: 256, so that five blocks of 128 threads fit an SM (with list_min_blocks below)
    return std::is_same<S, CorrStage>::value ? 256
                                             : (sizeof(typename S::Rec) <= 32 ? 320 : (sizeof(typename S::Rec) <= 48 ? 224 : 0));
}

// resident blocks per SM that list_kernel<S> is compiled for (a register cap; 0: none).
// Corrections is latency bound: capped for five blocks (96 registers, a few bytes spilled)
// it ran 10.1 ms on the 2x256^3 box, against 11.0 ms at four and 10.3 ms uncapped.
template <class S>
struct list_min_blocks {
    static constexpr int value = 0;  // no register cap
};
template <>
struct list_min_blocks<CorrStage> {
    static constexpr int value = 5;
};

// index rows in flight in list_kernel<S>: 8 for the short pair terms (records of at most 32
// bytes and few registers), 4 for the long ones
template <class S>
__host__ __device__ constexpr int list_ahead() {
    return (std::is_same<S, GeomStage>::value || std::is_same<S, GeomAdjStage>::value) ? 8 : 4;
}

// Stages whose pair term is gated by the in-range test (every contribution of
// an out-of-range j is an exact zero): list_kernel runs their rows of entries
// as straight-line code, padding the end of a lane's list with i's own record
// moved 4 h + 1 away, so the compiler interleaves the entries' dependent
// chains (geometry 5.34 -> 4.88 ms, corrections 10.48 -> 10.11 ms on the
// 2x256^3 box).  Hydro is left out: four staged 112-byte records per lane
// cost it its occupancy (15.1 -> 22.6 ms).
template <class S>
struct flat_tail {
    static constexpr bool value = false;
};
template <>
struct flat_tail<GeomStage> {
    static constexpr bool value = true;
};
template <>
struct flat_tail<GeomAdjStage> {
    static constexpr bool value = true;
};
template <>
struct flat_tail<CorrStage> {
    static constexpr bool value = true;
};
template <>
struct flat_tail<ExtrasStage> {
    static constexpr bool value = true;
};

// Exact neighbour lists, one warp per i-group.  The warp stages the group's
// j table in shared memory (each distinct j of the group gathered once,
// shifted into the i frame), then each lane walks its own list of table
// indices.  Table entries beyond the staged capacity are gathered from global
// memory through the leaf's image table.
template <class S, bool kCount>
__global__ void __launch_bounds__(kThreads, list_min_blocks<S>::value) list_kernel(LeafView lv, typename S::P p,
                                                        const typename S::Rec *__restrict__ rec, GasLists gl,
                                                        double *__restrict__ cons_part) {
    using Rec = typename S::Rec;
    constexpr int kTab = table_cap<S>();
    extern __shared__ __align__(16) unsigned char list_dyn[];
    __shared__ double cons_sh[kWarps][4];
    __shared__ float4 itab_all[kWarps][kGroupImgCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *itab = itab_all[warp];
    Rec *table = reinterpret_cast<Rec *>(list_dyn) + (size_t)warp * kTab;
    double cons_acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t ngroups = group_count(gl.groups, gl.dgroups);
    for (int64_t grp = next_group(lv, -1, lane); grp < ngroups; grp = next_group(lv, grp, lane)) {
        const int64_t a = gl.gleaf[grp];
        const int q = (int)(grp - gl.gstart[a]);
        const int lo = lv.leaf_start[a];
        const int hi = S::kGasOnly ? lo + lv.leaf_ngas[a] : lv.leaf_start[a + 1];
        const int g0 = lo + 32 * q;
        const crk_image *imgs = lv.img + lv.img_start[a];
        const int nimg = lv.img_cnt[a];
        const bool staged = nimg <= kGroupImgCap;
        __syncwarp();  // the previous group's tables are no longer read
        if (staged) {
            for (int t = lane; t < nimg; t += 32) {
                const crk_image im = imgs[t];
                itab[t] = make_float4(im.sx, im.sy, im.sz, __int_as_float(lv.leaf_start[im.b]));
            }
            __syncwarp();
        }
        const uint32_t *U = gl.ucode + gl.uoff[grp];
        const int nu = gl.unum[grp];
        // table entry -> shifted record of j
        auto fetch = [&](uint32_t code) -> Rec {
            float4 t;
            if (staged) {
                t = itab[code >> 10];
            } else {
                const crk_image im = imgs[code >> 10];
                t = make_float4(im.sx, im.sy, im.sz, __int_as_float(lv.leaf_start[im.b]));
            }
            Rec r = rec[__float_as_int(t.w) + (int)(code & 1023u)];
            S::shift(r, t.x, t.y, t.z);
            return r;
        };
        if constexpr (kTab > 0) {
            const int ns = nu < kTab ? nu : kTab;
#pragma unroll 4
            for (int u = lane; u < ns; u += 32) table[u] = fetch(__ldg(U + u));
            __syncwarp();
        }
        auto entry = [&](int idx) -> Rec {
            if constexpr (kTab > 0) {
                if (idx < kTab) return table[idx];
            }
            return fetch(__ldg(U + idx));
        };
        const uint16_t *Lp = gl.list + (size_t)gl.goff[grp] * 32 + lane;
        const int i = g0 + lane;
        const bool act = i < hi;
        const Rec ri = rec[act ? i : g0];
        typename S::I st;
        S::init(p, st, ri, a, q, lane, stage_index(lv, act ? i : g0));
        const int c = act ? gl.cnt[i] : 0;
        // indices kAhead rows ahead, so their loads overlap the pair arithmetic (light pair terms
        // need more rows in flight to cover a DRAM latency)
        constexpr int kAhead = list_ahead<S>();
        if constexpr (kAhead == 4) {
            int k = 0;
            int nx0 = 0 < c ? __ldg(Lp) : 0, nx1 = 1 < c ? __ldg(Lp + 32) : 0, nx2 = 2 < c ? __ldg(Lp + 64) : 0,
                nx3 = 3 < c ? __ldg(Lp + 96) : 0;
            for (; k < c; k += 4) {
                const int i0 = nx0, i1 = nx1, i2 = nx2, i3 = nx3;
                const uint16_t *Lk = Lp + (size_t)(k + 4) * 32;
                nx0 = k + 4 < c ? __ldg(Lk) : 0;
                nx1 = k + 5 < c ? __ldg(Lk + 32) : 0;
                nx2 = k + 6 < c ? __ldg(Lk + 64) : 0;
                nx3 = k + 7 < c ? __ldg(Lk + 96) : 0;
                if constexpr (flat_tail<S>::value) {
                    Rec far = ri;  // past the end of the list: out of range, every term finite
                    far.x += 4.0f * ri.h + 1.0f;
                    const Rec e0 = entry(i0);
                    const Rec e1 = k + 1 < c ? entry(i1) : far;
                    const Rec e2 = k + 2 < c ? entry(i2) : far;
                    const Rec e3 = k + 3 < c ? entry(i3) : far;
                    S::template interact<kCount>(p, st, ri, e0);
                    S::template interact<kCount>(p, st, ri, e1);
                    S::template interact<kCount>(p, st, ri, e2);
                    S::template interact<kCount>(p, st, ri, e3);
                } else {
                    S::template interact<kCount>(p, st, ri, entry(i0));
                    if (k + 1 < c) S::template interact<kCount>(p, st, ri, entry(i1));
                    if (k + 2 < c) S::template interact<kCount>(p, st, ri, entry(i2));
                    if (k + 3 < c) S::template interact<kCount>(p, st, ri, entry(i3));
                }
            }
        } else {
            int nx[kAhead];
#pragma unroll
            for (int d = 0; d < kAhead; ++d) nx[d] = d < c ? __ldg(Lp + (size_t)d * 32) : 0;
            for (int k = 0; k < c; k += kAhead) {
                int cur[kAhead];
                const uint16_t *Lk = Lp + (size_t)(k + kAhead) * 32;
#pragma unroll
                for (int d = 0; d < kAhead; ++d) {
                    cur[d] = nx[d];
                    nx[d] = k + kAhead + d < c ? __ldg(Lk + (size_t)d * 32) : 0;
                }
                if constexpr (flat_tail<S>::value) {
                    Rec far = ri;
                    far.x += 4.0f * ri.h + 1.0f;
                    Rec e[kAhead];
#pragma unroll
                    for (int d = 0; d < kAhead; ++d) e[d] = (d == 0 || k + d < c) ? entry(cur[d]) : far;
#pragma unroll
                    for (int d = 0; d < kAhead; ++d) S::template interact<kCount>(p, st, ri, e[d]);
                } else {
                    S::template interact<kCount>(p, st, ri, entry(cur[0]));
#pragma unroll
                    for (int d = 1; d < kAhead; ++d)
                        if (k + d < c) S::template interact<kCount>(p, st, ri, entry(cur[d]));
                }
            }
        }
        if (act) S::finish(p, st, ri, lv.korder ? i : lv.kperm[i], i);
        if constexpr (S::kCons) {
            double cc[4] = {0.0, 0.0, 0.0, 0.0};
            if (act) S::cons_terms(p, st, ri, lv.korder ? i : lv.kperm[i], cc);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cc[kk] += __shfl_xor_sync(CRK_FULL_MASK, cc[kk], o);
                cons_acc[kk] += cc[kk];
            }
        }
        if (kCount) {
            int cn = act ? st.cnt - 1 : 0;
            int sw = c;  // candidate evaluations: the list entries
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cn += __shfl_xor_sync(CRK_FULL_MASK, cn, o);
                sw += __shfl_xor_sync(CRK_FULL_MASK, sw, o);
            }
            if (lane == 0 && cn) atomicAdd(p.count, (unsigned long long)cn);
            if (lane == 0 && p.swept && sw) atomicAdd(p.swept, (unsigned long long)sw);
        }
    }
    if constexpr (S::kCons) {
        if (cons_part) cons_block_partial(cons_sh, cons_acc, cons_part);
    }
}

// dynamic shared memory of list_kernel<S>, and the opt-in above the 48 KB default (once per kernel)
template <class S, bool kCount>
size_t list_kernel_smem() {
    const size_t bytes = (size_t)kWarps * table_cap<S>() * sizeof(typename S::Rec);
    static bool set = false;
    if (!set) {
        cudaFuncSetAttribute(list_kernel<S, kCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        set = true;
    }
    return bytes;
}

// resident blocks per SM of list_kernel<S> (registers and shared memory; once per kernel)
template <class S, bool kCount>
int list_kernel_resident() {
    static int nb = 0;
    if (!nb) {
        const size_t smem = list_kernel_smem<S, kCount>();
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, list_kernel<S, kCount>, kThreads, smem) != cudaSuccess) {
            cudaGetLastError();
            nb = 4;
        }
        if (nb < 1) nb = 1;
    }
    return nb;
}

// fixed-capacity list and table offsets: goff[g] = g capr, uoff[g] = g capt
__global__ void strided_offsets_kernel(int64_t m, int capr, int capt, int32_t *__restrict__ goff,
                                       int32_t *__restrict__ uoff) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < m) {
        goff[g] = (int32_t)(g * capr);
        uoff[g] = (int32_t)(g * capt);
    }
}

// groups of each leaf, and the leaf of each group (groups beyond the capacity cap are dropped)
__global__ void list_group_leaf_kernel(int64_t n_leaves, const int32_t *__restrict__ gstart,
                                       int32_t *__restrict__ gleaf, int64_t cap) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_leaves) return;
    for (int32_t g = gstart[a]; g < gstart[a + 1] && g < cap; ++g) gleaf[g] = (int32_t)a;
}

// a rebuild's group count and list overflow as bits of the leaves' status word
__global__ void lists_status_kernel(const int32_t *__restrict__ groups, int64_t cap, const int32_t *__restrict__ ovf,
                                    int32_t *__restrict__ status) {
    int32_t s = 0;
    if (*groups > cap) s |= CRK_LEAVES_GROUP_CAP;
    if (ovf && *ovf) s |= CRK_LEAVES_LIST_CAP;
    if (s) atomicOr(status, s);
}

__global__ void list_group_count_kernel(int64_t n_leaves, const int32_t *__restrict__ leaf_start,
                                        const int32_t *__restrict__ ngas, int gas, int32_t *__restrict__ ng) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_leaves) ng[a] = ((gas ? ngas[a] : leaf_start[a + 1] - leaf_start[a]) + 31) >> 5;
}

// per group: the longest list of its lanes (units of 32 entries once scanned)
__global__ void list_group_k_kernel(int64_t n_leaves, const int32_t *__restrict__ leaf_start,
                                    const int32_t *__restrict__ ngas, int gas, const int32_t *__restrict__ gstart,
                                    const int32_t *__restrict__ cnt, int32_t *__restrict__ gk) {
    int64_t a = blockIdx.x;
    if (a >= n_leaves) return;
    const int lo = leaf_start[a], hi = gas ? lo + ngas[a] : leaf_start[a + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int g0 = lo + warp * 32; g0 < hi; g0 += (blockDim.x >> 5) * 32) {
        int i = g0 + lane;
        int c = i < hi ? cnt[i] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(CRK_FULL_MASK, c, o));
        if (lane == 0) gk[gstart[a] + ((g0 - lo) >> 5)] = c;
    }
}

template <class S>
int run_stage(crk_ctx *ctx, const crk_leaves *lv, typename S::P p, bool gas_pairs, int kernel_id,
              double *cons = nullptr, bool korder = false) {
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null leaves");
    const int64_t n = lv->n;
    if (n == 0) return CRK_OK;
    using Rec = typename S::Rec;
    Rec *rec = (Rec *)crk_scratch(ctx, 4, sizeof(Rec) * (size_t)n);
    if (!rec) return crk_fail(ctx, CRK_ENOMEM, "stage scratch");
    const crk_nlist &nls = gas_pairs ? lv->gas_lists : lv->grav_lists;
    const bool lists = nls.list && ctx->variant[kernel_id] == CRK_VARIANT_LISTS;
    // one block per i-leaf, or (lists) one warp per i-group
    int64_t grid = lists ? (nls.groups + kWarps - 1) / kWarps : lv->n_leaves;
    if (grid < 1) grid = 1;
    if (grid > 2147483647LL) grid = 2147483647LL;
    const bool persistent = ctx->persist[kernel_id] != 0;
    if (persistent) {
        // persistent grid: resident blocks on every SM (lists: as many as fit; tiles: 4 blocks of
        // 128 threads per SM, the design point)
        int per_sm = 4;
        if (lists) per_sm = p.count ? list_kernel_resident<S, true>() : list_kernel_resident<S, false>();
        const int64_t g = (int64_t)ctx->num_sms * per_sm;
        if (g < grid) grid = g;
    }
    const bool halfwarp = !lists && ctx->variant[kernel_id] >= CRK_VARIANT_HALFWARP_SHFL &&
                          ctx->variant[kernel_id] <= CRK_VARIANT_HALFWARP_LOAD && has_halfwarp<S>::value;
    // half-warp arms take their conservation sums from the finished outputs, in cblocks partials
    const int64_t cblocks = std::min<int64_t>(crk_grid(n, 256), (int64_t)ctx->num_sms * 8);
    int64_t nparts = halfwarp ? cblocks : grid;
    double *part = nullptr;
    if (cons) {
        part = (double *)crk_scratch(ctx, 5, sizeof(double) * 4 * (size_t)nparts);
        if (!part) return crk_fail(ctx, CRK_ENOMEM, "stage scratch");
    }
    const float4 *kpos = gas_pairs ? lv->pos : lv->pos_g;          // gravity: species-mixed kernel order
    const int32_t *kperm = gas_pairs ? lv->kperm : lv->kperm_g;
    gather_kernel<S><<<crk_grid(n, 256), 256, 0, ctx->stream>>>(n, kpos, kperm, p, rec, korder ? 1 : 0);
    int32_t *queue = nullptr;
    if (persistent) {
        queue = (int32_t *)crk_scratch(ctx, 17, 64);
        if (!queue) return crk_fail(ctx, CRK_ENOMEM, "stage scratch");
        CRK_CUDA(ctx, cudaMemsetAsync(queue, 0, sizeof(int32_t), ctx->stream));
    }
    LeafView v{lv->leaf_start, lv->leaf_ngas, lv->bbox, lv->hmax, kpos, kperm,
               gas_pairs ? lv->himg_start : lv->gimg_start, gas_pairs ? lv->himg_cnt : lv->gimg_cnt,
               gas_pairs ? lv->himg : lv->gimg, lv->n_leaves, queue, korder ? 1 : 0, ctx->depth[kernel_id]};
    if (p.count) CRK_CUDA(ctx, cudaMemsetAsync(p.count, 0, sizeof(unsigned long long), ctx->stream));
    if (p.swept) CRK_CUDA(ctx, cudaMemsetAsync(p.swept, 0, sizeof(unsigned long long), ctx->stream));
    if (lists) {
        GasLists gl{nls.gstart, nls.goff, nls.cnt, nls.list, nls.uoff, nls.unum, nls.ucode, nls.gleaf, nls.groups,
                    nls.dgroups};
        if (p.count)
            list_kernel<S, true><<<(unsigned)grid, kThreads, list_kernel_smem<S, true>(), ctx->stream>>>(v, p, rec, gl,
                                                                                                       part);
        else
            list_kernel<S, false><<<(unsigned)grid, kThreads, list_kernel_smem<S, false>(), ctx->stream>>>(v, p, rec, gl,
                                                                                                         part);
    } else if (halfwarp) {
        if constexpr (has_halfwarp<S>::value) {
            typename S::P q = p;
            if constexpr (S::kCons) {
                if (cons && !q.dv3) {  // the Energy pass: its recomputed force, for the conservation sums
                    q.dv3 = (float *)crk_scratch(ctx, 35, sizeof(float) * 3 * (size_t)n);
                    if (!q.dv3) return crk_fail(ctx, CRK_ENOMEM, "stage scratch");
                }
            }
            S::zero_outputs(q, ctx->stream);
            const int ex = ctx->variant[kernel_id] - CRK_VARIANT_HALFWARP_SHFL;
            const unsigned gg = (unsigned)grid;
            if (p.count) {
                if (ex == 0) pair_kernel_halfwarp<S, true, 0><<<gg, kThreads, 0, ctx->stream>>>(v, q, rec, part);
                else if (ex == 1) pair_kernel_halfwarp<S, true, 1><<<gg, kThreads, 0, ctx->stream>>>(v, q, rec, part);
                else pair_kernel_halfwarp<S, true, 2><<<gg, kThreads, 0, ctx->stream>>>(v, q, rec, part);
            } else {
                if (ex == 0) pair_kernel_halfwarp<S, false, 0><<<gg, kThreads, 0, ctx->stream>>>(v, q, rec, part);
                else if (ex == 1) pair_kernel_halfwarp<S, false, 1><<<gg, kThreads, 0, ctx->stream>>>(v, q, rec, part);
                else pair_kernel_halfwarp<S, false, 2><<<gg, kThreads, 0, ctx->stream>>>(v, q, rec, part);
            }
            if constexpr (S::kCons) {
                if (cons) {
                    halfwarp_cons_kernel<S><<<(unsigned)cblocks, 256, 0, ctx->stream>>>(n, kpos, kperm, korder ? 1 : 0,
                                                                                         q, part);
                    ++ctx->launches;
                }
            }
        }
    } else if constexpr (!S::kAllVariants) {  // built for lists and tiles only
        if (p.count)
            pair_kernel<S, true><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
        else
            pair_kernel<S, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
    } else {
        if (ctx->variant[kernel_id] == CRK_VARIANT_SPLIT8 && S::kPair) {
            if constexpr (S::kPair) {
                // a bounded grid: every block's warps own a slot of the candidate buffer
                constexpr int kGcap = 4096;
                static int occ[2] = {0, 0};  // resident blocks per SM, from the kernel's registers and shared memory
                int &oc = occ[p.count ? 1 : 0];
                if (!oc) {
                    cudaFuncAttributes fa{};
                    const cudaError_t e = p.count ? cudaFuncGetAttributes(&fa, pair_kernel_split<S, true>)
                                                  : cudaFuncGetAttributes(&fa, pair_kernel_split<S, false>);
                    int by_regs = 16, by_smem = 16;
                    if (e == cudaSuccess && fa.numRegs > 0) {
                        const int regs = (fa.numRegs + 7) / 8 * 8;  // allocated per thread in units of 8
                        by_regs = 65536 / (regs * kThreads);
                        by_smem = (int)((228u * 1024u) / ((unsigned)fa.sharedSizeBytes + 1024u));
                    } else {
                        cudaGetLastError();
                    }
                    oc = std::max(1, std::min(16, std::min(by_regs, by_smem)));
                }
                const int64_t g = std::min<int64_t>(grid, (int64_t)ctx->num_sms * oc);
                Rec *gbuf = (Rec *)crk_scratch(ctx, 37, sizeof(Rec) * (size_t)g * kWarps * kGcap);
                if (!gbuf) return crk_fail(ctx, CRK_ENOMEM, "stage scratch");
                if (p.count)
                    pair_kernel_split<S, true><<<(unsigned)g, kThreads, 0, ctx->stream>>>(v, p, rec, gbuf, kGcap);
                else
                    pair_kernel_split<S, false><<<(unsigned)g, kThreads, 0, ctx->stream>>>(v, p, rec, gbuf, kGcap);
            }
        } else if (ctx->variant[kernel_id] == CRK_VARIANT_TILES16) {
            if constexpr (S::kPair) {  // gravity stages: packed two-candidate sweeps
                if (p.count)
                    pair_kernel_sub_pair<S, true><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
                else
                    pair_kernel_sub_pair<S, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
            } else {
                if (p.count)
                    pair_kernel_sub<S, 16, true><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
                else
                    pair_kernel_sub<S, 16, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
            }
        } else if (ctx->variant[kernel_id] == CRK_VARIANT_RING16 && !S::kCons) {
            if constexpr (!S::kCons) {
                if (p.count)
                    pair_kernel_ring<S, true><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
                else
                    pair_kernel_ring<S, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
            }
        } else if (ctx->variant[kernel_id] == CRK_VARIANT_TILES8) {
            if (p.count)
                pair_kernel_sub<S, 8, true><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
            else
                pair_kernel_sub<S, 8, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
        } else if (S::kPair && ctx->warps[kernel_id] == 2) {
            if constexpr (S::kPair) {  // two warps per i-leaf (persistent: twice the blocks per SM)
                const unsigned g2 = (unsigned)(persistent ? std::min<int64_t>(lv->n_leaves, 2 * grid) : grid);
                if (p.count)
                    pair_kernel<S, true, 2><<<g2, 64, 0, ctx->stream>>>(v, p, rec, part);
                else
                    pair_kernel<S, false, 2><<<g2, 64, 0, ctx->stream>>>(v, p, rec, part);
            }
        } else if (p.count) {
            pair_kernel<S, true><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
        } else {
            pair_kernel<S, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, part);
        }
    }
    if (cons) cons_reduce_kernel<<<1, 256, 0, ctx->stream>>>(part, nparts, cons);
    ctx->launches += 2 + (cons ? 1 : 0);
    CRK_LAUNCH_CHECK(ctx, "pair kernel");
    return CRK_OK;
}

}  // namespace

int grav_short(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const float *m, float *a3,
               int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !gp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !a3)) return crk_fail(ctx, CRK_EINVAL, "null array");
    if (gp->r_cut != lv->r_cut_grav) return crk_fail(ctx, CRK_ESTATE, "r_cut differs from the leaves' r_cut_grav");
    GravP p{};
    p.m = m;
    p.a3 = a3;
    p.rc2 = gp->r_cut * gp->r_cut;
    p.eps2 = gp->eps * gp->eps;
    for (int k = 0; k < 6; ++k) p.c[k] = gp->poly[k];
    p.n = lv->n;
    p.count = (unsigned long long *)pair_count;
    return run_stage<GravStage>(ctx, lv, p, false, CRK_K_GRAVITY);
}

int grav_short_adjoint(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const float *m,
                       const float *abar3, float *gx3, float *gm) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !gp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !abar3 || !gx3 || !gm)) return crk_fail(ctx, CRK_EINVAL, "null array");
    if (gp->r_cut != lv->r_cut_grav) return crk_fail(ctx, CRK_ESTATE, "r_cut differs from the leaves' r_cut_grav");
    GravAdjP p{};
    p.m = m;
    p.abar = abar3;
    p.gx3 = gx3;
    p.gm = gm;
    p.rc2 = gp->r_cut * gp->r_cut;
    p.eps2 = gp->eps * gp->eps;
    for (int k = 0; k < 6; ++k) p.c[k] = gp->poly[k];
    p.n = lv->n;
    p.count = nullptr;
    return run_stage<GravAdjStage>(ctx, lv, p, false, CRK_K_GRAVITY_ADJOINT);
}

int crk_geometry(crk_ctx *ctx, const crk_leaves *lv, const float *m, float *V, float *rho, int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null leaves");
    if (lv->n > 0 && (!m || !V || !rho)) return crk_fail(ctx, CRK_EINVAL, "null array");
    GeomP p{m, V, rho, lv->n, (unsigned long long *)pair_count};
    return run_stage<GeomStage>(ctx, lv, p, true, CRK_K_GEOMETRY);
}

int crk_geometry_adjoint(crk_ctx *ctx, const crk_leaves *lv, const float *m, const float *V, const float *rhobar,
                         const float *Vbar, float *gx3, float *gm) {
    if (!ctx) return CRK_EINVAL;
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null leaves");
    if (lv->n > 0 && (!m || !V || !rhobar || !gx3 || !gm)) return crk_fail(ctx, CRK_EINVAL, "null array");
    GeomAdjP p{m, V, rhobar, Vbar, gx3, gm, lv->n, nullptr};
    return run_stage<GeomAdjStage>(ctx, lv, p, true, CRK_K_GEOMETRY_ADJOINT);
}

int crk_corrections(crk_ctx *ctx, const crk_leaves *lv, const float *V, float *A, float *B, float *gradA,
                    float *gradB, int32_t *n_singular) {
    if (!ctx) return CRK_EINVAL;
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null leaves");
    if (lv->n > 0 && (!V || !A || !B || !gradA || !gradB)) return crk_fail(ctx, CRK_EINVAL, "null array");
    if (n_singular) CRK_CUDA(ctx, cudaMemsetAsync(n_singular, 0, sizeof(int32_t), ctx->stream));
    CorrP p{V, A, B, gradA, gradB, n_singular, lv->n, nullptr};
    return run_stage<CorrStage>(ctx, lv, p, true, CRK_K_CORRECTIONS);
}

int crk_hydro(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
              const float *u, const float *V, const float *rho, const float *A, const float *B, const float *gradA,
              const float *gradB, float *dvdt3, float *dudt, double *conservation, int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !hp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !v3 || !u || !V || !rho || !A || !B || !gradA || !gradB || !dvdt3 || !dudt))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    HydroP p{m, v3, u, V, rho, A, B, gradA, gradB, dvdt3, dudt, conservation,
             hp->gamma, hp->alpha, hp->beta, hp->eta2, lv->n, (unsigned long long *)pair_count};
    return run_stage<HydroStage>(ctx, lv, p, true, CRK_K_HYDRO, conservation);
}

int crk_extras(crk_ctx *ctx, const crk_leaves *lv, const float *m, const float *v3, const float *V, const float *A,
               const float *B, const float *gradA, const float *gradB, float *rho_r, float *dvdx,
               int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !v3 || !V || !A || !B || !gradA || !gradB || !rho_r || !dvdx))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    ExtrasP p{m, v3, V, A, B, gradA, gradB, rho_r, dvdx, lv->n, (unsigned long long *)pair_count};
    return run_stage<ExtrasStage>(ctx, lv, p, true, CRK_K_EXTRAS);
}

int crk_hydro_limited(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m,
                      const float *v3, const float *u, const float *V, const float *rho, const float *A,
                      const float *B, const float *gradA, const float *gradB, const float *dvdx, float *dvdt3,
                      float *dudt, double *conservation, int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !hp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !v3 || !u || !V || !rho || !A || !B || !gradA || !gradB || !dvdx || !dvdt3 || !dudt))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    HydroP p{m, v3, u, V, rho, A, B, gradA, gradB, dvdt3, dudt, conservation,
             hp->gamma, hp->alpha, hp->beta, hp->eta2, lv->n, (unsigned long long *)pair_count, dvdx};
    return run_stage<HydroLimStage>(ctx, lv, p, true, CRK_K_HYDRO, conservation);
}

int crk_hydro_accel(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
                    const float *u, const float *V, const float *rho, const float *A, const float *B,
                    const float *gradA, const float *gradB, const float *dvdx, float sig_beta, float *dvdt3,
                    uint32_t *vsig_h_max, double *conservation, int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !hp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !v3 || !u || !V || !rho || !A || !B || !gradA || !gradB || !dvdt3))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    if (!(sig_beta >= 0.0f)) return crk_fail(ctx, CRK_EINVAL, "sig_beta must be >= 0");
    HydroP p{m, v3, u, V, rho, A, B, gradA, gradB, dvdt3, nullptr, conservation,
             hp->gamma, hp->alpha, hp->beta, hp->eta2, lv->n, (unsigned long long *)pair_count, dvdx};
    p.vsig_h = vsig_h_max;
    p.sig_beta = sig_beta;
    if (dvdx) return run_stage<HydroAccelStage<true>>(ctx, lv, p, true, CRK_K_ACCEL, conservation);
    return run_stage<HydroAccelStage<false>>(ctx, lv, p, true, CRK_K_ACCEL, conservation);
}

int crk_hydro_energy(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
                     const float *u, const float *V, const float *rho, const float *A, const float *B,
                     const float *gradA, const float *gradB, const float *dvdx, const float *vstar3, float *dudt,
                     double *conservation, int64_t *pair_count) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !hp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !v3 || !u || !V || !rho || !A || !B || !gradA || !gradB || !vstar3 || !dudt))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    HydroP p{m, v3, u, V, rho, A, B, gradA, gradB, nullptr, dudt, conservation,
             hp->gamma, hp->alpha, hp->beta, hp->eta2, lv->n, (unsigned long long *)pair_count, dvdx};
    p.vstar = vstar3;
    if (dvdx) return run_stage<HydroEnergyStage<true>>(ctx, lv, p, true, CRK_K_ENERGY, conservation);
    return run_stage<HydroEnergyStage<false>>(ctx, lv, p, true, CRK_K_ENERGY, conservation);
}

int crk_corrections_adjoint(crk_ctx *ctx, const crk_leaves *lv, const float *V, const float *Abar,
                            const float *Bbar, const float *gradAbar, const float *gradBbar, float *xbar3,
                            float *Vbar, int32_t *n_singular) {
    if (!ctx) return CRK_EINVAL;
    if (!lv) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!V || !Abar || !Bbar || !gradAbar || !gradBbar || !xbar3 || !Vbar))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    const int64_t n = lv->n;
    if (n_singular) CRK_CUDA(ctx, cudaMemsetAsync(n_singular, 0, sizeof(int32_t), ctx->stream));
    if (n == 0) return CRK_OK;
    float *coef = (float *)crk_scratch(ctx, 33, sizeof(float) * kCorrCoef * (size_t)n);
    if (!coef) return crk_fail(ctx, CRK_ENOMEM, "adjoint scratch");
    CorrAdjP p{};
    p.V = V;
    p.n_singular = n_singular;
    p.n = n;
    p.Abar = Abar;
    p.Bbar = Bbar;
    p.gAbar = gradAbar;
    p.gBbar = gradBbar;
    p.coef = coef;
    int rc;
    if ((rc = run_stage<CorrAdjPrepStage>(ctx, lv, p, true, CRK_K_CORRECTIONS))) return rc;
    CorrAdjSweepP q{V, coef, xbar3, Vbar, n, nullptr, nullptr};
    return run_stage<CorrAdjStage>(ctx, lv, q, true, CRK_K_CORRECTIONS);
}

int crk_hydro_adjoint(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, const float *m, const float *v3,
                      const float *u, const float *V, const float *rho, const float *A, const float *B,
                      const float *gradA, const float *gradB, const float *dvbar3, const float *dubar, float *xbar3,
                      float *vbar3, float *ubar, float *mbar, float *Vbar, float *rhobar, float *Abar, float *Bbar3,
                      float *gradAbar3, float *gradBbar9) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !hp) return crk_fail(ctx, CRK_EINVAL, "null argument");
    if (lv->n > 0 && (!m || !v3 || !u || !V || !rho || !A || !B || !gradA || !gradB || !dvbar3 || !dubar || !xbar3 ||
                      !vbar3 || !ubar || !mbar || !Vbar || !rhobar || !Abar || !Bbar3 || !gradAbar3 || !gradBbar9))
        return crk_fail(ctx, CRK_EINVAL, "null array");
    HydroAdjP p{m,      v3,     u,     V,     rho,   A,         B,         gradA,     gradB,
                dvbar3, dubar,  xbar3, vbar3, ubar,  mbar,      Vbar,      rhobar,    Abar,
                Bbar3,  gradAbar3, gradBbar9, hp->gamma, hp->alpha, hp->beta, hp->eta2, lv->n, nullptr, nullptr};
    return run_stage<HydroAdjStage>(ctx, lv, p, true, CRK_K_HYDRO);
}

// reuse: a rebuild of one-pass gas lists into the buffers of the first build (group arrays with
// room for 1/8 more groups); no host synchronisation, overflows go to the leaves' status word.
template <bool kGas>
static int build_lists(crk_ctx *ctx, crk_leaves *lv, crk_nlist &out, bool reuse) {
    const int64_t nl = lv->n_leaves, n = lv->n;
    if (nl == 0 || n == 0 || (kGas && lv->n_gas == 0)) return CRK_OK;
    if (reuse && (!kGas || !out.onepass)) return crk_fail(ctx, CRK_ESTATE, "rebuild: lists without fixed capacities");
    cudaStream_t st = ctx->stream;
    using LS = ListStage<kGas>;
    int32_t *gstart = reuse ? out.gstart : (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)(nl + 1));
    int32_t *cnt = reuse ? out.cnt : (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)n);
    int32_t *ng = (int32_t *)crk_scratch(ctx, 6, sizeof(int32_t) * (size_t)(nl + 1));
    int32_t *tot = (int32_t *)crk_scratch(ctx, 7, 64);  // [0] groups, [1] rows, [2] table entries, [4] largest table
    if (!gstart || !cnt || !ng || !tot) return crk_fail(ctx, CRK_ENOMEM, "neighbour list allocation");
    CRK_CUDA(ctx, cudaMemsetAsync(ng, 0, sizeof(int32_t) * (size_t)(nl + 1), st));
    list_group_count_kernel<<<crk_grid(nl, 256), 256, 0, st>>>(nl, lv->leaf_start, lv->leaf_ngas, kGas, ng);
    ++ctx->launches;
    int rc = crk_exclusive_scan_i32(ctx, ng, gstart, nl + 1, tot);
    if (rc) return rc;
    int32_t *dgroups = lv->dev + (kGas ? 1 : 2);  // this build's group count, for the kernels
    CRK_CUDA(ctx, cudaMemcpyAsync(dgroups, tot, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    LeafView v{lv->leaf_start, lv->leaf_ngas, lv->bbox, lv->hmax, kGas ? lv->pos : lv->pos_g,
               kGas ? lv->kperm : lv->kperm_g, kGas ? lv->himg_start : lv->gimg_start,
               kGas ? lv->himg_cnt : lv->gimg_cnt, kGas ? lv->himg : lv->gimg, nl, nullptr, 0, 32};
    typename LS::Rec *rec = (typename LS::Rec *)crk_scratch(ctx, 4, sizeof(typename LS::Rec) * (size_t)n);
    if (!rec) return crk_fail(ctx, CRK_ENOMEM, "neighbour list scratch");
    const float rc2 = lv->r_cut_grav * lv->r_cut_grav;
    const int capr = kGasListCapRows, capt = kGasTableCap;
    if (reuse) {
        const int64_t capg = out.groups;
        list_group_leaf_kernel<<<crk_grid(nl, 256), 256, 0, st>>>(nl, gstart, out.gleaf, capg);
        gather_kernel<LS><<<crk_grid(n, 256), 256, 0, st>>>(n, v.pos, v.kperm, ListP{}, rec, 0);
        CRK_CUDA(ctx, cudaMemsetAsync(tot + 5, 0, sizeof(int32_t), st));
        ListP pf{out.list, out.ucode, gstart, out.goff, out.uoff, cnt, out.unum, nullptr, tot + 5, capr, capt, rc2, n,
                 nullptr};
        const GroupTable gt{gstart, out.gleaf, capg, dgroups};
        const unsigned gg = (unsigned)((capg + kWarps - 1) / kWarps > 0 ? (capg + kWarps - 1) / kWarps : 1);
        pair_group_kernel<LS, false><<<gg, kThreads, 0, st>>>(v, pf, rec, gt, nullptr);
        lists_status_kernel<<<1, 1, 0, st>>>(tot, capg, tot + 5, lv->dev);
        ctx->launches += 4;
        CRK_LAUNCH_CHECK(ctx, "neighbour lists");
        return CRK_OK;
    }
    int32_t ngroups = 0;
    CRK_CUDA(ctx, cudaMemcpyAsync(&ngroups, tot, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CRK_CUDA(ctx, cudaStreamSynchronize(st));
    // one-pass lists: room for 1/8 more groups than this build holds (a rebuild of moved particles reuses them)
    const int64_t capg = (int64_t)ngroups + ngroups / 8 + 64;
    int32_t *gleaf = (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)capg);
    if (!gleaf) return crk_fail(ctx, CRK_ENOMEM, "neighbour list allocation");
    list_group_leaf_kernel<<<crk_grid(nl, 256), 256, 0, st>>>(nl, gstart, gleaf, capg);
    const GroupTable gt{gstart, gleaf, ngroups, nullptr};
    const unsigned ggrid = (unsigned)((ngroups + kWarps - 1) / kWarps > 0 ? (ngroups + kWarps - 1) / kWarps : 1);
    int32_t *ucnt = (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)(capg + 1));
    if (!ucnt) return crk_fail(ctx, CRK_ENOMEM, "neighbour list allocation");
    gather_kernel<LS><<<crk_grid(n, 256), 256, 0, st>>>(n, v.pos, v.kperm, ListP{}, rec, 0);
    ctx->launches += 2;
    int32_t *goff = nullptr, *uoff = nullptr;
    uint16_t *list = nullptr;
    uint32_t *ucode = nullptr;
    int64_t entries = 0, tsize = 0;
    // Gas lists: one pass into fixed capacities (a lane's list and a group's table), which the
    // adaptive smoothing lengths keep well above the largest counts; the exact two-pass build
    // (count, scan, fill) runs only if something overflowed.
    bool done = false;
    if (kGas && capg * capt < 2147483647LL) {
        goff = (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)(capg + 1));
        uoff = (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)(capg + 1));
        list = (uint16_t *)crk_leaves_alloc(ctx, lv, sizeof(uint16_t) * (size_t)capg * capr * 32);
        ucode = (uint32_t *)crk_leaves_alloc(ctx, lv, sizeof(uint32_t) * (size_t)capg * capt);
        if (!goff || !uoff || !list || !ucode) return crk_fail(ctx, CRK_ENOMEM, "neighbour list allocation");
        strided_offsets_kernel<<<crk_grid(capg + 1, 256), 256, 0, st>>>(capg + 1, capr, capt, goff, uoff);
        CRK_CUDA(ctx, cudaMemsetAsync(tot + 5, 0, sizeof(int32_t), st));
        ListP pf{list, ucode, gstart, goff, uoff, cnt, ucnt, nullptr, tot + 5, capr, capt, rc2, n, nullptr};
        pair_group_kernel<LS, false><<<ggrid, kThreads, 0, st>>>(v, pf, rec, gt, nullptr);
        ctx->launches += 2;
        CRK_LAUNCH_CHECK(ctx, "neighbour lists");
        int32_t ovf = 1;
        CRK_CUDA(ctx, cudaMemcpyAsync(&ovf, tot + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CRK_CUDA(ctx, cudaStreamSynchronize(st));
        if (ovf == 0) {
            done = true;
            entries = (int64_t)capg * capr * 32;
            tsize = (int64_t)capg * capt;
        } else if (ctx->trace) {
            fprintf(stderr, "[crk] gas lists: a list or table exceeded its capacity, exact build\n");
        }
    }
    if (!done) {
        CRK_CUDA(ctx, cudaMemsetAsync(ucnt, 0, sizeof(int32_t) * (size_t)(ngroups + 1), st));
        CRK_CUDA(ctx, cudaMemsetAsync(tot + 4, 0, sizeof(int32_t), st));
        ListP pc{nullptr, nullptr, gstart, nullptr, nullptr, cnt, ucnt, tot + 4, nullptr, 2147483647, 2147483647,
                 rc2, n, nullptr};
        pair_group_kernel<LS, false><<<ggrid, kThreads, 0, st>>>(v, pc, rec, gt, nullptr);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "neighbour counts");
        goff = (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)(ngroups + 1));
        uoff = (int32_t *)crk_leaves_alloc(ctx, lv, sizeof(int32_t) * (size_t)(ngroups + 1));
        int32_t *gk = (int32_t *)crk_scratch(ctx, 8, sizeof(int32_t) * (size_t)(ngroups + 1));
        if (!goff || !uoff || !gk) return crk_fail(ctx, CRK_ENOMEM, "neighbour list allocation");
        CRK_CUDA(ctx, cudaMemsetAsync(gk, 0, sizeof(int32_t) * (size_t)(ngroups + 1), st));
        list_group_k_kernel<<<(unsigned)nl, kThreads, 0, st>>>(nl, lv->leaf_start, lv->leaf_ngas, kGas, gstart, cnt,
                                                               gk);
        ++ctx->launches;
        rc = crk_exclusive_scan_i32(ctx, gk, goff, ngroups + 1, tot + 1);
        if (rc) return rc;
        rc = crk_exclusive_scan_i32(ctx, ucnt, uoff, ngroups + 1, tot + 2);
        if (rc) return rc;
        int32_t sizes[5] = {0, 0, 0, 0, 0};
        CRK_CUDA(ctx, cudaMemcpyAsync(sizes, tot, sizeof(sizes), cudaMemcpyDeviceToHost, st));
        CRK_CUDA(ctx, cudaStreamSynchronize(st));
        const int32_t rows = sizes[1], umax = sizes[4];
        tsize = (int64_t)(uint32_t)sizes[2];
        // table indices are 16-bit, and the offsets 32-bit: without lists the kernels use tiles
        if (umax > 65535 || rows < 0 || sizes[2] < 0) {
            if (ctx->trace)
                fprintf(stderr, "[crk] %s lists skipped (largest group table %d)\n", kGas ? "gas" : "gravity", umax);
            return CRK_OK;
        }
        entries = (int64_t)rows * 32;
        list = (uint16_t *)crk_leaves_alloc(ctx, lv, sizeof(uint16_t) * (size_t)(entries > 0 ? entries : 1));
        ucode = (uint32_t *)crk_leaves_alloc(ctx, lv, sizeof(uint32_t) * (size_t)(tsize > 0 ? tsize : 1));
        if (!list || !ucode)
            return crk_fail(ctx, CRK_ENOMEM, "neighbour list allocation (%lld entries)", (long long)entries);
        ListP pf{list, ucode, gstart, goff, uoff, nullptr, nullptr, nullptr, nullptr, 2147483647, 2147483647,
                 rc2, n, nullptr};
        pair_group_kernel<LS, false><<<ggrid, kThreads, 0, st>>>(v, pf, rec, gt, nullptr);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "neighbour lists");
    }
    out.unum = ucnt;
    out.uoff = uoff;
    out.ucode = ucode;
    out.table = tsize;
    out.gstart = gstart;
    out.gleaf = gleaf;
    out.goff = goff;
    out.cnt = cnt;
    out.list = list;
    out.groups = done ? capg : ngroups;
    out.dgroups = dgroups;
    out.onepass = done;
    out.entries = entries;
    return CRK_OK;
}

int crk_build_lists(crk_ctx *ctx, crk_leaves *lv, bool gas, bool reuse) {
    return gas ? build_lists<true>(ctx, lv, lv->gas_lists, reuse) : build_lists<false>(ctx, lv, lv->grav_lists, reuse);
}

// ---------------------------------------------------------------------------
// Allocation-free short-range gravity (no counterpart in the paper).
//
// Some callers cannot let a library call cudaMalloc: an application whose own
// pool already owns the device memory, or a time-stepping loop that must not
// pay the device synchronisation that cudaMalloc/cudaFree can imply.  This
// entry point runs the same gravity kernels as grav_short, but its only
// scratch (the kernel-order particle records, 16 bytes per particle) lives in
// the file-scope array below, which every GPU that loads libcrk holds until
// the process exits: CRK_NOALLOC_MAX_PARTICLES x 16 bytes = 32 MiB.
namespace {
__device__ __align__(256) GravStage::Rec g_noalloc_rec[CRK_NOALLOC_MAX_PARTICLES];

constexpr int kNoAllocMaxDevices = 64;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};  // device address of g_noalloc_rec, per device
std::mutex g_noalloc_mu;
}  // namespace

int grav_short_noalloc(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const float *m, float *a3) {
    if (!ctx || !lv || !gp) return CRK_EINVAL;
    const int64_t n = lv->n;
    if (n > CRK_NOALLOC_MAX_PARTICLES) return CRK_ETOOLARGE;
    if (n > 0 && (!m || !a3)) return CRK_EINVAL;
    if (gp->r_cut != lv->r_cut_grav) return CRK_ESTATE;
    if (n == 0) return CRK_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return CRK_ESTATE;  // the context's device must be current
    }
    // set-up, once per device, with that device current: the host-side name of a
    // __device__ array is not a device address, so ask the runtime for it
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_rec) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return CRK_ECUDA;
            }
            g_noalloc_ptr[dev] = ptr;
        }
        base = g_noalloc_ptr[dev];
    }
    GravStage::Rec *rec = (GravStage::Rec *)base;
    GravP p{};
    p.m = m;
    p.a3 = a3;
    p.rc2 = gp->r_cut * gp->r_cut;
    p.eps2 = gp->eps * gp->eps;
    for (int k = 0; k < 6; ++k) p.c[k] = gp->poly[k];
    p.n = n;
    p.count = nullptr;
    // every record is rewritten before it is read, so nothing needs clearing
    gather_kernel<GravStage><<<crk_grid(n, 256), 256, 0, ctx->stream>>>(n, lv->pos_g, lv->kperm_g, p, rec, 0);
    LeafView v{lv->leaf_start, lv->leaf_ngas, lv->bbox, lv->hmax, lv->pos_g, lv->kperm_g, lv->gimg_start,
               lv->gimg_cnt, lv->gimg, lv->n_leaves, nullptr, 0, 32};
    const int64_t grid = lv->n_leaves < 1 ? 1 : lv->n_leaves;
    const crk_nlist &nls = lv->grav_lists;
    if (nls.list && ctx->variant[CRK_K_GRAVITY] == CRK_VARIANT_LISTS) {
        GasLists gl{nls.gstart, nls.goff, nls.cnt, nls.list, nls.uoff, nls.unum, nls.ucode, nls.gleaf, nls.groups,
                    nls.dgroups};
        const int64_t lgrid = (nls.groups + kWarps - 1) / kWarps;
        list_kernel<GravStage, false><<<(unsigned)(lgrid > 0 ? lgrid : 1), kThreads,
                                        list_kernel_smem<GravStage, false>(), ctx->stream>>>(v, p, rec, gl, nullptr);
    } else {
        pair_kernel<GravStage, false><<<(unsigned)grid, kThreads, 0, ctx->stream>>>(v, p, rec, nullptr);
    }
    ctx->launches += 2;
    return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

// ---------------------------------------------------------------------------
// Whole step with kernel-order intermediates.  The step's inputs are permuted
// into the two kernel orders once; every intermediate (V, rho, A, B, dA, dB,
// a, the cotangents) stays in kernel order, so it is written and read
// coalesced instead of being scattered to the caller's order and gathered
// back by the next kernel; the outputs the caller asked for are gathered back
// to the caller's order once at the end.
namespace {

// dst[c*n + q] = src[c*n + perm[q]] for c < ncomp (into kernel order)
__global__ void to_korder_kernel(int64_t n, int ncomp, const int32_t *__restrict__ perm, const float *__restrict__ src,
                                 float *__restrict__ dst) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t o = perm[q];
    for (int c = 0; c < ncomp; ++c) dst[c * n + q] = src[c * n + o];
}


// One column through a permutation: dst[o] = src[perm[o]] (o in the
// destination order).  One column per launch keeps the randomly read source
// (n floats) about the size of L2, so each 32-byte sector is fetched from DRAM
// about once; gathering many columns at once thrashes L2 (measured slower).
__global__ void permute_col_kernel(int64_t n, const int32_t *__restrict__ perm, const float *__restrict__ src,
                                   float *__restrict__ dst) {
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < n) dst[o] = __ldg(src + perm[o]);
}

__global__ void cotangent_kernel(int64_t n, const float *__restrict__ a_g, const float4 *__restrict__ pos,
                                 float *__restrict__ abar_g, float *__restrict__ rhob_k) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    if (abar_g)
        for (int c = 0; c < 3; ++c) abar_g[c * n + q] = 2.0f * a_g[c * n + q];
    if (rhob_k) rhob_k[q] = pos[q].w > 0.0f ? 1.0f : 0.0f;
}

}  // namespace

int crk_stage_forces(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
                     int limited, int gravity, float sig_beta, const float *m, const float *v3, const float *u,
                     uint32_t *vsig_h, int32_t *n_singular, float *w) {
    namespace K = crk_stage_cols;
    const int64_t n = lv->n;
    if (n == 0) return CRK_OK;
    auto C = [&](int k) { return w + (size_t)k * n; };
    cudaStream_t st = ctx->stream;
    const int g = crk_grid(n, 256);
    auto col = [&](float *dst, const float *src, const int32_t *perm) {
        permute_col_kernel<<<g, 256, 0, st>>>(n, perm, src, dst);
        ++ctx->launches;
    };
    col(C(K::m), m, lv->kperm);
    for (int c = 0; c < 3; ++c) col(C(K::v) + (size_t)c * n, v3 + (size_t)c * n, lv->kperm);
    col(C(K::u), u, lv->kperm);
    if (gravity) col(C(K::mg), m, lv->kperm_g);
    CRK_LAUNCH_CHECK(ctx, "stage inputs");
    int rc;
    {
        GeomP p{C(K::m), C(K::V), C(K::rho), n, nullptr, nullptr};
        if ((rc = run_stage<GeomStage>(ctx, lv, p, true, CRK_K_GEOMETRY, nullptr, true))) return rc;
    }
    {
        if (n_singular) CRK_CUDA(ctx, cudaMemsetAsync(n_singular, 0, sizeof(int32_t), st));
        CorrP p{C(K::V), C(K::A), C(K::B), C(K::gA), C(K::gB), n_singular, n, nullptr};
        if ((rc = run_stage<CorrStage>(ctx, lv, p, true, CRK_K_CORRECTIONS, nullptr, true))) return rc;
    }
    if (limited) {
        ExtrasP p{C(K::m), C(K::v), C(K::V), C(K::A), C(K::B), C(K::gA), C(K::gB), C(K::rhoR), C(K::dvdx), n, nullptr};
        if ((rc = run_stage<ExtrasStage>(ctx, lv, p, true, CRK_K_EXTRAS, nullptr, true))) return rc;
    }
    {
        HydroP p{C(K::m), C(K::v), C(K::u), C(K::V), C(limited ? K::rhoR : K::rho), C(K::A), C(K::B), C(K::gA),
                 C(K::gB), C(K::dv), nullptr, nullptr, hp->gamma, hp->alpha, hp->beta, hp->eta2, n, nullptr,
                 limited ? C(K::dvdx) : nullptr};
        p.vsig_h = vsig_h;
        p.sig_beta = sig_beta;
        if (limited) rc = run_stage<HydroAccelStage<true>>(ctx, lv, p, true, CRK_K_ACCEL, nullptr, true);
        else rc = run_stage<HydroAccelStage<false>>(ctx, lv, p, true, CRK_K_ACCEL, nullptr, true);
        if (rc) return rc;
    }
    if (gravity) {
        if (gp->r_cut != lv->r_cut_grav) return crk_fail(ctx, CRK_ESTATE, "r_cut differs from the leaves' r_cut_grav");
        GravP p{};
        p.m = C(K::mg);
        p.a3 = C(K::ag);
        p.rc2 = gp->r_cut * gp->r_cut;
        p.eps2 = gp->eps * gp->eps;
        for (int k = 0; k < 6; ++k) p.c[k] = gp->poly[k];
        p.n = n;
        if ((rc = run_stage<GravStage>(ctx, lv, p, false, CRK_K_GRAVITY, nullptr, true))) return rc;
    }
    return CRK_OK;
}

int crk_stage_energy(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp, int limited,
                     const float *vstar3, float *w, double *conservation) {
    namespace K = crk_stage_cols;
    const int64_t n = lv->n;
    if (n == 0) return CRK_OK;
    auto C = [&](int k) { return w + (size_t)k * n; };
    const float *vs = C(K::v);
    if (vstar3) {
        const int g = crk_grid(n, 256);
        for (int c = 0; c < 3; ++c) {
            permute_col_kernel<<<g, 256, 0, ctx->stream>>>(n, lv->kperm, vstar3 + (size_t)c * n,
                                                           C(K::vs) + (size_t)c * n);
            ++ctx->launches;
        }
        CRK_LAUNCH_CHECK(ctx, "stage v*");
        vs = C(K::vs);
    }
    HydroP p{C(K::m), C(K::v), C(K::u), C(K::V), C(limited ? K::rhoR : K::rho), C(K::A), C(K::B), C(K::gA),
             C(K::gB), nullptr, C(K::du), conservation, hp->gamma, hp->alpha, hp->beta, hp->eta2, n, nullptr,
             limited ? C(K::dvdx) : nullptr};
    p.vstar = vs;
    if (limited) return run_stage<HydroEnergyStage<true>>(ctx, lv, p, true, CRK_K_ENERGY, conservation, true);
    return run_stage<HydroEnergyStage<false>>(ctx, lv, p, true, CRK_K_ENERGY, conservation, true);
}

namespace {
// out[i] = a[i] + b[i] (+ c[i] when c is given), over cols columns of n
__global__ void add_cols_kernel(int64_t n, int cols, float *__restrict__ out, const float *__restrict__ a,
                                const float *__restrict__ b, const float *__restrict__ c) {
    const int64_t total = n * cols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = c ? a[i] + b[i] + c[i] : a[i] + b[i];
}
}  // namespace

int crk_hydro_chain_adjoint(crk_ctx *ctx, const crk_leaves *lv, const crk_hydro_params *hp,
                            const crk_chain_adjoint_io *io) {
    if (!ctx) return CRK_EINVAL;
    if (!lv || !hp || !io) return crk_fail(ctx, CRK_EINVAL, "null argument");
    const int64_t n = lv->n;
    if (io->n_singular) CRK_CUDA(ctx, cudaMemsetAsync(io->n_singular, 0, sizeof(int32_t), ctx->stream));
    if (n == 0) return CRK_OK;
    if (!io->m || !io->v3 || !io->u || !io->dvbar3 || !io->dubar) return crk_fail(ctx, CRK_EINVAL, "null array");
    // kernel-order columns
    enum : int {
        cm = 0, cv = 1, cu = 4, cdvb = 5, cdub = 8, cV = 9, crho = 10, cA = 11, cB = 12, cgA = 15, cgB = 18,
        cdv = 27, cdu = 30, cxh = 31, cvb = 34, cub = 37, cmh = 38, cVh = 39, crhob = 40, cAb = 41, cBb = 42,
        cgAb = 45, cgBb = 48, ccoef = 57, cxc = ccoef + kCorrCoef, cVc = cxc + 3, cxg = cVc + 1, cmg = cxg + 3,
        cols = cmg + 1
    };
    float *w = (float *)crk_scratch(ctx, 34, sizeof(float) * cols * (size_t)n);
    if (!w) return crk_fail(ctx, CRK_ENOMEM, "chain scratch");
    auto C = [&](int k) { return w + (size_t)k * n; };
    cudaStream_t st = ctx->stream;
    const int g = crk_grid(n, 256);
    auto col = [&](float *dst, const float *src, const int32_t *perm) {
        permute_col_kernel<<<g, 256, 0, st>>>(n, perm, src, dst);
        ++ctx->launches;
    };
    col(C(cm), io->m, lv->kperm);
    col(C(cu), io->u, lv->kperm);
    col(C(cdub), io->dubar, lv->kperm);
    for (int c = 0; c < 3; ++c) {
        col(C(cv) + (size_t)c * n, io->v3 + (size_t)c * n, lv->kperm);
        col(C(cdvb) + (size_t)c * n, io->dvbar3 + (size_t)c * n, lv->kperm);
    }
    CRK_LAUNCH_CHECK(ctx, "chain inputs");
    int rc;
    {
        GeomP p{C(cm), C(cV), C(crho), n, nullptr, nullptr};
        if ((rc = run_stage<GeomStage>(ctx, lv, p, true, CRK_K_GEOMETRY, nullptr, true))) return rc;
    }
    {
        CorrP p{C(cV), C(cA), C(cB), C(cgA), C(cgB), io->n_singular, n, nullptr};
        if ((rc = run_stage<CorrStage>(ctx, lv, p, true, CRK_K_CORRECTIONS, nullptr, true))) return rc;
    }
    if (io->dvdt3 || io->dudt) {
        HydroP p{C(cm), C(cv), C(cu), C(cV), C(crho), C(cA), C(cB), C(cgA), C(cgB), C(cdv), C(cdu), nullptr,
                 hp->gamma, hp->alpha, hp->beta, hp->eta2, n, nullptr};
        if ((rc = run_stage<HydroStage>(ctx, lv, p, true, CRK_K_HYDRO, nullptr, true))) return rc;
    }
    {
        HydroAdjP p{C(cm),  C(cv),  C(cu),   C(cV),   C(crho),   C(cA),  C(cB),  C(cgA),     C(cgB),
                    C(cdvb), C(cdub), C(cxh), C(cvb), C(cub), C(cmh), C(cVh), C(crhob), C(cAb),
                    C(cBb), C(cgAb), C(cgBb), hp->gamma, hp->alpha, hp->beta, hp->eta2, n, nullptr, nullptr};
        if ((rc = run_stage<HydroAdjStage>(ctx, lv, p, true, CRK_K_HYDRO, nullptr, true))) return rc;
    }
    {
        CorrAdjP p{};
        p.V = C(cV);
        p.n = n;
        p.Abar = C(cAb);
        p.Bbar = C(cBb);
        p.gAbar = C(cgAb);
        p.gBbar = C(cgBb);
        p.coef = C(ccoef);
        if ((rc = run_stage<CorrAdjPrepStage>(ctx, lv, p, true, CRK_K_CORRECTIONS, nullptr, true))) return rc;
        CorrAdjSweepP q{C(cV), C(ccoef), C(cxc), C(cVc), n, nullptr, nullptr};
        if ((rc = run_stage<CorrAdjStage>(ctx, lv, q, true, CRK_K_CORRECTIONS, nullptr, true))) return rc;
    }
    const int ge = g < 8 * ctx->num_sms ? g : 8 * ctx->num_sms;
    add_cols_kernel<<<ge, 256, 0, st>>>(n, 1, C(cVh), C(cVh), C(cVc), nullptr);  // Vbar = hydro + corrections
    ++ctx->launches;
    {
        GeomAdjP p{C(cm), C(cV), C(crhob), C(cVh), C(cxg), C(cmg), n, nullptr};
        if ((rc = run_stage<GeomAdjStage>(ctx, lv, p, true, CRK_K_GEOMETRY_ADJOINT, nullptr, true))) return rc;
    }
    add_cols_kernel<<<ge, 256, 0, st>>>(n, 3, C(cxh), C(cxh), C(cxc), C(cxg));  // xbar
    add_cols_kernel<<<ge, 256, 0, st>>>(n, 1, C(cmh), C(cmh), C(cmg), nullptr);  // mbar
    ctx->launches += 2;
    CRK_LAUNCH_CHECK(ctx, "chain sums");
    struct Out {
        float *dst;
        int src, comp;
    } outs[] = {{io->dvdt3, cdv, 3}, {io->dudt, cdu, 1}, {io->xbar3, cxh, 3},
                {io->mbar, cmh, 1},  {io->vbar3, cvb, 3}, {io->ubar, cub, 1}};
    for (const Out &o : outs)
        if (o.dst)
            for (int c = 0; c < o.comp; ++c) col(o.dst + (size_t)c * n, C(o.src) + (size_t)c * n, lv->kinv);
    CRK_LAUNCH_CHECK(ctx, "chain outputs");
    return CRK_OK;
}

int crk_step_fused(crk_ctx *ctx, const crk_leaves *lv, const crk_grav_params *gp, const crk_hydro_params *hp,
                   const crk_step_io *io) {
    const int64_t n = lv->n;
    if (n == 0) return CRK_OK;
    if (!io->m || !io->v3 || !io->u) return crk_fail(ctx, CRK_EINVAL, "step inputs m, v3, u are required");
    if (gp->r_cut != lv->r_cut_grav) return crk_fail(ctx, CRK_ESTATE, "r_cut differs from the leaves' r_cut_grav");
    float *buf = (float *)crk_scratch(ctx, 18, sizeof(float) * 58 * (size_t)n);
    if (!buf) return crk_fail(ctx, CRK_ENOMEM, "step scratch");
    float *cur = buf;
    auto take = [&](int k) { float *r = cur; cur += (size_t)k * n; return r; };
    float *m_k = take(1), *v_k = take(3), *u_k = take(1), *V_k = take(1), *rho_k = take(1), *A_k = take(1);
    float *B_k = take(3), *gA_k = take(3), *gB_k = take(9), *dv_k = take(3), *du_k = take(1), *rhob_k = take(1);
    float *Vb_k = take(1), *gx2_k = take(3), *gm2_k = take(1);
    float *m_g = take(1), *a_g = take(3), *abar_g = take(3), *gx_g = take(3), *gm_g = take(1);
    float *rhoR_k = take(1), *dvdx_k = take(9);
    cudaStream_t st = ctx->stream;
    const int g = crk_grid(n, 256);
    crk_step_mark(ctx, 0);
    {
        // inputs into the two kernel orders: m, v, u (gas order) and m (gravity order)
        auto col = [&](float *dst, const float *src, const int32_t *perm) {
            permute_col_kernel<<<g, 256, 0, st>>>(n, perm, src, dst);
            ++ctx->launches;
        };
        col(m_k, io->m, lv->kperm);
        for (int c = 0; c < 3; ++c) col(v_k + (size_t)c * n, io->v3 + (size_t)c * n, lv->kperm);
        col(u_k, io->u, lv->kperm);
        col(m_g, io->m, lv->kperm_g);
    }
    CRK_LAUNCH_CHECK(ctx, "step inputs");
    unsigned long long *cnt = (unsigned long long *)io->pair_count;
    unsigned long long *swc = cnt ? (unsigned long long *)io->swept_count : nullptr;
    int rc;
    {
        GeomP p{m_k, V_k, rho_k, n, cnt ? cnt + 0 : nullptr, swc ? swc + 0 : nullptr};
        if ((rc = run_stage<GeomStage>(ctx, lv, p, true, CRK_K_GEOMETRY, nullptr, true))) return rc;
    }
    crk_step_mark(ctx, 1);
    {
        if (io->n_singular) CRK_CUDA(ctx, cudaMemsetAsync(io->n_singular, 0, sizeof(int32_t), st));
        CorrP p{V_k, A_k, B_k, gA_k, gB_k, io->n_singular, n, nullptr};
        if ((rc = run_stage<CorrStage>(ctx, lv, p, true, CRK_K_CORRECTIONS, nullptr, true))) return rc;
    }
    if (io->extras) {
        ExtrasP p{m_k, v_k, V_k, A_k, B_k, gA_k, gB_k, rhoR_k, dvdx_k, n, nullptr};
        if ((rc = run_stage<ExtrasStage>(ctx, lv, p, true, CRK_K_EXTRAS, nullptr, true))) return rc;
    }
    crk_step_mark(ctx, 2);
    if (io->extras) {
        HydroP p{m_k, v_k, u_k, V_k, rhoR_k, A_k, B_k, gA_k, gB_k, dv_k, du_k, io->conservation,
                 hp->gamma, hp->alpha, hp->beta, hp->eta2, n, cnt ? cnt + 1 : nullptr, dvdx_k,
                 swc ? swc + 1 : nullptr};
        if ((rc = run_stage<HydroLimStage>(ctx, lv, p, true, CRK_K_HYDRO, io->conservation, true))) return rc;
    } else {
        HydroP p{m_k, v_k, u_k, V_k, rho_k, A_k, B_k, gA_k, gB_k, dv_k, du_k, io->conservation,
                 hp->gamma, hp->alpha, hp->beta, hp->eta2, n, cnt ? cnt + 1 : nullptr, nullptr,
                 swc ? swc + 1 : nullptr};
        if ((rc = run_stage<HydroStage>(ctx, lv, p, true, CRK_K_HYDRO, io->conservation, true))) return rc;
    }
    crk_step_mark(ctx, 3);
    {
        GravP p{};
        p.m = m_g;
        p.a3 = a_g;
        p.rc2 = gp->r_cut * gp->r_cut;
        p.eps2 = gp->eps * gp->eps;
        for (int k = 0; k < 6; ++k) p.c[k] = gp->poly[k];
        p.n = n;
        p.count = cnt ? cnt + 2 : nullptr;
        p.swept = swc ? swc + 2 : nullptr;
        if ((rc = run_stage<GravStage>(ctx, lv, p, false, CRK_K_GRAVITY, nullptr, true))) return rc;
    }
    crk_step_mark(ctx, 4);
    // cotangents: the caller's (permuted into kernel order) or those of sum |a|^2 + sum_gas rho
    if (io->abar3) to_korder_kernel<<<g, 256, 0, st>>>(n, 3, lv->kperm_g, io->abar3, abar_g);
    if (io->rhobar) to_korder_kernel<<<g, 256, 0, st>>>(n, 1, lv->kperm, io->rhobar, rhob_k);
    if (io->Vbar) to_korder_kernel<<<g, 256, 0, st>>>(n, 1, lv->kperm, io->Vbar, Vb_k);
    cotangent_kernel<<<g, 256, 0, st>>>(n, a_g, lv->pos, io->abar3 ? nullptr : abar_g, io->rhobar ? nullptr : rhob_k);
    ctx->launches += 1 + (io->abar3 != nullptr) + (io->rhobar != nullptr) + (io->Vbar != nullptr);
    CRK_LAUNCH_CHECK(ctx, "step cotangents");
    {
        GravAdjP p{};
        p.m = m_g;
        p.abar = abar_g;
        p.gx3 = gx_g;
        p.gm = gm_g;
        p.rc2 = gp->r_cut * gp->r_cut;
        p.eps2 = gp->eps * gp->eps;
        for (int k = 0; k < 6; ++k) p.c[k] = gp->poly[k];
        p.n = n;
        p.count = nullptr;
        if ((rc = run_stage<GravAdjStage>(ctx, lv, p, false, CRK_K_GRAVITY_ADJOINT, nullptr, true))) return rc;
    }
    crk_step_mark(ctx, 5);
    {
        GeomAdjP p{m_k, V_k, rhob_k, io->Vbar ? Vb_k : nullptr, gx2_k, gm2_k, n, nullptr};
        if ((rc = run_stage<GeomAdjStage>(ctx, lv, p, true, CRK_K_GEOMETRY_ADJOINT, nullptr, true))) return rc;
    }
    crk_step_mark(ctx, 6);
    // outputs back to the caller's order (only those asked for)
    struct Out {
        float *dst;
        const float *src;
        int comp;
        const int32_t *perm;
    } outs[] = {{io->V, V_k, 1, lv->kinv},          {io->rho, rho_k, 1, lv->kinv},     {io->A, A_k, 1, lv->kinv},
                {io->B, B_k, 3, lv->kinv},          {io->gradA, gA_k, 3, lv->kinv},    {io->gradB, gB_k, 9, lv->kinv},
                {io->dvdt3, dv_k, 3, lv->kinv},     {io->dudt, du_k, 1, lv->kinv},     {io->a3, a_g, 3, lv->kinv_g},
                {io->gx3_grav, gx_g, 3, lv->kinv_g}, {io->gm_grav, gm_g, 1, lv->kinv_g}, {io->gx3_geom, gx2_k, 3, lv->kinv},
                {io->gm_geom, gm2_k, 1, lv->kinv},   {io->extras ? io->rho_r : nullptr, rhoR_k, 1, lv->kinv},
                {io->extras ? io->dvdx : nullptr, dvdx_k, 9, lv->kinv}};
    for (const Out &o : outs)
        if (o.dst)
            for (int c = 0; c < o.comp; ++c) {
                permute_col_kernel<<<g, 256, 0, st>>>(n, o.perm, o.src + (size_t)c * n, o.dst + (size_t)c * n);
                ++ctx->launches;
            }
    CRK_LAUNCH_CHECK(ctx, "step outputs");
    crk_step_mark(ctx, 7);
    return CRK_OK;
}
