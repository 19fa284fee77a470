// cert_internal.cuh -- device-side building blocks of the certificate step.
//
// Shared by the CUDA translation units of libcert.so only.  Arithmetic on
// squared distances is the fixed FP32 order of the public header (cert.h):
// D(i,j) = ((dx*dx + dy*dy) + dz*dz), dx = x_j - x_i, every operation an
// explicit round-to-nearest intrinsic so that no FMA contraction can occur.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace certk {

constexpr int kThreads = 256;
constexpr int kScanItems = 8;                          // items per thread in a scan tile
constexpr int kScanLatencyTiles = 3 * 148;             // scan grids below this: latency issue order
constexpr int kScanTile = kThreads * kScanItems;       // 2048 items per tile
constexpr int kSearchChunk = 4 * kThreads;             // sorted slots per search CTA
constexpr int kSearchSmallGrid = 4 * 148;              // half-size search chunks up to one wave
static_assert(kScanTile % kSearchChunk == 0, "the flag padding (a multiple of the scan tile) covers every search chunk");
constexpr int kMedianSample = 1024;                    // points sampled for the medians
constexpr int kMaxSearchRes = 2048;                    // search-grid cells per axis, cap
constexpr int kMaxExtend = 16;                         // face extensions before a warp scans the scene
constexpr uint32_t kSpinLimit = 1u << 22;              // bounded device waits
constexpr int kNlognTable = 1 << 16;                   // entries of each FP64 table below
constexpr int kLogTables = 5;                           // k ln k, ln k, 1/k, 1/ln k, k ln k fixed point
constexpr int kNlognFixBits = 40;                       // k ln k as round(k ln k * 2^40) in an int64

// Motion grid: a coarse per-scene grid of kMotionRes<DIM> cells per axis (a
// power of two, so cell coordinates and cell faces are exact in FP32) holding
// the largest squared displacement of the step's points in each cell, and its
// dilation by one cell (the largest over the 3^d block around each cell).
// kMotionStride cells are reserved per scene.
constexpr int kMotionStride = 512;
template <int DIM>
struct MotionRes {
    static constexpr int R = (DIM == 3) ? 8 : 16;
    static constexpr int cells = (DIM == 3) ? R * R * R : R * R;
};
static_assert(MotionRes<3>::cells <= kMotionStride && MotionRes<2>::cells <= kMotionStride, "motion grid stride");

// Latched device status bits (returned by cert_sync_result).
enum : uint32_t { ST_TIMEOUT = 1u, ST_NONFINITE = 2u, ST_EBOUND = 4u, ST_INDEX = 8u };

// Debug builds (-DCERT_DEBUG_BOUNDS, libcert_debug.so): index checks at the
// points where the release code relies on construction (search ranges inside
// their scene, neighbour indices written into certificates); a failed check
// latches ST_INDEX, which the host returns as CERT_EINTERNAL.  In release
// builds the checks compile to nothing.
#ifdef CERT_DEBUG_BOUNDS
#define CERT_CHECK(status, cond)                        \
    do {                                                \
        if (!(cond)) atomicOr((status), certk::ST_INDEX); \
    } while (0)
#else
#define CERT_CHECK(status, cond) \
    do {                         \
    } while (0)
#endif

// Step kernel modes.
enum : int { MODE_INIT = 0, MODE_STEP = 1, MODE_REBUILD = 2 };

// Strategies (values of cert_strategy).
enum : int { STRAT_AUTO = 0, STRAT_INC = 1, STRAT_REB = 2, STRAT_ALL = 3, STRAT_THR = 4 };

// Constant per-scene description (uploaded once at init).
struct SceneParams {
    int32_t pt_off, n;             // points [pt_off, pt_off + n)
    int32_t bucket_off, bucket_mask;  // hashed search-grid buckets [bucket_off, +mask+1)
    int32_t h_off, g_h;            // entropy grid: cells [h_off, h_off + g_h^dim), g_h per axis
    int32_t ap_off, ap_nch;        // all-pairs partials: base index, chunks per query
    int32_t ap_chunk, g_default;   // all-pairs chunk length; default search resolution
    int32_t s_off;                 // first slot of the scene in the quad-padded sorted array (multiple of 4)
    int32_t pad1;
};

// Per-scene state carried across steps.
struct SceneState {
    int32_t g_cur, g_next;         // search-grid cells per axis (this step, next step)
    int32_t strategy;              // strategy applied this step
    int32_t prev_nfront;           // previous step's |F|
    float prev_fail_ratio;         // previous n_failed / max(1, n_frontier)
    float prev_pred_ratio;         // previous selector output ln t_inc - ln t_reb
    float med_c, med_d2;           // truncated medians of the pre-step certificates
    float pred_inc, pred_reb;
    float inv_g;                   // 1/g_cur, rounded to nearest (face positions of the search)
    int32_t pad0;
    double S;                      // cumulative clock: sum of the steps' eps_t (FP64)
};

// Per-scene accumulators, zeroed at the start of every step.
struct SceneAcc {
    uint32_t eps_bits;             // max squared displacement (bit pattern, >= 0)
    int32_t occ;                   // occupied entropy cells (C)
    int32_t n_failed, n_missed;
    int32_t failed_cells, frontier_cells;
    int32_t n_searched;
    int32_t n_rho, n_rho_hit;      // local heuristic rho_i > 1/2: flagged, flagged and failed
    int32_t pad;
    double s_fail;                 // sum over cells of n ln n, failures
    double s_front;                // sum over cells of n ln n, detected frontier
    double f_sum[4];               // geometry audit: sums of x, y, z, |p|^2 over the failures
    double a_sum[4];               // ... and over every point of the scene
    unsigned long long search_cyc; // cost audit: summed per-query search cycles
    unsigned long long refresh_cyc;// ... and per-point scatter + refresh cycles
};

struct Top3 {
    float d0, d1, d2;
    int j0, j1, j2;
};

// Four smallest keys: the search keeps (nn, nn2, nn3) and bounds the rest by the fourth.
struct Top4 {
    float d0, d1, d2, d3;
    int j0, j1, j2, j3;
};

// ----------------------------------------------------------------------------- arithmetic

template <int DIM>
__device__ __forceinline__ float sqdist(const float4 a, const float4 b)
{
    // a = point i (the query), b = point j; differences are (j - i).
    const float dx = __fsub_rn(b.x, a.x);
    const float dy = __fsub_rn(b.y, a.y);
    float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    if (DIM == 3) {
        const float dz = __fsub_rn(b.z, a.z);
        s = __fadd_rn(s, __fmul_rn(dz, dz));
    }
    return s;
}

// Squared distances of two candidates a, b to the query p.  The differences
// and squares use packed FP32 pairs (Blackwell f32x2 arithmetic, every
// element rounded to nearest on its own); the two additions stay scalar
// add.rn.f32, which the code generator never fuses with a multiply.  Each
// result therefore equals sqdist<DIM>(p, .) bit for bit.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

template <int DIM>
__device__ __forceinline__ void sqdist_pair(const float4 p, const float4 a, const float4 b, float &Da, float &Db)
{
    unsigned long long dx, dy, sx, sy;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(pack2(a.x, b.x)), "l"(pack2(p.x, p.x)));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(pack2(a.y, b.y)), "l"(pack2(p.y, p.y)));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sx) : "l"(dx));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sy) : "l"(dy));
    float xa, xb, ya, yb;
    unpack2(sx, xa, xb);
    unpack2(sy, ya, yb);
    Da = __fadd_rn(xa, ya);
    Db = __fadd_rn(xb, yb);
    if (DIM == 3) {
        unsigned long long dz, sz;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(pack2(a.z, b.z)), "l"(pack2(p.z, p.z)));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sz) : "l"(dz));
        float za, zb;
        unpack2(sz, za, zb);
        Da = __fadd_rn(Da, za);
        Db = __fadd_rn(Db, zb);
    }
}

// Squared distances of one candidate c to two queries whose coordinates are
// packed pairwise (qx = {x0, x1}, ...): packed differences and squares, scalar
// additions -- bit-identical to sqdist<DIM>(query, c) for each query.
template <int DIM>
__device__ __forceinline__ void sqdist_qpair(unsigned long long qx, unsigned long long qy, unsigned long long qz,
                                             const float4 c, float &D0, float &D1)
{
    unsigned long long dx, dy, sx, sy;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(pack2(c.x, c.x)), "l"(qx));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(pack2(c.y, c.y)), "l"(qy));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sx) : "l"(dx));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sy) : "l"(dy));
    float x0, x1, y0, y1;
    unpack2(sx, x0, x1);
    unpack2(sy, y0, y1);
    D0 = __fadd_rn(x0, y0);
    D1 = __fadd_rn(x1, y1);
    if (DIM == 3) {
        unsigned long long dz, sz;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(pack2(c.z, c.z)), "l"(qz));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(sz) : "l"(dz));
        float z0, z1;
        unpack2(sz, z0, z1);
        D0 = __fadd_rn(D0, z0);
        D1 = __fadd_rn(D1, z1);
    }
}

// Squared distances of four candidates, held as quad rows X = (x0..x3),
// Y, Z, to the query whose coordinates are packed twice (px = {x, x}, ...):
// packed differences and squares, scalar additions in the order of sqdist,
// so each result equals sqdist<DIM>(query, candidate k) bit for bit.
template <int DIM>
__device__ __forceinline__ void sqdist_quad(unsigned long long px, unsigned long long py, unsigned long long pz,
                                            const float4 X, const float4 Y, const float4 Z, float &D0, float &D1,
                                            float &D2, float &D3)
{
    unsigned long long ax, bx, ay, by;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ax) : "l"(pack2(X.x, X.y)), "l"(px));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bx) : "l"(pack2(X.z, X.w)), "l"(px));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ay) : "l"(pack2(Y.x, Y.y)), "l"(py));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(by) : "l"(pack2(Y.z, Y.w)), "l"(py));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(ax) : "l"(ax));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(bx) : "l"(bx));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(ay) : "l"(ay));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(by) : "l"(by));
    float x0, x1, x2, x3, y0, y1, y2, y3;
    unpack2(ax, x0, x1);
    unpack2(bx, x2, x3);
    unpack2(ay, y0, y1);
    unpack2(by, y2, y3);
    D0 = __fadd_rn(x0, y0);
    D1 = __fadd_rn(x1, y1);
    D2 = __fadd_rn(x2, y2);
    D3 = __fadd_rn(x3, y3);
    if (DIM == 3) {
        unsigned long long az, bz;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(az) : "l"(pack2(Z.x, Z.y)), "l"(pz));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bz) : "l"(pack2(Z.z, Z.w)), "l"(pz));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(az) : "l"(az));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(bz) : "l"(bz));
        float z0, z1, z2, z3;
        unpack2(az, z0, z1);
        unpack2(bz, z2, z3);
        D0 = __fadd_rn(D0, z0);
        D1 = __fadd_rn(D1, z1);
        D2 = __fadd_rn(D2, z2);
        D3 = __fadd_rn(D3, z3);
    }
}

// ----------------------------------------------------------------------------- sorted points

// The points in search-grid order are stored in quads: quad q holds slots
// 4q .. 4q+3 as four float4 rows (x0..x3), (y0..y3), (z0..z3), (index bits).
// Every scene starts on a quad (SceneParams::s_off); slots past a scene's end
// up to the next quad hold NaN coordinates and index -1, so a whole quad can
// be evaluated and the padding never enters a top-k.
__device__ __forceinline__ void sorted_store(float4 *quads, int k, float x, float y, float z, int id)
{
    float *f = reinterpret_cast<float *>(quads + (size_t)(k >> 2) * 4) + (k & 3);
    f[0] = x;
    f[4] = y;
    f[8] = z;
    f[12] = __int_as_float(id);
}

__device__ __forceinline__ int sorted_index(const float4 *quads, int k)
{
    return __float_as_int(reinterpret_cast<const float *>(quads + (size_t)(k >> 2) * 4)[12 + (k & 3)]);
}

// Cell coordinate of one axis: floor(x * g) clamped to [0, g-1].
__device__ __forceinline__ int cell_coord(float x, int g, float gf)
{
    const float t = __fmul_rn(x, gf);
    if (!(t >= 0.0f)) return 0;
    if (t >= gf) return g - 1;
    return (int)floorf(t);
}

// Motion-grid cell of a position: floor(x * R) per axis clamped to [0, R-1];
// R is a power of two, so x * R is exact.
template <int DIM>
__device__ __forceinline__ int motion_cell(const float4 p)
{
    constexpr int R = MotionRes<DIM>::R;
    const int mx = cell_coord(p.x, R, (float)R);
    const int my = cell_coord(p.y, R, (float)R);
    if (DIM == 2) return my * R + mx;
    return (cell_coord(p.z, R, (float)R) * R + my) * R + mx;
}

// Dilation of a scene's motion grid: dst[c] = max of src over the cells of the
// 3^d block around c (clamped to the grid), as one pass per axis (a max over
// a box is the composition of the max over its three edges).  t0 and t1 are
// shared-memory scratch of MotionRes<DIM>::cells words each; src and dst may
// be global or shared.  Called by all nt threads of the block (it holds
// barriers); thread tid produces cells tid, tid + nt, ...
template <int DIM>
__device__ __forceinline__ void dilate_motion(const uint32_t *src, uint32_t *t0, uint32_t *t1, uint32_t *dst,
                                              int tid, int nt)
{
    constexpr int R = MotionRes<DIM>::R, C = MotionRes<DIM>::cells;
    // axis 0 (x, stride 1): src -> t0
    for (int c = tid; c < C; c += nt) {
        const int x = c % R;
        uint32_t m = src[c];
        if (x > 0) m = max(m, src[c - 1]);
        if (x < R - 1) m = max(m, src[c + 1]);
        t0[c] = m;
    }
    __syncthreads();
    // axis 1 (y, stride R): t0 -> t1 (2-D: -> dst)
    uint32_t *d1 = (DIM == 3) ? t1 : dst;
    for (int c = tid; c < C; c += nt) {
        const int y = (c / R) % R;
        uint32_t m = t0[c];
        if (y > 0) m = max(m, t0[c - R]);
        if (y < R - 1) m = max(m, t0[c + R]);
        d1[c] = m;
    }
    if (DIM == 3) {
        __syncthreads();
        // axis 2 (z, stride R^2): t1 -> dst
        for (int c = tid; c < C; c += nt) {
            const int z = c / (R * R);
            uint32_t m = t1[c];
            if (z > 0) m = max(m, t1[c - R * R]);
            if (z < R - 1) m = max(m, t1[c + R * R]);
            dst[c] = m;
        }
    }
}

// Distance from p to the nearest face of the 3^d motion-grid block around its
// cell that is not on the grid edge (rounded down; +inf when every face is on
// the edge).  A point outside the block is at least this far from p: its cell
// lies beyond one of those faces (edge cells are clamped, nothing lies beyond).
template <int DIM>
__device__ __forceinline__ float motion_block_face(const float4 p)
{
    constexpr int R = MotionRes<DIM>::R;
    constexpr float inv = 1.0f / (float)R;   // exact: R is a power of two
    float f = __int_as_float(0x7f800000);
    const float c[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const int m = cell_coord(c[k], R, (float)R);
        if (m - 1 > 0) f = fminf(f, __fsub_rd(c[k], (float)(m - 1) * inv));
        if (m + 1 < R - 1) f = fminf(f, __fsub_rd((float)(m + 2) * inv, c[k]));
    }
    return f;
}

// Latched device status bits; the cells of a
// row occupy consecutive buckets (mod T).  When the whole grid fits in the
// bucket table (g^dim <= T) the mapping is the plain linear cell index and
// buckets never mix cells; otherwise the row is placed by a 32-bit integer
// finalizer (the MurmurHash3 fmix32 mixing steps) and collisions only add
// candidates, never remove one.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

template <int DIM>
__device__ __forceinline__ bool grid_is_dense(int g, int T)
{
    const long long cells = (DIM == 3) ? (long long)g * g * g : (long long)g * g;
    return cells <= (long long)T;
}

template <int DIM>
__device__ __forceinline__ uint32_t row_base(int cy, int cz, int g, bool dense)
{
    if (dense) return (DIM == 3) ? (uint32_t)((cz * g + cy) * g) : (uint32_t)(cy * g);
    return mix32((DIM == 3) ? ((uint32_t)cz * 0x10001u + (uint32_t)cy) : (uint32_t)cy);
}

template <typename T>
__device__ __forceinline__ void swapv(T &a, T &b)
{
    const T t = a;
    a = b;
    b = t;
}

__device__ __forceinline__ bool key_less(float da, int ja, float db, int jb)
{
    return da < db || (da == db && ja < jb);
}

__device__ __forceinline__ void top3_reset(Top3 &t)
{
    t.d0 = t.d1 = t.d2 = __int_as_float(0x7f800000);
    t.j0 = t.j1 = t.j2 = 0x7fffffff;
}

// Insert (D, j) keeping the three lexicographically smallest distinct keys.
// A candidate index already held is ignored (a hashed bucket may be visited twice).
__device__ __forceinline__ void top3_insert(Top3 &t, float D, int j)
{
    if (!key_less(D, j, t.d2, t.j2)) return;
    if (j == t.j0 || j == t.j1) return;
    if (key_less(D, j, t.d1, t.j1)) {
        t.d2 = t.d1;
        t.j2 = t.j1;
        if (key_less(D, j, t.d0, t.j0)) {
            t.d1 = t.d0;
            t.j1 = t.j0;
            t.d0 = D;
            t.j0 = j;
        } else {
            t.d1 = D;
            t.j1 = j;
        }
    } else {
        t.d2 = D;
        t.j2 = j;
    }
}

__device__ __forceinline__ void top4_reset(Top4 &t)
{
    t.d0 = t.d1 = t.d2 = t.d3 = __int_as_float(0x7f800000);
    t.j0 = t.j1 = t.j2 = t.j3 = 0x7fffffff;
}

// Insert (D, j) keeping the four lexicographically smallest distinct keys;
// an index already held is ignored.
__device__ __forceinline__ void top4_insert(Top4 &t, float D, int j)
{
    if (!key_less(D, j, t.d3, t.j3)) return;
    if (j == t.j0 || j == t.j1 || j == t.j2) return;
    if (key_less(D, j, t.d2, t.j2)) {
        t.d3 = t.d2;
        t.j3 = t.j2;
        if (key_less(D, j, t.d1, t.j1)) {
            t.d2 = t.d1;
            t.j2 = t.j1;
            if (key_less(D, j, t.d0, t.j0)) {
                t.d1 = t.d0;
                t.j1 = t.j0;
                t.d0 = D;
                t.j0 = j;
            } else {
                t.d1 = D;
                t.j1 = j;
            }
        } else {
            t.d2 = D;
            t.j2 = j;
        }
    } else {
        t.d3 = D;
        t.j3 = j;
    }
}

// Conservative lower bound on sqrt(x): correctly rounded down, then shrunk by
// 2^-20 relative to absorb the rounding of the squared distance itself.
__device__ __forceinline__ float sqrt_lower(float x)
{
    return __fmul_rd(__fsqrt_rd(x), 1.0f - 0x1p-20f);
}

__device__ __forceinline__ float eps_of(const SceneAcc *acc, int s)
{
    return __fsqrt_rn(__uint_as_float(acc[s].eps_bits));
}

// The host-computed FP64 tables, kNlognTable entries each, back to back:
// k ln k, ln k, 1/k, 1/ln k (0 for k < 2), and k ln k in fixed point.  FP64 logarithms and divisions
// are slow on this part; a lookup replaces each of them on the device.
__device__ __forceinline__ double tab_ln(const double *tab, int k) { return tab[kNlognTable + k]; }
__device__ __forceinline__ double tab_inv(const double *tab, int k) { return tab[2 * kNlognTable + k]; }
__device__ __forceinline__ double tab_inv_ln(const double *tab, int k) { return tab[3 * kNlognTable + k]; }
// k ln k in fixed point (kNlognFixBits fraction bits): sums of these are exact and
// order-independent, and any sum over a scene's cells stays below 2^58.
__device__ __forceinline__ long long tab_nlogn_fix(const double *tab, int k)
{
    return reinterpret_cast<const long long *>(tab + 4 * kNlognTable)[k];
}

// n ln n increment when a histogram count goes old -> old + 1 (FP64).
__device__ __forceinline__ double nlogn_step(const double *tab, int old)
{
    if (old + 1 < kNlognTable) return tab[old + 1] - tab[old];
    const double a = (double)old, b = (double)(old + 1);
    return b * log(b) - a * log(a);
}

// ----------------------------------------------------------------------------- memory order

__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// A 64-bit word that carries everything its reader needs (a flag and a value)
// needs no ordering against other memory: relaxed, single-copy atomic access.
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ----------------------------------------------------------------------------- warp helpers

constexpr unsigned kFull = 0xffffffffu;

// Lanes of a warp holding consecutive points form contiguous runs of equal
// scene id (scenes are contiguous ranges).  Each helper reduces within the run
// and lets the run's lowest lane issue one atomic.  s < 0 marks an idle lane.
// Scene of point (or sorted slot) i.  A context of one scene needs no lookup,
// so the loads that depend on the scene (its parameters and state) are not
// held up behind one: a lone scene's steps are chains of dependent accesses.
__device__ __forceinline__ int scene_of_point(const int32_t *scene_of, int n_scenes, int i)
{
    return n_scenes == 1 ? 0 : scene_of[i];
}

// Increment counter k of a per-bucket or per-entropy-cell count array and
// return its previous value.  c16: the counts are 16-bit, two per word (every
// scene has fewer than 65,536 points, so no count reaches 2^16 and the low
// half never carries into the high one); otherwise one 32-bit count per entry.
__device__ __forceinline__ int count_inc(int32_t *arr, int k, int c16)
{
    if (c16) {
        const uint32_t sh = (uint32_t)(k & 1) << 4;
        return (int)((atomicAdd(reinterpret_cast<uint32_t *>(arr) + (k >> 1), 1u << sh) >> sh) & 0xffffu);
    }
    return atomicAdd(arr + k, 1);
}

__device__ __forceinline__ unsigned scene_run_mask(int s)
{
    return __match_any_sync(kFull, s);
}

__device__ __forceinline__ bool run_leader(unsigned mask)
{
    return (int)(threadIdx.x & 31) == __ffs(mask) - 1;
}

__device__ __forceinline__ int run_sum_i32(unsigned mask, int v)
{
    return (int)__reduce_add_sync(mask, (unsigned)v);
}

__device__ __forceinline__ unsigned run_max_u32(unsigned mask, unsigned v)
{
    return __reduce_max_sync(mask, v);
}

__device__ __forceinline__ double run_sum_f64(unsigned mask, double v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double w = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32 && ((mask >> (lane + o)) & 1u)) v += w;
    }
    return v;  // complete in the run's lowest lane
}

// ----------------------------------------------------------------------------- block scan

// Exclusive scan of one value per thread across a block of NT threads (a
// multiple of 32, at most 1024); returns the exclusive prefix, and the block
// total through *total.  smem_warp holds NT / 32 words.
template <int NT = kThreads>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total, uint32_t *smem_warp)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 32 of them");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < NT / 32) ? smem_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) smem_warp[lane] = w;  // inclusive warp prefixes
    }
    __syncthreads();
    const uint32_t warp_base = warp ? smem_warp[warp - 1] : 0u;
    *total = smem_warp[NT / 32 - 1];
    return warp_base + x - v;
}

}  // namespace certk
