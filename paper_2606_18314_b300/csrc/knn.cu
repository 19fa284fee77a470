// knn.cu -- k-nearest-neighbour certificates (include/cert_knn.h).
//
// One scene per context.  The certificate of point i is its sorted list of
// S = k + 1 + kExtra candidates under the key (D, j) -- the k nearest, the
// (k+1)-th (whose gap c^(k)_i = d_{k+1} - d_k is the clearance) and kExtra
// spares -- plus L_i, a lower bound on the distance from i to every point
// outside the list.  A step (Algorithm 1, one rank further out):
//
//   k_knn_prepare   displacement D(p_i, p'_i) (kept in w), eps_t^2 by a max,
//                   bucket of p'_i in the hashed grid and its rank there
//   k_knn_scan_*    exclusive scan of the bucket counts -> bucket starts
//                   (three passes; the counts are zeroed for the next step)
//   k_knn_refresh   scatter of p'_i into bucket order; the frontier test
//                   c^(k) <= 4 eps_t + tau (Lemma 1); the O(k) refresh: the S
//                   stored candidates' fresh keys, sorted, hold the exact
//                   top-(k+1) when the (k+1)-th is below (L_i - shrink_i)^2,
//                   shrink_i >= |p'_i - p_i| + eps_t (triangle inequality);
//                   every other point joins the search list with a hint, the
//                   fresh (k+1)-th distance (k+1 points lie that close)
//   k_knn_search    grid search: the cells meeting the ball of 1.15 x hint
//                   (without a hint, the 3^d block of Algorithm 1), grown by
//                   whole layers until the (k+1)-th key is below the squared
//                   distance to every face not on the grid edge (Cor. A.2);
//                   a box of more than kMaxHintRows rows, or one still open
//                   after kMaxRings layers, goes to the far list
//   k_knn_heavy     one warp per query whose box held more than kHeavy
//                   candidates (a coarse cell over a dense cluster): the same
//                   box, 32 lanes at a time
//   k_knn_far       one block per far query: every point of the scene
//   k_knn_finalize  the step's scalars; the next step's grid from the median
//                   (k+1)-th distance of a 1024-point sample
//
// The grid is hashed as in the k = 2 path: the cells of one row map to
// consecutive buckets (mod T) from a mixed row base, T = next_pow2(n) (at
// most 2^23) buckets, so the cell side can follow the data without a dense
// table; a bucket shared by two rows only adds candidates, and a candidate
// seen twice is inserted once.  When the sample's (k+1)-th distances span two
// scales (upper over lower quartile >= kTwoLevelRatio, e.g. dense clusters in
// a sparse background) a second, coarser level is built from the upper
// quartile; each query searches the finer level whose box has at most
// kFineRows rows.  Both levels share one bucket array (level 1 at offset T)
// and one scan.  Lists are rank-major ([r * n + i]).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "cert_internal.cuh"
#include "cert_launch.h"
#include "cert_knn.h"

using namespace certk;

namespace {

constexpr int kKnnThreads = kThreads;                 // 256 (block_exclusive_scan assumes it)
constexpr int kCellTile = kThreads * 8;               // buckets per scan tile
constexpr int kMaxBucketsLog2 = 23;                   // per level; two levels share the scan
constexpr int kMaxParts = (2 << kMaxBucketsLog2) / kCellTile;   // 8192 = 256 threads x 32 partials
constexpr int kExtra = 2;                             // spare candidates beyond the (k+1)-th
constexpr int kMaxRings = 8;                          // layers grown before the far pass
constexpr int kMaxHintRows = 256;                     // rows of a hinted box; more go to the far pass
constexpr int kFineRows = 64;                         // rows of a level-0 box before level 1 is used
constexpr int kHeavy = 384;                           // candidates one thread scans before a warp takes over
constexpr float kTwoLevelRatio = 4.0f;                // quartile ratio of the distances for two levels
constexpr int kMaxGrid = 2048;                        // grid cells per axis, cap
constexpr int kSample = 1024;                         // points sampled for the median
constexpr float kKnnFaceSlack = 0x1p-17f;
constexpr float kKnnHintGrow = 1.15f;

struct KnnCounters {
    uint32_t eps_bits;       // max squared displacement (bit pattern of a non-negative float)
    int32_t need_count;      // entries of the search list
    int32_t far_count;       // entries of the far list
    int32_t heavy_count;     // entries of the heavy list
    int32_t n_frontier, n_failed, n_missed, n_searched;
    int32_t search_next;     // the search list's next unclaimed batch of 32 (k_knn_search)
};

// One level of the hashed grid.
struct KnnLevel {
    int32_t g;               // cells per axis
    float gf, inv_g;         // g as a float, 1/g rounded to nearest
    int32_t dense;           // g^dim <= T: the plain linear index, no collisions
};

// The grid of the current step (written by k_knn_finalize for the next).
struct KnnGrid {
    KnnLevel lv[2];
    int32_t levels;          // 1 or 2
};

struct KnnArgs {
    int n, k, S, T;          // points, k, stored ranks, buckets
    uint32_t mask;           // T - 1
    int mode, strategy;      // MODE_INIT / MODE_STEP; STRAT_INC / STRAT_REB
    float declared_eps, cell_scale;
    const float *in;         // caller's positions [n][dim]
    const float4 *pos_old;   // previous positions
    float4 *pos_new;         // this step's positions, w = squared displacement
    int32_t *bucket, *rank;  // [2][n] per level and point: bucket (level 1: + T), rank inside it
    int32_t *cnt;            // [2T] counts (zero between steps)
    int32_t *start;          // [2T + 1] bucket starts
    int32_t *part;           // [kMaxParts] per-tile sums
    float4 *spos;            // [2n] points in bucket order, level 0 then level 1: x, y, z, index bits
    int32_t *idx;            // [S][n]
    float *d2;               // [S][n]
    float *L;                // [n] lower bound; for search-list points, the hint
    uint8_t *front, *failed;
    int32_t *need, *far;     // search list, far list
    int32_t *heavy;          // queries handed from a thread to a warp
    KnnCounters *ctr;
    KnnGrid *grid;
    uint32_t *status;
    cert_knn_result *res;
};

__device__ __forceinline__ float knn_eps(const KnnCounters *c)
{
    return __fsqrt_rn(__uint_as_float(c->eps_bits));
}

template <int DIM>
__device__ __forceinline__ uint32_t knn_bucket(const KnnArgs &a, const KnnLevel &gr, float4 p)
{
    const int x = cell_coord(p.x, gr.g, gr.gf);
    const int y = cell_coord(p.y, gr.g, gr.gf);
    const int z = (DIM == 3) ? cell_coord(p.z, gr.g, gr.gf) : 0;
    return (row_base<DIM>(y, z, gr.g, gr.dense != 0) + (uint32_t)x) & a.mask;
}

// Insert (D, j) into the sorted list of KH keys, dropping the last, unless j
// is held already; the caller has checked that (D, j) is below the last key.
template <int KH>
__device__ __forceinline__ void list_insert(float (&d)[KH], int (&jj)[KH], float D, int J)
{
    bool dup = false;
#pragma unroll
    for (int s = 0; s < KH; ++s) dup |= jj[s] == J;
    if (dup) return;
    bool placed = false;
#pragma unroll
    for (int s = KH - 1; s > 0; --s) {
        if (!placed) {
            if (key_less(D, J, d[s - 1], jj[s - 1])) {
                d[s] = d[s - 1];
                jj[s] = jj[s - 1];
            } else {
                d[s] = D;
                jj[s] = J;
                placed = true;
            }
        }
    }
    if (!placed) {
        d[0] = D;
        jj[0] = J;
    }
}

template <int KH>
__device__ __forceinline__ void list_reset(float (&d)[KH], int (&jj)[KH])
{
#pragma unroll
    for (int s = 0; s < KH; ++s) {
        d[s] = __int_as_float(0x7f800000);
        jj[s] = 0x7fffffff;
    }
}

// v[r] for a runtime r without local memory.
template <int KH, typename T>
__device__ __forceinline__ T pick(const T (&v)[KH], int r, T dflt)
{
    T out = dflt;
#pragma unroll
    for (int s = 0; s < KH; ++s)
        if (s == r) out = v[s];
    return out;
}

// ---------------------------------------------------------------------------- prepare

template <int DIM>
__global__ void __launch_bounds__(kKnnThreads) k_knn_prepare(const KnnArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const KnnGrid gr = *a.grid;
    uint32_t dbits = 0u;
    if (i < a.n) {
        float4 p;
        p.x = a.in[(size_t)i * DIM];
        p.y = a.in[(size_t)i * DIM + 1];
        p.z = (DIM == 3) ? a.in[(size_t)i * DIM + 2] : 0.0f;
        p.w = 0.0f;
        if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) atomicOr(a.status, ST_NONFINITE);
        if (a.mode == MODE_STEP) {
            p.w = sqdist<DIM>(a.pos_old[i], p);      // D(p_i, p'_i), Algorithm 1's eps_t
            dbits = __float_as_uint(p.w);
        }
        a.pos_new[i] = p;
        const uint32_t b = knn_bucket<DIM>(a, gr.lv[0], p);
        a.bucket[i] = (int32_t)b;
        a.rank[i] = atomicAdd(&a.cnt[b], 1);
        if (gr.levels == 2) {
            const uint32_t b1 = (uint32_t)a.T + knn_bucket<DIM>(a, gr.lv[1], p);
            a.bucket[a.n + i] = (int32_t)b1;
            a.rank[a.n + i] = atomicAdd(&a.cnt[b1], 1);
        }
    }
    if (a.mode == MODE_STEP) {
        // non-negative floats order as their bit patterns
        const uint32_t m = __reduce_max_sync(kFull, dbits);
        if ((threadIdx.x & 31) == 0 && m) atomicMax(&a.ctr->eps_bits, m);
    }
}

// ---------------------------------------------------------------------------- scan of the bucket counts

__global__ void __launch_bounds__(kKnnThreads) k_knn_scan_reduce(const KnnArgs a)
{
    __shared__ uint32_t s_warp[kKnnThreads / 32];
    const int base = blockIdx.x * kCellTile + threadIdx.x * 8;
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (base + k < 2 * a.T) sum += (uint32_t)a.cnt[base + k];
    uint32_t tot;
    block_exclusive_scan(sum, &tot, s_warp);
    if (threadIdx.x == 0) a.part[blockIdx.x] = (int32_t)tot;
}

__global__ void __launch_bounds__(kKnnThreads) k_knn_scan_parts(const KnnArgs a, int nparts)
{
    __shared__ uint32_t s_warp[kKnnThreads / 32];
    constexpr int per = kMaxParts / kKnnThreads;   // 32
    const int base = threadIdx.x * per;
    uint32_t v[per];
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        v[k] = (base + k < nparts) ? (uint32_t)a.part[base + k] : 0u;
        sum += v[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(sum, &tot, s_warp);
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if (base + k < nparts) a.part[base + k] = (int32_t)run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kKnnThreads) k_knn_scan_down(const KnnArgs a)
{
    __shared__ uint32_t s_warp[kKnnThreads / 32];
    const int base = blockIdx.x * kCellTile + threadIdx.x * 8;
    uint32_t v[8];
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = (base + k < 2 * a.T) ? (uint32_t)a.cnt[base + k] : 0u;
        sum += v[k];
    }
    uint32_t tot;
    uint32_t run = (uint32_t)a.part[blockIdx.x] + block_exclusive_scan(sum, &tot, s_warp);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (base + k < 2 * a.T) {
            a.start[base + k] = (int32_t)run;
            a.cnt[base + k] = 0;              // ready for the next step's histogram
        }
        run += v[k];
    }
    // the total: n with one level, 2n with two
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kKnnThreads - 1) a.start[2 * a.T] = (int32_t)run;
}

// ---------------------------------------------------------------------------- refresh

__device__ __forceinline__ void append_list(int32_t *list, int32_t *count, bool take, int i)
{
    const unsigned m = __ballot_sync(kFull, take);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (take) list[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// Does the new top-k (hj[0..k)) hold a point outside the old one (oj[0..k))?
template <int KB, int KH>
__device__ __forceinline__ int set_changed(const int (&oj)[KB], const int (&hj)[KH], int k)
{
    int changed = 0;
#pragma unroll
    for (int s = 0; s < KB; ++s)
        if (s < k) {
            bool found = false;
#pragma unroll
            for (int r = 0; r < KB; ++r) found |= oj[r] == hj[s];
            changed |= !found;
        }
    return changed;
}

template <int DIM, int KB>
__global__ void __launch_bounds__(kKnnThreads) k_knn_refresh(const KnnArgs a)
{
    constexpr int KS = KB + 1 + kExtra;        // stored keys, compile-time bound
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.n;
    bool need = false;
    int inF = 0, changed = 0, missed = 0;
    if (valid) {
        const float4 p = a.pos_new[i];
        const float4 q = make_float4(p.x, p.y, p.z, __int_as_float(i));
        a.spos[a.start[a.bucket[i]] + a.rank[i]] = q;
        if (a.grid->levels == 2) a.spos[a.start[a.bucket[a.n + i]] + a.rank[a.n + i]] = q;
        if (a.mode != MODE_STEP) {
            need = true;
            a.L[i] = 0.0f;                     // no list yet: no hint
        } else {
            const int n = a.n, k = a.k, S = a.S;
            const float eps = knn_eps(a.ctr);
            // frontier from the pre-step certificate (Lemma 1 at rank k)
            const float dk = __fsqrt_rn(a.d2[(size_t)(k - 1) * n + i]);
            const float dk1 = __fsqrt_rn(a.d2[(size_t)k * n + i]);
            const float c = __fsub_rn(dk1, dk);
            const float tau = __fmul_rn(0x1p-20f, __fadd_rn(__fadd_rn(dk, dk1), eps));
            inF = (c <= __fadd_rn(__fmul_rn(4.0f, eps), tau)) ? 1 : 0;
            a.front[i] = (uint8_t)inF;
            // fresh keys of the stored candidates, sorted
            float hd[KS];
            int hj[KS], oj[KB];
            list_reset<KS>(hd, hj);
#pragma unroll
            for (int r = 0; r < KB; ++r) oj[r] = -1;
#pragma unroll
            for (int r = 0; r < KS; ++r) {
                if (r < S) {
                    // ranks 0 .. k always hold a point; a spare rank is -1 when
                    // the search that wrote the list found fewer candidates
                    const int j = a.idx[(size_t)r * n + i];
                    if (r < KB && r < k) oj[r] = j;
                    if ((unsigned)j < (unsigned)n) {
                        const float D = sqdist<DIM>(p, a.pos_new[j]);
                        if (key_less(D, j, hd[KS - 1], hj[KS - 1])) list_insert<KS>(hd, hj, D, j);
                    }
                }
            }
            const float Dk = pick<KS>(hd, k, 0.0f);
            // every point outside the stored list was at least L away and both
            // ends moved: now at least L - (|p'_i - p_i| + eps_t)
            const float shrink = __fmul_ru(__fadd_ru(__fsqrt_ru(p.w), eps), 1.0f + 0x1p-18f);
            const float Lnew = __fsub_rd(a.L[i], shrink);
            if (a.strategy == STRAT_INC && Lnew > 0.0f && __fmul_ru(Dk, 1.0f + 0x1p-19f) < __fmul_rd(Lnew, Lnew)) {
#pragma unroll
                for (int r = 0; r < KS; ++r)
                    if (r < S) {
                        a.idx[(size_t)r * n + i] = (hj[r] != 0x7fffffff) ? hj[r] : -1;
                        a.d2[(size_t)r * n + i] = hd[r];
                    }
                changed = set_changed<KB, KS>(oj, hj, k);
                a.L[i] = Lnew;
                a.failed[i] = (uint8_t)changed;
                missed = changed && !inF;
            } else {
                need = true;
                // k+1 points lie within the fresh (k+1)-th distance: the search
                // box needs to reach no farther
                a.L[i] = __fsqrt_ru(Dk);
            }
        }
    }
    append_list(a.need, &a.ctr->need_count, valid && need, i);
    if (a.mode == MODE_STEP) {
        const int f = __reduce_add_sync(kFull, inF);
        const int nc = __reduce_add_sync(kFull, changed);
        const int nm = __reduce_add_sync(kFull, missed);
        if ((threadIdx.x & 31) == 0) {
            if (f) atomicAdd(&a.ctr->n_frontier, f);
            if (nc) atomicAdd(&a.ctr->n_failed, nc);
            if (nm) atomicAdd(&a.ctr->n_missed, nm);
        }
    }
}

// ---------------------------------------------------------------------------- search

template <int DIM, int KH>
__device__ __forceinline__ void visit_slots(const KnnArgs &a, int lo, int hi, int step, const float4 p, int self,
                                            float (&hd)[KH], int (&hj)[KH])
{
    CERT_CHECK(a.status, lo >= 0 && hi <= 2 * a.n);
    for (int s = lo; s < hi; s += step) {
        const float4 q = a.spos[s];
        const int j = __float_as_int(q.w);
        const float D = sqdist<DIM>(p, q);
        if (j != self && key_less(D, j, hd[KH - 1], hj[KH - 1])) list_insert<KH>(hd, hj, D, j);
    }
}

// Cells [xl, xh] of row (y, z): consecutive buckets from the row base, split
// in two where they wrap around the table.
// Slot ranges of the cells [xl, xh] of row (y, z): consecutive buckets from
// the row base, split in two where they wrap around the table.
template <int DIM>
__device__ __forceinline__ int row_slots(const KnnArgs &a, const KnnLevel &gr, int boff, int y, int z, int xl,
                                         int xh, int2 &r0, int2 &r1)
{
    r0 = r1 = make_int2(0, 0);
    const int len = xh - xl + 1;
    if (len <= 0) return 0;
    const int32_t *st = a.start + boff;
    if (len >= a.T) {
        r0 = make_int2(st[0], st[a.T]);
        return 1;
    }
    const int b0 = (int)((row_base<DIM>(y, z, gr.g, gr.dense != 0) + (uint32_t)xl) & a.mask);
    if (b0 + len <= a.T) {
        r0 = make_int2(st[b0], st[b0 + len]);
        return 1;
    }
    r0 = make_int2(st[b0], st[a.T]);
    r1 = make_int2(st[0], st[b0 + len - a.T]);
    return 2;
}

// Visit one row with lanes [lane, lane + step, ...) of its slots; budget
// counts the candidates still allowed (a thread-level search gives up, and
// leaves the query to a warp, once it would exceed kHeavy).
template <int DIM, int KH>
__device__ __forceinline__ void visit_row(const KnnArgs &a, const KnnLevel &gr, int boff, int y, int z, int xl,
                                          int xh, const float4 p, int self, float (&hd)[KH], int (&hj)[KH],
                                          long long &budget, int lane = 0, int step = 1)
{
    int2 r0, r1;
    const int nr = row_slots<DIM>(a, gr, boff, y, z, xl, xh, r0, r1);
    if (nr == 0) return;
    budget -= (long long)(r0.y - r0.x) + (r1.y - r1.x);
    if (budget < 0) return;
    visit_slots<DIM, KH>(a, r0.x + lane, r0.y, step, p, self, hd, hj);
    if (nr == 2) visit_slots<DIM, KH>(a, r1.x + lane, r1.y, step, p, self, hd, hj);
}

// Visit the cells of box [x0,x1] x [y0,y1] x [z0,z1] that are not in the box
// [ox0,ox1] x [oy0,oy1] x [oz0,oz1] (pass ox0 > ox1 for none).
template <int DIM, int KH>
__device__ __forceinline__ void visit_shell(const KnnArgs &a, const KnnLevel &gr, int boff, int x0, int x1, int y0,
                                            int y1, int z0, int z1, int ox0, int ox1, int oy0, int oy1, int oz0,
                                            int oz1, const float4 p, int self, float (&hd)[KH], int (&hj)[KH],
                                            long long &budget, int lane = 0, int step = 1)
{
    for (int z = z0; z <= z1 && budget >= 0; ++z)
        for (int y = y0; y <= y1 && budget >= 0; ++y) {
            const bool inner = ox0 <= ox1 && y >= oy0 && y <= oy1 && z >= oz0 && z <= oz1;
            if (!inner) {
                visit_row<DIM, KH>(a, gr, boff, y, z, x0, x1, p, self, hd, hj, budget, lane, step);
            } else {
                visit_row<DIM, KH>(a, gr, boff, y, z, x0, ox0 - 1, p, self, hd, hj, budget, lane, step);
                visit_row<DIM, KH>(a, gr, boff, y, z, ox1 + 1, x1, p, self, hd, hj, budget, lane, step);
            }
        }
}

// The box of the cells of level gr that meet the ball of radius R about p.
template <int DIM>
__device__ __forceinline__ void ball_box(const KnnLevel &gr, const float4 p, float R, int &x0, int &x1, int &y0,
                                         int &y1, int &z0, int &z1)
{
    x0 = cell_coord(__fsub_rd(p.x, R), gr.g, gr.gf);
    x1 = cell_coord(__fadd_ru(p.x, R), gr.g, gr.gf);
    y0 = cell_coord(__fsub_rd(p.y, R), gr.g, gr.gf);
    y1 = cell_coord(__fadd_ru(p.y, R), gr.g, gr.gf);
    z0 = (DIM == 3) ? cell_coord(__fsub_rd(p.z, R), gr.g, gr.gf) : 0;
    z1 = (DIM == 3) ? cell_coord(__fadd_ru(p.z, R), gr.g, gr.gf) : 0;
}

// The first box of a query: the cells meeting the ball of radius 1.15 x hint
// (it holds k+1 points), on the coarse level when the fine box has more
// than kFineRows rows; without a hint the 3^d block of Algorithm 1.  Returns
// false when the box has more than kMaxHintRows rows (the far pass).
template <int DIM>
__device__ __forceinline__ bool query_box(const KnnArgs &a, const KnnGrid &grid, const float4 p, float hint,
                                          KnnLevel &gr, int &boff, int &x0, int &x1, int &y0, int &y1, int &z0,
                                          int &z1)
{
    gr = grid.lv[0];
    boff = 0;
    if (hint > 0.0f) {
        const float R = __fmul_ru(hint, kKnnHintGrow);
        ball_box<DIM>(gr, p, R, x0, x1, y0, y1, z0, z1);
        if (grid.levels == 2 && (y1 - y0 + 1) * (z1 - z0 + 1) > kFineRows) {
            gr = grid.lv[1];
            boff = a.T;
            ball_box<DIM>(gr, p, R, x0, x1, y0, y1, z0, z1);
        }
    } else {
        const int gm = gr.g - 1;
        const int cx = cell_coord(p.x, gr.g, gr.gf);
        const int cy = cell_coord(p.y, gr.g, gr.gf);
        const int cz = (DIM == 3) ? cell_coord(p.z, gr.g, gr.gf) : 0;
        x0 = max(cx - 1, 0);
        x1 = min(cx + 1, gm);
        y0 = max(cy - 1, 0);
        y1 = min(cy + 1, gm);
        z0 = (DIM == 3) ? max(cz - 1, 0) : 0;
        z1 = (DIM == 3) ? min(cz + 1, gm) : 0;
    }
    return (y1 - y0 + 1) * (z1 - z0 + 1) <= kMaxHintRows;
}

// Distance from p to the nearest face of the box that is not on the grid
// edge (+inf when the box covers the grid).
template <int DIM>
__device__ __forceinline__ float open_face(const KnnLevel &gr, const float4 p, int x0, int x1, int y0, int y1, int z0,
                                           int z1)
{
    const int gm = gr.g - 1;
    float f0 = __int_as_float(0x7f800000);
    if (x0 > 0) f0 = fminf(f0, __fsub_rn(p.x, __fmul_rn((float)x0, gr.inv_g)));
    if (x1 < gm) f0 = fminf(f0, __fsub_rn(__fmul_rn((float)(x1 + 1), gr.inv_g), p.x));
    if (y0 > 0) f0 = fminf(f0, __fsub_rn(p.y, __fmul_rn((float)y0, gr.inv_g)));
    if (y1 < gm) f0 = fminf(f0, __fsub_rn(__fmul_rn((float)(y1 + 1), gr.inv_g), p.y));
    if (DIM == 3 && z0 > 0) f0 = fminf(f0, __fsub_rn(p.z, __fmul_rn((float)z0, gr.inv_g)));
    if (DIM == 3 && z1 < gm) f0 = fminf(f0, __fsub_rn(__fmul_rn((float)(z1 + 1), gr.inv_g), p.z));
    return f0;
}

// The enclosure test of Cor. A.2 at rank k; on success Lout is the bound on
// every point outside the S kept keys.
__device__ __forceinline__ bool enclosed(float f0, float Dk, float Dnext, float &Lout)
{
    if (isinf(f0)) {                       // the box covers the grid
        Lout = sqrt_lower(Dnext);
        return true;
    }
    const float fs = __fsub_rd(f0, kKnnFaceSlack);
    if (fs > 0.0f && Dk < __int_as_float(0x7f800000) && __fmul_ru(Dk, 1.0f + 0x1p-19f) < __fmul_rd(fs, fs)) {
        Lout = fminf(sqrt_lower(Dnext), fs);
        return true;
    }
    return false;
}

// Write a finished list (ranks 0 .. S-1) and L, with the failure audit.
template <int KB, int KH>
__device__ __forceinline__ int write_list(const KnnArgs &a, int i, const float (&hd)[KH], const int (&hj)[KH],
                                          float Lout)
{
    const int n = a.n, k = a.k, S = a.S;
    int changed = 0;
    if (a.mode == MODE_STEP) {
        int oj[KB];
#pragma unroll
        for (int r = 0; r < KB; ++r) oj[r] = (r < k) ? a.idx[(size_t)r * n + i] : -1;
        changed = set_changed<KB, KH>(oj, hj, k);
        a.failed[i] = (uint8_t)changed;
    }
#pragma unroll
    for (int r = 0; r < KH; ++r)
        if (r <= k) CERT_CHECK(a.status, (unsigned)hj[r] < (unsigned)n);   // ranks 0 .. k always hold a point
#pragma unroll
    for (int r = 0; r < KH; ++r)
        if (r < S) {
            // a spare rank the search did not fill is stored as -1 (never gathered)
            a.idx[(size_t)r * n + i] = (hj[r] != 0x7fffffff) ? hj[r] : -1;
            a.d2[(size_t)r * n + i] = hd[r];
        }
    a.L[i] = Lout;
    return changed;
}

template <int DIM, int KB>
__global__ void __launch_bounds__(kKnnThreads) k_knn_search(const KnnArgs a)
{
    constexpr int KH = KB + 2 + kExtra;        // S kept, the (S+1)-th bounds the rest
    const int total = a.ctr->need_count;
    const KnnGrid grid = *a.grid;
    const int k = a.k, S = a.S;
    int searched = 0, changed_sum = 0, missed_sum = 0;
    // A warp claims the list's next batch of 32 queries (one per lane) when its
    // previous batch is done: the queries' costs vary widely, and a fixed
    // grid-stride share would leave the warps that drew cheap ones idle while a
    // few finish long ones.
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = atomicAdd(&a.ctr->search_next, 32);
        t0 = __shfl_sync(kFull, t0, 0);
        if (t0 >= total) break;
        const int t = t0 + lane;
        if (t >= total) continue;   // the last batch's idle lanes go straight to the next claim
        const int i = a.need[t];
        const float4 p = a.pos_new[i];
        KnnLevel gr;
        int boff, x0, x1, y0, y1, z0, z1;
        if (!query_box<DIM>(a, grid, p, a.L[i], gr, boff, x0, x1, y0, y1, z0, z1)) {
            a.far[atomicAdd(&a.ctr->far_count, 1)] = i;      // a few isolated points
            continue;
        }
        const int gm = gr.g - 1;
        float hd[KH];
        int hj[KH];
        list_reset<KH>(hd, hj);
        long long budget = kHeavy;
        visit_shell<DIM, KH>(a, gr, boff, x0, x1, y0, y1, z0, z1, 1, 0, 1, 0, 1, 0, p, i, hd, hj, budget);
        float Lout = 0.0f;
        int where = 0;                             // 0: done, 1: heavy list, 2: far list
        for (int ring = 0;; ++ring) {
            if (budget < 0) {
                where = 1;
                break;
            }
            const float f0 = open_face<DIM>(gr, p, x0, x1, y0, y1, z0, z1);
            if (enclosed(f0, pick<KH>(hd, k, __int_as_float(0x7f800000)), pick<KH>(hd, S, __int_as_float(0x7f800000)),
                         Lout))
                break;
            if (ring >= kMaxRings) {
                where = 2;
                break;
            }
            const int nx0 = max(x0 - 1, 0), nx1 = min(x1 + 1, gm);
            const int ny0 = max(y0 - 1, 0), ny1 = min(y1 + 1, gm);
            const int nz0 = (DIM == 3) ? max(z0 - 1, 0) : 0, nz1 = (DIM == 3) ? min(z1 + 1, gm) : 0;
            visit_shell<DIM, KH>(a, gr, boff, nx0, nx1, ny0, ny1, nz0, nz1, x0, x1, y0, y1, z0, z1, p, i, hd, hj,
                                 budget);
            x0 = nx0;
            x1 = nx1;
            y0 = ny0;
            y1 = ny1;
            z0 = nz0;
            z1 = nz1;
        }
        if (where == 1) {                          // too many candidates for one thread
            a.heavy[atomicAdd(&a.ctr->heavy_count, 1)] = i;
            continue;
        }
        if (where == 2) {
            a.far[atomicAdd(&a.ctr->far_count, 1)] = i;
            continue;
        }
        const int changed = write_list<KB, KH>(a, i, hd, hj, Lout);
        ++searched;
        changed_sum += changed;
        if (a.mode == MODE_STEP && changed && !a.front[i]) ++missed_sum;
    }
    if (a.mode == MODE_STEP) {
        const int ns = __reduce_add_sync(kFull, searched);
        const int nc = __reduce_add_sync(kFull, changed_sum);
        const int nm = __reduce_add_sync(kFull, missed_sum);
        if ((threadIdx.x & 31) == 0) {
            if (ns) atomicAdd(&a.ctr->n_searched, ns);
            if (nc) atomicAdd(&a.ctr->n_failed, nc);
            if (nm) atomicAdd(&a.ctr->n_missed, nm);
        }
    }
}

// ---------------------------------------------------------------------------- heavy pass

// Merge the lanes' lists of one warp into lane 0's, through shared memory.
template <int KH>
__device__ __forceinline__ void warp_merge(float (&hd)[KH], int (&hj)[KH], float (*s_d)[KH], int (*s_j)[KH])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < KH; ++r) {
        s_d[lane][r] = hd[r];
        s_j[lane][r] = hj[r];
    }
    __syncwarp();
    if (lane == 0)
        for (int l = 1; l < 32; ++l)
            for (int r = 0; r < KH; ++r) {
                const float D = s_d[l][r];
                const int j = s_j[l][r];
                if (j == 0x7fffffff || !key_less(D, j, hd[KH - 1], hj[KH - 1])) break;   // lists are sorted
                list_insert<KH>(hd, hj, D, j);
            }
    __syncwarp();
}

// One warp per query whose box held more than kHeavy candidates: the same
// box and layers, each lane taking every 32nd slot of each row.
template <int DIM, int KB>
__global__ void __launch_bounds__(kKnnThreads) k_knn_heavy(const KnnArgs a)
{
    constexpr int KH = KB + 2 + kExtra;
    constexpr int W = kKnnThreads / 32;
    __shared__ float s_d[W][32][KH];
    __shared__ int s_j[W][32][KH];
    const int total = a.ctr->heavy_count;
    const KnnGrid grid = *a.grid;
    const int k = a.k, S = a.S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x * W + warp; t < total; t += gridDim.x * W) {
        const int i = a.heavy[t];
        const float4 p = a.pos_new[i];
        KnnLevel gr;
        int boff, x0, x1, y0, y1, z0, z1;
        query_box<DIM>(a, grid, p, a.L[i], gr, boff, x0, x1, y0, y1, z0, z1);   // <= kMaxHintRows rows
        const int gm = gr.g - 1;
        float hd[KH];
        int hj[KH];
        list_reset<KH>(hd, hj);
        long long budget = 1LL << 62;      // never runs out
        visit_shell<DIM, KH>(a, gr, boff, x0, x1, y0, y1, z0, z1, 1, 0, 1, 0, 1, 0, p, i, hd, hj, budget, lane, 32);
        float Lout = 0.0f;
        bool done = false;
        for (int ring = 0;; ++ring) {
            warp_merge<KH>(hd, hj, s_d[warp], s_j[warp]);
            int ok = 0;
            if (lane == 0) {
                const float f0 = open_face<DIM>(gr, p, x0, x1, y0, y1, z0, z1);
                ok = enclosed(f0, pick<KH>(hd, k, __int_as_float(0x7f800000)),
                              pick<KH>(hd, S, __int_as_float(0x7f800000)), Lout) ? 1 : 0;
            }
            ok = __shfl_sync(kFull, ok, 0);
            if (ok) {
                done = true;
                break;
            }
            if (ring >= kMaxRings) break;
            const int nx0 = max(x0 - 1, 0), nx1 = min(x1 + 1, gm);
            const int ny0 = max(y0 - 1, 0), ny1 = min(y1 + 1, gm);
            const int nz0 = (DIM == 3) ? max(z0 - 1, 0) : 0, nz1 = (DIM == 3) ? min(z1 + 1, gm) : 0;
            visit_shell<DIM, KH>(a, gr, boff, nx0, nx1, ny0, ny1, nz0, nz1, x0, x1, y0, y1, z0, z1, p, i, hd, hj,
                                 budget, lane, 32);
            x0 = nx0;
            x1 = nx1;
            y0 = ny0;
            y1 = ny1;
            z0 = nz0;
            z1 = nz1;
        }
        if (lane != 0) continue;
        if (!done) {
            a.far[atomicAdd(&a.ctr->far_count, 1)] = i;
            continue;
        }
        const int changed = write_list<KB, KH>(a, i, hd, hj, Lout);
        if (a.mode == MODE_STEP) {
            atomicAdd(&a.ctr->n_searched, 1);
            if (changed) {
                atomicAdd(&a.ctr->n_failed, 1);
                if (!a.front[i]) atomicAdd(&a.ctr->n_missed, 1);
            }
        }
    }
}

// ---------------------------------------------------------------------------- far pass

// One block per far query: each thread keeps the top-KH of a strided share of
// the points; the lists are merged per warp, then across warps, through
// shared memory.
template <int DIM, int KB>
__global__ void __launch_bounds__(kKnnThreads) k_knn_far(const KnnArgs a)
{
    constexpr int KH = KB + 2 + kExtra;
    constexpr int W = kKnnThreads / 32;
    __shared__ float s_d[kKnnThreads][KH];
    __shared__ int s_j[kKnnThreads][KH];
    const int total = a.ctr->far_count;
    const int S = a.S;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int i = a.far[t];
        const float4 p = a.pos_new[i];
        float hd[KH];
        int hj[KH];
        list_reset<KH>(hd, hj);
        visit_slots<DIM, KH>(a, threadIdx.x, a.n, kKnnThreads, p, i, hd, hj);   // level 0: every point once
#pragma unroll
        for (int r = 0; r < KH; ++r) {
            s_d[threadIdx.x][r] = hd[r];
            s_j[threadIdx.x][r] = hj[r];
        }
        __syncthreads();
        if (threadIdx.x < W) {
            list_reset<KH>(hd, hj);
            for (int l = 0; l < 32; ++l)
                for (int r = 0; r < KH; ++r) {
                    const float D = s_d[threadIdx.x * 32 + l][r];
                    const int j = s_j[threadIdx.x * 32 + l][r];
                    if (j != 0x7fffffff && key_less(D, j, hd[KH - 1], hj[KH - 1])) list_insert<KH>(hd, hj, D, j);
                }
        }
        __syncthreads();
        if (threadIdx.x < W) {
#pragma unroll
            for (int r = 0; r < KH; ++r) {
                s_d[threadIdx.x][r] = hd[r];
                s_j[threadIdx.x][r] = hj[r];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            list_reset<KH>(hd, hj);
            for (int w = 0; w < W; ++w)
                for (int r = 0; r < KH; ++r) {
                    const float D = s_d[w][r];
                    const int j = s_j[w][r];
                    if (j != 0x7fffffff && key_less(D, j, hd[KH - 1], hj[KH - 1])) list_insert<KH>(hd, hj, D, j);
                }
            // every point was visited: L is the first key beyond the list
            const int changed = write_list<KB, KH>(a, i, hd, hj, sqrt_lower(pick<KH>(hd, S, __int_as_float(0x7f800000))));
            if (a.mode == MODE_STEP) {
                atomicAdd(&a.ctr->n_searched, 1);
                if (changed) {
                    atomicAdd(&a.ctr->n_failed, 1);
                    if (!a.front[i]) atomicAdd(&a.ctr->n_missed, 1);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------- finalize

// One block of kSample threads: the step's scalars, and the next step's grid
// from the median (k+1)-th squared distance of a strided sample.
template <int DIM>
__global__ void __launch_bounds__(kSample) k_knn_finalize(const KnnArgs a)
{
    __shared__ float s_v[kSample];
    const int n = a.n, k = a.k;
    const int m = min(n, kSample);
    const int tid = threadIdx.x;
    s_v[tid] = (tid < m) ? a.d2[(size_t)k * n + (int)(((long long)tid * n) / m)] : __int_as_float(0x7f800000);
    __syncthreads();
    // bitonic sort of the sample, ascending
    for (int size = 2; size <= kSample; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int j = tid ^ stride;
            if (j > tid) {
                const bool up = (tid & size) == 0;
                const float x = s_v[tid], y = s_v[j];
                if ((x > y) == up) {
                    s_v[tid] = y;
                    s_v[j] = x;
                }
            }
            __syncthreads();
        }
    if (tid != 0) return;
    // next grid: cell side >= cell_scale x a typical (k+1)-th distance -- the
    // median, or, when the quartiles are kTwoLevelRatio apart, the lower
    // quartile for level 0 and the upper for level 1
    const float q1 = __fsqrt_ru(s_v[(m - 1) / 4]), q2 = __fsqrt_ru(s_v[(m - 1) / 2]);
    const float q3 = __fsqrt_ru(s_v[(3 * (m - 1)) / 4]);
    const bool two = q1 > 0.0f && isfinite(q3) && q3 >= __fmul_rn(kTwoLevelRatio, q1);
    const KnnGrid used = *a.grid;
    KnnGrid gr;
    gr.levels = two ? 2 : 1;
    for (int l = 0; l < 2; ++l) {
        const float side = __fmul_ru(a.cell_scale, two ? (l ? q3 : q1) : q2);
        int g = (side > 0.0f && isfinite(side)) ? (int)fminf((float)kMaxGrid, floorf(__frcp_rd(side))) : kMaxGrid;
        g = max(1, min(g, kMaxGrid));
        gr.lv[l].g = g;
        gr.lv[l].gf = (float)g;
        gr.lv[l].inv_g = __frcp_rn((float)g);
        const long long cells = (DIM == 3) ? (long long)g * g * g : (long long)g * g;
        gr.lv[l].dense = cells <= (long long)a.T ? 1 : 0;
    }
    *a.grid = gr;

    const KnnCounters c = *a.ctr;
    cert_knn_result r;
    r.eps_t = a.mode == MODE_STEP ? knn_eps(a.ctr) : 0.0f;
    r.n_frontier = c.n_frontier;
    r.n_failed = c.n_failed;
    r.n_missed = c.n_missed;
    r.n_false = c.n_frontier - (c.n_failed - c.n_missed);
    r.n_searched = a.mode == MODE_STEP ? c.n_searched : c.need_count;
    r.grid_res = used.lv[0].g;
    r.strategy = a.mode == MODE_STEP ? a.strategy : STRAT_REB;
    r.grid_res_coarse = used.levels == 2 ? used.lv[1].g : 0;
    r.n_far = c.far_count;
    *a.res = r;
    if (a.mode == MODE_STEP && r.eps_t > __fmul_ru(a.declared_eps, 1.0f + 0x1p-20f)) atomicOr(a.status, ST_EBOUND);
}

}  // namespace

// ============================================================================ host side

struct cert_knn_ctx {
    int dim = 0, k = 0, S = 0, kb = 0, T = 0;
    int64_t n = 0;
    float cell_scale = 1.0f;
    int cur = 0;                     // pos[cur] holds the current positions
    void *block = nullptr;           // one allocation for every buffer
    float4 *pos[2] = {nullptr, nullptr};
    int32_t *bucket = nullptr, *rank = nullptr, *cnt = nullptr, *start = nullptr, *part = nullptr;
    int32_t *need = nullptr, *far = nullptr, *heavy = nullptr;
    float4 *spos = nullptr;
    int32_t *idx = nullptr;
    float *d2 = nullptr, *L = nullptr;
    uint8_t *front = nullptr, *failed = nullptr;
    KnnCounters *ctr = nullptr;
    KnnGrid *grid = nullptr;
    uint32_t *status = nullptr;
    cert_knn_result *res = nullptr;
    cudaStream_t last = nullptr;
    int sms = 148;
};

static cert_status knn_fail(cert_status code, const std::string &msg)
{
    record_thread_error(msg.c_str());
    return code;
}

#define KCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return knn_fail(CERT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static KnnArgs knn_args(cert_knn_ctx *c, int mode, int strategy, float eps, const float *in)
{
    KnnArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = (int)c->n;
    a.k = c->k;
    a.S = c->S;
    a.T = c->T;
    a.mask = (uint32_t)(c->T - 1);
    a.mode = mode;
    a.strategy = strategy;
    a.declared_eps = eps;
    a.cell_scale = c->cell_scale;
    a.in = in;
    a.pos_old = c->pos[c->cur];
    a.pos_new = c->pos[c->cur ^ 1];
    a.bucket = c->bucket;
    a.rank = c->rank;
    a.cnt = c->cnt;
    a.start = c->start;
    a.part = c->part;
    a.spos = c->spos;
    a.idx = c->idx;
    a.d2 = c->d2;
    a.L = c->L;
    a.front = c->front;
    a.failed = c->failed;
    a.need = c->need;
    a.far = c->far;
    a.heavy = c->heavy;
    a.ctr = c->ctr;
    a.grid = c->grid;
    a.status = c->status;
    a.res = c->res;
    return a;
}

// Phase boundaries for cert_knn_profile: ev[0..kKnnPhases] recorded between
// the phases when non-null.
constexpr int kKnnPhases = 5;   // prepare, scan, refresh, search (+ far), finalize

template <int DIM, int KB>
static void launch_knn(const KnnArgs &a, int nblk, int sblk, int fblk, int nparts, cudaStream_t s, cudaEvent_t *ev)
{
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], s);
    };
    mark(0);
    k_knn_prepare<DIM><<<nblk, kKnnThreads, 0, s>>>(a);
    mark(1);
    k_knn_scan_reduce<<<nparts, kKnnThreads, 0, s>>>(a);
    k_knn_scan_parts<<<1, kKnnThreads, 0, s>>>(a, nparts);
    k_knn_scan_down<<<nparts, kKnnThreads, 0, s>>>(a);
    mark(2);
    k_knn_refresh<DIM, KB><<<nblk, kKnnThreads, 0, s>>>(a);
    mark(3);
    k_knn_search<DIM, KB><<<sblk, kKnnThreads, 0, s>>>(a);
    k_knn_heavy<DIM, KB><<<fblk, kKnnThreads, 0, s>>>(a);
    k_knn_far<DIM, KB><<<fblk, kKnnThreads, 0, s>>>(a);
    mark(4);
    k_knn_finalize<DIM><<<1, kSample, 0, s>>>(a);
    mark(5);
}

template <int DIM>
static void launch_knn_dim(const KnnArgs &a, int kb, int nblk, int sblk, int fblk, int nparts, cudaStream_t s,
                           cudaEvent_t *ev)
{
    switch (kb) {
    case 2: launch_knn<DIM, 2>(a, nblk, sblk, fblk, nparts, s, ev); break;
    case 4: launch_knn<DIM, 4>(a, nblk, sblk, fblk, nparts, s, ev); break;
    case 8: launch_knn<DIM, 8>(a, nblk, sblk, fblk, nparts, s, ev); break;
    default: launch_knn<DIM, 16>(a, nblk, sblk, fblk, nparts, s, ev); break;
    }
}

static cert_status knn_run(cert_knn_ctx *c, int mode, int strategy, float eps, const float *in, cudaStream_t s,
                           cudaEvent_t *ev = nullptr)
{
    KCK(cudaMemsetAsync(c->ctr, 0, sizeof(KnnCounters), s));
    const KnnArgs a = knn_args(c, mode, strategy, eps, in);
    const int nblk = (int)((c->n + kKnnThreads - 1) / kKnnThreads);
    const int sblk = std::min(nblk, c->sms * 8);
    const int fblk = c->sms * 2;
    const int nparts = (2 * c->T + kCellTile - 1) / kCellTile;
    if (c->dim == 2)
        launch_knn_dim<2>(a, c->kb, nblk, sblk, fblk, nparts, s, ev);
    else
        launch_knn_dim<3>(a, c->kb, nblk, sblk, fblk, nparts, s, ev);
    KCK(cudaGetLastError());
    c->cur ^= 1;
    c->last = s;
    return CERT_OK;
}

extern "C" {

cert_status cert_knn_init(cert_knn_ctx **out, const cert_knn_config *cfg, const float *d_pos, void *stream)
{
    if (!out) return knn_fail(CERT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || !d_pos) return knn_fail(CERT_EINVAL, "cfg or d_pos is NULL");
    if (cfg->dim != 2 && cfg->dim != 3) return knn_fail(CERT_EINVAL, "dim must be 2 or 3");
    if (cfg->k < 1 || cfg->k > CERT_KNN_MAX_K) return knn_fail(CERT_EINVAL, "k must be in 1 .. 16");
    if (cfg->n < (int64_t)cfg->k + 2 || cfg->n >= (int64_t(1) << 31))
        return knn_fail(CERT_EINVAL, "n must satisfy k + 2 <= n < 2^31");
    if (!(cfg->cell_scale >= 0.0f) || !std::isfinite(cfg->cell_scale))
        return knn_fail(CERT_EINVAL, "cell_scale must be finite and >= 0");
    if (cfg->reserved) return knn_fail(CERT_EINVAL, "reserved field must be zero");
    cudaStream_t s = (cudaStream_t)stream;

    cert_knn_ctx *c = new cert_knn_ctx();
    c->dim = cfg->dim;
    c->k = cfg->k;
    c->n = cfg->n;
    c->S = std::min<int64_t>(c->k + 1 + kExtra, c->n - 1);
    c->kb = c->k <= 2 ? 2 : c->k <= 4 ? 4 : c->k <= 8 ? 8 : 16;
    c->cell_scale = cfg->cell_scale > 0.0f ? cfg->cell_scale : 1.0f;
    c->T = 1;
    while (c->T < c->n && c->T < (1 << kMaxBucketsLog2)) c->T <<= 1;
    // the first grid: the (k+1)-th distance of a uniform set in the unit
    // domain, ((k+1) / (n V_d))^(1/d), times the scale
    const double vd = c->dim == 2 ? M_PI : 4.0 * M_PI / 3.0;
    const double h = c->cell_scale * std::pow((double)(c->k + 1) / ((double)c->n * vd), 1.0 / c->dim);
    KnnGrid g0;
    std::memset(&g0, 0, sizeof(g0));
    g0.levels = 1;
    g0.lv[0].g = (int)std::max(1.0, std::min((double)kMaxGrid, std::floor(1.0 / h)));
    g0.lv[0].gf = (float)g0.lv[0].g;
    g0.lv[0].inv_g = 1.0f / (float)g0.lv[0].g;
    const double cells = std::pow((double)g0.lv[0].g, c->dim);
    g0.lv[0].dense = cells <= (double)c->T ? 1 : 0;
    g0.lv[1] = g0.lv[0];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);

    const int64_t n = c->n, S = c->S;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t o_pos0 = take(n * sizeof(float4)), o_pos1 = take(n * sizeof(float4));
    const size_t o_bucket = take(2 * n * 4), o_rank = take(2 * n * 4), o_cnt = take(2 * size_t(c->T) * 4);
    const size_t o_start = take(size_t(2 * c->T + 1) * 4), o_part = take(size_t(kMaxParts) * 4);
    const size_t o_need = take(n * 4), o_far = take(n * 4), o_heavy = take(n * 4);
    const size_t o_spos = take(2 * n * sizeof(float4));
    const size_t o_idx = take(S * n * 4), o_d2 = take(S * n * 4), o_L = take(n * 4);
    const size_t o_front = take(n), o_failed = take(n);
    const size_t o_ctr = take(sizeof(KnnCounters)), o_grid = take(sizeof(KnnGrid)), o_status = take(4);
    const size_t o_res = take(sizeof(cert_knn_result));
    if (cudaMalloc(&c->block, off) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return knn_fail(CERT_ENOMEM, "device allocation failed");
    }
    char *b = (char *)c->block;
    c->pos[0] = (float4 *)(b + o_pos0);
    c->pos[1] = (float4 *)(b + o_pos1);
    c->bucket = (int32_t *)(b + o_bucket);
    c->rank = (int32_t *)(b + o_rank);
    c->cnt = (int32_t *)(b + o_cnt);
    c->start = (int32_t *)(b + o_start);
    c->part = (int32_t *)(b + o_part);
    c->need = (int32_t *)(b + o_need);
    c->far = (int32_t *)(b + o_far);
    c->heavy = (int32_t *)(b + o_heavy);
    c->spos = (float4 *)(b + o_spos);
    c->idx = (int32_t *)(b + o_idx);
    c->d2 = (float *)(b + o_d2);
    c->L = (float *)(b + o_L);
    c->front = (uint8_t *)(b + o_front);
    c->failed = (uint8_t *)(b + o_failed);
    c->ctr = (KnnCounters *)(b + o_ctr);
    c->grid = (KnnGrid *)(b + o_grid);
    c->status = (uint32_t *)(b + o_status);
    c->res = (cert_knn_result *)(b + o_res);
    cert_status rc = CERT_OK;
    cudaError_t e = cudaMemsetAsync(c->block, 0, off, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->grid, &g0, sizeof(KnnGrid), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);      // g0 lives on this stack frame
    if (e == cudaSuccess) rc = knn_run(c, MODE_INIT, STRAT_REB, 0.0f, d_pos, s);
    else rc = knn_fail(CERT_ECUDA, std::string("context set-up: ") + cudaGetErrorString(e));
    if (rc != CERT_OK) {
        cudaFree(c->block);
        delete c;
        return rc;
    }
    *out = c;
    return CERT_OK;
}

cert_status cert_knn_step(cert_knn_ctx *c, const float *d_pos_new, float eps, int32_t strategy, void *stream)
{
    if (!c || !d_pos_new) return knn_fail(CERT_EINVAL, "ctx or d_pos_new is NULL");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return knn_fail(CERT_EINVAL, "eps must be finite and >= 0");
    if (strategy != CERT_INCREMENTAL && strategy != CERT_REBUILD)
        return knn_fail(CERT_EINVAL, "strategy must be CERT_INCREMENTAL or CERT_REBUILD");
    return knn_run(c, MODE_STEP, strategy == CERT_INCREMENTAL ? STRAT_INC : STRAT_REB, eps, d_pos_new,
                   (cudaStream_t)stream);
}

cert_status cert_knn_profile(cert_knn_ctx *c, const float *d_pos_new, float eps, int32_t strategy, float *h_ms,
                             void *stream)
{
    if (!c || !d_pos_new || !h_ms) return knn_fail(CERT_EINVAL, "ctx, d_pos_new or h_ms is NULL");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return knn_fail(CERT_EINVAL, "eps must be finite and >= 0");
    if (strategy != CERT_INCREMENTAL && strategy != CERT_REBUILD)
        return knn_fail(CERT_EINVAL, "strategy must be CERT_INCREMENTAL or CERT_REBUILD");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[kKnnPhases + 1] = {};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k <= kKnnPhases && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    cert_status rc = CERT_OK;
    if (e == cudaSuccess) {
        rc = knn_run(c, MODE_STEP, strategy == CERT_INCREMENTAL ? STRAT_INC : STRAT_REB, eps, d_pos_new, s, ev);
        e = cudaEventSynchronize(ev[kKnnPhases]);
        for (int k = 0; k < kKnnPhases && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&h_ms[k], ev[k], ev[k + 1]);
    }
    for (int k = 0; k <= kKnnPhases; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    if (rc != CERT_OK) return rc;
    if (e != cudaSuccess) return knn_fail(CERT_ECUDA, std::string("profile events: ") + cudaGetErrorString(e));
    return CERT_OK;
}

cert_status cert_knn_get_views(const cert_knn_ctx *c, cert_knn_views *out)
{
    if (!c || !out) return knn_fail(CERT_EINVAL, "ctx or out is NULL");
    out->idx = c->idx;
    out->d2 = c->d2;
    out->frontier = c->front;
    out->failed = c->failed;
    out->result = c->res;
    out->n = c->n;
    out->k = c->k;
    out->dim = c->dim;
    return CERT_OK;
}

cert_status cert_knn_sync_result(cert_knn_ctx *c, cert_knn_result *out)
{
    if (!c) return knn_fail(CERT_EINVAL, "ctx is NULL");
    KCK(cudaStreamSynchronize(c->last));
    if (out) KCK(cudaMemcpy(out, c->res, sizeof(cert_knn_result), cudaMemcpyDeviceToHost));
    uint32_t st = 0;
    KCK(cudaMemcpy(&st, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    KCK(cudaMemset(c->status, 0, sizeof(uint32_t)));
    if (st & ST_INDEX) return knn_fail(CERT_EINTERNAL, "an internal index check failed (debug build)");
    if (st & ST_NONFINITE) return knn_fail(CERT_EINVAL, "non-finite coordinate in the positions");
    if (st & ST_EBOUND) return knn_fail(CERT_EBOUND, "measured eps_t exceeded the declared eps");
    return CERT_OK;
}

void cert_knn_destroy(cert_knn_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->last);
    cudaFree(c->block);
    delete c;
}

}  // extern "C"
