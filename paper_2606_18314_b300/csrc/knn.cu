// knn.cu -- k-nearest-neighbour certificates (include/cert_knn.h).
//
// One scene per context.  The certificate of point i is its top-(k+1) list
// under the key (D, j) -- the k nearest and the (k+1)-th, whose gap
// c^(k)_i = d_{k+1} - d_k is the clearance -- plus L_i, a lower bound on the
// distance from i to every point outside the list.  A step (Algorithm 1, one
// rank further out):
//
//   k_knn_prepare   displacement D(p_i, p'_i) (kept in w), eps_t^2 by a max,
//                   cell of p'_i in a dense grid over [0,1]^d and its rank in
//                   the cell (the counting sort's histogram)
//   k_knn_scan_*    exclusive scan of the cell counts -> cell starts (three
//                   passes; the counts are zeroed for the next step)
//   k_knn_refresh   scatter of p'_i into cell order; the frontier test
//                   c^(k) <= 4 eps_t + tau (Lemma 1); the O(k) refresh: the k+1
//                   stored neighbours' fresh keys, sorted, are the exact
//                   top-(k+1) when the largest is below (L_i - shrink_i)^2,
//                   shrink_i >= |p'_i - p_i| + eps_t (triangle inequality);
//                   every other point joins the search list
//   k_knn_search    grid search of the list: the 3^d block of the query's cell,
//                   then whole rings, until the (k+1)-th key is below the
//                   squared distance to every face not on the grid edge
//                   (Cor. A.2); keeps k+2 keys so that L_i = the (k+2)-th
//   k_knn_finalize  the per-step scalars
//
// Lists are rank-major ([r * n + i]) so that a warp's loads of one rank are
// coalesced.  Failure of a certificate = the SET of its k nearest changed.
#include <cmath>
#include <cstring>
#include <string>

#include "cert_internal.cuh"
#include "cert_launch.h"
#include "cert_knn.h"

using namespace certk;

namespace {

constexpr int kKnnThreads = kThreads;                 // 256 (block_exclusive_scan assumes it)
constexpr int kCellTile = kThreads * 8;               // cells per scan tile
constexpr int64_t kMaxCells = int64_t(1) << 24;
constexpr int kMaxParts = int(kMaxCells / kCellTile);  // 8192 = 256 threads x 32 partials
constexpr float kKnnFaceSlack = 0x1p-17f;

struct KnnCounters {
    uint32_t eps_bits;       // max squared displacement (bit pattern of a non-negative float)
    int32_t need_count;      // entries of the search list
    int32_t n_frontier, n_failed, n_missed, n_searched;
};

struct KnnArgs {
    int n, k, g, cells;
    float gf, inv_g;
    int mode, strategy;      // MODE_INIT / MODE_STEP / MODE_REBUILD; STRAT_INC / STRAT_REB
    float declared_eps;
    const float *in;         // caller's positions [n][dim]
    const float4 *pos_old;   // previous positions (w unused)
    float4 *pos_new;         // this step's positions, w = squared displacement
    int32_t *key, *rank;     // per point: cell, rank inside the cell
    int32_t *cnt;            // [cells] counts (zero between steps)
    int32_t *start;          // [cells + 1] cell starts
    int32_t *part;           // [kMaxParts] per-tile sums
    float4 *spos;            // points in cell order: x, y, z, index bits
    int32_t *idx;            // [k+1][n]
    float *d2;               // [k+1][n]
    float *L;                // [n]
    uint8_t *front, *failed;
    int32_t *need;           // search list
    KnnCounters *ctr;
    uint32_t *status;
    cert_knn_result *res;
};

__device__ __forceinline__ float knn_eps(const KnnCounters *c)
{
    return __fsqrt_rn(__uint_as_float(c->eps_bits));
}

template <int DIM>
__device__ __forceinline__ int knn_cell(const KnnArgs &a, float4 p)
{
    const int x = cell_coord(p.x, a.g, a.gf);
    const int y = cell_coord(p.y, a.g, a.gf);
    if (DIM == 2) return y * a.g + x;
    const int z = cell_coord(p.z, a.g, a.gf);
    return (z * a.g + y) * a.g + x;
}

// Insert (D, j) into the sorted list (d, j) of KH keys, dropping the last; the
// caller has checked that (D, j) is below the last key.
template <int KH>
__device__ __forceinline__ void list_insert(float (&d)[KH], int (&jj)[KH], float D, int J)
{
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

// d[r] for a runtime r < KH without local memory.
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
        const int c = knn_cell<DIM>(a, p);
        a.key[i] = c;
        a.rank[i] = atomicAdd(&a.cnt[c], 1);
    }
    if (a.mode == MODE_STEP) {
        // non-negative floats order as their bit patterns
        const uint32_t m = __reduce_max_sync(kFull, dbits);
        if ((threadIdx.x & 31) == 0 && m) atomicMax(&a.ctr->eps_bits, m);
    }
}

// ---------------------------------------------------------------------------- scan of the cell counts

__global__ void __launch_bounds__(kKnnThreads) k_knn_scan_reduce(const KnnArgs a)
{
    __shared__ uint32_t s_warp[kKnnThreads / 32];
    const int base = blockIdx.x * kCellTile + threadIdx.x * 8;
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (base + k < a.cells) sum += (uint32_t)a.cnt[base + k];
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
        v[k] = (base + k < a.cells) ? (uint32_t)a.cnt[base + k] : 0u;
        sum += v[k];
    }
    uint32_t tot;
    uint32_t run = (uint32_t)a.part[blockIdx.x] + block_exclusive_scan(sum, &tot, s_warp);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (base + k < a.cells) {
            a.start[base + k] = (int32_t)run;
            a.cnt[base + k] = 0;              // ready for the next step's histogram
        }
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.start[a.cells] = a.n;
}

// ---------------------------------------------------------------------------- refresh

__device__ __forceinline__ void append_need(const KnnArgs &a, bool need, int i)
{
    const unsigned m = __ballot_sync(kFull, need);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&a.ctr->need_count, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (need) a.need[base + __popc(m & ((1u << lane) - 1u))] = i;
}

template <int DIM, int KB>
__global__ void __launch_bounds__(kKnnThreads) k_knn_refresh(const KnnArgs a)
{
    constexpr int KS = KB + 1;                 // stored keys, compile-time bound
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.n;
    bool need = false;
    int inF = 0, changed = 0, missed = 0;
    if (valid) {
        const float4 p = a.pos_new[i];
        a.spos[a.start[a.key[i]] + a.rank[i]] = make_float4(p.x, p.y, p.z, __int_as_float(i));
        if (a.mode != MODE_STEP) {
            need = true;
        } else {
            const int n = a.n, k = a.k, K1 = k + 1;
            const float eps = knn_eps(a.ctr);
            // frontier from the pre-step certificate (Lemma 1 at rank k)
            const float dk = __fsqrt_rn(a.d2[(size_t)(k - 1) * n + i]);
            const float dk1 = __fsqrt_rn(a.d2[(size_t)k * n + i]);
            const float c = __fsub_rn(dk1, dk);
            const float tau = __fmul_rn(0x1p-20f, __fadd_rn(__fadd_rn(dk, dk1), eps));
            inF = (c <= __fadd_rn(__fmul_rn(4.0f, eps), tau)) ? 1 : 0;
            a.front[i] = (uint8_t)inF;
            if (a.strategy == STRAT_REB) {
                need = true;
            } else {
                float hd[KS];
                int hj[KS];
                int old_last = -1;
#pragma unroll
                for (int r = 0; r < KS; ++r) {
                    hd[r] = __int_as_float(0x7f800000);
                    hj[r] = 0x7fffffff;
                }
#pragma unroll
                for (int r = 0; r < KS; ++r) {
                    if (r < K1) {
                        const int j = a.idx[(size_t)r * n + i];
                        if (r == k) old_last = j;
                        const float D = sqdist<DIM>(p, a.pos_new[j]);
                        if (key_less(D, j, hd[KS - 1], hj[KS - 1])) list_insert<KS>(hd, hj, D, j);
                    }
                }
                // every point outside the stored list was at least L away and
                // both ends moved: now at least L - (|p'_i - p_i| + eps_t)
                const float shrink = __fmul_ru(__fadd_ru(__fsqrt_ru(p.w), eps), 1.0f + 0x1p-18f);
                const float Lnew = __fsub_rd(a.L[i], shrink);
                const float Dlast = pick<KS>(hd, k, 0.0f);
                if (Lnew > 0.0f && __fmul_ru(Dlast, 1.0f + 0x1p-19f) < __fmul_rd(Lnew, Lnew)) {
#pragma unroll
                    for (int r = 0; r < KS; ++r)
                        if (r < K1) {
                            a.idx[(size_t)r * n + i] = hj[r];
                            a.d2[(size_t)r * n + i] = hd[r];
                            if (r < k && hj[r] == old_last) changed = 1;   // the (k+1)-th moved in
                        }
                    a.L[i] = Lnew;
                    a.failed[i] = (uint8_t)changed;
                    missed = changed && !inF;
                } else {
                    need = true;
                }
            }
        }
    }
    append_need(a, valid && need, i);
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
__device__ __forceinline__ void visit_cells(const KnnArgs &a, int row, int xl, int xh, const float4 p, int self,
                                            float (&hd)[KH], int (&hj)[KH])
{
    const int lo = a.start[row + xl];
    const int hi = a.start[row + xh + 1];
    for (int s = lo; s < hi; ++s) {
        const float4 q = a.spos[s];
        const int j = __float_as_int(q.w);
        const float D = sqdist<DIM>(p, q);
        if (j != self && key_less(D, j, hd[KH - 1], hj[KH - 1])) list_insert<KH>(hd, hj, D, j);
    }
}

template <int DIM, int KB>
__global__ void __launch_bounds__(kKnnThreads) k_knn_search(const KnnArgs a)
{
    constexpr int KH = KB + 2;                 // k+1 kept, the (k+2)-th bounds the rest
    const int total = a.ctr->need_count;
    const int n = a.n, k = a.k, K1 = k + 1, g = a.g, gm = a.g - 1;
    int searched = 0, changed_sum = 0, missed_sum = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int i = a.need[t];
        const float4 p = a.pos_new[i];
        const int cx = cell_coord(p.x, g, a.gf);
        const int cy = cell_coord(p.y, g, a.gf);
        const int cz = (DIM == 3) ? cell_coord(p.z, g, a.gf) : 0;
        float hd[KH];
        int hj[KH];
#pragma unroll
        for (int r = 0; r < KH; ++r) {
            hd[r] = __int_as_float(0x7f800000);
            hj[r] = 0x7fffffff;
        }
        const float inf = __int_as_float(0x7f800000);
        float Lout = 0.0f;
        for (int r = 1;; ++r) {
            // box of ring r, clamped; the previous box is that of ring r-1
            const int x0 = max(cx - r, 0), x1 = min(cx + r, gm);
            const int y0 = max(cy - r, 0), y1 = min(cy + r, gm);
            const int z0 = (DIM == 3) ? max(cz - r, 0) : 0, z1 = (DIM == 3) ? min(cz + r, gm) : 0;
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y) {
                    const int row = (DIM == 3) ? (z * g + y) * g : y * g;
                    const bool inner = r > 1 && abs(y - cy) < r && (DIM == 2 || abs(z - cz) < r);
                    if (!inner) {
                        visit_cells<DIM, KH>(a, row, x0, x1, p, i, hd, hj);
                    } else {
                        // the row was visited up to ring r-1: only its two new cells
                        if (cx - r >= 0) visit_cells<DIM, KH>(a, row, cx - r, cx - r, p, i, hd, hj);
                        if (cx + r <= gm) visit_cells<DIM, KH>(a, row, cx + r, cx + r, p, i, hd, hj);
                    }
                }
            // distance to the nearest face that is not on the grid edge
            float f0 = inf;
            if (x0 > 0) f0 = fminf(f0, __fsub_rn(p.x, __fmul_rn((float)x0, a.inv_g)));
            if (x1 < gm) f0 = fminf(f0, __fsub_rn(__fmul_rn((float)(x1 + 1), a.inv_g), p.x));
            if (y0 > 0) f0 = fminf(f0, __fsub_rn(p.y, __fmul_rn((float)y0, a.inv_g)));
            if (y1 < gm) f0 = fminf(f0, __fsub_rn(__fmul_rn((float)(y1 + 1), a.inv_g), p.y));
            if (DIM == 3 && z0 > 0) f0 = fminf(f0, __fsub_rn(p.z, __fmul_rn((float)z0, a.inv_g)));
            if (DIM == 3 && z1 < gm) f0 = fminf(f0, __fsub_rn(__fmul_rn((float)(z1 + 1), a.inv_g), p.z));
            const float Dk1 = pick<KH>(hd, k + 1, inf);
            if (isinf(f0)) {                       // the box covers the grid
                Lout = sqrt_lower(Dk1);
                break;
            }
            const float fs = __fsub_rd(f0, kKnnFaceSlack);
            const float Dk = pick<KH>(hd, k, inf);
            if (fs > 0.0f && Dk < inf && __fmul_ru(Dk, 1.0f + 0x1p-19f) < __fmul_rd(fs, fs)) {
                Lout = fminf(sqrt_lower(Dk1), fs);
                break;
            }
        }
        int changed = 0;
        if (a.mode == MODE_STEP) {
            // the set of the k nearest changed iff a new one is not among the old
            int oj[KB];
#pragma unroll
            for (int r = 0; r < KB; ++r) oj[r] = (r < k) ? a.idx[(size_t)r * n + i] : -1;
#pragma unroll
            for (int s = 0; s < KB; ++s) {
                if (s < k) {
                    bool found = false;
#pragma unroll
                    for (int r = 0; r < KB; ++r) found |= oj[r] == hj[s];
                    changed |= !found;
                }
            }
            a.failed[i] = (uint8_t)changed;
        }
#pragma unroll
        for (int r = 0; r < KH; ++r)
            if (r < K1) {
                a.idx[(size_t)r * n + i] = hj[r];
                a.d2[(size_t)r * n + i] = hd[r];
            }
        a.L[i] = Lout;
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

// ---------------------------------------------------------------------------- finalize

__global__ void k_knn_finalize(const KnnArgs a)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const KnnCounters c = *a.ctr;
    cert_knn_result r;
    r.eps_t = a.mode == MODE_STEP ? knn_eps(a.ctr) : 0.0f;
    r.n_frontier = c.n_frontier;
    r.n_failed = c.n_failed;
    r.n_missed = c.n_missed;
    r.n_false = c.n_frontier - (c.n_failed - c.n_missed);
    r.n_searched = a.mode == MODE_STEP ? c.n_searched : c.need_count;
    r.grid_res = a.g;
    r.strategy = a.mode == MODE_STEP ? a.strategy : STRAT_REB;
    *a.res = r;
    if (a.mode == MODE_STEP && r.eps_t > __fmul_ru(a.declared_eps, 1.0f + 0x1p-20f)) atomicOr(a.status, ST_EBOUND);
}

}  // namespace

// ============================================================================ host side

struct cert_knn_ctx {
    int dim = 0, k = 0, g = 0, cells = 0, kb = 0;
    int64_t n = 0;
    int cur = 0;                     // pos[cur] holds the current positions
    void *block = nullptr;           // one allocation for every buffer
    float4 *pos[2] = {nullptr, nullptr};
    int32_t *key = nullptr, *rank = nullptr, *cnt = nullptr, *start = nullptr, *part = nullptr, *need = nullptr;
    float4 *spos = nullptr;
    int32_t *idx = nullptr;
    float *d2 = nullptr, *L = nullptr;
    uint8_t *front = nullptr, *failed = nullptr;
    KnnCounters *ctr = nullptr;
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
    a.g = c->g;
    a.cells = c->cells;
    a.gf = (float)c->g;
    a.inv_g = 1.0f / (float)c->g;
    a.mode = mode;
    a.strategy = strategy;
    a.declared_eps = eps;
    a.in = in;
    a.pos_old = c->pos[c->cur];
    a.pos_new = c->pos[c->cur ^ 1];
    a.key = c->key;
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
    a.ctr = c->ctr;
    a.status = c->status;
    a.res = c->res;
    return a;
}

template <int DIM, int KB>
static void launch_knn(const KnnArgs &a, int nblk, int sblk, int nparts, cudaStream_t s)
{
    k_knn_prepare<DIM><<<nblk, kKnnThreads, 0, s>>>(a);
    k_knn_scan_reduce<<<nparts, kKnnThreads, 0, s>>>(a);
    k_knn_scan_parts<<<1, kKnnThreads, 0, s>>>(a, nparts);
    k_knn_scan_down<<<nparts, kKnnThreads, 0, s>>>(a);
    k_knn_refresh<DIM, KB><<<nblk, kKnnThreads, 0, s>>>(a);
    k_knn_search<DIM, KB><<<sblk, kKnnThreads, 0, s>>>(a);
    k_knn_finalize<<<1, 32, 0, s>>>(a);
}

template <int DIM>
static void launch_knn_dim(const KnnArgs &a, int kb, int nblk, int sblk, int nparts, cudaStream_t s)
{
    switch (kb) {
    case 2: launch_knn<DIM, 2>(a, nblk, sblk, nparts, s); break;
    case 4: launch_knn<DIM, 4>(a, nblk, sblk, nparts, s); break;
    case 8: launch_knn<DIM, 8>(a, nblk, sblk, nparts, s); break;
    default: launch_knn<DIM, 16>(a, nblk, sblk, nparts, s); break;
    }
}

static cert_status knn_run(cert_knn_ctx *c, int mode, int strategy, float eps, const float *in, cudaStream_t s)
{
    KCK(cudaMemsetAsync(c->ctr, 0, sizeof(KnnCounters), s));
    const KnnArgs a = knn_args(c, mode, strategy, eps, in);
    const int nblk = (int)((c->n + kKnnThreads - 1) / kKnnThreads);
    const int sblk = std::min(nblk, c->sms * 8);
    const int nparts = (c->cells + kCellTile - 1) / kCellTile;
    if (c->dim == 2)
        launch_knn_dim<2>(a, c->kb, nblk, sblk, nparts, s);
    else
        launch_knn_dim<3>(a, c->kb, nblk, sblk, nparts, s);
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
    c->kb = c->k <= 2 ? 2 : c->k <= 4 ? 4 : c->k <= 8 ? 8 : 16;
    // cell side = scale * ((k+1)/n)^(1/d): about scale^d (k+1) points per cell in a uniform set
    const double scale = cfg->cell_scale > 0.0f ? cfg->cell_scale : 1.0;
    const double h = scale * std::pow((double)(c->k + 1) / (double)c->n, 1.0 / c->dim);
    const int gmax = c->dim == 2 ? 4096 : 256;           // g^d <= 2^24
    c->g = (int)std::max(1.0, std::min((double)gmax, std::floor(1.0 / h)));
    c->cells = c->dim == 2 ? c->g * c->g : c->g * c->g * c->g;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);

    const int64_t n = c->n, K1 = c->k + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t o_pos0 = take(n * sizeof(float4)), o_pos1 = take(n * sizeof(float4));
    const size_t o_key = take(n * 4), o_rank = take(n * 4), o_cnt = take(size_t(c->cells) * 4);
    const size_t o_start = take(size_t(c->cells + 1) * 4), o_part = take(size_t(kMaxParts) * 4);
    const size_t o_need = take(n * 4), o_spos = take(n * sizeof(float4));
    const size_t o_idx = take(K1 * n * 4), o_d2 = take(K1 * n * 4), o_L = take(n * 4);
    const size_t o_front = take(n), o_failed = take(n);
    const size_t o_ctr = take(sizeof(KnnCounters)), o_status = take(4), o_res = take(sizeof(cert_knn_result));
    if (cudaMalloc(&c->block, off) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return knn_fail(CERT_ENOMEM, "device allocation failed");
    }
    char *b = (char *)c->block;
    c->pos[0] = (float4 *)(b + o_pos0);
    c->pos[1] = (float4 *)(b + o_pos1);
    c->key = (int32_t *)(b + o_key);
    c->rank = (int32_t *)(b + o_rank);
    c->cnt = (int32_t *)(b + o_cnt);
    c->start = (int32_t *)(b + o_start);
    c->part = (int32_t *)(b + o_part);
    c->need = (int32_t *)(b + o_need);
    c->spos = (float4 *)(b + o_spos);
    c->idx = (int32_t *)(b + o_idx);
    c->d2 = (float *)(b + o_d2);
    c->L = (float *)(b + o_L);
    c->front = (uint8_t *)(b + o_front);
    c->failed = (uint8_t *)(b + o_failed);
    c->ctr = (KnnCounters *)(b + o_ctr);
    c->status = (uint32_t *)(b + o_status);
    c->res = (cert_knn_result *)(b + o_res);
    cert_status rc = CERT_OK;
    cudaError_t e = cudaMemsetAsync(c->block, 0, off, s);
    if (e == cudaSuccess) rc = knn_run(c, MODE_INIT, STRAT_REB, 0.0f, d_pos, s);
    else rc = knn_fail(CERT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
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
