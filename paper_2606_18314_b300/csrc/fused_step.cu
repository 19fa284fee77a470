// fused_step.cu -- one launch per step: every phase of a scene in one CTA.
//
// The multi-kernel step (step_kernels.cu) runs each phase of Algorithm 1 as
// its own grid over every scene, so a step is seven dependent launches whose
// counters and histograms live in global memory.  For scenes of at most
// kFusedMaxN points this kernel runs the whole step of one scene in one CTA,
// scenes in parallel, one launch for the batch:
//
//   prepare   eps_t, the search-grid bucket and rank (counting sort), the
//             entropy-grid cell and occupancy
//   scan      bucket starts; the ascending frontier list F_t with the
//             frontier-cell histogram
//   select    medians, features, the strategy (select_scene)
//   refresh   scatter into cell order; O(1) refresh where provable
//   search    grid repair of the rest (grid_search), far queries by the CTA
//   finalize  H(F_t), the audit, the next step's grid (finalize_scene)
//
// with __syncthreads between phases.  Bucket counts, the entropy-cell
// histograms (16-bit counters, two per word), the search flags and the search
// list are in shared memory, so the per-point atomics are shared-memory
// atomics.  Positions, certificates and the sorted points stay in global
// memory (L1/L2), in the same layout as the multi-kernel step, so the two
// paths can alternate step by step.  Every result equals the multi-kernel
// step's bit for bit; only n_searched (the refresh's work split) may differ.
//
// Scenes of at most kFusedResMaxN points also keep their sorted points and
// bucket starts in shared memory, so the search walks its candidates there.
// A batch's CTAs are launched largest scene first, so the block scheduler
// hands scenes to SMs longest-first as SMs free up.
#include <algorithm>
#include <type_traits>

#include "cert_phases.cuh"

namespace certk {

// Shared-memory layout of one CTA (dynamic), in bytes, for scenes of at most
// MAXN points.  RES (MAXN <= kFusedResMaxN): the scene's sorted points (quads)
// and bucket starts are kept in shared memory too, so the search reads its
// candidates there instead of through L1/L2.
template <int NT, int MAXN>
struct FusedLayout {
    static constexpr bool RES = MAXN <= kFusedResMaxN;
    static constexpr int kMaxBuckets = MAXN;                                      // next_pow2(n) <= MAXN
    static constexpr int kRowsBytes = kFusedRows * NT * 8;                        // search row table
    static constexpr int kRegionA = kRowsBytes > (int)sizeof(SelectSmem) ? kRowsBytes : (int)sizeof(SelectSmem);
    static constexpr int kCnt = kRegionA;                                         // bucket counts, then search list
    static constexpr int kCntBytes = kMaxBuckets * 2;
    static constexpr int kHCells = (MAXN == kFusedMaxN) ? kFusedMaxHCells : 4096;  // g_h^d for n <= MAXN
    static constexpr int kHist = kCnt + kCntBytes;                                // entropy-cell counts
    static constexpr int kHistBytes = ((kHCells + 1) / 2) * 4;
    static constexpr int kFlag = (kHist + kHistBytes + 15) & ~15;                 // search flags, one bit per slot
    static constexpr int kFlagBytes = MAXN / 8;
    static constexpr int kQuads = kFlag + kFlagBytes;                             // RES: sorted points, quad layout
    static constexpr int kQuadBytes = RES ? MAXN * 16 : 0;
    static constexpr int kStart = kQuads + kQuadBytes;                            // RES: bucket starts [T + 1]
    static constexpr int kStartBytes = RES ? ((kMaxBuckets + 1) * 4 + 15) & ~15 : 0;
    static constexpr int kHcell = kStart + kStartBytes;                           // RES: entropy cell per point
    static constexpr int kHcellBytes = RES ? MAXN * 2 : 0;
    static constexpr int kMisc = kHcell + kHcellBytes;
    static constexpr int kMotion = kMisc + 2048;                                  // motion grid, its dilation
    static constexpr int kBytes = kMotion + 3 * kMotionStride * 4;
};

constexpr int kFixCache = 64;   // fixed-point k ln k entries cached in shared memory

struct FusedMisc {
    uint32_t warp[32];              // block-scan scratch
    uint32_t dmax;                  // max squared displacement (bit pattern)
    int occ, nF, frontier_cells, n_rho, strat, nsearch, nfar;
    int n_failed, n_missed, failed_cells, n_rho_hit, n_searched;
    unsigned long long s_front, s_fail;   // sums of n ln n, fixed point (tab_nlogn_fix)
    long long fix[kFixCache];       // the first entries of the fixed-point k ln k table
    double geo[8];                  // geometry audit: failed x, y, z, |p|^2; all x, y, z, |p|^2
    float fd[32][4];                // far queries: per-warp top-4 keys
    int fj[32][4];                  // ... and indices
};
static_assert(sizeof(FusedMisc) <= 2048, "misc region");

// Increment a 16-bit counter of a shared array packed two per word; returns
// the previous count (counts stay below 2^16: a scene has <= kFusedMaxN points).
__device__ __forceinline__ int smem_inc_u16(uint32_t *w, int idx)
{
    const uint32_t sh = (uint32_t)(idx & 1) << 4;
    const uint32_t old = atomicAdd(&w[idx >> 1], 1u << sh);
    return (int)((old >> sh) & 0xffffu);
}

__device__ __forceinline__ uint32_t smem_get_u16(const uint32_t *w, int idx)
{
    return (w[idx >> 1] >> ((uint32_t)(idx & 1) << 4)) & 0xffffu;
}

__device__ __forceinline__ int warp_sum_i(int v)
{
    return (int)__reduce_add_sync(kFull, (unsigned)v);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// One pass over a 16-bit histogram of `cells` cells (shared memory): the
// occupied cells and sum over cells of n_k ln n_k, added to *occupied and
// *s_fix.  The sum is in fixed point (tab_nlogn_fix), so it is exact and needs
// no FP64 arithmetic; cells holding one item add 1 ln 1 = 0, so only counts >= 2
// are looked up, the small ones in the shared copy `fix` of the first
// kFixCache entries.  Called by every thread of the block.
__device__ __forceinline__ void hist_sum(const uint32_t *hist, int cells, const double *tab,
                                         const long long *fix, int nt, int *occupied,
                                         unsigned long long *s_fix)
{
    int occ = 0;
    long long sum = 0;
    for (int w = threadIdx.x; w < (cells + 1) / 2; w += nt) {
        const uint32_t v = hist[w];
        const uint32_t c0 = v & 0xffffu, c1 = v >> 16;
        occ += (c0 != 0u) + (c1 != 0u);
        if (c0 >= 2u) sum += c0 < kFixCache ? fix[c0] : tab_nlogn_fix(tab, (int)c0);
        if (c1 >= 2u) sum += c1 < kFixCache ? fix[c1] : tab_nlogn_fix(tab, (int)c1);
    }
    occ = (int)__reduce_add_sync(kFull, (unsigned)occ);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if ((threadIdx.x & 31) == 0) {
        if (occ) atomicAdd(occupied, occ);
        if (sum) atomicAdd(s_fix, (unsigned long long)sum);
    }
}

__device__ __forceinline__ double fix_to_double(unsigned long long v)
{
    return ldexp((double)(long long)v, -kNlognFixBits);
}

template <int DIM, int NT, int MAXN>
__global__ void __launch_bounds__(NT, 1024 / NT) k_fused_step(const StepArgs a, const int32_t *order)
{
    using Lay = FusedLayout<NT, MAXN>;
    constexpr bool RES = Lay::RES;
    extern __shared__ __align__(16) unsigned char smem[];
    SelectSmem &sel = *reinterpret_cast<SelectSmem *>(smem);
    int2 *rng = reinterpret_cast<int2 *>(smem);                         // region A, search phase
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + Lay::kCnt);     // prepare, scan
    uint16_t *list = reinterpret_cast<uint16_t *>(smem + Lay::kCnt);    // search
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + Lay::kHist);
    uint32_t *flag = reinterpret_cast<uint32_t *>(smem + Lay::kFlag);
    FusedMisc &m = *reinterpret_cast<FusedMisc *>(smem + Lay::kMisc);
    float4 *s_quad = reinterpret_cast<float4 *>(smem + Lay::kQuads);    // RES
    int32_t *s_start = reinterpret_cast<int32_t *>(smem + Lay::kStart); // RES
    uint16_t *s_hcell = reinterpret_cast<uint16_t *>(smem + Lay::kHcell); // RES: entropy cell (< 4096)
    uint32_t *s_mgrid = reinterpret_cast<uint32_t *>(smem + Lay::kMotion);  // motion grid
    uint32_t *s_mdil = s_mgrid + kMotionStride;                            // ... dilated
    uint32_t *s_mtmp = s_mdil + kMotionStride;                             // ... scratch of the dilation

    const int s = order ? order[blockIdx.x] : (int)blockIdx.x;
    const SceneParams sp = a.sp[s];
    const int n = sp.n, off = sp.pt_off;
    const int T = sp.bucket_mask + 1;
    const int tid = threadIdx.x, lane = tid & 31;
    const int hcells = (DIM == 3) ? sp.g_h * sp.g_h * sp.g_h : sp.g_h * sp.g_h;
    const int g = a.st[s].g_cur;
    const float gf = (float)g;
    const bool dense = grid_is_dense<DIM>(g, T);

    // ---- zero the counters
    for (int k = tid; k < (T + 1) / 2; k += NT) cnt[k] = 0u;
    for (int k = tid; k < (hcells + 1) / 2; k += NT) hist[k] = 0u;
    for (int k = tid; k < MAXN / 32; k += NT) flag[k] = 0u;
    for (int k = tid; k < MotionRes<DIM>::cells; k += NT) s_mgrid[k] = 0u;
    for (int k = tid; k < kFixCache; k += NT) m.fix[k] = tab_nlogn_fix(a.nlogn, k);
    if (RES && tid < 16) {
        // the last quad's padding slots: NaN coordinates, index -1 (all-ones bits)
        reinterpret_cast<uint32_t *>(s_quad + (size_t)((n - 1) >> 2) * 4)[tid] = 0xffffffffu;
    }
    if (tid == 0) {
        m.dmax = 0u;
        m.occ = m.nF = m.frontier_cells = m.n_rho = m.nsearch = m.nfar = 0;
        m.n_failed = m.n_missed = m.failed_cells = m.n_rho_hit = m.n_searched = 0;
        m.s_front = m.s_fail = 0ull;
        for (int k = 0; k < 8; ++k) m.geo[k] = 0.0;
    }
    __syncthreads();

    // ---- prepare: eps_t (Algorithm 1), bucket + rank, entropy cell + occupancy (Def. 2)
    {
        uint32_t dmax = 0u;
        int occ = 0;
        const float ghf = (float)sp.g_h;
        for (int k = tid; k < n; k += NT) {
            const int i = off + k;
            const float *q = a.pos_in + (size_t)i * DIM;
            float4 p = make_float4(q[0], q[1], (DIM == 3) ? q[2] : 0.0f, 0.0f);
            const float4 po = a.pos_old[i];
            if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) atomicOr(a.status, ST_NONFINITE);
            const float D = sqdist<DIM>(po, p);
            dmax = max(dmax, (D >= 0.0f) ? __float_as_uint(D) : 0u);
            p.w = D;
            a.pos_new[i] = p;
            const int cx = cell_coord(p.x, g, gf);
            const int cy = cell_coord(p.y, g, gf);
            const int cz = (DIM == 3) ? cell_coord(p.z, g, gf) : 0;
            const int b = (int)((row_base<DIM>(cy, cz, g, dense) + (uint32_t)cx) & (uint32_t)sp.bucket_mask);
            const int rank = smem_inc_u16(cnt, b);
            if (D > 0.0f) atomicMax(&s_mgrid[motion_cell<DIM>(p)], __float_as_uint(D));
            a.brank[i] = make_int2(sp.bucket_off + b, rank);
            const int hx = cell_coord(p.x, sp.g_h, ghf);
            const int hy = cell_coord(p.y, sp.g_h, ghf);
            const int hc = (DIM == 3) ? (cell_coord(p.z, sp.g_h, ghf) * sp.g_h + hy) * sp.g_h + hx : hy * sp.g_h + hx;
            a.hcell[i] = hc;
            if (RES) s_hcell[k] = (uint16_t)hc;
            occ += smem_inc_u16(hist, hc) == 0;
        }
        dmax = __reduce_max_sync(kFull, dmax);
        occ = warp_sum_i(occ);
        if (lane == 0) {
            atomicMax(&m.dmax, dmax);
            atomicAdd(&m.occ, occ);
        }
    }
    __syncthreads();
    const float eps = __fsqrt_rn(__uint_as_float(m.dmax));

    // ---- scan (a): bucket starts, written where the search reads them
    {
        const int per = (T + NT - 1) / NT;
        const int b0 = min(T, tid * per), b1 = min(T, b0 + per);
        uint32_t sum = 0u;
        for (int b = b0; b < b1; ++b) sum += smem_get_u16(cnt, b);
        uint32_t tot;
        uint32_t run = block_exclusive_scan<NT>(sum, &tot, m.warp);
        for (int b = b0; b < b1; ++b) {
            if (RES)
                s_start[b] = off + (int)run;
            else
                a.bucket_start[sp.bucket_off + b] = off + (int)run;
            run += smem_get_u16(cnt, b);
        }
        if (RES && tid == 0) s_start[T] = off + n;
        // the refresh's local motion bound (s_mgrid serves as the second scratch)
        dilate_motion<DIM>(s_mgrid, s_mtmp, s_mgrid, s_mdil, tid, NT);
    }
    for (int k = tid; k < (hcells + 1) / 2; k += NT) hist[k] = 0u;   // occupancy done: frontier cells next
    __syncthreads();

    // ---- scan (b): the ascending frontier list (Algorithm 1, Lemma 1), the frontier-cell histogram
    {
        const int per = (n + NT - 1) / NT;   // <= 32 (n <= kFusedMaxN, NT >= 512)
        const int k0 = min(n, tid * per), k1 = min(n, k0 + per);
        uint32_t bits = 0u;
        int nf = 0, nr = 0;
        for (int k = k0; k < k1; ++k) {
            const int i = off + k;
            uint32_t r;
            const uint32_t f = frontier_item<DIM>(a, i, s, eps, &r);
            nr += (int)r;
            if (f) {
                bits |= 1u << (k - k0);
                ++nf;
                smem_inc_u16(hist, RES ? (int)s_hcell[k] : a.hcell[i]);
            }
        }
        uint32_t tot;
        uint32_t run = block_exclusive_scan<NT>((uint32_t)nf, &tot, m.warp);   // every count is in
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            a.frontier[off + (int)run++] = k0 + b;
        }
        nr = warp_sum_i(nr);
        if (lane == 0 && nr) atomicAdd(&m.n_rho, nr);
        if (tid == 0) m.nF = (int)tot;
        hist_sum(hist, hcells, a.nlogn, m.fix, NT, &m.frontier_cells, &m.s_front);
    }
    __syncthreads();
    for (int k = tid; k < (hcells + 1) / 2; k += NT) hist[k] = 0u;   // frontier cells done: failures next
    const int nF = m.nF;

    // ---- select: medians, features, strategy, next grid (one CTA per scene, as k_select);
    // its first barrier also orders the histogram's zeroing before the refresh
    {
        const int strat = select_scene<DIM, NT>(a, s, eps, nF, fix_to_double(m.s_front), m.occ, m.frontier_cells, sel);
        if (tid == 0) m.strat = strat;
    }
    __syncthreads();
    const bool inc = m.strat == STRAT_INC;

    // ---- refresh: scatter into cell order, O(1) refresh where provable
    int n_failed = 0, n_missed = 0, n_hit = 0;
    for (int k = tid; k < n; k += NT) {
        const int i = off + k;
        const int2 br = a.brank[i];
        const float4 p = a.pos_new[i];
        int slot = (RES ? s_start[br.x - sp.bucket_off] : a.bucket_start[br.x]) + br.y;
        if ((unsigned)(slot - off) >= (unsigned)n) {   // cannot happen: counts and ranks are exact here
            atomicOr(a.status, ST_INDEX);
            slot = i;
        }
        if (RES)
            sorted_store(s_quad, slot - off, p.x, p.y, p.z, i);
        else
            sorted_store(a.squad, slot - off + sp.s_off, p.x, p.y, p.z, i);
        int changed = 0;
        const bool need =
            refresh_point<DIM>(a, sp, eps, i, p, a.nn[i], a.nn2[i], a.nn3[i], a.L[i], inc, s_mdil, &changed);
        if (need) atomicOr(&flag[(slot - off) >> 5], 1u << ((slot - off) & 31));
        if (changed) {
            const uint32_t fl = a.inF[i];
            ++n_failed;
            n_missed += !(fl & 1u);
            n_hit += (int)(fl >> 1);
            smem_inc_u16(hist, RES ? (int)s_hcell[k] : a.hcell[i]);
        }
    }
    __syncthreads();

    // ---- search (a): flagged slots in ascending order (a warp's queries are neighbours)
    {
        int per = 1;
        while (per * NT < n) per <<= 1;      // a power of two <= 32: a thread's slots lie in one flag word
        const int k0 = tid * per;
        uint32_t bits = 0u;
        if (k0 < n) {
            const uint32_t w = flag[k0 >> 5];
            bits = (per == 32) ? w : ((w >> (k0 & 31)) & ((1u << per) - 1u));
        }
        uint32_t tot;
        uint32_t run = block_exclusive_scan<NT>((uint32_t)__popc(bits), &tot, m.warp);
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            list[run++] = (uint16_t)(k0 + b);
        }
        if (tid == 0) m.nsearch = (int)tot;
    }
    __syncthreads();
    const int Q = m.nsearch;

    // ---- search (b): grid repair (Algorithm 1's block loop, Cor. A.2).  When the
    // queries fit in half the block or less, G = 2 or 4 lanes share each query
    // (one round either way), which shortens the longest per-query chain.
    int cur = 0;   // scene-local index of the point being certified (RES: its cell is in s_hcell)
    auto hist_add = [&](int hc) { return smem_inc_u16(hist, RES ? (int)s_hcell[cur] : hc); };
    auto search_rounds = [&](auto gtag) {
        constexpr int G = decltype(gtag)::value;
        constexpr int NQ = NT / G;                      // queries per round
        const int gl = tid & (G - 1);           // lane within the query's group
        for (int r0 = 0; r0 < Q; r0 += NQ) {
            if (r0 + ((tid / G) & ~(32 / G - 1)) >= Q) break;    // whole idle warps leave together
            const int e = r0 + tid / G;
            if (e >= Q) continue;
            const int ls = list[e];
            int gi = RES ? sorted_index(s_quad, ls) : sorted_index(a.squad, ls + sp.s_off);
            if ((unsigned)(gi - off) >= (unsigned)n) {
                atomicOr(a.status, ST_INDEX);
                gi = off + ls;
            }
            const float4 q = a.pos_new[gi];
            SearchCtx c;
            c.squad = RES ? s_quad : a.squad;
            c.bstart = RES ? s_start : a.bucket_start;
#ifdef CERT_DEBUG_BOUNDS
            c.status = a.status;
#endif
            c.p = q;
            c.px2 = pack2(q.x, q.x);
            c.py2 = pack2(q.y, q.y);
            c.pz2 = pack2(q.z, q.z);
            c.gi = gi;
            c.pt_off = off;
            c.n = n;
            c.pad = RES ? -off : sp.s_off - off;     // sorted slot -> index in the quad array
            c.boff = RES ? 0 : sp.bucket_off;
            c.T = T;
            c.mask = (uint32_t)sp.bucket_mask;
            c.g = g;
            c.inv_g = a.st[s].inv_g;
            c.dense = dense;
            Top4 t;
            float L;
            cur = gi - off;
            const bool ok = grid_search<DIM, NQ, kFusedRows, G>(c, t, L, rng + tid / G, a.L[gi], gl);
            if (gl != 0) continue;                  // the group's lanes hold the same result
            if (ok) {
                const SearchOut o = write_certificate<false>(a, sp, gi, t, L, hist_add);
                n_failed += o.changed;
                n_missed += o.missed;
                n_hit += o.hit;
            } else {
                a.far_list[off + atomicAdd(&m.nfar, 1)] = gi;   // the scene's own segment of the far list
            }
        }
    };
    if (RES && 4 * Q <= NT)
        search_rounds(std::integral_constant<int, 4>());
    else if (RES && 2 * Q <= NT)
        search_rounds(std::integral_constant<int, 2>());
    else
        search_rounds(std::integral_constant<int, 1>());
    __syncthreads();

    // ---- search (c): far queries, each scanned by the whole CTA (every point seen: exact)
    const int nfar = m.nfar;
    for (int f = 0; f < nfar; ++f) {
        const int gi = a.far_list[off + f];
        const float4 p = a.pos_new[gi];
        const unsigned long long px = pack2(p.x, p.x), py = pack2(p.y, p.y), pz = pack2(p.z, p.z);
        Top4 t;
        top4_reset(t);
        const int qb = RES ? 0 : (sp.s_off >> 2);
        const int q1 = qb + ((n + 3) >> 2);
        for (int qd = qb + tid; qd < q1; qd += NT) {
            const float4 *r = (RES ? s_quad : a.squad) + (size_t)qd * 4;
            const float4 X = r[0], Y = r[1];
            const float4 Z = (DIM == 3) ? r[2] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 J = r[3];
            float D0, D1, D2, D3;
            sqdist_quad<DIM>(px, py, pz, X, Y, Z, D0, D1, D2, D3);
            const int j0 = __float_as_int(J.x), j1 = __float_as_int(J.y);
            const int j2 = __float_as_int(J.z), j3 = __float_as_int(J.w);
            if (D0 <= t.d3 && j0 != gi) top4_insert(t, D0, j0);
            if (D1 <= t.d3 && j1 != gi) top4_insert(t, D1, j1);
            if (D2 <= t.d3 && j2 != gi) top4_insert(t, D2, j2);
            if (D3 <= t.d3 && j3 != gi) top4_insert(t, D3, j3);
        }
        warp_merge_top4(t);
        if (lane == 0) {
            const int w = tid >> 5;
            m.fd[w][0] = t.d0; m.fd[w][1] = t.d1; m.fd[w][2] = t.d2; m.fd[w][3] = t.d3;
            m.fj[w][0] = t.j0; m.fj[w][1] = t.j1; m.fj[w][2] = t.j2; m.fj[w][3] = t.j3;
        }
        __syncthreads();
        if (tid == 0) {
            cur = gi - off;
            Top4 r;
            top4_reset(r);
            for (int w = 0; w < NT / 32; ++w)
                for (int k = 0; k < 4; ++k)
                    if (m.fj[w][k] != 0x7fffffff) top4_insert(r, m.fd[w][k], m.fj[w][k]);
            const SearchOut o = write_certificate<false>(a, sp, gi, r, sqrt_lower(r.d3), hist_add);
            n_failed += o.changed;
            n_missed += o.missed;
            n_hit += o.hit;
        }
        __syncthreads();
    }

    // ---- finalize: the step's accumulators, then H(F_t), the audit and the next grid
    if (a.audit & CERT_AUDIT_GEOMETRY) {
        double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = tid; k < n; k += NT) {
            const int i = off + k;
            const float4 p = a.pos_new[i];
            const double x = p.x, y = p.y, z = (DIM == 3) ? (double)p.z : 0.0;
            const double qq = x * x + y * y + z * z;
            v[4] += x;
            v[5] += y;
            v[6] += z;
            v[7] += qq;
            if (a.failed[i]) {
                v[0] += x;
                v[1] += y;
                v[2] += z;
                v[3] += qq;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double w = warp_sum_d(v[k]);
            if (lane == 0 && w != 0.0) atomicAdd(&m.geo[k], w);
        }
    }
    n_failed = warp_sum_i(n_failed);
    n_missed = warp_sum_i(n_missed);
    n_hit = warp_sum_i(n_hit);
    if (lane == 0 && n_failed) {
        atomicAdd(&m.n_failed, n_failed);
        atomicAdd(&m.n_missed, n_missed);
        atomicAdd(&m.n_rho_hit, n_hit);
    }
    // every failure is in the histogram (the search and far barriers above)
    hist_sum(hist, hcells, a.nlogn, m.fix, NT, &m.failed_cells, &m.s_fail);
    __syncthreads();
    if (tid == 0) {
        SceneAcc acc;
        acc.eps_bits = m.dmax;
        acc.occ = m.occ;
        acc.n_failed = m.n_failed;
        acc.n_missed = m.n_missed;
        acc.failed_cells = m.failed_cells;
        acc.frontier_cells = m.frontier_cells;
        acc.n_searched = Q;
        acc.n_rho = (a.audit & CERT_AUDIT_RHO) ? m.n_rho : 0;
        acc.n_rho_hit = (a.audit & CERT_AUDIT_RHO) ? m.n_rho_hit : 0;
        acc.pad = 0;
        acc.search_cyc = acc.refresh_cyc = 0ull;   // the cost audit runs the multi-kernel step
        acc.s_fail = fix_to_double(m.s_fail);
        acc.s_front = fix_to_double(m.s_front);
        for (int k = 0; k < 4; ++k) {
            acc.f_sum[k] = m.geo[k];
            acc.a_sum[k] = m.geo[4 + k];
        }
        a.fstart[s] = off;   // (the global accumulators stay zero: the multi-kernel step's invariant)
        finalize_scene(a, s, acc, nF, off);
    }
}

// ============================================================================ launcher

template <int DIM, int NT, int MAXN>
static cudaError_t launch_fused_dim(const StepArgs &a, const int32_t *order, cudaStream_t st)
{
    constexpr int bytes = FusedLayout<NT, MAXN>::kBytes;
    // per CTA at most 227 KB; CTAs per SM (1024 / NT) x (bytes + 1 KB reserved) within the SM's 228 KB
    static_assert(bytes <= 227 * 1024 && (1024 / NT) * (bytes + 1024) <= 228 * 1024, "fused step shared memory");
    // a host-side attribute of the function (not a stream operation): set on every launch,
    // so that each device the library launches on has it
    const cudaError_t e =
        cudaFuncSetAttribute(k_fused_step<DIM, NT, MAXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    k_fused_step<DIM, NT, MAXN><<<a.n_scenes, NT, bytes, st>>>(a, order);
    return cudaGetLastError();
}

cudaError_t launch_fused_step(const StepArgs &a, const int32_t *order, int block, bool resident, cudaStream_t st)
{
    if (resident)   // scene data resident in shared memory; 1024 threads
        return a.dim == 3 ? launch_fused_dim<3, 1024, kFusedResMaxN>(a, order, st)
                          : launch_fused_dim<2, 1024, kFusedResMaxN>(a, order, st);
    if (block == 1024)
        return a.dim == 3 ? launch_fused_dim<3, 1024, kFusedMaxN>(a, order, st)
                          : launch_fused_dim<2, 1024, kFusedMaxN>(a, order, st);
    return a.dim == 3 ? launch_fused_dim<3, 512, kFusedMaxN>(a, order, st)
                      : launch_fused_dim<2, 512, kFusedMaxN>(a, order, st);
}

}  // namespace certk
