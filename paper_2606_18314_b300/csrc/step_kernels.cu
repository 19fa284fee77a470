// step_kernels.cu -- the per-step kernels of the certificate-maintenance loop.
//
// One step (Algorithm 1 of the paper, every certificate exact afterwards as in
// Cor. A.2) runs as seven kernels over all scenes of a batch at once, after a
// clear of the per-step counters:
//
//   k_prepare          pack p' to float4, eps_t max-reduce (Alg. 1 first
//                      statement), search-grid bucket + rank (counting sort,
//                      histogram phase), entropy-grid cell + occupancy (Def. 2),
//                      the per-scene motion grid (largest step per coarse cell)
//   k_scan             decoupled look-back scans: bucket starts (counting sort,
//                      scan phase) and the ascending frontier list
//                      F = {i : c_i <= 4 eps_t + tau_i} (Alg. 1 second
//                      statement, Lemma 1) with the frontier-cell histogram
//   k_select           per scene: truncated medians, next search resolution,
//                      the strategy (forced, per-scene policy, Prop. 1's
//                      threshold or the learned selector), the motion grid's
//                      dilation
//   k_scatter_refresh  counting-sort scatter into cell order; O(1) refresh of
//                      every certificate that its extended certificate still
//                      proves (frontier points included)
//   k_search           grid repair of the flagged points: top-2 over a box of
//                      cells sized from the refresh's hint (else the 3^d block),
//                      widened until the runner-up is enclosed (Alg. 1 block
//                      loop; Cor. A.2 widening)
//   k_far              the queries whose box would grow too far: one CTA scans
//                      the whole scene
//   k_finalize         per scene: H(F_t) (Def. 2), audit counts, next grid
//
// Extended certificate (an addition to the paper's record, needed because the
// paper leaves d1, d2 of safe points stale while every certificate here is
// exact each step): besides (nn, d1^2, d2^2) each point keeps its runner-up
// index nn2, a third candidate nn3 and a lower bound L on the distance to
// every point other than the three.  A step changes the distance from i to
// any j by at most |p'_i - p_i| + |p'_j - p_j| (triangle inequality, as in
// Lemma 1), so L minus a bound on that bounds the next step (refresh_point,
// cert_phases.cuh: eps_t, else the local motion grid); when the second of the
// three fresh keys stays below it, the first two keys are the exact top-2,
// otherwise the point is repaired by a search.  The test is independent of the
// safety rule, so a frontier point it proves is repaired in O(1) too (a change
// of nn is then found by the reordering of the candidates).
#include <algorithm>

#include "cert_phases.cuh"

namespace certk {

// ============================================================================ k_prepare

// PER points per thread (strided by kThreads, so a warp's lanes still hold
// consecutive points): the loads, atomics and stores of the points are issued
// together, overlapping their latencies.  kPrepPer for grids that fill the GPU;
// a small grid takes fewer per thread and more CTAs (chosen at the launch).
constexpr int kPrepPer = 4;
constexpr int kSmallGridPrepare = 5 * 148;   // one wave of k_prepare (48 registers)

__device__ void order_chunks(const StepArgs &a, int nch, int *s_hist, int *s_start);

template <int DIM, int PER>
__global__ void __launch_bounds__(kThreads, 5) k_prepare(const StepArgs a)   // 48 registers: 5 CTAs per SM
{
    if (a.order_chunks > 0 && blockIdx.x == 0) {   // uniform in the CTA
        __shared__ int s_hist[32], s_start[32];
        order_chunks(a, a.order_chunks, s_hist, s_start);
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) {   // the scans' tickets and the far list start empty
        a.tile_ctr[threadIdx.x] = 0u;
        a.far_count[threadIdx.x] = 0;
    }
    const int base = blockIdx.x * (kThreads * PER) + threadIdx.x;
    int s[PER];
    float4 p[PER], po[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        s[k] = -1;
        p[k] = po[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < a.n_total) {
            s[k] = scene_of_point(a.scene_of, a.n_scenes, i);
            if (a.mode == MODE_REBUILD) {
                p[k] = a.pos_new[i];
            } else {
                const float *q = a.pos_in + (size_t)i * DIM;
                p[k].x = q[0];
                p[k].y = q[1];
                p[k].z = (DIM == 3) ? q[2] : 0.0f;
                if (a.mode == MODE_STEP) po[k] = a.pos_old[i];
            }
        }
    }
    unsigned dbits[PER];
    int first[PER], rank[PER], b[PER], hc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        dbits[k] = 0u;
        first[k] = 0;
        if (s[k] < 0) continue;
        if (a.mode != MODE_REBUILD) {
            if (!(isfinite(p[k].x) && isfinite(p[k].y) && isfinite(p[k].z))) atomicOr(a.status, ST_NONFINITE);
            if (a.mode == MODE_STEP) {
                // squared displacement of this point; kept in w for the refresh
                const float D = sqdist<DIM>(po[k], p[k]);
                dbits[k] = (D >= 0.0f) ? __float_as_uint(D) : 0u;
                p[k].w = D;
            }
            a.pos_new[i] = p[k];
        }
        const SceneParams sp = a.sp[s[k]];
        // hashed search grid: bucket of the cell, rank inside the bucket
        const int g = a.st[s[k]].g_cur;
        const float gf = (float)g;
        const int cx = cell_coord(p[k].x, g, gf);
        const int cy = cell_coord(p[k].y, g, gf);
        const int cz = (DIM == 3) ? cell_coord(p[k].z, g, gf) : 0;
        const bool dense = grid_is_dense<DIM>(g, sp.bucket_mask + 1);
        b[k] = sp.bucket_off + (int)((row_base<DIM>(cy, cz, g, dense) + (uint32_t)cx) & (uint32_t)sp.bucket_mask);
        rank[k] = count_inc(a.bucket_count, b[k], a.c16b);
        // the motion grid of the refresh's local bound (static points add nothing)
        // (read first: cells of dense scenes take hundreds of points, and their
        // maximum is reached early, so most of the atomics would serialise for nothing)
        if (dbits[k]) {
            uint32_t *mc = &a.mgrid[s[k] * kMotionStride + motion_cell<DIM>(p[k])];
            if (dbits[k] > __ldcg(mc)) atomicMax(mc, dbits[k]);
        }
        // entropy grid on the post-step position (Def. 2)
        if (a.mode != MODE_REBUILD) {
            const int gh = sp.g_h;
            const float ghf = (float)gh;
            const int hx = cell_coord(p[k].x, gh, ghf);
            const int hy = cell_coord(p[k].y, gh, ghf);
            hc[k] = (DIM == 3) ? (cell_coord(p[k].z, gh, ghf) * gh + hy) * gh + hx : hy * gh + hx;
            const int hg = sp.h_off + hc[k];   // the first point to mark the cell counts it
            const uint32_t bit = 1u << (hg & 31);
            first[k] = (atomicOr(&a.hocc[hg >> 5], bit) & bit) == 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        if (s[k] >= 0) {
            a.brank[i] = make_int2(b[k], rank[k]);
            if (a.mode != MODE_REBUILD) a.hcell[i] = hc[k];
        }
        const unsigned m = scene_run_mask(s[k]);
        const unsigned mx = run_max_u32(m, dbits[k]);
        const int occ = run_sum_i32(m, first[k]);
        if (s[k] >= 0 && run_leader(m)) {
            if (mx) atomicMax(&a.acc[s[k]].eps_bits, mx);
            if (occ) atomicAdd(&a.acc[s[k]].occ, occ);
        }
    }
}

// ============================================================================ k_scan

// Publish this tile's aggregate and look back over predecessors for the
// exclusive prefix (single-pass chained scan).  Called by warp 0 only.  A
// status word is (flag << 32) | value with flag 1 = the tile's aggregate,
// 2 = its inclusive prefix, 0 = not yet published; the word is all a reader
// needs, so relaxed accesses suffice (acquire / release cost 6 us a step).
// Every wait is bounded; on expiry the status word records a timeout and the
// (incorrect) partial prefix is used so that the kernel still terminates.
__device__ uint32_t lookback(uint64_t *tstat, int tile, uint32_t aggregate, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed_u64(&tstat[0], (2ull << 32) | aggregate);
        return 0u;
    }
    if (lane == 0) st_relaxed_u64(&tstat[tile], (1ull << 32) | aggregate);
    uint32_t excl = 0u;
    int p = tile - 1;
    uint32_t spins = 0u;
    for (;;) {
        const int idx = p - lane;
        const uint64_t v = (idx >= 0) ? ld_relaxed_u64(&tstat[idx]) : (2ull << 32);   // before tile 0: prefix 0
        const uint32_t flag = (uint32_t)(v >> 32);
        const unsigned incl = __ballot_sync(kFull, flag == 2u);
        const unsigned notready = __ballot_sync(kFull, flag == 0u);
        const int fi = incl ? (__ffs(incl) - 1) : 32;
        const unsigned relevant = (fi >= 31) ? kFull : ((2u << fi) - 1u);
        if (notready & relevant) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                break;
            }
            continue;
        }
        uint32_t val = (lane <= fi) ? (uint32_t)v : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
        excl += val;
        if (fi < 32) break;
        p -= 32;
    }
    if (lane == 0) st_relaxed_u64(&tstat[tile], (2ull << 32) | (excl + aggregate));
    return excl;
}

// LAT selects the issue order for grids smaller than one wave (a small scene,
// where a tile's per-thread chain of dependent accesses is the kernel's
// time): the frontier items' entropy cells are loaded with the flags and their
// atomics issued back to back.  The default order keeps 48 registers, five
// resident CTAs per SM, for the many-tile grids that are bound by resident CTAs.
template <int DIM, bool LAT, int ITEMS>
__global__ void __launch_bounds__(kThreads) k_scan(const StepArgs a)
{
    constexpr int TILE = kThreads * ITEMS;
    static_assert(ITEMS <= 2 || ITEMS % 8 == 0, "bucket counts load one, two, or four / eight (c16) at a time");
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_tile;
    __shared__ uint32_t s_excl;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    // Point tiles take the first tickets: they are the longer ones (the
    // frontier test and the cell atomics), so they start early and the short
    // bucket tiles fill in at the end.  Each chain still takes its tiles in order.
    const int t = s_tile;

    if (t >= a.ntiles_p) {
        // ---- bucket counts -> bucket starts (global exclusive scan over all scenes)
        const int tb = t - a.ntiles_p;
        const int base = tb * TILE + threadIdx.x * ITEMS;
        uint32_t v[ITEMS];
        if constexpr (ITEMS == 1) {
            v[0] = a.c16b ? (uint32_t)reinterpret_cast<const uint16_t *>(a.bucket_count)[base]
                          : (uint32_t)a.bucket_count[base];
        } else if (a.c16b) {   // 16-bit counts: ITEMS of them in ITEMS / 2 words
            const uint16_t *c16 = reinterpret_cast<const uint16_t *>(a.bucket_count) + base;
            if constexpr (ITEMS == 2) {
                const uint32_t w = *reinterpret_cast<const uint32_t *>(c16);
                v[0] = w & 0xffffu;
                v[ITEMS > 1 ? 1 : 0] = w >> 16;
            } else {
#pragma unroll
                for (int k = 0; k < ITEMS; k += 8) {
                    const uint4 w = *reinterpret_cast<const uint4 *>(c16 + k);
                    v[k] = w.x & 0xffffu;
                    v[k + 1] = w.x >> 16;
                    v[k + 2] = w.y & 0xffffu;
                    v[k + 3] = w.y >> 16;
                    v[k + 4] = w.z & 0xffffu;
                    v[k + 5] = w.z >> 16;
                    v[k + 6] = w.w & 0xffffu;
                    v[k + 7] = w.w >> 16;
                }
            }
        } else if constexpr (ITEMS == 2) {
            const int2 c2 = *reinterpret_cast<const int2 *>(a.bucket_count + base);
            v[0] = (uint32_t)c2.x;
            v[ITEMS > 1 ? 1 : 0] = (uint32_t)c2.y;
        } else {
#pragma unroll
            for (int k = 0; k < ITEMS; k += 4) {
                const int4 c4 = *reinterpret_cast<const int4 *>(a.bucket_count + base + k);
                v[k] = (uint32_t)c4.x;
                v[k + 1] = (uint32_t)c4.y;
                v[k + 2] = (uint32_t)c4.z;
                v[k + 3] = (uint32_t)c4.w;
            }
        }
        uint32_t sum = 0u;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) sum += v[k];
        uint32_t tot;
        const uint32_t pre = block_exclusive_scan(sum, &tot, s_warp);
        if (threadIdx.x < 32) {
            const uint32_t ex = lookback(a.tstat_b, tb, tot, a.status);
            if (threadIdx.x == 0) s_excl = ex;
        }
        __syncthreads();
        uint32_t run = s_excl + pre;
        int o[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            o[k] = (int)run;
            run += v[k];
        }
        if constexpr (ITEMS == 1) {
            a.bucket_start[base] = o[0];
        } else if constexpr (ITEMS == 2) {
            *reinterpret_cast<int2 *>(a.bucket_start + base) = make_int2(o[0], o[ITEMS > 1 ? 1 : 0]);
        } else {
#pragma unroll
            for (int k = 0; k < ITEMS; k += 4)
                *reinterpret_cast<int4 *>(a.bucket_start + base + k) = make_int4(o[k], o[k + 1], o[k + 2], o[k + 3]);
        }
        return;
    }

    // ---- frontier flags -> ascending frontier list (Algorithm 1, Lemma 1)
    const int tp = t;
    const int base = tp * TILE + threadIdx.x * ITEMS;
    uint32_t f[ITEMS];
    uint32_t rho = 0u;                 // bit k: item k flagged by the rho heuristic
    static_assert(ITEMS <= 32, "rho flags fit one word");
    int sc[ITEMS];
    int hc[ITEMS];                // LAT: entropy cell of a frontier item, loaded early
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int i = base + k;
        f[k] = 0u;
        sc[k] = -1;
        hc[k] = 0;
        if (i < a.n_total) {
            const int s = scene_of_point(a.scene_of, a.n_scenes, i);
            sc[k] = s;
            uint32_t r;
            f[k] = frontier_item<DIM>(a, i, s, eps_of(a.acc, s), &r);
            rho |= r << k;
            if (LAT && f[k]) hc[k] = a.hcell[i];
        }
        sum += f[k];
    }
    uint32_t tot;
    const uint32_t pre = block_exclusive_scan(sum, &tot, s_warp);
    if (threadIdx.x < 32) {
        const uint32_t ex = lookback(a.tstat_p, tp, tot, a.status);
        if (threadIdx.x == 0) s_excl = ex;
    }
    __syncthreads();
    uint32_t run = s_excl + pre;
    // a thread's consecutive points nearly always share one scene: accumulate
    // locally and reduce once per warp; a scene change inside them is flushed directly
    int cur = -1, acc_first = 0, acc_rho = 0;
    double acc_dl = 0.0;
    int old[ITEMS];               // LAT: the atomics' results, used after all are issued
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int i = base + k;
        const int s = sc[k];
        old[k] = -1;
        if (s >= 0) {
            if (!LAT && s != cur) {
                if (cur >= 0 && (acc_first || acc_dl != 0.0 || acc_rho)) {
                    if (acc_first) atomicAdd(&a.acc[cur].frontier_cells, acc_first);
                    if (acc_dl != 0.0) atomicAdd(&a.acc[cur].s_front, acc_dl);
                    if (acc_rho) atomicAdd(&a.acc[cur].n_rho, acc_rho);
                }
                cur = s;
                acc_first = 0;
                acc_dl = 0.0;
                acc_rho = 0;
            }
            if (!LAT) acc_rho += (int)((rho >> k) & 1u);
            const SceneParams &sp = a.sp[s];
            if (i == sp.pt_off) a.fstart[s] = (int)run;
            if (f[k]) {
                if (run < (uint32_t)a.n_total) a.frontier[run] = i - sp.pt_off;
                if (LAT) {
                    old[k] = count_inc(a.hcand, sp.h_off + hc[k], a.c16h);
                } else {
                    const int o = count_inc(a.hcand, sp.h_off + a.hcell[i], a.c16h);
                    acc_first += o == 0;
                    acc_dl += nlogn_step(a.nlogn, o);
                }
            }
            if (i == a.n_total - 1) a.fstart[a.n_scenes] = (int)(run + f[k]);
        }
        run += f[k];
    }
    if (LAT) {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int s = sc[k];
            if (s < 0) continue;
            if (s != cur) {
                if (cur >= 0 && (acc_first || acc_dl != 0.0 || acc_rho)) {
                    if (acc_first) atomicAdd(&a.acc[cur].frontier_cells, acc_first);
                    if (acc_dl != 0.0) atomicAdd(&a.acc[cur].s_front, acc_dl);
                    if (acc_rho) atomicAdd(&a.acc[cur].n_rho, acc_rho);
                }
                cur = s;
                acc_first = 0;
                acc_dl = 0.0;
                acc_rho = 0;
            }
            acc_rho += (int)((rho >> k) & 1u);
            if (old[k] >= 0) {
                acc_first += old[k] == 0;
                acc_dl += nlogn_step(a.nlogn, old[k]);
            }
        }
    }
    const unsigned m = scene_run_mask(cur);
    const int fc = run_sum_i32(m, acc_first);
    const double sd = run_sum_f64(m, acc_dl);
    const int nr = (a.audit & CERT_AUDIT_RHO) ? run_sum_i32(m, acc_rho) : 0;
    if (cur >= 0 && run_leader(m)) {
        if (fc) atomicAdd(&a.acc[cur].frontier_cells, fc);
        if (sd != 0.0) atomicAdd(&a.acc[cur].s_front, sd);
        if (nr) atomicAdd(&a.acc[cur].n_rho, nr);
    }
}

// ============================================================================ k_select

// One CTA per scene: select_scene (cert_phases.cuh) on the scan's results.
// NT threads per scene: 256 for batches; 1024 for fewer scenes than SMs,
// where each CTA's chain of dependent steps is the kernel's time and more
// threads shorten it (one median sample per thread instead of four).
// SPLIT (fewer scenes than SMs): 2 x n_scenes CTAs; the second n_scenes zero
// the scenes' failure counts and dilate their motion grids, in parallel with
// the selections instead of after them.
template <int DIM, int NT, bool SPLIT>
__global__ void __launch_bounds__(NT) k_select(const StepArgs a)
{
    __shared__ SelectSmem sm;
    __shared__ uint32_t s_mot[2][kMotionStride];
    const bool sel = !SPLIT || (int)blockIdx.x < a.n_scenes;   // uniform in the CTA
    const int s = sel ? (int)blockIdx.x : (int)blockIdx.x - a.n_scenes;
    if (sel) {
        const SceneAcc &acc = a.acc[s];
        const int nF = a.fstart[s + 1] - a.fstart[s];
        select_scene<DIM, NT>(a, s, eps_of(a.acc, s), nF, acc.s_front, acc.occ, acc.frontier_cells, sm);
        if (SPLIT) return;
    }
    {   // the scene's failure histogram starts empty (the refresh, search and far pass fill it)
        const SceneParams sp = a.sp[s];
        const int cells = (DIM == 3) ? sp.g_h * sp.g_h * sp.g_h : sp.g_h * sp.g_h;
        // (h_off is a multiple of 8: with 16-bit counts the scene's words are its own)
        const int w0 = a.c16h ? sp.h_off / 2 : sp.h_off;
        const int nw = a.c16h ? (cells + 1) / 2 : cells;
        for (int k = threadIdx.x; k < nw; k += NT) a.hfail[w0 + k] = 0;
    }
    if (a.mode == MODE_STEP)   // the refresh's local motion bound (k_scatter_refresh)
        dilate_motion<DIM>(a.mgrid + s * kMotionStride, s_mot[0], s_mot[1], a.mdil + s * kMotionStride,
                           threadIdx.x, NT);
}

// ============================================================================ k_scatter_refresh

// PER points per thread (strided by kThreads), their loads issued together:
// kScatPer for grids that fill the GPU, one for a small grid.
constexpr int kScatPer = 2;
constexpr int kSmallGridScatter = 6 * 148;   // one wave of k_scatter_refresh (42 registers)

template <int DIM, int PER, bool COST>
__global__ void __launch_bounds__(kThreads) k_scatter_refresh(const StepArgs a)
{
    const int base = blockIdx.x * (kThreads * PER) + threadIdx.x;
    const bool step = a.mode == MODE_STEP;
    int s[PER], na[PER], nb[PER], nc[PER];
    int2 br[PER];
    float4 p[PER];
    float Lold[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        s[k] = -1;
        na[k] = nb[k] = nc[k] = -1;
        Lold[k] = 0.0f;
        if (i < a.n_total) {
            s[k] = scene_of_point(a.scene_of, a.n_scenes, i);
            br[k] = a.brank[i];
            p[k] = a.pos_new[i];
            if (step) {
                na[k] = a.nn[i];
                nb[k] = a.nn2[i];
                nc[k] = a.nn3[i];
                Lold[k] = a.L[i];
            }
        }
    }
    int changed[PER], missed[PER], first[PER], hit[PER];
    double dl[PER];
    double cyc[PER];   // cost audit: this point's scatter + refresh cycles
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        changed[k] = missed[k] = first[k] = hit[k] = 0;
        dl[k] = 0.0;
        cyc[k] = 0.0;
        if (s[k] < 0) continue;
        const long long t0 = COST ? clock64() : 0;
        const SceneParams sp = a.sp[s[k]];
        int slot = a.bucket_start[br[k].x] + br[k].y;
        if ((unsigned)(slot - sp.pt_off) >= (unsigned)sp.n) {  // only after a timed-out scan
            atomicOr(a.status, ST_TIMEOUT);
            slot = i;
        }
        sorted_store(a.squad, slot - sp.pt_off + sp.s_off, p[k].x, p[k].y, p[k].z, i);
        bool need = true;
        if (step) {
            need = refresh_point<DIM>(a, sp, eps_of(a.acc, s[k]), i, p[k], na[k], nb[k], nc[k], Lold[k],
                                      a.st[s[k]].strategy == STRAT_INC, a.mdil + s[k] * kMotionStride,
                                      &changed[k]);
            if (changed[k]) {
                const uint32_t fl = a.inF[i];
                missed[k] = !(fl & 1u);
                hit[k] = (int)(fl >> 1);
                const int old = count_inc(a.hfail, sp.h_off + a.hcell[i], a.c16h);
                first[k] = old == 0;
                dl[k] = nlogn_step(a.nlogn, old);
            }
        }
        a.sflag[slot] = need ? 1 : 0;
        if (COST) cyc[k] = (double)(clock64() - t0);
    }
    if (!step) return;  // uniform across the grid
    if (COST) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const unsigned m = scene_run_mask(s[k]);
            const double c = run_sum_f64(m, cyc[k]);
            if (s[k] >= 0 && run_leader(m) && c > 0.0) atomicAdd(&a.acc[s[k]].refresh_cyc, (unsigned long long)c);
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const unsigned m = scene_run_mask(s[k]);
        const int ncg = run_sum_i32(m, changed[k]);
        if (__any_sync(kFull, ncg != 0)) {
            const int nm = run_sum_i32(m, missed[k]);
            const int fc = run_sum_i32(m, first[k]);
            const int nh = run_sum_i32(m, hit[k]);
            const double sd = run_sum_f64(m, dl[k]);
            if (s[k] >= 0 && run_leader(m) && ncg) {
                atomicAdd(&a.acc[s[k]].n_failed, ncg);
                atomicAdd(&a.acc[s[k]].n_missed, nm);
                if (nh) atomicAdd(&a.acc[s[k]].n_rho_hit, nh);
                atomicAdd(&a.acc[s[k]].failed_cells, fc);
                atomicAdd(&a.acc[s[k]].s_fail, sd);
            }
        }
    }
}

// ============================================================================ k_search

// One CTA compacts the flagged slots of CHUNK consecutive sorted slots
// (ascending, so a warp's queries are neighbours and share most rows), then
// searches them kThreads / G at a time, G lanes per query.  CHUNK is
// kSearchChunk with G = 1; a grid that fits one wave even at half that (a
// small or single scene) takes half-size chunks, so that a CTA's queries fit
// one round of kThreads instead of spilling a few stragglers into a second
// round on the critical path.  A grid that fits one wave at 64 slots per CTA
// (a scene of at most about 38,000 points) takes 64-slot chunks with G = 4
// lanes per query: the GPU has lanes to spare there, and each lane walks a
// quarter of its query's quads, which cuts the chain of dependent loads that
// bounds a lone query's latency.
// This CTA's share of a grid-stride zeroing of n16 16-byte words.  A call of
// its own: inlined at the end of k_search, its loop raised the search's spill
// loads from 44 to 100 bytes per thread.
__device__ __noinline__ void zero_span(int4 *p, long long n16)
{
    for (long long w = (long long)blockIdx.x * kThreads + threadIdx.x; w < n16; w += (long long)gridDim.x * kThreads)
        p[w] = make_int4(0, 0, 0, 0);
}

template <int DIM, int CHUNK, int G, bool COST>
__global__ void __launch_bounds__(kThreads, 4) k_search(const StepArgs a)   // 64 registers: 4 CTAs per SM
{
    constexpr int NR = (DIM == 3) ? 9 : 3;
    constexpr int NQ = kThreads / G;                       // queries per round
    constexpr int PER = CHUNK >= kThreads ? CHUNK / kThreads : 1;   // slots per thread in the compaction
    static_assert(PER == 1 || PER == 2 || PER == 4, "the flag load below reads one, two or four flags at once");
    static_assert(CHUNK >= kThreads || G * CHUNK <= kThreads, "a chunk of queries fits one round");
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_list[CHUNK];
    __shared__ int2 s_rng[(kMaxRows > NR ? kMaxRows : NR) * NQ];   // per-query row ranges, column-major
    __shared__ int s_next;                                          // G == 1: the next unclaimed batch
    // the batch's CTAs take their chunks heaviest first (k_chunk_order, from the
    // query counts the chunks had in the previous step)
    constexpr bool kOrdered = (CHUNK == kSearchChunk && G == 1);
    const int chunk = kOrdered ? a.chunk_order[blockIdx.x] : (int)blockIdx.x;
    const int base = chunk * CHUNK + threadIdx.x * PER;
    if (threadIdx.x == 0) s_next = kThreads;   // every warp's first batch of 32 is its own
    // flags beyond n_total are zero up to the padded length (a multiple of the
    // scan tile, itself a multiple of CHUNK); each flag byte is 0 or 1
    uint32_t fw = 0u;
    if (base < a.n_total && threadIdx.x * PER < CHUNK)
        fw = (PER == 4)   ? *reinterpret_cast<const uint32_t *>(a.sflag + base)
             : (PER == 2) ? (uint32_t)*reinterpret_cast<const uint16_t *>(a.sflag + base)
                          : (uint32_t)a.sflag[base];
    uint32_t count;
    if constexpr (CHUNK <= 32) {
        // a chunk of at most one warp's slots (small grids): warp 0 compacts it by
        // a ballot, one barrier instead of a block scan's
        __shared__ uint32_t s_count;
        if (threadIdx.x < 32) {
            const unsigned m = __ballot_sync(kFull, fw != 0u);
            if (fw) s_list[__popc(m & ((1u << threadIdx.x) - 1u))] = base;
            if (threadIdx.x == 0) s_count = (uint32_t)__popc(m);
        }
        __syncthreads();
        count = s_count;
    } else {
        uint32_t pre = block_exclusive_scan(__popc(fw), &count, s_warp);
#pragma unroll
        for (int u = 0; u < PER; ++u)
            if ((fw >> (8 * u)) & 0xffu) s_list[pre++] = base + u;
        if (kOrdered && threadIdx.x == 0) a.chunk_cnt[chunk] = (int)count;   // the next step's order
        __syncthreads();
    }

    // G == 1: a warp searches a batch of 32 consecutive queries, then claims the
    // CTA's next unclaimed batch, so warps that drew short boxes take more
    // batches instead of idling while one warp finishes its last.  G > 1 (small
    // grids, one round): NQ queries per round, G lanes each.
    const int gl = (G > 1) ? (int)(threadIdx.x % G) : 0;   // lane within the query's group
    const int lane = (int)(threadIdx.x & 31u);
    for (int r0 = (G == 1) ? (int)(threadIdx.x & ~31u) : 0;;) {
        if (r0 >= (int)count) break;
        if (G > 1 && r0 + (int)(threadIdx.x & ~31u) / G >= (int)count) break;  // whole idle warps leave together
        const int e = (G == 1) ? r0 + lane : r0 + (int)threadIdx.x / G;
        const bool active = e < (int)count;   // the same for the G lanes of a group
        int s = -1;
        SearchOut o = {0, 0, 0, 0, 0.0};
        const long long t0 = COST ? clock64() : 0;   // cost audit: this query's cycles
        if (active) {
            const int slot = s_list[e];
            s = scene_of_point(a.scene_of, a.n_scenes, slot);   // slot ranges of scenes equal their point ranges
            const SceneParams sp = a.sp[s];
            const SceneState &st = a.st[s];
            int gi = sorted_index(a.squad, slot - sp.pt_off + sp.s_off);
            if ((unsigned)(gi - sp.pt_off) >= (unsigned)sp.n) {  // only after a timed-out scan
                atomicOr(a.status, ST_TIMEOUT);
                gi = slot;
            }
            const float4 q = a.pos_new[gi];
            SearchCtx c;
            c.squad = a.squad;
            c.bstart = a.bucket_start;
#ifdef CERT_DEBUG_BOUNDS
            c.status = a.status;
#endif
            c.p = q;
            c.px2 = pack2(q.x, q.x);
            c.py2 = pack2(q.y, q.y);
            c.pz2 = pack2(q.z, q.z);
            c.gi = gi;
            c.pt_off = sp.pt_off;
            c.n = sp.n;
            c.pad = sp.s_off - sp.pt_off;
            c.boff = sp.bucket_off;
            c.T = sp.bucket_mask + 1;
            c.mask = (uint32_t)sp.bucket_mask;
            c.g = st.g_cur;
            c.inv_g = st.inv_g;
            c.dense = grid_is_dense<DIM>(c.g, c.T);
            Top4 t;
            float L;
            const float hint = (a.mode == MODE_STEP) ? a.L[gi] : 0.0f;   // written by the refresh
            const bool ok = grid_search<DIM, NQ, kMaxRows, G>(c, t, L, s_rng + threadIdx.x / G, hint, gl);
            if (gl == 0) {   // the group's lanes hold the same result; one writes it
                if (ok)
                    o = write_certificate(a, sp, gi, t, L,
                                          [&](int hc) { return count_inc(a.hfail, sp.h_off + hc, a.c16h); });
                else
                    a.far_list[atomicAdd(a.far_count, 1)] = slot;   // finished by k_far
            }
        }
        if (a.mode == MODE_STEP) {
            // slots of one scene are contiguous, so lanes form contiguous scene runs
            const unsigned m = scene_run_mask(s);
            const int nsr = run_sum_i32(m, (active && gl == 0) ? 1 : 0);
            const int nc = run_sum_i32(m, o.changed);
            const int nm = run_sum_i32(m, o.missed);
            const int fc = run_sum_i32(m, o.first);
            const int nh = run_sum_i32(m, o.hit);
            const double sd = run_sum_f64(m, o.dl);
            if (COST) {
                const double c = run_sum_f64(m, (active && gl == 0) ? (double)(clock64() - t0) : 0.0);
                if (s >= 0 && run_leader(m) && c > 0.0) atomicAdd(&a.acc[s].search_cyc, (unsigned long long)c);
            }
            if (s >= 0 && run_leader(m)) {
                atomicAdd(&a.acc[s].n_searched, nsr);
                if (nc) {
                    atomicAdd(&a.acc[s].n_failed, nc);
                    atomicAdd(&a.acc[s].n_missed, nm);
                    if (nh) atomicAdd(&a.acc[s].n_rho_hit, nh);
                    atomicAdd(&a.acc[s].failed_cells, fc);
                    atomicAdd(&a.acc[s].s_fail, sd);
                }
            }
        }
        if (G == 1) {   // the warp's next batch
            int nb = 0;
            if (lane == 0) nb = atomicAdd(&s_next, 32);
            r0 = __shfl_sync(kFull, nb, 0);
        } else {
            r0 += NQ;
        }
    }
    // the counters of the earlier phases are dead: zero them for the next call,
    // each warp once it has no query left (stores only)
    zero_span(a.ztail, a.ztail_n16);
}

// ============================================================================ chunk order

// The batch search's dispatch order: chunks sorted by the number of queries they
// had in the previous step, heaviest first (a counting sort on 32 classes of 32
// queries), so that long CTAs start early and the last ones dispatched are
// short; the SMs then run out of work together.  The order only schedules:
// every chunk is searched once whatever it is.  Run by one whole CTA (the first
// CTA of k_prepare, alongside its points: the counts come from the previous
// step's k_search, the order is read by this step's).
__device__ void order_chunks(const StepArgs &a, int nch, int *s_hist, int *s_start)
{
    if (threadIdx.x < 32) s_hist[threadIdx.x] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < nch; c += blockDim.x) atomicAdd(&s_hist[31 - min(31, a.chunk_cnt[c] >> 5)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < 32; ++b) {
            s_start[b] = run;
            run += s_hist[b];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nch; c += blockDim.x)
        a.chunk_order[atomicAdd(&s_start[31 - min(31, a.chunk_cnt[c] >> 5)], 1)] = c;
}

// ============================================================================ k_far

// Queries whose box would grow beyond kMaxExtend layers (points far from
// their neighbours relative to the scene's cell size).  One CTA per query
// scans the whole scene with coalesced loads, four in flight per thread, and
// merges the 256 partial top-3 lists; the result is exact (every point seen).
constexpr int kFarCtas = 2 * 148;

// Far queries first, first + stride, ... of the far list, each scanned by the
// whole CTA (kThreads threads) over its scene; the CTA's warps merge their top-4
// lists through s_d / s_j.
template <int DIM>
__device__ void far_items(const StepArgs &a, int first, int stride, float (*s_d)[4], int (*s_j)[4])
{
    const int nfar = *a.far_count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = first; item < nfar; item += stride) {
        const int slot = a.far_list[item];
        const int s = scene_of_point(a.scene_of, a.n_scenes, slot);
        const SceneParams sp = a.sp[s];
        int gi = sorted_index(a.squad, slot - sp.pt_off + sp.s_off);
        if ((unsigned)(gi - sp.pt_off) >= (unsigned)sp.n) gi = slot;
        const float4 p = a.pos_new[gi];
        const unsigned long long px = pack2(p.x, p.x), py = pack2(p.y, p.y), pz = pack2(p.z, p.z);
        Top4 t;
        top4_reset(t);
        // every quad of the scene, coalesced across the CTA
        const int q1 = (sp.s_off + sp.n + 3) >> 2;
        for (int q = (sp.s_off >> 2) + threadIdx.x; q < q1; q += kThreads) {
            const float4 *r = a.squad + (size_t)q * 4;
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
            s_d[warp][0] = t.d0; s_d[warp][1] = t.d1; s_d[warp][2] = t.d2; s_d[warp][3] = t.d3;
            s_j[warp][0] = t.j0; s_j[warp][1] = t.j1; s_j[warp][2] = t.j2; s_j[warp][3] = t.j3;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Top4 r;
            top4_reset(r);
            for (int w = 0; w < kThreads / 32; ++w)
                for (int k = 0; k < 4; ++k)
                    if (s_j[w][k] != 0x7fffffff) top4_insert(r, s_d[w][k], s_j[w][k]);
            const SearchOut o = write_certificate(a, sp, gi, r, sqrt_lower(r.d3),
                                                  [&](int hc) { return count_inc(a.hfail, sp.h_off + hc, a.c16h); });
            if (a.mode == MODE_STEP && o.changed) {
                atomicAdd(&a.acc[s].n_failed, 1);
                atomicAdd(&a.acc[s].n_missed, o.missed);
                if (o.hit) atomicAdd(&a.acc[s].n_rho_hit, 1);
                atomicAdd(&a.acc[s].failed_cells, o.first);
                atomicAdd(&a.acc[s].s_fail, o.dl);
            }
        }
        __syncthreads();
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_far(const StepArgs a)
{
    __shared__ float s_d[kThreads / 32][4];
    __shared__ int s_j[kThreads / 32][4];
    far_items<DIM>(a, blockIdx.x, gridDim.x, s_d, s_j);
}

// ============================================================================ k_geometry

// CERT_AUDIT_GEOMETRY only (launched when the flag is set): per scene, the
// FP64 sums of x, y, z and |p|^2 of the post-step positions of every point
// and of the failed points, for the radius of gyration in k_finalize.  Kept
// out of the repair kernels, which it would cost registers.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_geometry(const StepArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int s = -1;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    bool f = false;
    if (i < a.n_total) {
        s = scene_of_point(a.scene_of, a.n_scenes, i);
        p = a.pos_new[i];
        f = a.failed[i] != 0;
    }
    const double x = p.x, y = p.y, z = (DIM == 3) ? (double)p.z : 0.0;
    const double q = x * x + y * y + z * z;
    const unsigned m = scene_run_mask(s);
    const double v[4] = {x, y, z, q};
    double all[4], fail[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        all[k] = run_sum_f64(m, v[k]);
        fail[k] = run_sum_f64(m, f ? v[k] : 0.0);
    }
    if (s >= 0 && run_leader(m)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(&a.acc[s].a_sum[k], all[k]);
            if (fail[k] != 0.0) atomicAdd(&a.acc[s].f_sum[k], fail[k]);
        }
    }
}

// ============================================================================ k_finalize

// One thread per scene: finalize_scene (cert_phases.cuh); the scene's
// accumulators are then zeroed for the next call.
__global__ void k_finalize(const StepArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_scenes) return;
    const SceneAcc acc = a.acc[s];
    finalize_scene(a, s, acc, a.fstart[s + 1] - a.fstart[s], a.fstart[s]);
    a.acc[s] = SceneAcc{};
}

// ============================================================================ distances

__global__ void k_distances(const float *d1sq, const float *d2sq, float *d1, float *d2, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        d1[i] = __fsqrt_rn(d1sq[i]);
        d2[i] = __fsqrt_rn(d2sq[i]);
    }
}

// ============================================================================ launchers

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

template <int DIM, bool COST>
static void launch_scatter(const StepArgs &a, cudaStream_t st)
{
    if (nblk(a.n_total, kThreads) <= kSmallGridScatter)
        k_scatter_refresh<DIM, 1, COST><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(a);
    else
        k_scatter_refresh<DIM, kScatPer, COST><<<nblk(a.n_total, kThreads * kScatPer), kThreads, 0, st>>>(a);
}

template <int DIM, bool COST>
static void launch_search(const StepArgs &a, cudaStream_t st)
{
    if (nblk(a.n_total, kThreads / 8) <= kSearchSmallGrid)
        k_search<DIM, kThreads / 8, 8, COST><<<nblk(a.n_total, kThreads / 8), kThreads, 0, st>>>(a);
    else if (nblk(a.n_total, kThreads / 4) <= kSearchSmallGrid)
        k_search<DIM, kThreads / 4, 4, COST><<<nblk(a.n_total, kThreads / 4), kThreads, 0, st>>>(a);
    else if (nblk(a.n_total, kSearchChunk / 4) <= kSearchSmallGrid)
        k_search<DIM, kSearchChunk / 4, 1, COST><<<nblk(a.n_total, kSearchChunk / 4), kThreads, 0, st>>>(a);
    else if (nblk(a.n_total, kSearchChunk / 2) <= kSearchSmallGrid)
        k_search<DIM, kSearchChunk / 2, 1, COST><<<nblk(a.n_total, kSearchChunk / 2), kThreads, 0, st>>>(a);
    else   // chunk_order was written by k_prepare's first CTA (search_ordered)
        k_search<DIM, kSearchChunk, 1, COST><<<nblk(a.n_total, kSearchChunk), kThreads, 0, st>>>(a);
}

// Whether the search takes the batch's ordered full chunks (the last branch above).
static bool search_ordered(long long n)
{
    return nblk(n, kThreads / 4) > kSearchSmallGrid && nblk(n, kSearchChunk / 4) > kSearchSmallGrid &&
           nblk(n, kSearchChunk / 2) > kSearchSmallGrid;
}

template <int DIM>
static cudaError_t run_step_dim(const StepArgs &a, int phase, cudaStream_t st)
{
    switch (phase) {
    case PH_PREPARE: {
        StepArgs b = a;
        b.order_chunks = search_ordered(a.n_total) ? nblk(a.n_total, kSearchChunk) : 0;
        // the fewest points per thread whose grid still fits one wave (5 CTAs per SM)
        if (nblk(a.n_total, kThreads) <= kSmallGridPrepare)
            k_prepare<DIM, 1><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(b);
        else if (nblk(a.n_total, kThreads * 2) <= kSmallGridPrepare)
            k_prepare<DIM, 2><<<nblk(a.n_total, kThreads * 2), kThreads, 0, st>>>(b);
        else
            k_prepare<DIM, kPrepPer><<<nblk(a.n_total, kThreads * kPrepPer), kThreads, 0, st>>>(b);
        break;
    }
    case PH_SCAN:
        if ((a.ntiles_b + a.ntiles_p) * kScanItems <= 2 * 148) {
            // a very small grid (a single scene of up to about 18,000 points): eighth
            // tiles, one item per thread, still at most two CTAs per SM
            StepArgs b = a;
            b.ntiles_b = a.ntiles_b * kScanItems;
            b.ntiles_p = nblk(a.n_total, kThreads);
            k_scan<DIM, true, 1><<<b.ntiles_b + b.ntiles_p, kThreads, 0, st>>>(b);
        } else if (a.ntiles_b + a.ntiles_p < kScanLatencyTiles) {
            // a small grid: latency issue order and quarter tiles (two items per thread),
            // four times the CTAs and a quarter of each thread's chain
            StepArgs b = a;
            b.ntiles_b = a.ntiles_b * (kScanItems / 2);
            b.ntiles_p = nblk(a.n_total, kThreads * 2);
            k_scan<DIM, true, 2><<<b.ntiles_b + b.ntiles_p, kThreads, 0, st>>>(b);
        } else {
            k_scan<DIM, false, kScanItems><<<a.ntiles_b + a.ntiles_p, kThreads, 0, st>>>(a);
        }
        break;
    case PH_SELECT:
        if (a.n_scenes < 148)
            k_select<DIM, 1024, true><<<2 * a.n_scenes, 1024, 0, st>>>(a);
        else
            k_select<DIM, kThreads, false><<<a.n_scenes, kThreads, 0, st>>>(a);
        break;
    case PH_SCATTER:
        if (a.audit & CERT_AUDIT_COST)
            launch_scatter<DIM, true>(a, st);
        else
            launch_scatter<DIM, false>(a, st);
        break;
    case PH_SEARCH:
        if (a.audit & CERT_AUDIT_COST)
            launch_search<DIM, true>(a, st);
        else
            launch_search<DIM, false>(a, st);
        // far queries are rare: a small grid gets a few CTAs (each scans a whole scene per query)
        if (cudaPeekAtLastError() == cudaSuccess)
            k_far<DIM><<<std::min(kFarCtas, std::max(8, nblk(a.n_total, 4096))), kThreads, 0, st>>>(a);
        break;
    case PH_FINALIZE:
        if (a.mode == MODE_STEP && (a.audit & CERT_AUDIT_GEOMETRY))
            k_geometry<DIM><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(a);
        // one thread per scene, 32 per block: the FP64 logarithms of the entropies spread over
        // n_scenes / 32 SMs instead of a few
        if (cudaPeekAtLastError() == cudaSuccess) k_finalize<<<nblk(a.n_scenes, 32), 32, 0, st>>>(a);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_step_phase(const StepArgs &a, int phase, cudaStream_t st)
{
    return a.dim == 3 ? run_step_dim<3>(a, phase, st) : run_step_dim<2>(a, phase, st);
}

cudaError_t launch_distances(const float *d1sq, const float *d2sq, float *d1, float *d2, int n, cudaStream_t st)
{
    if (n > 0) k_distances<<<nblk(n, 256), 256, 0, st>>>(d1sq, d2sq, d1, d2, n);
    return cudaGetLastError();
}

}  // namespace certk
