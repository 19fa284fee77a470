// step_kernels.cu -- the per-step kernels of the certificate-maintenance loop.
//
// One step (Algorithm 1 of the paper, every certificate exact afterwards as in
// Cor. A.2) runs as five kernels over all scenes of a batch at once:
//
//   k_prepare          pack p' to float4, eps_t max-reduce (Alg. 1 first
//                      statement), search-grid bucket + rank (counting sort,
//                      histogram phase), entropy-grid cell + occupancy (Def. 2)
//   k_scan             decoupled look-back scans: bucket starts (counting sort,
//                      scan phase) and the ascending frontier list
//                      F = {i : c_i <= 4 eps_t + tau_i} (Alg. 1 second
//                      statement, Lemma 1) with the frontier-cell histogram
//   k_select           per scene: truncated medians, next search resolution,
//                      the strategy (forced, policy or learned selector)
//   k_scatter_refresh  counting-sort scatter into cell order; O(1) refresh of
//                      every certificate that its extended certificate still
//                      proves (frontier points included)
//   k_search           grid repair of the flagged points: top-2 over the 3^d
//                      block, widened until the runner-up is enclosed (Alg. 1
//                      block loop; Cor. A.2 widening)
//   k_finalize         per scene: H(F_t) (Def. 2), audit counts, next grid
//
// Extended certificate (an addition to the paper's record, needed because the
// paper leaves d1, d2 of safe points stale while every certificate here is
// exact each step): besides (nn, d1^2, d2^2) each point keeps its runner-up
// index nn2 and a lower bound L on the distance to every point other than nn
// and nn2.  A step changes the distance from i to any j by at most
// |p'_i - p_i| + eps_t (triangle inequality, as in Lemma 1), so L minus that
// bounds the next step; when both fresh distances to nn and nn2 stay below it
// the top-2 is exactly {nn, nn2} in fresh order, otherwise the point is
// repaired by a search.  The test is independent of the safety rule, so a
// frontier point it proves is repaired in O(1) too (a change of nn is then
// found by the reordering of {nn, nn2}).
#include "cert_internal.cuh"
#include "cert_launch.h"

namespace certk {

// ============================================================================ k_prepare

// PER points per thread (strided by kThreads, so a warp's lanes still hold
// consecutive points): the loads, atomics and stores of the points are issued
// together, overlapping their latencies.  kPrepPer for grids that fill the GPU;
// a small grid takes fewer per thread and more CTAs (chosen at the launch).
constexpr int kPrepPer = 4;
constexpr int kSmallGridPrepare = 5 * 148;   // one wave of k_prepare (48 registers)

template <int DIM, int PER>
__global__ void __launch_bounds__(kThreads, 5) k_prepare(const StepArgs a)   // 48 registers: 5 CTAs per SM
{
    const int base = blockIdx.x * (kThreads * PER) + threadIdx.x;
    int s[PER];
    float4 p[PER], po[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        s[k] = -1;
        p[k] = po[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < a.n_total) {
            s[k] = a.scene_of[i];
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
        rank[k] = atomicAdd(&a.bucket_count[b[k]], 1);
        // entropy grid on the post-step position (Def. 2)
        if (a.mode != MODE_REBUILD) {
            const int gh = sp.g_h;
            const float ghf = (float)gh;
            const int hx = cell_coord(p[k].x, gh, ghf);
            const int hy = cell_coord(p[k].y, gh, ghf);
            hc[k] = (DIM == 3) ? (cell_coord(p[k].z, gh, ghf) * gh + hy) * gh + hx : hy * gh + hx;
            first[k] = atomicAdd(&a.hocc[sp.h_off + hc[k]], 1) == 0;
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
template <int DIM, bool LAT>
__global__ void __launch_bounds__(kThreads) k_scan(const StepArgs a)
{
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_tile;
    __shared__ uint32_t s_excl;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const int t = s_tile;

    if (t < a.ntiles_b) {
        // ---- bucket counts -> bucket starts (global exclusive scan over all scenes)
        const int base = t * kScanTile + threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; k += 4) {
            const int4 c4 = *reinterpret_cast<const int4 *>(a.bucket_count + base + k);
            v[k] = (uint32_t)c4.x;
            v[k + 1] = (uint32_t)c4.y;
            v[k + 2] = (uint32_t)c4.z;
            v[k + 3] = (uint32_t)c4.w;
        }
        uint32_t sum = 0u;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) sum += v[k];
        uint32_t tot;
        const uint32_t pre = block_exclusive_scan(sum, &tot, s_warp);
        if (threadIdx.x < 32) {
            const uint32_t ex = lookback(a.tstat_b, t, tot, a.status);
            if (threadIdx.x == 0) s_excl = ex;
        }
        __syncthreads();
        uint32_t run = s_excl + pre;
        int o[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            o[k] = (int)run;
            run += v[k];
        }
#pragma unroll
        for (int k = 0; k < kScanItems; k += 4)
            *reinterpret_cast<int4 *>(a.bucket_start + base + k) = make_int4(o[k], o[k + 1], o[k + 2], o[k + 3]);
        return;
    }

    // ---- frontier flags -> ascending frontier list (Algorithm 1, Lemma 1)
    const int tp = t - a.ntiles_b;
    const int base = tp * kScanTile + threadIdx.x * kScanItems;
    uint32_t f[kScanItems];
    uint32_t rho = 0u;                 // bit k: item k flagged by the rho heuristic
    static_assert(kScanItems <= 32, "rho flags fit one word");
    int sc[kScanItems];
    int hc[kScanItems];                // LAT: entropy cell of a frontier item, loaded early
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = base + k;
        f[k] = 0u;
        sc[k] = -1;
        hc[k] = 0;
        if (i < a.n_total) {
            const int s = a.scene_of[i];
            sc[k] = s;
            const float eps = eps_of(a.acc, s);
            const float d1 = __fsqrt_rn(a.d1sq[i]);
            const float d2 = __fsqrt_rn(a.d2sq[i]);
            const float c = __fsub_rn(d2, d1);
            if (a.frontier_rule == CERT_FRONTIER_CLOCK) {
                // cumulative clock (Thm A.3): revisit last step's frontier from the
                // current certificates, then test 4 (S - S_i) against c^rev_i, in FP64
                const double S_prev = a.st[s].S;
                double S_i;
                float c_rev, g_rev;
                if (a.inF[i] & 1u) {
                    S_i = S_prev;
                    c_rev = c;
                    g_rev = __fadd_rn(d1, d2);
                    a.clk_s[i] = S_i;
                    a.clk_c[i] = c_rev;
                    a.clk_g[i] = g_rev;
                } else {
                    S_i = a.clk_s[i];
                    c_rev = a.clk_c[i];
                    g_rev = a.clk_g[i];
                }
                const double D = __dsub_rn(__dadd_rn(S_prev, (double)eps), S_i);
                const double rhs = __dadd_rn(__dmul_rn(4.0, D), __dmul_rn(0x1p-20, __dadd_rn((double)g_rev, D)));
                f[k] = ((double)c_rev <= rhs) ? 1u : 0u;
            } else {
                const float tau = __fmul_rn(0x1p-20f, __fadd_rn(__fadd_rn(d1, d2), eps));
                float motion;           // the rule's bound on how much c can shrink, over 2
                if (a.frontier_rule == CERT_FRONTIER_POINT) {
                    // per-point budget: point i moved by delta_i (k_prepare keeps its square in w)
                    motion = __fmul_rn(2.0f, __fadd_rn(__fsqrt_rn(a.pos_new[i].w), eps));
                } else {
                    motion = __fmul_rn(4.0f, eps);   // Algorithm 1, Lemma 1
                }
                f[k] = (c <= __fadd_rn(motion, tau)) ? 1u : 0u;
            }
            // the local heuristic of Sec. 3: rho_i = delta_i / c_i > 1/2, taken as
            // 2 delta_i > c_i on the FP32 values (exact: the doubling rounds nothing)
            uint32_t r = 0u;
            if (a.audit & CERT_AUDIT_RHO) {
                r = (__fmul_rn(2.0f, __fsqrt_rn(a.pos_new[i].w)) > c) ? 1u : 0u;
                rho |= r << k;
            }
            a.inF[i] = (uint8_t)(f[k] | (r << 1));
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
    int old[kScanItems];               // LAT: the atomics' results, used after all are issued
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
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
                    old[k] = atomicAdd(&a.hcand[sp.h_off + hc[k]], 1);
                } else {
                    const int o = atomicAdd(&a.hcand[sp.h_off + a.hcell[i]], 1);
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
        for (int k = 0; k < kScanItems; ++k) {
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

// Truncated order statistic: the rank-r smallest of the sampled values,
// truncated to its sign, exponent and top 3 mantissa bits.  Truncation is
// monotone, so that value is exactly the 12-bit bin (bits >> 20) in which the
// cumulative histogram first exceeds r: a 2048-bin shared histogram and one
// block scan replace a full sort.  Values are non-negative (or +inf).
constexpr int kTruncBins = 2048;

__device__ uint32_t trunc_select(const uint32_t *hist, int rank, uint32_t *s_warp, int *s_bin)
{
    constexpr int per = kTruncBins / kThreads;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) sum += hist[threadIdx.x * per + k];
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(sum, &tot, s_warp);
    if (pre <= (uint32_t)rank && (uint32_t)rank < pre + sum) {
        for (int k = 0; k < per; ++k) {
            pre += hist[threadIdx.x * per + k];
            if ((uint32_t)rank < pre) {
                *s_bin = threadIdx.x * per + k;
                break;
            }
        }
    }
    __syncthreads();
    const uint32_t bin = (uint32_t)*s_bin;
    __syncthreads();
    return bin << 20;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_select(const StepArgs a)
{
    __shared__ uint32_t s_hc[kTruncBins];
    __shared__ uint32_t s_hd[kTruncBins];
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_bin;
    __shared__ float s_feat[8];
    __shared__ __align__(16) float s_h1[64];
    __shared__ __align__(16) float s_h2[64];
    __shared__ float s_out[2];
    const int s = blockIdx.x;
    const SceneParams sp = a.sp[s];
    const int ns = min(sp.n, kMedianSample);
    for (int k = threadIdx.x; k < kTruncBins; k += kThreads) {
        s_hc[k] = 0u;
        s_hd[k] = 0u;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += kThreads) {
        const int i = sp.pt_off + k;
        const float d1 = __fsqrt_rn(a.d1sq[i]);
        const float d2 = __fsqrt_rn(a.d2sq[i]);
        // c >= 0 and d2 >= 0 (or +inf): bit patterns >> 20 lie in [0, 2047]; NaN is clamped
        atomicAdd(&s_hc[min(__float_as_uint(__fsub_rn(d2, d1)) >> 20, (uint32_t)kTruncBins - 1)], 1u);
        atomicAdd(&s_hd[min(__float_as_uint(d2) >> 20, (uint32_t)kTruncBins - 1)], 1u);
    }
    __syncthreads();
    // lower median of the clearances; the cell-size reference quantile of d2
    const float med_c = __uint_as_float(trunc_select(s_hc, (ns - 1) / 2, s_warp, &s_bin));
    const int qi = min(ns - 1, max(0, (int)(a.cell_quantile * (float)(ns - 1))));
    const float med_d2 = __uint_as_float(trunc_select(s_hd, qi, s_warp, &s_bin));

    int strat = STRAT_INC;
    if (a.mode == MODE_STEP) {
        strat = a.strategy;
        if (strat == STRAT_AUTO) strat = a.policy;
        // ---- the eight selector features of this step (stored every step)
        if (threadIdx.x == 0) {
            const SceneAcc acc = a.acc[s];
            const SceneState st = a.st[s];
            const int nF = a.fstart[s + 1] - a.fstart[s];
            const float eps = eps_of(a.acc, s);
            const double lnF = nF > 1 ? log((double)nF) : 0.0;
            const double Hc = (nF > 1 && acc.occ > 1)
                                  ? fmin(1.0, fmax(0.0, (lnF - acc.s_front / nF) / log((double)acc.occ)))
                                  : 0.0;
            float x[8];
            x[0] = (float)nF / (float)sp.n;                               // |F|/N
            x[1] = (float)Hc;                                             // H of the detected frontier
            x[2] = logf((float)sp.n);                                     // ln N
            x[3] = (float)DIM;                                            // d
            x[4] = log1pf(fminf(eps / fmaxf(med_c, 1e-30f), 1e6f));       // ln(1 + eps_t / med c)
            x[5] = acc.occ > 0 ? (float)acc.frontier_cells / (float)acc.occ : 0.0f;  // touched-cell fraction
            x[6] = st.prev_fail_ratio;                                    // previous failed / frontier
            x[7] = st.prev_pred_ratio;                                    // previous predicted ln ratio
            for (int k = 0; k < 8; ++k) {
                a.feat[s * 8 + k] = x[k];
                s_feat[k] = a.sel_norm ? (x[k] - a.sel_norm[k]) * a.sel_norm[8 + k] : x[k];
            }
            // Prop. 1 rule with the boundary P ~ 1/ln N measured in Sec. 4
            if (a.strategy == STRAT_THR) strat = (x[0] < 1.0f / x[2]) ? STRAT_INC : STRAT_REB;
        }
        if (a.strategy == STRAT_AUTO && a.sel_params != nullptr) {
            // ---- learned selector: MLP 8-64-64-2 on the normalised features -> argmin
            __syncthreads();
            const float *W1 = a.sel_params, *b1 = W1 + 64 * 8, *W2 = b1 + 64, *b2 = W2 + 64 * 64,
                        *W3 = b2 + 64, *b3 = W3 + 2 * 64;
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (threadIdx.x < 64) {
                const float4 wa = *reinterpret_cast<const float4 *>(W1 + threadIdx.x * 8);
                const float4 wb = *reinterpret_cast<const float4 *>(W1 + threadIdx.x * 8 + 4);
                float z = b1[threadIdx.x];
                z = fmaf(wa.x, s_feat[0], z);
                z = fmaf(wa.y, s_feat[1], z);
                z = fmaf(wa.z, s_feat[2], z);
                z = fmaf(wa.w, s_feat[3], z);
                z = fmaf(wb.x, s_feat[4], z);
                z = fmaf(wb.y, s_feat[5], z);
                z = fmaf(wb.z, s_feat[6], z);
                z = fmaf(wb.w, s_feat[7], z);
                s_h1[threadIdx.x] = fmaxf(z, 0.0f);
            }
            __syncthreads();
            {
                // layer 2 as a warp-cooperative product: warp w owns outputs 8w .. 8w+7,
                // lane l reads the row pair (2l, 2l+1), coalesced, then the warp reduces
                const float2 h = *reinterpret_cast<const float2 *>(s_h1 + 2 * lane);
                float z[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 w = *reinterpret_cast<const float2 *>(W2 + (warp * 8 + u) * 64 + 2 * lane);
                    z[u] = fmaf(w.x, h.x, w.y * h.y);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int u = 0; u < 8; ++u) z[u] += __shfl_xor_sync(kFull, z[u], o);
                if (lane < 8) {
                    float v = z[0];
#pragma unroll
                    for (int u = 1; u < 8; ++u)
                        if (lane == u) v = z[u];
                    s_h2[warp * 8 + lane] = fmaxf(v + b2[warp * 8 + lane], 0.0f);
                }
            }
            __syncthreads();
            if (warp < 2) {
                // output o = warp: lane l covers hidden units (2l, 2l+1)
                const float2 w = *reinterpret_cast<const float2 *>(W3 + warp * 64 + 2 * lane);
                const float2 h = *reinterpret_cast<const float2 *>(s_h2 + 2 * lane);
                float y = fmaf(w.x, h.x, w.y * h.y);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(kFull, y, o);
                if (lane == 0) s_out[warp] = y;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const float pi = s_out[0] + b3[0];
                const float pr = s_out[1] + b3[1];
                SceneState st = a.st[s];
                st.pred_inc = pi;
                st.pred_reb = pr;
                if (isfinite(pi) && isfinite(pr)) strat = (pi <= pr) ? STRAT_INC : STRAT_REB;
                st.prev_pred_ratio = isfinite(pi - pr) ? (pi - pr) : 0.0f;
                a.st[s] = st;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        SceneState st = a.st[s];
        st.med_c = med_c;
        st.med_d2 = med_d2;
        int g = sp.g_default;
        const float h = __fmul_rn(a.cell_scale, med_d2);
        if (h > 0.0f && isfinite(h)) {
            const float gg = ceilf(1.0f / h);
            g = (gg >= (float)kMaxSearchRes) ? kMaxSearchRes : max(1, (int)gg);
        }
        st.g_next = g;
        if (a.mode == MODE_STEP) st.strategy = strat;
        a.st[s] = st;
    }
}

// ============================================================================ k_scatter_refresh

// PER points per thread (strided by kThreads), their loads issued together:
// kScatPer for grids that fill the GPU, one for a small grid.
constexpr int kScatPer = 2;
constexpr int kSmallGridScatter = 6 * 148;   // one wave of k_scatter_refresh (42 registers)

template <int DIM, int PER>
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
            s[k] = a.scene_of[i];
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
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = base + k * kThreads;
        changed[k] = missed[k] = first[k] = hit[k] = 0;
        dl[k] = 0.0;
        if (s[k] < 0) continue;
        const SceneParams sp = a.sp[s[k]];
        int slot = a.bucket_start[br[k].x] + br[k].y;
        if ((unsigned)(slot - sp.pt_off) >= (unsigned)sp.n) {  // only after a timed-out scan
            atomicOr(a.status, ST_TIMEOUT);
            slot = i;
        }
        sorted_store(a.squad, slot - sp.pt_off + sp.s_off, p[k].x, p[k].y, p[k].z, i);
        bool need = true;
        if (step) {
            float hint = 0.0f;             // no box hint unless the candidates are valid
            if ((unsigned)na[k] < (unsigned)sp.n && (unsigned)nb[k] < (unsigned)sp.n) {
                // fresh keys of the three stored candidates, sorted
                const bool hc3 = (unsigned)nc[k] < (unsigned)sp.n;
                const float4 qa = a.pos_new[sp.pt_off + na[k]];
                const float4 qb = a.pos_new[sp.pt_off + nb[k]];
                const float4 qc = hc3 ? a.pos_new[sp.pt_off + nc[k]] : qa;
                float d1 = sqdist<DIM>(p[k], qa);
                float d2 = sqdist<DIM>(p[k], qb);
                float d3 = hc3 ? sqdist<DIM>(p[k], qc) : __int_as_float(0x7f800000);
                int j1 = na[k], j2 = nb[k], j3 = hc3 ? nc[k] : 0x7fffffff;
                if (key_less(d2, j2, d1, j1)) {
                    swapv(d1, d2);
                    swapv(j1, j2);
                }
                if (key_less(d3, j3, d2, j2)) {
                    swapv(d2, d3);
                    swapv(j2, j3);
                    if (key_less(d2, j2, d1, j1)) {
                        swapv(d1, d2);
                        swapv(j1, j2);
                    }
                }
                // any distance from i changed by at most |p'_i - p_i| + eps_t
                // (triangle inequality); both terms rounded up with slack
                const float shrink = __fmul_ru(__fadd_ru(__fsqrt_ru(p[k].w), eps_of(a.acc, s[k])), 1.0f + 0x1p-18f);
                const float Lnew = __fsub_rd(Lold[k], shrink);
                // a search of this point can size its box from the second key:
                // the fresh runner-up over all points is no farther
                hint = __fsqrt_ru(d2);
                // every point outside {nn, nn2, nn3} is now at least Lnew away, so
                // when the second key is closer the top-2 is the first two keys
                if (a.st[s[k]].strategy == STRAT_INC && Lnew > 0.0f &&
                    __fmul_ru(d2, 1.0f + 0x1p-19f) < __fmul_rd(Lnew, Lnew)) {
                    need = false;
                    a.nn[i] = j1;
                    a.nn2[i] = j2;
                    a.nn3[i] = (j3 != 0x7fffffff) ? j3 : -1;
                    a.d1sq[i] = d1;
                    a.d2sq[i] = d2;
                    a.L[i] = Lnew;
                    changed[k] = j1 != na[k];
                    a.failed[i] = (uint8_t)changed[k];
                    if (changed[k]) {
                        const uint32_t fl = a.inF[i];
                        missed[k] = !(fl & 1u);
                        hit[k] = (int)(fl >> 1);
                        const int old = atomicAdd(&a.hfail[sp.h_off + a.hcell[i]], 1);
                        first[k] = old == 0;
                        dl[k] = nlogn_step(a.nlogn, old);
                    }
                }
            }
            if (need) a.L[i] = hint;       // read by the search; replaced by its result
        }
        a.sflag[slot] = need ? 1 : 0;
    }
    if (!step) return;  // uniform across the grid
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

struct SearchCtx {
    const float4 *squad;
    const int *bstart;
    float4 p;
    unsigned long long px2, py2, pz2;   // query coordinates, each packed twice
    int gi;
    int pt_off, n, pad, boff, T;        // pad = s_off - pt_off (slot -> quad-array index)
    uint32_t mask;
    int g;
    float inv_g;
    bool dense;
#ifdef CERT_DEBUG_BOUNDS
    uint32_t *status;
#endif
};

// Visit the sorted slots [lo, hi) of the scene.  The range is widened to whole
// quads; the extra slots are other points of the same scene (visiting more
// points never changes a top-k) or NaN padding, which no comparison accepts.
// Each quad is four 16-byte loads and one packed evaluation, with the next
// quad's loads issued before the current quad's arithmetic; one test of the
// quad's minimum against the current fourth key skips the insertions.
template <int DIM>
__device__ __forceinline__ void visit_range(const SearchCtx &c, int lo, int hi, Top4 &t)
{
    lo = max(lo, c.pt_off);          // a bucket range never leaves its scene
    hi = min(hi, c.pt_off + c.n);
    if (lo >= hi) return;
    const int q0 = (lo + c.pad) >> 2;
    const int q1 = (hi + c.pad + 3) >> 2;
    CERT_CHECK(c.status, q0 >= ((c.pt_off + c.pad) >> 2) && q1 <= ((c.pt_off + c.n + c.pad + 3) >> 2));
    const float4 *r = c.squad + (size_t)q0 * 4;
    float4 X = r[0], Y = r[1];
    float4 Z = (DIM == 3) ? r[2] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = q0; q < q1; ++q) {
        const float4 cX = X, cY = Y, cZ = Z;
        const float4 *rc = r;
        r += 4;
        if (q + 1 < q1) {
            X = r[0];
            Y = r[1];
            if (DIM == 3) Z = r[2];
        }
        float D0, D1, D2, D3;
        sqdist_quad<DIM>(c.px2, c.py2, c.pz2, cX, cY, cZ, D0, D1, D2, D3);
        if (fminf(fminf(D0, D1), fminf(D2, D3)) <= t.d3) {
            const float4 J = rc[3];
            const int j0 = __float_as_int(J.x), j1 = __float_as_int(J.y);
            const int j2 = __float_as_int(J.z), j3 = __float_as_int(J.w);
            if (D0 <= t.d3 && j0 != c.gi) top4_insert(t, D0, j0);
            if (D1 <= t.d3 && j1 != c.gi) top4_insert(t, D1, j1);
            if (D2 <= t.d3 && j2 != c.gi) top4_insert(t, D2, j2);
            if (D3 <= t.d3 && j3 != c.gi) top4_insert(t, D3, j3);
        }
    }
}


// Walk the quad ranges rng[0..NR) (column stride kThreads) as one stream, the
// next quad's loads -- across row ends too -- issued before the current
// quad's arithmetic.
template <int DIM>
__device__ __forceinline__ void visit_quad_rows(const SearchCtx &c, const int2 *rng, int NR, Top4 &t)
{
    int k = 0;
    int2 rr = rng[0];
    int q = rr.x, qe = rr.y;
    while (q >= qe && k + 1 < NR) {
        ++k;
        rr = rng[k * kThreads];
        q = rr.x;
        qe = rr.y;
    }
    if (q >= qe) return;
#ifdef CERT_DEBUG_BOUNDS
    const int qmin = (c.pt_off + c.pad) >> 2, qmax = (c.pt_off + c.n + c.pad + 3) >> 2;
    for (int kk = 0; kk < NR; ++kk) {
        const int2 rk = rng[kk * kThreads];
        CERT_CHECK(c.status, rk.x >= rk.y || (rk.x >= qmin && rk.y <= qmax));
    }
#endif
    const float4 *r = c.squad + (size_t)q * 4;
    float4 X = r[0], Y = r[1];
    float4 Z = (DIM == 3) ? r[2] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (;;) {
        const float4 cX = X, cY = Y, cZ = Z;
        const float4 *rc = r;
        ++q;
        while (q >= qe && k + 1 < NR) {
            ++k;
            rr = rng[k * kThreads];
            q = rr.x;
            qe = rr.y;
        }
        const bool more = q < qe;
        if (more) {
            r = c.squad + (size_t)q * 4;
            X = r[0];
            Y = r[1];
            if (DIM == 3) Z = r[2];
        }
        float D0, D1, D2, D3;
        sqdist_quad<DIM>(c.px2, c.py2, c.pz2, cX, cY, cZ, D0, D1, D2, D3);
        if (fminf(fminf(D0, D1), fminf(D2, D3)) <= t.d3) {
            const float4 J = rc[3];
            const int j0 = __float_as_int(J.x), j1 = __float_as_int(J.y);
            const int j2 = __float_as_int(J.z), j3 = __float_as_int(J.w);
            if (D0 <= t.d3 && j0 != c.gi) top4_insert(t, D0, j0);
            if (D1 <= t.d3 && j1 != c.gi) top4_insert(t, D1, j1);
            if (D2 <= t.d3 && j2 != c.gi) top4_insert(t, D2, j2);
            if (D3 <= t.d3 && j3 != c.gi) top4_insert(t, D3, j3);
        }
        if (!more) break;
    }
}

// Slot range(s) of the cells [xl, xh] of row (yr, zr).  A row's cells are
// consecutive buckets; the second range is non-empty only when they wrap.
template <int DIM>
__device__ __forceinline__ void row_ranges(const SearchCtx &c, int yr, int zr, int xl, int xh, int &lo, int &hi,
                                           int &lo2, int &hi2)
{
    lo = hi = lo2 = hi2 = 0;
    xl = max(xl, 0);
    xh = min(xh, c.g - 1);
    if (xl > xh || yr < 0 || yr >= c.g || zr < 0 || zr >= c.g) return;
    const int len = xh - xl + 1;
    if (len >= c.T) {
        lo = c.pt_off;
        hi = c.pt_off + c.n;
        return;
    }
    const int b0 = (int)((row_base<DIM>(yr, zr, c.g, c.dense) + (uint32_t)xl) & c.mask);
    if (b0 + len <= c.T) {
        lo = c.bstart[c.boff + b0];
        hi = c.bstart[c.boff + b0 + len];
    } else {
        lo = c.bstart[c.boff + b0];
        hi = c.bstart[c.boff + c.T];
        lo2 = c.bstart[c.boff];
        hi2 = c.bstart[c.boff + b0 + len - c.T];
    }
}

template <int DIM>
__device__ __forceinline__ void visit_row(const SearchCtx &c, int yr, int zr, int xl, int xh, Top4 &t)
{
    int lo, hi, lo2, hi2;
    row_ranges<DIM>(c, yr, zr, xl, xh, lo, hi, lo2, hi2);
    visit_range<DIM>(c, lo, hi, t);
    if (hi2 > lo2) visit_range<DIM>(c, lo2, hi2, t);
}

constexpr float kFaceSlack = 0x1p-17f;   // >> FP error of cell assignment and face position
constexpr float kHintGrow = 1.15f;       // box radius / box hint (margin for the bound L)
constexpr int kMaxRows = 16;             // rows of a hinted box kept in the shared range table

// Thread-level grid search over a box of cells [x0,x1] x [y0,y1] x [z0,z1]
// holding the query's cell.  It starts as the 3^d block of Algorithm 1 and
// grows one cell layer at a time on the face nearest to the query -- the face
// that limits the enclosure -- until the runner-up is provably enclosed (its
// distance is below the distance to every face that is not on the grid
// edge; boundary cells are clamped and extend to infinity), as in Cor. A.2.
// Returns false after kMaxExtend layers; such a query is appended to the far
// list and finished by k_far.
template <int DIM>
__device__ __forceinline__ bool grid_search(const SearchCtx &c, Top4 &t, float &Lout, int2 *rng, float hint)
{
    const float gf = (float)c.g;
    const int cx = cell_coord(c.p.x, c.g, gf);
    const int cy = cell_coord(c.p.y, c.g, gf);
    const int cz = (DIM == 3) ? cell_coord(c.p.z, c.g, gf) : 0;
    const int gm = c.g - 1;
    top4_reset(t);
    // Every row's slot range is fetched first (independent loads) and kept, as
    // a range of quads, in this thread's column of the shared range table; the
    // rows are then walked as one quad stream, the query's own row first: its
    // nearest candidates set a tight fourth key early, so most quads of the
    // other rows skip the insertions.
    int x0, x1, y0, y1, z0, z1, nrows = 0;
    if (hint > 0.0f) {
        // The box of the cells that meet the ball of radius kHintGrow * hint:
        // the runner-up is at most hint away, so the enclosure test nearly
        // always passes without growing the box.
        const float R = __fmul_ru(hint, kHintGrow);
        x0 = cell_coord(__fsub_rd(c.p.x, R), c.g, gf);
        x1 = cell_coord(__fadd_ru(c.p.x, R), c.g, gf);
        y0 = cell_coord(__fsub_rd(c.p.y, R), c.g, gf);
        y1 = cell_coord(__fadd_ru(c.p.y, R), c.g, gf);
        z0 = (DIM == 3) ? cell_coord(__fsub_rd(c.p.z, R), c.g, gf) : 0;
        z1 = (DIM == 3) ? cell_coord(__fadd_ru(c.p.z, R), c.g, gf) : 0;
        if ((y1 - y0 + 1) * (z1 - z0 + 1) <= kMaxRows) {
            rng[0] = make_int2(0, 0);      // the own row's entry, filled in the loop
            nrows = 1;
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y) {
                    const int k = (y == cy && z == cz) ? 0 : nrows++;
                    int lo, hi, lo2, hi2;
                    row_ranges<DIM>(c, y, z, x0, x1, lo, hi, lo2, hi2);
                    if (hi2 > lo2) visit_range<DIM>(c, lo2, hi2, t);   // wrapped row: rare
                    lo = max(lo, c.pt_off);
                    hi = min(hi, c.pt_off + c.n);
                    rng[k * kThreads] = (lo < hi) ? make_int2((lo + c.pad) >> 2, (hi + c.pad + 3) >> 2)
                                                  : make_int2(0, 0);
                }
        }
    }
    if (nrows == 0) {
        // no usable hint: the 3^d block of Algorithm 1
        constexpr int NR = (DIM == 3) ? 9 : 3;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const int kr = (k + NR / 2) % NR;   // the query's own row first
            const int yr = cy + (kr % 3) - 1;
            const int zr = (DIM == 3) ? cz + (kr / 3) - 1 : 0;
            int lo, hi, lo2, hi2;
            row_ranges<DIM>(c, yr, zr, cx - 1, cx + 1, lo, hi, lo2, hi2);
            if (hi2 > lo2) visit_range<DIM>(c, lo2, hi2, t);   // wrapped row: rare
            lo = max(lo, c.pt_off);
            hi = min(hi, c.pt_off + c.n);
            rng[k * kThreads] = (lo < hi) ? make_int2((lo + c.pad) >> 2, (hi + c.pad + 3) >> 2) : make_int2(0, 0);
        }
        nrows = NR;
        x0 = max(cx - 1, 0);
        x1 = min(cx + 1, gm);
        y0 = max(cy - 1, 0);
        y1 = min(cy + 1, gm);
        z0 = (DIM == 3) ? max(cz - 1, 0) : 0;
        z1 = (DIM == 3) ? min(cz + 1, gm) : 0;
    }
    visit_quad_rows<DIM>(c, rng, nrows, t);

    const float inf = __int_as_float(0x7f800000);
    for (int ext = 0;; ++ext) {
        // distances to the six faces (+inf on the grid edge)
        float f[6];
        f[0] = x0 > 0 ? __fsub_rn(c.p.x, __fmul_rn((float)x0, c.inv_g)) : inf;
        f[1] = x1 < gm ? __fsub_rn(__fmul_rn((float)(x1 + 1), c.inv_g), c.p.x) : inf;
        f[2] = y0 > 0 ? __fsub_rn(c.p.y, __fmul_rn((float)y0, c.inv_g)) : inf;
        f[3] = y1 < gm ? __fsub_rn(__fmul_rn((float)(y1 + 1), c.inv_g), c.p.y) : inf;
        f[4] = (DIM == 3 && z0 > 0) ? __fsub_rn(c.p.z, __fmul_rn((float)z0, c.inv_g)) : inf;
        f[5] = (DIM == 3 && z1 < gm) ? __fsub_rn(__fmul_rn((float)(z1 + 1), c.inv_g), c.p.z) : inf;
        int side = 0;
        float f0 = f[0];
#pragma unroll
        for (int k = 1; k < 6; ++k)
            if (f[k] < f0) {
                f0 = f[k];
                side = k;
            }
        if (isinf(f0)) {  // the box covers the whole grid: everything was visited
            Lout = sqrt_lower(t.d3);
            return true;
        }
        const float fs = __fsub_rd(f0, kFaceSlack);
        if (t.j1 != 0x7fffffff && fs > 0.0f &&
            __fmul_ru(t.d1, 1.0f + 0x1p-19f) < __fmul_rd(fs, fs)) {  // runner-up provably enclosed
            Lout = fminf(sqrt_lower(t.d3), fs);
            return true;
        }
        if (ext >= kMaxExtend) return false;
        // grow the limiting face by one cell layer and visit the new cells
        switch (side) {
        case 0:
        case 1: {
            const int x = (side == 0) ? --x0 : ++x1;
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y) visit_row<DIM>(c, y, z, x, x, t);
            break;
        }
        case 2:
        case 3: {
            const int y = (side == 2) ? --y0 : ++y1;
            for (int z = z0; z <= z1; ++z) visit_row<DIM>(c, y, z, x0, x1, t);
            break;
        }
        default: {
            const int z = (side == 4) ? --z0 : ++z1;
            for (int y = y0; y <= y1; ++y) visit_row<DIM>(c, y, z, x0, x1, t);
            break;
        }
        }
    }
}

// Merge the warp's per-lane top-4 lists (butterfly; every lane ends with the result).
__device__ __forceinline__ void warp_merge_top4(Top4 &t)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float e0 = __shfl_xor_sync(kFull, t.d0, o), e1 = __shfl_xor_sync(kFull, t.d1, o),
                    e2 = __shfl_xor_sync(kFull, t.d2, o), e3 = __shfl_xor_sync(kFull, t.d3, o);
        const int k0 = __shfl_xor_sync(kFull, t.j0, o), k1 = __shfl_xor_sync(kFull, t.j1, o),
                  k2 = __shfl_xor_sync(kFull, t.j2, o), k3 = __shfl_xor_sync(kFull, t.j3, o);
        if (k0 != 0x7fffffff) top4_insert(t, e0, k0);
        if (k1 != 0x7fffffff) top4_insert(t, e1, k1);
        if (k2 != 0x7fffffff) top4_insert(t, e2, k2);
        if (k3 != 0x7fffffff) top4_insert(t, e3, k3);
    }
}

// Certificate write and failure audit of one searched point (thread level).
struct SearchOut {
    int changed, missed, first, hit;
    double dl;
};

__device__ __forceinline__ SearchOut write_certificate(const StepArgs &a, const SceneParams &sp, int gi,
                                                       const Top4 &t, float L)
{
    SearchOut o = {0, 0, 0, 0, 0.0};
    const int n1 = (t.j0 != 0x7fffffff) ? t.j0 - sp.pt_off : -1;
    const int n2 = (t.j1 != 0x7fffffff) ? t.j1 - sp.pt_off : -1;
    CERT_CHECK(a.status, (unsigned)(gi - sp.pt_off) < (unsigned)sp.n && (unsigned)n1 < (unsigned)sp.n &&
                             (unsigned)n2 < (unsigned)sp.n);
    if (a.mode == MODE_STEP) {
        o.changed = n1 != a.nn[gi];
        a.failed[gi] = (uint8_t)o.changed;
        if (o.changed) {
            const uint32_t fl = a.inF[gi];
            o.missed = !(fl & 1u);
            o.hit = (int)(fl >> 1);
            const int old = atomicAdd(&a.hfail[sp.h_off + a.hcell[gi]], 1);
            o.first = old == 0;
            o.dl = nlogn_step(a.nlogn, old);
        }
    }
    a.nn[gi] = n1;
    a.nn2[gi] = n2;
    a.nn3[gi] = (t.j2 != 0x7fffffff) ? t.j2 - sp.pt_off : -1;
    a.d1sq[gi] = t.d0;
    a.d2sq[gi] = t.d1;
    a.L[gi] = L;
    return o;
}

// One CTA compacts the flagged slots of CHUNK consecutive sorted slots
// (ascending, so a warp's queries are neighbours and share most rows), then
// searches them kThreads at a time.  CHUNK is kSearchChunk; a grid that fits
// one wave even at half that (a small or single scene) takes half-size chunks,
// so that a CTA's queries fit one round of kThreads instead of spilling a few
// stragglers into a second round on the critical path.
template <int DIM, int CHUNK>
__global__ void __launch_bounds__(kThreads, 4) k_search(const StepArgs a)   // 64 registers: 4 CTAs per SM
{
    constexpr int NR = (DIM == 3) ? 9 : 3;
    constexpr int PER = CHUNK / kThreads;   // slots per thread in the compaction
    static_assert(PER == 1 || PER == 2 || PER == 4, "the flag load below reads one, two or four flags at once");
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_list[CHUNK];
    __shared__ int2 s_rng[(kMaxRows > NR ? kMaxRows : NR) * kThreads];   // per-thread row ranges, column-major
    const int base = blockIdx.x * CHUNK + threadIdx.x * PER;
    // flags beyond n_total are zero up to the padded length (a multiple of the
    // scan tile, itself a multiple of CHUNK); each flag byte is 0 or 1
    uint32_t fw = 0u;
    if (base < a.n_total)
        fw = (PER == 4)   ? *reinterpret_cast<const uint32_t *>(a.sflag + base)
             : (PER == 2) ? (uint32_t)*reinterpret_cast<const uint16_t *>(a.sflag + base)
                          : (uint32_t)a.sflag[base];
    uint32_t count;
    uint32_t pre = block_exclusive_scan(__popc(fw), &count, s_warp);
#pragma unroll
    for (int u = 0; u < PER; ++u)
        if ((fw >> (8 * u)) & 0xffu) s_list[pre++] = base + u;
    __syncthreads();

    for (int r0 = 0; r0 < (int)count; r0 += kThreads) {
        if (r0 + (int)(threadIdx.x & ~31u) >= (int)count) break;  // whole idle warps leave together
        const int e = r0 + (int)threadIdx.x;
        const bool active = e < (int)count;
        int s = -1;
        SearchOut o = {0, 0, 0, 0, 0.0};
        if (active) {
            const int slot = s_list[e];
            s = a.scene_of[slot];        // slot ranges of scenes equal their point ranges
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
            if (grid_search<DIM>(c, t, L, s_rng + threadIdx.x, hint))
                o = write_certificate(a, sp, gi, t, L);
            else
                a.far_list[atomicAdd(a.far_count, 1)] = slot;   // finished by k_far
        }
        if (a.mode == MODE_STEP) {
            // slots of one scene are contiguous, so lanes form contiguous scene runs
            const unsigned m = scene_run_mask(s);
            const int nsr = run_sum_i32(m, active ? 1 : 0);
            const int nc = run_sum_i32(m, o.changed);
            const int nm = run_sum_i32(m, o.missed);
            const int fc = run_sum_i32(m, o.first);
            const int nh = run_sum_i32(m, o.hit);
            const double sd = run_sum_f64(m, o.dl);
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
    }
}

// ============================================================================ k_far

// Queries whose box would grow beyond kMaxExtend layers (points far from
// their neighbours relative to the scene's cell size).  One CTA per query
// scans the whole scene with coalesced loads, four in flight per thread, and
// merges the 256 partial top-3 lists; the result is exact (every point seen).
constexpr int kFarCtas = 2 * 148;

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_far(const StepArgs a)
{
    __shared__ float s_d[kThreads / 32][4];
    __shared__ int s_j[kThreads / 32][4];
    const int nfar = *a.far_count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < nfar; item += gridDim.x) {
        const int slot = a.far_list[item];
        const int s = a.scene_of[slot];
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
            const SearchOut o = write_certificate(a, sp, gi, r, sqrt_lower(r.d3));
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
        s = a.scene_of[i];
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

// sqrt(mean |p|^2 - |mean p|^2) from the FP64 sums of x, y, z, |p|^2 of n points
__device__ __forceinline__ double gyration_radius(const double *sum, int n)
{
    if (n < 2) return 0.0;
    const double inv = 1.0 / (double)n;
    const double mx = sum[0] * inv, my = sum[1] * inv, mz = sum[2] * inv;
    return sqrt(fmax(0.0, sum[3] * inv - (mx * mx + my * my + mz * mz)));
}

// ============================================================================ k_finalize

__device__ __forceinline__ double norm_entropy(int n, double s_nlogn, int C)
{
    // H = -sum q ln q / ln C with q = n_k / n, i.e. (ln n - (1/n) sum n_k ln n_k) / ln C
    if (n <= 1 || C <= 1) return 0.0;
    const double h = (log((double)n) - s_nlogn / (double)n) / log((double)C);
    return fmin(1.0, fmax(0.0, h));
}

__global__ void k_finalize(const StepArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_scenes) return;
    const SceneParams sp = a.sp[s];
    SceneState st = a.st[s];
    if (a.mode == MODE_STEP) {
        const SceneAcc acc = a.acc[s];
        const int nF = a.fstart[s + 1] - a.fstart[s];
        cert_scene_result r;
        r.eps_t = eps_of(a.acc, s);
        r.med_c = st.med_c;
        r.H = norm_entropy(acc.n_failed, acc.s_fail, acc.occ);
        r.H_cand = norm_entropy(nF, acc.s_front, acc.occ);
        r.n_frontier = nF;
        r.frontier_start = a.fstart[s];
        r.n_failed = acc.n_failed;
        r.n_missed = acc.n_missed;
        r.n_false = nF - (acc.n_failed - acc.n_missed);
        r.n_searched = acc.n_searched;
        r.failed_cells = acc.failed_cells;
        r.frontier_cells = acc.frontier_cells;
        r.occupied_cells = acc.occ;
        r.strategy = st.strategy;
        r.pred_inc = st.pred_inc;
        r.pred_reb = st.pred_reb;
        r.grid_res = sp.g_h;
        r.search_res = st.g_cur;
        r.n_rho = acc.n_rho;
        r.n_rho_hit = acc.n_rho_hit;
        r.gyration = 0.0;
        r.compactness = 0.0;
        if ((a.audit & CERT_AUDIT_GEOMETRY) && acc.n_failed > 0) {
            r.gyration = gyration_radius(acc.f_sum, acc.n_failed);
            const double all = gyration_radius(acc.a_sum, sp.n);
            r.compactness = all > 0.0 ? fmin(1.0, fmax(0.0, 1.0 - r.gyration / all)) : 1.0;
        }
        a.res[s] = r;
        if (r.eps_t > __fmul_ru(a.declared_eps, 1.0f + 0x1p-20f)) atomicOr(a.status, ST_EBOUND);
        st.prev_fail_ratio = (float)acc.n_failed / (float)max(1, nF);
        st.prev_nfront = nF;
        st.S = __dadd_rn(st.S, (double)r.eps_t);   // cumulative clock
    }
    st.g_cur = st.g_next;
    st.inv_g = __frcp_rn((float)st.g_cur);
    a.st[s] = st;
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

template <int DIM>
static cudaError_t run_step_dim(const StepArgs &a, int phase, cudaStream_t st)
{
    switch (phase) {
    case PH_PREPARE:
        // the fewest points per thread whose grid still fits one wave (5 CTAs per SM)
        if (nblk(a.n_total, kThreads) <= kSmallGridPrepare)
            k_prepare<DIM, 1><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(a);
        else if (nblk(a.n_total, kThreads * 2) <= kSmallGridPrepare)
            k_prepare<DIM, 2><<<nblk(a.n_total, kThreads * 2), kThreads, 0, st>>>(a);
        else
            k_prepare<DIM, kPrepPer><<<nblk(a.n_total, kThreads * kPrepPer), kThreads, 0, st>>>(a);
        break;
    case PH_SCAN:
        if (a.ntiles_b + a.ntiles_p < kScanLatencyTiles)
            k_scan<DIM, true><<<a.ntiles_b + a.ntiles_p, kThreads, 0, st>>>(a);
        else
            k_scan<DIM, false><<<a.ntiles_b + a.ntiles_p, kThreads, 0, st>>>(a);
        break;
    case PH_SELECT: k_select<DIM><<<a.n_scenes, kThreads, 0, st>>>(a); break;
    case PH_SCATTER:
        if (nblk(a.n_total, kThreads) <= kSmallGridScatter)
            k_scatter_refresh<DIM, 1><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(a);
        else
            k_scatter_refresh<DIM, kScatPer><<<nblk(a.n_total, kThreads * kScatPer), kThreads, 0, st>>>(a);
        break;
    case PH_SEARCH:
        if (nblk(a.n_total, kSearchChunk / 4) <= kSearchSmallGrid)
            k_search<DIM, kSearchChunk / 4><<<nblk(a.n_total, kSearchChunk / 4), kThreads, 0, st>>>(a);
        else if (nblk(a.n_total, kSearchChunk / 2) <= kSearchSmallGrid)
            k_search<DIM, kSearchChunk / 2><<<nblk(a.n_total, kSearchChunk / 2), kThreads, 0, st>>>(a);
        else
            k_search<DIM, kSearchChunk><<<nblk(a.n_total, kSearchChunk), kThreads, 0, st>>>(a);
        if (cudaPeekAtLastError() == cudaSuccess) k_far<DIM><<<kFarCtas, kThreads, 0, st>>>(a);
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
