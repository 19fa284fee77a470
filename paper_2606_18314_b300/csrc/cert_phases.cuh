// cert_phases.cuh -- the per-point and per-scene phases of one certificate
// step, shared by the multi-kernel step (step_kernels.cu: one kernel per
// phase over every scene of a batch) and the fused step (fused_step.cu: one
// CTA runs every phase of one scene).  Results do not depend on which runs
// them; only the amount of work (which points are searched) may differ.
#pragma once

#include "cert_internal.cuh"
#include "cert_launch.h"

namespace certk {

// ============================================================================ frontier test

// Frontier membership of point i of scene s (Algorithm 1's second statement,
// Lemma 1, with the rounding guard; or the per-point budget, or the
// cumulative clock of the per-step cost subsection), from its pre-step
// certificate.  Writes inF[i] (bit 0: in F_t; bit 1: flagged by the rho
// heuristic of Sec. 3 when audited) and the clock rule's revisit state.
// Returns the membership; *rho = the rho flag.
template <int DIM>
__device__ __forceinline__ uint32_t frontier_item(const StepArgs &a, int i, int s, float eps, uint32_t *rho)
{
    const float d1 = __fsqrt_rn(a.d1sq[i]);
    const float d2 = __fsqrt_rn(a.d2sq[i]);
    const float c = __fsub_rn(d2, d1);
    uint32_t f;
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
        f = ((double)c_rev <= rhs) ? 1u : 0u;
    } else {
        const float tau = __fmul_rn(0x1p-20f, __fadd_rn(__fadd_rn(d1, d2), eps));
        float motion;           // the rule's bound on how much c can shrink, over 2
        if (a.frontier_rule == CERT_FRONTIER_POINT) {
            // per-point budget: point i moved by delta_i (the prepare phase keeps its square in w)
            motion = __fmul_rn(2.0f, __fadd_rn(__fsqrt_rn(a.pos_new[i].w), eps));
        } else {
            motion = __fmul_rn(4.0f, eps);   // Algorithm 1, Lemma 1
        }
        f = (c <= __fadd_rn(motion, tau)) ? 1u : 0u;
    }
    // the local heuristic of Sec. 3: rho_i = delta_i / c_i > 1/2, taken as
    // 2 delta_i > c_i on the FP32 values (exact: the doubling rounds nothing)
    uint32_t r = 0u;
    if (a.audit & CERT_AUDIT_RHO) r = (__fmul_rn(2.0f, __fsqrt_rn(a.pos_new[i].w)) > c) ? 1u : 0u;
    a.inF[i] = (uint8_t)(f | (r << 1));
    *rho = r;
    return f;
}

// ============================================================================ finalize

// sqrt(mean |p|^2 - |mean p|^2) from the FP64 sums of x, y, z, |p|^2 of n points
__device__ __forceinline__ double gyration_radius(const double *sum, int n)
{
    if (n < 2) return 0.0;
    const double inv = 1.0 / (double)n;
    const double mx = sum[0] * inv, my = sum[1] * inv, mz = sum[2] * inv;
    return sqrt(fmax(0.0, sum[3] * inv - (mx * mx + my * my + mz * mz)));
}

// Normalised entropy of a histogram of n items over cells, C occupied cells
// in the scene, from s_nlogn = sum over cells of n_k ln n_k (Def. 2):
// H = -sum q ln q / ln C with q = n_k / n, i.e. (ln n - (1/n) s_nlogn) / ln C,
// in FP64, with ln n, 1/n and 1/ln C read from the host-computed tables.
__device__ __forceinline__ double norm_entropy(const double *tab, int n, double s_nlogn, int C)
{
    if (n <= 1 || C <= 1) return 0.0;
    double h;
    if (n < kNlognTable && C < kNlognTable)
        h = (tab_ln(tab, n) - s_nlogn * tab_inv(tab, n)) * tab_inv_ln(tab, C);
    else
        h = (log((double)n) - s_nlogn / (double)n) / log((double)C);
    return fmin(1.0, fmax(0.0, h));
}

// ============================================================================ select

// Truncated order statistic: the rank-r smallest of the sampled values,
// truncated to its sign, exponent and top 3 mantissa bits.  Truncation is
// monotone, so that value is exactly the 12-bit bin (bits >> 20) in which the
// cumulative histogram first exceeds r: a 2048-bin shared histogram and one
// block scan replace a full sort.  Values are non-negative (or +inf).
constexpr int kTruncBins = 2048;

// The two order statistics of select_scene in one pass: rank rc of the
// histogram hc and rank rd of hd, from one block scan of both bin counts
// packed into one word (each histogram holds at most kMedianSample <= 65,535
// values, so the low half never carries into the high one).  Returns the two
// truncated values in *vc and *vd (every thread).
template <int NT>
__device__ void trunc_select2(const uint32_t *hc, const uint32_t *hd, int rc, int rd, uint32_t *s_warp,
                              int *s_bin, uint32_t *vc, uint32_t *vd)
{
    constexpr int per = kTruncBins / NT;
    static_assert(per >= 1 && kTruncBins % NT == 0, "bins split evenly over the block");
    uint32_t sc = 0, sd = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        sc += hc[threadIdx.x * per + k];
        sd += hd[threadIdx.x * per + k];
    }
    uint32_t tot;
    const uint32_t pre = block_exclusive_scan<NT>(sc | (sd << 16), &tot, s_warp);
    uint32_t pc = pre & 0xffffu, pd = pre >> 16;
    if (pc <= (uint32_t)rc && (uint32_t)rc < pc + sc) {
        for (int k = 0; k < per; ++k) {
            pc += hc[threadIdx.x * per + k];
            if ((uint32_t)rc < pc) {
                s_bin[0] = threadIdx.x * per + k;
                break;
            }
        }
    }
    if (pd <= (uint32_t)rd && (uint32_t)rd < pd + sd) {
        for (int k = 0; k < per; ++k) {
            pd += hd[threadIdx.x * per + k];
            if ((uint32_t)rd < pd) {
                s_bin[1] = threadIdx.x * per + k;
                break;
            }
        }
    }
    __syncthreads();
    *vc = (uint32_t)s_bin[0] << 20;
    *vd = (uint32_t)s_bin[1] << 20;
    __syncthreads();
}

// Shared memory of select_scene.
struct SelectSmem {
    uint32_t hc[kTruncBins];
    uint32_t hd[kTruncBins];
    uint32_t warp[32];
    int bins[2];
    float feat[8];
    __align__(16) float h1[64];
    __align__(16) float h2[64];
    float out[2];
};

// Per-scene selection, run by a whole block of NT threads (NT >= 256): the
// truncated medians of the pre-step clearances and runner-up distances over
// the first min(n, kMedianSample) points, the eight selector features of the
// step, the strategy (forced, policy, Prop. 1's threshold or the learned
// MLP's argmin) and the next step's search resolution.  eps is the scene's
// eps_t; nF, s_front, occ and frontier_cells are the scan's results for it.  Writes the scene's
// state and features; returns the strategy applied.
template <int DIM, int NT>
__device__ int select_scene(const StepArgs &a, int s, float eps, int nF, double s_front, int occ,
                            int frontier_cells, SelectSmem &sm)
{
    static_assert(NT >= 256 && NT % 32 == 0, "the MLP layers use the first eight warps");
    const SceneParams sp = a.sp[s];
    const int ns = min(sp.n, kMedianSample);
    // thread 0: the scene's state, read once here and written once at the end,
    // and the frontier's entropy, whose table reads overlap the histograms
    SceneState st;
    double Hc = 0.0;
    if (threadIdx.x == 0) {
        st = a.st[s];
        if (a.mode == MODE_STEP) Hc = norm_entropy(a.nlogn, nF, s_front, occ);
    }
    for (int k = threadIdx.x; k < kTruncBins; k += NT) {
        sm.hc[k] = 0u;
        sm.hd[k] = 0u;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += NT) {
        const int i = sp.pt_off + k;
        const float d1 = __fsqrt_rn(a.d1sq[i]);
        const float d2 = __fsqrt_rn(a.d2sq[i]);
        // c >= 0 and d2 >= 0 (or +inf): bit patterns >> 20 lie in [0, 2047]; NaN is clamped
        atomicAdd(&sm.hc[min(__float_as_uint(__fsub_rn(d2, d1)) >> 20, (uint32_t)kTruncBins - 1)], 1u);
        atomicAdd(&sm.hd[min(__float_as_uint(d2) >> 20, (uint32_t)kTruncBins - 1)], 1u);
    }
    __syncthreads();
    // lower median of the clearances; the cell-size reference quantile of d2
    const int qi = min(ns - 1, max(0, (int)(a.cell_quantile * (float)(ns - 1))));
    uint32_t vc, vd;
    trunc_select2<NT>(sm.hc, sm.hd, (ns - 1) / 2, qi, sm.warp, sm.bins, &vc, &vd);
    const float med_c = __uint_as_float(vc);
    const float med_d2 = __uint_as_float(vd);

    int strat = STRAT_INC;
    if (a.mode == MODE_STEP) {
        strat = a.strategy;
        if (strat == STRAT_AUTO) strat = a.scene_policy ? a.scene_policy[s] : a.policy;
        // ---- the eight selector features of this step (stored every step)
        if (threadIdx.x == 0) {
            float x[8];
            x[0] = (float)nF / (float)sp.n;                               // |F|/N
            x[1] = (float)Hc;                                             // H of the detected frontier
            x[2] = logf((float)sp.n);                                     // ln N
            x[3] = (float)DIM;                                            // d
            x[4] = log1pf(fminf(eps / fmaxf(med_c, 1e-30f), 1e6f));       // ln(1 + eps_t / med c)
            x[5] = occ > 0 ? (float)frontier_cells / (float)occ : 0.0f;   // touched-cell fraction
            x[6] = st.prev_fail_ratio;                                    // previous failed / frontier
            x[7] = st.prev_pred_ratio;                                    // previous predicted ln ratio
            for (int k = 0; k < 8; ++k) {
                a.feat[s * 8 + k] = x[k];
                sm.feat[k] = a.sel_norm ? (x[k] - a.sel_norm[k]) * a.sel_norm[8 + k] : x[k];
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
                z = fmaf(wa.x, sm.feat[0], z);
                z = fmaf(wa.y, sm.feat[1], z);
                z = fmaf(wa.z, sm.feat[2], z);
                z = fmaf(wa.w, sm.feat[3], z);
                z = fmaf(wb.x, sm.feat[4], z);
                z = fmaf(wb.y, sm.feat[5], z);
                z = fmaf(wb.z, sm.feat[6], z);
                z = fmaf(wb.w, sm.feat[7], z);
                sm.h1[threadIdx.x] = fmaxf(z, 0.0f);
            }
            __syncthreads();
            if (warp < 8) {
                // layer 2 as a warp-cooperative product: warp w owns outputs 8w .. 8w+7,
                // lane l reads the row pair (2l, 2l+1), coalesced, then the warp reduces
                const float2 h = *reinterpret_cast<const float2 *>(sm.h1 + 2 * lane);
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
                    sm.h2[warp * 8 + lane] = fmaxf(v + b2[warp * 8 + lane], 0.0f);
                }
            }
            __syncthreads();
            if (warp < 2) {
                // output o = warp: lane l covers hidden units (2l, 2l+1)
                const float2 w = *reinterpret_cast<const float2 *>(W3 + warp * 64 + 2 * lane);
                const float2 h = *reinterpret_cast<const float2 *>(sm.h2 + 2 * lane);
                float y = fmaf(w.x, h.x, w.y * h.y);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(kFull, y, o);
                if (lane == 0) sm.out[warp] = y;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const float pi = sm.out[0] + b3[0];
                const float pr = sm.out[1] + b3[1];
                st.pred_inc = pi;
                st.pred_reb = pr;
                if (isfinite(pi) && isfinite(pr)) strat = (pi <= pr) ? STRAT_INC : STRAT_REB;
                st.prev_pred_ratio = isfinite(pi - pr) ? (pi - pr) : 0.0f;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
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
    return strat;   // valid in thread 0
}

// ============================================================================ refresh

// O(1) refresh of point i (an addition to the paper's record:
// every certificate is exact each step, Cor. A.2).  Every point other than
// the three stored candidates was at least L away; a step changes the
// distance from i to any j by at most |p'_i - p_i| + |p'_j - p_j| (triangle
// inequality, as in Lemma 1), so L minus a bound on that bounds the next
// step.  The bound is tried twice: first with eps_t for |p'_j - p_j| (the
// scene's largest step), then, if that fails, with the largest step among the
// points of the 3^d motion-grid block around p'_i (mdil: the scene's dilated
// motion grid), a bound that holds for every point inside the block, capped
// by the distance to the block's faces, which bounds every point outside it.
// The fresh keys of the three candidates are sorted; when the second is
// closer than the shrunk bound, the first two keys are the exact top-2 and
// the certificate is written (a change of nn is a failure: *changed = 1).
// Otherwise the point needs a search, and L[i] receives its box hint (the
// second fresh key's distance: the fresh runner-up over all points is no
// farther).  Returns true when the point needs a search.
template <int DIM>
__device__ __forceinline__ bool refresh_point(const StepArgs &a, const SceneParams &sp, float eps, int i, float4 p,
                                              int na, int nb, int nc, float Lold, bool inc, const uint32_t *mdil,
                                              int *changed)
{
    *changed = 0;
    float hint = 0.0f;             // no box hint unless the candidates are valid
    bool need = true;
    if ((unsigned)na < (unsigned)sp.n && (unsigned)nb < (unsigned)sp.n) {
        // fresh keys of the three stored candidates, sorted
        const bool hc3 = (unsigned)nc < (unsigned)sp.n;
        const float4 qa = a.pos_new[sp.pt_off + na];
        const float4 qb = a.pos_new[sp.pt_off + nb];
        const float4 qc = hc3 ? a.pos_new[sp.pt_off + nc] : qa;
        float d1 = sqdist<DIM>(p, qa);
        float d2 = sqdist<DIM>(p, qb);
        float d3 = hc3 ? sqdist<DIM>(p, qc) : __int_as_float(0x7f800000);
        int j1 = na, j2 = nb, j3 = hc3 ? nc : 0x7fffffff;
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
        const float own = __fsqrt_ru(p.w);
        const float shrink = __fmul_ru(__fadd_ru(own, eps), 1.0f + 0x1p-18f);
        float Lnew = __fsub_rd(Lold, shrink);
        hint = __fsqrt_ru(d2);
        const float d2g = __fmul_ru(d2, 1.0f + 0x1p-19f);
        bool ok = inc && Lnew > 0.0f && d2g < __fmul_rd(Lnew, Lnew);
        if (inc && !ok) {
            // the local bound: the points of the motion block moved at most
            // sqrt(mdil) each; the points outside it are beyond its faces
            const float dl = __fsqrt_ru(__uint_as_float(mdil[motion_cell<DIM>(p)]));
            const float sl = __fmul_ru(__fadd_ru(own, dl), 1.0f + 0x1p-18f);
            const float Lloc = fminf(__fsub_rd(Lold, sl), motion_block_face<DIM>(p));
            if (Lloc > Lnew) Lnew = Lloc;
            ok = Lnew > 0.0f && d2g < __fmul_rd(Lnew, Lnew);
        }
        // every point outside {nn, nn2, nn3} is now at least Lnew away, so
        // when the second key is closer the top-2 is the first two keys
        if (ok) {
            need = false;
            a.nn[i] = j1;
            a.nn2[i] = j2;
            a.nn3[i] = (j3 != 0x7fffffff) ? j3 : -1;
            a.d1sq[i] = d1;
            a.d2sq[i] = d2;
            a.L[i] = Lnew;
            *changed = j1 != na;
            a.failed[i] = (uint8_t)*changed;
        }
    }
    if (need) a.L[i] = hint;       // read by the search; replaced by its result
    return need;
}

// Per-scene end of a step (one thread): H(F_t) (Def. 2), H_cand, the audit
// counts and descriptors into the scene's result, the eps bound check, and
// the state carried to the next step (ratios, the cumulative clock, the
// next search grid).  acc holds the step's accumulators; nF and f0 are the
// scene's frontier length and its offset in the frontier array.
__device__ __forceinline__ void finalize_scene(const StepArgs &a, int s, const SceneAcc &acc, int nF, int f0)
{
    const SceneParams sp = a.sp[s];
    SceneState st = a.st[s];
    if (a.mode == MODE_STEP) {
        cert_scene_result r;
        r.eps_t = __fsqrt_rn(__uint_as_float(acc.eps_bits));
        r.med_c = st.med_c;
        r.H = norm_entropy(a.nlogn, acc.n_failed, acc.s_fail, acc.occ);
        r.H_cand = norm_entropy(a.nlogn, nF, acc.s_front, acc.occ);
        r.n_frontier = nF;
        r.frontier_start = f0;
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
        r.search_cycles = acc.search_cyc;
        r.refresh_cycles = acc.refresh_cyc;
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

// ============================================================================ search

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


// Walk the quad ranges rng[0..NR) (column stride STRIDE: one column per thread
// of the block) as one stream, the next quad's loads -- across row ends too --
// issued before the current quad's arithmetic.
template <int DIM, int STRIDE>
__device__ __forceinline__ void visit_quad_rows(const SearchCtx &c, const int2 *rng, int NR, Top4 &t)
{
    int k = 0;
    int2 rr = rng[0];
    int q = rr.x, qe = rr.y;
    while (q >= qe && k + 1 < NR) {
        ++k;
        rr = rng[k * STRIDE];
        q = rr.x;
        qe = rr.y;
    }
    if (q >= qe) return;
#ifdef CERT_DEBUG_BOUNDS
    const int qmin = (c.pt_off + c.pad) >> 2, qmax = (c.pt_off + c.n + c.pad + 3) >> 2;
    for (int kk = 0; kk < NR; ++kk) {
        const int2 rk = rng[kk * STRIDE];
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
            rr = rng[k * STRIDE];
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

// The same walk shared by G lanes of one query.  The query's rows are taken as
// one sequence of quads, and lane g (0 <= g < G) takes quads g, g + G, g + 2G,
// ... of it, so the lanes' shares differ by at most one quad whatever the row
// lengths (the group's merge waits for its slowest lane); each lane's next
// quad's loads are issued before the current quad's arithmetic, across row
// ends too.  The lanes' top-4 lists are merged afterwards.
template <int DIM, int STRIDE, int G>
__device__ __forceinline__ void visit_quad_rows_split(const SearchCtx &c, const int2 *rng, int NR, Top4 &t, int g)
{
#ifdef CERT_DEBUG_BOUNDS
    const int qmin = (c.pt_off + c.pad) >> 2, qmax = (c.pt_off + c.n + c.pad + 3) >> 2;
    for (int kk = 0; kk < NR; ++kk) {
        const int2 rk = rng[kk * STRIDE];
        CERT_CHECK(c.status, rk.x >= rk.y || (rk.x >= qmin && rk.y <= qmax));
    }
#endif
    int k = 0;
    int2 rr = rng[0];
    int off = g;   // this lane's position in row k, in quads
    while (off >= rr.y - rr.x && k + 1 < NR) {
        off -= max(rr.y - rr.x, 0);
        ++k;
        rr = rng[k * STRIDE];
    }
    if (off >= rr.y - rr.x) return;   // the rows hold no more than g quads
    const float4 *r = c.squad + (size_t)(rr.x + off) * 4;
    float4 X = r[0], Y = r[1];
    float4 Z = (DIM == 3) ? r[2] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (;;) {
        const float4 cX = X, cY = Y, cZ = Z;
        const float4 *rc = r;
        off += G;
        while (off >= rr.y - rr.x && k + 1 < NR) {
            off -= max(rr.y - rr.x, 0);
            ++k;
            rr = rng[k * STRIDE];
        }
        const bool more = off < rr.y - rr.x;
        if (more) {
            r = c.squad + (size_t)(rr.x + off) * 4;
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

// Merge the top-4 lists of the G lanes of a query (butterfly within the group
// of G consecutive lanes; every lane ends with the merged list).
template <int G>
__device__ __forceinline__ void group_merge_top4(Top4 &t)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = (G == 32) ? kFull : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const float e0 = __shfl_xor_sync(gmask, t.d0, o), e1 = __shfl_xor_sync(gmask, t.d1, o),
                    e2 = __shfl_xor_sync(gmask, t.d2, o), e3 = __shfl_xor_sync(gmask, t.d3, o);
        const int k0 = __shfl_xor_sync(gmask, t.j0, o), k1 = __shfl_xor_sync(gmask, t.j1, o),
                  k2 = __shfl_xor_sync(gmask, t.j2, o), k3 = __shfl_xor_sync(gmask, t.j3, o);
        if (k0 != 0x7fffffff) top4_insert(t, e0, k0);
        if (k1 != 0x7fffffff) top4_insert(t, e1, k1);
        if (k2 != 0x7fffffff) top4_insert(t, e2, k2);
        if (k3 != 0x7fffffff) top4_insert(t, e3, k3);
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
    // the end of the scene's last bucket is the end of the scene: a fused step
    // writes only its own scene's bucket starts
    const int end = c.pt_off + c.n;
    if (b0 + len < c.T) {
        lo = c.bstart[c.boff + b0];
        hi = c.bstart[c.boff + b0 + len];
    } else if (b0 + len == c.T) {
        lo = c.bstart[c.boff + b0];
        hi = end;
    } else {
        lo = c.bstart[c.boff + b0];
        hi = end;
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
//
// With G > 1, G consecutive lanes search the same query: each fills the rows
// k = g, g + G, ... of the query's row table (one shared column per group),
// walks its share of the quads, and the lanes merge their lists; the
// enclosure test and any growth then run identically in every lane of the
// group, so all of them return the same certificate.
template <int DIM, int STRIDE = kThreads, int MAXROWS = kMaxRows, int G = 1>
__device__ __forceinline__ bool grid_search(const SearchCtx &c, Top4 &t, float &Lout, int2 *rng, float hint,
                                            int g = 0)
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
        if ((y1 - y0 + 1) * (z1 - z0 + 1) <= MAXROWS) {
            if (g == 0) rng[0] = make_int2(0, 0);      // the own row's entry, filled in the loop (lane 0)
            nrows = 1;
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y) {
                    const int k = (y == cy && z == cz) ? 0 : nrows++;
                    if (G > 1 && k % G != g) continue;   // another lane of the group fills this row
                    int lo, hi, lo2, hi2;
                    row_ranges<DIM>(c, y, z, x0, x1, lo, hi, lo2, hi2);
                    if (hi2 > lo2) visit_range<DIM>(c, lo2, hi2, t);   // wrapped row: rare
                    lo = max(lo, c.pt_off);
                    hi = min(hi, c.pt_off + c.n);
                    rng[k * STRIDE] = (lo < hi) ? make_int2((lo + c.pad) >> 2, (hi + c.pad + 3) >> 2)
                                                  : make_int2(0, 0);
                }
        }
    }
    if (nrows == 0) {
        // no usable hint: the 3^d block of Algorithm 1
        constexpr int NR = (DIM == 3) ? 9 : 3;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            if (G > 1 && k % G != g) continue;   // another lane of the group fills this row
            const int kr = (k + NR / 2) % NR;   // the query's own row first
            const int yr = cy + (kr % 3) - 1;
            const int zr = (DIM == 3) ? cz + (kr / 3) - 1 : 0;
            int lo, hi, lo2, hi2;
            row_ranges<DIM>(c, yr, zr, cx - 1, cx + 1, lo, hi, lo2, hi2);
            if (hi2 > lo2) visit_range<DIM>(c, lo2, hi2, t);   // wrapped row: rare
            lo = max(lo, c.pt_off);
            hi = min(hi, c.pt_off + c.n);
            rng[k * STRIDE] = (lo < hi) ? make_int2((lo + c.pad) >> 2, (hi + c.pad + 3) >> 2) : make_int2(0, 0);
        }
        nrows = NR;
        x0 = max(cx - 1, 0);
        x1 = min(cx + 1, gm);
        y0 = max(cy - 1, 0);
        y1 = min(cy + 1, gm);
        z0 = (DIM == 3) ? max(cz - 1, 0) : 0;
        z1 = (DIM == 3) ? min(cz + 1, gm) : 0;
    }
    if (G == 1) {
        visit_quad_rows<DIM, STRIDE>(c, rng, nrows, t);
    } else {
        const unsigned lane = threadIdx.x & 31u;
        __syncwarp(((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));   // the group's row table is complete
        visit_quad_rows_split<DIM, STRIDE, G>(c, rng, nrows, t, g);
        group_merge_top4<G>(t);
    }

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
// hist_add(cell) adds one failure to the scene's entropy-cell histogram and
// returns the cell's previous count (a global or a shared-memory histogram).
struct SearchOut {
    int changed, missed, first, hit;
    double dl;
};

// With ACCOUNT false the caller sums the histogram itself afterwards: the
// failure is still added to it, but first and dl are left 0.
template <bool ACCOUNT = true, typename HistAdd>
__device__ __forceinline__ SearchOut write_certificate(const StepArgs &a, const SceneParams &sp, int gi,
                                                       const Top4 &t, float L, HistAdd hist_add)
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
            const int old = hist_add(a.hcell[gi]);
            if (ACCOUNT) {
                o.first = old == 0;
                o.dl = nlogn_step(a.nlogn, old);
            }
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

}  // namespace certk
