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
//                      safe certificates from the extended certificate
//   k_search           grid repair of the flagged points: top-2 over the 3^d
//                      block, widened until the runner-up is enclosed (Alg. 1
//                      block loop; Cor. A.2 widening)
//   k_finalize         per scene: H(F_t) (Def. 2), audit counts, next grid
//
// Extended certificate (an addition to the paper's record, needed because the
// paper leaves d1, d2 of safe points stale while every certificate here is
// exact each step): besides (nn, d1^2, d2^2) each point keeps its runner-up
// index nn2 and a lower bound L on the distance to every point other than nn
// and nn2.  A step moves any pair apart or together by at most 2 eps_t
// (triangle inequality, as in Lemma 1), so L - 2 eps_t bounds the next step;
// when both fresh distances to nn and nn2 stay below it the top-2 is exactly
// {nn, nn2} in fresh order, otherwise the point is repaired by a search.
#include "cert_internal.cuh"
#include "cert_launch.h"

namespace certk {

// ============================================================================ k_prepare

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_prepare(const StepArgs a)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const bool valid = i < a.n_total;
    int s = -1;
    unsigned dbits = 0u;
    int first = 0;
    if (valid) {
        s = a.scene_of[i];
        const SceneParams sp = a.sp[s];
        float4 p;
        if (a.mode == MODE_REBUILD) {
            p = a.pos_new[i];
        } else {
            const float *q = a.pos_in + (size_t)i * DIM;
            p.x = q[0];
            p.y = q[1];
            p.z = (DIM == 3) ? q[2] : 0.0f;
            p.w = 0.0f;
            if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) atomicOr(a.status, ST_NONFINITE);
            a.pos_new[i] = p;
            if (a.mode == MODE_STEP) {
                const float D = sqdist<DIM>(a.pos_old[i], p);
                dbits = (D >= 0.0f) ? __float_as_uint(D) : 0u;
            }
        }
        // hashed search grid: bucket of the cell, rank inside the bucket
        const int g = a.st[s].g_cur;
        const float gf = (float)g;
        const int cx = cell_coord(p.x, g, gf);
        const int cy = cell_coord(p.y, g, gf);
        const int cz = (DIM == 3) ? cell_coord(p.z, g, gf) : 0;
        const int b = sp.bucket_off + (int)((row_hash<DIM>(cy, cz) + (uint32_t)cx) & (uint32_t)sp.bucket_mask);
        const int rank = atomicAdd(&a.bucket_count[b], 1);
        a.brank[i] = make_int2(b, rank);
        // entropy grid on the post-step position (Def. 2)
        if (a.mode != MODE_REBUILD) {
            const int gh = sp.g_h;
            const float ghf = (float)gh;
            const int hx = cell_coord(p.x, gh, ghf);
            const int hy = cell_coord(p.y, gh, ghf);
            const int hc = (DIM == 3) ? (cell_coord(p.z, gh, ghf) * gh + hy) * gh + hx : hy * gh + hx;
            a.hcell[i] = hc;
            first = atomicAdd(&a.hocc[sp.h_off + hc], 1) == 0;
        }
    }
    const unsigned m = scene_run_mask(s);
    const unsigned mx = run_max_u32(m, dbits);
    const int occ = run_sum_i32(m, first);
    if (s >= 0 && run_leader(m)) {
        if (mx) atomicMax(&a.acc[s].eps_bits, mx);
        if (occ) atomicAdd(&a.acc[s].occ, occ);
    }
}

// ============================================================================ k_scan

// Publish this tile's aggregate and look back over predecessors for the
// exclusive prefix (single-pass chained scan).  Called by warp 0 only.  Every
// wait is bounded; on expiry the status word records a timeout and the
// (incorrect) partial prefix is used so that the kernel still terminates.
__device__ uint32_t lookback(uint64_t *tstat, int tile, uint32_t aggregate, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release_u64(&tstat[0], (2ull << 32) | aggregate);
        return 0u;
    }
    if (lane == 0) st_release_u64(&tstat[tile], (1ull << 32) | aggregate);
    uint32_t excl = 0u;
    int p = tile - 1;
    uint32_t spins = 0u;
    for (;;) {
        const int idx = p - lane;
        const uint64_t v = (idx >= 0) ? ld_acquire_u64(&tstat[idx]) : (2ull << 32);
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
    if (lane == 0) st_release_u64(&tstat[tile], (2ull << 32) | (excl + aggregate));
    return excl;
}

template <int DIM>
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
        const int4 c0 = *reinterpret_cast<const int4 *>(a.bucket_count + base);
        const int4 c1 = *reinterpret_cast<const int4 *>(a.bucket_count + base + 4);
        const uint32_t v[8] = {(uint32_t)c0.x, (uint32_t)c0.y, (uint32_t)c0.z, (uint32_t)c0.w,
                               (uint32_t)c1.x, (uint32_t)c1.y, (uint32_t)c1.z, (uint32_t)c1.w};
        uint32_t sum = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += v[k];
        uint32_t tot;
        const uint32_t pre = block_exclusive_scan(sum, &tot, s_warp);
        if (threadIdx.x < 32) {
            const uint32_t ex = lookback(a.tstat_b, t, tot, a.status);
            if (threadIdx.x == 0) s_excl = ex;
        }
        __syncthreads();
        uint32_t run = s_excl + pre;
        int o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            o[k] = (int)run;
            run += v[k];
        }
        *reinterpret_cast<int4 *>(a.bucket_start + base) = make_int4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<int4 *>(a.bucket_start + base + 4) = make_int4(o[4], o[5], o[6], o[7]);
        return;
    }

    // ---- frontier flags -> ascending frontier list (Algorithm 1, Lemma 1)
    const int tp = t - a.ntiles_b;
    const int base = tp * kScanTile + threadIdx.x * kScanItems;
    uint32_t f[8];
    int sc[8];
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = base + k;
        f[k] = 0u;
        sc[k] = -1;
        if (i < a.n_total) {
            const int s = a.scene_of[i];
            sc[k] = s;
            const float eps = eps_of(a.acc, s);
            const float d1 = __fsqrt_rn(a.d1sq[i]);
            const float d2 = __fsqrt_rn(a.d2sq[i]);
            const float c = __fsub_rn(d2, d1);
            const float tau = __fmul_rn(0x1p-20f, __fadd_rn(__fadd_rn(d1, d2), eps));
            const float rhs = __fadd_rn(__fmul_rn(4.0f, eps), tau);
            f[k] = (c <= rhs) ? 1u : 0u;
            a.inF[i] = (uint8_t)f[k];
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
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = base + k;
        const int s = sc[k];
        int first = 0;
        double dl = 0.0;
        if (s >= 0) {
            const SceneParams &sp = a.sp[s];
            if (i == sp.pt_off) a.fstart[s] = (int)run;
            if (f[k]) {
                if (run < (uint32_t)a.n_total) a.frontier[run] = i - sp.pt_off;
                const int old = atomicAdd(&a.hcand[sp.h_off + a.hcell[i]], 1);
                first = old == 0;
                dl = nlogn_step(a.nlogn, old);
            }
            if (i == a.n_total - 1) a.fstart[a.n_scenes] = (int)(run + f[k]);
        }
        run += f[k];
        const unsigned m = scene_run_mask(s);
        const int fc = run_sum_i32(m, first);
        const double sd = run_sum_f64(m, dl);
        if (s >= 0 && run_leader(m)) {
            if (fc) atomicAdd(&a.acc[s].frontier_cells, fc);
            if (sd != 0.0) atomicAdd(&a.acc[s].s_front, sd);
        }
    }
}

// ============================================================================ k_select

__device__ void bitonic_sort_1024(uint32_t *v)
{
    for (int k = 2; k <= kMedianSample; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int idx = threadIdx.x; idx < kMedianSample; idx += kThreads) {
                const int ixj = idx ^ j;
                if (ixj > idx) {
                    const uint32_t x = v[idx], y = v[ixj];
                    const bool up = (idx & k) == 0;
                    if ((x > y) == up) {
                        v[idx] = y;
                        v[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_select(const StepArgs a)
{
    __shared__ uint32_t s_c[kMedianSample];
    __shared__ uint32_t s_d[kMedianSample];
    __shared__ float s_feat[8];
    __shared__ float s_h1[64];
    __shared__ float s_h2[64];
    __shared__ float s_out[4];
    const int s = blockIdx.x;
    const SceneParams sp = a.sp[s];
    const int ns = min(sp.n, kMedianSample);
    for (int k = threadIdx.x; k < kMedianSample; k += kThreads) {
        uint32_t cb = 0x7f800000u, db = 0x7f800000u;
        if (k < ns) {
            const int i = sp.pt_off + k;
            const float d1 = __fsqrt_rn(a.d1sq[i]);
            const float d2 = __fsqrt_rn(a.d2sq[i]);
            cb = __float_as_uint(__fsub_rn(d2, d1));
            db = __float_as_uint(d2);
        }
        s_c[k] = cb;
        s_d[k] = db;
    }
    __syncthreads();
    bitonic_sort_1024(s_c);
    bitonic_sort_1024(s_d);
    const float med_c = __uint_as_float(s_c[(ns - 1) / 2] & 0xFFF00000u);
    const float med_d2 = __uint_as_float(s_d[(ns - 1) / 2] & 0xFFF00000u);

    int strat = STRAT_INC;
    if (a.mode == MODE_STEP) {
        strat = a.strategy;
        if (strat == STRAT_AUTO) strat = a.policy;
        if (a.strategy == STRAT_AUTO && a.sel_params != nullptr) {
            // ---- learned selector: 8 features -> MLP 8-64-64-2 -> argmin
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
                x[0] = (float)nF / (float)sp.n;
                x[1] = (float)Hc;
                x[2] = logf((float)sp.n);
                x[3] = (float)DIM;
                x[4] = log1pf(fminf(eps / fmaxf(med_c, 1e-30f), 1e6f));
                x[5] = acc.occ > 0 ? (float)acc.frontier_cells / (float)acc.occ : 0.0f;
                x[6] = st.prev_fail_ratio;
                x[7] = st.prev_pred_ratio;
                for (int k = 0; k < 8; ++k) s_feat[k] = (x[k] - a.sel_norm[k]) * a.sel_norm[8 + k];
            }
            __syncthreads();
            const float *W1 = a.sel_params, *b1 = W1 + 64 * 8, *W2 = b1 + 64, *b2 = W2 + 64 * 64,
                        *W3 = b2 + 64, *b3 = W3 + 2 * 64;
            if (threadIdx.x < 64) {
                float z = b1[threadIdx.x];
                for (int k = 0; k < 8; ++k) z = fmaf(W1[threadIdx.x * 8 + k], s_feat[k], z);
                s_h1[threadIdx.x] = fmaxf(z, 0.0f);
            }
            __syncthreads();
            if (threadIdx.x < 64) {
                float z = b2[threadIdx.x];
                for (int k = 0; k < 64; ++k) z = fmaf(W2[threadIdx.x * 64 + k], s_h1[k], z);
                s_h2[threadIdx.x] = fmaxf(z, 0.0f);
            }
            __syncthreads();
            if (threadIdx.x < 64) {
                float y0 = W3[threadIdx.x] * s_h2[threadIdx.x];
                float y1 = W3[64 + threadIdx.x] * s_h2[threadIdx.x];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    y0 += __shfl_xor_sync(kFull, y0, o);
                    y1 += __shfl_xor_sync(kFull, y1, o);
                }
                if ((threadIdx.x & 31) == 0) {
                    s_out[threadIdx.x >> 5] = y0;     // partial sums of the two warps
                    s_out[2 + (threadIdx.x >> 5)] = y1;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const float pi = s_out[0] + s_out[1] + b3[0];
                const float pr = s_out[2] + s_out[3] + b3[1];
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

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_scatter_refresh(const StepArgs a)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const bool valid = i < a.n_total;
    int s = -1, changed = 0, first = 0;
    double dl = 0.0;
    if (valid) {
        s = a.scene_of[i];
        const SceneParams sp = a.sp[s];
        const int2 br = a.brank[i];
        int slot = a.bucket_start[br.x] + br.y;
        if ((unsigned)slot >= (unsigned)a.n_total) {  // only after a timed-out scan
            atomicOr(a.status, ST_TIMEOUT);
            slot = i;
        }
        const float4 p = a.pos_new[i];
        a.sorted[slot] = make_float4(p.x, p.y, p.z, __int_as_float(i));
        bool need = true;
        if (a.mode == MODE_STEP && a.st[s].strategy == STRAT_INC && !a.inF[i]) {
            const int na = a.nn[i], nb = a.nn2[i];
            if ((unsigned)na < (unsigned)sp.n && (unsigned)nb < (unsigned)sp.n) {
                const float Da = sqdist<DIM>(p, a.pos_new[sp.pt_off + na]);
                const float Db = sqdist<DIM>(p, a.pos_new[sp.pt_off + nb]);
                const float two_eps_up = __fmul_ru(eps_of(a.acc, s), 2.0f + 0x1p-18f);
                const float Lnew = __fsub_rd(a.L[i], two_eps_up);
                if (Lnew > 0.0f && __fmul_ru(fmaxf(Da, Db), 1.0f + 0x1p-19f) < __fmul_rd(Lnew, Lnew)) {
                    need = false;
                    const bool sw = key_less(Db, nb, Da, na);
                    const int n1 = sw ? nb : na, n2 = sw ? na : nb;
                    a.nn[i] = n1;
                    a.nn2[i] = n2;
                    a.d1sq[i] = sw ? Db : Da;
                    a.d2sq[i] = sw ? Da : Db;
                    a.L[i] = Lnew;
                    changed = n1 != na;
                    a.failed[i] = (uint8_t)changed;
                    if (changed) {
                        const int old = atomicAdd(&a.hfail[sp.h_off + a.hcell[i]], 1);
                        first = old == 0;
                        dl = nlogn_step(a.nlogn, old);
                    }
                }
            }
        }
        a.sflag[slot] = need ? 1 : 0;
    }
    if (a.mode != MODE_STEP) return;  // uniform across the grid
    const unsigned m = scene_run_mask(s);
    const int nc = run_sum_i32(m, changed);
    const int fc = run_sum_i32(m, first);
    const double sd = run_sum_f64(m, dl);
    if (s >= 0 && run_leader(m) && nc) {
        // refreshed points are never in F, so each change here is also a miss
        atomicAdd(&a.acc[s].n_failed, nc);
        atomicAdd(&a.acc[s].n_missed, nc);
        atomicAdd(&a.acc[s].failed_cells, fc);
        atomicAdd(&a.acc[s].s_fail, sd);
    }
}

// ============================================================================ k_search

struct SearchCtx {
    const float4 *sorted;
    const int *bstart;
    float4 p;
    int gi;
    int pt_off, n, boff, T;
    uint32_t mask;
    int g;
};

template <int DIM>
__device__ __forceinline__ void visit_range(const SearchCtx &c, int lo, int hi, Top3 &t)
{
    lo = max(lo, c.pt_off);          // a bucket range never leaves its scene
    hi = min(hi, c.pt_off + c.n);
    for (int k = lo; k < hi; ++k) {
        const float4 q = c.sorted[k];
        const int j = __float_as_int(q.w);
        const float D = sqdist<DIM>(c.p, q);
        if (D <= t.d2 && j != c.gi) top3_insert(t, D, j);
    }
}

template <int DIM>
__device__ __forceinline__ void visit_row(const SearchCtx &c, int yr, int zr, int xl, int xh, Top3 &t)
{
    xl = max(xl, 0);
    xh = min(xh, c.g - 1);
    if (xl > xh) return;
    const int len = xh - xl + 1;
    if (len >= c.T) {
        visit_range<DIM>(c, c.pt_off, c.pt_off + c.n, t);
        return;
    }
    const int b0 = (int)((row_hash<DIM>(yr, zr) + (uint32_t)xl) & c.mask);
    if (b0 + len <= c.T) {
        visit_range<DIM>(c, c.bstart[c.boff + b0], c.bstart[c.boff + b0 + len], t);
    } else {
        visit_range<DIM>(c, c.bstart[c.boff + b0], c.bstart[c.boff + c.T], t);
        visit_range<DIM>(c, c.bstart[c.boff], c.bstart[c.boff + b0 + len - c.T], t);
    }
}

// Lower bound on the distance from p to any point outside the block of cells
// [c - r, c + r]^dim; +inf when every face of the block lies on the grid edge
// (boundary cells are clamped and so extend to infinity).
template <int DIM>
__device__ __forceinline__ float face_distance(const float4 p, int cx, int cy, int cz, int r, int g, float inv_g)
{
    float f = __int_as_float(0x7f800000);
    const int c3[3] = {cx, cy, cz};
    const float p3[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        if (c3[ax] - r > 0) f = fminf(f, __fsub_rn(p3[ax], __fmul_rn((float)(c3[ax] - r), inv_g)));
        if (c3[ax] + r < g - 1) f = fminf(f, __fsub_rn(__fmul_rn((float)(c3[ax] + r + 1), inv_g), p3[ax]));
    }
    return f;
}

constexpr float kFaceSlack = 0x1p-17f;   // >> FP error of cell assignment and face position

template <int DIM>
__device__ __forceinline__ void grid_search(const SearchCtx &c, Top3 &t, float &Lout)
{
    const float gf = (float)c.g;
    const float inv_g = __frcp_rn(gf);
    const int cx = cell_coord(c.p.x, c.g, gf);
    const int cy = cell_coord(c.p.y, c.g, gf);
    const int cz = (DIM == 3) ? cell_coord(c.p.z, c.g, gf) : 0;
    top3_reset(t);
    // ring 1: the 3^d block of Algorithm 1
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
        const int zr = cz + dz;
        if (zr < 0 || zr >= c.g) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yr = cy + dy;
            if (yr < 0 || yr >= c.g) continue;
            visit_row<DIM>(c, yr, zr, cx - 1, cx + 1, t);
        }
    }
    int r = 1;
    for (;;) {
        const float f0 = face_distance<DIM>(c.p, cx, cy, cz, r, c.g, inv_g);
        if (isinf(f0)) {  // the block covers the whole grid: everything was visited
            Lout = sqrt_lower(t.d2);
            return;
        }
        const float f = __fsub_rd(f0, kFaceSlack);
        if (t.j1 != 0x7fffffff && f > 0.0f &&
            __fmul_ru(t.d1, 1.0f + 0x1p-19f) < __fmul_rd(f, f)) {  // runner-up provably enclosed
            Lout = fminf(sqrt_lower(t.d2), f);
            return;
        }
        ++r;
        if (r > kWidenCap) {  // far from everything: scan the scene linearly
            visit_range<DIM>(c, c.pt_off, c.pt_off + c.n, t);
            Lout = sqrt_lower(t.d2);
            return;
        }
        // shell at Chebyshev radius r
        for (int dz = (DIM == 3 ? -r : 0); dz <= (DIM == 3 ? r : 0); ++dz) {
            const int zr = cz + dz;
            if (zr < 0 || zr >= c.g) continue;
            for (int dy = -r; dy <= r; ++dy) {
                const int yr = cy + dy;
                if (yr < 0 || yr >= c.g) continue;
                if (max(abs(dy), abs(dz)) == r) {
                    visit_row<DIM>(c, yr, zr, cx - r, cx + r, t);
                } else {
                    visit_row<DIM>(c, yr, zr, cx - r, cx - r, t);
                    visit_row<DIM>(c, yr, zr, cx + r, cx + r, t);
                }
            }
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_search(const StepArgs a)
{
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ int s_list[kSearchChunk];
    const int my = blockIdx.x * kSearchChunk + threadIdx.x;
    const uint32_t f = (my < a.n_total) ? (uint32_t)a.sflag[my] : 0u;
    uint32_t count;
    const uint32_t pre = block_exclusive_scan(f, &count, s_warp);
    if (f) s_list[pre] = my;
    __syncthreads();
    if ((int)(threadIdx.x & ~31u) >= (int)count) return;  // whole idle warps leave together
    const bool active = threadIdx.x < count;
    int s = -1, changed = 0, missed = 0, first = 0;
    double dl = 0.0;
    if (active) {
        const int slot = s_list[threadIdx.x];
        const float4 q = a.sorted[slot];
        int gi = __float_as_int(q.w);
        if ((unsigned)gi >= (unsigned)a.n_total) {  // only after a timed-out scan
            atomicOr(a.status, ST_TIMEOUT);
            gi = slot;
        }
        s = a.scene_of[gi];
        const SceneParams sp = a.sp[s];
        SearchCtx c;
        c.sorted = a.sorted;
        c.bstart = a.bucket_start;
        c.p = q;
        c.gi = gi;
        c.pt_off = sp.pt_off;
        c.n = sp.n;
        c.boff = sp.bucket_off;
        c.T = sp.bucket_mask + 1;
        c.mask = (uint32_t)sp.bucket_mask;
        c.g = a.st[s].g_cur;
        Top3 t;
        float L;
        grid_search<DIM>(c, t, L);
        const int n1 = (t.j0 != 0x7fffffff) ? t.j0 - sp.pt_off : -1;
        const int n2 = (t.j1 != 0x7fffffff) ? t.j1 - sp.pt_off : -1;
        if (a.mode == MODE_STEP) {
            changed = n1 != a.nn[gi];
            a.failed[gi] = (uint8_t)changed;
            if (changed) {
                missed = !a.inF[gi];
                const int old = atomicAdd(&a.hfail[sp.h_off + a.hcell[gi]], 1);
                first = old == 0;
                dl = nlogn_step(a.nlogn, old);
            }
        }
        a.nn[gi] = n1;
        a.nn2[gi] = n2;
        a.d1sq[gi] = t.d0;
        a.d2sq[gi] = t.d1;
        a.L[gi] = L;
    }
    if (a.mode != MODE_STEP) return;
    // slots of one scene are contiguous, so lanes form contiguous scene runs
    const unsigned m = scene_run_mask(s);
    const int nsr = run_sum_i32(m, active ? 1 : 0);
    const int nc = run_sum_i32(m, changed);
    const int nm = run_sum_i32(m, missed);
    const int fc = run_sum_i32(m, first);
    const double sd = run_sum_f64(m, dl);
    if (s >= 0 && run_leader(m)) {
        atomicAdd(&a.acc[s].n_searched, nsr);
        if (nc) {
            atomicAdd(&a.acc[s].n_failed, nc);
            atomicAdd(&a.acc[s].n_missed, nm);
            atomicAdd(&a.acc[s].failed_cells, fc);
            atomicAdd(&a.acc[s].s_fail, sd);
        }
    }
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
        a.res[s] = r;
        if (r.eps_t > __fmul_ru(a.declared_eps, 1.0f + 0x1p-20f)) atomicOr(a.status, ST_EBOUND);
        st.prev_fail_ratio = (float)acc.n_failed / (float)max(1, nF);
        st.prev_nfront = nF;
    }
    st.g_cur = st.g_next;
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
    case PH_PREPARE: k_prepare<DIM><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(a); break;
    case PH_SCAN: k_scan<DIM><<<a.ntiles_b + a.ntiles_p, kThreads, 0, st>>>(a); break;
    case PH_SELECT: k_select<DIM><<<a.n_scenes, kThreads, 0, st>>>(a); break;
    case PH_SCATTER: k_scatter_refresh<DIM><<<nblk(a.n_total, kThreads), kThreads, 0, st>>>(a); break;
    case PH_SEARCH: k_search<DIM><<<nblk(a.n_total, kSearchChunk), kThreads, 0, st>>>(a); break;
    case PH_FINALIZE: k_finalize<<<nblk(a.n_scenes, 128), 128, 0, st>>>(a); break;
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
