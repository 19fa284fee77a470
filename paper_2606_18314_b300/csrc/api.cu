// api.cu -- host implementation of the C ABI declared in include/cert.h.
//
// A context owns one device allocation carved into every buffer a batch of
// scenes needs; cert_init sizes it from the scene offsets and nothing is
// allocated afterwards (cert_allpairs, which has no context, uses the
// stream-ordered allocator).  Every call only enqueues work on the caller's
// stream, except cert_sync_result / cert_step_host / cert_destroy, which wait.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cert_internal.cuh"
#include "cert_launch.h"

using namespace certk;

struct cert_ctx {
    int dim = 0, S = 0;
    int64_t N = 0;
    float cell_scale = 3.5f;
    float cell_quantile = 0.5f;
    int bucket_factor = 1;
    int policy = STRAT_INC;
    int frontier_rule = CERT_FRONTIER_STEP;
    int audit = 0;
    double *clk_s = nullptr;       // cumulative-clock rule: S_i, c^rev_i, (d1 + d2)^rev_i per point
    float *clk_c = nullptr, *clk_g = nullptr;
    std::vector<SceneParams> h_sp;
    int n_buckets = 0, n_buckets_pad = 0, ntiles_b = 0, ntiles_p = 0;
    int64_t n_h = 0, ap_P = 0;
    int n_ap_items = 0;
    char *blob = nullptr;
    size_t blob_bytes = 0;
    // persistent buffers
    SceneParams *sp = nullptr;
    SceneState *st = nullptr;
    cert_scene_result *res = nullptr;
    uint32_t *status = nullptr;
    int32_t *fstart = nullptr, *scene_of = nullptr;
    float4 *pos[2] = {nullptr, nullptr};
    int cur = 0;
    int32_t *nn = nullptr, *nn2 = nullptr, *nn3 = nullptr;
    float *d1sq = nullptr, *d2sq = nullptr, *L = nullptr;
    int32_t *hcell = nullptr, *frontier = nullptr;
    uint8_t *inF = nullptr, *failed = nullptr, *sflag = nullptr;
    int2 *brank = nullptr;
    float4 *squad = nullptr;
    int64_t n_quads = 0;
    int32_t *bucket_start = nullptr;
    int32_t *far_list = nullptr, *far_count = nullptr;
    double *nlogn = nullptr;
    float *stage = nullptr;
    APItem *ap_items = nullptr;
    float *ap_pd = nullptr;
    int32_t *ap_pj = nullptr;
    float *sel_params = nullptr, *sel_norm = nullptr;
    bool have_sel = false;
    int32_t *scene_policy = nullptr;   // [S] per-scene policy under AUTO without a selector
    bool have_scene_policy = false;
    float *feat = nullptr;          // [S][8] selector features of the last step
    // snapshot of the mutable state (allocated by the first cert_snapshot)
    char *snap = nullptr;
    // pipelined host steps: a second staging buffer, a copy stream and events (created on first use);
    // each buffer parity's steps write their scalars to their own slot of res_ring, which a second
    // copy stream moves to the host while the next step runs
    float *stage2 = nullptr;
    cudaStream_t copy_stream = nullptr, d2h_stream = nullptr;
    cert_scene_result *res_ring = nullptr;    // [2][S]
    cert_scene_result *res_target = nullptr;  // where k_finalize writes (nullptr: res)
    cudaEvent_t ev_d2h[2] = {nullptr, nullptr};
    // one-step CUDA graphs replayed by the pipelined host steps, one per
    // (position buffer, staging buffer) parity; rebuilt when eps, the strategy
    // or a setting baked into the step arguments changes
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        float eps = 0.0f;
        int strategy = -1;
        uint64_t epoch = 0;
    } step_graph[4];
    cudaStream_t capture_stream = nullptr;
    uint64_t settings_epoch = 1;
    // fused step (one launch per step): eligibility, the path setting, the CTA order (largest scene first)
    bool fused_ok = false;
    int step_path = CERT_PATH_AUTO;
    int max_n = 0, max_T = 0;
    bool c16b = false, c16h = false;   // 16-bit bucket counts; 16-bit entropy-cell counts
    int32_t *order = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    size_t snap_bytes = 0;
    int snap_cur = 0;
    bool snap_valid = false;
    // Counters and accumulators the pipeline's kernels add into.  Zero at the
    // start of every multi-kernel step: the step's own kernels zero each one
    // once it is dead (StepArgs::ztail), the fused step leaves them untouched,
    // and zero_dirty (set by a CUDA error, which may have cut a step short)
    // makes the next step memset them first.
    char *zero = nullptr;
    size_t zero_bytes = 0, ztail_off = 0;
    bool zero_dirty = true;
    SceneAcc *acc = nullptr;
    uint32_t *tile_ctr = nullptr;
    uint64_t *tstat_b = nullptr, *tstat_p = nullptr;
    int32_t *bucket_count = nullptr, *hfail = nullptr, *hcand = nullptr;
    uint32_t *hocc = nullptr;   // one bit per entropy cell: occupied
    uint32_t *mgrid = nullptr, *mdil = nullptr;   // motion grid (k_search zeroes it once dilated) and its dilation
    int32_t *chunk_cnt = nullptr, *chunk_order = nullptr;   // batch search: chunk weights and dispatch order
    cudaStream_t last = nullptr;
    bool stepped = false;
    // phase profiling (diagnostics)
    std::vector<cudaEvent_t> prof_ev;
    int prof_max = 0, prof_n = 0;
    bool prof_on = false;
    std::string err;
};

static thread_local std::string g_err;

static cert_status fail(cert_ctx *ctx, cert_status code, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    g_err = msg;
    return code;
}

// Lets other translation units of the library set the calling thread's
// error text returned by cert_last_error(NULL).
namespace certk {
void record_thread_error(const char *msg) { g_err = msg; }
}  // namespace certk

static cert_status cuda_fail(cert_ctx *ctx, const char *what, cudaError_t e)
{
    if (ctx) {   // a step may have stopped short of the kernels that zero the counters
        ctx->zero_dirty = true;
        ++ctx->settings_epoch;   // and cached step graphs were captured without the memset
    }
    return fail(ctx, CERT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, call)                                               \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), #call, e_);  \
    } while (0)

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static int next_pow2(int64_t v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

static int entropy_res(int64_t n, int dim)
{
    int g = 1;
    for (;;) {
        int64_t p = 1;
        for (int a = 0; a < dim; ++a) p *= g;
        if (p >= n) return g;
        ++g;
    }
}

// Bump allocator over one device allocation (256-byte aligned pieces).
struct Carver {
    size_t off = 0;
    template <typename T>
    size_t take(int64_t count)
    {
        off = (off + 255) & ~size_t(255);
        const size_t at = off;
        off += size_t(count) * sizeof(T);
        return at;
    }
};

static StepArgs make_args(cert_ctx *c, int mode)
{
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.mode = mode;
    a.dim = c->dim;
    a.n_total = (int)c->N;
    a.n_scenes = c->S;
    a.scene_of = c->scene_of;
    a.sp = c->sp;
    a.st = c->st;
    a.acc = c->acc;
    a.status = c->status;
    a.bucket_count = c->bucket_count;
    a.mgrid = c->mgrid;
    a.chunk_cnt = c->chunk_cnt;
    a.chunk_order = c->chunk_order;
    a.mdil = c->mdil;
    a.bucket_start = c->bucket_start;
    a.brank = c->brank;
    a.squad = c->squad;
    a.sflag = c->sflag;
    a.far_list = c->far_list;
    a.far_count = c->far_count;
    a.nn = c->nn;
    a.nn2 = c->nn2;
    a.nn3 = c->nn3;
    a.d1sq = c->d1sq;
    a.d2sq = c->d2sq;
    a.L = c->L;
    a.hcell = c->hcell;
    a.hocc = c->hocc;
    a.hfail = c->hfail;
    a.hcand = c->hcand;
    a.c16b = c->c16b ? 1 : 0;
    a.c16h = c->c16h ? 1 : 0;
    a.inF = c->inF;
    a.failed = c->failed;
    a.frontier = c->frontier;
    a.fstart = c->fstart;
    a.tstat_b = c->tstat_b;
    a.tstat_p = c->tstat_p;
    a.ztail = reinterpret_cast<int4 *>(c->zero + c->ztail_off);
    a.ztail_n16 = (long long)((c->zero_bytes - c->ztail_off) / 16);
    a.tile_ctr = c->tile_ctr;
    a.ntiles_b = c->ntiles_b;
    a.ntiles_p = 0;
    a.nlogn = c->nlogn;
    a.res = c->res_target ? c->res_target : c->res;
    a.policy = c->policy;
    a.frontier_rule = c->frontier_rule;
    a.audit = c->audit;
    a.clk_s = c->clk_s;
    a.clk_c = c->clk_c;
    a.clk_g = c->clk_g;
    a.cell_scale = c->cell_scale;
    a.cell_quantile = c->cell_quantile;
    a.scene_policy = c->have_scene_policy ? c->scene_policy : nullptr;
    a.sel_params = c->have_sel ? c->sel_params : nullptr;
    a.sel_norm = c->have_sel ? c->sel_norm : nullptr;
    a.feat = c->feat;
    return a;
}

// The fused step (one launch per step, fused_step.cu) runs a step when every
// scene fits its limits, the strategy is not the all-pairs pass, and either it
// was asked for or, on CERT_PATH_AUTO, every scene is small enough to keep its
// sorted points in shared memory -- and either has at most kFusedAutoSingleN
// points or the batch holds at least kFusedAutoScenes scenes.  One CTA per
// scene makes the fused step as long as its largest scene's chain of dependent
// accesses on one SM, whatever the number of scenes up to one wave, while the
// multi-kernel step spreads every phase over the GPU and grows with the total.
// Measured (graph replay, mixed families, scenes log-uniform from 500 points):
// up to 1,000 or 2,000 points per scene the fused step is 0.53 to 1.01 of the
// multi-kernel step's time from 16 to 296 scenes; up to 4,000 points it is
// 1.32 to 1.60 with 16 to 64 scenes, 0.97 to 0.99 with 148 and 0.67 to 0.75
// with 296.  A lone scene crosses over between 2,000 and 4,000 points (d = 2:
// 0.033 vs 0.035 ms at 2,000, 0.056 vs 0.035 ms at 4,000; d = 3: 0.042 vs
// 0.039 and 0.060 vs 0.041 ms).  Larger scenes (N = 16,000, d = 3: 0.29 vs
// 0.044 ms per step; the 512-scene batch: 1.38 vs 0.65 ms) always take the
// multi-kernel step.
constexpr int kFusedAutoScenes = 148;   // one CTA per SM: a full wave of scenes
constexpr int kFusedAutoSingleN = 2560;
static bool fused_resident(const cert_ctx *c)
{
    return c->max_n <= kFusedResMaxN && c->max_T <= kFusedResMaxN;
}

static bool use_fused(const cert_ctx *c, int strategy)
{
    if (!c->fused_ok || strategy == STRAT_ALL || c->step_path == CERT_PATH_MULTI) return false;
    if (c->audit & CERT_AUDIT_COST) return false;   // the cost audit instruments the multi-kernel step
    if (c->step_path == CERT_PATH_FUSED) return true;
    return fused_resident(c) && (c->max_n <= kFusedAutoSingleN || c->S >= kFusedAutoScenes);
}

// CTA size of the fused step: 512 threads (two CTAs per SM) for batches that
// fill the GPU, 1024 for fewer scenes than SMs (more threads per scene).
static int fused_block(const cert_ctx *c) { return c->S >= 148 ? 512 : 1024; }

// Contexts of more than this many points keep 16-bit counts when their scenes
// allow it (cert_init).
constexpr int64_t kC16MinN = 262144;

// Grid build + full search of every point of the current positions
// (initial certificates and cert_rebuild).
static cert_status run_full(cert_ctx *c, int mode, const float *pos_in, cudaStream_t s)
{
    StepArgs a = make_args(c, mode);
    a.pos_in = pos_in;
    a.pos_new = c->pos[c->cur];
    CK(c, cudaMemsetAsync(c->zero, 0, c->zero_bytes, s));
    CK(c, launch_step_phase(a, PH_PREPARE, s));
    CK(c, launch_step_phase(a, PH_SCAN, s));
    CK(c, launch_step_phase(a, PH_SCATTER, s));
    CK(c, launch_step_phase(a, PH_SEARCH, s));
    CK(c, launch_step_phase(a, PH_SELECT, s));
    CK(c, launch_step_phase(a, PH_FINALIZE, s));
    c->zero_dirty = false;   // k_search, k_select and k_finalize zeroed what the kernels filled
    // clock rule: every certificate was just recomputed, so the next step's scan
    // revisits every point (resets S_i, c^rev_i and (d1 + d2)^rev_i)
    if (c->frontier_rule == CERT_FRONTIER_CLOCK) CK(c, cudaMemsetAsync(c->inF, 1, size_t(c->N), s));
    c->last = s;
    return CERT_OK;
}

extern "C" {

const char *cert_version(void) { return "certmaint-b300 0.2 (sm_103a)"; }

// The build passes each translation unit's source fingerprint (build.py).
#ifndef CERT_FP_STEP_KERNELS
#define CERT_FP_STEP_KERNELS "unknown"
#endif
#ifndef CERT_FP_ALLPAIRS
#define CERT_FP_ALLPAIRS "unknown"
#endif
#ifndef CERT_FP_KNN
#define CERT_FP_KNN "unknown"
#endif
#ifndef CERT_FP_MLP
#define CERT_FP_MLP "unknown"
#endif
#ifndef CERT_FP_API
#define CERT_FP_API "unknown"
#endif
#ifndef CERT_FP_ALLPAIRS_NOALLOC
#define CERT_FP_ALLPAIRS_NOALLOC "unknown"
#endif
#ifndef CERT_FP_FUSED_STEP
#define CERT_FP_FUSED_STEP "unknown"
#endif

const char *cert_source_fingerprint(const char *unit)
{
    if (!unit) return nullptr;
    static const struct {
        const char *name, *fp;
    } table[] = {{"step_kernels", CERT_FP_STEP_KERNELS}, {"allpairs", CERT_FP_ALLPAIRS},
                 {"knn", CERT_FP_KNN},                   {"mlp", CERT_FP_MLP},
                 {"api", CERT_FP_API},                   {"allpairs_noalloc", CERT_FP_ALLPAIRS_NOALLOC},
                 {"fused_step", CERT_FP_FUSED_STEP}};
    for (const auto &t : table)
        if (std::strcmp(unit, t.name) == 0) return t.fp;
    return nullptr;
}

const char *cert_last_error(const cert_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

cert_status cert_init(cert_ctx **out, const cert_config *cfg, const float *d_pos, void *stream)
{
    if (!out) return fail(nullptr, CERT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, CERT_EINVAL, "cfg is NULL");
    if (!d_pos) return fail(nullptr, CERT_EINVAL, "positions are NULL");
    if (cfg->dim != 2 && cfg->dim != 3) return fail(nullptr, CERT_EINVAL, "dim must be 2 or 3");
    if (cfg->n_scenes < 1) return fail(nullptr, CERT_EINVAL, "n_scenes must be >= 1");
    if (cfg->audit & ~(CERT_AUDIT_RHO | CERT_AUDIT_GEOMETRY | CERT_AUDIT_COST))
        return fail(nullptr, CERT_EINVAL, "unknown audit flag");
    if (cfg->frontier_rule < CERT_FRONTIER_STEP || cfg->frontier_rule > CERT_FRONTIER_CLOCK)
        return fail(nullptr, CERT_EINVAL, "unknown frontier_rule");
    if (cfg->bucket_factor != 0 && cfg->bucket_factor != 1 && cfg->bucket_factor != 2 && cfg->bucket_factor != 4 &&
        cfg->bucket_factor != 8)
        return fail(nullptr, CERT_EINVAL, "bucket_factor must be 0, 1, 2, 4 or 8");
    if (!(cfg->cell_quantile >= 0.0f && cfg->cell_quantile <= 1.0f))
        return fail(nullptr, CERT_EINVAL, "cell_quantile must be in [0, 1]");
    if (!(cfg->cell_scale >= 0.0f) || !std::isfinite(cfg->cell_scale))
        return fail(nullptr, CERT_EINVAL, "cell_scale must be finite and >= 0");
    if (cfg->policy < 0 || cfg->policy > STRAT_REB)
        return fail(nullptr, CERT_EINVAL, "policy must be AUTO, INCREMENTAL or REBUILD");
    std::vector<int64_t> off;
    if (cfg->offsets) {
        off.assign(cfg->offsets, cfg->offsets + cfg->n_scenes + 1);
    } else {
        if (cfg->n_scenes != 1) return fail(nullptr, CERT_EINVAL, "offsets required when n_scenes > 1");
        off = {0, cfg->n_total};
    }
    if (off[0] != 0) return fail(nullptr, CERT_EINVAL, "offsets[0] must be 0");
    for (int s = 0; s < cfg->n_scenes; ++s)
        if (off[s + 1] - off[s] < 3) return fail(nullptr, CERT_EINVAL, "every scene needs at least 3 points");
    if (off.back() >= (int64_t(1) << 31) - kScanTile) return fail(nullptr, CERT_EINVAL, "too many points");

    cert_ctx *c = new cert_ctx();
    c->dim = cfg->dim;
    c->S = cfg->n_scenes;
    c->N = off.back();
    c->cell_scale = cfg->cell_scale > 0.0f ? cfg->cell_scale : 3.5f;
    c->cell_quantile = cfg->cell_quantile > 0.0f ? cfg->cell_quantile : 0.5f;
    c->bucket_factor = cfg->bucket_factor > 0 ? cfg->bucket_factor : 1;
    c->policy = cfg->policy == STRAT_AUTO ? STRAT_INC : cfg->policy;
    c->frontier_rule = cfg->frontier_rule;
    c->audit = cfg->audit;
    cudaStream_t s = (cudaStream_t)stream;

    // ---- per-scene layout
    c->h_sp.resize(c->S);
    int64_t boff = 0, hoff = 0, apoff = 0, total_qb = 0, quads = 0;
    for (int k = 0; k < c->S; ++k) total_qb += ceil_div(off[k + 1] - off[k], kApQBlock);
    const int64_t nch_all = allpairs_chunks(total_qb, c->dim, 64);
    std::vector<APItem> items;
    for (int k = 0; k < c->S; ++k) {
        SceneParams &p = c->h_sp[k];
        std::memset(&p, 0, sizeof(p));
        const int64_t n = off[k + 1] - off[k];
        p.pt_off = (int32_t)off[k];
        p.n = (int32_t)n;
        p.s_off = (int32_t)(4 * quads);
        quads += ceil_div(n, 4);
        const int T = next_pow2(std::max<int64_t>(n, 16)) * c->bucket_factor;
        p.bucket_off = (int32_t)boff;
        p.bucket_mask = T - 1;
        boff += T;
        p.g_h = entropy_res(n, c->dim);
        p.h_off = (int32_t)hoff;   // a multiple of 8 (16-bit counts: 16-byte words of its own)
        hoff += ((int64_t)(std::pow((double)p.g_h, (double)c->dim) + 0.5) + 7) & ~int64_t(7);
        p.g_default = std::max(1, (int)std::floor(std::pow(n / 2.0, 1.0 / c->dim)));
        const int nch = (int)std::min<int64_t>(nch_all, ceil_div(n, 256));
        p.ap_nch = nch;
        p.ap_chunk = (int32_t)ceil_div(n, nch);
        p.ap_off = (int32_t)apoff;
        apoff += n * nch;
        const int nqb = (int)ceil_div(n, kApQBlock);
        for (int ch = 0; ch < nch; ++ch)
            for (int qb = 0; qb < nqb; ++qb) items.push_back({k, qb, ch, 0});
    }
    c->n_quads = quads;
    c->fused_ok = true;
    for (int k = 0; k < c->S; ++k) {
        const SceneParams &p = c->h_sp[k];
        const int64_t cells = (int64_t)std::pow((double)p.g_h, (double)c->dim) + 0.5;
        c->max_n = std::max(c->max_n, (int)p.n);
        c->max_T = std::max(c->max_T, (int)p.bucket_mask + 1);
        if (p.n > kFusedMaxN || p.bucket_mask + 1 > kFusedMaxBuckets || cells > kFusedMaxHCells) c->fused_ok = false;
    }
    // 16-bit counts (no scene reaches 65,536 points, so no count reaches 2^16)
    // for contexts of more than kC16MinN points, where the arrays' footprint
    // matters more than two counters sharing an atomic's word (measured: the
    // 512-scene batch 4.44e9 -> 4.48e9 point-updates/s; a lone scene of 16,000
    // points, whose atomics are its step's critical chain, 0.045 -> 0.047 ms)
    c->c16b = c->c16h = c->max_n < 65536 && c->N > kC16MinN;
    c->n_buckets = (int)boff;
    c->n_buckets_pad = (int)ceil_div(boff + 1, kScanTile) * kScanTile;
    c->ntiles_b = c->n_buckets_pad / kScanTile;
    c->ntiles_p = (int)ceil_div(c->N, kScanTile);
    c->n_h = hoff;
    c->ap_P = apoff;
    c->n_ap_items = (int)items.size();

    // ---- carve one allocation
    const int64_t N = c->N, S = c->S, Npad = ceil_div(N, kScanTile) * kScanTile;
    Carver cv;
    const size_t o_sp = cv.take<SceneParams>(S), o_st = cv.take<SceneState>(S),
                 o_res = cv.take<cert_scene_result>(S), o_status = cv.take<uint32_t>(4),
                 o_fstart = cv.take<int32_t>(S + 1), o_scene = cv.take<int32_t>(N),
                 o_pos0 = cv.take<float4>(N), o_pos1 = cv.take<float4>(N), o_nn = cv.take<int32_t>(N),
                 o_nn2 = cv.take<int32_t>(N), o_nn3 = cv.take<int32_t>(N), o_d1 = cv.take<float>(N), o_d2 = cv.take<float>(N),
                 o_L = cv.take<float>(N), o_hcell = cv.take<int32_t>(N), o_front = cv.take<int32_t>(N),
                 o_inF = cv.take<uint8_t>(Npad), o_failed = cv.take<uint8_t>(Npad),
                 o_sflag = cv.take<uint8_t>(Npad), o_brank = cv.take<int2>(N), o_sorted = cv.take<float4>(4 * c->n_quads),
                 o_bstart = cv.take<int32_t>(c->n_buckets_pad), o_far = cv.take<int32_t>(N),
                 o_nlogn = cv.take<double>(kLogTables * kNlognTable),
                 o_stage = cv.take<float>(N * c->dim), o_stage2 = cv.take<float>(N * c->dim), o_items = cv.take<APItem>(items.size()),
                 o_pd = cv.take<float>(3 * apoff), o_pj = cv.take<int32_t>(3 * apoff),
                 o_selp = cv.take<float>(8192), o_seln = cv.take<float>(16), o_feat = cv.take<float>(S * 8),
                 o_resring = cv.take<cert_scene_result>(2 * S), o_order = cv.take<int32_t>(S),
                 o_mdil = cv.take<uint32_t>(S * kMotionStride), o_spol = cv.take<int32_t>(S),
                 o_ccnt = cv.take<int32_t>(ceil_div(N, kSearchChunk)), o_cord = cv.take<int32_t>(ceil_div(N, kSearchChunk));
    const int64_t Nclk = (c->frontier_rule == CERT_FRONTIER_CLOCK) ? N : 0;
    const size_t o_clks = cv.take<double>(Nclk), o_clkc = cv.take<float>(Nclk), o_clkg = cv.take<float>(Nclk);
    cv.off = (cv.off + 255) & ~size_t(255);
    const size_t zero_begin = cv.off;
    const size_t o_acc = cv.take<SceneAcc>(S), o_ctr = cv.take<uint32_t>(4), o_farc = cv.take<int32_t>(4),
                 o_hfail = cv.take<int32_t>(c->c16h ? hoff / 2 : hoff);
    // the span k_search zeroes (StepArgs::ztail)
    const size_t o_tb = cv.take<uint64_t>(c->ntiles_b * kScanItems),
                 o_tp = cv.take<uint64_t>(ceil_div(N, kThreads)),   // small grids scan eighth tiles
                 o_bcount = cv.take<int32_t>(c->c16b ? c->n_buckets_pad / 2 : c->n_buckets_pad),
                 o_hocc = cv.take<uint32_t>(hoff / 32 + 1), o_hcand = cv.take<int32_t>(c->c16h ? hoff / 2 : hoff),
                 o_mgrid = cv.take<uint32_t>(S * kMotionStride);
    cv.off = (cv.off + 15) & ~size_t(15);
    c->zero_bytes = cv.off - zero_begin;
    c->ztail_off = o_tb - zero_begin;
    c->blob_bytes = cv.off;
    cudaError_t e = cudaMalloc((void **)&c->blob, c->blob_bytes);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, e == cudaErrorMemoryAllocation ? CERT_ENOMEM : CERT_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    char *b = c->blob;
    c->sp = (SceneParams *)(b + o_sp);
    c->st = (SceneState *)(b + o_st);
    c->res = (cert_scene_result *)(b + o_res);
    c->status = (uint32_t *)(b + o_status);
    c->fstart = (int32_t *)(b + o_fstart);
    c->scene_of = (int32_t *)(b + o_scene);
    c->pos[0] = (float4 *)(b + o_pos0);
    c->pos[1] = (float4 *)(b + o_pos1);
    c->nn = (int32_t *)(b + o_nn);
    c->nn2 = (int32_t *)(b + o_nn2);
    c->nn3 = (int32_t *)(b + o_nn3);
    c->d1sq = (float *)(b + o_d1);
    c->d2sq = (float *)(b + o_d2);
    c->L = (float *)(b + o_L);
    c->hcell = (int32_t *)(b + o_hcell);
    c->frontier = (int32_t *)(b + o_front);
    c->inF = (uint8_t *)(b + o_inF);
    c->failed = (uint8_t *)(b + o_failed);
    c->sflag = (uint8_t *)(b + o_sflag);
    c->brank = (int2 *)(b + o_brank);
    c->squad = (float4 *)(b + o_sorted);
    c->bucket_start = (int32_t *)(b + o_bstart);
    c->far_list = (int32_t *)(b + o_far);
    c->far_count = (int32_t *)(b + o_farc);
    c->nlogn = (double *)(b + o_nlogn);
    c->stage = (float *)(b + o_stage);
    c->stage2 = (float *)(b + o_stage2);
    c->res_ring = (cert_scene_result *)(b + o_resring);
    c->ap_items = (APItem *)(b + o_items);
    c->ap_pd = (float *)(b + o_pd);
    c->ap_pj = (int32_t *)(b + o_pj);
    c->sel_params = (float *)(b + o_selp);
    c->scene_policy = (int32_t *)(b + o_spol);
    c->sel_norm = (float *)(b + o_seln);
    c->feat = (float *)(b + o_feat);
    c->order = (int32_t *)(b + o_order);
    c->mdil = (uint32_t *)(b + o_mdil);
    c->chunk_cnt = (int32_t *)(b + o_ccnt);
    c->chunk_order = (int32_t *)(b + o_cord);
    c->mgrid = (uint32_t *)(b + o_mgrid);
    if (Nclk) {
        c->clk_s = (double *)(b + o_clks);
        c->clk_c = (float *)(b + o_clkc);
        c->clk_g = (float *)(b + o_clkg);
    }
    c->zero = b + zero_begin;
    c->acc = (SceneAcc *)(b + o_acc);
    c->tile_ctr = (uint32_t *)(b + o_ctr);
    c->tstat_b = (uint64_t *)(b + o_tb);
    c->tstat_p = (uint64_t *)(b + o_tp);
    c->bucket_count = (int32_t *)(b + o_bcount);
    c->hocc = (uint32_t *)(b + o_hocc);
    c->hfail = (int32_t *)(b + o_hfail);
    c->hcand = (int32_t *)(b + o_hcand);

    // ---- host-built tables
    std::vector<int32_t> scene_of(N);
    for (int k = 0; k < c->S; ++k)
        for (int64_t i = off[k]; i < off[k + 1]; ++i) scene_of[i] = k;
    // FP64 tables (cert_internal.cuh): k ln k, ln k, 1/k, 1/ln k, and k ln k in fixed point
    std::vector<double> nlogn(size_t(kLogTables) * kNlognTable, 0.0);
    for (int k = 1; k < kNlognTable; ++k) {
        const double lk = std::log((double)k);
        nlogn[k] = (double)k * lk;
        nlogn[size_t(kNlognTable) + k] = lk;
        nlogn[size_t(2) * kNlognTable + k] = 1.0 / (double)k;
        nlogn[size_t(3) * kNlognTable + k] = k >= 2 ? 1.0 / lk : 0.0;
        const long long fx = std::llround(std::ldexp((double)k * (long double)lk, kNlognFixBits));
        std::memcpy(&nlogn[size_t(4) * kNlognTable + k], &fx, sizeof(fx));
    }
    std::vector<SceneState> st0(S);
    for (int k = 0; k < c->S; ++k) {
        std::memset(&st0[k], 0, sizeof(SceneState));
        st0[k].g_cur = st0[k].g_next = c->h_sp[k].g_default;
        st0[k].inv_g = 1.0f / (float)st0[k].g_cur;
        st0[k].strategy = STRAT_INC;
    }
    cert_status rc = CERT_OK;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (rc != CERT_OK || bytes == 0) return;
        cudaError_t e2 = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
        if (e2 != cudaSuccess) rc = cuda_fail(c, "cudaMemcpyAsync", e2);
    };
    up(c->sp, c->h_sp.data(), S * sizeof(SceneParams));
    up(c->st, st0.data(), S * sizeof(SceneState));
    up(c->scene_of, scene_of.data(), N * sizeof(int32_t));
    up(c->nlogn, nlogn.data(), nlogn.size() * sizeof(double));
    up(c->ap_items, items.data(), items.size() * sizeof(APItem));
    // fused steps launch the largest scenes first (ties by index)
    std::vector<int32_t> order(S);
    for (int k = 0; k < c->S; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return c->h_sp[x].n > c->h_sp[y].n; });
    up(c->order, order.data(), S * sizeof(int32_t));
    if (rc == CERT_OK) {
        // padding bytes of the flag arrays and the result block start at zero
        cudaError_t e3 = cudaMemsetAsync(c->inF, 0, Npad, s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->failed, 0, Npad, s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->sflag, 0, Npad, s);
        // quad padding: all-ones bytes are NaN coordinates and index -1
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->squad, 0xff, (size_t)c->n_quads * 4 * sizeof(float4), s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->res, 0, S * sizeof(cert_scene_result), s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->status, 0, 4 * sizeof(uint32_t), s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->fstart, 0, (S + 1) * sizeof(int32_t), s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->feat, 0, S * 8 * sizeof(float), s);
        if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->chunk_cnt, 0, ceil_div(N, kSearchChunk) * sizeof(int32_t), s);
        if (e3 != cudaSuccess) rc = cuda_fail(c, "cudaMemsetAsync", e3);
    }
    if (rc == CERT_OK) rc = run_full(c, MODE_INIT, d_pos, s);
    if (rc != CERT_OK) {
        g_err = c->err;
        cudaStreamSynchronize(s);
        cudaFree(c->blob);
        delete c;
        return rc;
    }
    *out = c;
    return CERT_OK;
}

cert_status cert_step(cert_ctx *c, const float *d_pos_new, float eps, int32_t strategy, cert_views *out,
                      void *stream)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (!d_pos_new) return fail(c, CERT_EINVAL, "positions are NULL");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return fail(c, CERT_EINVAL, "eps must be finite and >= 0");
    if (strategy < STRAT_AUTO || strategy > STRAT_THR) return fail(c, CERT_EINVAL, "unknown strategy");
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(c, MODE_STEP);
    a.pos_in = d_pos_new;
    a.pos_old = c->pos[c->cur];
    a.pos_new = c->pos[c->cur ^ 1];
    a.declared_eps = eps;
    a.strategy = strategy;
    a.ntiles_p = c->ntiles_p;
    cudaEvent_t *ev = nullptr;
    if (c->prof_on && c->prof_n < c->prof_max) ev = &c->prof_ev[size_t(c->prof_n++) * (CERT_N_PHASES + 1)];
    auto mark = [&](int k) -> cudaError_t { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    if (use_fused(c, strategy)) {
        // one launch: every phase of every scene (phases 0-6 of the profile are empty)
        for (int k = 0; k <= 7; ++k) CK(c, mark(k));
        CK(c, launch_fused_step(a, c->order, fused_block(c), fused_resident(c), s));
        CK(c, mark(8));
        c->cur ^= 1;
        c->last = s;
        c->stepped = true;
        if (out) cert_get_views(c, out);
        return CERT_OK;
    }
    CK(c, mark(0));
    if (c->zero_dirty) CK(c, cudaMemsetAsync(c->zero, 0, c->zero_bytes, s));
    CK(c, mark(1));
    CK(c, launch_step_phase(a, PH_PREPARE, s));
    CK(c, mark(2));
    CK(c, launch_step_phase(a, PH_SCAN, s));
    CK(c, mark(3));
    CK(c, launch_step_phase(a, PH_SELECT, s));
    CK(c, mark(4));
    if (strategy == STRAT_ALL) {
        APArgs ap;
        std::memset(&ap, 0, sizeof(ap));
        ap.dim = c->dim;
        ap.pos = a.pos_new;
        ap.sp = c->sp;
        ap.items = c->ap_items;
        ap.n_items = c->n_ap_items;
        ap.pd = c->ap_pd;
        ap.pj = c->ap_pj;
        ap.P = c->ap_P;
        ap.status = c->status;
        CK(c, launch_allpairs(ap, s));
        CK(c, mark(5));
        APMergeOut mo;
        std::memset(&mo, 0, sizeof(mo));
        mo.step_mode = 1;
        mo.step = a;
        CK(c, launch_allpairs_merge(ap, mo, c->N, s));
        // no k_search on this path: zero its span here
        CK(c, cudaMemsetAsync(c->zero + c->ztail_off, 0, c->zero_bytes - c->ztail_off, s));
    } else {
        CK(c, launch_step_phase(a, PH_SCATTER, s));
        CK(c, mark(5));
        CK(c, launch_step_phase(a, PH_SEARCH, s));
    }
    CK(c, mark(6));
    CK(c, launch_step_phase(a, PH_FINALIZE, s));
    c->zero_dirty = false;
    CK(c, mark(7));
    CK(c, mark(8));
    c->cur ^= 1;
    c->last = s;
    c->stepped = true;
    if (out) cert_get_views(c, out);
    return CERT_OK;
}

cert_status cert_step_host(cert_ctx *c, const float *h_pos_new, float eps, int32_t strategy,
                           cert_scene_result *h_scenes, void *stream)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (!h_pos_new) return fail(c, CERT_EINVAL, "positions are NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CK(c, cudaMemcpyAsync(c->stage, h_pos_new, size_t(c->N) * c->dim * sizeof(float), cudaMemcpyHostToDevice, s));
    cert_status rc = cert_step(c, c->stage, eps, strategy, nullptr, stream);
    if (rc != CERT_OK) return rc;
    if (h_scenes)
        CK(c, cudaMemcpyAsync(h_scenes, c->res, size_t(c->S) * sizeof(cert_scene_result),
                              cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    return CERT_OK;
}

// One step on `stream` by replaying a captured graph of cert_step for this
// parity of the position and staging buffers (captured on first use).
static cert_status step_by_graph(cert_ctx *c, const float *stage, int b, float eps, int32_t strategy,
                                 cudaStream_t s)
{
    cert_ctx::StepGraph &g = c->step_graph[c->cur * 2 + b];
    if (!g.exec || g.eps != eps || g.strategy != strategy || g.epoch != c->settings_epoch) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        if (!c->capture_stream) CK(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
        const int cur0 = c->cur;
        const cudaStream_t last0 = c->last;
        const bool stepped0 = c->stepped, dirty0 = c->zero_dirty;
        CK(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
        c->res_target = c->res_ring + (size_t)b * c->S;   // this parity's result slot
        const cert_status rc = cert_step(c, stage, eps, strategy, nullptr, c->capture_stream);
        c->res_target = nullptr;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->capture_stream, &graph);
        c->cur = cur0;              // the capture enqueued nothing: undo its bookkeeping
        c->last = last0;
        c->stepped = stepped0;
        c->zero_dirty = dirty0;
        if (rc != CERT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        CK(c, e);
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(c, ei);
        g.eps = eps;
        g.strategy = strategy;
        g.epoch = c->settings_epoch;
    }
    CK(c, cudaGraphLaunch(g.exec, s));
    c->cur ^= 1;
    c->last = s;
    c->stepped = true;
    return CERT_OK;
}

cert_status cert_step_host_stream(cert_ctx *c, const float *const *h_frames, int32_t n_steps, float eps,
                                  int32_t strategy, cert_scene_result *h_scenes, void *stream)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (!h_frames) return fail(c, CERT_EINVAL, "frames are NULL");
    if (n_steps < 0) return fail(c, CERT_EINVAL, "n_steps < 0");
    for (int32_t k = 0; k < n_steps; ++k)
        if (!h_frames[k]) return fail(c, CERT_EINVAL, "a frame pointer is NULL");
    const int64_t frame = c->N * c->dim;
    if (!c->copy_stream) {
        CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        CK(c, cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            CK(c, cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
            CK(c, cudaEventCreateWithFlags(&c->ev_used[k], cudaEventDisableTiming));
            CK(c, cudaEventCreateWithFlags(&c->ev_d2h[k], cudaEventDisableTiming));
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    float *buf[2] = {c->stage, c->stage2};
    const size_t res_bytes = size_t(c->S) * sizeof(cert_scene_result);
    // both buffers and both result slots are free once the caller's stream has reached this point
    for (int k = 0; k < 2; ++k) {
        CK(c, cudaEventRecord(c->ev_used[k], s));
        CK(c, cudaEventRecord(c->ev_d2h[k], s));
    }
    for (int32_t k = 0; k < n_steps; ++k) {
        const int b = k & 1;
        // copy frame k while step k-1 runs; buffer b was last read by step k-2
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_used[b], 0));
        CK(c, cudaMemcpyAsync(buf[b], h_frames[k], size_t(frame) * sizeof(float),
                              cudaMemcpyHostToDevice, c->copy_stream));
        CK(c, cudaEventRecord(c->ev_copied[b], c->copy_stream));
        CK(c, cudaStreamWaitEvent(s, c->ev_copied[b], 0));
        // result slot b was last read back for step k-2 (long done by now)
        CK(c, cudaStreamWaitEvent(s, c->ev_d2h[b], 0));
        // replayed as a graph (fewer launch gaps) unless phase profiling is on; either
        // way step k's scalars land in result slot b
        cert_status rc;
        if (c->prof_on) {
            c->res_target = c->res_ring + (size_t)b * c->S;
            rc = cert_step(c, buf[b], eps, strategy, nullptr, stream);
            c->res_target = nullptr;
        } else {
            rc = step_by_graph(c, buf[b], b, eps, strategy, s);
        }
        if (rc != CERT_OK) return rc;
        CK(c, cudaEventRecord(c->ev_used[b], s));
        // the read-back waits for step k on its own stream, so step k+1 starts at once
        if (h_scenes) {
            CK(c, cudaStreamWaitEvent(c->d2h_stream, c->ev_used[b], 0));
            CK(c, cudaMemcpyAsync(h_scenes + (size_t)k * c->S, c->res_ring + (size_t)b * c->S, res_bytes,
                                  cudaMemcpyDeviceToHost, c->d2h_stream));
            CK(c, cudaEventRecord(c->ev_d2h[b], c->d2h_stream));
        }
    }
    // the last step's scalars also where cert_sync_result and the views read them
    if (n_steps > 0)
        CK(c, cudaMemcpyAsync(c->res, c->res_ring + (size_t)((n_steps - 1) & 1) * c->S, res_bytes,
                              cudaMemcpyDeviceToDevice, s));
    CK(c, cudaStreamSynchronize(c->d2h_stream));
    CK(c, cudaStreamSynchronize(s));
    return CERT_OK;
}

cert_status cert_rebuild(cert_ctx *c, void *stream)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    return run_full(c, MODE_REBUILD, nullptr, (cudaStream_t)stream);
}

cert_status cert_get_views(const cert_ctx *c, cert_views *out)
{
    if (!c || !out) return fail(const_cast<cert_ctx *>(c), CERT_EINVAL, "NULL argument");
    out->nn = c->nn;
    out->d1sq = c->d1sq;
    out->d2sq = c->d2sq;
    out->cell = c->hcell;
    out->frontier = c->frontier;
    out->failed = c->failed;
    out->scenes = c->res;
    out->n_total = c->N;
    out->n_scenes = c->S;
    out->dim = c->dim;
    return CERT_OK;
}

cert_status cert_sync_result(cert_ctx *c, cert_scene_result *h_scenes)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    CK(c, cudaStreamSynchronize(c->last));
    if (h_scenes) CK(c, cudaMemcpy(h_scenes, c->res, size_t(c->S) * sizeof(cert_scene_result), cudaMemcpyDeviceToHost));
    uint32_t st = 0;
    CK(c, cudaMemcpy(&st, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    CK(c, cudaMemset(c->status, 0, sizeof(uint32_t)));
    if (st & ST_INDEX) return fail(c, CERT_EINTERNAL, "an internal index check failed (debug build)");
    if (st & ST_TIMEOUT) return fail(c, CERT_ETIMEOUT, "a bounded device wait gave up");
    if (st & ST_NONFINITE) return fail(c, CERT_EINVAL, "non-finite coordinate in the positions");
    if (st & ST_EBOUND) return fail(c, CERT_EBOUND, "measured eps_t exceeded the declared eps");
    return CERT_OK;
}

cert_status cert_distances(cert_ctx *c, float *d_d1, float *d_d2, void *stream)
{
    if (!c || !d_d1 || !d_d2) return fail(c, CERT_EINVAL, "NULL argument");
    CK(c, launch_distances(c->d1sq, c->d2sq, d_d1, d_d2, (int)c->N, (cudaStream_t)stream));
    return CERT_OK;
}

cert_status cert_profile_begin(cert_ctx *c, int32_t max_steps)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (max_steps < 1 || max_steps > (1 << 20)) return fail(c, CERT_EINVAL, "max_steps out of range");
    const size_t need = size_t(max_steps) * (CERT_N_PHASES + 1);
    while (c->prof_ev.size() < need) {
        cudaEvent_t e;
        CK(c, cudaEventCreate(&e));
        c->prof_ev.push_back(e);
    }
    c->prof_max = max_steps;
    c->prof_n = 0;
    c->prof_on = true;
    return CERT_OK;
}

cert_status cert_profile_end(cert_ctx *c, float *h_ms, int32_t max_steps, int32_t *n_steps)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    c->prof_on = false;
    const int n = std::min(c->prof_n, std::max(0, (int)max_steps));
    if (n_steps) *n_steps = n;
    if (n > 0) CK(c, cudaEventSynchronize(c->prof_ev[size_t(n - 1) * (CERT_N_PHASES + 1) + CERT_N_PHASES]));
    for (int k = 0; k < n && h_ms; ++k) {
        cudaEvent_t *ev = &c->prof_ev[size_t(k) * (CERT_N_PHASES + 1)];
        for (int ph = 0; ph < CERT_N_PHASES; ++ph) {
            float ms = 0.0f;
            CK(c, cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]));
            h_ms[size_t(k) * CERT_N_PHASES + ph] = ms;
        }
    }
    c->prof_n = 0;
    return CERT_OK;
}

cert_status cert_set_cell_scale(cert_ctx *c, float scale)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (!(scale > 0.0f) || !std::isfinite(scale)) return fail(c, CERT_EINVAL, "cell_scale must be finite and > 0");
    c->cell_scale = scale;
    ++c->settings_epoch;
    return CERT_OK;
}

float cert_get_cell_scale(const cert_ctx *c) { return c ? c->cell_scale : 0.0f; }

cert_status cert_set_step_path(cert_ctx *c, int32_t path)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (path < CERT_PATH_AUTO || path > CERT_PATH_FUSED) return fail(c, CERT_EINVAL, "unknown step path");
    if (path == CERT_PATH_FUSED && !c->fused_ok)
        return fail(c, CERT_EINVAL, "a scene exceeds the fused step's limits (16,384 points, 16,384 search-grid buckets)");
    c->step_path = path;
    ++c->settings_epoch;
    return CERT_OK;
}

int32_t cert_get_step_path(const cert_ctx *c, int32_t strategy)
{
    if (!c) return -1;
    return use_fused(c, strategy) ? CERT_PATH_FUSED : CERT_PATH_MULTI;
}

cert_status cert_set_cell_quantile(cert_ctx *c, float q)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (!(q > 0.0f && q <= 1.0f)) return fail(c, CERT_EINVAL, "cell_quantile must be in (0, 1]");
    c->cell_quantile = q;
    ++c->settings_epoch;
    return CERT_OK;
}

cert_status cert_get_features(cert_ctx *c, float *h_feat)
{
    if (!c || !h_feat) return fail(c, CERT_EINVAL, "NULL argument");
    CK(c, cudaStreamSynchronize(c->last));
    CK(c, cudaMemcpy(h_feat, c->feat, size_t(c->S) * 8 * sizeof(float), cudaMemcpyDeviceToHost));
    return CERT_OK;
}

cert_status cert_selector_load(cert_ctx *c, const float *h_params, const float *h_norm)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    CK(c, cudaStreamSynchronize(c->last));
    if (!h_params) {
        c->have_sel = false;
        ++c->settings_epoch;
        return CERT_OK;
    }
    if (!h_norm) return fail(c, CERT_EINVAL, "feature normalisation is NULL");
    for (int k = 0; k < CERT_MLP_PARAMS; ++k)
        if (!std::isfinite(h_params[k])) return fail(c, CERT_EINVAL, "non-finite selector weight");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(h_norm[k])) return fail(c, CERT_EINVAL, "non-finite feature normalisation");
    CK(c, cudaMemcpy(c->sel_params, h_params, CERT_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->sel_norm, h_norm, 16 * sizeof(float), cudaMemcpyHostToDevice));
    c->have_sel = true;
    ++c->settings_epoch;
    return CERT_OK;
}

cert_status cert_set_scene_policy(cert_ctx *c, const int32_t *h_policy)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (h_policy)
        for (int k = 0; k < c->S; ++k)
            if (h_policy[k] != STRAT_INC && h_policy[k] != STRAT_REB)
                return fail(c, CERT_EINVAL, "scene policy must be INCREMENTAL or REBUILD");
    CK(c, cudaStreamSynchronize(c->last));
    if (h_policy) CK(c, cudaMemcpy(c->scene_policy, h_policy, size_t(c->S) * sizeof(int32_t), cudaMemcpyHostToDevice));
    c->have_scene_policy = h_policy != nullptr;
    ++c->settings_epoch;
    return CERT_OK;
}

// Pieces of the mutable state a snapshot covers (device pointer, bytes).
static std::vector<std::pair<void *, size_t>> snapshot_pieces(cert_ctx *c)
{
    const size_t N = size_t(c->N), S = size_t(c->S);
    return {{c->pos[c->cur], N * sizeof(float4)},  {c->nn, N * 4},         {c->nn2, N * 4},
            {c->nn3, N * 4},
            {c->d1sq, N * 4},                      {c->d2sq, N * 4},       {c->L, N * 4},
            {c->st, S * sizeof(SceneState)},      {c->res, S * sizeof(cert_scene_result)},
            {c->hcell, N * 4},                     {c->frontier, N * 4},   {c->fstart, (S + 1) * 4},
            {c->failed, N},                        {c->inF, N},            {c->feat, S * 8 * 4},
            {c->clk_s, c->clk_s ? N * 8 : 0},      {c->clk_c, c->clk_c ? N * 4 : 0},
            {c->clk_g, c->clk_g ? N * 4 : 0},
            // the search's per-chunk query counts, which order the next step's search:
            // runs from one snapshot all start from the same schedule
            {c->chunk_cnt, size_t(ceil_div(int64_t(N), kSearchChunk)) * 4}};
}

cert_status cert_snapshot(cert_ctx *c, void *stream)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    auto pieces = snapshot_pieces(c);
    size_t need = 0;
    for (auto &p : pieces) need += (p.second + 255) & ~size_t(255);
    if (!c->snap) {
        cudaError_t e = cudaMalloc((void **)&c->snap, need);
        if (e != cudaSuccess) return fail(c, CERT_ENOMEM, std::string("snapshot buffer: ") + cudaGetErrorString(e));
        c->snap_bytes = need;
    }
    size_t off = 0;
    for (auto &p : pieces) {
        if (!p.second) continue;
        CK(c, cudaMemcpyAsync(c->snap + off, p.first, p.second, cudaMemcpyDeviceToDevice, s));
        off += (p.second + 255) & ~size_t(255);
    }
    c->snap_cur = c->cur;
    c->snap_valid = true;
    c->last = s;
    return CERT_OK;
}

cert_status cert_restore(cert_ctx *c, void *stream)
{
    if (!c) return fail(nullptr, CERT_EINVAL, "ctx is NULL");
    if (!c->snap_valid) return fail(c, CERT_ESTATE, "no snapshot taken");
    cudaStream_t s = (cudaStream_t)stream;
    c->cur = c->snap_cur;
    auto pieces = snapshot_pieces(c);
    size_t off = 0;
    for (auto &p : pieces) {
        if (!p.second) continue;
        CK(c, cudaMemcpyAsync(p.first, c->snap + off, p.second, cudaMemcpyDeviceToDevice, s));
        off += (p.second + 255) & ~size_t(255);
    }
    c->last = s;
    return CERT_OK;
}

cert_status cert_autotune(cert_ctx *c, const float *d_frames, int64_t frame_stride, int32_t n_frames, float eps,
                          int32_t strategy, const float *h_scales, int32_t n_scales, float *h_ms, float *h_best,
                          void *stream)
{
    if (!c || !d_frames || !h_scales) return fail(c, CERT_EINVAL, "NULL argument");
    if (n_frames < 2 || n_scales < 1 || frame_stride < c->N * c->dim)
        return fail(c, CERT_EINVAL, "need n_frames >= 2, n_scales >= 1 and frame_stride >= n_total*dim");
    for (int k = 0; k < n_scales; ++k)
        if (!(h_scales[k] > 0.0f) || !std::isfinite(h_scales[k])) return fail(c, CERT_EINVAL, "bad candidate scale");
    cudaStream_t s = (cudaStream_t)stream;
    const float keep = c->cell_scale;
    cert_status rc = cert_snapshot(c, stream);
    if (rc != CERT_OK) return rc;
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    float best_ms = 0.0f, best = keep;
    for (int k = 0; k < n_scales && rc == CERT_OK; ++k) {
        rc = cert_restore(c, stream);
        c->cell_scale = h_scales[k];
        // the first step derives the search grid from the candidate scale
        if (rc == CERT_OK) rc = cert_step(c, d_frames, eps, strategy, nullptr, stream);
        if (rc == CERT_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = fail(c, CERT_ECUDA, "event");
        for (int f = 1; f < n_frames && rc == CERT_OK; ++f)
            rc = cert_step(c, d_frames + f * frame_stride, eps, strategy, nullptr, stream);
        if (rc == CERT_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = fail(c, CERT_ECUDA, "event");
        float ms = 0.0f;
        if (rc == CERT_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = fail(c, CERT_ECUDA, "event timing");
        if (h_ms) h_ms[k] = ms;
        if (rc == CERT_OK && (k == 0 || ms < best_ms)) {
            best_ms = ms;
            best = h_scales[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cert_status rc2 = cert_restore(c, stream);
    c->cell_scale = (rc == CERT_OK) ? best : keep;
    ++c->settings_epoch;
    if (h_best) *h_best = c->cell_scale;
    if (rc == CERT_OK) rc = rc2;
    // drop any status the probe steps latched (e.g. EBOUND from the caller's frames)
    if (rc == CERT_OK) CK(c, cudaMemsetAsync(c->status, 0, sizeof(uint32_t), s));
    return rc;
}

void cert_destroy(cert_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->snap) cudaFree(c->snap);
    for (int k = 0; k < 2; ++k) {
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
        if (c->ev_used[k]) cudaEventDestroy(c->ev_used[k]);
        if (c->ev_d2h[k]) cudaEventDestroy(c->ev_d2h[k]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->d2h_stream) cudaStreamDestroy(c->d2h_stream);
    for (auto &g : c->step_graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    cudaFree(c->blob);
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------- bounded-wait self-test

namespace certk {
// Spin on a flag nothing ever sets, exactly as the chained scan waits for a
// predecessor, but with a caller-given iteration limit; on expiry record the
// timeout in the status word and return.
__global__ void k_wait_selftest(const uint64_t *flag, uint32_t limit, uint32_t *status, uint32_t *spun)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t spins = 0;
    while ((ld_acquire_u64(flag) >> 32) == 0u) {
        if (++spins > limit) {
            atomicOr(status, ST_TIMEOUT);
            break;
        }
    }
    *spun = spins;
}
}  // namespace certk

extern "C" cert_status cert_selftest_bounded_wait(int32_t limit, uint32_t *h_status, uint32_t *h_spins)
{
    if (limit < 1 || limit > (1 << 24)) return fail(nullptr, CERT_EINVAL, "limit must be in [1, 2^24]");
    char *buf = nullptr;
    CK((cert_ctx *)nullptr, cudaMalloc((void **)&buf, 256));
    cudaError_t e = cudaMemset(buf, 0, 256);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>((const uint64_t *)buf, (uint32_t)limit, (uint32_t *)(buf + 64),
                                   (uint32_t *)(buf + 128));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    uint32_t st = 0, sp = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, buf + 64, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&sp, buf + 128, 4, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(nullptr, "cert_selftest_bounded_wait", e);
    if (h_status) *h_status = st;
    if (h_spins) *h_spins = sp;
    return (st & ST_TIMEOUT) ? CERT_ETIMEOUT : CERT_OK;
}

// ---------------------------------------------------------------- cert_allpairs

namespace certk {
__global__ void k_write_params(SceneParams *dst, SceneParams v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}
}  // namespace certk

extern "C" cert_status cert_allpairs(const float *d_pos, int64_t n, int32_t dim, const int32_t *d_queries,
                                     int64_t nq, int32_t *d_nn, float *d_d1sq, float *d_d2sq, void *stream)
{
    if (!d_pos || !d_nn || !d_d1sq || !d_d2sq) return fail(nullptr, CERT_EINVAL, "NULL argument");
    if (dim != 2 && dim != 3) return fail(nullptr, CERT_EINVAL, "dim must be 2 or 3");
    if (n < 3 || n >= (int64_t(1) << 31) / 2) return fail(nullptr, CERT_EINVAL, "need 3 <= n < 2^30");
    if (!d_queries) nq = n;
    if (nq < 0 || nq >= (int64_t(1) << 31) / 2) return fail(nullptr, CERT_EINVAL, "bad query count");
    if (nq == 0) return CERT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int nqb = (int)ceil_div(nq, kApQBlock);
    const int nch = allpairs_chunks_for(nqb, n, dim, (int)std::min<int64_t>(64, ceil_div(n, 256)));
    SceneParams p;
    std::memset(&p, 0, sizeof(p));
    p.pt_off = 0;
    p.n = (int32_t)n;
    p.ap_off = 0;
    p.ap_nch = nch;
    p.ap_chunk = (int32_t)ceil_div(n, nch);
    const long long P = (long long)nq * nch;
    Carver cv;
    const size_t o_pos = cv.take<float4>(n), o_sp = cv.take<SceneParams>(1), o_st = cv.take<uint32_t>(4),
                 o_pd = cv.take<float>(3 * P), o_pj = cv.take<int32_t>(3 * P);
    char *scratch = nullptr;
    CK((cert_ctx *)nullptr, cudaMallocAsync((void **)&scratch, cv.off, s));
    float4 *pos4 = (float4 *)(scratch + o_pos);
    SceneParams *dsp = (SceneParams *)(scratch + o_sp);
    uint32_t *status = (uint32_t *)(scratch + o_st);
    cudaError_t e = cudaMemsetAsync(status, 0, 16, s);
    if (e == cudaSuccess) {
        k_write_params<<<1, 32, 0, s>>>(dsp, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_pack(d_pos, (int)n, dim, pos4, status, s);
    APArgs ap;
    std::memset(&ap, 0, sizeof(ap));
    ap.dim = dim;
    ap.pos = pos4;
    ap.sp = dsp;
    ap.items = nullptr;
    ap.nqb = nqb;
    ap.n_items = nqb * nch;
    ap.queries = d_queries;
    ap.nq_list = (int)nq;
    ap.pd = (float *)(scratch + o_pd);
    ap.pj = (int32_t *)(scratch + o_pj);
    ap.P = P;
    ap.status = status;
    if (e == cudaSuccess) e = launch_allpairs(ap, s);
    APMergeOut mo;
    std::memset(&mo, 0, sizeof(mo));
    mo.nn = d_nn;
    mo.d1sq = d_d1sq;
    mo.d2sq = d_d2sq;
    if (e == cudaSuccess) e = launch_allpairs_merge(ap, mo, nq, s);
    uint32_t st = 0;
    bool have_st = false;
    if (e == cudaSuccess) e = allpairs_status_read(status, &st, &have_st, s);   // before the free below
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, "cert_allpairs launch", e);
    if (e2 != cudaSuccess) return cuda_fail(nullptr, "cudaFreeAsync", e2);
    return have_st ? allpairs_status_code(st) : CERT_OK;
}
