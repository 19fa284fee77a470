/*
 * cert.h -- C ABI of libcert.so: exact nearest-neighbour certificates for
 * points moving by small steps in 2-D and 3-D, maintained on one B300 GPU.
 *
 * Paper: "Repair Entropy in Dynamic Geometric Nearest-Neighbour Structures".
 *   certificate (nn_i, d1_i, d2_i), clearance c_i = d2_i - d1_i  ...... Sec. 2, Def. 1
 *   safety rule: c_i > 4 eps  =>  nn_i unchanged ..................... Lemma 1, Thm A.1
 *   one maintenance step (eps, frontier, cell update, block repair) .. Algorithm 1
 *   frontier entropy H(F_t) over the occupied index cells ............. Def. 2
 *   exactness of the widened-block repair ............................. Cor. A.2
 *   incremental repair vs rebuild vs exact all-pairs pass ............. Sec. 3 (strategies)
 *
 * Conventions (every entry point):
 *   - Positions are float32, contiguous [n][dim] (dim = 2 or 3), in DEVICE
 *     memory owned by the caller, unless the name ends in _host.  They are
 *     expected in the unit domain [0,1]^dim; points outside are clamped into
 *     the boundary index cells, which keeps every result exact.
 *   - Squared distances use the fixed FP32 order ((dx*dx + dy*dy) + dz*dz),
 *     dx = x_j - x_i, each operation rounded to nearest, no FMA.  Equal
 *     squared distances are ordered by the lower point index.
 *   - Indices in results are scene-local (0 .. n_s - 1).
 *   - A stream argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Entry points that take a stream only enqueue work and
 *     never synchronise, unless documented otherwise.
 *   - Errors: host-detectable argument errors return immediately, nothing is
 *     enqueued.  Device-side conditions (a bounded wait that gave up, a
 *     non-finite coordinate, eps_t above the declared eps) are latched in a
 *     device status word and reported by cert_sync_result.  No entry point
 *     throws, aborts or prints.
 *   - Thread safety: one context must not be used from two threads at once.
 */
#ifndef CERT_H
#define CERT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cert_ctx cert_ctx;

typedef enum {
    CERT_OK = 0,
    CERT_EINVAL = 1,   /* bad argument; or (latched) a non-finite coordinate      */
    CERT_ENOMEM = 2,   /* device allocation failed                                 */
    CERT_ECUDA = 3,    /* a CUDA runtime call failed; see cert_last_error          */
    CERT_ETIMEOUT = 4, /* (latched) a bounded device-side wait gave up             */
    CERT_EBOUND = 5,   /* (latched, warning) measured eps_t > declared eps         */
    CERT_ESTATE = 6,   /* call not valid in the context's current state            */
    CERT_EINTERNAL = 7 /* (latched, debug builds only: libcert_debug.so) an internal
                          index check failed -- a bug in this library, never the caller's */
} cert_status;

typedef enum {
    CERT_AUTO = 0,        /* per scene: the loaded selector's choice, else the policy */
    CERT_INCREMENTAL = 1, /* O(1) refresh where provable, grid repair of the rest (Alg. 1) */
    CERT_REBUILD = 2,     /* grid search for every point (O(N) rebuild)               */
    CERT_ALLPAIRS = 3,    /* exact all-pairs pass for every point (O(N^2))            */
    CERT_THRESHOLD = 4    /* per scene: incremental iff |F|/N < 1/ln N, else rebuild
                             (Prop. 1 with the boundary P ~ 1/log N of Sec. 4)       */
} cert_strategy;

/* Which points a step flags as its detected frontier F_t (the audit, H_cand and
 * the selector features use F_t; the certificates are exact under every rule).
 * Each rule carries the rounding guard tau_i = 2^-20 ((d1_i + d2_i) + x), with x
 * the rule's motion term, and none ever misses a failed certificate.
 *   CERT_FRONTIER_STEP   c_i <= 4 eps_t + tau_i (Algorithm 1, Lemma 1), the default.
 *   CERT_FRONTIER_POINT  c_i <= 2 (delta_i + eps_t) + tau_i with delta_i = |p'_i - p_i|:
 *                        Lemma 1's triangle inequality with point i's own
 *                        displacement, the per-point motion budget of Sec. 5.
 *   CERT_FRONTIER_CLOCK  the cumulative clock of the per-step cost subsection
 *                        (Thm A.3): S = sum of eps_t in FP64; a certificate last
 *                        revisited at clock S_i with clearance c^rev_i stays valid
 *                        while 4 (S - S_i) < c^rev_i, so F_t = {i : c^rev_i <=
 *                        4 (S - S_i) + 2^-20 ((d1 + d2)^rev_i + (S - S_i))}, in FP64;
 *                        the points of F_t are revisited (S_i, c^rev_i reset from
 *                        their post-step certificates).  cert_init and
 *                        cert_rebuild revisit every point. */
typedef enum {
    CERT_FRONTIER_STEP = 0,
    CERT_FRONTIER_POINT = 1,
    CERT_FRONTIER_CLOCK = 2
} cert_frontier_rule;

/* Batch description.  One context holds n_scenes independent scenes whose
 * points are concatenated in scene order: scene s owns points
 * offsets[s] .. offsets[s+1]-1 of every position / result array. */
typedef struct {
    int32_t dim;              /* 2 or 3                                               */
    int32_t n_scenes;         /* >= 1                                                 */
    const int64_t *offsets;   /* HOST array [n_scenes+1]; offsets[0] = 0, strictly
                                 increasing, every scene >= 3 points, total < 2^31;
                                 NULL allowed when n_scenes == 1 together with n_total */
    int64_t n_total;          /* total points (used when offsets == NULL)             */
    float cell_scale;         /* search-grid cell side / reference d2 (0 -> 3.5)      */
    int32_t policy;           /* strategy for CERT_AUTO without a selector (0 -> INCREMENTAL) */
    int32_t bucket_factor;    /* hashed-grid buckets per scene = factor x next_pow2(n);
                                 1, 2, 4 or 8 (0 -> 1)                                 */
    float cell_quantile;      /* reference d2 = this quantile of a scene's previous d2
                                 over its first min(n,1024) points, in (0,1] (0 -> 0.5) */
    int32_t frontier_rule;    /* cert_frontier_rule (0 -> CERT_FRONTIER_STEP)          */
    int32_t audit;            /* cert_audit flags (0: none); other bits are rejected     */
} cert_config;

/* Optional per-step audits (cert_config.audit, OR-ed).  Off, their fields of
 * cert_scene_result stay 0 and the step does no extra work.
 *   CERT_AUDIT_RHO       the local heuristic rho_i = delta_i / c_i > 1/2 of Sec. 3
 *                        and Table 1: n_rho, n_rho_hit.
 *   CERT_AUDIT_GEOMETRY  the spatial spread of the true failures, the frontier
 *                        descriptors of the paper's transition log (Sec. 6 dataset
 *                        columns, which the paper names but does not define):
 *                        gyration and compactness. */
typedef enum {
    CERT_AUDIT_RHO = 1,
    CERT_AUDIT_GEOMETRY = 2,
    CERT_AUDIT_COST = 4       /* per-scene cost attribution inside a batched step (no counterpart
                                 in the paper): search_cycles, refresh_cycles.  Runs the
                                 multi-kernel step (the fused step is not taken) */
} cert_audit;

/* Per-scene scalars of the last step.  Same layout on device and host. */
typedef struct {
    double H;                 /* entropy of the true failures over the entropy grid, Def. 2 */
    double H_cand;            /* entropy of the detected frontier F_t                         */
    float eps_t;              /* measured max_i ||p'_i - p_i||, Algorithm 1                   */
    float med_c;              /* lower median of the pre-step clearances over the first
                                 min(n,1024) points, truncated to 3 mantissa bits            */
    int32_t n_frontier;       /* |F_t| = #{i : c_i <= 4 eps_t + tau_i} (pre-step certificates) */
    int32_t frontier_start;   /* offset of this scene's frontier list in the frontier array  */
    int32_t n_failed;         /* #{i : nn_i changed across the step}                          */
    int32_t n_missed;         /* failed but not in F_t (Lemma 1: always 0)                    */
    int32_t n_false;          /* in F_t but not failed                                         */
    int32_t n_searched;       /* certificates recomputed by a search this step                */
    int32_t failed_cells;     /* m: entropy-grid cells the failures meet (Thm A.4)            */
    int32_t frontier_cells;   /* cells the detected frontier meets                             */
    int32_t occupied_cells;   /* C: cells holding at least one point                           */
    int32_t strategy;         /* cert_strategy applied to this scene                           */
    float pred_inc;           /* selector output: predicted ln step time, incremental (0 if none) */
    float pred_reb;           /* selector output: predicted ln step time, rebuild               */
    int32_t grid_res;         /* entropy-grid cells per axis (smallest g with g^dim >= n)      */
    int32_t search_res;       /* search-grid cells per axis used this step                      */
    int32_t n_rho;            /* CERT_AUDIT_RHO: #{i : 2 delta_i > c_i}, delta_i = |p'_i - p_i|
                                 and c_i the pre-step clearance, both FP32 (the heuristic
                                 rho_i > 1/2 of Sec. 3 and Table 1; a guess, not a bound)     */
    int32_t n_rho_hit;        /* CERT_AUDIT_RHO: flagged points whose nn changed; recall =
                                 n_rho_hit / n_failed, false = (n_rho - n_rho_hit) / n_rho      */
    double gyration;          /* CERT_AUDIT_GEOMETRY: radius of gyration of the failed points'
                                 post-step positions, sqrt(mean |p'_i - centroid|^2); 0 with
                                 fewer than two failures.  FP64 sums in any order: within
                                 1e-5 of the two-pass value                                   */
    double compactness;       /* CERT_AUDIT_GEOMETRY: 1 - gyration / (the same radius over all
                                 points of the scene), clamped to [0, 1]: 1 when the failures
                                 collapse to a point, near 0 when they spread like the scene;
                                 1 for a single failure, 0 without failures                   */
    uint64_t search_cycles;   /* CERT_AUDIT_COST: the SM clock cycles the scene's searches took,
                                 summed over its queries (each query from its set-up to its
                                 certificate write, on its lane's SM clock, waits for the warp's
                                 other lanes included).  Within a step the scenes' shares of the
                                 sum are their shares of the search kernel's time             */
    uint64_t refresh_cycles;  /* CERT_AUDIT_COST: the same for the scatter and O(1) refresh of
                                 the scene's points                                             */
} cert_scene_result;

/* Device views of the per-point results; valid until the next call that
 * modifies the context.  All arrays are [n_total] unless noted. */
typedef struct {
    const int32_t *nn;        /* nearest neighbour (scene-local index)                        */
    const float *d1sq;        /* squared distance to nn                                       */
    const float *d2sq;        /* squared distance to the runner-up                            */
    const int32_t *cell;      /* entropy-grid cell of the post-step position (scene-local)   */
    const int32_t *frontier;  /* ascending frontier lists, scene s at [frontier_start, +n_frontier) */
    const uint8_t *failed;    /* 1 where nn changed across the last step                      */
    const cert_scene_result *scenes; /* [n_scenes] device copy of the scalars                */
    int64_t n_total;
    int32_t n_scenes;
    int32_t dim;
} cert_views;

/* Create a context and compute the initial certificates of d_pos by a full
 * grid search (exact; Def. 1).  d_pos: device [n_total][dim] float32.
 * Allocates every device buffer the context will use; later calls on the
 * context allocate nothing.  On error *out is NULL. */
cert_status cert_init(cert_ctx **out, const cert_config *cfg, const float *d_pos, void *stream);

/* One maintenance step to positions d_pos_new (Algorithm 1, with every
 * certificate exact afterwards, Cor. A.2): eps_t, the ascending frontier from
 * the pre-step certificates, the index rebuild, the chosen strategy's repair,
 * failure marks, H(F_t) and the audit.  eps is the declared step bound (>= 0,
 * finite): the rule always uses the measured eps_t; eps_t > eps*(1+2^-20) only
 * latches CERT_EBOUND.  strategy: cert_strategy.  Stream-ordered, no host
 * synchronisation, no allocation, capturable in a CUDA graph.  out may be NULL. */
cert_status cert_step(cert_ctx *ctx, const float *d_pos_new, float eps, int32_t strategy,
                      cert_views *out, void *stream);

/* The same step with HOST buffers: copies h_pos_new (pinned for full speed)
 * to the device, runs cert_step, copies the per-scene scalars into
 * h_scenes[n_scenes] and synchronises the stream before returning. */
cert_status cert_step_host(cert_ctx *ctx, const float *h_pos_new, float eps, int32_t strategy,
                           cert_scene_result *h_scenes, void *stream);

/* n_steps consecutive steps from HOST frames, with the host-to-device copies
 * pipelined against the steps.  h_frames[k] is step k's positions,
 * [n_total][dim] float32 (pinned for full speed); the pointer table itself is
 * read on the host.  h_scenes should be pinned too: a copy into pageable
 * memory returns only when the step is done, which stops the overlap.
 * Frame k+1 is copied on the context's own copy stream,
 * into the other of two device staging buffers, while step k runs on
 * `stream`.  Step k writes its per-scene scalars into one of two device
 * result slots, and a second copy stream moves them to
 * h_scenes[k * n_scenes ...] (may be NULL) while step k+1 runs; after the
 * last step they are also where cert_sync_result and the views read them.
 * Results equal n_steps calls of cert_step_host.  Each step is replayed from
 * a CUDA graph of cert_step, captured on first use for each parity of the
 * position and staging buffers and captured again when eps, the strategy or
 * a setting that the step reads (cell scale, cell quantile, selector)
 * changes; with phase profiling on, the steps are launched directly.
 * Synchronises `stream` and the copy streams before returning.  Creates the
 * copy and capture streams and the events on first use; allocates no device
 * memory.  Errors:
 * CERT_EINVAL for a NULL table or frame, or n_steps < 0; CERT_ECUDA for a
 * failed copy or launch. */
cert_status cert_step_host_stream(cert_ctx *ctx, const float *const *h_frames, int32_t n_steps, float eps,
                                  int32_t strategy, cert_scene_result *h_scenes, void *stream);

/* Recompute every certificate of the current positions by a full grid search
 * (the O(N) rebuild of Sec. 3).  Step outputs (frontier, failures, H) keep the
 * values of the last step. */
cert_status cert_rebuild(cert_ctx *ctx, void *stream);

/* Views of the current results (no device work). */
cert_status cert_get_views(const cert_ctx *ctx, cert_views *out);

/* Wait for the context's last stream, copy the per-scene scalars to
 * h_scenes[n_scenes] (may be NULL), and return the latched device status
 * (CERT_OK, CERT_EBOUND, CERT_ETIMEOUT or CERT_EINVAL), clearing it. */
cert_status cert_sync_result(cert_ctx *ctx, cert_scene_result *h_scenes);

/* d1 = sqrtf(d1^2), d2 = sqrtf(d2^2) of every current certificate (correctly
 * rounded), written to caller device buffers [n_total]. */
cert_status cert_distances(cert_ctx *ctx, float *d_d1, float *d_d2, void *stream);

/* Exact all-pairs certificates (the paper's brute-force oracle pass, Sec. 3,
 * Table 2) of a single point set d_pos [n][dim] (n >= 3): for each query --
 * every point when d_queries is NULL, else the nq listed indices -- the top-2
 * over all j != query.  Outputs are caller device buffers of length n (or nq).
 * Uses library-managed scratch from the stream-ordered allocator.  The call
 * waits for its stream at the end and returns the status the kernels
 * latched: CERT_EINVAL for a non-finite coordinate, CERT_ETIMEOUT when a
 * bounded bulk-copy wait gave up (in both cases the outputs are not valid),
 * CERT_OK otherwise.  Enqueued inside a stream capture, it cannot wait: it
 * returns CERT_OK and the latched status is not read. */
cert_status cert_allpairs(const float *d_pos, int64_t n, int32_t dim, const int32_t *d_queries,
                          int64_t nq, int32_t *d_nn, float *d_d1sq, float *d_d2sq, void *stream);

/* Search-grid cell side of every scene = scale x (reference d2 of the
 * scene's previous certificates, see cell_quantile); takes effect from the
 * next step.  Only the
 * speed depends on it: certificates are exact for any scale > 0. */
cert_status cert_set_cell_scale(cert_ctx *ctx, float scale);
/* Quantile of the previous d2 (over the first min(n,1024) points, truncated
 * to 3 mantissa bits) that the cell side is a multiple of; in (0, 1]. */
cert_status cert_set_cell_quantile(cert_ctx *ctx, float quantile);
float cert_get_cell_scale(const cert_ctx *ctx);

/* How cert_step runs a step (no counterpart in the paper, which runs one
 * scene's phases as separate GPU passes):
 *   CERT_PATH_MULTI  one kernel per phase over every scene of the batch
 *                    (seven launches and a clear per step; any size);
 *   CERT_PATH_FUSED  one launch per step, one CTA per scene running every
 *                    phase, counters and histograms in shared memory; for
 *                    scenes of at most 16,384 points and 16,384 search-grid
 *                    buckets (next_pow2(n) x bucket_factor), and for every
 *                    strategy but CERT_ALLPAIRS (which always takes the
 *                    multi-kernel path);
 *   CERT_PATH_AUTO   (default) the fused step when no scene has more than
 *                    4,096 points or search-grid buckets -- such a scene's
 *                    sorted points and bucket starts then stay in shared
 *                    memory for the whole step -- and either none has more
 *                    than 2,560 points or the context holds 148 or more
 *                    scenes (a full wave of one CTA per SM); else the
 *                    multi-kernel step (one CTA per larger scene is slower
 *                    than spreading each phase over the GPU).
 * Both paths give the same results bit for bit (every certificate, flag,
 * count and H), except n_searched, which counts the work the refresh left to
 * the search.  cert_set_step_path returns CERT_EINVAL for CERT_PATH_FUSED on a
 * context whose scenes exceed the limits.  Takes effect from the next step. */
typedef enum { CERT_PATH_AUTO = 0, CERT_PATH_MULTI = 1, CERT_PATH_FUSED = 2 } cert_step_path;
cert_status cert_set_step_path(cert_ctx *ctx, int32_t path);
/* The path the next cert_step with this strategy takes (CERT_PATH_MULTI or
 * CERT_PATH_FUSED; -1 for a NULL context). */
int32_t cert_get_step_path(const cert_ctx *ctx, int32_t strategy);

/* Autotuner (the grid cell side of Sec. 2's uniform grid, chosen by timing):
 * for each of the n_scales candidate scales, restore the current state, run
 * one step on frame 0 (it builds the grid at that scale) and time steps on
 * frames 1 .. n_frames-1 with CUDA events; keep the fastest scale, restore
 * the state and write the per-candidate milliseconds to h_ms (may be NULL)
 * and the chosen scale to *h_best (may be NULL).  Frames are device
 * [n_total][dim] float32 arrays at d_frames + f * frame_stride, each within
 * eps of the previous one (the first within eps of the current state).
 * Synchronises; the first call allocates the snapshot buffer. */
cert_status cert_autotune(cert_ctx *ctx, const float *d_frames, int64_t frame_stride, int32_t n_frames,
                          float eps, int32_t strategy, const float *h_scales, int32_t n_scales, float *h_ms,
                          float *h_best, void *stream);

/* Copy the mutable state (positions, extended certificates, per-scene state,
 * the last step's outputs and the search's schedule) aside / put it back, so that several
 * strategies can be run and timed from identical state.  The first
 * cert_snapshot allocates its buffer (about 46 bytes per point); restore
 * without a snapshot returns CERT_ESTATE.  Stream-ordered. */
cert_status cert_snapshot(cert_ctx *ctx, void *stream);
cert_status cert_restore(cert_ctx *ctx, void *stream);

/* Selector features of the last step, h_feat[n_scenes][8] (synchronises):
 * |F|/N, H_cand, ln N, d, ln(1 + eps_t/med_c), touched-cell fraction m_F/C,
 * previous n_failed/max(1,|F|), previous predicted ln t_inc - ln t_reb. */
cert_status cert_get_features(cert_ctx *ctx, float *h_feat);

/* Number of selector parameters: W1[64][8], b1[64], W2[64][64], b2[64],
 * W3[2][64], b3[2] in this order (float32). */
#define CERT_MLP_PARAMS 4866

/* Load the repair-strategy selector (no counterpart in the paper; the
 * crossover it learns is the one Prop. 1 describes): an MLP 8-64-64-2 with
 * ReLU whose outputs predict ln step time of incremental repair and of
 * rebuild.  h_params[CERT_MLP_PARAMS]; h_norm[16] = feature mean[8] then
 * 1/std[8] applied before the first layer.  With a selector loaded,
 * CERT_AUTO picks, per scene and step, the strategy with the smaller
 * prediction (non-finite predictions fall back to the policy).  h_params ==
 * NULL unloads it.  Synchronises.  Never changes results, only the schedule. */
cert_status cert_selector_load(cert_ctx *ctx, const float *h_params, const float *h_norm);

/* Per-scene policy (no counterpart in the paper): h_policy[n_scenes] of
 * CERT_INCREMENTAL / CERT_REBUILD, used by CERT_AUTO in place of
 * cert_config.policy for scenes without a loaded selector's decision, so that
 * the strategy of every scene of a batch can be set by hand (for example to
 * measure what one scene family's choice costs inside the batch).  NULL
 * clears it.  Synchronises; CERT_EINVAL for other values.  Never changes
 * results, only the schedule. */
cert_status cert_set_scene_policy(cert_ctx *ctx, const int32_t *h_policy);

/* Selector training and batch inference on the device (no counterpart in
 * the paper).  X[n][8] raw features, normalised inside the kernels with
 * d_norm[16] (mean[8], 1/std[8]); T[n][2] targets (ln t_inc, ln t_reb);
 * Y[n][2] predictions.  cert_mlp_grad writes the gradient of
 * mean((y - t)^2) over all rows and both outputs into d_grad[CERT_MLP_PARAMS]
 * and the loss into *d_loss (may be NULL); it needs a caller workspace of
 * cert_mlp_workspace_bytes(n) bytes; the gradient is summed in a fixed order
 * (deterministic).  cert_mlp_adam applies one Adam update (Kingma & Ba) with
 * bias correction for step t >= 1.  All three only enqueue work. */
size_t cert_mlp_workspace_bytes(int64_t n);
cert_status cert_mlp_forward(const float *d_params, const float *d_norm, const float *d_X, int64_t n,
                             float *d_Y, void *stream);
cert_status cert_mlp_grad(const float *d_params, const float *d_norm, const float *d_X, const float *d_T,
                          int64_t n, float *d_grad, float *d_loss, void *d_work, size_t work_bytes, void *stream);
cert_status cert_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int32_t t, float lr,
                          float beta1, float beta2, float eps, void *stream);

/* Number of timed phases per step (see cert_profile_end). */
#define CERT_N_PHASES 8

/* Diagnostics: while enabled, cert_step records a CUDA event on its stream
 * before the first and after every phase of the next max_steps steps
 * (phases: 0 clear accumulators, 1 prepare, 2 scans, 3 select, 4 scatter and
 * refresh -- or all-pairs tiles, 5 grid search -- or all-pairs merge,
 * 6 finalize; 7 the fused step, whose one launch runs every phase and leaves
 * phases 0-6 empty, as a multi-kernel step leaves phase 7 empty).  Creates
 * the events here, so the timed steps allocate nothing. */
cert_status cert_profile_begin(cert_ctx *ctx, int32_t max_steps);

/* Stop recording, wait for the recorded steps and write h_ms[step][phase]
 * (milliseconds, CERT_N_PHASES per step) for *n_steps <= max_steps steps. */
cert_status cert_profile_end(cert_ctx *ctx, float *h_ms, int32_t max_steps, int32_t *n_steps);

/* cert_allpairs without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot let a library allocate device memory --
 * a real-time loop whose memory is fixed at start-up, a host whose device
 * memory belongs to another allocator (a framework's caching allocator, a
 * pre-reserved pool), or code that must not wait on the driver's allocator.
 * Same arguments, same results (bit for bit) as cert_allpairs.
 *   - Scratch is one file-scope device array of 32 MiB, held by every GPU that
 *     loads the library until the process exits.  A call needs about
 *     16 n + 24 nq k bytes (k = number of j-chunks, 1 to 64, chosen as in
 *     cert_allpairs but no more than the array holds); every call with
 *     n = nq <= 838,000 fits.  A call that would not fit returns CERT_EINVAL
 *     with the required size in cert_last_error(NULL); nothing is enqueued.
 *   - CUDA loads the library's device code into a context lazily, so the
 *     array's 32 MiB are committed by the driver at the first call on each
 *     device, and that first call can fail with out-of-memory (CERT_ECUDA).
 *     A caller with a fixed memory budget makes one call at start-up, before
 *     any stream capture.  Every call looks up the array's device address
 *     (cudaGetSymbolAddress) with the caller's device current.
 *   - All calls share the array: calls whose work overlaps on the GPU (for
 *     example on two streams at once) race and must be serialised.
 *   - Like cert_allpairs, the call waits for its stream at the end and
 *     returns the latched status: CERT_EINVAL for a non-finite coordinate,
 *     CERT_ETIMEOUT when a bounded bulk-copy wait gave up. */
cert_status cert_allpairs_noalloc(const float *d_pos, int64_t n, int32_t dim, const int32_t *d_queries,
                                  int64_t nq, int32_t *d_nn, float *d_d1sq, float *d_d2sq, void *stream);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * thread spins on a flag that nothing sets, the way a chained-scan tile
 * waits for its predecessor, and gives up after `limit` polls (1 .. 2^24),
 * latching the timeout bit.  Returns CERT_ETIMEOUT when the wait expired as
 * designed (the context stays usable), *h_status = latched bits, *h_spins =
 * polls made.  Synchronises the device; allocates 256 bytes. */
cert_status cert_selftest_bounded_wait(int32_t limit, uint32_t *h_status, uint32_t *h_spins);

/* Release every resource of the context (synchronises it first). */
void cert_destroy(cert_ctx *ctx);

/* Text of the last error on this context (ctx == NULL: of the calling thread). */
const char *cert_last_error(const cert_ctx *ctx);

/* Library version string. */
const char *cert_version(void);

/* Source fingerprint of one translation unit of this build (no counterpart in
 * the paper): the first 16 hex digits of the SHA-256 of the unit's source file
 * and every header, computed by the build.  `unit` is the source's base name
 * without extension ("step_kernels", "fused_step", "allpairs", "knn", "mlp",
 * "api", "allpairs_noalloc").  A profiler measurement of a kernel is valid for the
 * build whose fingerprint it was taken on.  Returns a static string, or NULL
 * for an unknown unit. */
const char *cert_source_fingerprint(const char *unit);

#ifdef __cplusplus
}
#endif

#endif /* CERT_H */
