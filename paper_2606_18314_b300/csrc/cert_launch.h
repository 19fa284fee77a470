// cert_launch.h -- argument blocks and launch wrappers shared by the
// translation units of libcert.so (host code calls these; kernels live in
// step_kernels.cu, allpairs.cu and mlp.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cert.h"

namespace certk {

struct SceneParams;
struct SceneState;
struct SceneAcc;

enum : int { PH_PREPARE = 0, PH_SCAN, PH_SELECT, PH_SCATTER, PH_SEARCH, PH_FINALIZE };

// Everything a step kernel may touch.  Passed by value as a kernel parameter.
struct StepArgs {
    int mode;                      // MODE_INIT / MODE_STEP / MODE_REBUILD
    int dim;
    int n_total, n_scenes;
    const float *pos_in;           // caller positions [n][dim] (INIT, STEP)
    const float4 *pos_old;         // previous positions (STEP)
    float4 *pos_new;               // positions of this step (written in INIT/STEP)
    const int32_t *scene_of;       // [n] scene of every point
    const SceneParams *sp;
    SceneState *st;
    SceneAcc *acc;
    uint32_t *status;
    // hashed search grid (counting sort by bucket)
    int32_t *bucket_count;         // [n_buckets_pad]
    int32_t *bucket_start;         // [n_buckets_pad]
    int2 *brank;                   // [n] (bucket, rank in bucket)
    float4 *squad;                 // points in bucket order, quad layout (sorted_store), padded per scene
    uint32_t *mgrid;               // [n_scenes][kMotionStride] max squared displacement per motion cell (bits)
    uint32_t *mdil;                // [n_scenes][kMotionStride] its dilation by one cell
    uint8_t *sflag;                // [n_pad] by sorted slot: 1 = search this point
    int32_t *far_list;             // [n] sorted slots left to the far pass
    int32_t *chunk_cnt;            // [n_chunks] queries each batch search chunk had (kept for the next step)
    int32_t *chunk_order;          // [n_chunks] the search's CTA -> chunk map, heaviest chunks first
    int order_chunks;              // k_prepare's first CTA orders this many chunks (0: the search is unordered)
    int32_t *far_count;            // number of entries in far_list (zeroed by k_prepare)
    // certificates
    int frontier_rule;             // cert_frontier_rule
    int audit;                     // cert_audit flags: rho (inF bit 1), geometry (position sums)
    double *clk_s;                 // clock rule, per point: clock of the last revisit
    float *clk_c, *clk_g;          // ... and c, d1 + d2 of the certificate then
    int32_t *nn, *nn2, *nn3;       // nearest, runner-up, third stored candidate (-1: none)
    float *d1sq, *d2sq, *L;        // L: lower bound on the distance to every other point
    // step outputs
    int32_t *hcell, *hfail, *hcand;  // entropy cell per point; failures and frontier points per cell
    int c16b, c16h;                // 16-bit counts (count_inc): bucket_count; hfail and hcand
    uint32_t *hocc;                // occupied entropy cells, one bit per cell (global index h_off + cell)
    uint8_t *inF, *failed;         // inF bit 0: in F_t; bit 1: rho-flagged (CERT_AUDIT_RHO)
    int32_t *frontier, *fstart;
    // chained-scan state
    uint64_t *tstat_b, *tstat_p;
    uint32_t *tile_ctr;            // chained scans' tile tickets (zeroed by k_prepare)
    int ntiles_b, ntiles_p;
    // Counters that k_prepare, k_scan and k_select accumulate (the scan tile
    // states, bucket counts, occupancy, frontier-cell and motion grids): one
    // 16-byte-aligned span that k_search zeroes for the next call once they
    // are dead.  hfail is zeroed per scene by k_select, acc[s] by k_finalize
    // after reading it; so every call that ends with k_search and k_finalize
    // leaves them all zero and the next step needs no memset.
    int4 *ztail;
    long long ztail_n16;           // 16-byte words of the span
    const double *nlogn;
    cert_scene_result *res;
    float declared_eps;
    int strategy, policy;
    float cell_scale;
    float cell_quantile;
    const int32_t *scene_policy;   // [n_scenes] strategy of each scene under AUTO without a selector (NULL: policy)
    const float *sel_params;       // selector weights (NULL: none loaded)
    const float *sel_norm;         // feature mean[8], 1/std[8] (NULL: none loaded)
    float *feat;                   // [n_scenes][8] selector features of the last step
};

cudaError_t launch_step_phase(const StepArgs &a, int phase, cudaStream_t st);

// ---------------------------------------------------------------- fused step

// Limits of the fused step (one CTA runs every phase of one scene, counters in
// shared memory; fused_step.cu): points per scene, search-grid buckets per
// scene (16-bit counters), entropy-grid cells per scene (26^3), row-range
// table entries per thread.
constexpr int kFusedMaxN = 16384;
constexpr int kFusedMaxBuckets = 16384;
constexpr int kFusedMaxHCells = 17576;
constexpr int kFusedRows = 9;
// Scenes of at most this many points keep their sorted points and bucket
// starts in shared memory during a fused step.
constexpr int kFusedResMaxN = 4096;
// One step of every scene (MODE_STEP, any strategy but all-pairs) in one
// launch: CTA b runs scene order[b] (order may be NULL: scene b), block =
// 512 or 1024 threads.  resident: every scene has at most kFusedResMaxN points
// and search-grid buckets, so its sorted points and bucket starts are kept in
// shared memory (1024 threads; block is ignored).
cudaError_t launch_fused_step(const StepArgs &a, const int32_t *order, int block, bool resident, cudaStream_t st);
cudaError_t launch_distances(const float *d1sq, const float *d2sq, float *d1, float *d2, int n,
                             cudaStream_t st);

// ---------------------------------------------------------------- all-pairs

// Work item of the all-pairs kernel: scene, query block, j-chunk.
struct APItem {
    int32_t s, qb, chunk, pad;
};

struct APArgs {
    int dim;
    const float4 *pos;             // points in index order
    const SceneParams *sp;         // per scene: pt_off, n, ap_off, ap_nch, ap_chunk
    const APItem *items;           // one per block; NULL: scene 0, item = (b % nqb, b / nqb)
    int n_items;
    int nqb;                       // query blocks of scene 0 when items == NULL
    const int32_t *queries;        // NULL: every point of each scene; else list (scene 0, local indices)
    int nq_list;                   // length of the list
    float *pd;                     // partial keys [3][P]
    int32_t *pj;                   // partial indices [3][P]
    long long P;
    uint32_t *status;
};

// Outputs of the merge: ABI mode writes (nn, d1^2, d2^2) of each query; step
// mode writes the full extended certificate of every point plus the audit.
struct APMergeOut {
    int32_t *nn;
    float *d1sq, *d2sq;
    int step_mode;                 // 1: StepArgs fields below are used
    StepArgs step;
};

constexpr int kApThreads = 128;
constexpr int kApQ = 4;                        // queries per thread
constexpr int kApQBlock = kApThreads * kApQ;   // queries per block
constexpr int kApTile = 2048;                  // candidates staged per shared-memory tile

cudaError_t launch_allpairs(const APArgs &a, cudaStream_t st);
// j-chunks per query block that fill whole waves of resident k_allpairs CTAs (1 <= result <= cap).
int allpairs_chunks(long long qblocks, int dim, int cap);
int allpairs_chunks_for(long long qblocks, long long n, int dim, int cap);
cudaError_t launch_allpairs_merge(const APArgs &a, const APMergeOut &o, long long n_queries_total,
                                  cudaStream_t st);
cudaError_t launch_pack(const float *pos, int n, int dim, float4 *out, uint32_t *status, cudaStream_t st);
// Wait for the all-pairs work on st and copy its latched status word to *h_status
// (*read = true).  A stream under capture cannot be waited on: then nothing is
// read (*read = false) and the capture is left intact.
cudaError_t allpairs_status_read(const uint32_t *d_status, uint32_t *h_status, bool *read, cudaStream_t st);
// cert_status of latched status bits: a failed debug check, a wait that gave up,
// a non-finite coordinate, in this order of precedence; CERT_OK for none.
cert_status allpairs_status_code(uint32_t st);

// Sets the text cert_last_error(NULL) returns on the calling thread.
void record_thread_error(const char *msg);

}  // namespace certk
