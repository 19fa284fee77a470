/*
 * cert_knn.h -- C ABI of libcert.so, k-nearest-neighbour certificates: the
 * exact k nearest neighbours of every point (a kNN graph), maintained on one
 * GPU while the points move by small steps.
 *
 * Paper: "Repair Entropy in Dynamic Geometric Nearest-Neighbour Structures".
 * The paper studies the k = 2 certificate (nn_i, d1_i, d2_i) and leaves richer
 * certificates, k-nearest-neighbour graphs among them, open (Sec. 6).  This is
 * the same method one rank further out:
 *   certificate of point i: its k nearest neighbours, ordered by the key
 *   (D, j) (squared distance, then index), and the clearance
 *   c^(k)_i = d_{k+1,i} - d_{k,i} (k = 1 is Def. 1's c_i = d2_i - d1_i) ..... Def. 1
 *   safety rule: every distance from i changes by at most 2 eps_t in a step,
 *   so the SET of the k nearest is unchanged while c^(k)_i > 4 eps_t ........ Lemma 1
 *   one step: eps_t, the frontier {c^(k) <= 4 eps_t + tau}, the index
 *   rebuild, repair of every certificate the bound L below cannot prove ..... Algorithm 1
 *   exactness of a search box: a key is final once it is below the squared
 *   distance to every face of the box that is not on the grid edge ......... Cor. A.2
 *
 * The conventions of cert.h hold (device positions [n][dim] float32 in the
 * unit domain, points outside it clamped into the boundary cells; FP32 fixed
 * order distances; lowest index first among equal keys; stream-ordered calls
 * that never synchronise unless documented; argument errors returned at once,
 * device conditions latched and returned by cert_knn_sync_result).  A
 * context has no error text of its own: after a failed call,
 * cert_last_error(NULL) gives the calling thread's last message.
 *
 * A context holds one point set (one scene).  Everything it allocates is
 * allocated by cert_knn_init; cert_knn_step allocates nothing, never
 * synchronises and can be captured in a CUDA graph.  Steps alternate between
 * two internal position buffers: a graph replays correctly when the context
 * has taken an even number of steps since the capture began (capture two
 * steps, and keep any steps between replays even in number).
 */
#ifndef CERT_KNN_H
#define CERT_KNN_H

#include <stdint.h>

#include "cert.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CERT_KNN_MAX_K 16

typedef struct cert_knn_ctx cert_knn_ctx;

typedef struct {
    int32_t dim;          /* 2 or 3                                                     */
    int32_t k;            /* neighbours per point, 1 .. CERT_KNN_MAX_K                  */
    int64_t n;            /* points, k + 2 <= n < 2^31                                   */
    float cell_scale;     /* grid cell side = cell_scale x the median (k+1)-th distance of
                             a 1024-point sample of the previous step (0 -> 1.0); the
                             first grid assumes a uniform set in the unit domain.  The
                             grid is hashed into next_pow2(n) buckets (at most 2^24),
                             so any resolution up to 2048 cells per axis fits          */
    int32_t reserved;     /* must be zero                                               */
} cert_knn_config;

/* Per-step scalars.  Same layout on device and host. */
typedef struct {
    float eps_t;          /* measured max_i |p'_i - p_i|                                 */
    int32_t n_frontier;   /* #{i : c^(k)_i <= 4 eps_t + tau_i}, tau_i = 2^-20 ((d_k + d_{k+1}) + eps_t),
                             from the pre-step certificates                              */
    int32_t n_failed;     /* #{i : the set of the k nearest of i changed}                */
    int32_t n_missed;     /* failed but not in the frontier (Lemma 1: always 0)          */
    int32_t n_false;      /* in the frontier but not failed                               */
    int32_t n_searched;   /* certificates recomputed by a search this step (grid or, for
                             the few whose box would be too large, every point)       */
    int32_t grid_res;     /* grid cells per axis (the fine level)                         */
    int32_t strategy;     /* CERT_INCREMENTAL or CERT_REBUILD                              */
    int32_t grid_res_coarse; /* cells per axis of the coarse level, 0 when the grid had one  */
    int32_t n_far;        /* searches whose box was too large, done over every point       */
} cert_knn_result;

/* Device views, valid until the next call on the context.  The lists are
 * rank-major: entry r of point i is at [r * n + i]; ranks 0 .. k hold the
 * k nearest and the (k+1)-th, which fixes the clearance (two further ranks
 * follow in the same arrays: spare candidates for the refresh, not exact). */
typedef struct {
    const int32_t *idx;      /* [k+1][n] neighbour indices, ascending key (D, j)      */
    const float *d2;         /* [k+1][n] their squared distances                       */
    const uint8_t *frontier; /* [n] 1 where c^(k)_i <= 4 eps_t + tau_i this step        */
    const uint8_t *failed;   /* [n] 1 where the set of the k nearest changed this step  */
    const cert_knn_result *result; /* device copy of the scalars                       */
    int64_t n;
    int32_t k, dim;
} cert_knn_views;

/* Create a context and compute the exact k+1 nearest neighbours of every
 * point of d_pos (device [n][dim] float32) by a full grid search.  Validates
 * cfg (dim, k, n, cell_scale >= 0 and finite, reserved == 0) before touching the
 * device.  On error *out is NULL. */
cert_status cert_knn_init(cert_knn_ctx **out, const cert_knn_config *cfg, const float *d_pos, void *stream);

/* One step to positions d_pos_new (device [n][dim] float32): eps_t, the
 * frontier from the pre-step certificates, the grid rebuild, then, for
 * strategy CERT_INCREMENTAL, an O(k) refresh of every certificate whose lower
 * bound L still proves it (L_i <- L_i - (|p'_i - p_i| + eps_t) with upward
 * rounding slack, as in the k = 2 path) and a grid search of the rest; for
 * CERT_REBUILD a grid search of every point.  Failure marks and the audit.
 * eps is the declared bound (>= 0, finite); eps_t > eps (1 + 2^-20) only
 * latches CERT_EBOUND.  Other strategies are rejected (CERT_EINVAL). */
cert_status cert_knn_step(cert_knn_ctx *ctx, const float *d_pos_new, float eps, int32_t strategy, void *stream);

/* Diagnostics: the same step as cert_knn_step, with CUDA events between its
 * phases; synchronises and writes the phase times in ms to h_ms[5]: prepare
 * (displacement, eps_t, cells), scan (cell starts), refresh (scatter,
 * frontier, O(k) refresh), search, finalize.  Not capturable. */
cert_status cert_knn_profile(cert_knn_ctx *ctx, const float *d_pos_new, float eps, int32_t strategy, float *h_ms,
                             void *stream);

/* Pointers to the current lists and flags (no device work). */
cert_status cert_knn_get_views(const cert_knn_ctx *ctx, cert_knn_views *out);

/* Synchronise the context's last stream, copy the scalars of the last step to
 * *out (may be NULL) and return, then clear, the latched device status. */
cert_status cert_knn_sync_result(cert_knn_ctx *ctx, cert_knn_result *out);

/* Release everything; NULL is a no-op. */
void cert_knn_destroy(cert_knn_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CERT_KNN_H */
