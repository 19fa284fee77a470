// allpairs.cu -- exact all-pairs top-2 (the paper's brute-force oracle pass,
// "rtx_full_rebuild" / "rtx_frontier_oracle" of Sec. 3, throughput in Table 2).
//
// Each CTA owns (scene, block of 512 queries, one j-chunk).  The chunk's
// coordinates are staged into shared memory 2048 points at a time by a TMA bulk
// copy (cp.async.bulk + mbarrier), every thread keeps the running top-3 of its
// four queries in registers, and candidates are visited in ascending index so
// a strict '<' realises the lowest-index tie-break inside a chunk.  Distances
// of a candidate to two queries come from one packed FP32 pair operation
// (f32x2 differences and squares, scalar additions; bit-identical).  Chunks are
// merged afterwards in chunk order with the full lexicographic key, which
// gives a deterministic result independent of how the j-range was split.
// The work is plain FP32 arithmetic (no tensor cores: the inner dimension is
// d <= 3 and the fixed rounding order forbids the |x|^2 + |y|^2 - 2xy form).
#include <algorithm>

#include "cert_internal.cuh"
#include "cert_launch.h"

namespace certk {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Candidates staged per TMA copy; the staged tile is rewritten as candidate
// pairs (xa, xb, ya, yb) and (za, zb), so that one 16-byte and one 8-byte
// shared load give each coordinate of two candidates as one f32x2 operand.
constexpr int kApStage = 1024;

// Squared distances of two candidates (coordinates packed pairwise: cx =
// {xa, xb}, ...) to the query whose coordinates are packed twice (px = {x,
// x}, ...): packed differences and squares, scalar additions -- bit-identical
// to sqdist<DIM>(query, candidate) for each candidate.
template <int DIM>
__device__ __forceinline__ void sqdist_cpair(unsigned long long px, unsigned long long py, unsigned long long pz,
                                             unsigned long long cx, unsigned long long cy, unsigned long long cz,
                                             float &Da, float &Db)
{
    unsigned long long dx, dy;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(cx), "l"(px));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(cy), "l"(py));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(dx) : "l"(dx));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(dy) : "l"(dy));
    float xa, xb, ya, yb;
    unpack2(dx, xa, xb);
    unpack2(dy, ya, yb);
    Da = __fadd_rn(xa, ya);
    Db = __fadd_rn(xb, yb);
    if (DIM == 3) {
        unsigned long long dz;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(cz), "l"(pz));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(dz) : "l"(dz));
        float za, zb;
        unpack2(dz, za, zb);
        Da = __fadd_rn(Da, za);
        Db = __fadd_rn(Db, zb);
    }
}

// One converted tile (npair candidate pairs, the first with index jb) against
// this thread's kApQ queries.  Candidates are visited in ascending index, so
// the strict '<' keeps the lowest index among equal distances.
template <int DIM, bool CHECK_SELF>
__device__ __forceinline__ void visit_pairs(const float4 *s_xy, const float2 *s_z, int npair, int jb,
                                            const unsigned long long *px, const unsigned long long *py,
                                            const unsigned long long *pz, const int *qi, Top3 *t)
{
    for (int pp = 0; pp < npair; ++pp) {
        const float4 xy = s_xy[pp];
        const float2 zz = (DIM == 3) ? s_z[pp] : make_float2(0.f, 0.f);
        const unsigned long long cx = pack2(xy.x, xy.y), cy = pack2(xy.z, xy.w), cz = pack2(zz.x, zz.y);
        const int ja = jb + 2 * pp, jn = ja + 1;
#pragma unroll
        for (int k = 0; k < kApQ; ++k) {
            float Da, Db;
            sqdist_cpair<DIM>(px[k], py[k], pz[k], cx, cy, cz, Da, Db);
            if (fminf(Da, Db) < t[k].d2) {
                if (Da < t[k].d2 && (!CHECK_SELF || ja != qi[k])) top3_insert(t[k], Da, ja);
                if (Db < t[k].d2 && (!CHECK_SELF || jn != qi[k])) top3_insert(t[k], Db, jn);
            }
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(kApThreads) k_allpairs(const APArgs a)
{
    __shared__ __align__(128) float4 s_tile[kApStage];        // TMA staging (x, y, z, w) per candidate
    __shared__ __align__(16) float4 s_xy[kApStage / 2];       // (xa, xb, ya, yb) per candidate pair
    __shared__ __align__(16) float2 s_z[kApStage / 2];        // (za, zb)
    __shared__ __align__(8) uint64_t s_bar;

    APItem it;
    if (a.items) {
        it = a.items[blockIdx.x];
    } else {
        it.s = 0;
        it.qb = blockIdx.x % a.nqb;
        it.chunk = blockIdx.x / a.nqb;
    }
    const SceneParams sp = a.sp[it.s];
    const int nq = a.queries ? a.nq_list : sp.n;

    float4 qp[kApQ];
    int qi[kApQ];
    Top3 t[kApQ];
#pragma unroll
    for (int k = 0; k < kApQ; ++k) {
        const int q = it.qb * kApQBlock + k * kApThreads + threadIdx.x;
        int loc = -1;
        if (q < nq) loc = a.queries ? a.queries[q] : q;
        const bool ok = (unsigned)loc < (unsigned)sp.n;
        qi[k] = ok ? sp.pt_off + loc : -1;
        qp[k] = ok ? a.pos[sp.pt_off + loc] : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        top3_reset(t[k]);
    }
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // each query's coordinates packed twice for the f32x2 arithmetic
    unsigned long long px[kApQ], py[kApQ], pz[kApQ];
#pragma unroll
    for (int k = 0; k < kApQ; ++k) {
        px[k] = pack2(qp[k].x, qp[k].x);
        py[k] = pack2(qp[k].y, qp[k].y);
        pz[k] = pack2(qp[k].z, qp[k].z);
    }
    const int j0 = it.chunk * sp.ap_chunk;
    const int j1 = min(sp.n, j0 + sp.ap_chunk);
    const int qlo = it.qb * kApQBlock;
    uint32_t phase = 0;
    // the first tile's copy; each later one is issued once the previous tile
    // has been converted, so it overlaps the distance work
    if (threadIdx.x == 0 && j0 < j1) {
        const int len = min(kApStage, j1 - j0);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar, (uint32_t)len * 16u);
        bulk_copy_g2s(s_tile, a.pos + sp.pt_off + j0, (uint32_t)len * 16u, &s_bar);
    }
    for (int jt = j0; jt < j1; jt += kApStage) {
        const int len = min(kApStage, j1 - jt);
        uint32_t spins = 0;
        bool ready;
        while (!(ready = mbar_try_wait(&s_bar, phase)))
            if (++spins > kSpinLimit) break;
        if (!ready) atomicOr(a.status, ST_TIMEOUT);
        if (__syncthreads_or(!ready)) break;
        phase ^= 1u;
        // staged candidates -> pairs; an odd tail is paired with a NaN candidate
        const int npair = (len + 1) >> 1;
        for (int pp = threadIdx.x; pp < npair; pp += kApThreads) {
            const float4 ca = s_tile[2 * pp];
            const float4 cb = (2 * pp + 1 < len) ? s_tile[2 * pp + 1]
                                                 : make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                                                               __int_as_float(0x7fc00000), 0.f);
            s_xy[pp] = make_float4(ca.x, cb.x, ca.y, cb.y);
            s_z[pp] = make_float2(ca.z, cb.z);
        }
        __syncthreads();
        if (threadIdx.x == 0 && jt + kApStage < j1) {
            const int ln = min(kApStage, j1 - jt - kApStage);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar, (uint32_t)ln * 16u);
            bulk_copy_g2s(s_tile, a.pos + sp.pt_off + jt + kApStage, (uint32_t)ln * 16u, &s_bar);
        }
        const int jb = sp.pt_off + jt;
        // a tile can hold one of this CTA's own queries only where the index
        // ranges meet (always possible for a query list); elsewhere the
        // self-exclusion test is dropped from the inner loop
        const bool own = a.queries != nullptr || (jt < qlo + kApQBlock && jt + len > qlo);
        if (own)
            visit_pairs<DIM, true>(s_xy, s_z, npair, jb, px, py, pz, qi, t);
        else
            visit_pairs<DIM, false>(s_xy, s_z, npair, jb, px, py, pz, qi, t);
        __syncthreads();
    }

#pragma unroll
    for (int k = 0; k < kApQ; ++k) {
        const int q = it.qb * kApQBlock + k * kApThreads + threadIdx.x;
        if (q < nq) {
            const long long slot = (long long)sp.ap_off + (long long)it.chunk * nq + q;
            a.pd[slot] = t[k].d0;
            a.pd[a.P + slot] = t[k].d1;
            a.pd[2 * a.P + slot] = t[k].d2;
            a.pj[slot] = t[k].j0;
            a.pj[a.P + slot] = t[k].j1;
            a.pj[2 * a.P + slot] = t[k].j2;
        }
    }
}

__device__ __forceinline__ void merge_partials(const APArgs &a, const SceneParams &sp, int nq, int q, Top3 &t)
{
    top3_reset(t);
    for (int c = 0; c < sp.ap_nch; ++c) {
        const long long slot = (long long)sp.ap_off + (long long)c * nq + q;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int j = a.pj[r * a.P + slot];
            if (j != 0x7fffffff) top3_insert(t, a.pd[r * a.P + slot], j);
        }
    }
}

// ABI mode: one thread per query of scene 0.
__global__ void k_allpairs_merge_abi(const APArgs a, const APMergeOut o)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.nq_list) return;
    const SceneParams sp = a.sp[0];
    const int loc = a.queries ? a.queries[q] : q;
    if ((unsigned)loc >= (unsigned)sp.n) {
        o.nn[q] = -1;
        o.d1sq[q] = __int_as_float(0x7fc00000);
        o.d2sq[q] = __int_as_float(0x7fc00000);
        return;
    }
    Top3 t;
    merge_partials(a, sp, a.nq_list, q, t);
    o.nn[q] = (t.j0 != 0x7fffffff) ? t.j0 - sp.pt_off : -1;
    o.d1sq[q] = t.d0;
    o.d2sq[q] = t.d1;
}

// Step mode: one thread per point of every scene; writes the extended
// certificate and the failure audit exactly as the grid search does.
__global__ void k_allpairs_merge_step(const APArgs a, const APMergeOut o)
{
    const StepArgs &sa = o.step;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < sa.n_total;
    int s = -1, changed = 0, missed = 0, first = 0, hit = 0;
    double dl = 0.0;
    if (valid) {
        s = sa.scene_of[i];
        const SceneParams sp = a.sp[s];
        Top3 t;
        merge_partials(a, sp, sp.n, i - sp.pt_off, t);
        const int n1 = (t.j0 != 0x7fffffff) ? t.j0 - sp.pt_off : -1;
        const int n2 = (t.j1 != 0x7fffffff) ? t.j1 - sp.pt_off : -1;
        CERT_CHECK(sa.status, (unsigned)n1 < (unsigned)sp.n && (unsigned)n2 < (unsigned)sp.n);
        changed = n1 != sa.nn[i];
        sa.failed[i] = (uint8_t)changed;
        if (changed) {
            const uint32_t fl = sa.inF[i];   // bit 0: in F_t, bit 1: rho-flagged
            missed = !(fl & 1u);
            hit = (int)(fl >> 1);
            const int old = count_inc(sa.hfail, sp.h_off + sa.hcell[i], sa.c16h);
            first = old == 0;
            dl = nlogn_step(sa.nlogn, old);
        }
        sa.nn[i] = n1;
        sa.nn2[i] = n2;
        sa.nn3[i] = (t.j2 != 0x7fffffff) ? t.j2 - sp.pt_off : -1;
        sa.d1sq[i] = t.d0;
        sa.d2sq[i] = t.d1;
        sa.L[i] = sqrt_lower(t.d2);   // every point beyond the top-3 is at least this far
    }
    const unsigned m = scene_run_mask(s);
    const int nsr = run_sum_i32(m, valid ? 1 : 0);
    const int nc = run_sum_i32(m, changed);
    const int nm = run_sum_i32(m, missed);
    const int fc = run_sum_i32(m, first);
    const int nh = run_sum_i32(m, hit);
    const double sd = run_sum_f64(m, dl);
    if (s >= 0 && run_leader(m)) {
        atomicAdd(&sa.acc[s].n_searched, nsr);
        if (nc) {
            atomicAdd(&sa.acc[s].n_failed, nc);
            atomicAdd(&sa.acc[s].n_missed, nm);
            if (nh) atomicAdd(&sa.acc[s].n_rho_hit, nh);
            atomicAdd(&sa.acc[s].failed_cells, fc);
            atomicAdd(&sa.acc[s].s_fail, sd);
        }
    }
}

template <int DIM>
__global__ void k_pack(const float *pos, int n, float4 *out, uint32_t *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *q = pos + (size_t)i * DIM;
    const float4 p = make_float4(q[0], q[1], DIM == 3 ? q[2] : 0.0f, 0.0f);
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) atomicOr(status, ST_NONFINITE);
    out[i] = p;
}

// j-chunks for one point set of n candidates: the count that minimises the
// time of the grid, modelled as (waves of resident CTAs) x (chunk length +
// a fixed cost of kApChunkFixed candidates per CTA); ties go to fewer chunks
// (a smaller merge).
int allpairs_chunks_for(long long qblocks, long long n, int dim, int cap)
{
    constexpr long long kApChunkFixed = 256;
    int dev = 0, sms = 1, bps = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        sms = 148;
    const cudaError_t e = (dim == 3) ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_allpairs<3>, kApThreads, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_allpairs<2>, kApThreads, 0);
    if (e != cudaSuccess || bps < 1) bps = 1;
    const long long wave = (long long)sms * bps;
    cap = std::max(1, std::min(cap, 64));
    int best = 1;
    long long best_cost = -1;
    for (int nch = 1; nch <= cap; ++nch) {
        const long long waves = (qblocks * nch + wave - 1) / wave;
        const long long cost = waves * ((n + nch - 1) / nch + kApChunkFixed);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = nch;
        }
    }
    return best;
}

int allpairs_chunks(long long qblocks, int dim, int cap)
{
    // j-chunks per query block so that the grid fills whole waves of resident
    // CTAs: the smallest count giving at least one full wave at >= 90% of the
    // last wave, else the best fill found
    int dev = 0, sms = 1, bps = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        sms = 148;
    const cudaError_t e = (dim == 3) ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_allpairs<3>, kApThreads, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_allpairs<2>, kApThreads, 0);
    if (e != cudaSuccess || bps < 1) bps = 1;
    const long long wave = (long long)sms * bps;
    cap = std::max(1, std::min(cap, 64));
    int best = 1;
    double best_fill = -1.0;
    for (int nch = 1; nch <= cap; ++nch) {
        const long long ctas = qblocks * nch;
        const long long waves = (ctas + wave - 1) / wave;
        const double fill = (double)ctas / (double)(waves * wave);
        if (ctas >= wave && fill >= 0.9) return nch;
        if (fill > best_fill + 1e-9) {
            best_fill = fill;
            best = nch;
        }
    }
    return best;
}

cudaError_t launch_allpairs(const APArgs &a, cudaStream_t st)
{
    if (a.n_items <= 0) return cudaSuccess;
    if (a.dim == 3)
        k_allpairs<3><<<a.n_items, kApThreads, 0, st>>>(a);
    else
        k_allpairs<2><<<a.n_items, kApThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_allpairs_merge(const APArgs &a, const APMergeOut &o, long long n_queries_total, cudaStream_t st)
{
    const int blocks = (int)((n_queries_total + 255) / 256);
    if (blocks <= 0) return cudaSuccess;
    if (o.step_mode)
        k_allpairs_merge_step<<<blocks, 256, 0, st>>>(a, o);
    else
        k_allpairs_merge_abi<<<blocks, 256, 0, st>>>(a, o);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *pos, int n, int dim, float4 *out, uint32_t *status, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256;
    if (dim == 3)
        k_pack<3><<<blocks, 256, 0, st>>>(pos, n, out, status);
    else
        k_pack<2><<<blocks, 256, 0, st>>>(pos, n, out, status);
    return cudaGetLastError();
}

cudaError_t allpairs_status_read(const uint32_t *d_status, uint32_t *h_status, bool *read, cudaStream_t st)
{
    *read = false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
    e = cudaMemcpyAsync(h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *read = e == cudaSuccess;
    return e;
}

cert_status allpairs_status_code(uint32_t st)
{
    const char *msg = nullptr;
    cert_status code = CERT_OK;
    if (st & ST_INDEX) {
        code = CERT_EINTERNAL;
        msg = "cert_allpairs: an internal index check failed (debug build)";
    } else if (st & ST_TIMEOUT) {
        code = CERT_ETIMEOUT;
        msg = "cert_allpairs: a bounded bulk-copy wait gave up; the results are not valid";
    } else if (st & ST_NONFINITE) {
        code = CERT_EINVAL;
        msg = "cert_allpairs: non-finite coordinate in the positions; the results are not valid";
    }
    if (msg) record_thread_error(msg);
    return code;
}

}  // namespace certk
