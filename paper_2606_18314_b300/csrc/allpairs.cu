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

// One staged tile against this thread's kApQ queries (packed in pairs).
template <int DIM, bool CHECK_SELF>
__device__ __forceinline__ void visit_tile(const float4 *s_tile, int len, int jb, const unsigned long long *qx,
                                           const unsigned long long *qy, const unsigned long long *qz,
                                           const int *qi, Top3 *t)
{
    for (int jj = 0; jj < len; ++jj) {
        const float4 c = s_tile[jj];
        const int j = jb + jj;
#pragma unroll
        for (int k = 0; k < kApQ; k += 2) {
            float D0, D1;
            sqdist_qpair<DIM>(qx[k / 2], qy[k / 2], qz[k / 2], c, D0, D1);
            if (D0 < t[k].d2 && (!CHECK_SELF || j != qi[k])) top3_insert(t[k], D0, j);
            if (D1 < t[k + 1].d2 && (!CHECK_SELF || j != qi[k + 1])) top3_insert(t[k + 1], D1, j);
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(kApThreads) k_allpairs(const APArgs a)
{
    __shared__ __align__(128) float4 s_tile[kApTile];
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

    // queries packed pairwise for the f32x2 arithmetic
    unsigned long long qx[kApQ / 2], qy[kApQ / 2], qz[kApQ / 2];
#pragma unroll
    for (int k = 0; k < kApQ / 2; ++k) {
        qx[k] = pack2(qp[2 * k].x, qp[2 * k + 1].x);
        qy[k] = pack2(qp[2 * k].y, qp[2 * k + 1].y);
        qz[k] = pack2(qp[2 * k].z, qp[2 * k + 1].z);
    }
    const int j0 = it.chunk * sp.ap_chunk;
    const int j1 = min(sp.n, j0 + sp.ap_chunk);
    uint32_t phase = 0;
    for (int jt = j0; jt < j1; jt += kApTile) {
        const int len = min(kApTile, j1 - jt);
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar, (uint32_t)len * 16u);
            bulk_copy_g2s(s_tile, a.pos + sp.pt_off + jt, (uint32_t)len * 16u, &s_bar);
        }
        uint32_t spins = 0;
        bool ready;
        while (!(ready = mbar_try_wait(&s_bar, phase)))
            if (++spins > kSpinLimit) break;
        if (!ready) atomicOr(a.status, ST_TIMEOUT);
        if (__syncthreads_or(!ready)) break;
        phase ^= 1u;
        const int jb = sp.pt_off + jt;
        // a tile can hold one of this CTA's own queries only where the index
        // ranges meet (always possible for a query list); elsewhere the
        // self-exclusion test is dropped from the inner loop
        const int qlo = it.qb * kApQBlock;
        const bool own = a.queries != nullptr || (jt < qlo + kApQBlock && jt + len > qlo);
        if (own)
            visit_tile<DIM, true>(s_tile, len, jb, qx, qy, qz, qi, t);
        else
            visit_tile<DIM, false>(s_tile, len, jb, qx, qy, qz, qi, t);
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
    int s = -1, changed = 0, missed = 0, first = 0;
    double dl = 0.0;
    if (valid) {
        s = sa.scene_of[i];
        const SceneParams sp = a.sp[s];
        Top3 t;
        merge_partials(a, sp, sp.n, i - sp.pt_off, t);
        const int n1 = (t.j0 != 0x7fffffff) ? t.j0 - sp.pt_off : -1;
        const int n2 = (t.j1 != 0x7fffffff) ? t.j1 - sp.pt_off : -1;
        changed = n1 != sa.nn[i];
        sa.failed[i] = (uint8_t)changed;
        if (changed) {
            missed = !sa.inF[i];
            const int old = atomicAdd(&sa.hfail[sp.h_off + sa.hcell[i]], 1);
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
    const double sd = run_sum_f64(m, dl);
    if (s >= 0 && run_leader(m)) {
        atomicAdd(&sa.acc[s].n_searched, nsr);
        if (nc) {
            atomicAdd(&sa.acc[s].n_failed, nc);
            atomicAdd(&sa.acc[s].n_missed, nm);
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

}  // namespace certk
