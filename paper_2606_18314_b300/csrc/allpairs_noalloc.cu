// allpairs_noalloc.cu -- cert_allpairs for callers that cannot allocate.
//
// cert_allpairs takes its scratch (packed coordinates and the per-chunk
// partial top-3 lists) from the stream-ordered allocator on every call.  Some
// callers cannot let a library allocate device memory: a real-time loop whose
// memory budget is fixed at start-up, a host whose device memory is owned by
// another allocator (a framework's caching allocator or a pre-reserved pool),
// or code that must never wait on the driver's allocator.  This variant runs
// the same kernels with its scratch in one file-scope device array of fixed
// size, so a call allocates nothing.
//
// The array is a static __device__ symbol: every GPU that loads the library
// holds kNoAllocScratchBytes of it until the process exits.  CUDA loads a
// module into a context lazily, so the array's memory is committed by the
// driver when this module first loads on a device -- at the first call on
// that device, in the address lookup below.  That first call can therefore
// fail with out-of-memory (CERT_ECUDA); a caller with a fixed memory budget
// makes it at start-up, and makes it before any stream capture.  Host code
// cannot use the symbol's name as a device address, so every call looks the
// address up with cudaGetSymbolAddress, with the caller's device current.
// All calls share the one array and it keeps the last call's contents: the
// status word is cleared on every call and every partial slot a call reads is
// written by the same call.  Calls whose work overlaps on the GPU (two streams
// at once) race on the array; serialise them.  The call waits for its stream
// at the end and returns the status the kernels latched (a non-finite
// coordinate, a bulk-copy wait that gave up).
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "cert_internal.cuh"
#include "cert_launch.h"

namespace certk {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

__global__ void k_noalloc_write_params(SceneParams *dst, SceneParams v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

// Device address of the scratch array in the current device's context.  It is
// looked up on every call rather than cached per device ordinal: after a
// cudaDeviceReset the module is loaded again into a new context, and an
// address cached from the old one would no longer be mapped.  Once the module
// is loaded the lookup is a table read.
static cudaError_t noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace certk

using namespace certk;

static cert_status noalloc_fail(cert_status code, const char *msg)
{
    record_thread_error(msg);
    return code;
}

extern "C" cert_status cert_allpairs_noalloc(const float *d_pos, int64_t n, int32_t dim, const int32_t *d_queries,
                                             int64_t nq, int32_t *d_nn, float *d_d1sq, float *d_d2sq,
                                             void *stream)
{
    if (!d_pos || !d_nn || !d_d1sq || !d_d2sq) return noalloc_fail(CERT_EINVAL, "NULL argument");
    if (dim != 2 && dim != 3) return noalloc_fail(CERT_EINVAL, "dim must be 2 or 3");
    if (n < 3 || n >= (int64_t(1) << 30)) return noalloc_fail(CERT_EINVAL, "need 3 <= n < 2^30");
    if (!d_queries) nq = n;
    if (nq < 0 || nq >= (int64_t(1) << 30)) return noalloc_fail(CERT_EINVAL, "bad query count");
    if (nq == 0) return CERT_OK;

    // Same decomposition as cert_allpairs (512 queries per CTA, the j-chunk
    // count from the same wave-time model), with the chunk count also capped by
    // the scratch it needs.
    const int64_t nqb = (nq + kApQBlock - 1) / kApQBlock;
    const int64_t room = (int64_t)kNoAllocScratchBytes - (int64_t)align256(size_t(n) * sizeof(float4)) - 4096;
    const int64_t fit = room > 0 ? room / (nq * int64_t(6 * sizeof(float))) : 1;
    const int64_t nch = allpairs_chunks_for(nqb, n, dim, (int)std::max<int64_t>(
                                                      1, std::min<int64_t>({fit, (n + 255) / 256, int64_t(64)})));
    const long long P = (long long)nq * nch;
    const size_t o_pos = 0;
    const size_t o_sp = align256(o_pos + size_t(n) * sizeof(float4));
    const size_t o_st = align256(o_sp + sizeof(SceneParams));
    const size_t o_pd = align256(o_st + 16);
    const size_t o_pj = align256(o_pd + size_t(3) * P * sizeof(float));
    const size_t need = align256(o_pj + size_t(3) * P * sizeof(int32_t));
    if (need > kNoAllocScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "cert_allpairs_noalloc: n=%lld, nq=%lld needs %zu bytes of scratch; the static array holds %zu",
                      (long long)n, (long long)nq, need, kNoAllocScratchBytes);
        return noalloc_fail(CERT_EINVAL, msg);
    }
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return noalloc_fail(CERT_ECUDA, cudaGetErrorString(e));
    char *scratch = (char *)base;
    cudaStream_t s = (cudaStream_t)stream;

    SceneParams p;
    std::memset(&p, 0, sizeof(p));
    p.n = (int32_t)n;
    p.ap_nch = (int32_t)nch;
    p.ap_chunk = (int32_t)((n + nch - 1) / nch);
    float4 *pos4 = (float4 *)(scratch + o_pos);
    SceneParams *dsp = (SceneParams *)(scratch + o_sp);
    uint32_t *status = (uint32_t *)(scratch + o_st);

    e = cudaMemsetAsync(status, 0, 16, s);   // the array keeps the previous call's contents
    if (e == cudaSuccess) {
        k_noalloc_write_params<<<1, 32, 0, s>>>(dsp, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_pack(d_pos, (int)n, dim, pos4, status, s);
    APArgs ap;
    std::memset(&ap, 0, sizeof(ap));
    ap.dim = dim;
    ap.pos = pos4;
    ap.sp = dsp;
    ap.items = nullptr;
    ap.nqb = (int)nqb;
    ap.n_items = (int)(nqb * nch);
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
    if (e == cudaSuccess) e = allpairs_status_read(status, &st, &have_st, s);
    if (e != cudaSuccess) return noalloc_fail(CERT_ECUDA, cudaGetErrorString(e));
    return have_st ? allpairs_status_code(st) : CERT_OK;
}
