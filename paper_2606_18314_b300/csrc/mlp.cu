// mlp.cu -- the repair-strategy selector network on the device.
//
// The selector (no counterpart in the paper; it learns the repair/rebuild
// crossover that Prop. 1 describes) is an MLP 8 -> 64 -> 64 -> 2 with ReLU
// after each hidden layer.  Its inputs are the step features, normalised as
// x' = (x - mean) * inv_std; its outputs predict ln step time of incremental
// repair and of rebuild.  Loss: mean over rows and both outputs of (y - t)^2.
//
// Training kernels: each CTA owns 64-row tiles of the batch; the weights, the
// tile's pre-activations and back-propagated errors, and the CTA's gradient
// accumulators live in shared memory, with every gradient element owned by
// one thread (no atomics).  CTA partial gradients are summed in CTA order by
// a second kernel, so gradients are deterministic.  Adam is elementwise.
// FP32 CUDA cores: a batch is a few MFLOP, far too small for tensor cores to
// matter, and this runs off the per-step path.
#include <algorithm>
#include <cstring>

#include "cert_internal.cuh"
#include "cert_launch.h"

namespace certk {

constexpr int kIn = 8, kHid = 64, kOut = 2;
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kOut * kHid, kNP = kB3 + kOut;   // 4866
constexpr int kRows = 64;           // rows per tile
constexpr int kMlpThreads = 256;
static_assert(kNP == CERT_MLP_PARAMS, "parameter layout");

struct MlpSmem {
    float w[kNP];                   // parameters
    float w2t[kHid * kHid];         // W2 transposed: lanes that vary the output unit read consecutive words
    float g[kNP];                   // this CTA's gradient accumulators
    float x[kRows][kIn];            // normalised inputs
    float z1[kRows][kHid];          // pre-activations, then errors of layer 1
    float z2[kRows][kHid];          // pre-activations of layer 2
    float d2[kRows][kHid];          // errors of layer 2
    float dy[kRows][kOut];
    float red[kMlpThreads / 32];
};

__device__ void mlp_load_params(MlpSmem &m, const float *p)
{
    for (int k = threadIdx.x; k < kNP; k += kMlpThreads) m.w[k] = p[k];
    for (int e = threadIdx.x; e < kHid * kHid; e += kMlpThreads) {
        const int h = e / kHid, k = e % kHid;
        m.w2t[k * kHid + h] = p[kW2 + e];
    }
}

// Forward pass of one tile: fills x, z1, z2 and returns nothing; y via out.
__device__ void mlp_tile_forward(MlpSmem &m, const float *X, const float *norm, long long row0, long long n)
{
    for (int e = threadIdx.x; e < kRows * kIn; e += kMlpThreads) {
        const int r = e / kIn, k = e % kIn;
        const long long row = row0 + r;
        m.x[r][k] = row < n ? (X[row * kIn + k] - norm[k]) * norm[kIn + k] : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kRows * kHid; e += kMlpThreads) {
        const int r = e / kHid, h = e % kHid;
        float z = m.w[kB1 + h];
#pragma unroll
        for (int k = 0; k < kIn; ++k) z = fmaf(m.w[kW1 + h * kIn + k], m.x[r][k], z);
        m.z1[r][h] = z;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kRows * kHid; e += kMlpThreads) {
        const int r = e / kHid, h = e % kHid;
        float z = m.w[kB2 + h];
        for (int k = 0; k < kHid; ++k) z = fmaf(m.w2t[k * kHid + h], fmaxf(m.z1[r][k], 0.0f), z);
        m.z2[r][h] = z;
    }
    __syncthreads();
}

__device__ __forceinline__ float mlp_out(const MlpSmem &m, int r, int o)
{
    float y = m.w[kB3 + o];
    for (int k = 0; k < kHid; ++k) y = fmaf(m.w[kW3 + o * kHid + k], fmaxf(m.z2[r][k], 0.0f), y);
    return y;
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float *params, const float *norm, const float *X,
                                                            long long n, float *Y)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem &m = *reinterpret_cast<MlpSmem *>(smem_raw);
    mlp_load_params(m, params);
    __syncthreads();
    for (long long row0 = (long long)blockIdx.x * kRows; row0 < n; row0 += (long long)gridDim.x * kRows) {
        mlp_tile_forward(m, X, norm, row0, n);
        if (threadIdx.x < kRows * kOut) {
            const int r = threadIdx.x / kOut, o = threadIdx.x % kOut;
            if (row0 + r < n) Y[(row0 + r) * kOut + o] = mlp_out(m, r, o);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_grad_partial(const float *params, const float *norm,
                                                                 const float *X, const float *T, long long n,
                                                                 float *work)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem &m = *reinterpret_cast<MlpSmem *>(smem_raw);
    mlp_load_params(m, params);
    for (int k = threadIdx.x; k < kNP; k += kMlpThreads) m.g[k] = 0.0f;
    float loss = 0.0f;
    const float scale = 2.0f / (float)(n * kOut);   // d mean((y-t)^2) / dy
    __syncthreads();
    for (long long row0 = (long long)blockIdx.x * kRows; row0 < n; row0 += (long long)gridDim.x * kRows) {
        mlp_tile_forward(m, X, norm, row0, n);
        if (threadIdx.x < kRows * kOut) {
            const int r = threadIdx.x / kOut, o = threadIdx.x % kOut;
            const long long row = row0 + r;
            float d = 0.0f;
            if (row < n) {
                const float e = mlp_out(m, r, o) - T[row * kOut + o];
                loss = fmaf(e, e, loss);
                d = scale * e;
            }
            m.dy[r][o] = d;
        }
        __syncthreads();
        // output layer gradients and the error of layer 2
        for (int e = threadIdx.x; e < kOut * kHid + kOut; e += kMlpThreads) {
            float acc = 0.0f;
            if (e < kOut * kHid) {
                const int o = e / kHid, k = e % kHid;
                for (int r = 0; r < kRows; ++r) acc = fmaf(m.dy[r][o], fmaxf(m.z2[r][k], 0.0f), acc);
                m.g[kW3 + e] += acc;
            } else {
                const int o = e - kOut * kHid;
                for (int r = 0; r < kRows; ++r) acc += m.dy[r][o];
                m.g[kB3 + o] += acc;
            }
        }
        for (int e = threadIdx.x; e < kRows * kHid; e += kMlpThreads) {
            const int r = e / kHid, k = e % kHid;
            float d = 0.0f;
#pragma unroll
            for (int o = 0; o < kOut; ++o) d = fmaf(m.dy[r][o], m.w[kW3 + o * kHid + k], d);
            m.d2[r][k] = m.z2[r][k] > 0.0f ? d : 0.0f;
        }
        __syncthreads();
        // layer 2 gradients
        for (int e = threadIdx.x; e < kHid * kHid + kHid; e += kMlpThreads) {
            float acc = 0.0f;
            if (e < kHid * kHid) {
                const int h = e / kHid, k = e % kHid;
                for (int r = 0; r < kRows; ++r) acc = fmaf(m.d2[r][h], fmaxf(m.z1[r][k], 0.0f), acc);
                m.g[kW2 + e] += acc;
            } else {
                const int h = e - kHid * kHid;
                for (int r = 0; r < kRows; ++r) acc += m.d2[r][h];
                m.g[kB2 + h] += acc;
            }
        }
        __syncthreads();
        // error of layer 1, written over z1 (each element read before it is overwritten by its owner)
        for (int e = threadIdx.x; e < kRows * kHid; e += kMlpThreads) {
            const int r = e / kHid, k = e % kHid;
            float d = 0.0f;
            for (int h = 0; h < kHid; ++h) d = fmaf(m.d2[r][h], m.w[kW2 + h * kHid + k], d);
            m.z1[r][k] = m.z1[r][k] > 0.0f ? d : 0.0f;   // only this thread touches element (r, k)
        }
        __syncthreads();
        // layer 1 gradients
        for (int e = threadIdx.x; e < kHid * kIn + kHid; e += kMlpThreads) {
            float acc = 0.0f;
            if (e < kHid * kIn) {
                const int h = e / kIn, k = e % kIn;
                for (int r = 0; r < kRows; ++r) acc = fmaf(m.z1[r][h], m.x[r][k], acc);
                m.g[kW1 + e] += acc;
            } else {
                const int h = e - kHid * kIn;
                for (int r = 0; r < kRows; ++r) acc += m.z1[r][h];
                m.g[kB1 + h] += acc;
            }
        }
        __syncthreads();
    }
    // CTA loss: warp sums, then thread 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(kFull, loss, o);
    if ((threadIdx.x & 31) == 0) m.red[threadIdx.x >> 5] = loss;
    __syncthreads();
    float *out = work + (size_t)blockIdx.x * (kNP + 1);
    for (int k = threadIdx.x; k < kNP; k += kMlpThreads) out[k] = m.g[k];
    if (threadIdx.x == 0) {
        float tot = 0.0f;
        for (int w = 0; w < kMlpThreads / 32; ++w) tot += m.red[w];
        out[kNP] = tot;
    }
}

// Sum the CTA partials in CTA order; loss = sum of squared errors / (2n).
__global__ void k_mlp_grad_reduce(const float *work, int parts, long long n, float *grad, float *loss)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kNP) return;
    float acc = 0.0f;
    for (int p = 0; p < parts; ++p) acc += work[(size_t)p * (kNP + 1) + k];
    if (k < kNP)
        grad[k] = acc;
    else if (loss)
        *loss = acc / (float)(n * kOut);
}

__global__ void k_mlp_adam(float *p, const float *g, float *mo, float *ve, float lr, float b1, float b2, float eps,
                           float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNP) return;
    const float gk = g[k];
    const float m = b1 * mo[k] + (1.0f - b1) * gk;
    const float v = b2 * ve[k] + (1.0f - b2) * gk * gk;
    mo[k] = m;
    ve[k] = v;
    p[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

static int mlp_ctas(long long n)
{
    const long long tiles = (n + kRows - 1) / kRows;
    return (int)std::max<long long>(1, std::min<long long>(tiles, 148));
}

}  // namespace certk

using namespace certk;

static cert_status mlp_fail(cert_status code, const char *msg)
{
    record_thread_error(msg);
    return code;
}

static cudaError_t mlp_smem_setup()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MlpSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(MlpSmem));
    if (e == cudaSuccess) done = true;
    return e;
}

extern "C" size_t cert_mlp_workspace_bytes(int64_t n)
{
    return (size_t)mlp_ctas(n) * (kNP + 1) * sizeof(float);
}

extern "C" cert_status cert_mlp_forward(const float *d_params, const float *d_norm, const float *d_X, int64_t n,
                                        float *d_Y, void *stream)
{
    if (!d_params || !d_norm || !d_X || !d_Y) return mlp_fail(CERT_EINVAL, "NULL argument");
    if (n <= 0) return n == 0 ? CERT_OK : mlp_fail(CERT_EINVAL, "n < 0");
    cudaError_t e = mlp_smem_setup();
    if (e == cudaSuccess) {
        k_mlp_forward<<<mlp_ctas(n), kMlpThreads, sizeof(MlpSmem), (cudaStream_t)stream>>>(d_params, d_norm, d_X, n,
                                                                                            d_Y);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? CERT_OK : mlp_fail(CERT_ECUDA, cudaGetErrorString(e));
}

extern "C" cert_status cert_mlp_grad(const float *d_params, const float *d_norm, const float *d_X, const float *d_T,
                                     int64_t n, float *d_grad, float *d_loss, void *d_work, size_t work_bytes,
                                     void *stream)
{
    if (!d_params || !d_norm || !d_X || !d_T || !d_grad || !d_work) return mlp_fail(CERT_EINVAL, "NULL argument");
    if (n <= 0) return mlp_fail(CERT_EINVAL, "n must be > 0");
    if (work_bytes < cert_mlp_workspace_bytes(n)) return mlp_fail(CERT_EINVAL, "workspace too small");
    cudaError_t e = mlp_smem_setup();
    const int parts = mlp_ctas(n);
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) {
        k_mlp_grad_partial<<<parts, kMlpThreads, sizeof(MlpSmem), s>>>(d_params, d_norm, d_X, d_T, n, (float *)d_work);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_mlp_grad_reduce<<<(kNP + 1 + 255) / 256, 256, 0, s>>>((const float *)d_work, parts, n, d_grad, d_loss);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? CERT_OK : mlp_fail(CERT_ECUDA, cudaGetErrorString(e));
}

extern "C" cert_status cert_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int32_t t,
                                     float lr, float beta1, float beta2, float eps, void *stream)
{
    if (!d_params || !d_grad || !d_m || !d_v) return mlp_fail(CERT_EINVAL, "NULL argument");
    if (t < 1) return mlp_fail(CERT_EINVAL, "Adam step counts from 1");
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_mlp_adam<<<(kNP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps,
                                                                     c1, c2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CERT_OK : mlp_fail(CERT_ECUDA, cudaGetErrorString(e));
}
