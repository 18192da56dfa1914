// probe.cu -- FMA throughput probes (diagnostics; no counterpart in the paper).
//
// The aperture kernels are bound by FP32 issue, and the float64 parts of the
// path (pixel centres, guard-band decisions, weight sums) by B300's narrow
// FP64 pipe.  These kernels measure both ceilings on the running GPU: every
// thread runs eight independent fused multiply-add chains, a -> a b + c,
// with b and c kernel arguments (so nothing folds at compile time) and
// |b| < 1 (so the chains stay bounded).  The result is written only when it
// equals an impossible value, which keeps the chains alive without memory
// traffic.  A third form runs the chains on float32 pairs through the
// packed two-lane FMA instruction.
#include <cuda_runtime.h>

#include "smart_internal.cuh"

namespace smart {
namespace {

__device__ double g_probe_sink;

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int64_t iters, T b, T c) {
    T a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = (T)(threadIdx.x & 7) * (T)1e-3 + (T)i;
    for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < PROBE_UNROLL; ++r) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == (T)-1.2345e30) g_probe_sink = (double)s;
}

// float32 pairs: every FMA instruction is a packed two-lane one (sm_100 and
// later), 16 FMAs per chain step instead of 8
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe_x2(int64_t iters, float b, float c) {
    float2 a[PROBE_CHAINS];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i)
        a[i] = make_float2((float)(threadIdx.x & 7) * 1e-3f + (float)i, (float)(threadIdx.x & 3) * 2e-3f + (float)i);
    for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < PROBE_UNROLL; ++r) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
        }
    }
    float s = 0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i].x + a[i].y;
    if (s == -1.2345e30f) g_probe_sink = (double)s;
}

}  // namespace
}  // namespace smart

using namespace smart;

extern "C" smart_status smart_fma_probe(int bits, int64_t iters, int ctas_per_sm, void *cuda_stream,
                                        double *flops) {
    if ((bits != 32 && bits != 64 && bits != (32 | SMART_PROBE_PACKED)) || iters <= 0 || ctas_per_sm < 1 ||
        ctas_per_sm > 8 || !flops)
        return SMART_E_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SMART_E_CUDA;
    const unsigned grid = (unsigned)(nsm * ctas_per_sm);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (bits == 32) k_fma_probe<float><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999f, 1e-7f);
    else if (bits == 64) k_fma_probe<double><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999999, 1e-10);
    else k_fma_probe_x2<<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999f, 1e-7f);
    if (cudaGetLastError() != cudaSuccess) return SMART_E_CUDA;
    *flops = 2.0 * (double)grid * PROBE_THREADS * (double)iters * PROBE_UNROLL * PROBE_CHAINS *
             (bits == 64 || bits == 32 ? 1.0 : 2.0);
    return SMART_OK;
}
