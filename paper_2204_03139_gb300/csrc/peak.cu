// Measured FP32 FMA throughput of the device: the denominator the Chamfer kernel's roofline
// fraction is cross-checked against (the paper has no counterpart: this is a measurement aid).
//
// Every thread runs independent FMA chains (scalar fmaf, or packed __ffma2_rn on float2),
// enough of them to cover the pipe latency, at full occupancy on every SM. The multiplier is
// just below 1 and the addend small, so the values stay normal and never overflow; the sum of
// the chains is stored (to a file-scope sink, under a condition that never holds but that the
// compiler cannot decide) so that nothing is optimised away. No memory is allocated.
#include "dc_internal.cuh"

namespace dc {

namespace {

constexpr int RATE_THREADS = 256;
constexpr int RATE_CHAINS = 16;  // FP32 lane operations per thread per iteration

__device__ float g_fma_sink;

template <bool PACKED>
__global__ void __launch_bounds__(RATE_THREADS) k_fma_rate(int iters, float seed) {
    const float m = 0.99999988f, c = 1e-7f;
    float acc = 0.0f;
    if (PACKED) {
        float2 a[RATE_CHAINS / 2];
#pragma unroll
        for (int k = 0; k < RATE_CHAINS / 2; ++k)
            a[k] = make_float2(seed + k, seed + 0.5f * k + threadIdx.x * 1e-3f);
        const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < RATE_CHAINS / 2; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
        }
#pragma unroll
        for (int k = 0; k < RATE_CHAINS / 2; ++k) acc += a[k].x + a[k].y;
    } else {
        float a[RATE_CHAINS];
#pragma unroll
        for (int k = 0; k < RATE_CHAINS; ++k) a[k] = seed + k + threadIdx.x * 1e-3f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < RATE_CHAINS; ++k) a[k] = __fmaf_rn(a[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < RATE_CHAINS; ++k) acc += a[k];
    }
    // never true: every chain starts positive and a m + c with m, c > 0 stays positive
    if (acc == -1.0f) g_fma_sink = acc;
}

}  // namespace

}  // namespace dc

extern "C" int dc_fp32_fma_rate(int packed, int iters, double* flop_per_s,
                                dc_stream_t stream) {
    using namespace dc;
    if (!flop_per_s || iters <= 0) return DC_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DC_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, packed ? (const void*)k_fma_rate<true> : (const void*)k_fma_rate<false>,
        RATE_THREADS, 0);
    if (sms <= 0 || per_sm <= 0) return DC_ECUDA;
    const int grid = sms * per_sm;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (!e) {
        for (int rep = 0; rep < 2 && !e; ++rep) {  // the first launch warms up
            cudaEventRecord(e0, s);
            if (packed)
                k_fma_rate<true><<<grid, RATE_THREADS, 0, s>>>(iters, 1.0f);
            else
                k_fma_rate<false><<<grid, RATE_THREADS, 0, s>>>(iters, 1.0f);
            cudaEventRecord(e1, s);
            e = cudaGetLastError();
            if (!e) e = cudaEventSynchronize(e1);
        }
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e || ms <= 0.0f) return DC_ECUDA;
    const double lane_ops = (double)grid * RATE_THREADS * RATE_CHAINS * (double)iters;
    *flop_per_s = 2.0 * lane_ops / (ms * 1e-3);  // an FMA is 2 flop
    return DC_OK;
}
