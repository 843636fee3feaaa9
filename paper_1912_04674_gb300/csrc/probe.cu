// Measurement helper: the FP64 fused multiply-add rate of the current device.
//
// The FP64 form of the particle passes is bound by the FP64 pipe, whose rate on this part
// is a small fraction of the FP32 rate; its roofline is taken against this measured rate
// rather than a datasheet figure.  Every thread runs kChains independent FMA chains (enough
// independent work to cover the pipe's latency), each value staying near 1 so that no
// denormal or overflow path is taken; the sums are stored so the work cannot be removed.
#include "lpic.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma(int iters, double *out) {
    double v[kChains];
    const double b = 1.0 - 1.0 / 4096.0, c = 1.0 / 4096.0;   // fixed point of v = b v + c is 1
#pragma unroll
    for (int q = 0; q < kChains; q++) v[q] = 1.0 + (threadIdx.x + q) * 1e-9;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int q = 0; q < kChains; q++) v[q] = fma(v[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; q++) s += v[q];
    if (s == 12345.678) out[0] = s;   // never true; keeps the chains live
    if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

}  // namespace

extern "C" lpic_status lpic_probe_fp64_fma(int32_t iters, double *out_dev, int64_t *flops,
                                           void *cuda_stream) {
    if (iters < 1 || !out_dev || !flops) return LPIC_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LPIC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LPIC_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma, kThreads, 0) != cudaSuccess)
        return LPIC_ECUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    (void)cudaGetLastError();
    k_dfma<<<blocks, kThreads, 0, (cudaStream_t)cuda_stream>>>(iters, out_dev);
    if (cudaGetLastError() != cudaSuccess) return LPIC_ECUDA;
    *flops = 2LL * kChains * (long long)iters * blocks * kThreads;
    return LPIC_OK;
}
