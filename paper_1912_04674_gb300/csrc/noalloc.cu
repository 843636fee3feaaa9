// Allocation-free envelope statistics (peak |A| and second-moment waist).
//
// For callers that cannot call cudaMalloc: code running where the CUDA allocator is off
// limits (a host framework that owns all device memory through its own pool, a real-time
// loop whose memory is fixed up front, a plug-in that may only use memory it was handed).
// It computes the same two numbers as lpic_diagnose(LPIC_DIAG_A_ABS_MAX / LPIC_DIAG_WAIST),
// but from an envelope array the caller passes in, and keeps its only scratch -- one
// partial result per thread block -- in a fixed array in this file's device memory.
#include <mutex>

#include "lpic.h"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerBlock = 4096;                 // nodes reduced by one block
constexpr int kMaxBlocks = 4096;                     // scratch slots
constexpr long long kMaxNodes = (long long)kNodesPerBlock * kMaxBlocks;   // 16,777,216
constexpr int kMaxDevices = 64;

// Per-block partials {max |A|^2, sum |A|^2 r^2 v, sum |A|^2 v}: 4096 x 3 doubles = 96 KiB,
// held by every device that loads the library until the process exits.
static __device__ __align__(256) double g_partials[kMaxBlocks * 3];

std::mutex g_setup_lock;
double *g_partials_addr[kMaxDevices] = {};

__global__ void k_partials(const double2 *__restrict__ a, int nx, int nr, double dr, long long n,
                           double *part) {
    double m = 0.0, s2 = 0.0, s0 = 0.0;
    const long long base = (long long)blockIdx.x * kNodesPerBlock;
    for (int t = threadIdx.x; t < kNodesPerBlock; t += kThreads) {
        const long long k = base + t;
        if (k >= n) break;
        const int j = (int)(k % (nr + 1));
        const double2 v = a[k];
        const double I = v.x * v.x + v.y * v.y;
        const double r = j * dr;
        const double vol = j == 0 ? 0.125 * dr * dr : r * dr;   // node volume / (2 pi dx)
        m = fmax(m, I);
        s0 += I * vol;
        s2 += I * vol * r * r;
    }
    __shared__ double sh[3][kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = m; sh[1][wid] = s2; sh[2][wid] = s0; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kThreads / 32; q++) {
            m = fmax(m, sh[0][q]);
            s2 += sh[1][q];
            s0 += sh[2][q];
        }
        part[3 * blockIdx.x + 0] = m;   // every used slot is written: nothing to clear
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = s0;
    }
}

__global__ void k_finish(const double *part, int nblocks, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = 0.0, s2 = 0.0, s0 = 0.0;
    for (int b = 0; b < nblocks; b++) {   // fixed order: the result is reproducible
        m = fmax(m, part[3 * b]);
        s2 += part[3 * b + 1];
        s0 += part[3 * b + 2];
    }
    out[0] = sqrt(m);
    out[1] = s0 > 0.0 ? sqrt(2.0 * s2 / s0) : 0.0;
}

}  // namespace

extern "C" lpic_status lpic_envelope_stats_noalloc(const void *a_dev, int32_t nx, int32_t nr,
                                                   double dr, double *out_dev, void *cuda_stream) {
    if (!a_dev || !out_dev || nx < 1 || nr < 1 || !(dr > 0.0)) return LPIC_EINVAL;
    const long long n = ((long long)nx + 1) * ((long long)nr + 1);
    if (n > kMaxNodes) return LPIC_EBUFSIZE;   // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LPIC_ECUDA;
    double *part = nullptr;
    {
        // Once per device, with that device current: the host-side name g_partials is only
        // a stand-in, so ask the runtime for the array's device address.
        std::lock_guard<std::mutex> lock(g_setup_lock);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return LPIC_ECUDA;
            g_partials_addr[dev] = (double *)p;
        }
        part = g_partials_addr[dev];
    }
    const int nblocks = (int)((n + kNodesPerBlock - 1) / kNodesPerBlock);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    (void)cudaGetLastError();   // an error left by the caller's earlier work is not ours to report
    k_partials<<<nblocks, kThreads, 0, st>>>((const double2 *)a_dev, nx, nr, dr, n, part);
    if (cudaGetLastError() != cudaSuccess) return LPIC_ECUDA;
    k_finish<<<1, 32, 0, st>>>(part, nblocks, out_dev);
    return cudaGetLastError() == cudaSuccess ? LPIC_OK : LPIC_ECUDA;
}
