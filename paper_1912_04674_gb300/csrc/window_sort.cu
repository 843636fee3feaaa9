// Moving window (shift bookkeeping, guard zeroing, plasma injection at the front), step
// counter advance, and the periodic counting sort of particles by cell.
#include "lpic_internal.cuh"
#include "window.cuh"

namespace lpic {

namespace {

constexpr int TPB = 256;

// One part of the window step of one simulation (window.cuh): parts of kWindowThreads threads.
template <class R> __device__ __forceinline__ void window_body(const SimDev<R> &S, int part, int nparts) {
    __shared__ ColumnPlan<R> cp;
    window_fill<R>(S, part * blockDim.x + threadIdx.x, nparts * blockDim.x, false, cp);
    window_done<R>(S, (unsigned)nparts);
}

// Fused form over a batch: items {simulation, part, parts of that simulation}.
template <class R> __global__ void k_window_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        window_body<R>(pk.v[it.x], it.y, it.z);
        __syncthreads();   // the body's block-level bookkeeping must not overlap the next item
    }
}

// ---- counting sort by window cell (x-major, r fastest, like the grid) -------------------
// Cell key of slots k = k0, k0 + stride, ... < k1 and the per-cell counts.
template <class R>
__device__ __forceinline__ void sort_count_span(const SimDev<R> &S, int *key, int *count, int k0, int k1, int stride) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const long long s = S.d->shift;
    const int ncell = S.geo.nx * S.geo.nr;
    const R idr = S.k.idr;
    for (int k = k0; k < k1; k += stride) {
        const int ix = P.ix[k];
        int c;
        if (ix == kDead) {
            c = ncell;
        } else {
            const R y = P.y[k], z = P.z[k];
            int j = (int)(sqrt_<R>(y * y + z * z) * idr);
            j = min(max(j, 0), S.geo.nr - 1);
            int i = (int)((long long)ix - s);
            i = min(max(i, 0), S.geo.nx - 1);
            c = i * S.geo.nr + j;
        }
        key[k] = c;
        // particles are near-sorted: one atomic per group of lanes with the same cell
        const unsigned grp = __match_any_sync(__activemask(), c);
        if ((int)(__ffs(grp) - 1) == (int)(threadIdx.x & 31)) atomicAdd(count + c, __popc(grp));
    }
}

template <class R> __global__ void k_sort_count(SimDev<R> S, int *key, int *count) {
    sort_count_span<R>(S, key, count, blockIdx.x * blockDim.x + threadIdx.x, S.d->np, gridDim.x * blockDim.x);
}

// Exclusive scan of count[0..n) in place, three phases over blocks of 4096 items.
constexpr int SB = 1024, SI = 4;
__device__ __forceinline__ int block_exclusive_scan(int v, int *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (SB / 32) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const int before = wid > 0 ? sh[wid - 1] : 0;
    const int total = sh[SB / 32 - 1];
    __syncthreads();
    sh[32] = total;
    return before + x - v;
}

__device__ __forceinline__ void scan_blocks_body(int *data, int n, int *blocksum, int b) {
    __shared__ int sh[40];
    const int base = b * SB * SI + threadIdx.x * SI;
    int v[SI], tsum = 0;
#pragma unroll
    for (int q = 0; q < SI; q++) {
        v[q] = base + q < n ? data[base + q] : 0;
        tsum += v[q];
    }
    int ex = block_exclusive_scan(tsum, sh);
#pragma unroll
    for (int q = 0; q < SI; q++) {
        if (base + q < n) data[base + q] = ex;
        ex += v[q];
    }
    if (threadIdx.x == 0) blocksum[b] = sh[32];
    __syncthreads();   // sh is reused by the next call of this block
}

__device__ __forceinline__ void scan_top_body(int *blocksum, int nb) {  // nb <= SB*SI
    __shared__ int sh[40];
    const int base = threadIdx.x * SI;
    int v[SI], tsum = 0;
#pragma unroll
    for (int q = 0; q < SI; q++) {
        v[q] = base + q < nb ? blocksum[base + q] : 0;
        tsum += v[q];
    }
    int ex = block_exclusive_scan(tsum, sh);
#pragma unroll
    for (int q = 0; q < SI; q++) {
        if (base + q < nb) blocksum[base + q] = ex;
        ex += v[q];
    }
    __syncthreads();
}

__device__ __forceinline__ void scan_add_body(int *data, int n, const int *blocksum, int b) {
    const int add = blocksum[b];
    const int base = b * SB * SI + threadIdx.x * SI;
#pragma unroll
    for (int q = 0; q < SI; q++)
        if (base + q < n) data[base + q] += add;
}

__global__ void k_scan_blocks(int *data, int n, int *blocksum) { scan_blocks_body(data, n, blocksum, blockIdx.x); }
__global__ void k_scan_top(int *blocksum, int nb) { scan_top_body(blocksum, nb); }
__global__ void k_scan_add(int *data, int n, const int *blocksum) { scan_add_body(data, n, blocksum, blockIdx.x); }

// Scatter of slots k = k0, k0 + stride, ... < k1 to their cells' cursors (dead slots drop).
template <class R>
__device__ __forceinline__ void sort_scatter_span(const SimDev<R> &S, const int *key, int *cursor, int k0, int k1,
                                                  int stride) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Parts<R> out = S.d->pbuf ? S.p[0] : S.p[1];
    const int ncell = S.geo.nx * S.geo.nr;
    for (int k = k0; k < k1; k += stride) {
        const int c = key[k];
        // one atomic per group of lanes with the same cell; ranks within the group by lane
        const unsigned grp = __match_any_sync(__activemask(), c);
        const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
        int base = 0;
        if (lane == leader && c != ncell) base = atomicAdd(cursor + c, __popc(grp));
        base = __shfl_sync(grp, base, leader);
        if (c == ncell) continue;  // dead: dropped
        const int d = base + __popc(grp & ((1u << lane) - 1u));
        out.ix[d] = P.ix[k];
        out.ox[d] = P.ox[k];
        out.y[d] = P.y[k];
        out.z[d] = P.z[k];
        out.px[d] = P.px[k];
        out.py[d] = P.py[k];
        out.pz[d] = P.pz[k];
        out.w[d] = P.w[k];
        out.id[d] = P.id[k];
    }
}

template <class R>
__global__ void k_sort_scatter(SimDev<R> S, const int *key, int *cursor) {
    sort_scatter_span<R>(S, key, cursor, blockIdx.x * blockDim.x + threadIdx.x, S.d->np, gridDim.x * blockDim.x);
}

// After the scatter cursor[c] = end of cell c, so cursor[ncell-1] is the alive count.
template <class R> __device__ __forceinline__ void sort_finish_body(const SimDev<R> &S, const int *cursor) {
    const int ncell = S.geo.nx * S.geo.nr;
    const int alive = ncell > 0 ? cursor[ncell - 1] : 0;
    S.d->np = alive;
    S.d->n_alive = alive;
    S.d->pbuf ^= 1;
}
template <class R> __global__ void k_sort_finish(SimDev<R> S, const int *cursor) { sort_finish_body<R>(S, cursor); }

// ---- fused counting sort over a pack of simulations (those with due[slot] != 0) --------
template <class R>
__global__ void __launch_bounds__(SB) k_sort_clear_multi(const __grid_constant__ SimPack<R> pk, const int *due,
                                                         const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        if (!due[it.x]) continue;
        const SimDev<R> &S = pk.v[it.x];
        const int nc = S.geo.nx * S.geo.nr + 2;
        const int base = it.y * SB * SI + threadIdx.x * SI;
#pragma unroll
        for (int q = 0; q < SI; q++)
            if (base + q < nc) S.sb.count[base + q] = 0;
    }
}
template <class R>
__global__ void __launch_bounds__(TPB) k_sort_count_multi(const __grid_constant__ SimPack<R> pk, const int *due,
                                                          const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        if (!due[it.x]) continue;
        const SimDev<R> &S = pk.v[it.x];
        const int np = S.d->np;
        const long long b0 = (long long)it.y * it.w;
        const int begin = b0 < np ? (int)b0 : np, end = min(begin + it.w, np);
        sort_count_span<R>(S, S.sb.key, S.sb.count, begin + threadIdx.x, end, TPB);
    }
}
template <class R>
__global__ void __launch_bounds__(SB) k_scan_blocks_multi(const __grid_constant__ SimPack<R> pk, const int *due,
                                                          const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        if (!due[it.x]) continue;   // block-uniform: the whole block skips or takes the item
        const SimDev<R> &S = pk.v[it.x];
        scan_blocks_body(S.sb.count, S.geo.nx * S.geo.nr + 1, S.sb.blocksum, it.y);
    }
}
template <class R>
__global__ void __launch_bounds__(SB) k_scan_top_multi(const __grid_constant__ SimPack<R> pk, const int *due,
                                                       const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        if (!due[it.x]) continue;
        const SimDev<R> &S = pk.v[it.x];
        scan_top_body(S.sb.blocksum, sort_blocks(S.geo));
    }
}
template <class R>
__global__ void __launch_bounds__(SB) k_scan_add_multi(const __grid_constant__ SimPack<R> pk, const int *due,
                                                       const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        if (!due[it.x]) continue;
        const SimDev<R> &S = pk.v[it.x];
        scan_add_body(S.sb.count, S.geo.nx * S.geo.nr + 1, S.sb.blocksum, it.y);
    }
}
template <class R>
__global__ void __launch_bounds__(TPB) k_sort_scatter_multi(const __grid_constant__ SimPack<R> pk, const int *due,
                                                            const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        if (!due[it.x]) continue;
        const SimDev<R> &S = pk.v[it.x];
        const int np = S.d->np;
        const long long b0 = (long long)it.y * it.w;
        const int begin = b0 < np ? (int)b0 : np, end = min(begin + it.w, np);
        sort_scatter_span<R>(S, S.sb.key, S.sb.count, begin + threadIdx.x, end, TPB);
    }
}
template <class R>
__global__ void k_sort_finish_multi(const __grid_constant__ SimPack<R> pk, const int *due, const int4 *items, int n) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    const int4 it = items[w];
    if (due[it.x]) sort_finish_body<R>(pk.v[it.x], pk.v[it.x].sb.count);
}

inline int pgrid(int n) {
    int b = (n + TPB - 1) / TPB;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

}  // namespace

int window_parts(const Geo &g, int work) {
    int blocks = (work + kWindowThreads - 1) / kWindowThreads;
    return blocks < 1 ? 1 : (blocks > 152 * 8 ? 152 * 8 : blocks);
}

template <class R> void launch_window_multi(const SimPack<R> &pk, const int4 *items, int n, cudaStream_t st) {
    if (n > 0) k_window_multi<R><<<n < 152 * 8 ? n : 152 * 8, kWindowThreads, 0, st>>>(pk, items, n);
}

// Exclusive scan of n <= SB*SI*SB*SI ints in place.
void scan_exclusive(int *data, int n, int *blocksum, cudaStream_t st) {
    const int per = SB * SI;
    const int nb = (n + per - 1) / per;
    k_scan_blocks<<<nb, SB, 0, st>>>(data, n, blocksum);
    k_scan_top<<<1, SB, 0, st>>>(blocksum, nb);
    k_scan_add<<<nb, SB, 0, st>>>(data, n, blocksum);
}

template <class R>
void launch_sort(const SimDev<R> &S, int np_upper, int *key, int *count, int *blocksum,
                 cudaStream_t st) {
    const int ncell = S.geo.nx * S.geo.nr;
    cudaMemsetAsync(count, 0, sizeof(int) * (ncell + 1), st);
    k_sort_count<R><<<pgrid(np_upper), TPB, 0, st>>>(S, key, count);
    scan_exclusive(count, ncell + 1, blocksum, st);
    k_sort_scatter<R><<<pgrid(np_upper), TPB, 0, st>>>(S, key, count);
    k_sort_finish<R><<<1, 1, 0, st>>>(S, count);
}

template <class R>
void launch_sort_multi(const SimPack<R> &pk, const int *due, const int4 *blocks, int nblocks,
                       const int4 *slots, int nslots, const int4 *sims, int nsims, cudaStream_t st) {
    if (nsims <= 0) return;
    const int gb = nblocks < 152 * 2 ? nblocks : 152 * 2;     // 1024-thread blocks, 2 per SM
    const int gs = nslots < 152 * 8 ? nslots : 152 * 8;       // 256-thread blocks, 8 per SM
    if (gb > 0) k_sort_clear_multi<R><<<gb, SB, 0, st>>>(pk, due, blocks, nblocks);
    if (gs > 0) k_sort_count_multi<R><<<gs, TPB, 0, st>>>(pk, due, slots, nslots);
    if (gb > 0) k_scan_blocks_multi<R><<<gb, SB, 0, st>>>(pk, due, blocks, nblocks);
    k_scan_top_multi<R><<<nsims, SB, 0, st>>>(pk, due, sims, nsims);
    if (gb > 0) k_scan_add_multi<R><<<gb, SB, 0, st>>>(pk, due, blocks, nblocks);
    if (gs > 0) k_sort_scatter_multi<R><<<gs, TPB, 0, st>>>(pk, due, slots, nslots);
    k_sort_finish_multi<R><<<(nsims + 63) / 64, 64, 0, st>>>(pk, due, sims, nsims);
}

#define INST(R)                                                                          \
    template void launch_sort_multi<R>(const SimPack<R> &, const int *, const int4 *, int, \
                                       const int4 *, int, const int4 *, int, cudaStream_t); \
    template void launch_window_multi<R>(const SimPack<R> &, const int4 *, int, cudaStream_t); \
    template void launch_sort<R>(const SimDev<R> &, int, int *, int *, int *, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace lpic
