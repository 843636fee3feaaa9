// x-slab decomposition: the exchange between two adjacent slabs of one window after a step
// (lpic_slab_exchange).  Sec. 3 of the paper parallelises the envelope solver like a standard
// Yee scheme: sub-domains that trade guard cells.  Here the slabs overlap by 2*halo columns;
// each computes its whole window (owned columns plus halos) every step, and afterwards the
// owner's values replace the halo values, so that wrong boundary values at a slab's edges
// never reach the columns it owns.
#include "lpic_internal.cuh"

namespace lpic {

namespace {

constexpr int TPB = 256;
constexpr unsigned FULL = 0xffffffffu;

// ncols whole physical columns of one persistent array, from local column cs of the source
// slab to local column cd of the destination (columns are contiguous in both: P elements each).
template <class T>
__device__ __forceinline__ void copy_cols(const T *src, int offs, int cs, T *dst, int offd, int cd, int ncols, int P) {
    const long long n = (long long)ncols * P;
    const T *s = src + (long long)(offs + kG + cs) * P;
    T *d = dst + (long long)(offd + kG + cd) * P;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        d[k] = s[k];
}

// blockIdx.y picks the array and the direction.  Right to left: nodes [B, B+halo] and cells
// [B, B+halo) (right's local columns from halo); left to right: nodes and cells [B-halo, B)
// into right's local columns [0, halo).
template <class R> __global__ void k_slab_fields(SimDev<R> L, SimDev<R> Rt, int B_L, int halo) {
    const int offL = L.d->off, offR = Rt.d->off, P = L.geo.P;
    const int task = blockIdx.y, arr = task % 5;
    const bool to_left = task < 5;
    const bool node = arr != 0 && arr != 2;   // Ex and B_theta are cell-centred in x
    const SimDev<R> &S = to_left ? Rt : L;
    const SimDev<R> &D = to_left ? L : Rt;
    const int offs = to_left ? offR : offL, offd = to_left ? offL : offR;
    const int cs = to_left ? halo : B_L - halo, cd = to_left ? B_L : 0;
    const int n = to_left ? halo + (node ? 1 : 0) : halo;
    switch (arr) {
    case 0: copy_cols(S.f.ex, offs, cs, D.f.ex, offd, cd, n, P); break;
    case 1: copy_cols(S.f.er, offs, cs, D.f.er, offd, cd, n, P); break;
    case 2: copy_cols(S.f.bt, offs, cs, D.f.bt, offd, cd, n, P); break;
    default: copy_cols(S.f.a[arr - 3], offs, cs, D.f.a[arr - 3], offd, cd, n, P); break;
    }
}

// Remove the electrons whose local cell is outside [lo, hi), and list the freed slots (up to
// fcap of them, warp-aggregated) for the appends of the same exchange.
template <class R> __global__ void k_slab_keep(SimDev<R> S, int lo, int hi, int *freed, int fcap) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const long long sh = S.d->shift;
    const int np = S.d->np;
    const int lane = threadIdx.x & 31;
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < np; base += gridDim.x * blockDim.x) {
        const int k = base + lane;
        const int ix = k < np ? P.ix[k] : kDead;
        const long long irel = (long long)ix - sh;
        const bool drop = ix != kDead && (irel < lo || irel >= hi);
        const unsigned m = __ballot_sync(FULL, drop);
        if (!m) continue;
        int first = 0;
        if (lane == 0) first = atomicAdd(&S.d->nfree, __popc(m));
        first = __shfl_sync(FULL, first, 0);
        if (!drop) continue;
        P.ix[k] = kDead;
        const int t = first + __popc(m & ((1u << lane) - 1u));
        if (t < fcap) freed[t] = k;
    }
}

// Append the source's electrons in its local cells [lo, hi) to the destination: the slots its
// removal freed first (they sit where the halo cells' electrons were sorted), then slots from
// its np on (warp-aggregated claims).  Slots beyond the capacity are not written and latch
// ERR_CAPACITY.
template <class R> __global__ void k_slab_append(SimDev<R> Src, SimDev<R> Dst, int lo, int hi, const int *freed,
                                                 int fcap) {
    const Parts<R> P = Src.d->pbuf ? Src.p[1] : Src.p[0];
    const Parts<R> Q = Dst.d->pbuf ? Dst.p[1] : Dst.p[0];
    const long long sh = Src.d->shift;
    const int np = Src.d->np, cap = Dst.ph.cap;
    const int nfree = min(Dst.d->nfree, fcap), np0 = Dst.d->np;
    const int lane = threadIdx.x & 31;
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < np; base += gridDim.x * blockDim.x) {
        const int k = base + lane;
        const int ix = k < np ? P.ix[k] : kDead;
        const long long irel = (long long)ix - sh;
        const bool sel = ix != kDead && irel >= lo && irel < hi;
        const unsigned m = __ballot_sync(FULL, sel);
        if (!m) continue;
        int first = 0;
        if (lane == 0) first = atomicAdd(&Dst.d->ntaken, __popc(m));
        first = __shfl_sync(FULL, first, 0);
        if (!sel) continue;
        const int t = first + __popc(m & ((1u << lane) - 1u));
        const long long slot = t < nfree ? (long long)freed[t] : (long long)np0 + (t - nfree);
        if (slot >= cap) {
            atomicOr(&Dst.d->err, (int)ERR_CAPACITY);
            continue;
        }
        Q.ix[slot] = ix;
        Q.ox[slot] = P.ox[k];
        Q.y[slot] = P.y[k];
        Q.z[slot] = P.z[k];
        Q.px[slot] = P.px[k];
        Q.py[slot] = P.py[k];
        Q.pz[slot] = P.pz[k];
        Q.w[slot] = P.w[k];
        Q.id[slot] = P.id[k];
    }
}

// np grows by the appends that found no freed slot (within the capacity); the counters are
// zeroed for the next exchange.
template <class R> __global__ void k_slab_settle(SimDev<R> S, int fcap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int nfree = min(S.d->nfree, fcap);
        const long long grown = (long long)S.d->np + max(S.d->ntaken - nfree, 0);
        S.d->np = (int)(grown < S.ph.cap ? grown : S.ph.cap);
        S.d->nfree = 0;
        S.d->ntaken = 0;
    }
}

int blocks_for(long long n) {
    long long b = (n + TPB - 1) / TPB;
    return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

}  // namespace

// B_L: the boundary in the left slab's local columns; freeL / freeR: scratch for fcap slot
// indices of each side (its staging area).  Both slabs' np are read on the device, so the
// particle kernels are sized for the capacities.  The appends read np of the destination as
// the keep left it: the destination's removal runs first, both removals before the appends.
template <class R>
void launch_slab_exchange(const SimDev<R> &L, const SimDev<R> &Rt, int B_L, int halo, int *freeL, int *freeR,
                          int fcap, cudaStream_t st) {
    const long long cols = (long long)(halo + 1) * L.geo.P;
    k_slab_fields<R><<<dim3(blocks_for(cols), 10), TPB, 0, st>>>(L, Rt, B_L, halo);
    k_slab_keep<R><<<blocks_for(L.ph.cap), TPB, 0, st>>>(L, -(1 << 30), B_L, freeL, fcap);
    k_slab_keep<R><<<blocks_for(Rt.ph.cap), TPB, 0, st>>>(Rt, halo, 1 << 30, freeR, fcap);
    k_slab_append<R><<<blocks_for(Rt.ph.cap), TPB, 0, st>>>(Rt, L, halo, 2 * halo, freeL, fcap);
    k_slab_append<R><<<blocks_for(L.ph.cap), TPB, 0, st>>>(L, Rt, B_L - halo, B_L, freeR, fcap);
    k_slab_settle<R><<<1, 32, 0, st>>>(L, fcap);
    k_slab_settle<R><<<1, 32, 0, st>>>(Rt, fcap);
}

template void launch_slab_exchange<double>(const SimDev<double> &, const SimDev<double> &, int, int, int *, int *,
                                           int, cudaStream_t);
template void launch_slab_exchange<float>(const SimDev<float> &, const SimDev<float> &, int, int, int *, int *, int,
                                          cudaStream_t);

}  // namespace lpic
