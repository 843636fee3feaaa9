// End-of-step moving window (paper Sec. 4 runs use a window moving at c), shared by the
// window kernels of window_sort.cu and by the Ampere launch of fields.cu that folds the window
// step into itself.  If the window shifts after step n, the live window slides one physical
// column, the guard columns of the persistent arrays on both sides of the new window are zeroed
// (the new front column of A and Er is among them), and the new last cell column is filled with
// the plasma lattice at slots [np, np + count).  Every block of the launch then counts itself
// done; the last one advances the counters (no block waits for another).
#pragma once
#include "lpic_internal.cuh"

namespace lpic {

// Zeroing and injection by threads tid, tid + nth, ...  (a block-uniform call; cp is the block's
// shared column plan).  skip_e0: leave Ex, Er and B_theta of the new column -1 (the old column 0,
// which Ampere may still be writing, or reading for its column 1, in the same launch) to the
// next step's prepass.
template <class R>
__device__ __forceinline__ void window_fill(const SimDev<R> &S, int tid, int nth, bool skip_e0, ColumnPlan<R> &cp) {
    const long long n = S.d->step, s = S.d->shift;
    if (!window_shifts(S.ph, n, s)) return;
    const Geo g = S.geo;
    const int noff = S.d->off + 1;
    // columns i in [-kG, -1] and [nx, nx+kG] of the new window
    const int ncz = 2 * kG + 1;
    for (int t = tid; t < ncz * g.P; t += nth) {
        const int cc = t / g.P, j = t - cc * g.P;
        const int i = cc < kG ? cc - kG : g.nx + (cc - kG);
        const long long id = g.at(noff, i, j);
        if (!(skip_e0 && i == -1)) {
            S.f.ex[id] = (R)0;
            S.f.er[id] = (R)0;
            S.f.bt[id] = (R)0;
        }
        typename Cplx<R>::t zc;
        zc.x = (R)0;
        zc.y = (R)0;
        S.f.a[0][id] = zc;
        S.f.a[1][id] = zc;
    }
    if (S.ph.have_plasma && S.ph.inject) {
        const long long c = s + g.nx;   // lab column of the new last cell column
        const int lt = threadIdx.y * blockDim.x + threadIdx.x;
        if (lt == 0) column_plan<R>(S.ph, c, cp);
        __syncthreads();
        const int np = S.d->np;
        const int count = column_particles<R>(S.ph, cp, g.nr);
        if (np + count <= S.ph.cap)
            for (int t = tid; t < count; t += nth) lattice_emit<R>(S, cp, c, t, np + t);
    }
}

// Every window block calls this at its end (nblocks: the window blocks for this simulation).
// The last one to arrive advances step, shift, offset, particle count and envelope buffer.
template <class R> __device__ __forceinline__ void window_done(const SimDev<R> &S, unsigned nblocks) {
    __shared__ int last;
    const int lt = threadIdx.y * blockDim.x + threadIdx.x;
    __syncthreads();
    if (lt == 0) {
        __threadfence();
        last = atomicAdd(&S.d->done, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    Desc *d = S.d;
    const long long n = d->step, s = d->shift;
    const bool shifting = window_shifts(S.ph, n, s);
    const Geo g = S.geo;
    if (lt == 0) {
        d->done = 0;
        d->last_shift = shifting ? 1 : 0;
        if (shifting) {
            if (S.ph.have_plasma && S.ph.inject) {
                ColumnPlan<R> cp;
                column_plan<R>(S.ph, s + g.nx, cp);
                const int count = column_particles<R>(S.ph, cp, g.nr);
                if (d->np + count <= S.ph.cap) d->np += count;
                else d->err |= ERR_CAPACITY;
            }
            d->shift = s + 1;
            d->off += 1;
        }
        d->step = n + 1;
        d->abuf ^= 1;
    }
}

}  // namespace lpic
