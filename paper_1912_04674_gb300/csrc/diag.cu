// Diagnostics (reductions on the device, small results copied back by api.cu), canonical
// FP64 dumps and uploads of grid arrays and particles.
#include "lpic_internal.cuh"

namespace lpic {

namespace {

constexpr int TPB = 256;

inline int pgrid(long long n) {
    long long b = (n + TPB - 1) / TPB;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : (int)b);
}

__device__ __forceinline__ void atomic_max_nonneg(double *p, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

template <class R> __global__ void k_ex_axis(SimDev<R> S, double *out) {
    const int off = S.d->off;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.geo.nx; i += gridDim.x * blockDim.x)
        out[i] = (double)S.f.ex[S.geo.at(off, i, 0)];
}

// out[0] = max |A^n|, out[1] = sum |A|^2 r^2 V, out[2] = sum |A|^2 V (V: node volume / 2 pi dx)
template <class R> __global__ void k_amax_waist(SimDev<R> S, double *out) {
    const Geo g = S.geo;
    const int off = S.d->off;
    const auto *A = S.f.a[S.d->abuf];
    const long long n = (long long)(g.nx + 1) * (g.nr + 1);
    double m = 0.0, s2 = 0.0, s0 = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / (g.nr + 1)), j = (int)(t - (long long)i * (g.nr + 1));
        auto a = A[g.at(off, i, j)];
        const double I = (double)a.x * a.x + (double)a.y * a.y;
        m = fmax(m, I);
        const double r = j * S.ph.dr;
        const double v = j == 0 ? 0.125 * S.ph.dr * S.ph.dr : r * S.ph.dr;
        s0 += I * v;
        s2 += I * v * r * r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(out, sqrt(m));
        atomicAdd(out + 1, s2);
        atomicAdd(out + 2, s0);
    }
}

// Continuity residual of the last step on interior nodes i in [1, nx-1], j in [0, nr-1]:
// out[0] = max |dQ/dt + div I|, out[1] = max |div I|, I = J times face area, i.e. the charge
// the deposit moved through each face, over dt.
template <class R> __global__ void k_cont(SimDev<R> S, double *out) {
    const Geo g = S.geo;
    const int off = S.d->off - S.d->last_shift;  // the window the last step deposited on
    const double dt = S.ph.dt;
    // interior columns; with the current filter, also away from the `passes` columns at each
    // end, where filtering on the window only (zero outside) breaks the discrete continuity
    const int edge = 1 + S.ph.filter_passes;
    const long long n = (long long)(g.nx + 1 - 2 * edge) * g.nr;
    double rmax = 0.0, dmax = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = edge + (int)(t / g.nr), j = (int)(t % g.nr);
        const double ixp = S.f.jxu[g.at(off, i, j)], ixm = S.f.jxu[g.at(off, i - 1, j)];
        const double irp = S.f.jru[g.at(off, i, j)];
        const double irm = j == 0 ? 0.0 : S.f.jru[g.at(off, i, j - 1)];
        const double div = ((ixp - ixm) + (irp - irm)) / dt;
        const double res = S.f.dqu[g.at(off, i, j)] / dt + div;
        rmax = fmax(rmax, fabs(res));
        dmax = fmax(dmax, fabs(div));
    }
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(out, rmax);
        atomic_max_nonneg(out + 1, dmax);
    }
}

// ---- beam parameters of the accelerated electrons (Table BeamParams quantities) -----------
// Energy gamma - 1 of slot k in FP64, without contraction, so that a particle state gives the
// same bits here and in any other IEEE evaluation of sqrt(1 + px^2 + py^2 + pz^2) - 1.
template <class R> __device__ __forceinline__ double beam_energy(const Parts<R> &P, int k) {
    const double px = P.px[k], py = P.py[k], pz = P.pz[k];
    const double s = __dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(px, px)), __dmul_rn(py, py)), __dmul_rn(pz, pz));
    return __dsub_rn(sqrt(s), 1.0);
}

// out = {max energy, count} over alive particles with p_x > thr.
template <class R> __global__ void k_beam_max(SimDev<R> S, double thr, double *out) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const int np = S.d->np;
    double m = 0.0, c = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        if (P.ix[k] == kDead || !((double)P.px[k] > thr)) continue;
        m = fmax(m, beam_energy<R>(P, k));
        c += 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0 && c > 0) {
        atomic_max_nonneg(out, m);
        atomicAdd(out + 1, c);
    }
}

// w-weighted energy histogram, bins of `width` over [0, nbins*width) (the last bin takes the top).
template <class R> __global__ void k_beam_hist(SimDev<R> S, double thr, double width, int nbins, double *hist) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const int np = S.d->np;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        if (P.ix[k] == kDead || !((double)P.px[k] > thr)) continue;
        const double b = floor(__ddiv_rn(beam_energy<R>(P, k), width));
        atomicAdd(hist + (b < (double)(nbins - 1) ? (int)b : nbins - 1), (double)P.w[k]);
    }
}

// Sums over the beam (|E - e_peak| <= fwhm): w, wE, wE^2, then for u = y, z: w u, w u^2, w p_u,
// w p_u^2, w u p_u; and the count.  out: 14 doubles.
template <class R>
__global__ void k_beam_moments(SimDev<R> S, double thr, double e_peak, double fwhm, double *out) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const int np = S.d->np;
    double a[14];
#pragma unroll
    for (int q = 0; q < 14; q++) a[q] = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        if (P.ix[k] == kDead || !((double)P.px[k] > thr)) continue;
        const double e = beam_energy<R>(P, k);
        if (!(fabs(e - e_peak) <= fwhm)) continue;
        const double w = P.w[k], y = P.y[k], z = P.z[k], py = P.py[k], pz = P.pz[k];
        a[0] += w; a[1] += w * e; a[2] += w * e * e;
        a[3] += w * y; a[4] += w * y * y; a[5] += w * py; a[6] += w * py * py; a[7] += w * y * py;
        a[8] += w * z; a[9] += w * z * z; a[10] += w * pz; a[11] += w * pz * pz; a[12] += w * z * pz;
        a[13] += 1.0;
    }
#pragma unroll
    for (int q = 0; q < 14; q++)
        for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
    if ((threadIdx.x & 31) == 0 && a[13] > 0)
        for (int q = 0; q < 14; q++) atomicAdd(out + q, a[q]);
}

// out = {count, sum w, sum w (g-1), sum w (g-1)^2} over alive particles with p_x > thr.
template <class R> __global__ void k_accel(SimDev<R> S, double thr, double *out) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const int np = S.d->np;
    double c = 0, sw = 0, s1 = 0, s2 = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        if (P.ix[k] == kDead) continue;
        const double px = P.px[k], py = P.py[k], pz = P.pz[k], w = P.w[k];
        if (!(px > thr)) continue;
        const double e = sqrt(1.0 + px * px + py * py + pz * pz) - 1.0;
        c += 1.0;
        sw += w;
        s1 += w * e;
        s2 += w * e * e;
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0 && c > 0) {
        atomicAdd(out, c);
        atomicAdd(out + 1, sw);
        atomicAdd(out + 2, s1);
        atomicAdd(out + 3, s2);
    }
}

// Canonical shape of a grid array kind: rows (i count) x cols (j count), complex flag.
__host__ __device__ inline void kind_shape(int kind, int nx, int nr, int &ni, int &nj, int &cplx) {
    cplx = 0;
    switch (kind) {
    case 10: case 16: ni = nx; nj = nr + 1; break;          // Ex, Jx
    case 11: case 17: ni = nx + 1; nj = nr; break;          // Er, Jr
    case 12: ni = nx; nj = nr; break;                       // Bt
    case 13: case 14: ni = nx + 1; nj = nr + 1; cplx = 1; break;
    default: ni = nx + 1; nj = nr + 1; break;               // chi, dq
    }
}

template <class R> __global__ void k_dump_field(SimDev<R> S, int kind, int c0, int c1, double *st) {
    int ni, nj, cplx;
    kind_shape(kind, S.geo.nx, S.geo.nr, ni, nj, cplx);
    // per-step deposits (chi, J, dQ) are read on the window of the step that made them
    const int off = S.d->off - (kind >= 15 ? S.d->last_shift : 0);
    const long long n = (long long)(c1 - c0) * nj;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = c0 + (int)(t / nj), j = (int)(t % nj);
        const long long id = S.geo.at(off, i, j);
        switch (kind) {
        case 10: st[t] = S.f.ex[id]; break;
        case 11: st[t] = S.f.er[id]; break;
        case 12: st[t] = S.f.bt[id]; break;
        case 13: case 14: {
            auto a = S.f.a[kind == 13 ? S.d->abuf : (S.d->abuf ^ 1)][id];
            st[2 * t] = a.x;
            st[2 * t + 1] = a.y;
            break;
        }
        case 15: st[t] = S.f.chi[id] * row_ichi(S.ph, j); break;
        case 16: st[t] = S.f.jxu[id] * row_ijx(S.ph, j); break;
        case 17: st[t] = S.f.jru[id] * row_ijr(S.ph, j); break;
        case 18: st[t] = S.f.dqu[id]; break;
        }
    }
}

template <class R>
__global__ void k_upload_field(SimDev<R> S, int kind, int c0, int c1, const double *st) {
    int ni, nj, cplx;
    kind_shape(kind, S.geo.nx, S.geo.nr, ni, nj, cplx);
    const int off = S.d->off;
    const long long n = (long long)(c1 - c0) * nj;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = c0 + (int)(t / nj), j = (int)(t % nj);
        const long long id = S.geo.at(off, i, j);
        switch (kind) {
        case 10: S.f.ex[id] = (R)st[t]; break;
        case 11: S.f.er[id] = (R)st[t]; break;
        case 12: S.f.bt[id] = (R)st[t]; break;
        case 13: case 14: {
            typename Cplx<R>::t v;
            v.x = (R)st[2 * t];
            v.y = (R)st[2 * t + 1];
            S.f.a[kind == 13 ? S.d->abuf : (S.d->abuf ^ 1)][id] = v;
            break;
        }
        }
    }
}

// Deterministic alive compaction: per-block counts, scan, then per-block ordered write.
template <class R> __global__ void k_alive_count(SimDev<R> S, int *blockcnt) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const int np = S.d->np;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool alive = k < np && P.ix[k] != kDead;
    const int c = __syncthreads_count(alive);
    if (threadIdx.x == 0) blockcnt[blockIdx.x] = c;
}
// total = sum of the per-block counts; written before the in-place exclusive scan
__global__ void k_sum_small(const int *v, int n, int *total) {
    int s = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += v[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += sh[q];
        *total = t;
    }
}
template <class R> __global__ void k_alive_write(SimDev<R> S, const int *blockbase, int *idx) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    __shared__ int wsum[TPB / 32];
    const int np = S.d->np;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool alive = k < np && P.ix[k] != kDead;
    const unsigned m = __ballot_sync(0xffffffffu, alive);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int q = 0; q < wid; q++) before += wsum[q];
    if (alive) idx[blockbase[blockIdx.x] + before + __popc(m & ((1u << lane) - 1u))] = k;
}

template <class R>
__global__ void k_dump_particles(SimDev<R> S, const int *idx, int k0, int k1, int comp, double *st) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k1 - k0; t += gridDim.x * blockDim.x) {
        const int k = idx[k0 + t];
        double v;
        switch (comp) {
        case 0: v = ((double)P.ix[k] + (double)P.ox[k]) * S.ph.dx; break;
        case 1: v = P.y[k]; break;
        case 2: v = P.z[k]; break;
        case 3: v = P.px[k]; break;
        case 4: v = P.py[k]; break;
        case 5: v = P.pz[k]; break;
        default: v = P.w[k]; break;
        }
        st[t] = v;
    }
}

// Upload of component comp of particles [k0, k1) from doubles.  x is split into the lab
// cell index and the in-cell offset.
template <class R>
__global__ void k_upload_particles(SimDev<R> S, int k0, int k1, int comp, const double *st) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k1 - k0; t += gridDim.x * blockDim.x) {
        const int k = k0 + t;
        const double v = st[t];
        switch (comp) {
        case 0: {
            const double xn = v / S.ph.dx;
            const double fl = floor(xn);
            P.ix[k] = (int)fl;
            R o = (R)(xn - fl);
            if (o >= (R)1) { o = (R)0; P.ix[k] += 1; }
            P.ox[k] = o;
            P.id[k] = (uint64_t)k;
            break;
        }
        case 1: P.y[k] = (R)v; break;
        case 2: P.z[k] = (R)v; break;
        case 3: P.px[k] = (R)v; break;
        case 4: P.py[k] = (R)v; break;
        case 5: P.pz[k] = (R)v; break;
        default: P.w[k] = (R)v; break;
        }
    }
}

// The particle store in its own layout (LPIC_DIAG_PARTICLES_NATIVE), component comp of
// particles [k0, k1): 0 the id (uint64), 1-7 the in-cell offset, y, z, px, py, pz, w (R), 8
// the lab cell (int32).  mode 0: buf[t] = component of slot idx[k0+t] (dump); mode 1: the
// component of slot k0+t = buf[t] (upload).  Plain copies of the stored bits.
template <class R> __device__ __forceinline__ R *native_comp(const Parts<R> &P, int comp) {
    switch (comp) {
    case 1: return P.ox;
    case 2: return P.y;
    case 3: return P.z;
    case 4: return P.px;
    case 5: return P.py;
    case 6: return P.pz;
    default: return P.w;
    }
}
template <class R>
__global__ void k_native(SimDev<R> S, const int *idx, int k0, int k1, int comp, void *buf, int mode) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    R *a = native_comp<R>(P, comp);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k1 - k0; t += gridDim.x * blockDim.x) {
        const int k = mode == 0 ? idx[k0 + t] : k0 + t;
        if (comp == 0) {
            if (mode == 0) static_cast<uint64_t *>(buf)[t] = P.id[k];
            else P.id[k] = static_cast<const uint64_t *>(buf)[t];
        } else if (comp == 8) {
            if (mode == 0) static_cast<int *>(buf)[t] = P.ix[k];
            else P.ix[k] = static_cast<const int *>(buf)[t];
        } else {
            if (mode == 0) static_cast<R *>(buf)[t] = a[k];
            else a[k] = static_cast<const R *>(buf)[t];
        }
    }
}

// mode 0: out[t] = id[idx[k0+t]] (dump);  mode 1: id[k0+t] = stage[t] (upload)
template <class R>
__global__ void k_ids(SimDev<R> S, const int *idx, int k0, int k1, const uint64_t *stage,
                      uint64_t *out, int mode) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k1 - k0; t += gridDim.x * blockDim.x) {
        if (mode == 0) out[t] = P.id[idx[k0 + t]];
        else P.id[k0 + t] = stage[t];
    }
}

// After an upload of n particles: remove those outside the window / r range, set counts.
template <class R> __global__ void k_finish_upload(SimDev<R> S, int n) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const long long s = S.d->shift;
    const double rmax = S.geo.nr * S.ph.dr;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long irel = (long long)P.ix[k] - s;
        const double y = P.y[k], z = P.z[k];
        if (irel < 0 || irel >= S.geo.nx || sqrt(y * y + z * z) >= rmax) P.ix[k] = kDead;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.d->np = n;
        S.d->n_alive = n;
    }
}

}  // namespace

template <class R> void launch_diag_ex_axis(const SimDev<R> &S, double *out, cudaStream_t st) {
    k_ex_axis<R><<<pgrid(S.geo.nx), TPB, 0, st>>>(S, out);
}
template <class R> void launch_diag_amax_waist(const SimDev<R> &S, double *out3, cudaStream_t st) {
    cudaMemsetAsync(out3, 0, 3 * sizeof(double), st);
    k_amax_waist<R><<<pgrid((long long)(S.geo.nx + 1) * (S.geo.nr + 1)), TPB, 0, st>>>(S, out3);
}
template <class R> void launch_diag_cont(const SimDev<R> &S, double *out2, cudaStream_t st) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    k_cont<R><<<pgrid((long long)S.geo.nx * S.geo.nr), TPB, 0, st>>>(S, out2);
}
template <class R>
void launch_diag_accel(const SimDev<R> &S, int np_upper, double thr, double *out4, cudaStream_t st) {
    cudaMemsetAsync(out4, 0, 4 * sizeof(double), st);
    k_accel<R><<<pgrid(np_upper), TPB, 0, st>>>(S, thr, out4);
}
template <class R>
void launch_beam_max(const SimDev<R> &S, int np_upper, double thr, double *out2, cudaStream_t st) {
    cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    k_beam_max<R><<<pgrid(np_upper), TPB, 0, st>>>(S, thr, out2);
}
template <class R>
void launch_beam_hist(const SimDev<R> &S, int np_upper, double thr, double width, int nbins, double *hist,
                      cudaStream_t st) {
    cudaMemsetAsync(hist, 0, nbins * sizeof(double), st);
    k_beam_hist<R><<<pgrid(np_upper), TPB, 0, st>>>(S, thr, width, nbins, hist);
}
template <class R>
void launch_beam_moments(const SimDev<R> &S, int np_upper, double thr, double e_peak, double fwhm, double *out14,
                         cudaStream_t st) {
    cudaMemsetAsync(out14, 0, 14 * sizeof(double), st);
    k_beam_moments<R><<<pgrid(np_upper), TPB, 0, st>>>(S, thr, e_peak, fwhm, out14);
}
template <class R>
void launch_dump_field(const SimDev<R> &S, int kind, int c0, int c1, double *stage, cudaStream_t st) {
    int ni, nj, cp;
    kind_shape(kind, S.geo.nx, S.geo.nr, ni, nj, cp);
    k_dump_field<R><<<pgrid((long long)(c1 - c0) * nj), TPB, 0, st>>>(S, kind, c0, c1, stage);
}
template <class R>
void launch_upload_field(const SimDev<R> &S, int kind, int c0, int c1, const double *stage,
                         cudaStream_t st) {
    int ni, nj, cp;
    kind_shape(kind, S.geo.nx, S.geo.nr, ni, nj, cp);
    k_upload_field<R><<<pgrid((long long)(c1 - c0) * nj), TPB, 0, st>>>(S, kind, c0, c1, stage);
}
template <class R>
void launch_alive_index(const SimDev<R> &S, int np_upper, int *idx, int *blockcnt, int *d_count,
                        cudaStream_t st) {
    const int nb = np_upper > 0 ? (np_upper + TPB - 1) / TPB : 1;
    k_alive_count<R><<<nb, TPB, 0, st>>>(S, blockcnt);
    k_sum_small<<<1, 1024, 0, st>>>(blockcnt, nb, d_count);
    scan_exclusive(blockcnt, nb, d_count + 1, st);   // d_count[1..] is the scan's block scratch
    k_alive_write<R><<<nb, TPB, 0, st>>>(S, blockcnt, idx);
}
template <class R>
void launch_dump_particles(const SimDev<R> &S, const int *idx, int k0, int k1, int comp,
                           double *stage, cudaStream_t st) {
    k_dump_particles<R><<<pgrid(k1 - k0), TPB, 0, st>>>(S, idx, k0, k1, comp, stage);
}
template <class R>
void launch_upload_particles(const SimDev<R> &S, int k0, int k1, int comp, const double *stage,
                             cudaStream_t st) {
    k_upload_particles<R><<<pgrid(k1 - k0), TPB, 0, st>>>(S, k0, k1, comp, stage);
}
template <class R>
void launch_set_ids(const SimDev<R> &S, const int *idx, int k0, int k1, const uint64_t *stage,
                    uint64_t *out, int mode, cudaStream_t st) {
    k_ids<R><<<pgrid(k1 - k0), TPB, 0, st>>>(S, idx, k0, k1, stage, out, mode);
}
template <class R>
void launch_native_particles(const SimDev<R> &S, const int *idx, int k0, int k1, int comp, void *buf, int mode,
                             cudaStream_t st) {
    if (k1 > k0) k_native<R><<<pgrid(k1 - k0), TPB, 0, st>>>(S, idx, k0, k1, comp, buf, mode);
}
template <class R> void launch_finish_upload(const SimDev<R> &S, int n, cudaStream_t st) {
    k_finish_upload<R><<<pgrid(n), TPB, 0, st>>>(S, n);
}

#define INST(R)                                                                                 \
    template void launch_diag_ex_axis<R>(const SimDev<R> &, double *, cudaStream_t);            \
    template void launch_diag_amax_waist<R>(const SimDev<R> &, double *, cudaStream_t);         \
    template void launch_diag_cont<R>(const SimDev<R> &, double *, cudaStream_t);               \
    template void launch_diag_accel<R>(const SimDev<R> &, int, double, double *, cudaStream_t); \
    template void launch_beam_max<R>(const SimDev<R> &, int, double, double *, cudaStream_t);   \
    template void launch_beam_hist<R>(const SimDev<R> &, int, double, double, int, double *,    \
                                      cudaStream_t);                                            \
    template void launch_beam_moments<R>(const SimDev<R> &, int, double, double, double, double *, \
                                         cudaStream_t);                                         \
    template void launch_dump_field<R>(const SimDev<R> &, int, int, int, double *, cudaStream_t); \
    template void launch_upload_field<R>(const SimDev<R> &, int, int, int, const double *,      \
                                         cudaStream_t);                                         \
    template void launch_alive_index<R>(const SimDev<R> &, int, int *, int *, int *, cudaStream_t); \
    template void launch_dump_particles<R>(const SimDev<R> &, const int *, int, int, int, double *, \
                                           cudaStream_t);                                       \
    template void launch_native_particles<R>(const SimDev<R> &, const int *, int, int, int, void *, int, \
                                             cudaStream_t);                                     \
    template void launch_upload_particles<R>(const SimDev<R> &, int, int, int, const double *,  \
                                             cudaStream_t);                                     \
    template void launch_set_ids<R>(const SimDev<R> &, const int *, int, int, const uint64_t *, \
                                    uint64_t *, int, cudaStream_t);                             \
    template void launch_finish_upload<R>(const SimDev<R> &, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace lpic
