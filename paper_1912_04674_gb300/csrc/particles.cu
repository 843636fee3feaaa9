// Particle kernels: pass A (gather, Cartesian projection, chi deposit, ponderomotive Boris
// momentum push), pass B (time-centred position push, charge-conserving current deposit,
// removal at the window edges) and the lattice loader.
//
// One thread per particle slot, grid-stride over the slot count held on the device.
// Particles are kept counting-sorted by cell, so the threads of a warp gather from a few
// neighbouring columns (L1 hits) and the FP64 atomics of a warp land on a few lines.
#include "lpic_internal.cuh"

namespace lpic {

namespace {

constexpr int TPB = 256;

// Linear-weight position of a particle on the four grids a gather can use.
template <class R> struct Loc {
    int ip, id;    // primal / dual x index (window-relative) of the lower node
    R fp, fd;      // their fractions
    int jp, jd;    // primal / dual r index (jd may be -1: odd ghost row)
    R gp, gd;
};

template <class R>
__device__ __forceinline__ Loc<R> locate(int irel, R ox, R rn, int nx, int nr) {
    Loc<R> L;
    irel = min(max(irel, -1), nx);
    L.ip = irel;
    L.fp = ox;
    R u = ox - (R)0.5;
    if (u < (R)0) { L.id = irel - 1; L.fd = u + (R)1; } else { L.id = irel; L.fd = u; }
    int j0 = min((int)rn, nr);
    L.jp = j0;
    L.gp = rn - (R)j0;
    R v = rn - (R)0.5;
    if (v < (R)0) { L.jd = -1; L.gd = v + (R)1; } else { L.jd = min((int)v, nr); L.gd = v - (R)L.jd; }
    return L;
}

// Gather with weights (1-f)(1-g), f(1-g), (1-f)g, fg; for odd-in-r quantities the ghost row
// j = -1 reads -F(j = 0).
template <class R>
__device__ __forceinline__ R gather4(const R *__restrict__ F, const Geo &geo, int off, int i,
                                     R f, int j, R gw, bool odd_ghost) {
    const long long b = geo.at(off, i, j < 0 ? 0 : j);
    R f00 = __ldg(F + b), f10 = __ldg(F + b + geo.P);
    R f01, f11;
    if (j < 0 && odd_ghost) {
        f01 = f00; f11 = f10; f00 = -f00; f10 = -f10;
    } else {
        f01 = __ldg(F + b + 1); f11 = __ldg(F + b + geo.P + 1);
    }
    return ((R)1 - f) * ((R)1 - gw) * f00 + f * ((R)1 - gw) * f10 + ((R)1 - f) * gw * f01 +
           f * gw * f11;
}

__device__ __forceinline__ void red_add(double *p, double v) {
    if (v != 0.0) atomicAdd(p, v);
}

// Pass A (paper Eqs. EquationsOfMotion and motion_equations_cartesian, modified Boris of
// Sec. 3; chi projected like a charge density divided by gamma, Sec. 2-3):
//   g0 = sqrt(1+|p|^2+Phi), p* = p + dt/2 (qE - gradPhi/(2 g0)), gt = sqrt(1+|p*|^2+Phi),
//   chi += q^2 w S/(gt V_chi),  F = qE - gradPhi/(2 gt),  Boris rotation with g- .
template <class R> __global__ void __launch_bounds__(TPB) k_pass_a(SimDev<R> S) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Geo geo = S.geo;
    const int off = S.d->off, np = S.d->np;
    const long long shift = S.d->shift;
    const R dt = (R)S.ph.dt, hdt = (R)(0.5 * S.ph.dt), idr = (R)(1.0 / S.ph.dr);
    const double cv0 = 3.0 / (kPi * S.ph.dr * S.ph.dr * S.ph.dx);      // 1/V_chi(axis)
    const double cv1 = 1.0 / (2.0 * kPi * S.ph.dr * S.ph.dr * S.ph.dx); // j/V_chi(j)
    const R q = (R)-1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const int ix = P.ix[k];
        if (ix == kDead) continue;
        const int irel = (int)((long long)ix - shift);
        const R ox = P.ox[k], y = P.y[k], z = P.z[k], w = P.w[k];
        R px = P.px[k], py = P.py[k], pz = P.pz[k];
        const R r = sqrt(y * y + z * z);
        R ct = (R)1, st = (R)0;
        if (r > (R)0) { ct = y / r; st = z / r; }
        const Loc<R> L = locate<R>(irel, ox, r * idr, geo.nx, geo.nr);
        const R exg = gather4<R>(S.f.ex, geo, off, L.id, L.fd, L.jp, L.gp, false);
        const R erg = gather4<R>(S.f.er, geo, off, L.ip, L.fp, L.jd, L.gd, true);
        const R btg = gather4<R>(S.f.btn, geo, off, L.id, L.fd, L.jd, L.gd, true);
        const R phg = gather4<R>(S.f.phi, geo, off, L.ip, L.fp, L.jp, L.gp, false);
        const R gxg = gather4<R>(S.f.gx, geo, off, L.ip, L.fp, L.jp, L.gp, false);
        const R grg = gather4<R>(S.f.gr, geo, off, L.ip, L.fp, L.jp, L.gp, false);
        const R Ex = exg, Ey = erg * ct, Ez = erg * st;
        const R By = -btg * st, Bz = btg * ct;               // Bx = 0
        const R Gx = gxg, Gy = grg * ct, Gz = grg * st;

        const R g0 = sqrt((R)1 + px * px + py * py + pz * pz + phg);
        const R i2g0 = (R)0.5 / g0;
        const R sx = px + hdt * (q * Ex - Gx * i2g0);
        const R sy = py + hdt * (q * Ey - Gy * i2g0);
        const R sz = pz + hdt * (q * Ez - Gz * i2g0);
        const R gt = sqrt((R)1 + sx * sx + sy * sy + sz * sz + phg);

        // susceptibility deposit on the primal nodes
        {
            const double base = (double)w / (double)gt;
            const double wx0 = (double)((R)1 - L.fp), wx1 = (double)L.fp;
            const double wr0 = (double)((R)1 - L.gp), wr1 = (double)L.gp;
            const double iv0 = L.jp == 0 ? cv0 : cv1 / L.jp;
            const double iv1 = cv1 / (L.jp + 1);
            const long long b = geo.at(off, L.ip, L.jp);
            red_add(S.f.chi + b, base * wx0 * wr0 * iv0);
            red_add(S.f.chi + b + geo.P, base * wx1 * wr0 * iv0);
            red_add(S.f.chi + b + 1, base * wx0 * wr1 * iv1);
            red_add(S.f.chi + b + geo.P + 1, base * wx1 * wr1 * iv1);
        }

        const R i2gt = (R)0.5 / gt;
        const R Fx = q * Ex - Gx * i2gt, Fy = q * Ey - Gy * i2gt, Fz = q * Ez - Gz * i2gt;
        const R mx = px + hdt * Fx, my = py + hdt * Fy, mz = pz + hdt * Fz;
        const R gm = sqrt((R)1 + mx * mx + my * my + mz * mz + phg);
        const R tf = q * hdt / gm;
        const R ty = tf * By, tz = tf * Bz;                  // tx = 0
        const R t2 = ty * ty + tz * tz;
        const R sf = (R)2 / ((R)1 + t2);
        const R vy = sf * ty, vz = sf * tz;
        // p' = p- + p- x t ; p+ = p- + p' x s   (t and s have no x component)
        const R ppx = mx + (my * tz - mz * ty);
        const R ppy = my + (-mx * tz);
        const R ppz = mz + (mx * ty);
        const R plx = mx + (ppy * vz - ppz * vy);
        const R ply = my + (-ppx * vz);
        const R plz = mz + (ppx * vy);
        P.px[k] = plx + hdt * Fx;
        P.py[k] = ply + hdt * Fy;
        P.pz[k] = plz + hdt * Fz;
    }
}

template <class R> __device__ __forceinline__ void shape3(int i0, R f, int base, R *s) {
    s[0] = s[1] = s[2] = (R)0;
    s[i0 - base] = (R)1 - f;
    s[i0 - base + 1] = f;
}

// Pass B: Phi^{n+1/2} at x^n, gbar = sqrt(1+|p|^2+Phi^{n+1/2}), x^{n+1} = x^n + dt p/gbar;
// charge-conserving current in the (x, r) index plane (Esirkepov decomposition):
//   Wx = DSx (S0r + DSr/2), Wr = DSr (S0x + DSx/2),
//   Jx(i+1/2,j) = (-q w/dt) sum_{k<=i} Wx(k,j) / (V_j/dx),
//   Jr(i,j+1/2) = (-q w/dt) sum_{l<=j} Wr(i,l) / (2 pi r_{j+1/2} dx).
// Particles leaving the next step's window (x < 0, x >= Nx dx) or reaching r >= r_max are
// marked dead after their deposit.
template <class R> __global__ void __launch_bounds__(TPB) k_pass_b(SimDev<R> S) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Geo geo = S.geo;
    const int off = S.d->off, np = S.d->np;
    const long long shift = S.d->shift, step = S.d->step;
    const int snext = window_shifts(S.ph, step, shift) ? 1 : 0;
    const R dt = (R)S.ph.dt, idr = (R)(1.0 / S.ph.dr), dtdx = (R)(S.ph.dt / S.ph.dx);
    const double rmax = geo.nr * S.ph.dr;
    const double ax0 = 1.0 / (kPi * 0.25 * S.ph.dr * S.ph.dr);       // 1/(V_0/dx)
    const double ax1 = 1.0 / (2.0 * kPi * S.ph.dr * S.ph.dr);        // j/(V_j/dx)
    const double ar = 1.0 / (2.0 * kPi * S.ph.dr * S.ph.dx);         // (j+1/2)*(1/area_r)
    const double jfac = 1.0 / S.ph.dt;                               // -q/dt, q = -1
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const int ix = P.ix[k];
        if (ix == kDead) continue;
        const int irel = (int)((long long)ix - shift);
        const R ox = P.ox[k], y = P.y[k], z = P.z[k], w = P.w[k];
        const R px = P.px[k], py = P.py[k], pz = P.pz[k];
        const R r0 = sqrt(y * y + z * z);
        const R rn0 = r0 * idr;
        const Loc<R> L = locate<R>(irel, ox, rn0, geo.nx, geo.nr);
        const R ph = gather4<R>(S.f.phih, geo, off, L.ip, L.fp, L.jp, L.gp, false);
        const R gbar = sqrt((R)1 + px * px + py * py + pz * pz + ph);
        const R ig = (R)1 / gbar;
        // The current is a difference of shape factors at two nearby positions: move x as
        // an in-cell offset, and take the new radius as r^n plus the radial step in the
        // cancellation-free form (dy (y0+y1) + dz (z0+z1)) / (r0 + r1).
        R ox1 = ox + dtdx * px * ig;
        const R dy = dt * py * ig, dz = dt * pz * ig;
        const R y1 = y + dy, z1 = z + dz;
        // a particle moves less than one cell per step (dt < dx, dt < dr); the clamps only
        // keep the 3-node shape window in range for non-finite input
        int di = min(max((int)floor(ox1), -1), 1);
        ox1 -= (R)di;
        if (ox1 >= (R)1) { ox1 -= (R)1; di = min(di + 1, 1); }
        const int ia = L.ip, ib = L.ip + di;
        const R r1 = sqrt(y1 * y1 + z1 * z1);
        const R rsum = r0 + r1;
        const R step_r = rsum > (R)0 ? (dy * (y + y1) + dz * (z + z1)) / rsum : (R)0;
        R rn1 = rn0 + step_r * idr;
        if (rn1 < (R)0) rn1 = (R)0;
        const int ja = L.jp, jb = min(max((int)rn1, ja - 1), ja + 1);
        const R fra = L.gp, frb = rn1 - (R)jb;
        const int imin = min(ia, ib), jmin = min(ja, jb);
        R s0x[3], s1x[3], s0r[3], s1r[3], dsx[3], dsr[3];
        shape3<R>(ia, ox, imin, s0x);
        shape3<R>(ib, ox1, imin, s1x);
        shape3<R>(ja, fra, jmin, s0r);
        shape3<R>(jb, frb, jmin, s1r);
#pragma unroll
        for (int c = 0; c < 3; c++) { dsx[c] = s1x[c] - s0x[c]; dsr[c] = s1r[c] - s0r[c]; }
        const double qf = (double)w * jfac;
        const long long b = geo.at(off, imin, jmin);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            const int j = jmin + l;
            const double inva = j == 0 ? ax0 : ax1 / j;
            R acc = (R)0;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                acc += dsx[c] * (s0r[l] + (R)0.5 * dsr[l]);
                red_add(S.f.jx + b + (long long)c * geo.P + l, qf * (double)acc * inva);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            R acc = (R)0;
#pragma unroll
            for (int l = 0; l < 2; l++) {
                acc += dsr[l] * (s0x[c] + (R)0.5 * dsx[c]);
                const double inva = ar / ((double)(jmin + l) + 0.5);
                red_add(S.f.jr + b + (long long)c * geo.P + l, qf * (double)acc * inva);
            }
        }
        if (S.ph.track_dq) {
            const double qw = -(double)w;
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int l = 0; l < 3; l++)
                    red_add(S.f.dq + b + (long long)c * geo.P + l,
                            qw * (double)(s1x[c] * s1r[l] - s0x[c] * s0r[l]));
        }
        const int irel_next = ib - snext;
        const bool dead = irel_next < 0 || irel_next >= geo.nx || (double)r1 >= rmax;
        P.ix[k] = dead ? kDead : ix + di;
        P.ox[k] = ox1;
        P.y[k] = y1;
        P.z[k] = z1;
    }
}

}  // namespace



namespace {
template <class R>
__global__ void k_load_columns(SimDev<R> S, const int *__restrict__ colbase, int ncols, int total) {
    const long long s = S.d->shift;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int lo = 0, hi = ncols;  // colbase[lo] <= t < colbase[hi]
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (colbase[mid] <= t) lo = mid; else hi = mid;
        }
        lattice_particle<R>(S, s + lo, t - colbase[lo], t);
    }
}
}  // namespace

inline int pgrid(int n) {
    int b = (n + TPB - 1) / TPB;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

template <class R> void launch_pass_a(const SimDev<R> &S, int np_upper, cudaStream_t st) {
    k_pass_a<R><<<pgrid(np_upper), TPB, 0, st>>>(S);
}
template <class R> void launch_pass_b(const SimDev<R> &S, int np_upper, cudaStream_t st) {
    k_pass_b<R><<<pgrid(np_upper), TPB, 0, st>>>(S);
}
template <class R> void launch_load_columns(const SimDev<R> &S, const int *d_colbase, int ncols,
                                            int total, cudaStream_t st) {
    if (total > 0) k_load_columns<R><<<pgrid(total), TPB, 0, st>>>(S, d_colbase, ncols, total);
}

#define INST(R)                                                                             \
    template void launch_pass_a<R>(const SimDev<R> &, int, cudaStream_t);                   \
    template void launch_pass_b<R>(const SimDev<R> &, int, cudaStream_t);                   \
    template void launch_load_columns<R>(const SimDev<R> &, const int *, int, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace lpic
