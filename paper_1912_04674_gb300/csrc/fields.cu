// Grid kernels: Faraday + per-step node quantities, envelope solve, Ampere, envelope
// initialisation, live-region relocation.
//
// Thread mapping: threadIdx.x runs along the radial index j (contiguous in memory),
// threadIdx.y and the grid's y along the column index i.  In FP32_MIXED mode the axis
// row j = 0 of the envelope and of the Ex update is computed in FP64 (the 1/r and 4/dr
// axis terms); everything else in the working precision R.
#include "lpic_internal.cuh"
#include "window.cuh"

namespace lpic {

namespace {

constexpr int BX = 32, BY = 4;   // 4 rows: twice the envelope's FP64 axis blocks (measured 15 % faster envelope)

template <class R> __device__ __forceinline__ R sq(R v) { return v * v; }

// Faraday (Eq. MaxwellEqsCylindrical, first equation, FDTD of Sec. 3) on cells, B^n for the
// gathers, Phi^n = |A^n|^2/2 (Sec. 2) and its centred differences (Sec. 3) on nodes, and
// the clearing of the FP64 accumulators.  Every element of the live window incl. guards is
// written, so the per-step arrays always read zero outside their valid range.
// Tile (bx, by) of one simulation: threads run over j = bx*BX + tx, i = by*BY + ty - kG.
template <class R> __device__ __forceinline__ void prepass_tile(const SimDev<R> &S, int bx, int by) {
    const Geo g = S.geo;
    const int off = S.d->off;
    const int j = bx * BX + threadIdx.x;
    const int i = by * BY + (int)threadIdx.y - kG;
    if (bx == 0 && by == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        S.d->off_step = off;
        S.d->ticket = 0;   // for pass A
    }
    if (j >= g.P || i > g.nx + kG) return;
    const long long id = g.at(off, i, j);
    const R dt = S.k.dt, idx_ = S.k.idx, idr = S.k.idr;
    if (i == -1) {
        // the guard column left of the window: the Ampere launch that folds in the window step
        // leaves E and B_theta there (its old column 0) for this kernel to zero
        S.f.ex[id] = (R)0;
        S.f.er[id] = (R)0;
        S.f.bt[id] = (R)0;
    }

    R btn_here = (R)0;
    if (i >= 0 && i < g.nx && j < g.nr) {
        R bold = S.f.bt[id];
        R dexdr = (S.f.ex[id + 1] - S.f.ex[id]) * idr;
        R derdx = (S.f.er[g.at(off, i + 1, j)] - S.f.er[id]) * idx_;
        R bnew = bold + dt * (dexdr - derdx);
        S.f.bt[id] = bnew;
        btn_here = (R)0.5 * (bold + bnew);
    }
    if constexpr (sizeof(R) == 8) S.f.btn[id] = btn_here;   // FP32 gathers read the x-pairs below
    if constexpr (sizeof(R) == 4) {
        // x-pairs for the FP32 gathers, record (i, j) = (F(i, j), F(i+1, j)) for nodes i in
        // [-1, nx+1], j in [-1, nr+1].  E is not written by this kernel outside column -1 (whose
        // values are zero: its own thread knows them), so a thread reads its right neighbour.
        // B is updated in place, so B^n of node (i, j) is stored by its own thread into both
        // records that hold it: (i, j).x and (i-1, j).y (separate 4-byte words, no two threads
        // write the same one).  Row -1 holds the odd mirror, the negated row 0 (read for Er and
        // Btheta only).
        if (i >= -1 && i <= g.nx + 1 && j <= g.nr + 1) {
            float *bq = reinterpret_cast<float *>(S.f.btq);
            const long long P = g.P;
            bq[2 * (long long)id] = btn_here;
            if (i >= 0) bq[2 * ((long long)id - P) + 1] = btn_here;   // (i-1, j).y (column -2 unread)
            const bool guard = i == -1;
            const R ex0 = guard ? (R)0 : S.f.ex[id], er0 = guard ? (R)0 : S.f.er[id];
            const R ex1 = S.f.ex[id + P], er1 = S.f.er[id + P];
            S.f.exq[id] = make_float2(ex0, ex1);
            S.f.erq[id] = make_float2(er0, er1);
            if (j == 0) {
                S.f.exq[id - 1] = make_float2(-ex0, -ex1);
                S.f.erq[id - 1] = make_float2(-er0, -er1);
                bq[2 * ((long long)id - 1)] = -btn_here;                          // (i, -1).x
                if (i >= 0) bq[2 * ((long long)id - 1 - P) + 1] = -btn_here;      // (i-1, -1).y
            }
        }
    }

    Q4<R> q4;
    q4.phi = q4.gx = q4.gr = q4.pad = (R)0;
    if (i >= 0 && i <= g.nx && j <= g.nr) {
        const auto *A = S.f.a[S.d->abuf];
        auto c = A[id];
        auto xp = A[g.at(off, i + 1, j)];   // guard columns of A are zero
        auto xm = A[g.at(off, i - 1, j)];
        const R phxp = (R)0.5 * (xp.x * xp.x + xp.y * xp.y);
        const R phxm = (R)0.5 * (xm.x * xm.x + xm.y * xm.y);
        q4.phi = (R)0.5 * (c.x * c.x + c.y * c.y);
        q4.gx = (phxp - phxm) * S.k.hidx;
        if (j > 0) {
            auto rp = A[id + 1];             // row nr+1 is a zero guard
            auto rm = A[id - 1];
            const R phrp = (R)0.5 * (rp.x * rp.x + rp.y * rp.y);
            const R phrm = (R)0.5 * (rm.x * rm.x + rm.y * rm.y);
            q4.gr = (phrp - phrm) * S.k.hidr;
        }
    }
    S.f.pg[id] = q4;
    S.f.chi[id] = 0.0;
    S.f.jx[id] = 0.0;
    S.f.jr[id] = 0.0;
    if (S.ph.track_dq) S.f.dq[id] = 0.0;
}

template <class R> __global__ void k_prepass(SimDev<R> S) { prepass_tile<R>(S, blockIdx.x, blockIdx.y); }

// One node of Eq. (envelope_solver) in compute precision C:
//   A^{n+1} = (1+i dt)/(1+dt^2) [2A^n - (1+i dt)A^{n-1} + dt^2 (lap A - chi A + 2i dA/dx)].
// inv2rj = 1/(2 dr r_j) (unused on the axis row, whose radial part is 4 (A_1 - A_0)/dr^2).
template <class C, class V>
__device__ __forceinline__ void envelope_node(V cin, V xpin, V xmin, V rpin, V rmin, V amin,
                                              C chi, bool axis, C idx2, C idr2, C inv2rj,
                                              C hidx, C t, C t2, C p, C pt, C &ore, C &oim) {
    const C cx = (C)cin.x, cy = (C)cin.y;
    const C xpx = (C)xpin.x, xpy = (C)xpin.y, xmx = (C)xmin.x, xmy = (C)xmin.y;
    C lx = (xpx - (C)2 * cx + xmx) * idx2;
    C ly = (xpy - (C)2 * cy + xmy) * idx2;
    if (axis) {
        lx += (C)4 * ((C)rpin.x - cx) * idr2;
        ly += (C)4 * ((C)rpin.y - cy) * idr2;
    } else {
        const C rpx = (C)rpin.x, rpy = (C)rpin.y, rmx = (C)rmin.x, rmy = (C)rmin.y;
        lx += (rpx - (C)2 * cx + rmx) * idr2 + (rpx - rmx) * inv2rj;
        ly += (rpy - (C)2 * cy + rmy) * idr2 + (rpy - rmy) * inv2rj;
    }
    const C dxr = (xpx - xmx) * hidx, dxi = (xpy - xmy) * hidx;
    const C amx = (C)amin.x, amy = (C)amin.y;
    // bracket: lap - chi A + 2i dA/dx
    const C bx = lx - chi * cx - (C)2 * dxi;
    const C by = ly - chi * cy + (C)2 * dxr;
    const C rx = (C)2 * cx - (amx - t * amy) + t2 * bx;
    const C ry = (C)2 * cy - (amy + t * amx) + t2 * by;
    ore = p * rx - pt * ry;
    oim = p * ry + pt * rx;
}

// Envelope solve on the off-axis nodes in the working precision; A^{n+1} overwrites A^{n-1}
// in place (each node reads only its own A^{n-1}); Phi^{n+1/2} = (Phi^n + Phi^{n+1})/2 for the
// position push.  The axis row is done in FP64 by the extra last column of blocks.
template <class R> __device__ __forceinline__ void envelope_store(const SimDev<R> &S, int id, int ab,
                                                                  typename Cplx<R>::t c, R nre, R nim) {
    typename Cplx<R>::t o;
    o.x = nre;
    o.y = nim;
    S.f.a[ab ^ 1][id] = o;
    S.f.phih[id] = (R)0.5 * ((R)0.5 * (c.x * c.x + c.y * c.y) + (R)0.5 * (nre * nre + nim * nim));
}

template <class R> __device__ __forceinline__ void envelope_axis_node(const SimDev<R> &S, int i);

// Tile (bx, by): off-axis nodes j = 1 + bx*BX + tx, i = by*BY + ty; axis tile by takes the
// axis nodes i = by*BX*BY + (ty*BX + tx), one per thread (FP64), so that every lane of its
// warps does FP64 work (only the first ceil((Nx+1)/(BX*BY)) axis tiles have nodes).
template <class R>
__device__ __forceinline__ void envelope_tile(const SimDev<R> &S, int bx, int by, bool axis) {
    const Geo g = S.geo;
    const int off = S.d->off;
    if (axis) {
        const int i = by * BX * BY + threadIdx.y * BX + threadIdx.x;
        if (i <= g.nx) envelope_axis_node<R>(S, i);
        return;
    }
    const int j = 1 + bx * BX + threadIdx.x;
    const int i = by * BY + threadIdx.y;
    if (j > g.nr || i > g.nx) return;
    const int ab = S.d->abuf;
    const auto *A = S.f.a[ab];
    const int id = g.at(off, i, j);
    const auto c = A[id];
    const Kc<R> &K = S.k;
    R nre, nim;
    envelope_node<R>(c, A[g.at(off, i + 1, j)], A[g.at(off, i - 1, j)], A[id + 1], A[id - 1],
                     S.f.a[ab ^ 1][id], from_acc<R>(S.f.chi[id]) * K.tab[T_CHI * g.P + j], false, K.idx2,
                     K.idr2, K.tab[T_ENV1R * g.P + j], K.hidx, K.dt, K.dt2, K.envp, K.envpt, nre, nim);
    envelope_store<R>(S, id, ab, c, nre, nim);
}

template <class R> __global__ void k_envelope(SimDev<R> S) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) S.d->ticket = 0;   // for pass B
    envelope_tile<R>(S, blockIdx.x, blockIdx.y, blockIdx.x == gridDim.x - 1);
}

// The axis row j = 0 (even symmetry: radial part 4 (A_1 - A_0)/dr^2) in FP64, node (i, 0).
template <class R> __device__ __forceinline__ void envelope_axis_node(const SimDev<R> &S, int i) {
    const Geo g = S.geo;
    const int off = S.d->off;
    const int ab = S.d->abuf;
    const auto *A = S.f.a[ab];
    const int id = g.at(off, i, 0);
    const auto c = A[id];
    const Kc<R> &K = S.k;
    double dre, dim;
    envelope_node<double>(c, A[g.at(off, i + 1, 0)], A[g.at(off, i - 1, 0)], A[id + 1], c,
                          S.f.a[ab ^ 1][id], S.f.chi[id] * axis_factor(K.tab, g.P, 0), true, K.d_idx2, K.d_idr2, 0.0, K.d_hidx,
                          K.d_dt, K.d_dt2, K.d_envp, K.d_envpt, dre, dim);
    envelope_store<R>(S, id, ab, c, (R)dre, (R)dim);
}

// Ampere (Eq. MaxwellEqsCylindrical, second and third equations): Er on (i, j+1/2) with
// Er = 0 on the x ends; Ex on (i+1/2, j) with the axis row 4 B_{1/2}/dr and Ex = 0 at r_max.
template <class R> __device__ __forceinline__ void ampere_tile(const SimDev<R> &S, int off, int bx, int by) {
    const Geo g = S.geo;
    const int j = bx * BX + threadIdx.x;
    const int i = by * BY + threadIdx.y;
    if (j > g.nr || i > g.nx) return;
    const long long id = g.at(off, i, j);
    const R dt = S.k.dt;
    if (j < g.nr) {
        if (i == 0 || i == g.nx) {
            S.f.er[id] = (R)0;
        } else {
            R dbdx = (S.f.bt[id] - S.f.bt[g.at(off, i - 1, j)]) * S.k.idx;
            S.f.er[id] += dt * (-dbdx - from_acc<R>(S.f.jru[id]) * S.k.tab[T_JR * g.P + j]);
        }
    }
    if (i < g.nx) {
        if (j == g.nr) {
            S.f.ex[id] = (R)0;
        } else if (j == 0) {  // axis row in FP64
            double curl = S.k.d_4idr * (double)S.f.bt[id];
            S.f.ex[id] = (R)((double)S.f.ex[id] + S.k.d_dt * (curl - S.f.jxu[id] * axis_factor(S.k.tab, g.P, 1)));
        } else {
            R curl = S.k.tab[T_AMPP * g.P + j] * S.f.bt[id] - S.k.tab[T_AMPM * g.P + j] * S.f.bt[id - 1];
            S.f.ex[id] += dt * (curl - from_acc<R>(S.f.jxu[id]) * S.k.tab[T_JX * g.P + j]);
        }
    }
}

template <class R> __global__ void k_ampere(SimDev<R> S) { ampere_tile<R>(S, S.d->off, blockIdx.x, blockIdx.y); }

// Ampere with the step's moving-window work folded into the same launch: blocks [0, gw) zero
// the new guard columns and inject the plasma of the new front column (first, so that their
// latency-bound work starts with the launch), and the last of them advances the counters; the
// other blocks are the Ampere tiles, one per block.  Ampere addresses the grid through the
// offset the step began with (off_step), so it does not matter when the window blocks move
// `off`; E and B_theta of the old column 0, which Ampere updates and which becomes the guard
// column -1, are zeroed by the next step's prepass.  One launch instead of two, and no Ampere
// block waits for or counts anything.
template <class R> __global__ void __launch_bounds__(BX * BY) k_ampere_window(SimDev<R> S, int tiles_x, int gw) {
    const int b = blockIdx.x;
    if (b < gw) {
        __shared__ ColumnPlan<R> cp;
        window_fill<R>(S, b * (BX * BY) + threadIdx.y * BX + threadIdx.x, gw * (BX * BY), true, cp);
        window_done<R>(S, (unsigned)gw);
    } else {
        const int t = b - gw;
        ampere_tile<R>(S, S.d->off_step, t % tiles_x, t / tiles_x);
    }
}

// Binomial current filter (Sec. 4: an uncompensated binomial filter of 7 passes against
// numerical Cherenkov radiation): each pass replaces F_i by (F_{i-1} + 2 F_i + F_{i+1})/4 along x,
// F = 0 outside the window, on Jx, Jr and, when tracked, the charge change dQ (so that the
// filtered current keeps continuity with the filtered charge); working precision.  Tile
// (bx, by): rows j = bx*BX + tx, interior columns [by*FX, by*FX + FX).  The tile also holds
// `passes` halo columns on each side; their values go stale one column per pass, which never
// reaches the interior.  Tiles read the deposit arrays and write separate ones, so no tile
// reads a neighbour's output.  A tile whose halo lies inside the window applies the composed
// filter, the convolution with C(2p, k)/4^p, in one sweep; tiles at the window's ends run
// the passes one by one with the zero-outside rule.
constexpr int FX = 32;
template <class R>
__device__ __forceinline__ void filter_array(const double *F, double *out, const Geo &g, int off, int ni, int nj,
                                             int i0, int j, int passes, R (*t)[BX]) {
    const int tx = threadIdx.x, ty = threadIdx.y, W = FX + 2 * passes;
    for (int c = ty; c < W; c += BY) {
        const int i = i0 - passes + c;
        t[c][tx] = (i >= 0 && i < ni && j < nj) ? from_acc<R>(F[g.at(off, i, j)]) : (R)0;
    }
    __syncthreads();
    if (i0 - passes >= 0 && i0 + FX + passes <= ni) {
        // the tile and its halo lie inside the window: the passes compose to one convolution
        // with the binomial weights C(2p, k) / 4^p, with no boundary to re-apply between them
        __shared__ R wk[2 * kFilterMaxPasses + 1];
        if (tx == 0 && ty == 0) {
            R v = (R)1;
            for (int p = 0; p < 2 * passes; p++) v *= (R)0.5;   // 4^-p
            for (int k = 0; k <= 2 * passes; k++) {
                wk[k] = v;
                v = v * (R)(2 * passes - k) / (R)(k + 1);
            }
        }
        __syncthreads();
        for (int c = passes + ty; c < passes + FX; c += BY) {
            R acc = (R)0;
            for (int k = 0; k <= 2 * passes; k++) acc += wk[k] * t[c - passes + k][tx];
            const int i = i0 - passes + c;
            if (j < nj) out[g.at(off, i, j)] = to_acc(acc);
        }
        __syncthreads();   // the tile is reused by the next call
        return;
    }
    constexpr int NC = (FX + 2 * kFilterMaxPasses + BY - 1) / BY;
    for (int p = 0; p < passes; p++) {
        R nv[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) {
            const int c = ty + q * BY, i = i0 - passes + c;
            R v = (R)0;
            if (c < W && i >= 0 && i < ni) {
                const R l = c > 0 ? t[c - 1][tx] : (R)0;
                const R r = c < W - 1 ? t[c + 1][tx] : (R)0;
                v = (R)0.25 * l + (R)0.5 * t[c][tx] + (R)0.25 * r;
            }
            nv[q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NC; q++) {
            const int c = ty + q * BY;
            if (c < W) t[c][tx] = nv[q];
        }
        __syncthreads();
    }
    for (int c = passes + ty; c < passes + FX; c += BY) {
        const int i = i0 - passes + c;
        if (i < ni && j < nj) out[g.at(off, i, j)] = to_acc(t[c][tx]);
    }
    __syncthreads();   // the tile is reused by the next array
}

// Array `which` (0 Jx, 1 Jr, 2 dQ) of tile (bx, by).
template <class R> __device__ __forceinline__ void filter_tile(const SimDev<R> &S, int bx, int by, int which) {
    __shared__ R t[FX + 2 * kFilterMaxPasses][BX];
    const Geo g = S.geo;
    const int off = S.d->off, passes = S.ph.filter_passes;
    const int j = bx * BX + threadIdx.x, i0 = by * FX;
    if (which == 0) filter_array<R>(S.f.jx, S.f.jxu, g, off, g.nx, g.nr + 1, i0, j, passes, t);
    else if (which == 1) filter_array<R>(S.f.jr, S.f.jru, g, off, g.nx + 1, g.nr, i0, j, passes, t);
    else if (S.ph.track_dq) filter_array<R>(S.f.dq, S.f.dqu, g, off, g.nx + 1, g.nr + 1, i0, j, passes, t);
}

template <class R> __global__ void __launch_bounds__(BX * BY) k_filter(SimDev<R> S) {
    filter_tile<R>(S, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Fused forms over a batch: each block walks work items {simulation, bx, by, flag}.
template <class R>
__global__ void __launch_bounds__(BX * BY) k_prepass_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        prepass_tile<R>(pk.v[it.x], it.y, it.z);
    }
}
template <class R>
__global__ void __launch_bounds__(BX * BY) k_envelope_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        envelope_tile<R>(pk.v[it.x], it.y, it.z, it.w != 0);
    }
}
template <class R>
__global__ void __launch_bounds__(BX * BY) k_ampere_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        ampere_tile<R>(pk.v[it.x], pk.v[it.x].d->off, it.y, it.z);
    }
}
template <class R>
__global__ void __launch_bounds__(BX * BY) k_filter_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n) {
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int4 it = items[w];
        filter_tile<R>(pk.v[it.x], it.y, it.z, it.w);
    }
}

// Paraxial focused Gaussian pulse at t = 0 and t = -dt (paper Sec. 4 benchmarks):
// A = a0/D exp(-r^2/(w0^2 D)) exp(-(x-t-xc)^2/L^2), D = 1 + i (x-xf)/xR, xR = w0^2/2.
template <class R> __global__ void k_init_envelope(SimDev<R> S, double a0, double w0, double L,
                                                   double xc, double xf) {
    const Geo g = S.geo;
    const int off = S.d->off;
    const int j = blockIdx.x * BX + threadIdx.x;
    const int i = blockIdx.y * BY + threadIdx.y;
    if (j > g.nr || i > g.nx) return;
    const double x = (double)(S.d->shift + i) * S.ph.dx, r = j * S.ph.dr;
    const double xr = 0.5 * w0 * w0;
    const double u = (x - xf) / xr;                 // D = 1 + i u
    const double inv = 1.0 / (1.0 + u * u);         // 1/D = (1 - i u) inv
    const double er = -(r * r) / (w0 * w0) * inv;   // -r^2/(w0^2 D) = er (1 - i u)
    const double mag = exp(er);
    double sphase, cphase;
    sincos(-er * u, &sphase, &cphase);
    // a0/D * exp(er) * e^{-i er u}
    const double dre = a0 * inv, dim = -a0 * inv * u;
    const double bre = dre * cphase - dim * sphase, bim = dre * sphase + dim * cphase;
    const long long id = g.at(off, i, j);
    for (int lev = 0; lev < 2; lev++) {
        const double t = lev == 0 ? 0.0 : -S.ph.dt;
        const double lon = (x - t - xc) / L;
        const double env = mag * exp(-lon * lon);
        typename Cplx<R>::t v;
        v.x = (R)(bre * env);
        v.y = (R)(bim * env);
        S.f.a[S.d->abuf ^ lev][id] = v;
    }
}

template <class R> __global__ void k_relocate(SimDev<R> S, int new_off) {
    const Geo g = S.geo;
    const int off = S.d->off;
    const long long n = (long long)g.nlive * g.P;
    const long long src0 = (long long)off * g.P, dst0 = (long long)new_off * g.P;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        S.f.ex[dst0 + k] = S.f.ex[src0 + k];
        S.f.er[dst0 + k] = S.f.er[src0 + k];
        S.f.bt[dst0 + k] = S.f.bt[src0 + k];
        S.f.a[0][dst0 + k] = S.f.a[0][src0 + k];
        S.f.a[1][dst0 + k] = S.f.a[1][src0 + k];
    }
}
template <class R> __global__ void k_set_off(SimDev<R> S, int new_off) { S.d->off = new_off; }

inline dim3 grid2(int nj, int ni) { return dim3((nj + BX - 1) / BX, (ni + BY - 1) / BY); }

}  // namespace

template <class R> void launch_prepass(const SimDev<R> &S, cudaStream_t st) {
    k_prepass<R><<<grid2(S.geo.P, S.geo.nlive), dim3(BX, BY), 0, st>>>(S);
}
template <class R> void launch_envelope(const SimDev<R> &S, cudaStream_t st) {
    dim3 g = grid2(S.geo.nr, S.geo.nx + 1);
    g.x += 1;   // the axis-row blocks
    k_envelope<R><<<g, dim3(BX, BY), 0, st>>>(S);
}
template <class R> void launch_ampere(const SimDev<R> &S, cudaStream_t st) {
    k_ampere<R><<<grid2(S.geo.nr + 1, S.geo.nx + 1), dim3(BX, BY), 0, st>>>(S);
}
template <class R> void launch_ampere_window(const SimDev<R> &S, int inj_upper, cudaStream_t st) {
    const dim3 t = grid2(S.geo.nr + 1, S.geo.nx + 1);
    int work = (2 * kG + 1) * S.geo.P;
    if (inj_upper > work) work = inj_upper;
    const int gw = (work + BX * BY - 1) / (BX * BY);
    k_ampere_window<R><<<(int)(t.x * t.y) + gw, dim3(BX, BY), 0, st>>>(S, (int)t.x, gw);
}
template <class R> void launch_filter(const SimDev<R> &S, cudaStream_t st) {
    int tx, ty;
    grid_tiles(S.geo, 3, tx, ty);
    if (S.ph.filter_passes > 0) k_filter<R><<<dim3(tx, ty, S.ph.track_dq ? 3 : 2), dim3(BX, BY), 0, st>>>(S);
}
template <class R> void launch_init_envelope(const SimDev<R> &S, double a0, double w0, double L,
                                            double xc, double xf, cudaStream_t st) {
    k_init_envelope<R><<<grid2(S.geo.nr + 1, S.geo.nx + 1), dim3(BX, BY), 0, st>>>(S, a0, w0, L,
                                                                                   xc, xf);
}
// Copies the live region of the persistent arrays to physical offset new_off (regions
// must not overlap) and updates the descriptor.
template <class R> void launch_relocate(const SimDev<R> &S, int new_off, cudaStream_t st) {
    k_relocate<R><<<1216, 256, 0, st>>>(S, new_off);
    k_set_off<R><<<1, 1, 0, st>>>(S, new_off);
}

// Tile grids of one simulation (the single-simulation launches use the same tiling).
void grid_tiles(const Geo &g, int phase, int &tx, int &ty) {
    if (phase == 0) { tx = (g.P + BX - 1) / BX; ty = (g.nlive + BY - 1) / BY; }          // prepass
    else if (phase == 1) { tx = (g.nr + BX - 1) / BX + 1; ty = (g.nx + 1 + BY - 1) / BY; } // envelope
    else if (phase == 2) { tx = (g.nr + 1 + BX - 1) / BX; ty = (g.nx + 1 + BY - 1) / BY; } // ampere
    else { tx = (g.nr + 1 + BX - 1) / BX; ty = (g.nx + 1 + FX - 1) / FX; }                 // filter
}

template <class K> int resident(K *kernel, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
}

template <class R>
void launch_grid_multi(int phase, const SimPack<R> &pk, const int4 *items, int n, cudaStream_t st) {
    if (n <= 0) return;
    static int res[4] = {0, 0, 0, 0};
    const dim3 blk(BX, BY);
    if (phase == 0) {
        if (!res[0]) res[0] = resident(k_prepass_multi<R>, BX * BY);
        k_prepass_multi<R><<<n < res[0] ? n : res[0], blk, 0, st>>>(pk, items, n);
    } else if (phase == 1) {
        if (!res[1]) res[1] = resident(k_envelope_multi<R>, BX * BY);
        k_envelope_multi<R><<<n < res[1] ? n : res[1], blk, 0, st>>>(pk, items, n);
    } else if (phase == 2) {
        if (!res[2]) res[2] = resident(k_ampere_multi<R>, BX * BY);
        k_ampere_multi<R><<<n < res[2] ? n : res[2], blk, 0, st>>>(pk, items, n);
    } else {
        if (!res[3]) res[3] = resident(k_filter_multi<R>, BX * BY);
        k_filter_multi<R><<<n < res[3] ? n : res[3], blk, 0, st>>>(pk, items, n);
    }
}

#define INST(R)                                                                              \
    template void launch_grid_multi<R>(int, const SimPack<R> &, const int4 *, int, cudaStream_t); \
    template void launch_prepass<R>(const SimDev<R> &, cudaStream_t);                        \
    template void launch_envelope<R>(const SimDev<R> &, cudaStream_t);                       \
    template void launch_ampere<R>(const SimDev<R> &, cudaStream_t);                         \
    template void launch_ampere_window<R>(const SimDev<R> &, int, cudaStream_t);             \
    template void launch_filter<R>(const SimDev<R> &, cudaStream_t);                         \
    template void launch_init_envelope<R>(const SimDev<R> &, double, double, double, double, \
                                          double, cudaStream_t);                             \
    template void launch_relocate<R>(const SimDev<R> &, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace lpic
