// Particle kernels: pass A (gather, Cartesian projection, chi deposit, ponderomotive Boris
// momentum push), pass B (time-centred position push, charge-conserving current deposit,
// removal at the window edges) and the lattice loader.
//
// Each block walks particle slots in block-sized groups (a block-uniform loop: every lane
// takes part in the warp reductions and the blocks may synchronise); the FP32 passes take two
// neighbouring slots per thread.  Particles are kept counting-sorted by cell, so runs of
// neighbouring lanes deposit onto the same nodes: each deposit is first summed over the warp's
// particles of its cell (exact, in integers, in FP32: warp-private shared-memory buckets in
// pass A, a segmented shuffle reduction over runs of lanes in pass B and in FP64), and only one
// lane per cell and deposit issues the FP64 global atomic.
#include <mutex>

#include "lpic_internal.cuh"

namespace lpic {

namespace {

constexpr int TPB = 256;
constexpr int TPB_B = 128;   // pass B: measured 2 % faster than 256 (pass A is not)
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned kNoKey = 0xffffffffu;

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
// j = -1 reads -F(j = 0) (selects, no branch).
template <class R>
__device__ __forceinline__ R gather4(const R *__restrict__ F, const Geo &geo, int off, int i,
                                     R f, int j, R gw, bool odd_ghost) {
    const bool ghost = odd_ghost && j < 0;
    const int b = geo.at(off, i, j < 0 ? 0 : j);
    const int up = ghost ? 0 : 1;
    const R l0 = __ldg(F + b), l1 = __ldg(F + b + geo.P);
    const R f01 = __ldg(F + b + up), f11 = __ldg(F + b + geo.P + up);
    const R f00 = ghost ? -l0 : l0, f10 = ghost ? -l1 : l1;
    const R lo = f00 + f * (f10 - f00), hi = f01 + f * (f11 - f01);
    return lo + gw * (hi - lo);
}



__device__ __forceinline__ void atom_add(double *p, double v) {
    if (v != 0.0) atomicAdd(p, v);
}
__device__ __forceinline__ void atom_add(double *p, float v) {
    if (v != 0.0f) atomicAdd(p, f2d_bits(v));
}

// ---- warp runs ----------------------------------------------------------------------------
// Particles are counting-sorted by cell, so lanes that deposit onto the same node sit next to
// each other: a warp splits into a few runs of consecutive lanes with equal key.  Lane l's run
// spans [head, end); lane l + o belongs to it iff l + o < end, so the segmented reductions
// below need no per-step membership shuffles.
struct Run {
    int head, end;   // first lane and one past the last lane of this lane's run
};
__device__ __forceinline__ Run run_of(unsigned key) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned prev = __shfl_up_sync(FULL, key, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0u || prev != key);
    const unsigned le = 0xffffffffu >> (31u - lane);          // lanes 0..lane
    Run r;
    r.head = 31 - __clz(heads & le);
    const unsigned after = heads & ~le;
    r.end = after ? __ffs(after) - 1 : 32;
    return r;
}

// Segmented suffix sums: afterwards the head lane of each run holds the run's sums.
// Stages stop at the warp's longest run (sorted particles rarely make runs of 32 lanes).
template <class T, int N> __device__ __forceinline__ void run_sums(const Run &r, T (&v)[N]) {
    const int lane = threadIdx.x & 31;
    const int span = (int)__reduce_max_sync(FULL, (unsigned)(r.end - r.head));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        if (o >= span) break;
        const bool in = lane + o < r.end;
#pragma unroll
        for (int q = 0; q < N; q++) {
            const T t = __shfl_down_sync(FULL, v[q], o);
            if (in) v[q] += t;
        }
    }
}

// q * 2^(e - 151) in FP64, exactly (|q| < 2^31, q != 0, 25 <= e <= 255): the integer converts
// to FP64 exactly (one conversion per value, issued by the run heads only), and the power of
// two is added to its exponent field, which stays in the normal range for these q and e.
// (Measured faster than assembling the bits with 32-bit integer operations.)
__device__ __forceinline__ double scaled_int_to_double(int q, int e) {
    const double d = (double)q;
    return __hiloint2double(__double2hiint(d) + ((e - 151) << 20), __double2loint(d));
}

// Deposit of each run's four values (row factors already applied; the lanes of a run share
// the key, hence the addresses) to addr[q] in FP64.
// FP32: summed exactly.  Value q belongs to group m = q*M/4 with bound bnd[m] >= |value|; every
// value of group m in the warp is scaled by 2^(151 - e_m), e_m the largest exponent field among
// the warp's group-m bounds (so that 32 scaled values cannot overflow 31 bits), rounded to an
// integer (one rounding of at most 2^-25 of the warp's largest bound), and the run's integers
// are summed exactly; the head lane turns each sum into FP64 exactly and adds it.  A
// non-finite value in the warp makes its group's deposits NaN.
template <int M>
__device__ __forceinline__ void run_deposit(const Run &r, unsigned key, const float (&v)[4], const float (&bnd)[M],
                                            double *const (&addr)[4]) {
    int qi[4], ec[M];
    bool bad[M];
#pragma unroll
    for (int m = 0; m < M; m++) {
        const unsigned e = ((unsigned)__float_as_uint(bnd[m]) >> 23) & 0xffu;
        const int emax = (int)__reduce_max_sync(FULL, e);
        bad[m] = emax == 255;
        ec[m] = min(max(emax, 25), 254);
        const float sc = __uint_as_float((unsigned)(278 - ec[m]) << 23);   // 2^(151 - ec)
#pragma unroll
        for (int q = m * 4 / M; q < (m + 1) * 4 / M; q++) qi[q] = bad[m] ? 0 : __float2int_rn(v[q] * sc);
    }
    run_sums<int, 4>(r, qi);
    if (key == kNoKey || (int)(threadIdx.x & 31) != r.head) return;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int m = q * M / 4;
        if (bad[m]) atomicAdd(addr[q], __longlong_as_double(0x7ff8000000000000ll));
        else if (qi[q] != 0) atomicAdd(addr[q], scaled_int_to_double(qi[q], ec[m]));
    }
}
template <int M>
__device__ __forceinline__ void run_deposit(const Run &r, unsigned key, const double (&v)[4], const double (&)[M],
                                            double *const (&addr)[4]) {
    double s[4] = {v[0], v[1], v[2], v[3]};
    run_sums<double, 4>(r, s);
    if (key == kNoKey || (int)(threadIdx.x & 31) != r.head) return;
#pragma unroll
    for (int q = 0; q < 4; q++) atom_add(addr[q], s[q]);
}

// Particle registers of one slot.
template <class R> struct PReg {
    int ix;
    R ox, y, z, px, py, pz, w;
};
// Slot k if k < lim (the end of the block's chunk), else an empty slot.
template <class R> __device__ __forceinline__ PReg<R> load_particle(const Parts<R> &P, int k, int lim) {
    PReg<R> q;
    const bool in = k < lim;
    const int kk = in ? k : 0;
    q.ix = in ? P.ix[kk] : kDead;
    q.ox = in ? P.ox[kk] : (R)0;
    q.y = in ? P.y[kk] : (R)0;
    q.z = in ? P.z[kk] : (R)0;
    q.px = in ? P.px[kk] : (R)0;
    q.py = in ? P.py[kk] : (R)0;
    q.pz = in ? P.pz[kk] : (R)0;
    q.w = in ? P.w[kk] : (R)0;
    return q;
}

// Work split of the single-simulation particle passes: each block first takes a contiguous share
// of num/den of the slots, in units of U slots (one iteration of the block), then single units
// of the rest from the descriptor's ticket counter (zeroed by the kernel before), so that the
// blocks of the SMs that finish their share early take more of the end.  With equal shares
// only, the SMs' active cycles spread by 5-7 % of the launch (ncu sm__cycles_active min, avg,
// max) and the launch lasted as long as the slowest.  Measured (3 alternating runs each): pass
// A 0.0923 ms with equal shares, 0.0896 at 7/8, 0.0883 at 15/16, 0.0904 at 31/32, 0.092 at
// 3/4, 0.098 at 1/2;
// pass B 0.0925, 0.0905 at 7/8, 0.0945 at 15/16, 0.0915 at 3/4.  Each unit handed out costs
// the ticket's round trip with the block waiting at a barrier; claiming the next unit one
// iteration ahead (hiding that round trip) measured slower in pass B (spills) and within 0.5 %
// in pass A.  The one-particle-per-thread passes (FP64, and FP32 pass B with the charge change)
// take 7/8.
struct Split {
    int sbeg, send;   // the block's contiguous share
    int dyn0, nunits; // first unit handed out by ticket, number of units
};
__device__ __forceinline__ Split split_slots(int np, int vb, int nvb, int U, int num, int den) {
    Split s;
    s.nunits = (np + U - 1) / U;
    const int per = (int)((long long)s.nunits * num / den / nvb);
    s.sbeg = (int)min((long long)vb * per * U, (long long)np);
    s.send = (int)min((long long)(vb + 1) * per * U, (long long)np);
    s.dyn0 = nvb * per;
    return s;
}
// The block's next unit (block-uniform; every thread calls it).
__device__ __forceinline__ int next_unit(int *ticket, int dyn0) {
    __shared__ int w;
    __syncthreads();   // every thread has read the previous unit
    if (threadIdx.x == 0) w = dyn0 + atomicAdd(ticket, 1);
    __syncthreads();
    return w;
}

// Pass A (paper Eqs. EquationsOfMotion and motion_equations_cartesian, modified Boris of
// Sec. 3; chi projected like a charge density divided by gamma, Sec. 2-3):
//   g0 = sqrt(1+|p|^2+Phi), p* = p + dt/2 (qE - gradPhi/(2 g0)), gt = sqrt(1+|p*|^2+Phi),
//   chi += q^2 w S/(gt V_chi),  F = qE - gradPhi/(2 gt),  Boris rotation with g- .
// Every lane computes (a hole or a lane past the end works on harmless zeros or stale
// values) and the results are masked, so the loop body has no data-dependent branch.
// Slots of block vb of nvb (single launch: near-equal contiguous chunks of the live slots),
// or of item vb of a fixed size csize > 0 (fused launches), clipped to the live slots.
__device__ __forceinline__ int2 slot_range(int np, int vb, int nvb, int csize) {
    int chunk = csize;
    if (chunk <= 0) chunk = ((np + nvb - 1) / nvb + TPB - 1) / TPB * TPB;
    const long long b = (long long)vb * chunk;
    const int begin = b < np ? (int)b : np;
    return make_int2(begin, min(begin + chunk, np));
}

// Gather from x-pairs (FP32 pass A): the same weights and the same sum as gather4, with the
// two columns of a row in one 8-byte record and the next row in the next record (an immediate
// offset from the first); row -1 holds the odd mirror.
__device__ __forceinline__ float gather_q(const float2 *__restrict__ G, const Geo &geo, int off, int i, float f,
                                          int j, float gw) {
    const float2 *r = G + geo.at(off, i, j);
    const float2 c0 = __ldg(r), c1 = __ldg(r + 1);
    const float lo = c0.x + f * (c0.y - c0.x), hi = c1.x + f * (c1.y - c1.x);
    return lo + gw * (hi - lo);
}

// A (Phi, dPhi/dx, dPhi/dr) record through the read-only data path (the array is not written
// during the pass; measured 5 % off FP32 pass A against plain loads).
__device__ __forceinline__ Q4<float> ldg_q4(const Q4<float> *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    Q4<float> q;
    q.phi = v.x;
    q.gx = v.y;
    q.gr = v.z;
    q.pad = v.w;
    return q;
}
__device__ __forceinline__ Q4<double> ldg_q4(const Q4<double> *p) {
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p)), v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    Q4<double> q;
    q.phi = v0.x;
    q.gx = v0.y;
    q.gr = v1.x;
    q.pad = v1.y;
    return q;
}

// Results of pass A for one particle: its susceptibility deposit (four primal nodes from b,
// row factors applied, with a bound on their size) and its new momentum.
template <class R> struct AOut {
    unsigned key;   // b, or kNoKey for a hole
    int b;
    R v[4], bnd;
    R px, py, pz;
};

template <class R>
__device__ __forceinline__ AOut<R> a_particle(const SimDev<R> &S, const Geo &geo, int off, long long shift,
                                              int ix, R ox, R y, R z, R px, R py, R pz, R w) {
    const R hdt = S.k.hdt, idr = S.k.idr;
    const R q = (R)-1;
    const bool alive = ix != kDead;
    const int irel = (int)((long long)ix - shift);
    const R r2 = y * y + z * z;
    const bool onaxis = !(r2 > (R)0);
    const R ir = onaxis ? (R)0 : rsqrt_<R>(r2);
    const R r = r2 * ir, ct = onaxis ? (R)1 : y * ir, st = z * ir;
    const Loc<R> L = locate<R>(irel, ox, r * idr, geo.nx, geo.nr);
    const R exg = gather4<R>(S.f.ex, geo, off, L.id, L.fd, L.jp, L.gp, false);
    const R erg = gather4<R>(S.f.er, geo, off, L.ip, L.fp, L.jd, L.gd, true);
    const R btg = gather4<R>(S.f.btn, geo, off, L.id, L.fd, L.jd, L.gd, true);
    // Phi, dPhi/dx, dPhi/dr share the primal weights: one 4-vector load per corner
    const int b = geo.at(off, L.ip, L.jp);
    const R wx0 = (R)1 - L.fp, wr0 = (R)1 - L.gp;
    const R w00 = wx0 * wr0, w10 = L.fp * wr0, w01 = wx0 * L.gp, w11 = L.fp * L.gp;
    const Q4<R> q00 = ldg_q4(S.f.pg + b), q10 = ldg_q4(S.f.pg + b + geo.P);
    const Q4<R> q01 = ldg_q4(S.f.pg + b + 1), q11 = ldg_q4(S.f.pg + b + geo.P + 1);
    const R phg = w00 * q00.phi + w10 * q10.phi + w01 * q01.phi + w11 * q11.phi;
    const R gxg = w00 * q00.gx + w10 * q10.gx + w01 * q01.gx + w11 * q11.gx;
    const R grg = w00 * q00.gr + w10 * q10.gr + w01 * q01.gr + w11 * q11.gr;
    const R Ex = exg, Ey = erg * ct, Ez = erg * st;
    const R By = -btg * st, Bz = btg * ct;               // Bx = 0
    const R Gx = gxg, Gy = grg * ct, Gz = grg * st;

    const R i2g0 = (R)0.5 * rsqrt_<R>((R)1 + px * px + py * py + pz * pz + phg);
    const R sx = px + hdt * (q * Ex - Gx * i2g0);
    const R sy = py + hdt * (q * Ey - Gy * i2g0);
    const R sz = pz + hdt * (q * Ez - Gz * i2g0);
    const R rgt = rsqrt_<R>((R)1 + sx * sx + sy * sy + sz * sz + phg);   // 1/gt

    // susceptibility: w S/gt on the four primal nodes (q^2/m = 1); the envelope applies 1/V_chi
    // per row
    AOut<R> o;
    const R base_w = alive ? w * rgt : (R)0;
    o.v[0] = base_w * w00; o.v[1] = base_w * w10; o.v[2] = base_w * w01; o.v[3] = base_w * w11;
    o.bnd = base_w;
    o.key = alive ? (unsigned)b : kNoKey;
    o.b = b;

    const R i2gt = (R)0.5 * rgt;
    const R Fx = q * Ex - Gx * i2gt, Fy = q * Ey - Gy * i2gt, Fz = q * Ez - Gz * i2gt;
    const R mx = px + hdt * Fx, my = py + hdt * Fy, mz = pz + hdt * Fz;
    const R tf = q * hdt * rsqrt_<R>((R)1 + mx * mx + my * my + mz * mz + phg);
    const R ty = tf * By, tz = tf * Bz;                  // tx = 0
    const R sf = (R)2 / ((R)1 + ty * ty + tz * tz);
    const R vy = sf * ty, vz = sf * tz;
    // p' = p- + p- x t ; p+ = p- + p' x s   (t and s have no x component)
    const R ppx = mx + (my * tz - mz * ty);
    const R ppy = my + (-mx * tz);
    const R ppz = mz + (mx * ty);
    o.px = mx + (ppy * vz - ppz * vy) + hdt * Fx;
    o.py = my + (-ppx * vz) + hdt * Fy;
    o.pz = mz + (ppx * vy) + hdt * Fz;
    return o;
}

template <class R> __device__ __forceinline__ void pass_a_body(const SimDev<R> &S, int vb, int nvb, int csize) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Geo geo = S.geo;
    const int off = S.d->off, np = S.d->np;
    const long long shift = S.d->shift;
    // each block walks contiguous runs of slots, so that its successive iterations gather from
    // neighbouring cells (field lines stay in L1)
    auto range = [&](int begin, int end) {
        int k = begin + threadIdx.x;
        PReg<R> cur = load_particle<R>(P, k, end);
        for (int base = begin; base < end; base += TPB, k += TPB) {
            const PReg<R> nxt = load_particle<R>(P, k + TPB, end);   // prefetch
            const AOut<R> o = a_particle<R>(S, geo, off, shift, cur.ix, cur.ox, cur.y, cur.z, cur.px, cur.py,
                                            cur.pz, cur.w);
            if (cur.ix != kDead) {
                P.px[k] = o.px;
                P.py[k] = o.py;
                P.pz[k] = o.pz;
            }
            const Run run = run_of(o.key);
            const R bnd[1] = {o.bnd};
            double *const addr[4] = {S.f.chi + o.b, S.f.chi + o.b + geo.P, S.f.chi + o.b + 1,
                                     S.f.chi + o.b + geo.P + 1};
            run_deposit<1>(run, o.key, o.v, bnd, addr);
            cur = nxt;
        }
    };
    if (csize > 0) {   // a work item of a fused launch
        const int2 rg = slot_range(np, vb, nvb, csize);
        range(rg.x, rg.y);
        return;
    }
    const Split sp = split_slots(np, vb, nvb, TPB, 7, 8);   // the work split of the FP32 passes
    range(sp.sbeg, sp.send);
    for (;;) {
        const int u = next_unit(&S.d->ticket, sp.dyn0);
        if (u >= sp.nunits) break;
        range(u * TPB, min(u * TPB + TPB, np));
    }
}

// ---- FP32: two neighbouring particles per thread ----------------------------------------------
// Thread t of a block takes slots 2t and 2t+1 of each group of 2*TPB (8-byte vector loads and
// stores), and the warp deposits its 64 particles as one sequence: element a then element b of
// lane 0, then of lane 1, ...  Within a lane, b absorbs a when their cells agree.  A chain is a
// run of lanes whose single (absorbed) element continues the previous lane's b cell; chains are
// summed by a segmented prefix scan, so the chain's last lane holds its sum.  A lane whose a
// and b differ deposits a itself, adding the sum of the chain that ends on the previous lane
// when that chain has a's cell; a chain's last lane deposits b's sum unless the next lane's
// first element continues it.  Values are scaled by 2^(150 - e) (64 values per warp) and the
// sums are exact in 32-bit integers.  (Measured 12 % faster than one particle per thread:
// fewer load, reduction and atomic instructions per particle.)  The push of the pair runs in
// packed FP32x2 arithmetic (a_pair, b_pair): 30 fewer thread instructions per particle in
// pass A (292 -> 262) and 15 in pass B, 4-6 % off each pass.  Pass A deposits through the
// warp's shared-memory node buckets instead (node_bucket_deposit: per-cell buckets took pass A
// from 0.105 to 0.101 ms, per-node ones to 0.093 ms); in pass B per-cell buckets cut
// instructions as well but the pass ran 2 % slower, so it keeps the runs.

// The position half of a pair (carried one iteration ahead) and the rest (loaded at the top
// of the iteration that uses it).  Particle data is read and written once per pass: it goes
// through the caches as streaming data (evict first), which leaves L2 to the field arrays
// the gathers read (measured 2.5 % off the step).
struct PPos {
    int2 ix;
    float2 ox, y, z;
};
struct PMom {
    float2 px, py, pz, w;
};
__device__ __forceinline__ float2 ld_pair(const float *a, int k, bool two, bool one) {
    if (two) return __ldcs(reinterpret_cast<const float2 *>(a + k));
    return make_float2(one ? __ldcs(a + k) : 0.f, 0.f);
}
__device__ __forceinline__ PPos load_pos(const Parts<float> &P, int k, int lim) {
    const bool two = k + 1 < lim, one = k < lim;
    PPos q;
    if (two) q.ix = __ldcs(reinterpret_cast<const int2 *>(P.ix + k));
    else q.ix = make_int2(one ? __ldcs(P.ix + k) : kDead, kDead);
    q.ox = ld_pair(P.ox, k, two, one);
    q.y = ld_pair(P.y, k, two, one);
    q.z = ld_pair(P.z, k, two, one);
    return q;
}
__device__ __forceinline__ PMom load_mom(const Parts<float> &P, int k, int lim) {
    const bool two = k + 1 < lim, one = k < lim;
    PMom q;
    q.px = ld_pair(P.px, k, two, one);
    q.py = ld_pair(P.py, k, two, one);
    q.pz = ld_pair(P.pz, k, two, one);
    q.w = ld_pair(P.w, k, two, one);
    return q;
}

// ---- packed FP32x2 arithmetic ------------------------------------------------------------------
// The sm_100 family's paired FP32 instructions apply one IEEE operation (round to nearest) to
// both halves of a float2.  The FP32 passes hold the two particles of a lane as such pairs
// (x: the first slot, y: the second), so each elementwise step of their push is one
// instruction for both particles.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }

// locate() for a pair: the same indices and fractions.
struct Loc2 {
    int ipa, ipb, ida, idb, jpa, jpb, jda, jdb;
    float2 fp, fd, gp, gd;
};
__device__ __forceinline__ Loc2 locate2(int ia, int ib, float2 ox, float2 rn, int nx, int nr) {
    Loc2 L;
    L.ipa = min(max(ia, -1), nx);
    L.ipb = min(max(ib, -1), nx);
    L.fp = ox;
    const float2 u = add2(ox, dup2(-0.5f));
    const bool ua = u.x < 0.f, ub = u.y < 0.f;
    L.ida = ua ? L.ipa - 1 : L.ipa;
    L.idb = ub ? L.ipb - 1 : L.ipb;
    L.fd = add2(u, make_float2(ua ? 1.f : 0.f, ub ? 1.f : 0.f));
    L.jpa = min((int)rn.x, nr);
    L.jpb = min((int)rn.y, nr);
    L.gp = sub2(rn, make_float2((float)L.jpa, (float)L.jpb));
    const float2 v = add2(rn, dup2(-0.5f));
    L.jda = v.x < 0.f ? -1 : min((int)v.x, nr);
    L.jdb = v.y < 0.f ? -1 : min((int)v.y, nr);
    L.gd = sub2(v, make_float2((float)L.jda, (float)L.jdb));   // v + 1 on the ghost row
    return L;
}

// Phi, dPhi/dx, dPhi/dr of one particle from the four records of its primal cell.
__device__ __forceinline__ void gather_pg(const Q4<float> *__restrict__ pg, int b, int P, float w00, float w10,
                                          float w01, float w11, float &ph, float &gx, float &gr) {
    const Q4<float> q00 = ldg_q4(pg + b), q10 = ldg_q4(pg + b + P);
    const Q4<float> q01 = ldg_q4(pg + b + 1), q11 = ldg_q4(pg + b + P + 1);
    ph = w00 * q00.phi + w10 * q10.phi + w01 * q01.phi + w11 * q11.phi;
    gx = w00 * q00.gx + w10 * q10.gx + w01 * q01.gx + w11 * q11.gx;
    gr = w00 * q00.gr + w10 * q10.gr + w01 * q01.gr + w11 * q11.gr;
}

// Pass A for the two particles of a lane: a_particle's arithmetic (gathers per particle, the
// rest in pairs).  With q = -1 the signs are folded: F' = E + Grad Phi/(2 g) = -F, and with
// h = hdt B_theta / g-, the rotation vector is t = (0, h sin, -h cos).
__device__ __forceinline__ void a_pair(const SimDev<float> &S, const Geo &geo, int off, long long shift,
                                       const PPos &c, const PMom &m, AOut<float> &oa, AOut<float> &ob) {
    const float hdt = S.k.hdt;
    const bool la = c.ix.x != kDead, lb = c.ix.y != kDead;
    const float2 r2 = fma2(c.y, c.y, mul2(c.z, c.z));
    const bool axa = !(r2.x > 0.f), axb = !(r2.y > 0.f);
    const float2 ir = make_float2(axa ? 0.f : rsqrtf(r2.x), axb ? 0.f : rsqrtf(r2.y));
    float2 ct = mul2(c.y, ir);
    ct.x = axa ? 1.f : ct.x;
    ct.y = axb ? 1.f : ct.y;
    const float2 st = mul2(c.z, ir);
    const float2 rn = mul2(mul2(r2, ir), dup2(S.k.idr));
    const Loc2 L = locate2((int)((long long)c.ix.x - shift), (int)((long long)c.ix.y - shift), c.ox, rn,
                           geo.nx, geo.nr);
    // live particles have id >= -1; the clamp keeps holes (irel = -1) in the arrays
    const int ida = L.ida < -1 ? -1 : L.ida, idb = L.idb < -1 ? -1 : L.idb;
    float2 ex, er, bt;
    ex.x = gather_q(S.f.exq, geo, off, ida, L.fd.x, L.jpa, L.gp.x);
    ex.y = gather_q(S.f.exq, geo, off, idb, L.fd.y, L.jpb, L.gp.y);
    er.x = gather_q(S.f.erq, geo, off, L.ipa, L.fp.x, L.jda, L.gd.x);
    er.y = gather_q(S.f.erq, geo, off, L.ipb, L.fp.y, L.jdb, L.gd.y);
    bt.x = gather_q(S.f.btq, geo, off, ida, L.fd.x, L.jda, L.gd.x);
    bt.y = gather_q(S.f.btq, geo, off, idb, L.fd.y, L.jdb, L.gd.y);
    const int ba = geo.at(off, L.ipa, L.jpa), bb = geo.at(off, L.ipb, L.jpb);
    const float2 one = dup2(1.f);
    const float2 wx0 = sub2(one, L.fp), wr0 = sub2(one, L.gp);
    const float2 w00 = mul2(wx0, wr0), w10 = mul2(L.fp, wr0), w01 = mul2(wx0, L.gp), w11 = mul2(L.fp, L.gp);
    float2 ph, gx, gr;
    gather_pg(S.f.pg, ba, geo.P, w00.x, w10.x, w01.x, w11.x, ph.x, gx.x, gr.x);
    gather_pg(S.f.pg, bb, geo.P, w00.y, w10.y, w01.y, w11.y, ph.y, gx.y, gr.y);
    const float2 ey = mul2(er, ct), ez = mul2(er, st);
    const float2 gy = mul2(gr, ct), gz = mul2(gr, st);
    const float2 onep = add2(one, ph);
    const float2 nh = dup2(-hdt);

    // half-step momenta p* = p - hdt (E + Grad Phi/(2 g0)), g0 = sqrt(1 + |p|^2 + Phi)
    const float2 i2g0 = mul2(dup2(0.5f), rsqrt2(fma2(m.pz, m.pz, fma2(m.py, m.py, fma2(m.px, m.px, onep)))));
    const float2 sx = fma2(nh, fma2(gx, i2g0, ex), m.px);
    const float2 sy = fma2(nh, fma2(gy, i2g0, ey), m.py);
    const float2 sz = fma2(nh, fma2(gz, i2g0, ez), m.pz);
    const float2 rgt = rsqrt2(fma2(sz, sz, fma2(sy, sy, fma2(sx, sx, onep))));   // 1/gt

    // susceptibility: w S/gt on the four primal nodes (the envelope applies 1/V_chi per row)
    const float2 bw = mul2(m.w, rgt);
    const float2 bwl = make_float2(la ? bw.x : 0.f, lb ? bw.y : 0.f);
    const float2 v0 = mul2(bwl, w00), v1 = mul2(bwl, w10), v2 = mul2(bwl, w01), v3 = mul2(bwl, w11);
    oa.v[0] = v0.x; oa.v[1] = v1.x; oa.v[2] = v2.x; oa.v[3] = v3.x;
    ob.v[0] = v0.y; ob.v[1] = v1.y; ob.v[2] = v2.y; ob.v[3] = v3.y;
    oa.bnd = bwl.x;
    ob.bnd = bwl.y;
    oa.key = la ? (unsigned)ba : kNoKey;
    ob.key = lb ? (unsigned)bb : kNoKey;
    oa.b = ba;
    ob.b = bb;

    // p- = p - hdt F',  g- = sqrt(1 + |p-|^2 + Phi)
    const float2 i2gt = mul2(dup2(0.5f), rgt);
    const float2 fx = fma2(gx, i2gt, ex), fy = fma2(gy, i2gt, ey), fz = fma2(gz, i2gt, ez);
    const float2 mx = fma2(nh, fx, m.px), my = fma2(nh, fy, m.py), mz = fma2(nh, fz, m.pz);
    const float2 h = mul2(mul2(dup2(hdt), bt), rsqrt2(fma2(mz, mz, fma2(my, my, fma2(mx, mx, onep)))));
    const float2 ty = mul2(h, st), ntz = mul2(h, ct);                  // t_y and -t_z
    const float2 d = fma2(ntz, ntz, fma2(ty, ty, one));
    const float2 sf = make_float2(2.f / d.x, 2.f / d.y);
    const float2 vy = mul2(sf, ty), nvz = mul2(sf, ntz);              // s_y and -s_z
    // p' = p- + p- x t ;  p+ = p- + p' x s ;  p^{n+1/2} = p+ - hdt F'
    const float2 ppx = sub2(mx, fma2(my, ntz, mul2(mz, ty)));
    const float2 ppy = fma2(mx, ntz, my);
    const float2 ppz = fma2(mx, ty, mz);
    const float2 opx = fma2(nh, fx, sub2(mx, fma2(ppy, nvz, mul2(ppz, vy))));
    const float2 opy = fma2(nh, fy, fma2(ppx, nvz, my));
    const float2 opz = fma2(nh, fz, fma2(ppx, vy, mz));
    oa.px = opx.x; oa.py = opy.x; oa.pz = opz.x;
    ob.px = opx.y; ob.py = opy.y; ob.pz = opz.y;
}

// Deposit of a warp's 64 elements (see above); v*[q] belong to group q*M/4 with bounds
// bnd[m] >= |value| over both elements.
// Value q of an element with cell base b goes to base[q][b + o[q]].
template <int M>
__device__ __forceinline__ void pair_deposit(unsigned ka, unsigned kb, const float (&va)[4], const float (&vb)[4],
                                             const float (&bnd)[M], int ba, int bb, double *const (&base)[4],
                                             const int (&o)[4]) {
    const int lane = threadIdx.x & 31;
    int ec[M];
    float sc[M];
    bool bad[M], anybad = false;
#pragma unroll
    for (int m = 0; m < M; m++) {
        const unsigned e = ((unsigned)__float_as_uint(bnd[m]) >> 23) & 0xffu;
        const int emax = (int)__reduce_max_sync(FULL, e);
        bad[m] = emax == 255;
        anybad |= bad[m];
        ec[m] = min(max(emax, 25), 254);
        sc[m] = __uint_as_float((unsigned)(277 - ec[m]) << 23);   // 2^(150 - ec)
    }
    if (anybad) {   // warp-uniform, rare: every element deposits alone, NaN in a bad group
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int m = q * M / 4;
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            const int qa = bad[m] ? 0 : __float2int_rn(va[q] * sc[m]);
            const int qb = bad[m] ? 0 : __float2int_rn(vb[q] * sc[m]);
            if (ka != kNoKey && (bad[m] || qa != 0))
                atomicAdd(base[q] + ba + o[q], bad[m] ? nan : scaled_int_to_double(qa, ec[m] + 1));
            if (kb != kNoKey && (bad[m] || qb != 0))
                atomicAdd(base[q] + bb + o[q], bad[m] ? nan : scaled_int_to_double(qb, ec[m] + 1));
        }
        return;
    }
    int qa[4], qb[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        qa[q] = __float2int_rn(va[q] * sc[q * M / 4]);
        qb[q] = __float2int_rn(vb[q] * sc[q * M / 4]);
    }
    const bool fold = ka == kb;              // a joins b (also when both are holes)
#pragma unroll
    for (int q = 0; q < 4; q++) qb[q] += fold ? qa[q] : 0;
    const unsigned kprev = __shfl_up_sync(FULL, kb, 1);
    const bool has_prev = lane > 0;
    const bool cont = has_prev && fold && kb == kprev;              // b continues the previous chain
    const bool a_joins = has_prev && !fold && ka == kprev;          // a closes the previous chain
    const unsigned absorb = __ballot_sync(FULL, cont || a_joins);
    const unsigned starts = __ballot_sync(FULL, !cont);
    const unsigned le = 0xffffffffu >> (31u - (unsigned)lane);
    const int head = 31 - __clz(starts & le);                      // first lane of this chain
    const int span = (int)__reduce_max_sync(FULL, (unsigned)(lane - head + 1));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (d >= span) break;
        const bool in = lane - d >= head;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int t = __shfl_up_sync(FULL, qb[q], d);
            if (in) qb[q] += t;
        }
    }
    // the previous lane's chain sum, for an a that closes it
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int t = __shfl_up_sync(FULL, qb[q], 1);
        if (a_joins) qa[q] += t;
    }
    const bool dep_a = !fold && ka != kNoKey;
    const bool dep_b = kb != kNoKey && (lane == 31 || !((absorb >> (lane + 1)) & 1u));
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int m = q * M / 4;
        if (dep_a && qa[q] != 0) atomicAdd(base[q] + ba + o[q], scaled_int_to_double(qa[q], ec[m] + 1));
        if (dep_b && qb[q] != 0) atomicAdd(base[q] + bb + o[q], scaled_int_to_double(qb[q], ec[m] + 1));
    }
}

// chi deposit of a warp's 64 elements through warp-private node buckets in shared memory:
// seg0[r] sums the values of node k0 + r, seg1[r] those of node k0 + P + r (k0 the warp's
// lowest cell key; an element of cell k0 + r adds w00 to seg0[r], w01 to seg0[r+1], w10 to
// seg1[r], w11 to seg1[r+1]), so that a node shared by neighbouring cells takes one
// reduction.  Sorted keys are consecutive within a column and jump by P - Nr + 1 between
// columns, so a warp's elements (about 4 cells) fit in the 31 cells from k0.  Values are
// scaled as in pair_deposit (one scale per warp, 64 values: exact in 32-bit integers); each
// element adds its four integers with shared-memory atomics, then lane r turns seg0[r] and
// seg1[r] into FP64 exactly, adds them to their nodes and zeroes them.  Elements outside the
// 31 cells (far from their sorted place) add their values alone; a non-finite value in the
// warp makes its deposits NaN.
__device__ __forceinline__ void node_bucket_deposit(int *seg, unsigned ka, unsigned kb, const float (&va)[4],
                                                    const float (&vb)[4], float bnd, int ba, int bb, double *chi,
                                                    int P) {
    const int lane = threadIdx.x & 31;
    const unsigned e = ((unsigned)__float_as_uint(bnd) >> 23) & 0xffu;
    const int emax = (int)__reduce_max_sync(FULL, e);
    const int ec = min(max(emax, 25), 254);
    const float sc = __uint_as_float((unsigned)(277 - ec) << 23);   // 2^(150 - ec)
    const int o[4] = {0, P, 1, P + 1};
    if (emax == 255) {   // warp-uniform, rare: every element deposits NaN
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (ka != kNoKey) atomicAdd(chi + ba + o[q], nan);
            if (kb != kNoKey) atomicAdd(chi + bb + o[q], nan);
        }
        return;
    }
    int qa[4], qb[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        qa[q] = __float2int_rn(va[q] * sc);
        qb[q] = __float2int_rn(vb[q] * sc);
    }
    if (ka == kb) {   // a joins b (also when both are holes)
#pragma unroll
        for (int q = 0; q < 4; q++) qb[q] += qa[q];
        ka = kNoKey;
    }
    const unsigned k0 = __reduce_min_sync(FULL, min(ka, kb));
    const bool ina = ka != kNoKey && ka - k0 < 31u;
    const bool inb = kb != kNoKey && kb - k0 < 31u;
    int *const s0 = seg, *const s1 = seg + 32;
    if (ina) {
        const int r = (int)(ka - k0);
        atomicAdd(s0 + r, qa[0]); atomicAdd(s0 + r + 1, qa[2]); atomicAdd(s1 + r, qa[1]); atomicAdd(s1 + r + 1, qa[3]);
    }
    if (inb) {
        const int r = (int)(kb - k0);
        atomicAdd(s0 + r, qb[0]); atomicAdd(s0 + r + 1, qb[2]); atomicAdd(s1 + r, qb[1]); atomicAdd(s1 + r + 1, qb[3]);
    }
    __syncwarp();
    const int v0 = s0[lane], v1 = s1[lane];
    const int n0 = (int)(k0 + (unsigned)lane);
    if (v0 != 0) {   // (scaled_int_to_double is defined for q != 0 only)
        s0[lane] = 0;
        atomicAdd(chi + n0, scaled_int_to_double(v0, ec + 1));
    }
    if (v1 != 0) {
        s1[lane] = 0;
        atomicAdd(chi + n0 + P, scaled_int_to_double(v1, ec + 1));
    }
    __syncwarp();
    const bool oa = ka != kNoKey && !ina, ob = kb != kNoKey && !inb;
    if (__any_sync(FULL, oa || ob)) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (oa && qa[q] != 0) atomicAdd(chi + ba + o[q], scaled_int_to_double(qa[q], ec + 1));
            if (ob && qb[q] != 0) atomicAdd(chi + bb + o[q], scaled_int_to_double(qb[q], ec + 1));
        }
    }
}

// Slots [begin, end) of pass A (begin even).
__device__ __forceinline__ void pass_a_range(const SimDev<float> &S, const Parts<float> &P, const Geo &geo, int off,
                                             long long shift, int *seg, int begin, int end) {
    int k = begin + 2 * threadIdx.x;
    PPos cur = load_pos(P, k, end);
    for (int base = begin; base < end; base += 2 * TPB, k += 2 * TPB) {
        const PMom m = load_mom(P, k, end);
        const PPos nxt = load_pos(P, k + 2 * TPB, end);   // prefetch
        const bool la = cur.ix.x != kDead, lb = cur.ix.y != kDead;
        AOut<float> a, b;
        a_pair(S, geo, off, shift, cur, m, a, b);
        // the pair's new momenta as 8-byte stores (measured 5 % faster than storing each
        // particle's as soon as it is pushed)
        if (la && lb) {
            __stcs(reinterpret_cast<float2 *>(P.px + k), make_float2(a.px, b.px));
            __stcs(reinterpret_cast<float2 *>(P.py + k), make_float2(a.py, b.py));
            __stcs(reinterpret_cast<float2 *>(P.pz + k), make_float2(a.pz, b.pz));
        } else {
            if (la) { __stcs(P.px + k, a.px); __stcs(P.py + k, a.py); __stcs(P.pz + k, a.pz); }
            if (lb) { __stcs(P.px + k + 1, b.px); __stcs(P.py + k + 1, b.py); __stcs(P.pz + k + 1, b.pz); }
        }
        node_bucket_deposit(seg, a.key, b.key, a.v, b.v, a.bnd > b.bnd ? a.bnd : b.bnd, a.b, b.b, S.f.chi, geo.P);
        cur = nxt;
    }
}

template <> __device__ __forceinline__ void pass_a_body<float>(const SimDev<float> &S, int vb, int nvb, int csize) {
    const Parts<float> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Geo geo = S.geo;
    const int off = S.d->off, np = S.d->np;
    const long long shift = S.d->shift;
    __shared__ int segs[TPB / 32][64];
    int *seg = segs[threadIdx.x >> 5];
    seg[threadIdx.x & 31] = 0;
    seg[32 + (threadIdx.x & 31)] = 0;
    __syncwarp();
    if (csize > 0) {   // a work item of a fused launch
        const int2 rg = slot_range(np, vb, nvb, csize);   // begin is even: chunks are multiples of TPB
        pass_a_range(S, P, geo, off, shift, seg, rg.x, rg.y);
        return;
    }
    constexpr int U = 2 * TPB;
    const Split sp = split_slots(np, vb, nvb, U, 15, 16);
    pass_a_range(S, P, geo, off, shift, seg, sp.sbeg, sp.send);
    for (;;) {
        const int u = next_unit(&S.d->ticket, sp.dyn0);
        if (u >= sp.nunits) break;
        pass_a_range(S, P, geo, off, shift, seg, u * U, min(u * U + U, np));
    }
}

template <class R> __global__ void __launch_bounds__(TPB, sizeof(R) == 4 ? 4 : 3) k_pass_a(SimDev<R> S) {
    pass_a_body<R>(S, blockIdx.x, gridDim.x, 0);
}

// Linear shape of a particle in cell i0 with fraction f, on the nodes base, base+1, base+2
// (i0 is base or base+1); written with selects so the arrays stay in registers.
template <class R> __device__ __forceinline__ void shape3(int i0, R f, int base, R *s) {
    const bool lo = i0 == base;
    s[0] = lo ? (R)1 - f : (R)0;
    s[1] = lo ? f : (R)1 - f;
    s[2] = lo ? (R)0 : f;
}

// Cell-crossing particles of one warp, parked until the warp can process 32 of them at once.
constexpr int QW = 96;                 // entries per warp: drained at 32 once per iteration, in
                                       // which at most 64 join (two particles per lane)
constexpr int NWARP = TPB_B / 32;
template <class R> struct CrossQueue {
    int ia[NWARP][QW], ja[NWARP][QW], di[NWARP][QW], dj[NWARP][QW];
    R fa[NWARP][QW], fb[NWARP][QW], fra[NWARP][QW], frb[NWARP][QW], w[NWARP][QW];
};

// General charge-conserving deposit (3x3 window) of one crossing move.
template <class R>
__device__ __forceinline__ void deposit_general(const SimDev<R> &S, int off, int ia, int ib,
                                                R fa, R fb, int ja, int jb, R fra, R frb, R w) {
    const Geo &geo = S.geo;
    const int imin = min(ia, ib), jmin = min(ja, jb);
    R s0x[3], s1x[3], s0r[3], s1r[3], dsx[3], dsr[3];
    shape3<R>(ia, fa, imin, s0x);
    shape3<R>(ib, fb, imin, s1x);
    shape3<R>(ja, fra, jmin, s0r);
    shape3<R>(jb, frb, jmin, s1r);
#pragma unroll
    for (int cc = 0; cc < 3; cc++) { dsx[cc] = s1x[cc] - s0x[cc]; dsr[cc] = s1r[cc] - s0r[cc]; }
    const int bb = geo.at(off, imin, jmin);
#pragma unroll
    for (int l = 0; l < 3; l++) {
        R acc = (R)0;
#pragma unroll
        for (int cc = 0; cc < 2; cc++) {
            acc += dsx[cc] * (s0r[l] + (R)0.5 * dsr[l]);
            atom_add(S.f.jx + bb + cc * geo.P + l, w * acc);
        }
    }
#pragma unroll
    for (int cc = 0; cc < 3; cc++) {
        R acc = (R)0;
#pragma unroll
        for (int l = 0; l < 2; l++) {
            acc += dsr[l] * (s0x[cc] + (R)0.5 * dsx[cc]);
            atom_add(S.f.jr + bb + cc * geo.P + l, w * acc);
        }
    }
}

// Process this warp's queued moves [0, n) (n is warp-uniform), one per lane at a time.
template <class R>
__device__ __forceinline__ void drain_queue(const SimDev<R> &S, int off, CrossQueue<R> &Q, int wq, int n) {
    __syncwarp();
    for (int t = threadIdx.x & 31; t < n; t += 32)
        deposit_general<R>(S, off, Q.ia[wq][t], Q.ia[wq][t] + Q.di[wq][t], Q.fa[wq][t], Q.fb[wq][t],
                           Q.ja[wq][t], Q.ja[wq][t] + Q.dj[wq][t], Q.fra[wq][t], Q.frb[wq][t], Q.w[wq][t]);
    __syncwarp();
}

// Pass B: Phi^{n+1/2} at x^n, gbar = sqrt(1+|p|^2+Phi^{n+1/2}), x^{n+1} = x^n + dt p/gbar;
// charge-conserving current in the (x, r) index plane (Esirkepov decomposition):
//   Wx = DSx (S0r + DSr/2), Wr = DSr (S0x + DSx/2),
//   Jx(i+1/2,j) = (-q w/dt) sum_{k<=i} Wx(k,j) / (V_j/dx),
//   Jr(i,j+1/2) = (-q w/dt) sum_{l<=j} Wr(i,l) / (2 pi r_{j+1/2} dx);
// the deposit is the charge -q w sum Wx (sum Wr) through each face, and Ampere applies the
// per-row factors 1/(dt V_j/dx) and 1/(dt 2 pi r_{j+1/2} dx).
// A particle that stays in its cell has only four non-zero terms,
//   Jx(i+1/2, j)   ~ -w dx_ (1 - rbar),  Jx(i+1/2, j+1) ~ -w dx_ rbar,
//   Jr(i, j+1/2)   ~ -w dr_ (1 - xbar),  Jr(i+1, j+1/2) ~ -w dr_ xbar,
// (dx_, dr_ the in-cell displacements, xbar, rbar the mean fractions); those are summed over
// the run of lanes sharing the cell before the atomics.  Cell-crossing particles (a few per
// cent) are queued per warp in shared memory and take the 3x3 general form 32 at a time, so
// that their slow path runs on full warps.  Particles leaving the next step's window (x < 0,
// x >= Nx dx) or reaching r >= r_max are marked dead after their deposit.
// Results of pass B for one particle.
template <class R> struct BOut {
    unsigned key;              // b for a particle that stays in its cell, else kNoKey
    int b;                     // its cell base (window-relative node index)
    R v[4], bnd[2];            // charge through the faces of Jx(i+1/2, j), Jx(i+1/2, j+1),
                               // Jr(i, j+1/2), Jr(i+1, j+1/2)
    bool cross;                // alive and leaving its cell: the general deposit
    int ia, ja, di, dj;        // the move, in cells
    R fa, fb, fra, frb;        // in-cell fractions before and after
    int ixn;                   // new lab cell (kDead when the particle leaves)
    R ox1, y1, z1;
    bool nonfinite;            // alive with a non-finite new position (latched as ERR_NONFINITE)
};

template <class R>
__device__ __forceinline__ BOut<R> b_particle(const SimDev<R> &S, const Geo &geo, int off, long long shift,
                                              int snext, int ix, R ox, R y, R z, R px, R py, R pz, R w) {
    const R dt = S.k.dt, idr = S.k.idr, dtdx = S.k.dtdx;
    const R rmax = S.k.rmax;
    const bool alive = ix != kDead;
    const int irel = (int)((long long)ix - shift);
    const R r0 = sqrt_<R>(y * y + z * z);
    const R rn0 = r0 * idr;
    const Loc<R> L = locate<R>(irel, ox, rn0, geo.nx, geo.nr);
    const R ph = gather4<R>(S.f.phih, geo, off, L.ip, L.fp, L.jp, L.gp, false);
    const R ig = rsqrt_<R>((R)1 + px * px + py * py + pz * pz + ph);   // 1/gbar
    // The current is a difference of shape factors at two nearby positions: move x as
    // an in-cell offset, and take the new radius as r^n plus the radial step in the
    // cancellation-free form (dy (y0+y1) + dz (z0+z1)) / (r0 + r1).
    R ox1 = ox + dtdx * px * ig;
    const R dy = dt * py * ig, dz = dt * pz * ig;
    const R y1 = y + dy, z1 = z + dz;
    // a particle moves less than one cell per step (dt < dx, dt < dr); the clamps only
    // keep the 3-node shape window in range for non-finite input
    int di = min(max(floor_int<R>(ox1), -1), 1);
    ox1 -= (R)di;
    if (ox1 >= (R)1) { ox1 -= (R)1; di = min(di + 1, 1); }
    const int ia = L.ip;
    const R r1 = sqrt_<R>(y1 * y1 + z1 * z1);
    const R rsum = r0 + r1;
    const R step_r = rsum > (R)0 ? (dy * (y + y1) + dz * (z + z1)) / rsum : (R)0;
    R rn1 = rn0 + step_r * idr;
    rn1 = rn1 < (R)0 ? (R)0 : rn1;
    const int ja = L.jp, jb = min(max((int)rn1, ja - 1), ja + 1);
    const R fra = L.gp, frb = rn1 - (R)jb;
    const bool stays = di == 0 && ja == jb;

    BOut<R> o;
    const R ddx = ox1 - ox, ddr = frb - fra;
    const R xbar = (R)0.5 * (ox + ox1), rbar = (R)0.5 * (fra + frb);
    const bool fast = alive && stays;
    const R bx = fast ? w * ddx : (R)0, br = fast ? w * ddr : (R)0;
    // the charge moved through the two x faces and the r face (Ampere applies the row factors
    // 1/(dt A_j) and 1/(dt 2 pi r_{j+1/2} dx))
    const R cx = -bx, cr = -br;
    o.v[0] = cx * ((R)1 - rbar);
    o.v[1] = cx * rbar;
    o.v[2] = cr * ((R)1 - xbar);
    o.v[3] = cr * xbar;
    o.bnd[0] = fabs_<R>(bx);
    o.bnd[1] = fabs_<R>(br);
    o.b = geo.at(off, ia, ja);
    o.key = fast ? (unsigned)o.b : kNoKey;
    o.cross = alive && !stays;
    o.ia = ia; o.ja = ja; o.di = di; o.dj = jb - ja;
    o.fa = ox; o.fb = ox1; o.fra = fra; o.frb = frb;
    const int irel_next = ia + di - snext;
    const bool dead = irel_next < 0 || irel_next >= geo.nx || r1 >= rmax;
    o.ixn = dead ? kDead : ix + di;
    o.ox1 = ox1; o.y1 = y1; o.z1 = z1;
    o.nonfinite = alive && !(fabs_<R>(ox1 + y1 + z1) <= (R)3.0e38);   // NaN or infinity
    return o;
}

// A non-finite pushed position (from a non-finite momentum or field) is latched in the
// descriptor, one atomic per warp that saw one; lpic_step reports it as LPIC_ENONFINITE.
__device__ __forceinline__ void latch_nonfinite(Desc *d, bool bad) {
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(&d->err, (int)ERR_NONFINITE);
}

// Park this warp's crossing moves in the queue (queued: same value on every lane).
template <class R>
__device__ __forceinline__ void enqueue_cross(CrossQueue<R> &Q, int wq, int &queued, const BOut<R> &o, R w) {
    const int lane = threadIdx.x & 31;
    const unsigned cm = __ballot_sync(FULL, o.cross);
    if (o.cross) {
        const int slot = queued + __popc(cm & ((1u << lane) - 1u));
        Q.ia[wq][slot] = o.ia; Q.ja[wq][slot] = o.ja; Q.di[wq][slot] = o.di; Q.dj[wq][slot] = o.dj;
        Q.fa[wq][slot] = o.fa; Q.fb[wq][slot] = o.fb; Q.fra[wq][slot] = o.fra; Q.frb[wq][slot] = o.frb;
        Q.w[wq][slot] = w;
    }
    queued += __popc(cm);
}

// Diagnostic only (a separate instantiation): charge change q w (S1 - S0), general form.
template <class R>
__device__ __forceinline__ void charge_change(const SimDev<R> &S, const Geo &geo, int off, const BOut<R> &o, R w) {
    const int ib = o.ia + o.di, jb = o.ja + o.dj, imin = min(o.ia, ib), jmin = min(o.ja, jb);
    R s0x[3], s1x[3], s0r[3], s1r[3];
    shape3<R>(o.ia, o.fa, imin, s0x);
    shape3<R>(ib, o.fb, imin, s1x);
    shape3<R>(o.ja, o.fra, jmin, s0r);
    shape3<R>(jb, o.frb, jmin, s1r);
    const int bb = geo.at(off, imin, jmin);
#pragma unroll
    for (int cc = 0; cc < 3; cc++)
#pragma unroll
        for (int l = 0; l < 3; l++)
            atom_add(S.f.dq + bb + cc * geo.P + l, -(double)w * (double)(s1x[cc] * s1r[l] - s0x[cc] * s0r[l]));
}

template <class R, bool DQ> __device__ __forceinline__ void pass_b_body(const SimDev<R> &S, int vb, int nvb, int csize) {
    __shared__ CrossQueue<R> Q;
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Geo geo = S.geo;
    const int off = S.d->off, np = S.d->np;
    const long long shift = S.d->shift, step = S.d->step;
    const int snext = window_shifts(S.ph, step, shift) ? 1 : 0;
    const int wq = threadIdx.x >> 5;
    int queued = 0;   // same value on every lane of the warp
    // each block walks contiguous runs of slots (see pass A)
    auto range = [&](int begin, int end) {
        int k = begin + threadIdx.x;
        PReg<R> cur = load_particle<R>(P, k, end);
        for (int base = begin; base < end; base += TPB_B, k += TPB_B) {
            const PReg<R> nxt = load_particle<R>(P, k + TPB_B, end);   // prefetch
            const BOut<R> o = b_particle<R>(S, geo, off, shift, snext, cur.ix, cur.ox, cur.y, cur.z, cur.px,
                                            cur.py, cur.pz, cur.w);
            enqueue_cross<R>(Q, wq, queued, o, cur.w);
            latch_nonfinite(S.d, o.nonfinite);
            const bool alive = cur.ix != kDead;
            if (DQ && alive) charge_change<R>(S, geo, off, o, cur.w);
            if (alive) {
                P.ix[k] = o.ixn;
                P.ox[k] = o.ox1;
                P.y[k] = o.y1;
                P.z[k] = o.z1;
            }
            const Run run = run_of(o.key);
            double *const addr[4] = {S.f.jx + o.b, S.f.jx + o.b + 1, S.f.jr + o.b, S.f.jr + o.b + geo.P};
            run_deposit<2>(run, o.key, o.v, o.bnd, addr);
            // at most 32 join per iteration, so draining at 32 keeps the queue within QW
            if (queued >= 32) {
                drain_queue<R>(S, off, Q, wq, queued);
                queued = 0;
            }
            cur = nxt;
        }
    };
    if (csize > 0) {   // a work item of a fused launch
        const int2 rg = slot_range(np, vb, nvb, csize);
        range(rg.x, rg.y);
    } else {
        const Split sp = split_slots(np, vb, nvb, TPB_B, 7, 8);   // the work split of the FP32 passes
        range(sp.sbeg, sp.send);
        for (;;) {
            const int u = next_unit(&S.d->ticket, sp.dyn0);
            if (u >= sp.nunits) break;
            range(u * TPB_B, min(u * TPB_B + TPB_B, np));
        }
    }
    drain_queue<R>(S, off, Q, wq, queued);
}

// Pass B for the two particles of a lane: b_particle's arithmetic (the Phi gather per
// particle, the rest in pairs).  The deposit values come out with their signs folded:
// -w dx_ = w (ox - ox1) and -w dr_ = w (fra - frb).
__device__ __forceinline__ void b_pair(const SimDev<float> &S, const Geo &geo, int off, long long shift, int snext,
                                       const PPos &c, const PMom &m, BOut<float> &oa, BOut<float> &ob) {
    const float rmax = S.k.rmax;
    const bool la = c.ix.x != kDead, lb = c.ix.y != kDead;
    const float2 one = dup2(1.f);
    const float2 q0 = fma2(c.y, c.y, mul2(c.z, c.z));
    const float2 r0 = make_float2(sqrtf(q0.x), sqrtf(q0.y));
    const float2 rn0 = mul2(r0, dup2(S.k.idr));
    const Loc2 L = locate2((int)((long long)c.ix.x - shift), (int)((long long)c.ix.y - shift), c.ox, rn0,
                           geo.nx, geo.nr);
    float2 ph;
    ph.x = gather4<float>(S.f.phih, geo, off, L.ipa, L.fp.x, L.jpa, L.gp.x, false);
    ph.y = gather4<float>(S.f.phih, geo, off, L.ipb, L.fp.y, L.jpb, L.gp.y, false);
    const float2 ig = rsqrt2(fma2(m.pz, m.pz, fma2(m.py, m.py, fma2(m.px, m.px, add2(one, ph)))));   // 1/gbar
    // x moves as an in-cell offset; r^{n+1} = r^n + (dy (y0+y1) + dz (z0+z1)) / (r0 + r1)
    float2 ox1 = fma2(mul2(dup2(S.k.dtdx), m.px), ig, c.ox);
    const float2 dtv = dup2(S.k.dt);
    const float2 dy = mul2(mul2(dtv, m.py), ig), dz = mul2(mul2(dtv, m.pz), ig);
    const float2 y1 = add2(c.y, dy), z1 = add2(c.z, dz);
    int dia = min(max(floor_int<float>(ox1.x), -1), 1), dib = min(max(floor_int<float>(ox1.y), -1), 1);
    ox1 = sub2(ox1, make_float2((float)dia, (float)dib));
    if (ox1.x >= 1.f) { ox1.x -= 1.f; dia = min(dia + 1, 1); }
    if (ox1.y >= 1.f) { ox1.y -= 1.f; dib = min(dib + 1, 1); }
    const float2 q1 = fma2(y1, y1, mul2(z1, z1));
    const float2 r1 = make_float2(sqrtf(q1.x), sqrtf(q1.y));
    const float2 rsum = add2(r0, r1);
    const float2 num = fma2(dy, add2(c.y, y1), mul2(dz, add2(c.z, z1)));
    const float2 step_r = make_float2(rsum.x > 0.f ? num.x / rsum.x : 0.f, rsum.y > 0.f ? num.y / rsum.y : 0.f);
    float2 rn1 = fma2(step_r, dup2(S.k.idr), rn0);
    rn1.x = rn1.x < 0.f ? 0.f : rn1.x;
    rn1.y = rn1.y < 0.f ? 0.f : rn1.y;
    const int jba = min(max((int)rn1.x, L.jpa - 1), L.jpa + 1), jbb = min(max((int)rn1.y, L.jpb - 1), L.jpb + 1);
    const float2 frb = sub2(rn1, make_float2((float)jba, (float)jbb));
    const bool sta = dia == 0 && L.jpa == jba, stb = dib == 0 && L.jpb == jbb;
    const bool fa = la && sta, fb = lb && stb;
    const float2 half = dup2(0.5f);
    const float2 xbar = mul2(half, add2(c.ox, ox1)), rbar = mul2(half, add2(L.gp, frb));
    float2 cx = mul2(m.w, sub2(c.ox, ox1)), cr = mul2(m.w, sub2(L.gp, frb));
    cx = make_float2(fa ? cx.x : 0.f, fb ? cx.y : 0.f);
    cr = make_float2(fa ? cr.x : 0.f, fb ? cr.y : 0.f);
    const float2 v0 = mul2(cx, sub2(one, rbar)), v1 = mul2(cx, rbar);
    const float2 v2 = mul2(cr, sub2(one, xbar)), v3 = mul2(cr, xbar);
    oa.v[0] = v0.x; oa.v[1] = v1.x; oa.v[2] = v2.x; oa.v[3] = v3.x;
    ob.v[0] = v0.y; ob.v[1] = v1.y; ob.v[2] = v2.y; ob.v[3] = v3.y;
    oa.bnd[0] = fabsf(cx.x); oa.bnd[1] = fabsf(cr.x);
    ob.bnd[0] = fabsf(cx.y); ob.bnd[1] = fabsf(cr.y);
    oa.b = geo.at(off, L.ipa, L.jpa);
    ob.b = geo.at(off, L.ipb, L.jpb);
    oa.key = fa ? (unsigned)oa.b : kNoKey;
    ob.key = fb ? (unsigned)ob.b : kNoKey;
    oa.cross = la && !sta;
    ob.cross = lb && !stb;
    oa.ia = L.ipa; oa.ja = L.jpa; oa.di = dia; oa.dj = jba - L.jpa;
    ob.ia = L.ipb; ob.ja = L.jpb; ob.di = dib; ob.dj = jbb - L.jpb;
    oa.fa = c.ox.x; oa.fb = ox1.x; oa.fra = L.gp.x; oa.frb = frb.x;
    ob.fa = c.ox.y; ob.fb = ox1.y; ob.fra = L.gp.y; ob.frb = frb.y;
    const int na = L.ipa + dia - snext, nb = L.ipb + dib - snext;
    oa.ixn = (na < 0 || na >= geo.nx || r1.x >= rmax) ? kDead : c.ix.x + dia;
    ob.ixn = (nb < 0 || nb >= geo.nx || r1.y >= rmax) ? kDead : c.ix.y + dib;
    oa.ox1 = ox1.x; oa.y1 = y1.x; oa.z1 = z1.x;
    ob.ox1 = ox1.y; ob.y1 = y1.y; ob.z1 = z1.y;
    const float2 sum = add2(add2(ox1, y1), z1);
    oa.nonfinite = la && !(fabsf(sum.x) <= 3.0e38f);   // NaN or infinity
    ob.nonfinite = lb && !(fabsf(sum.y) <= 3.0e38f);
}

// FP32: two neighbouring particles per thread, as in pass A, pushed together in packed FP32x2
// arithmetic (b_pair; 6 % faster than one particle after the other); the crossing moves of both
// join the queue, which is drained at one place per iteration (one inlined copy of the general
// deposit, not two).  Unlike pass A, the momenta are carried one iteration ahead too: they fit
// in 64 registers here (8 blocks of 128 per SM instead of 9 at 56 registers; 1.7 % faster).
// This function: slots [begin, end) (begin even); queued: the warp's crossing queue fill.
__device__ __forceinline__ void pass_b_range(const SimDev<float> &S, const Parts<float> &P, const Geo &geo, int off,
                                             long long shift, int snext, CrossQueue<float> &Q, int wq, int &queued,
                                             int begin, int end) {
    int k = begin + 2 * threadIdx.x;
    PPos cur = load_pos(P, k, end);
    PMom mcur = load_mom(P, k, end);
    for (int base = begin; base < end; base += 2 * TPB_B, k += 2 * TPB_B) {
        const PMom m = mcur;
        const PPos nxt = load_pos(P, k + 2 * TPB_B, end);   // prefetch
        mcur = load_mom(P, k + 2 * TPB_B, end);
        BOut<float> a, b;
        b_pair(S, geo, off, shift, snext, cur, m, a, b);
        enqueue_cross<float>(Q, wq, queued, a, m.w.x);
        enqueue_cross<float>(Q, wq, queued, b, m.w.y);
        latch_nonfinite(S.d, a.nonfinite || b.nonfinite);
        const bool la = cur.ix.x != kDead, lb = cur.ix.y != kDead;
        if (la && lb) {
            __stcs(reinterpret_cast<int2 *>(P.ix + k), make_int2(a.ixn, b.ixn));
            __stcs(reinterpret_cast<float2 *>(P.ox + k), make_float2(a.ox1, b.ox1));
            __stcs(reinterpret_cast<float2 *>(P.y + k), make_float2(a.y1, b.y1));
            __stcs(reinterpret_cast<float2 *>(P.z + k), make_float2(a.z1, b.z1));
        } else {
            if (la) { P.ix[k] = a.ixn; P.ox[k] = a.ox1; P.y[k] = a.y1; P.z[k] = a.z1; }
            if (lb) { P.ix[k + 1] = b.ixn; P.ox[k + 1] = b.ox1; P.y[k + 1] = b.y1; P.z[k + 1] = b.z1; }
        }
        const float bnd[2] = {a.bnd[0] > b.bnd[0] ? a.bnd[0] : b.bnd[0], a.bnd[1] > b.bnd[1] ? a.bnd[1] : b.bnd[1]};
        double *const base_q[4] = {S.f.jx, S.f.jx, S.f.jr, S.f.jr};
        const int o[4] = {0, 1, 0, geo.P};
        pair_deposit<2>(a.key, b.key, a.v, b.v, bnd, a.b, b.b, base_q, o);
        if (queued >= 32) {
            drain_queue<float>(S, off, Q, wq, queued);
            queued = 0;
        }
        cur = nxt;
    }
}

template <>
__device__ __forceinline__ void pass_b_body<float, false>(const SimDev<float> &S, int vb, int nvb, int csize) {
    __shared__ CrossQueue<float> Q;
    const Parts<float> P = S.d->pbuf ? S.p[1] : S.p[0];
    const Geo geo = S.geo;
    const int off = S.d->off, np = S.d->np;
    const long long shift = S.d->shift, step = S.d->step;
    const int snext = window_shifts(S.ph, step, shift) ? 1 : 0;
    const int wq = threadIdx.x >> 5;
    int queued = 0;   // same value on every lane of the warp
    if (csize > 0) {   // a work item of a fused launch
        const int2 rg = slot_range(np, vb, nvb, csize);   // begin is even: chunks are multiples of 2 * TPB_B
        pass_b_range(S, P, geo, off, shift, snext, Q, wq, queued, rg.x, rg.y);
    } else {
        constexpr int U = 2 * TPB_B;
        const Split sp = split_slots(np, vb, nvb, U, 7, 8);
        pass_b_range(S, P, geo, off, shift, snext, Q, wq, queued, sp.sbeg, sp.send);
        for (;;) {
            const int u = next_unit(&S.d->ticket, sp.dyn0);
            if (u >= sp.nunits) break;
            pass_b_range(S, P, geo, off, shift, snext, Q, wq, queued, u * U, min(u * U + U, np));
        }
    }
    drain_queue<float>(S, off, Q, wq, queued);
}

template <class R, bool DQ>
__global__ void __launch_bounds__(TPB_B, sizeof(R) == 4 ? 8 : 6) k_pass_b(SimDev<R> S) {
    pass_b_body<R, DQ>(S, blockIdx.x, gridDim.x, 0);
}

// Fused forms over a batch: blocks take work items {simulation, item, 0, slots per item} in
// turn from a ticket counter (zeroed before the launch), so that the blocks that drew cheap
// items take more of them and the launch ends with little tail.
__device__ __forceinline__ int next_item(int *ticket) {
    __shared__ int w;
    __syncthreads();   // every thread has read the previous ticket
    if (threadIdx.x == 0) w = atomicAdd(ticket, 1);
    __syncthreads();
    return w;
}
template <class R>
__global__ void __launch_bounds__(TPB, sizeof(R) == 4 ? 4 : 3) k_pass_a_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n, int *ticket) {
    for (int w = next_item(ticket); w < n; w = next_item(ticket)) {
        const int4 it = items[w];
        pass_a_body<R>(pk.v[it.x], it.y, it.z, it.w);
    }
}
template <class R, bool DQ>
__global__ void __launch_bounds__(TPB_B, sizeof(R) == 4 ? 8 : 6) k_pass_b_multi(const __grid_constant__ SimPack<R> pk, const int4 *items, int n, int *ticket) {
    for (int w = next_item(ticket); w < n; w = next_item(ticket)) {
        const int4 it = items[w];
        pass_b_body<R, DQ>(pk.v[it.x], it.y, it.z, it.w);
    }
}

template <class R>
__global__ void k_load_columns(SimDev<R> S, const int *__restrict__ colbase, int ncols, int total) {
    const long long s = S.d->shift;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int lo = 0, hi = ncols;  // colbase[lo] <= t < colbase[hi]
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (colbase[mid] <= t) lo = mid; else hi = mid;
        }
        ColumnPlan<R> cp;
        column_plan<R>(S.ph, s + lo, cp);
        if (t - colbase[lo] < column_particles<R>(S.ph, cp, S.geo.nr)) lattice_emit<R>(S, cp, s + lo, t - colbase[lo], t);
    }
}

inline int pgrid(int n) {
    int b = (n + TPB - 1) / TPB;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

// Blocks of a particle kernel that are resident on the whole device at once (the kernels
// loop over particle groups, so one resident wave is enough); cached per kernel address
// (kernels of one signature share a function type, so the address is the key).
template <class K> int resident_blocks(K *kernel, int threads = TPB) {
    static std::mutex lock;
    static const void *keys[8] = {};
    static int vals[8] = {};
    std::lock_guard<std::mutex> g(lock);
    for (int q = 0; q < 8; q++)
        if (keys[q] == (const void *)kernel) return vals[q];
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    const int v = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
    for (int q = 0; q < 8; q++)
        if (!keys[q]) { keys[q] = (const void *)kernel; vals[q] = v; break; }
    return v;
}

inline int particle_grid(int np_upper, int resident, int threads = TPB) {
    const int need = (np_upper + threads - 1) / threads;
    return need < 1 ? 1 : (need < resident ? need : resident);
}

}  // namespace

template <class R> void launch_pass_a(const SimDev<R> &S, int np_upper, cudaStream_t st) {
    k_pass_a<R><<<particle_grid(np_upper, resident_blocks(k_pass_a<R>)), TPB, 0, st>>>(S);
}
template <class R> void launch_pass_b(const SimDev<R> &S, int np_upper, cudaStream_t st) {
    if (S.ph.track_dq)
        k_pass_b<R, true><<<particle_grid(np_upper, resident_blocks(k_pass_b<R, true>, TPB_B), TPB_B), TPB_B, 0, st>>>(S);
    else
        k_pass_b<R, false><<<particle_grid(np_upper, resident_blocks(k_pass_b<R, false>, TPB_B), TPB_B), TPB_B, 0, st>>>(S);
}
template <class R> void launch_load_columns(const SimDev<R> &S, const int *d_colbase, int ncols,
                                            int total, cudaStream_t st) {
    if (total > 0) k_load_columns<R><<<pgrid(total), TPB, 0, st>>>(S, d_colbase, ncols, total);
}

template <class R>
void launch_particles_multi(int phase, bool dq, const SimPack<R> &pk, const int4 *items, int n,
                            int *ticket, cudaStream_t st) {
    if (n <= 0) return;
    int g;
    if (phase == 0) {
        g = resident_blocks(k_pass_a_multi<R>);
        k_pass_a_multi<R><<<n < g ? n : g, TPB, 0, st>>>(pk, items, n, ticket);
    } else if (dq) {
        g = resident_blocks(k_pass_b_multi<R, true>, TPB_B);
        k_pass_b_multi<R, true><<<n < g ? n : g, TPB_B, 0, st>>>(pk, items, n, ticket);
    } else {
        g = resident_blocks(k_pass_b_multi<R, false>, TPB_B);
        k_pass_b_multi<R, false><<<n < g ? n : g, TPB_B, 0, st>>>(pk, items, n, ticket);
    }
}

#define INST(R)                                                                             \
    template void launch_particles_multi<R>(int, bool, const SimPack<R> &, const int4 *, int, \
                                            int *, cudaStream_t);                           \
    template void launch_pass_a<R>(const SimDev<R> &, int, cudaStream_t);                   \
    template void launch_pass_b<R>(const SimDev<R> &, int, cudaStream_t);                   \
    template void launch_load_columns<R>(const SimDev<R> &, const int *, int, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace lpic
