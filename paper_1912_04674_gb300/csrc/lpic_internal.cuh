// Internal declarations of the lpic CUDA library (not part of the C ABI).
//
// Device data layout (one caller-owned buffer, sub-allocated by api.cu):
//   * grid arrays: column-major in x ("r fastest"), column stride P >= nr+3 elements,
//     kG guard columns on both sides of the live window, and a sliding physical column
//     offset `off` so that a moving-window shift is a pointer slide plus the zeroing of
//     the guard columns, not a copy of the grid (api.cu relocates the live region when
//     the slide reaches the end of the allocation);
//   * particles: structure of arrays, x kept as an int32 lab-frame cell index plus an
//     in-cell offset in [0,1) of the working precision R, so the window shift never
//     touches particles and FP32 keeps full resolution far from the origin.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lpic {

constexpr int kG = 2;                    // guard columns on each side of the live window
constexpr int32_t kDead = INT32_MIN;     // ix of a removed particle (a hole until compaction)
constexpr double kPi = 3.14159265358979323846;

enum ErrBits : int { ERR_CAPACITY = 1, ERR_NONFINITE = 2 };

// Device-resident per-simulation counters, read by every kernel so that a captured CUDA
// graph replays correctly step after step.
struct Desc {
    long long step;    // n
    long long shift;   // s: lab x of window column 0 is s*dx
    int off;           // sliding physical column offset of the grid arrays
    int np;            // particle slots in use (alive + holes)
    int n_alive;       // alive count after the last compaction
    int err;           // ErrBits, sticky
    int abuf;          // index of the buffer holding A^n (the other holds A^{n-1})
    int pbuf;          // index of the particle buffer in use (the other is the sort target)
    int last_shift;    // 1 if the last step ended with a window shift (its deposits sit one
                       // physical column before the current window)
    unsigned done;     // blocks of the window kernel finished this step (last one advances)
    int off_step;      // `off` as the step began (copied by the prepass): Ampere reads it while
                       // the window step, in the same launch, may already have advanced `off`
    int nfree;         // slab exchange: slots freed by its removal (listed in the staging area)
    int ntaken;        // slab exchange: appended electrons so far (freed slots first)
    int ticket;        // units handed out by the FP32 particle passes (zeroed by the kernel before)
};
static_assert(sizeof(Desc) == 64, "Desc is one 64-byte line");

template <class R> struct Cplx;
template <> struct Cplx<double> { using t = double2; };
template <> struct Cplx<float> { using t = float2; };

struct Geo {
    int nx, nr;   // cells
    int P;        // column stride in elements
    int ncol;     // physical columns of every grid array
    int nlive;    // nx + 1 + 2*kG columns of the live window (incl. guards)
    // element index; every grid array has fewer than 2^31 elements (checked at set-up)
    __host__ __device__ __forceinline__ int at(int off, int i, int j) const {
        return (off + kG + i) * P + j;
    }
};

// Phi^n and its two centred differences at one node, loaded together by the gathers.
template <class R> struct alignas(4 * sizeof(R)) Q4 {
    R phi, gx, gr, pad;
};

template <class R> struct Fields {
    R *ex, *er, *bt;                 // persistent: E^n, B^{n-1/2} -> B^{n+1/2}
    typename Cplx<R>::t *a[2];       // persistent: A^n = a[abuf], A^{n-1} = a[abuf^1]
    R *btn, *phih;                   // per step: B^n (FP64 contexts; FP32 reads btq), Phi^{n+1/2}
    Q4<R> *pg;                       // per step: (Phi^n, dPhi/dx, dPhi/dr)
    // per step, FP32 contexts only (else null): E^n and B^n as pairs of x neighbours,
    // element (i, j) = (F(i, j), F(i+1, j)), so that a gather reads two adjacent 8-byte
    // records; the element of row -1 (the spare last row of the previous column) is
    // (-F(i, 0), -F(i+1, 0)), the odd mirror of Er and Btheta across the axis
    typename Cplx<R>::t *exq, *erq, *btq;
    double *chi, *jx, *jr, *dq;      // per step FP64 accumulators (deposit targets), before
                                     // their row factors (RowTab): chi sum w S/gamma, Jx and
                                     // Jr the charge through each face in the step
    // the current (and charge change) the fields see: the deposit targets, or, with the
    // binomial filter on, separate arrays the filter writes from them
    double *jxu, *jru, *dqu;
};

template <class R> struct Parts {
    int32_t *ix;
    R *ox, *y, *z, *px, *py, *pz, *w;
    uint64_t *id;
};

struct Phys {
    double dx, dr, dt;
    int moving_window;
    int have_plasma;
    double n0, x_start, ramp_len;
    int ppcx, ppcr, ppct;
    unsigned long long seed;
    int cap;
    int track_dq;
    int filter_passes;   // binomial current filter passes after the deposit (0: off)
    int x0;              // x-slab: global window column of column 0 (0 for a whole window)
    int inject;          // 1: the moving window injects plasma at the front column
    // host-computed reciprocals for the lattice generator
    double inv_ramp, inv_ppcx, inv_ppcr, inv_ppct, wfac;  // wfac = 2 pi dr dx / ppc
};

// Per-row tables (device, P entries each, working precision), filled once at set-up.
// The particle passes deposit per-row-free sums (chi: sum w S / gamma; Jx, Jr: the charge
// moved through each face in the step), and the grid kernels that read them apply these row
// factors (one multiply per node instead of one per particle and node).
enum RowTab : int {
    T_CHI = 0,   // 1 / V_chi(j)
    T_JX,        // (1/dt) / (V_j / dx): current from a charge flux through an x face
    T_JR,        // (1/dt) / (2 pi r_{j+1/2} dx): through an r face
    T_ENV1R,     // 1 / (2 dr r_j), j >= 1 (envelope radial term)
    T_AMPP,      // r_{j+1/2} / (r_j dr), j >= 1 (Ampere)
    T_AMPM,      // r_{j-1/2} / (r_j dr), j >= 1
    NTAB
};

// The row factors in FP64 (the host tables and the FP64 axis rows use these; dumps too).
// Volumes (G7): V_j = 2 pi j dr^2 dx (j >= 1), charge and current V_0 = pi (dr/2)^2 dx,
// susceptibility V_chi,0 = pi dr^2 dx / 3.
__host__ __device__ __forceinline__ double row_ichi(const Phys &ph, int j) {
    const double vchi = j == 0 ? kPi * ph.dr * ph.dr * ph.dx / 3.0 : 2.0 * kPi * j * ph.dr * ph.dr * ph.dx;
    return 1.0 / vchi;
}
__host__ __device__ __forceinline__ double row_ijx(const Phys &ph, int j) {
    const double vq = j == 0 ? kPi * 0.25 * ph.dr * ph.dr * ph.dx : 2.0 * kPi * j * ph.dr * ph.dr * ph.dx;
    return (1.0 / ph.dt) / (vq / ph.dx);
}
__host__ __device__ __forceinline__ double row_ijr(const Phys &ph, int j) {
    return (1.0 / ph.dt) / (2.0 * kPi * (j + 0.5) * ph.dr * ph.dx);
}

// The FP64 factors of the axis rows (envelope: 1/V_chi,0; Ampere: 1/(dt V_0/dx)) follow the
// working-precision row tables in device memory (FP64 divisions are slow on this part).
constexpr int kAxisFactors = 2;
template <class R> __device__ __forceinline__ double axis_factor(const R *tab, int P, int which) {
    return reinterpret_cast<const double *>(tab + (size_t)NTAB * P)[which];
}

// Constants of one simulation, computed on the host (FP64 is a slow pipe on this part,
// so no kernel derives them per thread).
template <class R> struct Kc {
    R dt, hdt, idx, idr, dtdx, hidx, hidr, idx2, idr2, dt2, envp, envpt;
    double d_dt, d_dt2, d_idx2, d_idr2, d_hidx, d_envp, d_envpt, d_4idr;  // FP64 axis rows
    R rmax;         // Nr dr: particles at r >= rmax leave
    R lat_ippcx, lat_ippcr, lat_ippct, lat_dr, lat_wfac;   // plasma lattice (1/ppc, dr, 2 pi dr dx / ppc)
    const R *tab;   // NTAB x P row tables
};

// Scratch of the counting sort: key per slot, ncell + 2 counters, scan block sums.
struct SortBufs {
    int *key, *count, *blocksum;
};

template <class R> struct SimDev {
    Geo geo;
    Phys ph;
    Kc<R> k;
    Desc *d;
    Fields<R> f;
    Parts<R> p[2];   // p[d->pbuf] in use; the counting sort scatters into the other
    SortBufs sb;
};

// ---- shared device helpers -------------------------------------------------------------
// Square roots, absolute values and floors in the working precision, spelled out so that FP32 code never
// takes a double-precision overload.
template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }
template <class R> __device__ __forceinline__ R sqrt_(R x);
template <> __device__ __forceinline__ float sqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double sqrt_<double>(double x) { return ::sqrt(x); }
template <class R> __device__ __forceinline__ R fabs_(R x);
template <> __device__ __forceinline__ float fabs_<float>(float x) { return fabsf(x); }
template <> __device__ __forceinline__ double fabs_<double>(double x) { return ::fabs(x); }
// FP64 accumulator -> working precision.  For FP32, round to nearest even from the IEEE-754
// fields with integer operations (the FP64 pipe, which the hardware conversion would use, is
// slow on this part); magnitudes below the FP32 normal range flush to a signed zero, like the
// FP32 kernels' arithmetic; overflow gives infinity and NaN stays NaN.
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;        // FP32 exponent field
    const unsigned mf = ((hi & 0xfffffu) << 3) | (lo >> 29);      // top 23 of 52 mantissa bits
    const unsigned rest = lo & 0x1fffffffu, half = 0x10000000u;   // the 29 dropped bits
    const unsigned up = (rest > half || (rest == half && (mf & 1u))) ? 1u : 0u;
    const unsigned fin = ((unsigned)e << 23) + mf + up;           // a carry rounds into the exponent
    const bool special = ((hi >> 20) & 0x7ffu) == 0x7ffu;
    const unsigned nan_or_inf = 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
    const unsigned bits = special ? nan_or_inf : (e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : fin));
    return __uint_as_float(sgn | bits);
}
// FP32 -> FP64 from the IEEE-754 field layouts with integer operations (the FP64 pipe is
// slow on this part): exponent rebiased by 1023 - 127 = 896, mantissa widened.  FP32
// subnormals (< 1.2e-38) become 0; infinities and NaNs stay what they are.
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x), sgn = u & 0x80000000u, m = u & 0x7fffffffu;
    const bool tiny = m < 0x00800000u, special = m >= 0x7f800000u;
    const unsigned hi_n = sgn | ((m >> 3) + (896u << 20));
    const unsigned hi_s = sgn | 0x7ff00000u | ((m & 0x007fffffu) >> 3);
    const unsigned hi = tiny ? sgn : (special ? hi_s : hi_n);
    const unsigned lo = tiny ? 0u : (m << 29);
    return __hiloint2double((int)hi, (int)lo);
}

template <class R> __device__ __forceinline__ R from_acc(double x);
template <> __device__ __forceinline__ float from_acc<float>(double x) { return d2f_bits(x); }
template <> __device__ __forceinline__ double from_acc<double>(double x) { return x; }
__device__ __forceinline__ double to_acc(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_acc(double x) { return x; }

template <class R> __device__ __forceinline__ int floor_int(R x);
template <> __device__ __forceinline__ int floor_int<float>(float x) { return __float2int_rd(x); }
template <> __device__ __forceinline__ int floor_int<double>(double x) { return __double2int_rd(x); }

__host__ __device__ __forceinline__ double plasma_density(const Phys &ph, double xlab) {
    if (xlab < ph.x_start) return 0.0;
    if (ph.ramp_len > 0.0 && xlab < ph.x_start + ph.ramp_len)
        return ph.n0 * (xlab - ph.x_start) * ph.inv_ramp;
    return ph.n0;
}

// lab x of lattice slice a of lab column c
__host__ __device__ __forceinline__ double lattice_x(const Phys &ph, long long c, int a) {
    return ((double)c + (a + 0.5) * ph.inv_ppcx) * ph.dx;
}

// k-th output of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                                  unsigned long long k) {
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Does the window shift after step n (window speed c)?  s is the context's shift counter,
// the lab cell of its column 0: the global shift count plus the slab offset x0.  Same double
// arithmetic on host and device.
__host__ __device__ __forceinline__ bool window_shifts(const Phys &ph, long long n, long long s) {
    return ph.moving_window && (double)(n + 1) * ph.dt >= (double)(s - ph.x0 + 1) * ph.dx;
}

// Plasma lattice of lab column c (regular ppc_x x ppc_r x ppc_theta per cell, weight
// n(x) 2 pi r dr dx / ppc; the densities of the Sec. 4 runs): the x slices a that carry
// plasma and their densities, computed once per column.
template <class R> struct ColumnPlan {
    int nv;
    int valid[16];
    R dens[16];
};
template <class R>
__device__ __forceinline__ void column_plan(const Phys &ph, long long c, ColumnPlan<R> &cp) {
    cp.nv = 0;
    for (int a = 0; a < ph.ppcx && a < 16; a++) {
        const double n = plasma_density(ph, lattice_x(ph, c, a));
        if (n > 0.0) {
            cp.valid[cp.nv] = a;
            cp.dens[cp.nv] = (R)n;
            cp.nv++;
        }
    }
}
template <class R> __device__ __forceinline__ int column_particles(const Phys &ph, const ColumnPlan<R> &cp, int nr) {
    return cp.nv * ph.ppcr * ph.ppct * nr;
}

// Particle `local` of column c (enumerating (j, valid slice, b, k)) into `slot`; local must be
// below column_particles.  FP64 evaluates the lattice in FP64; FP32 in FP32 (its positions are
// FP32 anyway), with the azimuthal offset u from the top 24 bits of the SplitMix64 output.
template <class R>
__device__ __forceinline__ void lattice_emit(const SimDev<R> &S, const ColumnPlan<R> &cp, long long c, int local,
                                             int slot) {
    const Phys &ph = S.ph;
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const int perj = cp.nv * ph.ppcr * ph.ppct;
    const int j = local / perj;
    int rem = local - j * perj;
    const int av = rem / (ph.ppcr * ph.ppct);
    rem -= av * ph.ppcr * ph.ppct;
    const int b = rem / ph.ppct, kk = rem - b * ph.ppct;
    const int a = cp.valid[av];
    const unsigned long long cell = (unsigned long long)c * S.geo.nr + (unsigned long long)j;
    const unsigned long long h = splitmix64(ph.seed, cell + 1);
    if (sizeof(R) == 4) {
        const float r = ((float)j + ((float)b + 0.5f) * (float)S.k.lat_ippcr) * (float)S.k.lat_dr;
        const float u = (float)(unsigned)(h >> 40) * 5.9604644775390625e-08f;   // 2^-24
        float sn, cs;
        sincospif(2.0f * ((float)kk + u) * (float)S.k.lat_ippct, &sn, &cs);
        P.ox[slot] = (R)(((float)a + 0.5f) * (float)S.k.lat_ippcx);
        P.y[slot] = (R)(r * cs);
        P.z[slot] = (R)(r * sn);
        P.w[slot] = (R)((float)cp.dens[av] * r * (float)S.k.lat_wfac);
    } else {
        const double r = (j + (b + 0.5) * ph.inv_ppcr) * ph.dr;
        const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
        double sd, cd;
        sincos(2.0 * kPi * ((kk + u) * ph.inv_ppct), &sd, &cd);
        P.ox[slot] = (R)((a + 0.5) * ph.inv_ppcx);
        P.y[slot] = (R)(r * cd);
        P.z[slot] = (R)(r * sd);
        P.w[slot] = (R)((double)cp.dens[av] * r * ph.wfac);
    }
    P.ix[slot] = (int)c;
    P.px[slot] = (R)0;
    P.py[slot] = (R)0;
    P.pz[slot] = (R)0;
    P.id[slot] = ((cell * ph.ppcx + a) * ph.ppcr + b) * ph.ppct + kk;
}

// ---- launchers (defined in the kernel translation units) --------------------------------
template <class R> void launch_prepass(const SimDev<R> &S, cudaStream_t st);
template <class R> void launch_pass_a(const SimDev<R> &S, int np_upper, cudaStream_t st);
template <class R> void launch_envelope(const SimDev<R> &S, cudaStream_t st);
template <class R> void launch_pass_b(const SimDev<R> &S, int np_upper, cudaStream_t st);
template <class R> void launch_ampere(const SimDev<R> &S, cudaStream_t st);
// Ampere and the end-of-step window (guard zeroing, injection, counters) in one launch
template <class R> void launch_ampere_window(const SimDev<R> &S, int inj_upper, cudaStream_t st);
template <class R> void launch_filter(const SimDev<R> &S, cudaStream_t st);
constexpr int kFilterMaxPasses = 16;

template <class R> void launch_init_envelope(const SimDev<R> &S, double a0, double w0, double L,
                                            double xc, double xf, cudaStream_t st);
template <class R> void launch_load_columns(const SimDev<R> &S, const int *d_colbase, int ncols,
                                            int total, cudaStream_t st);
template <class R> void launch_relocate(const SimDev<R> &S, int new_off, cudaStream_t st);

// ---- x-slab exchange (slab.cu): halo columns of the persistent arrays from the owner, then
// the electrons: remove those outside [lo, hi) (local cells) from each side and append the
// other side's electrons in its halo cells, into the slots the removal freed first (freeL,
// freeR: scratch for fcap slot indices per side).
template <class R>
void launch_slab_exchange(const SimDev<R> &L, const SimDev<R> &Rt, int B_L, int halo, int *freeL, int *freeR,
                          int fcap, cudaStream_t st);

// ---- injected bunch: its charge from particle slots [k0, k0 + n), the discrete Gauss-law solve
// (preconditioned CG to relative residual tol, at most max_iter iterations) and the addition of
// its fields to E^n, B^{n-1/2}; returns the iterations, *res the final relative residual.
size_t bunch_scratch_bytes(const Geo &g);
template <class R>
int bunch_solve_and_add(const SimDev<R> &S, int k0, int n, double gamma, void *scratch, double *d_dot, double tol,
                        int max_iter, cudaStream_t st, double *res_out);

// ---- fused batch forms: one launch per phase over work items {sim, a, b, c} -------------
// The views of the simulations of one fused launch travel by value in the kernel's
// parameter space (a __grid_constant__ pack, read through the constant cache like a single
// simulation's view, so the bodies keep the register budget of the single kernels).
// 46 views of at most 696 bytes plus the other arguments fit the 32,764-byte limit.
constexpr int kPackMax = 46;
template <class R> struct SimPack { SimDev<R> v[kPackMax]; };
static_assert(sizeof(SimPack<double>) + 2 * sizeof(void *) + 2 * sizeof(int) <= 32764 &&
                  sizeof(SimPack<float>) + 2 * sizeof(void *) + 2 * sizeof(int) <= 32764,
              "a pack of views must fit the kernel parameter space");
// grid phases 0 prepass, 1 envelope (c = axis tile), 2 ampere, 3 current filter: items
// {sim, bx, by, c}
void grid_tiles(const Geo &g, int phase, int &tx, int &ty);
template <class R>
void launch_grid_multi(int phase, const SimPack<R> &pk, const int4 *items, int n, cudaStream_t st);
// particle phases (0 pass A, 1 pass B): items {sim, item, 0, slots per item}, item covering
// slots [item * size, (item + 1) * size) clipped to the live slots; blocks draw the items
// from *ticket, which must be zero when the launch starts
template <class R>
void launch_particles_multi(int phase, bool dq, const SimPack<R> &pk, const int4 *items, int n,
                            int *ticket, cudaStream_t st);
// window: items {sim, part, parts of sim, 0}
template <class R> void launch_window_multi(const SimPack<R> &pk, const int4 *items, int n, cudaStream_t st);
// counting sort of the simulations with due[slot] != 0, seven launches: clear, count, scan
// blocks, scan top, scan add, scatter, finish.  blocks: items {sim, block of 4096 counters,
// 0, 0} (clear and scans); slots: particle items as for the passes; sims: {sim, 0, 0, 0}.
template <class R>
void launch_sort_multi(const SimPack<R> &pk, const int *due, const int4 *blocks, int nblocks,
                       const int4 *slots, int nslots, const int4 *sims, int nsims, cudaStream_t st);
constexpr int kSortLaunchesMulti = 7;
__host__ __device__ inline int sort_blocks(const Geo &g) { return (g.nx * g.nr + 1 + 4095) / 4096; }
constexpr int kWindowThreads = 64;
int window_parts(const Geo &g, int work);   // parts of one simulation's window step in the fused batch launch

// exclusive scan of n ints in place (n <= 4096 * 4096); blocksum: ceil(n/4096)+1 ints
void scan_exclusive(int *data, int n, int *blocksum, cudaStream_t st);

// counting sort by cell; `alt` receives the sorted particles; scratch ints:
// key[cap], count[ncell+1], blocksum[...]
template <class R> void launch_sort(const SimDev<R> &S, int np_upper, int *key, int *count,
                                    int *blocksum, cudaStream_t st);

// diagnostics (results in `out`, device doubles / uint64)
template <class R> void launch_diag_ex_axis(const SimDev<R> &S, double *out, cudaStream_t st);
template <class R> void launch_diag_amax_waist(const SimDev<R> &S, double *out3, cudaStream_t st);
template <class R> void launch_diag_cont(const SimDev<R> &S, double *out2, cudaStream_t st);
template <class R> void launch_beam_max(const SimDev<R> &S, int np_upper, double thr, double *out2, cudaStream_t st);
template <class R> void launch_beam_hist(const SimDev<R> &S, int np_upper, double thr, double width, int nbins,
                                         double *hist, cudaStream_t st);
template <class R> void launch_beam_moments(const SimDev<R> &S, int np_upper, double thr, double e_peak,
                                            double fwhm, double *out14, cudaStream_t st);
constexpr int kBeamBins = 256;
template <class R> void launch_diag_accel(const SimDev<R> &S, int np_upper, double thr,
                                          double *out4, cudaStream_t st);
// canonical dump / upload of one grid array (kind as in lpic_diag_kind), columns [c0, c1)
template <class R> void launch_dump_field(const SimDev<R> &S, int kind, int c0, int c1,
                                          double *stage, cudaStream_t st);
template <class R> void launch_upload_field(const SimDev<R> &S, int kind, int c0, int c1,
                                            const double *stage, cudaStream_t st);
// alive-particle compaction index list (deterministic order); returns count via *d_count
template <class R> void launch_alive_index(const SimDev<R> &S, int np_upper, int *idx,
                                           int *blockcnt, int *d_count, cudaStream_t st);
template <class R> void launch_dump_particles(const SimDev<R> &S, const int *idx, int k0, int k1,
                                              int comp, double *stage, cudaStream_t st);
template <class R> void launch_native_particles(const SimDev<R> &S, const int *idx, int k0, int k1,
                                                int comp, void *buf, int mode, cudaStream_t st);
template <class R> void launch_upload_particles(const SimDev<R> &S, int k0, int k1, int comp,
                                                const double *stage, cudaStream_t st);
template <class R> void launch_set_ids(const SimDev<R> &S, const int *idx, int k0, int k1,
                                       const uint64_t *stage, uint64_t *out, int mode,
                                       cudaStream_t st);
template <class R> void launch_finish_upload(const SimDev<R> &S, int n, cudaStream_t st);

}  // namespace lpic
