/*
 * lpic.h -- C ABI of the GB300 (sm_103a) implementation of one timestep of the
 * cylindrical (azimuthal mode m=0) laser-envelope particle-in-cell method of
 * Massimo et al., arXiv:1912.04674.
 *
 * Normalised units throughout (paper Sec. 2): lengths in c/w0, time in 1/w0,
 * fields in m c w0/e, densities in n_c.  Macro-particles are electrons
 * (q = -1, m = 1) over an immobile neutralising ion background.
 *
 * Memory and streams.  The caller owns ONE device buffer of
 * lpic_required_bytes() bytes and the CUDA stream; the library sub-allocates
 * every grid, particle and scratch array from that buffer and never calls
 * cudaMalloc.  Every call that launches work enqueues it on the context's
 * stream and returns without synchronising, except lpic_diagnose and
 * lpic_upload, which synchronise that stream.  The caller must not touch the
 * buffer while work is in flight.  A context is used by one host thread at a
 * time.
 *
 * Errors.  Every call returns an lpic_status; nothing is thrown across the ABI.
 * lpic_last_error() gives a message for the last failing call on a context.
 * Errors found on the device (particle capacity exhausted, a non-finite value)
 * are latched in the context and reported by the next call.
 *
 * Canonical grid layout used by dumps and uploads: [i][j], radial index j
 * fastest, FP64 (complex values as (re, im) pairs), with the staggering
 *   A, chi, Phi, dq : (i, j)        i in [0,Nx], j in [0,Nr]   (Nx+1) x (Nr+1)
 *   Ex, Jx          : (i+1/2, j)    i in [0,Nx-1], j in [0,Nr] Nx x (Nr+1)
 *   Er, Jr          : (i, j+1/2)    i in [0,Nx], j in [0,Nr-1] (Nx+1) x Nr
 *   Bt              : (i+1/2, j+1/2)                           Nx x Nr
 * (paper Sec. 3: Yee-like cell with Lifschitz centring, envelope centred like E).
 */
#ifndef LPIC_H
#define LPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpic_ctx lpic_ctx;
typedef struct lpic_batch lpic_batch;

typedef enum {
    LPIC_OK = 0,
    LPIC_EINVAL = 1,         /* bad argument or size                                   */
    LPIC_ECFL = 2,           /* time step outside the stability region of a solver    */
    LPIC_ENOMEM_BUDGET = 3,  /* caller buffer smaller than lpic_required_bytes        */
    LPIC_EBUFSIZE = 4,       /* output buffer too small, or particle capacity exceeded */
    LPIC_ECUDA = 5,          /* a CUDA runtime call failed                             */
    LPIC_ETIMEOUT = 6,       /* a bounded device wait gave up                          */
    LPIC_ENONFINITE = 7,     /* a NaN/Inf: a diagnostic's result or a pushed position  */
    LPIC_ESTATE = 8          /* call out of order (e.g. step before init)              */
} lpic_status;

typedef enum {
    LPIC_FP64 = 0,           /* everything in FP64                                        */
    LPIC_FP32_MIXED = 1      /* FP32 push/gather/stencils, int cell + FP32 offset
                                positions, FP64 axis rows and FP64 J/chi accumulation      */
} lpic_precision;

/* Grid and time step (paper Sec. 3; benchmarks of Sec. 4 use dt = 0.8 dx or 0.9 dx). */
typedef struct {
    int32_t nx, nr;              /* cells in x and r; r_max = nr*dr; Nx*Nr < 2^31           */
    double dx, dr, dt;           /* must satisfy the stability limits of lpic_check_params  */
    int32_t moving_window;       /* 1: window moves at c (shift one cell when (n+1)dt >= (s+1)dx) */
    int32_t sort_every;          /* counting sort + compaction of particles every k steps (>=1) */
    int64_t particle_capacity;   /* particle slots; lpic_particle_capacity() gives a value  */
    int32_t track_continuity;    /* 1: also deposit the per-step charge change (diagnostic) */
    double accel_px_min;         /* p_x threshold of "accelerated" electrons; <= 0 means 10 */
    int32_t filter_passes;       /* binomial current filter after each deposit (Sec. 4 nonlinear
                                    run: 7 passes): each pass replaces Jx, Jr (and the tracked
                                    charge change) by (F_{i-1} + 2F_i + F_{i+1})/4 along x, zero
                                    outside the window; 0 = off, at most 16                   */
    int32_t slab_x0;             /* x-slab decomposition (lpic_slab_exchange): global window
                                    column of this grid's column 0 when the grid is one slab of
                                    a wider window, else 0.  The context's shift counter then
                                    reads s + slab_x0 (the lab cell of its column 0) and the
                                    moving window still shifts when (n+1)dt >= (s+1)dx        */
    int32_t slab_front_interior; /* 1: this slab's front column lies inside the global window,
                                    so the moving window injects no plasma there (the exchange
                                    fills it); 0 for the front slab or a whole window          */
} lpic_grid_params;

/* Gaussian envelope (paper Sec. 4; paraxial focused pulse, field profile exp(-xi^2/L^2)). */
typedef struct {
    double a0, w0, L;            /* peak |A|, waist, 1/e field half-length                  */
    double x_center, x_focus;    /* lab-frame pulse centre at t=0 and focal plane           */
} lpic_laser_params;

/* Plasma: density n0 (n_c), zero before x_start, linear up-ramp of length ramp_len;
 * regular lattice of ppc_x * ppc_r * ppc_theta particles per (x, r) cell (paper Sec. 4
 * uses 6 per cell; the build's workloads 2x2x4), azimuthal offset from SplitMix64(seed). */
typedef struct {
    double n0, x_start, ramp_len;
    int32_t ppc_x, ppc_r, ppc_theta;
    uint64_t seed;
} lpic_plasma_params;

typedef enum {
    LPIC_DIAG_EX_AXIS = 0,       /* Nx doubles: Ex(i+1/2, r=0) (paper Sec. 4, on-axis wake)  */
    LPIC_DIAG_A_ABS_MAX = 1,     /* 1 double: max |A| over the grid                          */
    LPIC_DIAG_WAIST = 2,         /* 1 double: sqrt(2 <r^2>) weighted by |A|^2 (Sec. 4, w(x)) */
    LPIC_DIAG_CONT_RESIDUAL = 3, /* 1 double: max_ij |dQ/dt + div I| / max_ij |div I| over
                                    interior nodes for the last step (needs track_continuity) */
    LPIC_DIAG_ACCEL_ENERGY = 4,  /* 4 doubles: count, sum w, weighted mean and rms of gamma-1
                                    over alive electrons with p_x > accel_px_min            */
    LPIC_DIAG_COUNTERS = 5,      /* 4 int64: step n, window shift s, particle slots, alive   */
    LPIC_DIAG_BEAM = 6,          /* 12 doubles, the injected-beam parameters of Table BeamParams
                                    (Sec. 4) over alive electrons with p_x > accel_px_min:
                                    {n_accel, n_beam, charge (sum w), E_peak, FWHM, dE/E,
                                    eps_y, eps_z, eps_mean, mean E, E_max, bins}.  E = gamma-1
                                    (m c^2); spectrum = w-weighted histogram of E in 256 bins
                                    over [0, E_max]; E_peak = centre of the first largest bin;
                                    FWHM from the half-maximum crossings (linear interpolation
                                    between bin centres); beam = |E - E_peak| <= FWHM;
                                    dE/E = rms E over the beam / E_peak; eps_u =
                                    sqrt(s_uu s_pp - s_up^2) of the beam's central moments
                                    (c/w0 units), u = y, z.  All zero without accelerated e-. */
    LPIC_DIAG_EX = 10, LPIC_DIAG_ER = 11, LPIC_DIAG_BT = 12,
    LPIC_DIAG_A = 13,            /* A^n, complex (re,im)                                     */
    LPIC_DIAG_AM = 14,           /* A^{n-1}, complex (re,im)                                 */
    LPIC_DIAG_CHI = 15, LPIC_DIAG_JX = 16, LPIC_DIAG_JR = 17, LPIC_DIAG_DQ = 18,
                                 /* chi, J, dQ: deposits of the last step, on that step's window
                                    (before its moving-window shift)                        */
    LPIC_DIAG_PARTICLES = 20,    /* 7 x n doubles, SoA: x(lab), y, z, px, py, pz, w          */
    LPIC_DIAG_PARTICLE_IDS = 21, /* n uint64 ids, same order as LPIC_DIAG_PARTICLES          */
    LPIC_DIAG_PARTICLES_NATIVE = 22
                                 /* the particle store as the context holds it (checkpoint
                                    form), same particles and order as LPIC_DIAG_PARTICLES:
                                    n uint64 ids, then 7 blocks of n values in the working
                                    precision (float for LPIC_FP32_MIXED, double for
                                    LPIC_FP64): in-cell x offset in [0, 1), y, z, px, py, pz,
                                    w; then n int32 lab cell indices (x = (cell + offset) dx).
                                    12 + 7 x 4 = 40 bytes per electron in FP32_MIXED, 68 in
                                    FP64; every block starts aligned to its element size.
                                    Dump and upload are bit-exact.                          */
} lpic_diag_kind;

/* Stability and consistency check of the parameters, host only (needs no GPU).
 * Limits (dt, dx, dr):
 *   Yee m=0:   dt * sqrt(4/dx^2 + 4.842/dr^2) < 2      (4.842/dr^2: spectral radius of
 *              the discrete radial operator including the axis row)
 *   envelope:  dt^2 [(2 + 2 sqrt(1+dx^2))/dx^2 + 4.842/dr^2] <= 2 + 2 sqrt(1+dt^2)
 *              dt^2 (2 sqrt(1+dx^2) - 2)/dx^2              <= 2 sqrt(1+dt^2) - 2
 *              (roots of the centred scheme of Eq. envelope_solver on the unit circle)
 *   particles: dt < dx and dt < dr (a particle moves less than one cell per step)
 * Returns LPIC_OK, LPIC_EINVAL or LPIC_ECFL; writes a message into msg (may be NULL). */
lpic_status lpic_check_params(const lpic_grid_params *g, const lpic_plasma_params *p,
                              char *msg, size_t msg_cap);

/* Particle slots needed for plasma p on grid g: the full window, 10% more for electrons
 * that travel with the window (trapped or pushed ahead of the pulse) while fresh plasma is
 * injected, and the injection of (sort_every + 2) window shifts between compactions.
 * 0 for p == NULL. */
int64_t lpic_particle_capacity(const lpic_grid_params *g, const lpic_plasma_params *p);

/* Bytes of the caller-owned device buffer for grid g (with g->particle_capacity) in
 * precision prec; 0 if the parameters are invalid. */
size_t lpic_required_bytes(const lpic_grid_params *g, lpic_precision prec);

/* Create a context on the current CUDA device (paper Sec. 3: the 2D (x,r) grid).
 * device_buf: caller-owned, >= lpic_required_bytes(g, prec) bytes, 256-byte aligned,
 * must stay valid until lpic_destroy.  cuda_stream: a cudaStream_t (NULL = default).
 * Zeroes all fields; no particles.  *out is set only on LPIC_OK. */
lpic_status lpic_init_grid(lpic_ctx **out, const lpic_grid_params *g, lpic_precision prec,
                           void *device_buf, size_t buf_bytes, void *cuda_stream);

/* Write the Gaussian envelope A^0 (t=0) and A^{-1} (t=-dt) on the current window
 * (paper Sec. 4 benchmarks; paraxial focused Gaussian, xR = w0^2/2). */
lpic_status lpic_init_envelope(lpic_ctx *ctx, const lpic_laser_params *laser);

/* Load the plasma lattice on every cell column of the current window and remember the
 * profile for injection at the moving-window front (paper Sec. 4: uniform plasma,
 * regular particles per cell).  Cold (p = 0).  LPIC_EBUFSIZE if the capacity is short. */
lpic_status lpic_load_plasma(lpic_ctx *ctx, const lpic_plasma_params *plasma);

/* Advance nsteps timesteps (paper Sec. 3, the 3D envelope loop order):
 * Faraday -> gather/chi deposit/ponderomotive Boris -> envelope solve (Eq. envelope_solver)
 * -> position push/charge-conserving current -> Ampere -> moving window/injection,
 * with a counting sort every sort_every steps.  Asynchronous on the context stream.  The
 * steps are replayed from CUDA graphs recorded on first use (eight steps per replay where none
 * of them sorts or relocates the window, else one); with kernel timing on
 * (lpic_set_kernel_timing) they are launched kernel by kernel instead.  The state reached is
 * the same either way, up to the order of the FP64 atomic additions.
 * Conditions the kernels latch (plasma injection beyond the capacity: LPIC_EBUFSIZE; a
 * particle pushed to a non-finite position: LPIC_ENONFINITE) are returned by the next
 * lpic_step whose predecessor has completed, or by the next lpic_diagnose. */
lpic_status lpic_step(lpic_ctx *ctx, int nsteps);

/* Read an observable into host memory host_out (capacity cap bytes); *written gets the
 * byte count.  Synchronises the context stream.  LPIC_EBUFSIZE if cap is too small
 * (*written then holds the size needed); LPIC_ENONFINITE if a returned scalar is NaN/Inf
 * or a step latched a non-finite particle position. */
lpic_status lpic_diagnose(lpic_ctx *ctx, lpic_diag_kind kind, void *host_out, size_t cap,
                          size_t *written);

/* Asynchronous form of lpic_diagnose for the on-axis wake (LPIC_DIAG_EX_AXIS, same layout:
 * Nx doubles): enqueues the read into host_out on the context stream and returns without
 * synchronising, so that a caller can consume step n's wake while step n+1 runs.  host_out
 * should be page-locked: if the device can address it (cudaHostAlloc, cudaHostRegister, a
 * pinned torch tensor, 8-byte aligned) the kernel writes the wake into it directly, with no
 * copy on the stream; other page-locked memory is filled by a copy from the staging area, and
 * a pageable destination makes that copy synchronous.  host_out holds the result once the
 * stream has passed this call (an event recorded after it, or any synchronising call) and must
 * stay valid until then.  Errors: LPIC_EINVAL for another kind
 * or a NULL host_out, LPIC_EBUFSIZE if cap < Nx * 8; device-side errors of earlier steps are
 * reported by the next synchronising call. */
lpic_status lpic_diagnose_async(lpic_ctx *ctx, lpic_diag_kind kind, void *host_out, size_t cap);

/* Overwrite a part of the state from host memory in the dump layout of the same kind
 * (checkpoint restore, or starting from another implementation's state).  Accepts
 * LPIC_DIAG_EX/ER/BT/A/AM (exact sizes), LPIC_DIAG_PARTICLES (7n doubles: replaces the
 * particle set by n particles, ids reset to 0..n-1), LPIC_DIAG_PARTICLE_IDS (n ids for the
 * current set), LPIC_DIAG_PARTICLES_NATIVE (n electrons in the context's own layout and
 * precision, ids included: a dump of this kind restores the particle store bit for bit) and
 * LPIC_DIAG_COUNTERS (step and shift; the other two entries are ignored).  A particle upload
 * marks electrons outside the window or at r >= r_max as removed, and restarts the sort
 * cadence (the next counting sort comes sort_every steps later).  Field dumps and uploads are
 * exact in both precisions (FP32 values pass through FP64 unchanged), so the field kinds, the
 * native particles and the counters together are a checkpoint.
 * Page-locked host memory that the device can address (cudaHostAlloc, cudaHostRegister, a
 * pinned torch tensor) and that is 8-byte aligned is read by the conversion kernels in place
 * over the host link; other host memory goes through the library's staging area in chunks.
 * Synchronises the context stream. */
lpic_status lpic_upload(lpic_ctx *ctx, lpic_diag_kind kind, const void *host_in, size_t bytes);

/* Tracing.  Launches of every kernel family are always counted; while timing is enabled,
 * lpic_step also records a CUDA event pair around each launch on the context stream.
 * lpic_kernel_stats writes, for up to cap families, the launch count since lpic_init_grid
 * and the device milliseconds accumulated while timing was on (it synchronises the stream
 * and then clears the accumulated times); *n gets the number of families.  Family k is
 * named by lpic_kernel_name(k) (NULL past the last). */
lpic_status lpic_set_kernel_timing(lpic_ctx *ctx, int enable);
lpic_status lpic_kernel_stats(lpic_ctx *ctx, int64_t *launches, double *ms, int cap, int *n);
const char *lpic_kernel_name(int k);

/* Allocation-free envelope statistics.  The paper has no counterpart: this is a service for
 * callers that cannot call cudaMalloc -- code whose device memory all comes from a pool it
 * was handed (a host framework with its own allocator, a plug-in, a real-time loop whose
 * memory is fixed before it starts) -- and so cannot create a context either.
 * Computes, like lpic_diagnose(LPIC_DIAG_A_ABS_MAX) and lpic_diagnose(LPIC_DIAG_WAIST),
 *   out_dev[0] = max |A|,  out_dev[1] = sqrt(2 <r^2>) weighted by |A|^2 (node volumes),
 * from a_dev: the envelope in the canonical dump layout of LPIC_DIAG_A ((nx+1) x (nr+1)
 * complex FP64 (re, im) pairs, radial index fastest), in device memory the caller owns.
 * out_dev: 2 doubles of caller-owned device memory.  Asynchronous on cuda_stream.
 * It allocates nothing: its scratch (one partial per 4096 nodes) is a fixed 96 KiB array in
 * the library's device memory, present on every device that loads the library until the
 * process exits, which limits the input to (nx+1)(nr+1) <= 16,777,216 nodes (LPIC_EBUFSIZE
 * beyond).  The first call on a device looks up that array's device address (with the
 * device current) and keeps it for the life of the process; make that first call before
 * any stream capture.  A cudaDeviceReset of that device invalidates the kept address: do
 * not call this entry point on a device after resetting it.  Every call rewrites
 * the partials it uses, so nothing carries over, but all calls share the one array: calls
 * that overlap on the GPU (on different streams, or from several threads) race.
 * Returns LPIC_OK, LPIC_EINVAL (NULL pointer, sizes < 1, dr <= 0), LPIC_EBUFSIZE or
 * LPIC_ECUDA. */
lpic_status lpic_envelope_stats_noalloc(const void *a_dev, int32_t nx, int32_t nr, double dr,
                                        double *out_dev, void *cuda_stream);

/* x-slab decomposition of one simulation (Sec. 3: the envelope solver parallelises with the
 * strategies of a standard Yee scheme, i.e. sub-domains that exchange guard cells; Sec. 4 runs
 * it on patches).  left and right are contexts of the same precision, nr, dx, dr, dt and step
 * counter, on the same stream, holding adjacent slabs of one window: left covers global columns
 * [x0_L, x0_L + nx_L], right starts at x0_R (their slab_x0), and they overlap by 2*halo columns
 * around the boundary B = x0_R + halo = x0_L + nx_L - halo; left owns the cells below B and
 * right the cells from B on.  After both have completed the same step, this call enqueues:
 *   - E, B_theta, A^n and A^{n-1} of the owner copied into the other's halo columns (right's
 *     nodes [B, B+halo] and cells [B, B+halo) into left; left's [B-halo, B) into right);
 *   - left's electrons in cells >= B and right's in cells < B removed, then right's
 *     electrons in cells [B, B+halo) appended to left and left's in [B-halo, B) appended to
 *     right (same ids: the owner keeps its own), each into the slots its removal freed first
 *     (listed in the context's staging area) and then past its slots in use,
 * so that each slab computes its owned columns of the next step exactly as one whole window
 * would: one step's phases reach at most 6 columns from a wrong boundary value (Faraday,
 * gather, deposit, envelope, position push, current, Ampere and the window shift), so halo >= 8
 * (>= 8 + filter_passes with the current filter) and every slab must own >= halo columns.
 * Layout: the copies move whole columns of the persistent arrays (the sliding offsets of
 * the two contexts are read on the device).  Errors: LPIC_EINVAL for mismatched contexts or a
 * boundary that does not match the slab_x0/nx values; an append beyond a context's particle
 * capacity is latched (LPIC_EBUFSIZE from that context's next call). */
lpic_status lpic_slab_exchange(lpic_ctx *left, lpic_ctx *right, int32_t halo);

/* Measurement helper (the paper has no counterpart): enqueues on cuda_stream one launch that
 * keeps every SM's FP64 pipe busy with fused multiply-adds (8 independent chains of `iters`
 * FMAs per thread, one resident wave of blocks), for timing the FP64 peak that bounds the FP64
 * particle passes.  *flops gets the launch's FP64 operations (FMA = 2); out_dev: 2 doubles of
 * caller-owned device memory the launch writes.  LPIC_EINVAL (iters < 1, NULL), LPIC_ECUDA. */
lpic_status lpic_probe_fp64_fma(int32_t iters, double *out_dev, int64_t *flops, void *cuda_stream);

/* Release the context (host memory only; the device buffer stays the caller's). */
lpic_status lpic_destroy(lpic_ctx *ctx);

/* ---- externally injected relativistic bunch (Sec. 3: the field initialisation of a bunch
 * in uniform motion, in cylindrical symmetry) -------------------------------------------------
 * Appends n electrons (host_parts: 7 x n doubles, SoA as for LPIC_DIAG_PARTICLES: lab x, y,
 * z, px, py, pz, w; ids 2^63 + a running count) and adds to E^n and B^{n-1/2} the fields of
 * their charge moving along x at beta = sqrt(1 - 1/gamma^2):
 *   E = -(dphi/dx / gamma^2, dphi/dr),  B_theta = beta E_r moved back by beta dt/2,
 * phi from the flux-form discrete Gauss law of the Yee grid (the divergence the Maxwell solver
 * conserves) with no x flux through the window ends and phi = 0 at r_max, solved by
 * preconditioned conjugate gradients to a relative residual of 1e-12 (at most 2000
 * iterations).  scratch: caller-owned device memory of lpic_bunch_scratch_bytes, 256-byte
 * aligned, free again when the call returns.  Synchronous.  Errors: LPIC_EINVAL (gamma <= 1,
 * non-finite input, bad scratch), LPIC_EBUFSIZE (capacity), LPIC_ENONFINITE (no convergence). */
size_t lpic_bunch_scratch_bytes(const lpic_ctx *ctx);
lpic_status lpic_inject_bunch(lpic_ctx *ctx, const double *host_parts, int64_t n, double gamma, void *scratch,
                              size_t scratch_bytes);

/* Message of the last failing call on ctx (or of the last failing lpic_init_grid /
 * lpic_batch_create on this thread when ctx is NULL).  Never NULL. */
const char *lpic_last_error(const lpic_ctx *ctx);

/* ---- batched form: many independent simulations advanced together ------------------
 * The paper runs one simulation at a time; a parametric scan (a0, density, waist, grid
 * size) is many independent runs of the same step (Sec. 2-3 equations, unchanged).  The
 * batch advances them together: one step is a fixed sequence of fused persistent launches
 * (prepass, pass A, envelope, pass B, Ampere, window), each walking a work list of
 * {simulation, tile or block of particle slots} items over every active simulation,
 * recorded once per set of active simulations in a CUDA graph and replayed; the blocks of
 * the particle passes draw their items from ticket counters.  The periodic counting sorts
 * of the simulations due at a step are seven more fused launches in a second graph;
 * relocation stays per simulation, on the batch stream.  A tuning (lpic_batch_set_tuning)
 * can instead replay each simulation's own step graph.
 * All contexts must share one precision and one device, be initialised
 * (lpic_init_envelope done), and appear once.  The contexts keep their own buffers. */

/* Device bytes the batch needs for its sort flags, item tickets and work lists (0 if the
 * contexts are invalid).  Depends on the contexts' shapes. */
size_t lpic_batch_required_bytes(lpic_ctx *const *ctxs, int n);

/* device_buf: caller-owned, 256-byte aligned, at least lpic_batch_required_bytes bytes,
 * alive and untouched until lpic_batch_destroy.  cuda_stream: the batch stream.
 * Errors: LPIC_EINVAL (bad contexts or alignment), LPIC_ENOMEM_BUDGET (buffer too small),
 * LPIC_ECUDA; the message is lpic_last_error(NULL). */
lpic_status lpic_batch_create(lpic_batch **out, lpic_ctx *const *ctxs, int n, void *device_buf,
                              size_t buf_bytes, void *cuda_stream);
/* Advance simulation k by steps_per_ctx[k] >= 0 steps; simulations with fewer steps
 * drop out of the later launches (their items leave the work lists).  Asynchronous on the
 * batch stream, ordered after earlier work on each context's stream; later calls on a
 * context's stream are ordered after it.  Device-side errors of one simulation (particle
 * capacity) are reported by that context's next lpic_diagnose. */
lpic_status lpic_batch_step(lpic_batch *b, const int *steps_per_ctx);
/* Tuning of the fused launches, effective at the next lpic_batch_step:
 * particles_per_item: particle slots per work item of the fused particle passes (a
 *   multiple of 256 in [1024, 1048576]; default 4096).  Smaller items balance the blocks
 *   better, larger ones cost less per item.
 * packs: split the simulations into this many packs (0: as few as the parameter space
 *   allows, one per 46 simulations), each with its own launch sequence as a parallel branch
 *   of the graph, so that phases of different packs overlap on the device.  -1: no fused
 *   launches; each step replays every simulation's own step graph (lpic_step) on its own
 *   stream, in turn, which overlaps better for batches of large simulations.
 * The binding's autotuner picks both by timing real steps.  Errors: LPIC_EINVAL. */
lpic_status lpic_batch_set_tuning(lpic_batch *b, int32_t particles_per_item, int32_t packs);
/* Kernels the batch has enqueued so far (fused launches, relocations and sorts). */
int64_t lpic_batch_launches(const lpic_batch *b);
/* Message of the last failing call on b.  Never NULL. */
const char *lpic_batch_last_error(const lpic_batch *b);
lpic_status lpic_batch_destroy(lpic_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* LPIC_H */
