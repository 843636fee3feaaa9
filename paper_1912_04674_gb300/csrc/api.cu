// Host side of the C ABI declared in include/lpic.h: parameter checks, memory planning
// inside the caller's buffer, step orchestration, diagnostics, uploads, batched form.
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "lpic.h"
#include "lpic_internal.cuh"

using namespace lpic;

namespace {

thread_local std::string g_thread_err;
constexpr size_t kAlign = 256;
constexpr size_t kStageBytes = size_t(8) << 20;
constexpr double kRadialSpectral = 4.842;  // sup of dr^2 x spectral radius, m=0 radial operator

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }


void msgf(char *msg, size_t cap, const char *fmt, double a = 0, double b = 0) {
    if (msg && cap) snprintf(msg, cap, fmt, a, b);
}

lpic_status check_params(const lpic_grid_params *g, const lpic_plasma_params *p, char *msg,
                         size_t cap) {
    if (!g) { msgf(msg, cap, "grid params are NULL"); return LPIC_EINVAL; }
    if (g->nx < 2 || g->nr < 2) { msgf(msg, cap, "nx=%g and nr=%g must be >= 2", g->nx, g->nr); return LPIC_EINVAL; }
    if (g->nr > 65536) { msgf(msg, cap, "nr=%g exceeds 65536", g->nr); return LPIC_EINVAL; }
    if ((long long)(g->nr + 6) * 2 * (g->nx + 1 + 2 * kG) * 4 >= (1LL << 31)) {
        msgf(msg, cap, "grid of nx=%g, nr=%g too large for 32-bit element indices", g->nx, g->nr);
        return LPIC_EINVAL;
    }
    if ((long long)g->nx * g->nr + 1 > (long long)4096 * 4096) {
        msgf(msg, cap, "nx*nr=%g cells exceeds the counting-sort limit 16777215", (double)g->nx * g->nr);
        return LPIC_EINVAL;
    }
    const double dx = g->dx, dr = g->dr, dt = g->dt;
    if (!(dx > 0 && dr > 0 && dt > 0) || !std::isfinite(dx) || !std::isfinite(dr) || !std::isfinite(dt)) {
        msgf(msg, cap, "dx, dr, dt must be positive and finite");
        return LPIC_EINVAL;
    }
    if (g->particle_capacity < 0 || g->particle_capacity > (int64_t)INT32_MAX / 2) {
        msgf(msg, cap, "particle_capacity=%g out of range", (double)g->particle_capacity);
        return LPIC_EINVAL;
    }
    if (g->filter_passes < 0 || g->filter_passes > kFilterMaxPasses) {
        msgf(msg, cap, "filter_passes=%g outside [0, %g]", g->filter_passes, kFilterMaxPasses);
        return LPIC_EINVAL;
    }
    if (g->slab_x0 < 0 || (g->slab_front_interior != 0 && g->slab_front_interior != 1)) {
        msgf(msg, cap, "slab_x0 must be >= 0 and slab_front_interior 0 or 1");
        return LPIC_EINVAL;
    }
    if (g->particle_capacity > 0 && g->sort_every < 1) {
        msgf(msg, cap, "sort_every must be >= 1 when particles are present");
        return LPIC_EINVAL;
    }
    // Yee m=0 leapfrog: dt * omega_max < 2
    const double wmax = std::sqrt(4.0 / (dx * dx) + kRadialSpectral / (dr * dr));
    if (!(dt * wmax < 2.0)) {
        msgf(msg, cap, "Yee stability: dt=%g >= %g", dt, 2.0 / wmax);
        return LPIC_ECFL;
    }
    // envelope scheme: both characteristic roots on the unit circle for every mode
    const double sx = std::sqrt(1.0 + dx * dx), st = std::sqrt(1.0 + dt * dt);
    const double kmax = (2.0 + 2.0 * sx) / (dx * dx) + kRadialSpectral / (dr * dr);
    const double kneg = (2.0 * sx - 2.0) / (dx * dx);
    if (!(dt * dt * kmax <= 2.0 + 2.0 * st) || !(dt * dt * kneg <= 2.0 * st - 2.0)) {
        msgf(msg, cap, "envelope stability: dt=%g outside the stable range (dx=%g)", dt, dx);
        return LPIC_ECFL;
    }
    if (!(dt < dx && dt < dr)) {
        msgf(msg, cap, "particle step: dt=%g must be below min(dx, dr)=%g", dt, std::fmin(dx, dr));
        return LPIC_ECFL;
    }
    if (p) {
        if (!(p->n0 >= 0) || !std::isfinite(p->n0) || !(p->ramp_len >= 0) || !std::isfinite(p->x_start)) {
            msgf(msg, cap, "plasma: n0 >= 0, ramp_len >= 0 and finite values required");
            return LPIC_EINVAL;
        }
        if (p->ppc_x < 1 || p->ppc_x > 16 || p->ppc_r < 1 || p->ppc_theta < 1 ||
            (long long)p->ppc_x * p->ppc_r * p->ppc_theta > 1024) {
            msgf(msg, cap, "plasma: ppc_x in [1,16], ppc_r, ppc_theta >= 1, product <= 1024");
            return LPIC_EINVAL;
        }
    }
    if (msg && cap) msg[0] = 0;
    return LPIC_OK;
}

struct Layout {
    size_t desc, tab, grid[18], parts[2][9], key, count, blocksum, blockcnt, icount, diag, stage, total;
    int P, nlive, ncol;
};

Layout make_layout(const lpic_grid_params *g, lpic_precision prec) {
    Layout L{};
    const size_t rs = prec == LPIC_FP64 ? 8 : 4;
    L.P = ((g->nr + 3) + 3) / 4 * 4;  // rows up to nr+2 are touched by the 3x3 deposit window
    L.nlive = g->nx + 1 + 2 * kG;
    L.ncol = g->moving_window ? 2 * L.nlive : L.nlive;
    const size_t cells = (size_t)L.P * L.ncol;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
    L.desc = take(sizeof(Desc));
    L.tab = take((size_t)NTAB * L.P * rs + kAxisFactors * sizeof(double));
    // ex er bt btn phih (R), pg (4R), exq erq (2R, FP32 only), a0 a1 (2R), chi jx jr dq
    // (double), [14-16 filter], btq (2R, FP32 only)
    const bool paired = prec != LPIC_FP64;
    for (int k = 0; k < 5; k++) L.grid[k] = take(cells * rs);
    L.grid[5] = take(cells * 4 * rs);
    L.grid[6] = paired ? take(cells * 2 * rs) : 0;
    L.grid[7] = paired ? take(cells * 2 * rs) : 0;
    for (int k = 8; k < 10; k++) L.grid[k] = take(cells * 2 * rs);
    for (int k = 10; k < 14; k++) L.grid[k] = take(cells * 8);
    // filtered current and charge change (only with the binomial filter on)
    for (int k = 14; k < 17; k++) L.grid[k] = g->filter_passes > 0 ? take(cells * 8) : 0;
    L.grid[17] = paired ? take(cells * 2 * rs) : 0;
    const size_t cap = (size_t)g->particle_capacity;
    for (int b = 0; b < 2; b++) {
        L.parts[b][0] = take(cap * 4);                          // ix
        for (int k = 1; k < 8; k++) L.parts[b][k] = take(cap * rs);  // ox y z px py pz w
        L.parts[b][8] = take(cap * 8);                          // id
    }
    const size_t ncell = (size_t)g->nx * g->nr;
    L.key = take((cap + 1) * 4);
    L.count = take((ncell + 2) * 4);
    L.blocksum = take(((ncell + 1 + 4095) / 4096 + 1) * 4);
    L.blockcnt = take((cap / 256 + 2) * 4);
    L.icount = take(((cap / 256 + 2) / 4096 + 4) * 4);   // count + scan block scratch
    L.diag = take(16 * 8);
    size_t col_bytes = (size_t)(g->nr + 1) * 16;
    size_t stage = kStageBytes;
    if (stage < col_bytes) stage = col_bytes;
    L.stage = take(stage);
    L.total = o;
    return L;
}

int valid_a_count(const Phys &ph, long long c) {
    int nv = 0;
    for (int a = 0; a < ph.ppcx; a++)
        if (plasma_density(ph, lattice_x(ph, c, a)) > 0.0) nv++;
    return nv;
}

// Host-side constants and per-row tables of one simulation.
template <class R> Kc<R> make_consts(const Phys &ph, int nr, const R *tab_dev) {
    Kc<R> k{};
    const double dx = ph.dx, dr = ph.dr, dt = ph.dt;
    k.dt = (R)dt;
    k.hdt = (R)(0.5 * dt);
    k.idx = (R)(1.0 / dx);
    k.idr = (R)(1.0 / dr);
    k.dtdx = (R)(dt / dx);
    k.hidx = (R)(0.5 / dx);
    k.hidr = (R)(0.5 / dr);
    k.idx2 = (R)(1.0 / (dx * dx));
    k.idr2 = (R)(1.0 / (dr * dr));
    k.dt2 = (R)(dt * dt);
    k.envp = (R)(1.0 / (1.0 + dt * dt));
    k.envpt = (R)(dt / (1.0 + dt * dt));
    k.d_dt = dt;
    k.d_dt2 = dt * dt;
    k.d_idx2 = 1.0 / (dx * dx);
    k.d_idr2 = 1.0 / (dr * dr);
    k.d_hidx = 0.5 / dx;
    k.d_envp = 1.0 / (1.0 + dt * dt);
    k.d_envpt = dt / (1.0 + dt * dt);
    k.d_4idr = 4.0 / dr;
    k.rmax = (R)(nr * dr);
    k.lat_ippcx = (R)ph.inv_ppcx;
    k.lat_ippcr = (R)ph.inv_ppcr;
    k.lat_ippct = (R)ph.inv_ppct;
    k.lat_dr = (R)dr;
    k.lat_wfac = (R)ph.wfac;
    k.tab = tab_dev;
    return k;
}

std::vector<double> row_tables(const Phys &ph, int P) {
    std::vector<double> t((size_t)NTAB * P, 0.0);
    const double dr = ph.dr;
    for (int j = 0; j < P; j++) {
        t[(size_t)T_CHI * P + j] = row_ichi(ph, j);
        t[(size_t)T_JX * P + j] = row_ijx(ph, j);
        t[(size_t)T_JR * P + j] = row_ijr(ph, j);
        if (j > 0) {
            t[(size_t)T_ENV1R * P + j] = 1.0 / (2.0 * dr * (j * dr));
            t[(size_t)T_AMPP * P + j] = ((j + 0.5) * dr) / ((j * dr) * dr);
            t[(size_t)T_AMPM * P + j] = ((j - 0.5) * dr) / ((j * dr) * dr);
        }
    }
    return t;
}

}  // namespace

struct lpic_ctx {
    lpic_precision prec;
    lpic_grid_params g;
    Phys ph{};
    Geo geo{};
    cudaStream_t st = nullptr;
    char *buf = nullptr;
    size_t bytes = 0;
    Layout L{};
    SimDev<double> sd{};
    SimDev<float> sf{};
    Desc *d_desc = nullptr;
    int *key = nullptr, *count = nullptr, *blocksum = nullptr, *blockcnt = nullptr, *icount = nullptr;
    double *diag = nullptr;
    char *stage = nullptr;
    size_t stage_bytes = 0;
    // host mirrors of the deterministic counters
    long long step = 0, shift = 0;
    int off = 0;
    long long np_upper = 0;
    int since_sort = 0;
    unsigned long long bunch_ids = 0;   // injected-bunch particles so far
    Desc *h_desc = nullptr;          // pinned
    cudaEvent_t ev = nullptr;
    bool ev_pending = false;
    std::string err;
    bool envelope_set = false;
    // tracing
    static constexpr int kFamilies = 9;
    long long launches[kFamilies] = {};
    double ms[kFamilies] = {};
    bool timing = false;
    struct Span { int fam; cudaEvent_t a, b; };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> ev_pool;

    lpic_status fail(lpic_status s, const std::string &m) { err = m; return s; }
    lpic_status cuda_fail(cudaError_t e, const char *where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return LPIC_ECUDA;
    }
    // one step, one step followed by the sort, and kMultiSteps steps without a sort, recorded
    // as CUDA graphs and replayed while kernel timing is off; launches per replay by family
    static constexpr int kMultiSteps = 8;
    cudaGraphExec_t step_exec[3] = {nullptr, nullptr, nullptr};
    long long step_launches[3][9] = {};
    void drop_step_graphs() {
        for (auto &e : step_exec)
            if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    }
    void sync_views() {   // after a change of the physics parameters (plasma loading)
        sd.ph = ph;
        sf.ph = ph;
        sd.k = make_consts<double>(ph, geo.nr, sd.k.tab);
        sf.k = make_consts<float>(ph, geo.nr, sf.k.tab);
        drop_step_graphs();   // the recorded launches carry the old views
    }
    template <class F> void dispatch(F &&f) {
        if (prec == LPIC_FP64) f(sd); else f(sf);
    }
};

namespace {

const char *const kFamilyNames[lpic_ctx::kFamilies] = {
    "prepass", "pass_a", "envelope", "pass_b", "ampere", "window", "sort", "relocate", "filter"};
enum Fam { F_PREPASS, F_PASS_A, F_ENVELOPE, F_PASS_B, F_AMPERE, F_WINDOW, F_SORT, F_RELOCATE, F_FILTER };
constexpr int kSortLaunches = 6;  // memset-free launches of one counting sort

cudaEvent_t pool_event(lpic_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch through f, counting it as family `fam` (nlaunch kernels) and, when timing is on,
// bracketing it with events on stream st.
template <class F> void traced(lpic_ctx *c, int fam, int nlaunch, cudaStream_t st, F &&f) {
    c->launches[fam] += nlaunch;
    if (!c->timing) { f(); return; }
    lpic_ctx::Span sp{fam, pool_event(c), pool_event(c)};
    cudaEventRecord(sp.a, st);
    f();
    cudaEventRecord(sp.b, st);
    c->spans.push_back(sp);
}

template <class R> void fill_views(lpic_ctx *c, SimDev<R> &S) {
    char *b = c->buf;
    const Layout &L = c->L;
    S.geo = c->geo;
    S.ph = c->ph;
    S.k = make_consts<R>(c->ph, c->geo.nr, (const R *)(c->buf + c->L.tab));
    S.d = c->d_desc;
    S.f.ex = (R *)(b + L.grid[0]);
    S.f.er = (R *)(b + L.grid[1]);
    S.f.bt = (R *)(b + L.grid[2]);
    S.f.btn = (R *)(b + L.grid[3]);
    S.f.phih = (R *)(b + L.grid[4]);
    S.f.pg = (Q4<R> *)(b + L.grid[5]);
    using CT = typename Cplx<R>::t;
    S.f.exq = L.grid[6] ? (CT *)(b + L.grid[6]) : nullptr;
    S.f.erq = L.grid[7] ? (CT *)(b + L.grid[7]) : nullptr;
    S.f.btq = L.grid[17] ? (CT *)(b + L.grid[17]) : nullptr;
    S.f.a[0] = (typename Cplx<R>::t *)(b + L.grid[8]);
    S.f.a[1] = (typename Cplx<R>::t *)(b + L.grid[9]);
    S.f.chi = (double *)(b + L.grid[10]);
    S.f.jx = (double *)(b + L.grid[11]);
    S.f.jr = (double *)(b + L.grid[12]);
    S.f.dq = (double *)(b + L.grid[13]);
    const bool filt = c->ph.filter_passes > 0;
    S.f.jxu = filt ? (double *)(b + L.grid[14]) : S.f.jx;
    S.f.jru = filt ? (double *)(b + L.grid[15]) : S.f.jr;
    S.f.dqu = filt ? (double *)(b + L.grid[16]) : S.f.dq;
    for (int k = 0; k < 2; k++) {
        S.p[k].ix = (int32_t *)(b + L.parts[k][0]);
        S.p[k].ox = (R *)(b + L.parts[k][1]);
        S.p[k].y = (R *)(b + L.parts[k][2]);
        S.p[k].z = (R *)(b + L.parts[k][3]);
        S.p[k].px = (R *)(b + L.parts[k][4]);
        S.p[k].py = (R *)(b + L.parts[k][5]);
        S.p[k].pz = (R *)(b + L.parts[k][6]);
        S.p[k].w = (R *)(b + L.parts[k][7]);
        S.p[k].id = (uint64_t *)(b + L.parts[k][8]);
    }
    S.sb.key = (int *)(b + L.key);
    S.sb.count = (int *)(b + L.count);
    S.sb.blocksum = (int *)(b + L.blocksum);
}

lpic_status pull_desc(lpic_ctx *c) {
    cudaError_t e = cudaMemcpyAsync(c->h_desc, c->d_desc, sizeof(Desc), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "pull_desc");
    return LPIC_OK;
}
lpic_status push_desc(lpic_ctx *c) {
    cudaError_t e = cudaMemcpyAsync(c->d_desc, c->h_desc, sizeof(Desc), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "push_desc");
    return LPIC_OK;
}

lpic_status device_errors(lpic_ctx *c, const Desc &d) {
    if (d.err & ERR_CAPACITY)
        return c->fail(LPIC_EBUFSIZE, "particle capacity exhausted (plasma injection or slab exchange) "
                                      "(raise particle_capacity or lower sort_every)");
    if (d.err & ERR_NONFINITE)
        return c->fail(LPIC_ENONFINITE, "a particle was pushed to a non-finite position "
                                        "(non-finite momentum or field)");
    return LPIC_OK;
}

// Errors latched on the device by earlier asynchronous steps, if their copy has landed.
lpic_status deferred_errors(lpic_ctx *c) {
    if (!c->ev_pending) return LPIC_OK;
    cudaError_t q = cudaEventQuery(c->ev);
    if (q == cudaErrorNotReady) return LPIC_OK;
    c->ev_pending = false;
    if (q != cudaSuccess) return c->cuda_fail(q, "step");
    return device_errors(c, *c->h_desc);
}

int launch_cap(const lpic_ctx *c) {
    long long n = c->np_upper < c->g.particle_capacity ? c->np_upper : c->g.particle_capacity;
    return (int)n;
}

// Host part of one step before its launches: relocate the live region when the slide
// reaches the end of the allocation.
void pre_step(lpic_ctx *c, cudaStream_t st) {
    if (c->g.moving_window && c->off + c->geo.nlive + 1 > c->geo.ncol) {
        traced(c, F_RELOCATE, 2, st, [&] { c->dispatch([&](auto &S) { launch_relocate(S, 0, st); }); });
        c->off = 0;
    }
}

template <class S_>
void enqueue_step_kernels(lpic_ctx *c, const S_ &S, int npl, int inj, cudaStream_t st) {
    traced(c, F_PREPASS, 1, st, [&] { launch_prepass(S, st); });
    if (npl > 0) traced(c, F_PASS_A, 1, st, [&] { launch_pass_a(S, npl, st); });
    traced(c, F_ENVELOPE, 1, st, [&] { launch_envelope(S, st); });
    if (npl > 0) traced(c, F_PASS_B, 1, st, [&] { launch_pass_b(S, npl, st); });
    if (S.ph.filter_passes > 0) traced(c, F_FILTER, 1, st, [&] { launch_filter(S, st); });
    // Ampere and the moving-window step share one launch (counted as Ampere)
    traced(c, F_AMPERE, 1, st, [&] { launch_ampere_window(S, inj, st); });
}

int inj_upper(const lpic_ctx *c) {
    return c->ph.have_plasma ? c->ph.ppcx * c->ph.ppcr * c->ph.ppct * c->geo.nr : 0;
}

// Host mirror update for one step; true when the periodic sort follows the step.
bool advance_mirror(lpic_ctx *c) {
    if (window_shifts(c->ph, c->step, c->shift)) {
        c->shift += 1;
        c->off += 1;
        if (c->ph.have_plasma && c->ph.inject)
            c->np_upper += (long long)valid_a_count(c->ph, c->shift + c->geo.nx - 1) * c->ph.ppcr *
                           c->ph.ppct * c->geo.nr;
    }
    c->step += 1;
    if (c->g.particle_capacity > 0 && c->np_upper > 0 && ++c->since_sort >= c->g.sort_every) {
        c->since_sort = 0;
        return true;
    }
    return false;
}

// Host mirror update after one step's launches, and the periodic sort.
void post_step(lpic_ctx *c, cudaStream_t st) {
    if (advance_mirror(c)) {
        const int npl = launch_cap(c);
        traced(c, F_SORT, kSortLaunches, st, [&] {
            c->dispatch([&](auto &S) { launch_sort(S, npl, c->key, c->count, c->blocksum, st); });
        });
    }
}

void record_status_copy(lpic_ctx *c) {
    cudaMemcpyAsync(c->h_desc, c->d_desc, sizeof(Desc), cudaMemcpyDeviceToHost, c->st);
    cudaEventRecord(c->ev, c->st);
    c->ev_pending = true;
}

}  // namespace

// ====================================================================================== API

extern "C" {

lpic_status lpic_check_params(const lpic_grid_params *g, const lpic_plasma_params *p, char *msg,
                              size_t msg_cap) {
    return check_params(g, p, msg, msg_cap);
}

int64_t lpic_particle_capacity(const lpic_grid_params *g, const lpic_plasma_params *p) {
    if (!g || !p) return 0;
    const int64_t ppc = (int64_t)p->ppc_x * p->ppc_r * p->ppc_theta;
    const int64_t full = (int64_t)g->nx * g->nr * ppc;
    // electrons trapped in the wake or pushed ahead of the pulse ride with the window while
    // fresh plasma keeps arriving: 10% over the full window
    int64_t cap = full + full / 10 + 1024;
    if (g->moving_window) cap += (int64_t)(g->sort_every > 0 ? g->sort_every + 2 : 3) * g->nr * ppc;
    return cap;
}

size_t lpic_required_bytes(const lpic_grid_params *g, lpic_precision prec) {
    if (check_params(g, nullptr, nullptr, 0) != LPIC_OK) return 0;
    if (prec != LPIC_FP64 && prec != LPIC_FP32_MIXED) return 0;
    return make_layout(g, prec).total;
}

lpic_status lpic_init_grid(lpic_ctx **out, const lpic_grid_params *g, lpic_precision prec,
                           void *device_buf, size_t buf_bytes, void *cuda_stream) {
    char m[256];
    if (!out) { g_thread_err = "out is NULL"; return LPIC_EINVAL; }
    lpic_status s = check_params(g, nullptr, m, sizeof m);
    if (s != LPIC_OK) { g_thread_err = m; return s; }
    if (prec != LPIC_FP64 && prec != LPIC_FP32_MIXED) { g_thread_err = "bad precision"; return LPIC_EINVAL; }
    if (!device_buf || ((uintptr_t)device_buf & (kAlign - 1))) {
        g_thread_err = "device_buf must be non-NULL and 256-byte aligned";
        return LPIC_EINVAL;
    }
    Layout L = make_layout(g, prec);
    if (buf_bytes < L.total) {
        g_thread_err = "device buffer of " + std::to_string(buf_bytes) + " bytes is smaller than the " +
                       std::to_string(L.total) + " required";
        return LPIC_ENOMEM_BUDGET;
    }
    lpic_ctx *c = new lpic_ctx();
    c->prec = prec;
    c->g = *g;
    c->L = L;
    c->st = (cudaStream_t)cuda_stream;
    c->buf = (char *)device_buf;
    c->bytes = buf_bytes;
    c->geo.nx = g->nx;
    c->geo.nr = g->nr;
    c->geo.P = L.P;
    c->geo.ncol = L.ncol;
    c->geo.nlive = L.nlive;
    c->ph.dx = g->dx;
    c->ph.dr = g->dr;
    c->ph.dt = g->dt;
    c->ph.moving_window = g->moving_window ? 1 : 0;
    c->ph.cap = (int)g->particle_capacity;
    c->ph.track_dq = g->track_continuity ? 1 : 0;
    c->ph.filter_passes = g->filter_passes;
    c->ph.x0 = g->slab_x0;
    c->ph.inject = g->slab_front_interior ? 0 : 1;
    c->d_desc = (Desc *)(c->buf + L.desc);
    c->key = (int *)(c->buf + L.key);
    c->count = (int *)(c->buf + L.count);
    c->blocksum = (int *)(c->buf + L.blocksum);
    c->blockcnt = (int *)(c->buf + L.blockcnt);
    c->icount = (int *)(c->buf + L.icount);
    c->diag = (double *)(c->buf + L.diag);
    c->stage = c->buf + L.stage;
    c->stage_bytes = L.total - L.stage;
    fill_views(c, c->sd);
    fill_views(c, c->sf);
    std::vector<double> tab = row_tables(c->ph, L.P);
    std::vector<float> tabf(tab.begin(), tab.end());
    cudaError_t e = cudaMallocHost((void **)&c->h_desc, sizeof(Desc));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->buf, 0, L.total, c->st);
    if (e == cudaSuccess)
        e = prec == LPIC_FP64
                ? cudaMemcpyAsync(c->buf + L.tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, c->st)
                : cudaMemcpyAsync(c->buf + L.tab, tabf.data(), tabf.size() * 4, cudaMemcpyHostToDevice, c->st);
    // the FP64 factors of the axis rows, after the working-precision tables
    static_assert(kAxisFactors == 2, "axis factors: 1/V_chi,0 and 1/(dt V_0/dx)");
    const double axis[kAxisFactors] = {row_ichi(c->ph, 0), row_ijx(c->ph, 0)};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->buf + L.tab + (size_t)NTAB * L.P * (prec == LPIC_FP64 ? 8 : 4), axis, sizeof axis,
                            cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);   // `axis` lives on this stack frame
    if (e != cudaSuccess) {
        g_thread_err = std::string("lpic_init_grid: ") + cudaGetErrorString(e);
        if (c->h_desc) cudaFreeHost(c->h_desc);
        delete c;
        return LPIC_ECUDA;
    }
    memset(c->h_desc, 0, sizeof(Desc));
    if ((s = push_desc(c)) != LPIC_OK) {
        g_thread_err = c->err;
        cudaFreeHost(c->h_desc);
        delete c;
        return s;
    }
    *out = c;
    return LPIC_OK;
}

lpic_status lpic_init_envelope(lpic_ctx *c, const lpic_laser_params *la) {
    if (!c || !la) return c ? c->fail(LPIC_EINVAL, "laser params are NULL") : LPIC_EINVAL;
    if (!(la->w0 > 0) || !(la->L > 0) || !std::isfinite(la->a0) || !std::isfinite(la->x_center) ||
        !std::isfinite(la->x_focus))
        return c->fail(LPIC_EINVAL, "laser: w0 > 0, L > 0 and finite a0, x_center, x_focus required");
    c->dispatch([&](auto &S) { launch_init_envelope(S, la->a0, la->w0, la->L, la->x_center, la->x_focus, c->st); });
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->cuda_fail(e, "lpic_init_envelope");
    c->envelope_set = true;
    return LPIC_OK;
}

lpic_status lpic_load_plasma(lpic_ctx *c, const lpic_plasma_params *p) {
    if (!c) return LPIC_EINVAL;
    char m[256];
    lpic_status s = check_params(&c->g, p, m, sizeof m);
    if (s != LPIC_OK) return c->fail(s, m);
    if (!p) return c->fail(LPIC_EINVAL, "plasma params are NULL");
    if ((s = pull_desc(c)) != LPIC_OK) return s;
    Phys ph = c->ph;
    ph.have_plasma = 1;
    ph.n0 = p->n0;
    ph.x_start = p->x_start;
    ph.ramp_len = p->ramp_len;
    ph.ppcx = p->ppc_x;
    ph.ppcr = p->ppc_r;
    ph.ppct = p->ppc_theta;
    ph.seed = p->seed;
    ph.inv_ramp = p->ramp_len > 0 ? 1.0 / p->ramp_len : 0.0;
    ph.inv_ppcx = 1.0 / p->ppc_x;
    ph.inv_ppcr = 1.0 / p->ppc_r;
    ph.inv_ppct = 1.0 / p->ppc_theta;
    ph.wfac = 2.0 * kPi * c->ph.dr * c->ph.dx / ((double)p->ppc_x * p->ppc_r * p->ppc_theta);
    std::vector<int> colbase(c->geo.nx + 1, 0);
    long long total = 0;
    for (int i = 0; i < c->geo.nx; i++) {
        colbase[i] = (int)total;
        total += (long long)valid_a_count(ph, c->shift + i) * ph.ppcr * ph.ppct * c->geo.nr;
        if (total > c->g.particle_capacity) break;
    }
    colbase[c->geo.nx] = (int)(total < INT32_MAX ? total : INT32_MAX);
    const long long np0 = c->h_desc->np;
    if (np0 != 0) return c->fail(LPIC_ESTATE, "lpic_load_plasma: particles already loaded");
    const long long headroom = c->g.moving_window
                                   ? (long long)(c->g.sort_every + 2) * ph.ppcx * ph.ppcr * ph.ppct * c->geo.nr
                                   : 0;
    if (total + headroom > c->g.particle_capacity)
        return c->fail(LPIC_EBUFSIZE, "particle_capacity " + std::to_string(c->g.particle_capacity) +
                                          " < " + std::to_string(total + headroom) +
                                          " (window plus injection headroom)");
    if (colbase.size() * sizeof(int) > c->stage_bytes) return c->fail(LPIC_EINVAL, "nx too large for staging");
    c->ph = ph;
    c->sync_views();
    cudaError_t e = cudaMemcpyAsync(c->stage, colbase.data(), colbase.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "lpic_load_plasma");
    c->dispatch([&](auto &S) { launch_load_columns(S, (const int *)c->stage, c->geo.nx, (int)total, c->st); });
    c->h_desc->np = (int)total;
    c->h_desc->n_alive = (int)total;
    if ((s = push_desc(c)) != LPIC_OK) return s;  // synchronises: colbase may go
    e = cudaGetLastError();
    if (e != cudaSuccess) return c->cuda_fail(e, "lpic_load_plasma");
    c->np_upper = total;
    c->since_sort = 0;
    return LPIC_OK;
}

// Record one step (with_sort: followed by the counting sort) as a CUDA graph.  The particle
// kernels are sized for the whole capacity (they read the live count from the device), so the
// graph stays valid while the particle count changes.
// mode 0: one step; 1: one step and the sort; 2: kMultiSteps steps (no sort, no relocation)
lpic_status capture_step(lpic_ctx *c, int mode) {
    static_assert(lpic_ctx::kFamilies == 9, "step_launches is sized for the kernel families");
    long long before[lpic_ctx::kFamilies];
    memcpy(before, c->launches, sizeof before);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return c->cuda_fail(e, "step capture");
    const int npl = (int)c->g.particle_capacity, inj = inj_upper(c);
    c->dispatch([&](auto &S) {
        for (int g = 0; g < (mode == 2 ? lpic_ctx::kMultiSteps : 1); g++) enqueue_step_kernels(c, S, npl, inj, c->st);
        if (mode == 1)
            traced(c, F_SORT, kSortLaunches, c->st, [&] { launch_sort(S, npl, c->key, c->count, c->blocksum, c->st); });
    });
    e = cudaStreamEndCapture(c->st, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_exec[mode], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (int f = 0; f < lpic_ctx::kFamilies; f++) {
        c->step_launches[mode][f] = c->launches[f] - before[f];
        c->launches[f] = before[f];
    }
    return e == cudaSuccess ? LPIC_OK : c->cuda_fail(e, "step graph");
}

lpic_status lpic_step(lpic_ctx *c, int nsteps) {
    if (!c) return LPIC_EINVAL;
    if (nsteps < 0) return c->fail(LPIC_EINVAL, "nsteps < 0");
    lpic_status s = deferred_errors(c);
    if (s != LPIC_OK) return s;
    for (int k = 0; k < nsteps; k++) {
        // kMultiSteps steps in one replay when none of them sorts or relocates (the window
        // slides the offset by at most one column a step)
        const int G = lpic_ctx::kMultiSteps;
        if (!c->timing && nsteps - k >= G && c->since_sort + G < c->g.sort_every &&
            (!c->g.moving_window || c->off + G + c->geo.nlive + 1 <= c->geo.ncol)) {
            for (int g = 0; g < G; g++) (void)advance_mirror(c);   // no sort: since_sort stays below
            if (!c->step_exec[2] && (s = capture_step(c, 2)) != LPIC_OK) return s;
            cudaError_t e = cudaGraphLaunch(c->step_exec[2], c->st);
            if (e != cudaSuccess) return c->cuda_fail(e, "lpic_step");
            for (int f = 0; f < lpic_ctx::kFamilies; f++) c->launches[f] += c->step_launches[2][f];
            k += G - 1;
            continue;
        }
        pre_step(c, c->st);
        if (c->timing) {   // kernel by kernel, bracketed with events
            const int npl = launch_cap(c), inj = inj_upper(c);
            c->dispatch([&](auto &S) { enqueue_step_kernels(c, S, npl, inj, c->st); });
            post_step(c, c->st);
            continue;
        }
        const int sort = advance_mirror(c) ? 1 : 0;   // host mirrors of this step; sort after it?
        if (!c->step_exec[sort] && (s = capture_step(c, sort)) != LPIC_OK) return s;
        cudaError_t e = cudaGraphLaunch(c->step_exec[sort], c->st);
        if (e != cudaSuccess) return c->cuda_fail(e, "lpic_step");
        for (int f = 0; f < lpic_ctx::kFamilies; f++) c->launches[f] += c->step_launches[sort][f];
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->cuda_fail(e, "lpic_step");
    record_status_copy(c);
    return LPIC_OK;
}

lpic_status lpic_diagnose_async(lpic_ctx *c, lpic_diag_kind kind, void *host_out, size_t cap) {
    if (!c) return LPIC_EINVAL;
    if (kind != LPIC_DIAG_EX_AXIS || !host_out)
        return c->fail(LPIC_EINVAL, "lpic_diagnose_async: LPIC_DIAG_EX_AXIS into a non-NULL buffer only");
    const size_t n = (size_t)c->geo.nx * sizeof(double);
    if (cap < n) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
    // Page-locked host memory the device can address: the kernel writes the wake into it
    // directly (no copy on the stream between two steps).  Else through the staging area,
    // which is reused only by later work on the same stream, after this copy.
    cudaPointerAttributes pa{};
    void *mapped = nullptr;
    if (cudaPointerGetAttributes(&pa, host_out) == cudaSuccess) {
        if (pa.type == cudaMemoryTypeHost && pa.devicePointer && (uintptr_t)pa.devicePointer % 8 == 0)
            mapped = pa.devicePointer;
    } else {
        (void)cudaGetLastError();   // not a CUDA-known pointer: pageable memory
    }
    cudaError_t e = cudaSuccess;
    if (mapped) {
        c->dispatch([&](auto &S) { launch_diag_ex_axis(S, (double *)mapped, c->st); });
    } else {
        c->dispatch([&](auto &S) { launch_diag_ex_axis(S, (double *)c->stage, c->st); });
        e = cudaMemcpyAsync(host_out, c->stage, n, cudaMemcpyDeviceToHost, c->st);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? LPIC_OK : c->cuda_fail(e, "lpic_diagnose_async");
}

lpic_status lpic_diagnose(lpic_ctx *c, lpic_diag_kind kind, void *host_out, size_t cap,
                          size_t *written) {
    if (!c) return LPIC_EINVAL;
    if (written) *written = 0;
    lpic_status s = pull_desc(c);
    if (s != LPIC_OK) return s;
    c->ev_pending = false;
    if ((s = device_errors(c, *c->h_desc)) != LPIC_OK) return s;
    const Desc d = *c->h_desc;
    const int nx = c->geo.nx, nr = c->geo.nr;
    auto need = [&](size_t n) -> bool {
        if (written) *written = n;
        return cap >= n && (n == 0 || host_out);
    };
    auto copy_back = [&](void *dst, const void *src, size_t n) -> lpic_status {
        cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e == cudaSuccess) e = cudaGetLastError();
        return e == cudaSuccess ? LPIC_OK : c->cuda_fail(e, "lpic_diagnose");
    };
    switch (kind) {
    case LPIC_DIAG_EX_AXIS: {
        if (!need(nx * sizeof(double))) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        c->dispatch([&](auto &S) { launch_diag_ex_axis(S, (double *)c->stage, c->st); });
        return copy_back(host_out, c->stage, nx * sizeof(double));
    }
    case LPIC_DIAG_A_ABS_MAX:
    case LPIC_DIAG_WAIST: {
        if (!need(sizeof(double))) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        double h[3];
        c->dispatch([&](auto &S) { launch_diag_amax_waist(S, c->diag, c->st); });
        if ((s = copy_back(h, c->diag, sizeof h)) != LPIC_OK) return s;
        double v = kind == LPIC_DIAG_A_ABS_MAX ? h[0] : (h[2] > 0 ? std::sqrt(2.0 * h[1] / h[2]) : 0.0);
        memcpy(host_out, &v, sizeof v);
        return std::isfinite(v) ? LPIC_OK : c->fail(LPIC_ENONFINITE, "non-finite envelope");
    }
    case LPIC_DIAG_CONT_RESIDUAL: {
        if (!need(sizeof(double))) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        if (!c->ph.track_dq) return c->fail(LPIC_ESTATE, "track_continuity is off");
        double h[2];
        c->dispatch([&](auto &S) { launch_diag_cont(S, c->diag, c->st); });
        if ((s = copy_back(h, c->diag, sizeof h)) != LPIC_OK) return s;
        double v = h[1] > 0 ? h[0] / h[1] : 0.0;
        memcpy(host_out, &v, sizeof v);
        return std::isfinite(v) ? LPIC_OK : c->fail(LPIC_ENONFINITE, "non-finite current");
    }
    case LPIC_DIAG_ACCEL_ENERGY: {
        if (!need(4 * sizeof(double))) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        double h[4];
        const double thr = c->g.accel_px_min > 0 ? c->g.accel_px_min : 10.0;
        c->dispatch([&](auto &S) { launch_diag_accel(S, launch_cap(c), thr, c->diag, c->st); });
        if ((s = copy_back(h, c->diag, sizeof h)) != LPIC_OK) return s;
        double o[4] = {h[0], h[1], 0.0, 0.0};
        if (h[1] > 0) {
            o[2] = h[2] / h[1];
            o[3] = std::sqrt(std::fmax(h[3] / h[1] - o[2] * o[2], 0.0));
        }
        memcpy(host_out, o, sizeof o);
        return LPIC_OK;
    }
    case LPIC_DIAG_BEAM: {
        if (!need(12 * sizeof(double))) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        const double thr = c->g.accel_px_min > 0 ? c->g.accel_px_min : 10.0;
        const int npl = launch_cap(c), nb = kBeamBins;
        double o[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, (double)nb};
        double mx[2];
        c->dispatch([&](auto &S) { launch_beam_max(S, npl, thr, c->diag, c->st); });
        if ((s = copy_back(mx, c->diag, sizeof mx)) != LPIC_OK) return s;
        o[0] = mx[1];
        o[10] = mx[0];
        if (mx[1] > 0) {
            // spectrum, its peak and half-maximum crossings (host side: nb values)
            const double width = mx[0] > 0 ? mx[0] / nb : 1.0;
            std::vector<double> hist(nb);
            c->dispatch([&](auto &S) { launch_beam_hist(S, npl, thr, width, nb, (double *)c->stage, c->st); });
            if ((s = copy_back(hist.data(), c->stage, nb * sizeof(double))) != LPIC_OK) return s;
            int kp = 0;
            for (int b = 1; b < nb; b++)
                if (hist[b] > hist[kp]) kp = b;
            const double half = 0.5 * hist[kp];
            auto crossing = [&](int step) {
                int b = kp;
                while (b + step >= 0 && b + step < nb && hist[b + step] >= half) b += step;
                const int nx_ = b + step;
                const double hn = (nx_ >= 0 && nx_ < nb) ? hist[nx_] : 0.0;
                const double t = hist[b] != hn ? (hist[b] - half) / (hist[b] - hn) : 0.0;
                return (b + 0.5) * width + step * t * width;
            };
            const double e_peak = (kp + 0.5) * width, fwhm = crossing(1) - crossing(-1);
            o[3] = e_peak;
            o[4] = fwhm;
            double m[14];
            c->dispatch([&](auto &S) { launch_beam_moments(S, npl, thr, e_peak, fwhm, c->diag, c->st); });
            if ((s = copy_back(m, c->diag, sizeof m)) != LPIC_OK) return s;
            o[1] = m[13];
            o[2] = m[0];
            if (m[0] > 0) {
                const double q = m[0], em = m[1] / q;
                o[9] = em;
                o[5] = std::sqrt(std::fmax(m[2] / q - em * em, 0.0)) / e_peak;
                for (int u = 0; u < 2; u++) {
                    const double *a = m + 3 + 5 * u;
                    const double mu = a[0] / q, mp = a[2] / q;
                    const double suu = a[1] / q - mu * mu, spp = a[3] / q - mp * mp, sup = a[4] / q - mu * mp;
                    o[6 + u] = std::sqrt(std::fmax(suu * spp - sup * sup, 0.0));
                }
                o[8] = 0.5 * (o[6] + o[7]);
            }
        }
        memcpy(host_out, o, sizeof o);
        return LPIC_OK;
    }
    case LPIC_DIAG_COUNTERS: {
        if (!need(4 * sizeof(int64_t))) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        c->dispatch([&](auto &S) { launch_alive_index(S, launch_cap(c), c->key, c->blockcnt, c->icount, c->st); });
        int alive = 0;
        if ((s = copy_back(&alive, c->icount, sizeof alive)) != LPIC_OK) return s;
        int64_t o[4] = {d.step, d.shift, d.np, alive};
        memcpy(host_out, o, sizeof o);
        return LPIC_OK;
    }
    case LPIC_DIAG_EX: case LPIC_DIAG_ER: case LPIC_DIAG_BT: case LPIC_DIAG_A: case LPIC_DIAG_AM:
    case LPIC_DIAG_CHI: case LPIC_DIAG_JX: case LPIC_DIAG_JR: case LPIC_DIAG_DQ: {
        int ni, nj, cp = 0;
        switch (kind) {
        case LPIC_DIAG_EX: case LPIC_DIAG_JX: ni = nx; nj = nr + 1; break;
        case LPIC_DIAG_ER: case LPIC_DIAG_JR: ni = nx + 1; nj = nr; break;
        case LPIC_DIAG_BT: ni = nx; nj = nr; break;
        case LPIC_DIAG_A: case LPIC_DIAG_AM: ni = nx + 1; nj = nr + 1; cp = 1; break;
        default: ni = nx + 1; nj = nr + 1; break;
        }
        const size_t colb = (size_t)nj * sizeof(double) * (cp ? 2 : 1);
        if (!need(colb * ni)) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        const int per = (int)(c->stage_bytes / colb);
        for (int c0 = 0; c0 < ni; c0 += per) {
            const int c1 = c0 + per < ni ? c0 + per : ni;
            c->dispatch([&](auto &S) { launch_dump_field(S, (int)kind, c0, c1, (double *)c->stage, c->st); });
            if ((s = copy_back((char *)host_out + colb * c0, c->stage, colb * (c1 - c0))) != LPIC_OK) return s;
        }
        return LPIC_OK;
    }
    case LPIC_DIAG_PARTICLES:
    case LPIC_DIAG_PARTICLE_IDS: {
        c->dispatch([&](auto &S) { launch_alive_index(S, launch_cap(c), c->key, c->blockcnt, c->icount, c->st); });
        int n = 0;
        if ((s = copy_back(&n, c->icount, sizeof n)) != LPIC_OK) return s;
        const size_t per_p = kind == LPIC_DIAG_PARTICLES ? 7 * sizeof(double) : sizeof(uint64_t);
        if (!need(per_p * n)) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        const int chunk = (int)(c->stage_bytes / 8);
        if (kind == LPIC_DIAG_PARTICLE_IDS) {
            for (int k0 = 0; k0 < n; k0 += chunk) {
                const int k1 = k0 + chunk < n ? k0 + chunk : n;
                c->dispatch([&](auto &S) { launch_set_ids(S, c->key, k0, k1, nullptr, (uint64_t *)c->stage, 0, c->st); });
                if ((s = copy_back((uint64_t *)host_out + k0, c->stage, 8 * (size_t)(k1 - k0))) != LPIC_OK) return s;
            }
            return LPIC_OK;
        }
        for (int comp = 0; comp < 7; comp++)
            for (int k0 = 0; k0 < n; k0 += chunk) {
                const int k1 = k0 + chunk < n ? k0 + chunk : n;
                c->dispatch([&](auto &S) { launch_dump_particles(S, c->key, k0, k1, comp, (double *)c->stage, c->st); });
                if ((s = copy_back((double *)host_out + (size_t)comp * n + k0, c->stage, 8 * (size_t)(k1 - k0))) != LPIC_OK)
                    return s;
            }
        return LPIC_OK;
    }
    case LPIC_DIAG_PARTICLES_NATIVE: {
        c->dispatch([&](auto &S) { launch_alive_index(S, launch_cap(c), c->key, c->blockcnt, c->icount, c->st); });
        int n = 0;
        if ((s = copy_back(&n, c->icount, sizeof n)) != LPIC_OK) return s;
        const size_t es = c->prec == LPIC_FP64 ? 8 : 4;
        if (!need((12 + 7 * es) * (size_t)n)) return c->fail(LPIC_EBUFSIZE, "output buffer too small");
        const int chunk = (int)(c->stage_bytes / 8);
        size_t at = 0;
        for (int comp = 0; comp < 9; comp++) {
            const size_t esz = comp == 0 ? 8 : comp == 8 ? 4 : es;
            for (int k0 = 0; k0 < n; k0 += chunk) {
                const int k1 = k0 + chunk < n ? k0 + chunk : n;
                c->dispatch([&](auto &S) { launch_native_particles(S, c->key, k0, k1, comp, c->stage, 0, c->st); });
                if ((s = copy_back((char *)host_out + at + esz * k0, c->stage, esz * (size_t)(k1 - k0))) != LPIC_OK)
                    return s;
            }
            at += esz * (size_t)n;
        }
        return LPIC_OK;
    }
    }
    return c->fail(LPIC_EINVAL, "unknown diagnostic kind");
}

lpic_status lpic_upload(lpic_ctx *c, lpic_diag_kind kind, const void *host_in, size_t bytes) {
    if (!c) return LPIC_EINVAL;
    if (!host_in && bytes) return c->fail(LPIC_EINVAL, "host_in is NULL");
    lpic_status s = pull_desc(c);
    if (s != LPIC_OK) return s;
    const int nx = c->geo.nx, nr = c->geo.nr;
    auto h2d = [&](void *dst, const void *src, size_t n) -> lpic_status {
        cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->st);
        return e == cudaSuccess ? LPIC_OK : c->cuda_fail(e, "lpic_upload");
    };
    auto finish = [&]() -> lpic_status {
        cudaError_t e = cudaStreamSynchronize(c->st);
        if (e == cudaSuccess) e = cudaGetLastError();
        return e == cudaSuccess ? LPIC_OK : c->cuda_fail(e, "lpic_upload");
    };
    // Page-locked host memory the device can address (cudaHostAlloc / cudaHostRegister with
    // unified addressing): the conversion kernels read it in place over the host link, in one
    // pass, instead of through the staging area chunk by chunk.  Only 8-byte aligned buffers:
    // the kernels read doubles and 64-bit ids from it.
    const void *mapped = nullptr;
    if (host_in) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, host_in) == cudaSuccess) {
            if (pa.type == cudaMemoryTypeHost && pa.devicePointer && (uintptr_t)pa.devicePointer % 8 == 0)
                mapped = pa.devicePointer;
        } else {
            (void)cudaGetLastError();   // not a CUDA-known pointer: pageable memory
        }
    }
    switch (kind) {
    case LPIC_DIAG_COUNTERS: {
        if (bytes != 4 * sizeof(int64_t)) return c->fail(LPIC_EINVAL, "counters: 4 int64 expected");
        int64_t v[4];
        memcpy(v, host_in, sizeof v);
        if (v[0] < 0 || v[1] < 0) return c->fail(LPIC_EINVAL, "counters must be >= 0");
        c->h_desc->step = v[0];
        c->h_desc->shift = v[1];
        if ((s = push_desc(c)) != LPIC_OK) return s;
        c->step = v[0];
        c->shift = v[1];
        return LPIC_OK;
    }
    case LPIC_DIAG_EX: case LPIC_DIAG_ER: case LPIC_DIAG_BT: case LPIC_DIAG_A: case LPIC_DIAG_AM: {
        int ni, nj, cp = 0;
        switch (kind) {
        case LPIC_DIAG_EX: ni = nx; nj = nr + 1; break;
        case LPIC_DIAG_ER: ni = nx + 1; nj = nr; break;
        case LPIC_DIAG_BT: ni = nx; nj = nr; break;
        default: ni = nx + 1; nj = nr + 1; cp = 1; break;
        }
        const size_t colb = (size_t)nj * sizeof(double) * (cp ? 2 : 1);
        if (bytes != colb * ni) return c->fail(LPIC_EINVAL, "upload: wrong size for this array");
        if (mapped) {
            c->dispatch([&](auto &S) { launch_upload_field(S, (int)kind, 0, ni, (const double *)mapped, c->st); });
            return finish();
        }
        const int per = (int)(c->stage_bytes / colb);
        for (int c0 = 0; c0 < ni; c0 += per) {
            const int c1 = c0 + per < ni ? c0 + per : ni;
            if ((s = h2d(c->stage, (const char *)host_in + colb * c0, colb * (c1 - c0))) != LPIC_OK) return s;
            c->dispatch([&](auto &S) { launch_upload_field(S, (int)kind, c0, c1, (const double *)c->stage, c->st); });
        }
        return finish();
    }
    case LPIC_DIAG_PARTICLES: {
        if (bytes % (7 * sizeof(double))) return c->fail(LPIC_EINVAL, "particles: 7n doubles expected");
        const long long n = (long long)(bytes / (7 * sizeof(double)));
        if (n > c->g.particle_capacity) return c->fail(LPIC_EBUFSIZE, "more particles than capacity");
        const int chunk = mapped ? (int)(n > 0 ? n : 1) : (int)(c->stage_bytes / 8);
        for (int comp = 0; comp < 7; comp++)
            for (long long k0 = 0; k0 < n; k0 += chunk) {
                if (mapped) {
                    c->dispatch([&](auto &S) {
                        launch_upload_particles(S, 0, (int)n, comp, (const double *)mapped + comp * n, c->st);
                    });
                    continue;
                }
                const long long k1 = k0 + chunk < n ? k0 + chunk : n;
                if ((s = h2d(c->stage, (const double *)host_in + comp * n + k0, 8 * (size_t)(k1 - k0))) != LPIC_OK)
                    return s;
                c->dispatch([&](auto &S) { launch_upload_particles(S, (int)k0, (int)k1, comp, (const double *)c->stage, c->st); });
            }
        c->dispatch([&](auto &S) { launch_finish_upload(S, (int)n, c->st); });
        c->np_upper = n;
        c->since_sort = 0;
        return finish();
    }
    case LPIC_DIAG_PARTICLES_NATIVE: {
        const size_t es = c->prec == LPIC_FP64 ? 8 : 4, per = 12 + 7 * es;
        if (bytes % per) return c->fail(LPIC_EINVAL, "native particles: 12 + 7 x element bytes per electron expected");
        const long long n = (long long)(bytes / per);
        if (n > c->g.particle_capacity) return c->fail(LPIC_EBUFSIZE, "more particles than capacity");
        // the blocks are the particle arrays themselves: plain copies into slots [0, n) of the
        // current buffer (the copy engines move them; no conversion kernel)
        const int pb = c->h_desc->pbuf;
        c->dispatch([&](auto &S) {
            const auto &P = S.p[pb ? 1 : 0];
            void *const dst[9] = {P.id, P.ox, P.y, P.z, P.px, P.py, P.pz, P.w, P.ix};
            size_t at = 0;
            for (int comp = 0; comp < 9 && s == LPIC_OK; comp++) {
                const size_t b = (comp == 0 ? 8 : comp == 8 ? 4 : es) * (size_t)n;
                if (b) s = h2d(dst[comp], (const char *)host_in + at, b);
                at += b;
            }
        });
        if (s != LPIC_OK) return s;
        c->dispatch([&](auto &S) { launch_finish_upload(S, (int)n, c->st); });
        c->np_upper = n;
        c->since_sort = 0;
        return finish();
    }
    case LPIC_DIAG_PARTICLE_IDS: {
        const long long n = (long long)(bytes / sizeof(uint64_t));
        if (bytes % 8 || n != c->h_desc->np)
            return c->fail(LPIC_EINVAL, "ids: one uint64 per particle slot expected");
        if (mapped) {
            c->dispatch([&](auto &S) {
                launch_set_ids(S, nullptr, 0, (int)n, (const uint64_t *)mapped, nullptr, 1, c->st);
            });
            return finish();
        }
        const int chunk = (int)(c->stage_bytes / 8);
        for (long long k0 = 0; k0 < n; k0 += chunk) {
            const long long k1 = k0 + chunk < n ? k0 + chunk : n;
            if ((s = h2d(c->stage, (const uint64_t *)host_in + k0, 8 * (size_t)(k1 - k0))) != LPIC_OK) return s;
            c->dispatch([&](auto &S) { launch_set_ids(S, nullptr, (int)k0, (int)k1, (const uint64_t *)c->stage, nullptr, 1, c->st); });
        }
        return finish();
    }
    default:
        return c->fail(LPIC_EINVAL, "this kind cannot be uploaded");
    }
}

lpic_status lpic_slab_exchange(lpic_ctx *l, lpic_ctx *r, int32_t halo) {
    if (!l || !r || l == r) return l ? l->fail(LPIC_EINVAL, "slab exchange: two distinct contexts needed") : LPIC_EINVAL;
    auto bad = [&](const char *m) { r->fail(LPIC_EINVAL, m); return l->fail(LPIC_EINVAL, m); };
    if (l->prec != r->prec || l->geo.nr != r->geo.nr || l->geo.P != r->geo.P || l->ph.dx != r->ph.dx ||
        l->ph.dr != r->ph.dr || l->ph.dt != r->ph.dt || l->ph.moving_window != r->ph.moving_window)
        return bad("slab exchange: precision, nr, dx, dr, dt and the window rule must match");
    if (l->st != r->st) return bad("slab exchange: both contexts must use the same stream");
    if (halo < 1 || l->geo.nx < 2 * halo || r->geo.nx < 2 * halo)
        return bad("slab exchange: halo >= 1 and each slab at least 2*halo columns wide");
    const long long B = (long long)r->ph.x0 + halo;
    if (B != (long long)l->ph.x0 + l->geo.nx - halo) return bad("slab exchange: slab_x0/nx do not meet at B");
    if (l->step != r->step || l->shift - l->ph.x0 != r->shift - r->ph.x0)
        return bad("slab exchange: the slabs are not at the same step and window shift");
    lpic_status s = deferred_errors(l);
    if (s == LPIC_OK) s = deferred_errors(r);
    if (s != LPIC_OK) return s;
    const int B_L = (int)(B - l->ph.x0);
    // the freed-slot lists live in each side's staging area (free between calls)
    const size_t fb = l->stage_bytes < r->stage_bytes ? l->stage_bytes : r->stage_bytes;
    const int fcap = (int)(fb / sizeof(int) < (size_t)(1 << 30) ? fb / sizeof(int) : (size_t)(1 << 30));
    if (l->prec == LPIC_FP64)
        launch_slab_exchange<double>(l->sd, r->sd, B_L, halo, (int *)l->stage, (int *)r->stage, fcap, l->st);
    else
        launch_slab_exchange<float>(l->sf, r->sf, B_L, halo, (int *)l->stage, (int *)r->stage, fcap, l->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return l->cuda_fail(e, "lpic_slab_exchange");
    // appended electrons: the launch bounds and the next sort cover every slot
    l->np_upper = l->g.particle_capacity;
    r->np_upper = r->g.particle_capacity;
    record_status_copy(l);
    record_status_copy(r);
    return LPIC_OK;
}

size_t lpic_bunch_scratch_bytes(const lpic_ctx *c) { return c ? bunch_scratch_bytes(c->geo) : 0; }

lpic_status lpic_inject_bunch(lpic_ctx *c, const double *host_parts, int64_t n, double gamma, void *scratch,
                              size_t scratch_bytes) {
    if (!c) return LPIC_EINVAL;
    if (!(gamma > 1.0) || !std::isfinite(gamma)) return c->fail(LPIC_EINVAL, "inject_bunch: gamma must be > 1");
    if (n < 0 || (n > 0 && !host_parts)) return c->fail(LPIC_EINVAL, "inject_bunch: bad particle array");
    if (!scratch || ((uintptr_t)scratch % 256) != 0 || scratch_bytes < bunch_scratch_bytes(c->geo))
        return c->fail(LPIC_EINVAL, "inject_bunch: scratch must be 256-byte aligned and hold lpic_bunch_scratch_bytes");
    for (int64_t k = 0; k < 7 * n; k++)
        if (!std::isfinite(host_parts[k])) return c->fail(LPIC_EINVAL, "inject_bunch: non-finite particle value");
    {   // every electron inside the window: x in [s dx, (s + Nx) dx), r < r_max
        const double x0 = c->shift * c->ph.dx, x1 = (c->shift + c->geo.nx) * c->ph.dx, rmax = c->geo.nr * c->ph.dr;
        for (int64_t k = 0; k < n; k++) {
            const double x = host_parts[k], y = host_parts[n + k], z = host_parts[2 * n + k];
            if (!(x >= x0 && x < x1) || !(std::sqrt(y * y + z * z) < rmax))
                return c->fail(LPIC_EINVAL, "inject_bunch: an electron lies outside the window");
        }
    }
    lpic_status s = pull_desc(c);
    if (s != LPIC_OK) return s;
    const long long np0 = c->h_desc->np;
    if (np0 + n > c->g.particle_capacity) return c->fail(LPIC_EBUFSIZE, "inject_bunch: particle capacity exceeded");
    auto h2d = [&](void *dst, const void *src, size_t bytes) -> lpic_status {
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);   // the stage is reused next
        return e == cudaSuccess ? LPIC_OK : c->cuda_fail(e, "inject_bunch");
    };
    // append the particles at slots [np0, np0 + n)
    const int chunk = (int)(c->stage_bytes / 8);
    for (int comp = 0; comp < 7; comp++)
        for (long long k0 = 0; k0 < n; k0 += chunk) {
            const long long k1 = k0 + chunk < n ? k0 + chunk : n;
            if ((s = h2d(c->stage, host_parts + comp * n + k0, 8 * (size_t)(k1 - k0))) != LPIC_OK) return s;
            c->dispatch([&](auto &S) { launch_upload_particles(S, (int)(np0 + k0), (int)(np0 + k1), comp, (const double *)c->stage, c->st); });
        }
    std::vector<uint64_t> ids;
    for (long long k0 = 0; k0 < n; k0 += chunk) {
        const long long k1 = k0 + chunk < n ? k0 + chunk : n;
        ids.resize(k1 - k0);
        for (long long t = k0; t < k1; t++) ids[t - k0] = (1ull << 63) + c->bunch_ids + (unsigned long long)t;
        if ((s = h2d(c->stage, ids.data(), 8 * ids.size())) != LPIC_OK) return s;
        c->dispatch([&](auto &S) { launch_set_ids(S, nullptr, (int)(np0 + k0), (int)(np0 + k1), (const uint64_t *)c->stage, nullptr, 1, c->st); });
    }
    c->bunch_ids += (unsigned long long)n;
    c->h_desc->np = (int)(np0 + n);
    c->h_desc->n_alive += (int)n;
    if ((s = push_desc(c)) != LPIC_OK) return s;
    c->np_upper = np0 + n > c->np_upper ? np0 + n : c->np_upper;
    // fields of the bunch
    int iters = 0;
    double res = 0.0;
    c->dispatch([&](auto &S) {
        iters = bunch_solve_and_add(S, (int)np0, (int)n, gamma, scratch, c->diag, 1e-12, 2000, c->st, &res);
    });
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return c->cuda_fail(e, "inject_bunch");
    if (!(res <= 1e-12) || !std::isfinite(res)) return c->fail(LPIC_ENONFINITE, "inject_bunch: the field solve did not converge");
    (void)iters;
    return LPIC_OK;
}

lpic_status lpic_set_kernel_timing(lpic_ctx *c, int enable) {
    if (!c) return LPIC_EINVAL;
    c->timing = enable != 0;
    return LPIC_OK;
}

lpic_status lpic_kernel_stats(lpic_ctx *c, int64_t *launches, double *ms, int cap, int *n) {
    if (!c) return LPIC_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return c->cuda_fail(e, "lpic_kernel_stats");
    for (auto &sp : c->spans) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, sp.a, sp.b) == cudaSuccess) c->ms[sp.fam] += t;
        c->ev_pool.push_back(sp.a);
        c->ev_pool.push_back(sp.b);
    }
    c->spans.clear();
    const int m = cap < lpic_ctx::kFamilies ? cap : lpic_ctx::kFamilies;
    for (int k = 0; k < m; k++) {
        if (launches) launches[k] = c->launches[k];
        if (ms) ms[k] = c->ms[k];
        c->ms[k] = 0.0;
    }
    if (n) *n = lpic_ctx::kFamilies;
    return LPIC_OK;
}

const char *lpic_kernel_name(int k) {
    return (k >= 0 && k < lpic_ctx::kFamilies) ? kFamilyNames[k] : nullptr;
}

lpic_status lpic_destroy(lpic_ctx *c) {
    if (!c) return LPIC_EINVAL;
    cudaStreamSynchronize(c->st);
    c->drop_step_graphs();
    for (auto &sp : c->spans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->h_desc) cudaFreeHost(c->h_desc);
    delete c;
    return LPIC_OK;
}

const char *lpic_last_error(const lpic_ctx *c) {
    if (c) return c->err.c_str();
    return g_thread_err.c_str();
}

}  // extern "C"

// ============================================================================ batched form
//
// One step of a batch is a fixed sequence of fused launches (prepass, pass A, envelope,
// pass B, Ampere, window), each a persistent grid walking a work list of items
// {simulation, tile or virtual block, ...} over the active simulations.  The simulations'
// views travel in the launches' parameter space, up to kPackMax per launch; larger batches
// are split into packs of near-equal size whose launch sequences run as parallel branches.
// The device buffer the caller provides holds the work lists.  The sequence is recorded in a
// CUDA graph once per active set and replayed every step; relocation of a slid-out window
// and the periodic sort stay per simulation, enqueued on the batch stream between replays,
// because the host decides when they are due.

namespace {
// work lists: prepass, pass A (and the sort's count and scatter), envelope, pass B, pass B
// (dq), ampere, window, sort counter blocks, one item per simulation, current filter
constexpr int kBatchLists = 10;
enum { BL_PREPASS, BL_SLOTS, BL_ENVELOPE, BL_PASSB, BL_PASSB_DQ, BL_AMPERE, BL_WINDOW, BL_SORTBLK, BL_SIMS, BL_FILTER };
constexpr int kDefaultChunk = 4096, kMinChunk = 1024, kMaxChunk = 1 << 20;

int window_work(const lpic_ctx *c) {
    int work = (2 * kG + 1) * c->geo.P;
    const int inj = c->ph.have_plasma ? c->ph.ppcx * c->ph.ppcr * c->ph.ppct * c->geo.nr : 0;
    return inj > work ? inj : work;
}

int pack_count(int n) { return (n + kPackMax - 1) / kPackMax; }
// Head of the batch buffer: n sort flags, then three item tickets per pack (pass A, pass B,
// pass B with the charge change; at most n packs).
constexpr int kTicketsPerPack = 3;
size_t flags_bytes(int n) { return ((size_t)n * (1 + kTicketsPerPack) * sizeof(int) + 255) / 256 * 256; }

// Upper bound of the work items over all lists with every simulation active.
size_t batch_items_bound(lpic_ctx *const *ctxs, int n) {
    size_t items = 0;
    for (int k = 0; k < n; k++) {
        int tx, ty;
        for (int ph = 0; ph < 3; ph++) {
            grid_tiles(ctxs[k]->geo, ph, tx, ty);
            items += (size_t)tx * ty;
        }
        items += (size_t)window_parts(ctxs[k]->geo, window_work(ctxs[k]));
        items += 2 * (size_t)((ctxs[k]->g.particle_capacity + kMinChunk - 1) / kMinChunk);
        items += (size_t)sort_blocks(ctxs[k]->geo) + 1;
        if (ctxs[k]->ph.filter_passes > 0) {
            int tx, ty;
            grid_tiles(ctxs[k]->geo, 3, tx, ty);
            items += 3 * (size_t)tx * ty;
        }
    }
    return items;
}
}  // namespace

struct lpic_batch {
    std::vector<lpic_ctx *> ctx;
    lpic_precision prec = LPIC_FP64;
    cudaStream_t st = nullptr;
    int *due = nullptr;                     // caller's device buffer: sort flags, tickets, items
    int *tickets = nullptr;
    int4 *items = nullptr;
    size_t items_cap = 0;
    cudaEvent_t ev = nullptr;
    std::vector<cudaStream_t> aux;          // branches of packs 1.. in the graph
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // one step; one step and the sorts
    std::vector<char> active_key;
    std::vector<int> order;                 // context index of each flag (pack order)
    int chunk = kDefaultChunk;              // particle slots per work item
    int packs = 0;                          // packs requested (0: as few as the views allow)
    int per_replay[2] = {0, 0};             // kernels per graph replay
    long long launches = 0;                 // kernels enqueued by the batch (fused + relocation)
    std::string err;
};

namespace {
void drop_graphs(lpic_batch *b) {
    for (auto &e : b->exec)
        if (e) { cudaGraphExecDestroy(e); e = nullptr; }
}

void batch_release(lpic_batch *b) {
    drop_graphs(b);
    if (b->ev) cudaEventDestroy(b->ev);
    for (auto s : b->aux) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
}

template <class R> SimDev<R> &view_of(lpic_ctx *c);
template <> SimDev<double> &view_of<double>(lpic_ctx *c) { return c->sd; }
template <> SimDev<float> &view_of<float>(lpic_ctx *c) { return c->sf; }

// Work lists of one pack (sims: context indices of its simulations, pack slot = position).
// Particle lists cut each simulation's slots [0, capacity) into items of b->chunk slots;
// items are interleaved across simulations (all first items, then all second items, ...)
// so that the items past a simulation's live slots, which end at once, spread over the
// blocks instead of piling onto a few.
void plan_pack(const lpic_batch *b, const std::vector<int> &sims, std::vector<int4> L[kBatchLists]) {
    const int nact = (int)sims.size();
    int most = 0;
    for (int slot = 0; slot < nact; slot++) {
        const lpic_ctx *c = b->ctx[sims[slot]];
        const int grid_list[3] = {BL_PREPASS, BL_ENVELOPE, BL_AMPERE};
        for (int ph = 0; ph < 3; ph++) {
            int tx, ty;
            grid_tiles(c->geo, ph, tx, ty);
            for (int by = 0; by < ty; by++)
                for (int bx = 0; bx < tx; bx++)
                    L[grid_list[ph]].push_back(make_int4(slot, bx, by, ph == 1 && bx == tx - 1 ? 1 : 0));
        }
        if (c->ph.filter_passes > 0) {
            int tx, ty;
            grid_tiles(c->geo, 3, tx, ty);
            for (int a = 0; a < (c->ph.track_dq ? 3 : 2); a++)   // Jx, Jr, dQ
                for (int by = 0; by < ty; by++)
                    for (int bx = 0; bx < tx; bx++) L[BL_FILTER].push_back(make_int4(slot, bx, by, a));
        }
        const int parts = window_parts(c->geo, window_work(c));
        for (int v = 0; v < parts; v++) L[BL_WINDOW].push_back(make_int4(slot, v, parts, 0));
        const int nb = sort_blocks(c->geo);
        for (int v = 0; v < nb; v++) L[BL_SORTBLK].push_back(make_int4(slot, v, 0, 0));
        L[BL_SIMS].push_back(make_int4(slot, 0, 0, 0));
        const long long ni = (c->g.particle_capacity + b->chunk - 1) / b->chunk;
        if (ni > most) most = (int)ni;
    }
    for (int v = 0; v < most; v++)
        for (int slot = 0; slot < nact; slot++) {
            const lpic_ctx *c = b->ctx[sims[slot]];
            if ((long long)v * b->chunk >= c->g.particle_capacity) continue;
            const int4 it = make_int4(slot, v, 0, b->chunk);
            L[BL_SLOTS].push_back(it);
            L[c->ph.track_dq ? BL_PASSB_DQ : BL_PASSB].push_back(it);
        }
}

// Upload the work lists, then record one step of the active set, without and with the
// sorts (the sort launches act on the simulations whose flag is set before the replay).
template <class R> lpic_status batch_capture(lpic_batch *b, const std::vector<char> &active) {
    drop_graphs(b);
    std::vector<int> act;
    for (size_t k = 0; k < b->ctx.size(); k++)
        if (active[k]) act.push_back((int)k);
    int npk = pack_count((int)act.size());
    if (b->packs > npk) npk = b->packs < (int)act.size() ? b->packs : (int)act.size();
    if (npk < 1) npk = 1;
    // packs of near-equal size
    std::vector<std::vector<int>> packs(npk);
    for (size_t q = 0; q < act.size(); q++) packs[q * npk / act.size()].push_back(act[q]);
    std::vector<int4> host;
    std::vector<std::array<size_t, kBatchLists>> start(npk);
    std::vector<std::array<int, kBatchLists>> count(npk);
    std::vector<int> flag0(npk);
    b->order.clear();
    for (int p = 0; p < npk; p++) {
        std::vector<int4> L[kBatchLists];
        plan_pack(b, packs[p], L);
        for (int q = 0; q < kBatchLists; q++) {
            start[p][q] = host.size();
            count[p][q] = (int)L[q].size();
            host.insert(host.end(), L[q].begin(), L[q].end());
        }
        flag0[p] = (int)b->order.size();
        b->order.insert(b->order.end(), packs[p].begin(), packs[p].end());
    }
    if (host.size() > b->items_cap) { b->err = "batch: work lists exceed the buffer"; return LPIC_EBUFSIZE; }
    // a pageable source: the copy returns once the source has been staged
    cudaError_t e = host.empty() ? cudaSuccess
                                 : cudaMemcpyAsync(b->items, host.data(), host.size() * sizeof(int4),
                                                   cudaMemcpyHostToDevice, b->st);
    if (e != cudaSuccess) { b->err = std::string("batch upload: ") + cudaGetErrorString(e); return LPIC_ECUDA; }
    while ((int)b->aux.size() < npk - 1) {
        cudaStream_t s = nullptr;
        cudaEvent_t j = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e != cudaSuccess) { b->err = std::string("batch: ") + cudaGetErrorString(e); return LPIC_ECUDA; }
        b->aux.push_back(s);
        b->join.push_back(j);
    }
    std::unique_ptr<SimPack<R>> pk(new SimPack<R>());
    for (int g = 0; g < 2; g++) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return LPIC_ECUDA; }
        cudaMemsetAsync(b->tickets, 0, (size_t)npk * kTicketsPerPack * sizeof(int), b->st);
        cudaEventRecord(b->ev, b->st);
        int nl = 0;
        for (int p = 0; p < npk; p++) {
            cudaStream_t st = p == 0 ? b->st : b->aux[p - 1];
            if (p > 0) cudaStreamWaitEvent(st, b->ev, 0);
            for (size_t q = 0; q < packs[p].size(); q++) pk->v[q] = view_of<R>(b->ctx[packs[p][q]]);
            const auto &cn = count[p];
            auto it = [&](int q) { return (const int4 *)(b->items + start[p][q]); };
            for (int q : {BL_PREPASS, BL_SLOTS, BL_ENVELOPE, BL_PASSB, BL_PASSB_DQ, BL_FILTER, BL_AMPERE, BL_WINDOW})
                nl += cn[q] > 0;
            launch_grid_multi<R>(0, *pk, it(BL_PREPASS), cn[BL_PREPASS], st);
            int *tk = b->tickets + (size_t)p * kTicketsPerPack;
            launch_particles_multi<R>(0, false, *pk, it(BL_SLOTS), cn[BL_SLOTS], tk, st);
            launch_grid_multi<R>(1, *pk, it(BL_ENVELOPE), cn[BL_ENVELOPE], st);
            launch_particles_multi<R>(1, false, *pk, it(BL_PASSB), cn[BL_PASSB], tk + 1, st);
            launch_particles_multi<R>(1, true, *pk, it(BL_PASSB_DQ), cn[BL_PASSB_DQ], tk + 2, st);
            launch_grid_multi<R>(3, *pk, it(BL_FILTER), cn[BL_FILTER], st);
            launch_grid_multi<R>(2, *pk, it(BL_AMPERE), cn[BL_AMPERE], st);
            launch_window_multi<R>(*pk, it(BL_WINDOW), cn[BL_WINDOW], st);
            if (g == 1 && cn[BL_SIMS] > 0) {
                launch_sort_multi<R>(*pk, b->due + flag0[p], it(BL_SORTBLK), cn[BL_SORTBLK], it(BL_SLOTS),
                                     cn[BL_SLOTS], it(BL_SIMS), cn[BL_SIMS], st);
                nl += kSortLaunchesMulti - (cn[BL_SORTBLK] > 0 ? 0 : 3) - (cn[BL_SLOTS] > 0 ? 0 : 2);
            }
            if (p > 0) {
                cudaEventRecord(b->join[p - 1], st);
                cudaStreamWaitEvent(b->st, b->join[p - 1], 0);
            }
        }
        e = cudaStreamEndCapture(b->st, &graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[g], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) { b->err = std::string("graph: ") + cudaGetErrorString(e); return LPIC_ECUDA; }
        b->per_replay[g] = nl;
    }
    b->active_key = active;
    return LPIC_OK;
}
}  // namespace

extern "C" {

size_t lpic_batch_required_bytes(lpic_ctx *const *ctxs, int n) {
    if (!ctxs || n <= 0) return 0;
    for (int k = 0; k < n; k++)
        if (!ctxs[k] || ctxs[k]->prec != ctxs[0]->prec) return 0;
    return flags_bytes(n) + batch_items_bound(ctxs, n) * sizeof(int4);
}

lpic_status lpic_batch_create(lpic_batch **out, lpic_ctx *const *ctxs, int n, void *device_buf,
                              size_t buf_bytes, void *cuda_stream) {
    if (!out || !ctxs || n <= 0) { g_thread_err = "batch: bad arguments"; return LPIC_EINVAL; }
    for (int k = 0; k < n; k++)
        if (!ctxs[k] || ctxs[k]->prec != ctxs[0]->prec || !ctxs[k]->envelope_set) {
            g_thread_err = "batch: contexts must be non-NULL, initialised and share one precision";
            return LPIC_EINVAL;
        }
    for (int k = 0; k < n; k++)
        for (int q = k + 1; q < n; q++)
            if (ctxs[k] == ctxs[q]) { g_thread_err = "batch: a context appears twice"; return LPIC_EINVAL; }
    const size_t need = lpic_batch_required_bytes(ctxs, n);
    if (!device_buf || ((uintptr_t)device_buf % 256) != 0) {
        g_thread_err = "batch: device_buf must be non-NULL and 256-byte aligned";
        return LPIC_EINVAL;
    }
    if (buf_bytes < need) { g_thread_err = "batch: device_buf smaller than lpic_batch_required_bytes"; return LPIC_ENOMEM_BUDGET; }
    lpic_batch *b = new lpic_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->prec = ctxs[0]->prec;
    b->st = (cudaStream_t)cuda_stream;
    b->due = (int *)device_buf;
    b->tickets = b->due + n;
    b->items = (int4 *)((char *)device_buf + flags_bytes(n));
    b->items_cap = (buf_bytes - flags_bytes(n)) / sizeof(int4);
    cudaError_t e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_thread_err = std::string("batch: ") + cudaGetErrorString(e);
        batch_release(b);
        delete b;
        return LPIC_ECUDA;
    }
    *out = b;
    return LPIC_OK;
}

lpic_status lpic_batch_step(lpic_batch *b, const int *steps) {
    if (!b || !steps) return LPIC_EINVAL;
    const size_t n = b->ctx.size();
    int maxs = 0;
    for (size_t k = 0; k < n; k++) {
        if (steps[k] < 0) { b->err = "batch: negative step count"; return LPIC_EINVAL; }
        if (steps[k] > maxs) maxs = steps[k];
    }
    if (maxs == 0) return LPIC_OK;
    if (b->packs < 0) {
        // each simulation's own step graph on its own stream, in turn, after earlier work on
        // the batch stream; later work on the batch stream comes after all of them
        cudaEventRecord(b->ev, b->st);
        for (size_t k = 0; k < n; k++) cudaStreamWaitEvent(b->ctx[k]->st, b->ev, 0);
        lpic_status s = LPIC_OK;
        for (int t = 0; t < maxs && s == LPIC_OK; t++)
            for (size_t k = 0; k < n && s == LPIC_OK; k++) {
                if (steps[k] <= t) continue;
                lpic_ctx *c = b->ctx[k];
                long long before = 0, after = 0;
                for (int f = 0; f < lpic_ctx::kFamilies; f++) before += c->launches[f];
                s = lpic_step(c, 1);
                if (s != LPIC_OK) b->err = "batch: simulation " + std::to_string(k) + ": " + c->err;
                for (int f = 0; f < lpic_ctx::kFamilies; f++) after += c->launches[f];
                b->launches += after - before;
            }
        // also after a failed step: the batch stream waits for whatever was enqueued
        for (size_t k = 0; k < n; k++) {
            cudaEventRecord(b->ev, b->ctx[k]->st);
            cudaStreamWaitEvent(b->st, b->ev, 0);
        }
        if (s != LPIC_OK) return s;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return LPIC_ECUDA; }
        return LPIC_OK;
    }
    // order after earlier work on the contexts' own streams
    for (size_t k = 0; k < n; k++) {
        cudaEventRecord(b->ev, b->ctx[k]->st);
        cudaStreamWaitEvent(b->st, b->ev, 0);
    }
    std::vector<char> active(n), sort(n);
    std::vector<int> flags;
    for (int t = 0; t < maxs; t++) {
        for (size_t k = 0; k < n; k++) active[k] = steps[k] > t;
        for (size_t k = 0; k < n; k++)
            if (active[k]) {
                const long long r0 = b->ctx[k]->launches[F_RELOCATE];
                pre_step(b->ctx[k], b->st);
                b->launches += b->ctx[k]->launches[F_RELOCATE] - r0;
            }
        if (!b->exec[0] || active != b->active_key) {
            lpic_status s = b->prec == LPIC_FP64 ? batch_capture<double>(b, active) : batch_capture<float>(b, active);
            if (s != LPIC_OK) return s;
        }
        bool any = false;
        for (size_t k = 0; k < n; k++) {
            sort[k] = active[k] && advance_mirror(b->ctx[k]);
            any = any || sort[k];
        }
        if (any) {
            flags.resize(b->order.size());
            for (size_t q = 0; q < b->order.size(); q++) flags[q] = sort[b->order[q]] ? 1 : 0;
            // a pageable source: the copy returns once the source has been staged
            cudaError_t e = cudaMemcpyAsync(b->due, flags.data(), flags.size() * sizeof(int),
                                            cudaMemcpyHostToDevice, b->st);
            if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return LPIC_ECUDA; }
        }
        cudaError_t e = cudaGraphLaunch(b->exec[any ? 1 : 0], b->st);
        if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return LPIC_ECUDA; }
        b->launches += b->per_replay[any ? 1 : 0];
    }
    // later calls on a context's own stream come after this batch step
    cudaEventRecord(b->ev, b->st);
    for (size_t k = 0; k < n; k++) cudaStreamWaitEvent(b->ctx[k]->st, b->ev, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { b->err = cudaGetErrorString(e); return LPIC_ECUDA; }
    return LPIC_OK;
}

lpic_status lpic_batch_set_tuning(lpic_batch *b, int32_t particles_per_item, int32_t packs) {
    if (!b) return LPIC_EINVAL;
    if (particles_per_item < kMinChunk || particles_per_item > kMaxChunk || particles_per_item % 256) {
        b->err = "batch: particles_per_item must be a multiple of 256 in [1024, 1048576]";
        return LPIC_EINVAL;
    }
    if (packs < -1) { b->err = "batch: packs must be >= -1"; return LPIC_EINVAL; }
    if (particles_per_item != b->chunk || packs != b->packs) {
        b->chunk = particles_per_item;
        b->packs = packs;
        drop_graphs(b);   // re-planned at the next step
    }
    return LPIC_OK;
}

int64_t lpic_batch_launches(const lpic_batch *b) { return b ? b->launches : -1; }

const char *lpic_batch_last_error(const lpic_batch *b) { return b ? b->err.c_str() : "batch: NULL"; }

lpic_status lpic_batch_destroy(lpic_batch *b) {
    if (!b) return LPIC_EINVAL;
    cudaStreamSynchronize(b->st);
    batch_release(b);
    delete b;
    return LPIC_OK;
}

}  // extern "C"
