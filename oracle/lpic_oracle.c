/*
 * lpic_oracle.c -- plain, slow, FP64 CPU oracle of one timestep of the
 * cylindrical (azimuthal mode m=0) laser-envelope particle-in-cell method of
 * Massimo et al., "Efficient cylindrical envelope modeling for laser
 * wakefield acceleration" (arXiv:1912.04674).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header
 * or constant table with the CUDA library; it is written for a reader who
 * checks it against the paper by eye: one node or one particle at a time, in
 * the order the method states, no blocking, fusion or reordering.
 *
 * Units are the paper's normalised units (Sec. 2): lengths c/w0, time 1/w0,
 * fields m c w0 / e, densities n_c.  Macro-particles are electrons, q=-1, m=1;
 * ions are an immobile neutralising background and are not stored.
 *
 * Grid (reading of Fig. 1, which is not printed; Lifschitz-type centring):
 *   primal nodes x_i = i dx (window-relative), r_j = j dr, j=0 on the axis.
 *   A (envelope, complex), chi, Phi at (i, j)          i in [0,Nx], j in [0,Nr]
 *   Ex, Jx at (i+1/2, j)                               i in [0,Nx-1], j in [0,Nr]
 *   Er, Jr at (i, j+1/2)                               i in [0,Nx],   j in [0,Nr-1]
 *   Bt at (i+1/2, j+1/2)                               i in [0,Nx-1], j in [0,Nr-1]
 * All arrays are stored [i][j] with j (radial) fastest.
 *
 * Time levels at the start of step n: x^n, p^{n-1/2}, E^n, B^{n-1/2},
 * A^n, A^{n-1}.  The envelope is centred in time like E (Sec. 3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

#define PI 3.14159265358979323846

typedef struct osim {
    int nx, nr;
    double dx, dr, dt;
    int moving_window;
    long step;   /* n */
    long shift;  /* s: window origin is s*dx in the lab frame */
    /* fields */
    double *ex, *er, *bt, *btn;          /* btn: B^n, the interpolated average */
    double complex *a, *am;              /* A^n, A^{n-1} */
    double *chi, *jx, *jr;
    double *dq;                          /* charge change of the last step (diagnostic) */
    /* node scratch */
    double *phi, *dphix, *dphir, *phih;
    /* particles: x is kept as the lab cell index ix and the in-cell offset ox in [0,1)
     * (x_lab = (ix + ox) dx), so that a displacement is never lost against the size of
     * the lab coordinate */
    long np, cap;
    long *ix;
    double *ox, *y, *z, *px, *py, *pz, *w;
    uint64_t *id;
    /* plasma profile kept for injection at the moving window front */
    int have_plasma;
    double n0, x_start, ramp_len;
    int ppcx, ppcr, ppct;
    uint64_t seed;
    /* current filter: passes of the binomial filter after the deposit (0: off) */
    int filter_passes;
} osim;

/* ------------------------------------------------------------------ sizes */
static long n_node(const osim *s) { return (long)(s->nx + 1) * (s->nr + 1); }
static long n_ex(const osim *s) { return (long)s->nx * (s->nr + 1); }
static long n_er(const osim *s) { return (long)(s->nx + 1) * s->nr; }
static long n_bt(const osim *s) { return (long)s->nx * s->nr; }

static void *zalloc(long n, long sz) { return calloc((size_t)(n > 0 ? n : 1), (size_t)sz); }

osim *osim_create(int nx, int nr, double dx, double dr, double dt, int moving_window)
{
    osim *s = (osim *)calloc(1, sizeof(osim));
    s->nx = nx; s->nr = nr; s->dx = dx; s->dr = dr; s->dt = dt;
    s->moving_window = moving_window;
    s->ex = zalloc(n_ex(s), sizeof(double));
    s->jx = zalloc(n_ex(s), sizeof(double));
    s->er = zalloc(n_er(s), sizeof(double));
    s->jr = zalloc(n_er(s), sizeof(double));
    s->bt = zalloc(n_bt(s), sizeof(double));
    s->btn = zalloc(n_bt(s), sizeof(double));
    s->a = zalloc(n_node(s), sizeof(double complex));
    s->am = zalloc(n_node(s), sizeof(double complex));
    s->chi = zalloc(n_node(s), sizeof(double));
    s->dq = zalloc(n_node(s), sizeof(double));
    s->phi = zalloc(n_node(s), sizeof(double));
    s->dphix = zalloc(n_node(s), sizeof(double));
    s->dphir = zalloc(n_node(s), sizeof(double));
    s->phih = zalloc(n_node(s), sizeof(double));
    return s;
}

void osim_free(osim *s)
{
    if (!s) return;
    free(s->ex); free(s->jx); free(s->er); free(s->jr); free(s->bt); free(s->btn);
    free(s->a); free(s->am); free(s->chi); free(s->dq);
    free(s->phi); free(s->dphix); free(s->dphir); free(s->phih);
    free(s->ix); free(s->ox); free(s->y); free(s->z); free(s->px); free(s->py); free(s->pz);
    free(s->w); free(s->id);
    free(s);
}

/* particle storage ------------------------------------------------------- */
void osim_reserve(osim *s, long cap)
{
    if (cap <= s->cap) return;
    s->ix = realloc(s->ix, cap * sizeof(long));
    s->ox = realloc(s->ox, cap * sizeof(double));
    s->y = realloc(s->y, cap * sizeof(double));
    s->z = realloc(s->z, cap * sizeof(double));
    s->px = realloc(s->px, cap * sizeof(double));
    s->py = realloc(s->py, cap * sizeof(double));
    s->pz = realloc(s->pz, cap * sizeof(double));
    s->w = realloc(s->w, cap * sizeof(double));
    s->id = realloc(s->id, cap * sizeof(uint64_t));
    s->cap = cap;
}

/* Set the particle count (tests write the arrays afterwards). */
void osim_set_np(osim *s, long np)
{
    osim_reserve(s, np > 0 ? np : 1);
    s->np = np;
}

static void push_particle(osim *s, long ix, double ox, double y, double z, double w, uint64_t id)
{
    if (s->np == s->cap) osim_reserve(s, s->cap ? 2 * s->cap : 1024);
    long k = s->np++;
    s->ix[k] = ix; s->ox[k] = ox; s->y[k] = y; s->z[k] = z;
    s->px[k] = 0.0; s->py[k] = 0.0; s->pz[k] = 0.0;
    s->w[k] = w; s->id[k] = id;
}

/* -------------------------------------------------------------- envelope init
 * Paraxial focused Gaussian pulse (Sec. 4 benchmarks use a Gaussian pulse;
 * its vacuum solution of 2i dA/dx + lap_perp A = 0 is the Rayleigh beam):
 *   A(x,r,t) = a0/D exp(-r^2/(w0^2 D)) exp(-(x-t-xc)^2/L^2),
 *   D = 1 + i (x-xf)/xR,  xR = w0^2/2.
 * A^0 at t=0 and A^{-1} at t=-dt on the initial window (shift 0).
 */
static double complex gaussian_pulse(double x, double r, double t, double a0, double w0,
                                     double L, double xc, double xf)
{
    double xr_ = 0.5 * w0 * w0;
    double complex D = 1.0 + I * ((x - xf) / xr_);
    double lon = (x - t - xc) / L;
    return a0 / D * cexp(-(r * r) / (w0 * w0 * D)) * exp(-lon * lon);
}

void osim_init_envelope(osim *s, double a0, double w0, double L, double xc, double xf)
{
    double x0 = s->shift * s->dx;
    for (int i = 0; i <= s->nx; i++)
        for (int j = 0; j <= s->nr; j++) {
            double x = x0 + i * s->dx, r = j * s->dr;
            s->a[i * (s->nr + 1) + j] = gaussian_pulse(x, r, 0.0, a0, w0, L, xc, xf);
            s->am[i * (s->nr + 1) + j] = gaussian_pulse(x, r, -s->dt, a0, w0, L, xc, xf);
        }
}

/* ------------------------------------------------------------ plasma loading
 * SplitMix64 (Steele, Lea, Flood 2014): the k-th output of the generator
 * seeded with `seed` is mix(seed + k*0x9E3779B97F4A7C15).  The random
 * azimuthal offset of cell c is the (c+1)-th output.
 */
uint64_t osim_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double density(const osim *s, double xlab)
{
    if (xlab < s->x_start) return 0.0;
    if (s->ramp_len > 0.0 && xlab < s->x_start + s->ramp_len)
        return s->n0 * (xlab - s->x_start) / s->ramp_len;
    return s->n0;
}

/* Load the regular lattice of one lab cell column c (lab x in [c dx, (c+1) dx)):
 * ppcx x ppcr positions per (x,r) cell at fractions (a+1/2)/ppcx, (b+1/2)/ppcr,
 * and ppct azimuthal samples theta_k = 2 pi (k+u)/ppct, u from SplitMix64.
 * Weight: density times the ring volume 2 pi r dr dx shared by the cell's
 * particles, so that the weights of a cell sum to n times its annulus volume. */
static void load_column(osim *s, long c)
{
    for (int j = 0; j < s->nr; j++) {
        uint64_t cell = (uint64_t)c * (uint64_t)s->nr + (uint64_t)j;
        double u = (double)(osim_splitmix64(s->seed, cell + 1) >> 11) * (1.0 / 9007199254740992.0);
        for (int a = 0; a < s->ppcx; a++) {
            double frac = (a + 0.5) / s->ppcx;
            double xlab = (c + frac) * s->dx;
            double n = density(s, xlab);
            if (n <= 0.0) continue;
            for (int b = 0; b < s->ppcr; b++) {
                double r = (j + (b + 0.5) / s->ppcr) * s->dr;
                double w = n * 2.0 * PI * r * s->dr * s->dx / (s->ppcx * s->ppcr * s->ppct);
                for (int k = 0; k < s->ppct; k++) {
                    double th = 2.0 * PI * (k + u) / s->ppct;
                    uint64_t pid = ((cell * s->ppcx + a) * s->ppcr + b) * s->ppct + k;
                    push_particle(s, c, frac, r * cos(th), r * sin(th), w, pid);
                }
            }
        }
    }
}

void osim_load_plasma(osim *s, double n0, double x_start, double ramp_len,
                      int ppcx, int ppcr, int ppct, uint64_t seed)
{
    s->have_plasma = 1;
    s->n0 = n0; s->x_start = x_start; s->ramp_len = ramp_len;
    s->ppcx = ppcx; s->ppcr = ppcr; s->ppct = ppct; s->seed = seed;
    for (int i = 0; i < s->nx; i++) load_column(s, s->shift + i);
}

/* ------------------------------------------------------------------ Faraday
 * Eq. (MaxwellEqsCylindrical), first equation, Yee-centred (Sec. 3):
 * B^{n+1/2} = B^{n-1/2} + dt [ dEx/dr - dEr/dx ];  B^n = (B^{n-1/2}+B^{n+1/2})/2.
 */
void osim_faraday(osim *s)
{
    int nx = s->nx, nr = s->nr;
    for (int i = 0; i < nx; i++)
        for (int j = 0; j < nr; j++) {
            double dexdr = (s->ex[i * (nr + 1) + j + 1] - s->ex[i * (nr + 1) + j]) / s->dr;
            double derdx = (s->er[(i + 1) * nr + j] - s->er[i * nr + j]) / s->dx;
            double bold = s->bt[i * nr + j];
            double bnew = bold + s->dt * (dexdr - derdx);
            s->bt[i * nr + j] = bnew;
            s->btn[i * nr + j] = 0.5 * (bold + bnew);
        }
}

/* ------------------------------------------------------------------ Ampere
 * Eq. (MaxwellEqsCylindrical), second and third equations:
 *   Er += dt [ -dBt/dx - Jr ]                           (Er = 0 on the x ends)
 *   Ex += dt [ (r_{j+1/2} B_{j+1/2} - r_{j-1/2} B_{j-1/2}) / (r_j dr) - Jx ]
 *   axis (j=0):  Ex += dt [ 4 B_{1/2} / dr - Jx ]       (Stokes on the disc r<dr/2)
 *   Ex = 0 at r = r_max (perfect conductor).
 */
void osim_ampere(osim *s)
{
    int nx = s->nx, nr = s->nr;
    for (int i = 0; i <= nx; i++)
        for (int j = 0; j < nr; j++) {
            if (i == 0 || i == nx) { s->er[i * nr + j] = 0.0; continue; }
            double dbdx = (s->bt[i * nr + j] - s->bt[(i - 1) * nr + j]) / s->dx;
            s->er[i * nr + j] += s->dt * (-dbdx - s->jr[i * nr + j]);
        }
    for (int i = 0; i < nx; i++)
        for (int j = 0; j <= nr; j++) {
            double *e = &s->ex[i * (nr + 1) + j];
            if (j == nr) { *e = 0.0; continue; }
            double curl;
            if (j == 0) {
                curl = 4.0 * s->bt[i * nr + 0] / s->dr;
            } else {
                double rp = (j + 0.5) * s->dr, rm = (j - 0.5) * s->dr, rj = j * s->dr;
                curl = (rp * s->bt[i * nr + j] - rm * s->bt[i * nr + j - 1]) / (rj * s->dr);
            }
            *e += s->dt * (curl - s->jx[i * (nr + 1) + j]);
        }
}

/* ------------------------------------------------------------------ gathers
 * Linear (area) weights on a grid whose first point sits at (sx, sr) cells;
 * points outside the grid read zero, except the radial ghost row j=-1 of a
 * radially staggered (odd in r) quantity, which reads -F(j=0).
 */
static double grid_at(const double *F, int ni, int nj, int i, int j, int odd_r)
{
    if (i < 0 || i >= ni) return 0.0;
    if (j == -1 && odd_r) return -F[i * nj + 0];
    if (j < 0 || j >= nj) return 0.0;
    return F[i * nj + j];
}

static double gather(const double *F, int ni, int nj, double sx, double sr,
                     long icell, double fcell, double rn)
{
    /* x position = icell + fcell (window cells), fcell in [0,1) */
    double u = fcell - sx;
    long i0 = icell;
    if (u < 0.0) { u += 1.0; i0 -= 1; }
    double v = rn - sr;
    int j0 = (int)floor(v);
    double fu = u, fv = v - j0;
    int odd = (sr != 0.0);
    return (1.0 - fu) * (1.0 - fv) * grid_at(F, ni, nj, (int)i0, j0, odd)
         + fu * (1.0 - fv) * grid_at(F, ni, nj, (int)(i0 + 1), j0, odd)
         + (1.0 - fu) * fv * grid_at(F, ni, nj, (int)i0, j0 + 1, odd)
         + fu * fv * grid_at(F, ni, nj, (int)(i0 + 1), j0 + 1, odd);
}

/* Node volumes.  Ring volume 2 pi r_j dr dx for j>=1.  The axis node:
 *  - charge and current use pi (dr/2)^2 dx, the disc the axis curl 4B/dr is
 *    exact on, so that the discrete Gauss law is kept;
 *  - the susceptibility uses pi dr^2 dx / 3, the volume that linear weights
 *    give a uniform density on the axis node. */
static double vol_q(const osim *s, int j)
{
    return j == 0 ? PI * 0.25 * s->dr * s->dr * s->dx : 2.0 * PI * j * s->dr * s->dr * s->dx;
}
static double vol_chi(const osim *s, int j)
{
    return j == 0 ? PI * s->dr * s->dr * s->dx / 3.0 : 2.0 * PI * j * s->dr * s->dr * s->dx;
}

/* Phi = |A|^2/2 at nodes (Sec. 2) and its centred differences (Sec. 3):
 * dPhi/dx = (Phi_{i+1}-Phi_{i-1})/(2dx) with Phi=0 outside [0,Nx];
 * dPhi/dr = (Phi_{j+1}-Phi_{j-1})/(2dr), 0 on the axis, Phi_{Nr+1}=0. */
static void ponderomotive_nodes(osim *s)
{
    int nx = s->nx, nr = s->nr, nj = nr + 1;
    for (long k = 0; k < n_node(s); k++) {
        double complex a = s->a[k];
        s->phi[k] = 0.5 * (creal(a) * creal(a) + cimag(a) * cimag(a));
    }
    for (int i = 0; i <= nx; i++)
        for (int j = 0; j <= nr; j++) {
            double pxp = i < nx ? s->phi[(i + 1) * nj + j] : 0.0;
            double pxm = i > 0 ? s->phi[(i - 1) * nj + j] : 0.0;
            s->dphix[i * nj + j] = (pxp - pxm) / (2.0 * s->dx);
            if (j == 0) { s->dphir[i * nj + j] = 0.0; continue; }
            double prp = j < nr ? s->phi[i * nj + j + 1] : 0.0;
            double prm = s->phi[i * nj + j - 1];
            s->dphir[i * nj + j] = (prp - prm) / (2.0 * s->dr);
        }
}

/* ------------------------------------------------------------- particle pass A
 * For every particle at x^n (Eqs. EquationsOfMotion, motion_equations_cartesian):
 *  1. gather Ex, Er, Bt (B^n), Phi, dPhi/dx, dPhi/dr with linear weights;
 *  2. project to 3D Cartesian: cos = y/r, sin = z/r (r=0: cos=1, sin=0),
 *     E = (Ex, Er cos, Er sin), B = Bt (0, -sin, cos), grad Phi = (dx, dr cos, dr sin);
 *  3. time-centred ponderomotive Lorentz factor
 *        g0 = sqrt(1 + |p^{n-1/2}|^2 + Phi),
 *        p* = p^{n-1/2} + dt/2 (q E - grad Phi/(2 g0)),   gt = sqrt(1 + |p*|^2 + Phi);
 *  4. susceptibility deposit chi += q^2/m w S /(gt V_chi)  (Sec. 2: charge density / gamma);
 *  5. ponderomotive Boris push with F = q E - grad Phi/(2 gt):
 *        p- = p + dt/2 F,  g- = sqrt(1+|p-|^2+Phi),  t = q B dt/(2 g-),  s = 2t/(1+t^2),
 *        p' = p- + p- x t,  p+ = p- + p' x s,  p^{n+1/2} = p+ + dt/2 F.
 */
void osim_pass_a(osim *s)
{
    int nx = s->nx, nr = s->nr;
    const double q = -1.0;
    double hdt = 0.5 * s->dt;
    ponderomotive_nodes(s);
    memset(s->chi, 0, n_node(s) * sizeof(double));
    for (long k = 0; k < s->np; k++) {
        long ic = s->ix[k] - s->shift;
        double fx = s->ox[k];
        double r = sqrt(s->y[k] * s->y[k] + s->z[k] * s->z[k]);
        double rn = r / s->dr;
        double ct = 1.0, st = 0.0;
        if (r > 0.0) { ct = s->y[k] / r; st = s->z[k] / r; }
        double exg = gather(s->ex, nx, nr + 1, 0.5, 0.0, ic, fx, rn);
        double erg = gather(s->er, nx + 1, nr, 0.0, 0.5, ic, fx, rn);
        double btg = gather(s->btn, nx, nr, 0.5, 0.5, ic, fx, rn);
        double phg = gather(s->phi, nx + 1, nr + 1, 0.0, 0.0, ic, fx, rn);
        double gxg = gather(s->dphix, nx + 1, nr + 1, 0.0, 0.0, ic, fx, rn);
        double grg = gather(s->dphir, nx + 1, nr + 1, 0.0, 0.0, ic, fx, rn);
        double E[3] = {exg, erg * ct, erg * st};
        double B[3] = {0.0, -btg * st, btg * ct};
        double G[3] = {gxg, grg * ct, grg * st};
        double p[3] = {s->px[k], s->py[k], s->pz[k]};

        double g0 = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + phg);
        double ps[3];
        for (int c = 0; c < 3; c++) ps[c] = p[c] + hdt * (q * E[c] - G[c] / (2.0 * g0));
        double gt = sqrt(1.0 + ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2] + phg);

        /* susceptibility deposit with the primal linear weights */
        int i0 = (int)ic, j0 = (int)floor(rn);
        double fr = rn - j0;
        for (int di = 0; di < 2; di++)
            for (int dj = 0; dj < 2; dj++) {
                int i = i0 + di, j = j0 + dj;
                if (i < 0 || i > nx || j < 0 || j > nr) continue;
                double sw = (di ? fx : 1.0 - fx) * (dj ? fr : 1.0 - fr);
                s->chi[i * (nr + 1) + j] += q * q * s->w[k] * sw / (gt * vol_chi(s, j));
            }

        double F[3];
        for (int c = 0; c < 3; c++) F[c] = q * E[c] - G[c] / (2.0 * gt);
        double pm[3];
        for (int c = 0; c < 3; c++) pm[c] = p[c] + hdt * F[c];
        double gm = sqrt(1.0 + pm[0] * pm[0] + pm[1] * pm[1] + pm[2] * pm[2] + phg);
        double t[3], sv[3];
        for (int c = 0; c < 3; c++) t[c] = q * B[c] * hdt / gm;
        double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        for (int c = 0; c < 3; c++) sv[c] = 2.0 * t[c] / (1.0 + t2);
        double pp[3] = {pm[0] + (pm[1] * t[2] - pm[2] * t[1]),
                        pm[1] + (pm[2] * t[0] - pm[0] * t[2]),
                        pm[2] + (pm[0] * t[1] - pm[1] * t[0])};
        double pl[3] = {pm[0] + (pp[1] * sv[2] - pp[2] * sv[1]),
                        pm[1] + (pp[2] * sv[0] - pp[0] * sv[2]),
                        pm[2] + (pp[0] * sv[1] - pp[1] * sv[0])};
        s->px[k] = pl[0] + hdt * F[0];
        s->py[k] = pl[1] + hdt * F[1];
        s->pz[k] = pl[2] + hdt * F[2];
    }
}

/* ------------------------------------------------------------ envelope solver
 * Eq. (envelope_solver), with the dt^2 factor on the whole bracket (the
 * centred discretisation of Eq. envelope_equation gives it there) and dz read
 * as dx:
 *   A^{n+1} = (1+i dt)/(1+dt^2) [ 2A^n - (1+i dt) A^{n-1}
 *              + dt^2 ( lap A^n - chi^n A^n + 2i (A_{i+1}-A_{i-1})/(2dx) ) ],
 *   lap A = (A_{i+1}-2A+A_{i-1})/dx^2 + (A_{j+1}-2A+A_{j-1})/dr^2
 *           + (A_{j+1}-A_{j-1})/(2 dr r_j),
 *   axis (j=0, A even in r):  radial part = 4 (A_{i,1} - A_{i,0}) / dr^2.
 * A = 0 at i=-1, i=Nx+1 and j=Nr+1.  Afterwards A^{n-1} <- A^n, A^n <- A^{n+1}.
 */
void osim_envelope(osim *s)
{
    int nx = s->nx, nr = s->nr, nj = nr + 1;
    double dt = s->dt, dx = s->dx, dr = s->dr;
    double complex *an = (double complex *)malloc(n_node(s) * sizeof(double complex));
    double complex pre = (1.0 + I * dt) / (1.0 + dt * dt);
    for (int i = 0; i <= nx; i++)
        for (int j = 0; j <= nr; j++) {
            double complex c = s->a[i * nj + j];
            double complex xp = i < nx ? s->a[(i + 1) * nj + j] : 0.0;
            double complex xm = i > 0 ? s->a[(i - 1) * nj + j] : 0.0;
            double complex lap = (xp - 2.0 * c + xm) / (dx * dx);
            if (j == 0) {
                lap += 4.0 * (s->a[i * nj + 1] - c) / (dr * dr);
            } else {
                double complex rp = j < nr ? s->a[i * nj + j + 1] : 0.0;
                double complex rm = s->a[i * nj + j - 1];
                lap += (rp - 2.0 * c + rm) / (dr * dr) + (rp - rm) / (2.0 * dr * (j * dr));
            }
            double complex ddx = (xp - xm) / (2.0 * dx);
            double complex rhs = 2.0 * c - (1.0 + I * dt) * s->am[i * nj + j]
                               + dt * dt * (lap - s->chi[i * nj + j] * c + 2.0 * I * ddx);
            an[i * nj + j] = pre * rhs;
        }
    for (long k = 0; k < n_node(s); k++) {
        s->am[k] = s->a[k];
        s->a[k] = an[k];
    }
    free(an);
}

/* ------------------------------------------------------------- particle pass B
 * Position push with the time-centred ponderomotive potential
 *   Phi^{n+1/2} = (Phi^n + Phi^{n+1})/2 gathered at x^n,
 *   gbar = sqrt(1 + |p^{n+1/2}|^2 + Phi^{n+1/2}),   x^{n+1} = x^n + dt p^{n+1/2}/gbar,
 * then charge-conserving (Esirkepov-type) deposition of Jx, Jr in the (x,r)
 * index plane.  With S0, S1 the linear shapes at (x^n, r^n), (x^{n+1}, r^{n+1})
 * on a 3x3 node window and DS = S1 - S0:
 *   Wx = DSx (S0r + DSr/2),  Wr = DSr (S0x + DSx/2),
 *   Ix(i+1/2, j) = -(q w/dt) sum_{k<=i} Wx(k, j),   Jx = Ix / (V_j/dx),
 *   Ir(i, j+1/2) = -(q w/dt) sum_{l<=j} Wr(i, l),   Jr = Ir / (2 pi r_{j+1/2} dx),
 * so that dQ/dt + (Ix_{i+1/2}-Ix_{i-1/2}) + (Ir_{j+1/2}-Ir_{j-1/2}) = 0 node by node.
 * Contributions to points outside the grid are discarded.  The charge change
 * q w DS is also recorded (diagnostic of the continuity residual).
 *
 * DS is a difference of shape factors at two nearby positions, so both positions are
 * taken relative to the particle's cell: x as (cell, offset) moved by dt v_x/dx, and the
 * new radius as r^n + dr_step with the radial step in the cancellation-free form
 *   dr_step = (dy (y^n + y^{n+1}) + dz (z^n + z^{n+1})) / (r^n + r^{n+1}),
 * dy = dt p_y/gbar, dz = dt p_z/gbar (the identity r1^2 - r0^2 = (r1 - r0)(r1 + r0)).
 */
static void shape3(long i0, double f, long base, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    out[i0 - base] = 1.0 - f;
    out[i0 - base + 1] = f;
}

void osim_pass_b(osim *s)
{
    int nx = s->nx, nr = s->nr;
    const double q = -1.0;
    double dt = s->dt;
    for (long k = 0; k < n_node(s); k++)
        s->phih[k] = 0.5 * (0.5 * (creal(s->a[k]) * creal(s->a[k]) + cimag(s->a[k]) * cimag(s->a[k]))
                          + 0.5 * (creal(s->am[k]) * creal(s->am[k]) + cimag(s->am[k]) * cimag(s->am[k])));
    memset(s->jx, 0, n_ex(s) * sizeof(double));
    memset(s->jr, 0, n_er(s) * sizeof(double));
    memset(s->dq, 0, n_node(s) * sizeof(double));
    for (long k = 0; k < s->np; k++) {
        long ia = s->ix[k] - s->shift;
        double fa = s->ox[k];
        double y0 = s->y[k], z0 = s->z[k];
        double r0 = sqrt(y0 * y0 + z0 * z0);
        double rn0 = r0 / s->dr;
        double ph = gather(s->phih, nx + 1, nr + 1, 0.0, 0.0, ia, fa, rn0);
        double p2 = s->px[k] * s->px[k] + s->py[k] * s->py[k] + s->pz[k] * s->pz[k];
        double gbar = sqrt(1.0 + p2 + ph);
        double ddx = dt * s->px[k] / gbar, ddy = dt * s->py[k] / gbar, ddz = dt * s->pz[k] / gbar;
        /* x: offset push within the cell frame */
        double fb = fa + ddx / s->dx;
        long ib = ia + (long)floor(fb);
        fb -= floor(fb);
        s->ix[k] += ib - ia;
        s->ox[k] = fb;
        /* r: new radius from the radial step */
        double y1 = y0 + ddy, z1 = z0 + ddz;
        double r1 = sqrt(y1 * y1 + z1 * z1);
        double step_r = (r0 + r1 > 0.0) ? (ddy * (y0 + y1) + ddz * (z0 + z1)) / (r0 + r1) : 0.0;
        double rn1 = rn0 + step_r / s->dr;
        if (rn1 < 0.0) rn1 = 0.0;
        s->y[k] = y1;
        s->z[k] = z1;

        int ja = (int)floor(rn0), jb = (int)floor(rn1);
        long imin = ia < ib ? ia : ib;
        int jmin = ja < jb ? ja : jb;
        double s0x[3], s1x[3], s0r[3], s1r[3], dsx[3], dsr[3];
        shape3(ia, fa, imin, s0x); shape3(ib, fb, imin, s1x);
        shape3(ja, rn0 - ja, jmin, s0r); shape3(jb, rn1 - jb, jmin, s1r);
        for (int c = 0; c < 3; c++) { dsx[c] = s1x[c] - s0x[c]; dsr[c] = s1r[c] - s0r[c]; }
        double qw = q * s->w[k];
        for (int l = 0; l < 3; l++) {          /* Jx on faces imin+1/2, imin+3/2 */
            int j = jmin + l;
            double acc = 0.0;
            for (int c = 0; c < 2; c++) {
                acc += dsx[c] * (s0r[l] + 0.5 * dsr[l]);
                long i = imin + c;
                if (i < 0 || i >= nx || j < 0 || j > nr) continue;
                double area = vol_q(s, j) / s->dx;
                s->jx[i * (nr + 1) + j] += -qw / dt * acc / area;
            }
        }
        for (int c = 0; c < 3; c++) {          /* Jr on faces jmin+1/2, jmin+3/2 */
            long i = imin + c;
            double acc = 0.0;
            for (int l = 0; l < 2; l++) {
                acc += dsr[l] * (s0x[c] + 0.5 * dsx[c]);
                int j = jmin + l;
                if (i < 0 || i > nx || j < 0 || j >= nr) continue;
                double area = 2.0 * PI * (j + 0.5) * s->dr * s->dx;
                s->jr[i * nr + j] += -qw / dt * acc / area;
            }
        }
        for (int c = 0; c < 3; c++)
            for (int l = 0; l < 3; l++) {
                long i = imin + c;
                int j = jmin + l;
                if (i < 0 || i > nx || j < 0 || j > nr) continue;
                s->dq[i * (nr + 1) + j] += qw * (s1x[c] * s1r[l] - s0x[c] * s0r[l]);
            }
    }
}

/* --------------------------------------------------------------- moving window
 * The window moves at c: after step n completes (time (n+1) dt), if
 * (n+1) dt >= (s+1) dx the grids shift one column towards -x, the new front
 * column is zero, and fresh plasma is loaded in the new last cell column.
 * Then particles outside the window (x < 0, x >= Nx dx) or at r >= r_max are
 * removed.  Also advances the step counter.
 */
static void shift_array(double *F, int ni, int nj)
{
    memmove(F, F + nj, (size_t)(ni - 1) * nj * sizeof(double));
    memset(F + (long)(ni - 1) * nj, 0, (size_t)nj * sizeof(double));
}
static void shift_carray(double complex *F, int ni, int nj)
{
    memmove(F, F + nj, (size_t)(ni - 1) * nj * sizeof(double complex));
    for (int j = 0; j < nj; j++) F[(long)(ni - 1) * nj + j] = 0.0;
}

void osim_window(osim *s)
{
    int nx = s->nx, nr = s->nr;
    s->step += 1;
    if (s->moving_window && (double)s->step * s->dt >= (double)(s->shift + 1) * s->dx) {
        s->shift += 1;
        shift_array(s->ex, nx, nr + 1);
        shift_array(s->er, nx + 1, nr);
        shift_array(s->bt, nx, nr);
        shift_carray(s->a, nx + 1, nr + 1);
        shift_carray(s->am, nx + 1, nr + 1);
        if (s->have_plasma) load_column(s, s->shift + nx - 1);
    }
    double rmax = nr * s->dr;
    long keep = 0;
    for (long k = 0; k < s->np; k++) {
        long ic = s->ix[k] - s->shift;
        double r = sqrt(s->y[k] * s->y[k] + s->z[k] * s->z[k]);
        if (ic < 0 || ic >= nx || r >= rmax) continue;
        s->ix[keep] = s->ix[k]; s->ox[keep] = s->ox[k];
        s->y[keep] = s->y[k]; s->z[keep] = s->z[k];
        s->px[keep] = s->px[k]; s->py[keep] = s->py[k]; s->pz[keep] = s->pz[k];
        s->w[keep] = s->w[k]; s->id[keep] = s->id[k];
        keep++;
    }
    s->np = keep;
}

/* --------------------------------------------------------------- current filter
 * Sec. 4 (nonlinear benchmark): an uncompensated binomial filter of 7 passes is applied
 * against numerical Cherenkov radiation.  Reading: one pass replaces every value F_i of Jx
 * and Jr along x by (F_{i-1} + 2 F_i + F_{i+1}) / 4, with F = 0 outside the window; the
 * charge change dq of the step takes the same passes, so that the filtered current keeps the
 * continuity equation with the filtered charge.  Radial filtering is not applied.
 */
static void binomial_pass_x(double *F, int ni, int nj, double *tmp)
{
    memcpy(tmp, F, (size_t)ni * nj * sizeof(double));
    for (int i = 0; i < ni; i++)
        for (int j = 0; j < nj; j++) {
            double left = i > 0 ? tmp[(i - 1) * nj + j] : 0.0;
            double right = i < ni - 1 ? tmp[(i + 1) * nj + j] : 0.0;
            F[i * nj + j] = 0.25 * left + 0.5 * tmp[i * nj + j] + 0.25 * right;
        }
}

void osim_set_filter(osim *s, int passes) { s->filter_passes = passes > 0 ? passes : 0; }

void osim_filter(osim *s)
{
    double *tmp = (double *)malloc((size_t)n_node(s) * sizeof(double));
    for (int p = 0; p < s->filter_passes; p++) {
        binomial_pass_x(s->jx, s->nx, s->nr + 1, tmp);
        binomial_pass_x(s->jr, s->nx + 1, s->nr, tmp);
        binomial_pass_x(s->dq, s->nx + 1, s->nr + 1, tmp);
    }
    free(tmp);
}

/* One full timestep in the order of the 3D envelope loop the paper follows (Sec. 3). */
void osim_step(osim *s)
{
    osim_faraday(s);
    osim_pass_a(s);
    osim_envelope(s);
    osim_pass_b(s);
    if (s->filter_passes > 0) osim_filter(s);
    osim_ampere(s);
    osim_window(s);
}

void osim_run(osim *s, long nsteps)
{
    for (long k = 0; k < nsteps; k++) osim_step(s);
}

/* ------------------------------------------------------------------ accessors */
enum { F_EX = 0, F_ER, F_BT, F_BTN, F_A, F_AM, F_CHI, F_JX, F_JR, F_DQ, F_PHI, F_DPHIX, F_DPHIR, F_PHIH };
void *osim_field(osim *s, int which)
{
    switch (which) {
    case F_EX: return s->ex;   case F_ER: return s->er;   case F_BT: return s->bt;
    case F_BTN: return s->btn; case F_A: return s->a;     case F_AM: return s->am;
    case F_CHI: return s->chi; case F_JX: return s->jx;   case F_JR: return s->jr;
    case F_DQ: return s->dq;   case F_PHI: return s->phi; case F_DPHIX: return s->dphix;
    case F_DPHIR: return s->dphir; case F_PHIH: return s->phih;
    }
    return 0;
}
enum { P_X = 0, P_Y, P_Z, P_PX, P_PY, P_PZ, P_W, P_ID };
void *osim_particles(osim *s, int which)
{
    switch (which) {
    case P_X: return 0;      case P_Y: return s->y;   case P_Z: return s->z;
    case P_PX: return s->px; case P_PY: return s->py; case P_PZ: return s->pz;
    case P_W: return s->w;   case P_ID: return s->id;
    }
    return 0;
}
/* Lab-frame x of every particle, (ix + ox) dx, and its inverse. */
void osim_get_x(const osim *s, double *out)
{
    for (long k = 0; k < s->np; k++) out[k] = ((double)s->ix[k] + s->ox[k]) * s->dx;
}
void osim_set_x(osim *s, const double *in)
{
    for (long k = 0; k < s->np; k++) {
        double u = in[k] / s->dx, f = floor(u);
        s->ix[k] = (long)f;
        s->ox[k] = u - f;
        if (s->ox[k] >= 1.0) { s->ox[k] = 0.0; s->ix[k] += 1; }
    }
}
long osim_np(const osim *s) { return s->np; }
long osim_step_index(const osim *s) { return s->step; }
long osim_shift(const osim *s) { return s->shift; }
void osim_set_counters(osim *s, long step, long shift) { s->step = step; s->shift = shift; }
