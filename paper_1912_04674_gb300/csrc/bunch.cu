// Externally injected relativistic bunch (Sec. 3: the field initialisation of a bunch in
// uniform motion, carried over to cylindrical symmetry): the bunch is appended to the particle
// set and the fields of a charge moving along x at beta are added to E and B,
//   E = -(dphi/dx / gamma^2, dphi/dr),  B_theta = beta E_r (at t - dt/2),
// phi solving the flux-form discrete Gauss law of the Yee grid on the nodes (i, j), j < Nr:
//   sum over the four faces of (area x flux) = Q_ij,
// which is symmetric positive definite: x faces couple (i, j) to (i +- 1, j) with
// cx_j = A_j / (gamma^2 dx) (A_j the ring area of the charge volume, pi dr^2/4 on the axis),
// r faces couple (i, j) to (i, j +- 1) with cr_j = 2 pi dx r_{j+1/2} / dr, no flux through the
// window's x ends and phi = 0 on the wall j = Nr.  Solved by conjugate gradients preconditioned
// with the radial line of each column (the x coupling is 1/gamma^2 weaker).  Vectors are FP64
// in the caller's scratch buffer, indexed i*Nr + j.
#include <vector>

#include "lpic_internal.cuh"

namespace lpic {

namespace {

constexpr int TB = 256;

struct Coef {
    double dx, dr, g2;   // g2 = gamma^2
};
__device__ __forceinline__ double ring_area(const Coef &c, int j) {
    return j == 0 ? kPi * 0.25 * c.dr * c.dr : 2.0 * kPi * j * c.dr * c.dr;
}
__device__ __forceinline__ double cx_of(const Coef &c, int j) { return ring_area(c, j) / (c.g2 * c.dx); }
__device__ __forceinline__ double cr_of(const Coef &c, int j) { return 2.0 * kPi * c.dx * (j + 0.5); }   // 2 pi dx r_{j+1/2} / dr

// Q_ij = sum q w S_x S_r of the bunch particles in slots [k0, k0 + n) (q = -1), from the values
// the simulation holds (so that the initial field matches the charge the deposits will move)
template <class R>
__global__ void k_bunch_charge(SimDev<R> S, int k0, int n, double *__restrict__ q) {
    const Parts<R> P = S.d->pbuf ? S.p[1] : S.p[0];
    const long long shift = S.d->shift;
    const int nx = S.geo.nx, nr = S.geo.nr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int k = k0 + t;
        if (P.ix[k] == kDead) continue;
        const double y = P.y[k], z = P.z[k], w = P.w[k];
        const int i0 = (int)((long long)P.ix[k] - shift);
        const double fx = P.ox[k], rn = sqrt(y * y + z * z) / S.ph.dr;
        const int j0 = (int)floor(rn);
        const double fr = rn - j0;
        for (int di = 0; di < 2; di++)
            for (int dj = 0; dj < 2; dj++) {
                const int i = i0 + di, j = j0 + dj;
                if (i < 0 || i > nx || j < 0 || j >= nr) continue;   // phi = 0 on the wall j = Nr
                atomicAdd(q + (size_t)i * nr + j, -w * (di ? fx : 1.0 - fx) * (dj ? fr : 1.0 - fr));
            }
    }
}

// y = K x
__global__ void k_bunch_apply(Coef c, int nx, int nr, const double *__restrict__ x, double *__restrict__ y) {
    const long long n = (long long)(nx + 1) * nr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / nr), j = (int)(t - (long long)i * nr);
        const double cx = cx_of(c, j), crp = cr_of(c, j), crm = j > 0 ? cr_of(c, j - 1) : 0.0;
        const double v = x[t];
        double acc = (crp + crm) * v;
        if (j + 1 < nr) acc -= crp * x[t + 1];
        if (j > 0) acc -= crm * x[t - 1];
        if (i > 0) acc += cx * (v - x[t - nr]);
        if (i < nx) acc += cx * (v - x[t + nr]);
        y[t] = acc;
    }
}

// z = M^-1 r, M the radial tridiagonal line of each column with the x coupling on its diagonal
// (Thomas algorithm, one thread per column).  The elimination factors depend only on j and on
// whether the column is an end column (one x neighbour) or not (two): tab holds, for each,
// 1/den_j and the modified upper diagonal c'_j, computed once on the host.
__global__ void k_bunch_precond(Coef c, int nx, int nr, const double *__restrict__ tab, const double *__restrict__ r,
                                double *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nx) return;
    const double *inv = tab + (i > 0 && i < nx ? 0 : 2 * nr), *cpj = inv + nr;
    const size_t base = (size_t)i * nr;
    double prev = 0.0;
    for (int j = 0; j < nr; j++) {
        const double lower = j > 0 ? -cr_of(c, j - 1) : 0.0;
        prev = (r[base + j] - lower * prev) * inv[j];
        z[base + j] = prev;
    }
    for (int j = nr - 2; j >= 0; j--) z[base + j] -= cpj[j] * z[base + j + 1];
}

// out[slot] += sum a_t b_t
__global__ void k_bunch_dot(const double *__restrict__ a, const double *__restrict__ b, long long n, double *out) {
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        s += a[t] * b[t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double sh[TB / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < TB / 32; q++) t += sh[q];
        atomicAdd(out, t);
    }
}

// x += alpha p, r -= alpha Ap
__global__ void k_bunch_update(double alpha, long long n, const double *__restrict__ p, const double *__restrict__ ap,
                               double *__restrict__ x, double *__restrict__ r) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        x[t] += alpha * p[t];
        r[t] -= alpha * ap[t];
    }
}

// p = z + beta p
__global__ void k_bunch_direction(double beta, long long n, const double *__restrict__ z, double *__restrict__ p) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        p[t] = z[t] + beta * p[t];
}

// Add the bunch fields from phi to E^n and B^{n-1/2}.
template <class R>
__global__ void k_bunch_fields(SimDev<R> S, Coef c, double beta, double f, const double *__restrict__ phi) {
    const Geo g = S.geo;
    const int off = S.d->off, nx = g.nx, nr = g.nr;
    auto ph = [&](int i, int j) { return j < nr ? phi[(size_t)i * nr + j] : 0.0; };
    const long long n = (long long)(nx + 1) * (nr + 1);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / (nr + 1)), j = (int)(t - (long long)i * (nr + 1));
        const long long id = g.at(off, i, j);
        if (i < nx) S.f.ex[id] += (R)(-(ph(i + 1, j) - ph(i, j)) / (c.g2 * c.dx));
        if (j < nr) {
            const double er_i = -(ph(i, j + 1) - ph(i, j)) / c.dr;
            if (i > 0 && i < nx) S.f.er[id] += (R)er_i;    // Er = 0 on the x ends (conductor)
            if (i < nx) {
                const double er_n = -(ph(i + 1, j + 1) - ph(i + 1, j)) / c.dr;
                S.f.bt[id] += (R)(beta * ((1.0 - f) * er_i + f * er_n));
            }
        }
    }
}

inline int grid_for(long long n) {
    long long b = (n + TB - 1) / TB;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

size_t bunch_scratch_bytes(const Geo &g) {
    return (6 * (size_t)(g.nx + 1) * g.nr + 4 * (size_t)g.nr) * sizeof(double) + 256;
}

template <class R>
int bunch_solve_and_add(const SimDev<R> &S, int k0, int n, double gamma, void *scratch, double *d_dot, double tol,
                        int max_iter, cudaStream_t st, double *res_out) {
    const Geo g = S.geo;
    const int nx = g.nx, nr = g.nr;
    const long long m = (long long)(nx + 1) * nr;
    double *q = (double *)scratch, *x = q + m, *r = x + m, *z = r + m, *p = z + m, *ap = p + m, *tab = ap + m;
    const Coef c{S.ph.dx, S.ph.dr, gamma * gamma};
    {   // elimination factors of the line preconditioner: inner columns, then end columns
        std::vector<double> h(4 * (size_t)nr);
        for (int e = 0; e < 2; e++) {
            const double nxn = e == 0 ? 2.0 : 1.0;
            double *inv = h.data() + 2 * (size_t)nr * e, *cpj = inv + nr, prev_c = 0.0;
            for (int j = 0; j < nr; j++) {
                const double area = j == 0 ? kPi * 0.25 * c.dr * c.dr : 2.0 * kPi * j * c.dr * c.dr;
                const double crp = 2.0 * kPi * c.dx * (j + 0.5), crm = j > 0 ? 2.0 * kPi * c.dx * (j - 0.5) : 0.0;
                const double diag = crp + crm + nxn * area / (c.g2 * c.dx);
                const double lower = j > 0 ? -crm : 0.0, upper = j + 1 < nr ? -crp : 0.0;
                const double den = diag - lower * prev_c;
                inv[j] = 1.0 / den;
                prev_c = upper / den;
                cpj[j] = prev_c;
            }
        }
        cudaMemcpyAsync(tab, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);   // h is a host temporary
    }
    const double beta = sqrt(1.0 - 1.0 / (gamma * gamma));
    cudaMemsetAsync(q, 0, 2 * m * sizeof(double), st);   // q and x
    if (n > 0) k_bunch_charge<R><<<grid_for(n), TB, 0, st>>>(S, k0, n, q);
    cudaMemcpyAsync(r, q, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
    auto dot = [&](const double *a, const double *b) -> double {
        double h = 0.0;
        cudaMemsetAsync(d_dot, 0, sizeof(double), st);
        k_bunch_dot<<<grid_for(m), TB, 0, st>>>(a, b, m, d_dot);
        cudaMemcpyAsync(&h, d_dot, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return h;
    };
    const double bb = dot(q, q);
    int it = 0;
    double rr = bb;
    if (bb > 0) {
        k_bunch_precond<<<(nx + 1 + TB - 1) / TB, TB, 0, st>>>(c, nx, nr, tab, r, z);
        cudaMemcpyAsync(p, z, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
        double rz = dot(r, z);
        for (it = 1; it <= max_iter; it++) {
            k_bunch_apply<<<grid_for(m), TB, 0, st>>>(c, nx, nr, p, ap);
            const double pap = dot(p, ap);
            if (!(pap > 0)) break;
            const double alpha = rz / pap;
            k_bunch_update<<<grid_for(m), TB, 0, st>>>(alpha, m, p, ap, x, r);
            rr = dot(r, r);
            if (rr <= tol * tol * bb) break;
            k_bunch_precond<<<(nx + 1 + TB - 1) / TB, TB, 0, st>>>(c, nx, nr, tab, r, z);
            const double rz_new = dot(r, z);
            k_bunch_direction<<<grid_for(m), TB, 0, st>>>(rz_new / rz, m, z, p);
            rz = rz_new;
        }
    }
    if (res_out) *res_out = bb > 0 ? sqrt(rr / bb) : 0.0;
    const double f = 0.5 + beta * S.ph.dt / (2.0 * S.ph.dx);
    k_bunch_fields<R><<<grid_for((long long)(nx + 1) * (nr + 1)), TB, 0, st>>>(S, c, beta, f, x);
    return it;
}

#define INST(R)                                                                                   \
    template int bunch_solve_and_add<R>(const SimDev<R> &, int, int, double, void *, double *, double, \
                                        int, cudaStream_t, double *);
INST(double)
INST(float)
#undef INST

}  // namespace lpic
