"""Pin P10: brute-force recomputation of every stencil and deposit of the oracle on an 8 x 8
grid, node by node, at 50 significant digits.

The reference below is written from the equations (Sec. 2-3: Eqs. MaxwellEqsCylindrical,
envelope_solver, EquationsOfMotion, motion_equations_cartesian) and the readings of the
paper listed in the design notes (G1-G9), in a deliberately different form from the
oracle: linear shape factors are hat functions of the distance to *every* node of a
(staggered) grid, summed over the whole grid instead of a two-node window, radial odd
ghosts are explicit mirror nodes at r = -dr/2, and the Esirkepov prefix sums run over the
whole column.  Each phase of the oracle is run alone on random fields and particles and
compared with the reference to 1e-13 of the largest value.
"""
import numpy as np
import pytest

from oracle.oracle import OSim

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

NX, NR, DX, DR, DT = 8, 8, 0.69, 1.5, 0.5
TOL = 1e-13
Q = -1


def M(v):
    return mp.mpf(float(v))


def fresh(seed):
    o = OSim(NX, NR, DX, DR, DT, False)
    rng = np.random.default_rng(seed)
    for name in ("ex", "er", "bt", "btn", "jx", "jr", "chi"):
        f = o.field(name)
        f[:] = rng.standard_normal(f.shape)
    for name in ("a", "am"):
        f = o.field(name)
        f[:] = rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)
    return o, rng


def close(got, want):
    got = np.asarray(got, dtype=complex if np.iscomplexobj(got) else float)
    want = np.asarray(want, dtype=got.dtype)
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max() / scale
    assert err < TOL, err


def hat(u):
    """Linear shape factor of a point at distance u (in cells) from a node."""
    u = abs(u)
    return 1 - u if u < 1 else mp.mpf(0)


# ---------------------------------------------------------------- Yee (Eq. MaxwellEqsCylindrical)
def test_p10_faraday():
    o, _ = fresh(1)
    ex, er, b0 = o.field("ex").copy(), o.field("er").copy(), o.field("bt").copy()
    o.faraday()
    want = np.zeros((NX, NR))
    wantn = np.zeros((NX, NR))
    for i in range(NX):          # Bt at (i+1/2, j+1/2)
        for j in range(NR):
            curl = (M(ex[i, j + 1]) - M(ex[i, j])) / M(DR) - (M(er[i + 1, j]) - M(er[i, j])) / M(DX)
            bn = M(b0[i, j]) + M(DT) * curl
            want[i, j] = float(bn)
            wantn[i, j] = float((M(b0[i, j]) + bn) / 2)
    close(o.field("bt"), want)
    close(o.field("btn"), wantn)


def test_p10_ampere():
    o, _ = fresh(2)
    ex, er, bt = o.field("ex").copy(), o.field("er").copy(), o.field("bt").copy()
    jx, jr = o.field("jx").copy(), o.field("jr").copy()
    o.ampere()
    want_er = np.zeros_like(er)
    for i in range(NX + 1):      # Er at (i, j+1/2); perfect conductor at both x ends
        for j in range(NR):
            if i in (0, NX):
                continue
            want_er[i, j] = float(M(er[i, j]) + M(DT) * (-(M(bt[i, j]) - M(bt[i - 1, j])) / M(DX) - M(jr[i, j])))
    want_ex = np.zeros_like(ex)
    for i in range(NX):          # Ex at (i+1/2, j); Ex = 0 at r_max
        for j in range(NR + 1):
            if j == NR:
                continue
            if j == 0:           # Stokes on the disc r < dr/2: 2 pi (dr/2) B / (pi (dr/2)^2)
                rot = 2 * mp.pi * (M(DR) / 2) * M(bt[i, 0]) / (mp.pi * (M(DR) / 2) ** 2)
            else:
                rp, rm, rj = (j + mp.mpf(1) / 2) * M(DR), (j - mp.mpf(1) / 2) * M(DR), j * M(DR)
                rot = (rp * M(bt[i, j]) - rm * M(bt[i, j - 1])) / (rj * M(DR))
            want_ex[i, j] = float(M(ex[i, j]) + M(DT) * (rot - M(jx[i, j])))
    close(o.field("er"), want_er)
    close(o.field("ex"), want_ex)


# ---------------------------------------------------------------- envelope (Eq. envelope_solver)
def test_p10_envelope():
    o, _ = fresh(3)
    a, am, chi = o.field("a").copy(), o.field("am").copy(), o.field("chi").copy()
    o.envelope()

    def A(i, j):                 # Dirichlet 0 outside; even in r across the axis
        if i < 0 or i > NX or j > NR:
            return mp.mpc(0)
        if j < 0:
            j = -j
        return mp.mpc(a[i, j].real, a[i, j].imag)

    dt, dx, dr = M(DT), M(DX), M(DR)
    want = np.zeros_like(a)
    for i in range(NX + 1):
        for j in range(NR + 1):
            c = A(i, j)
            lap_x = (A(i + 1, j) - 2 * c + A(i - 1, j)) / dx**2
            if j == 0:
                # (1/r) d/dr (r dA/dr) -> 2 d2A/dr2 on the axis; with the even ghost
                # A(-1) = A(1) this is 4 (A_1 - A_0) / dr^2
                lap_r = 2 * (A(i, 1) - 2 * c + A(i, -1)) / dr**2
            else:
                lap_r = (A(i, j + 1) - 2 * c + A(i, j - 1)) / dr**2 + (A(i, j + 1) - A(i, j - 1)) / (2 * dr * j * dr)
            d_x = (A(i + 1, j) - A(i - 1, j)) / (2 * dx)
            bracket = lap_x + lap_r - M(chi[i, j]) * c + 2j * d_x
            # (A+ - 2A + A-)/dt^2 - 2i (A+ - A-)/(2dt) = bracket, solved for A+
            rhs = 2 * c - mp.mpc(am[i, j].real, am[i, j].imag) * (1 + 1j * dt) + dt**2 * bracket
            want[i, j] = complex(rhs / (1 - 1j * dt))
    close(o.field("a"), want)
    close(o.field("am"), a)


# ---------------------------------------------------------------- particles
def particles(rng, n=6):
    x = rng.uniform(1.5 * DX, 6.0 * DX, n)
    r = np.concatenate([[0.2 * DR, 0.45 * DR], rng.uniform(0.6 * DR, 6.0 * DR, n - 2)])
    th = rng.uniform(0, 2 * np.pi, n)
    return dict(x=x, y=r * np.cos(th), z=r * np.sin(th), px=0.3 * rng.standard_normal(n),
                py=0.3 * rng.standard_normal(n), pz=0.3 * rng.standard_normal(n),
                w=rng.uniform(0.5, 2.0, n))


def gather_hat(F, x, r, sx, sr, odd):
    """Sum over every point of a grid whose point (i, j) sits at ((i+sx) dx, (j+sr) dr)."""
    ni, nj = F.shape
    acc = mp.mpf(0)
    for i in range(ni):
        wx = hat(x / M(DX) - (i + sx))
        if wx == 0:
            continue
        for j in range(nj):
            acc += wx * hat(r / M(DR) - (j + sr)) * M(F[i, j])
        if odd:                  # mirror point below the axis carries -F(i, 0)
            acc += wx * hat(r / M(DR) - (-1 + sr)) * (-M(F[i, 0]))
    return acc


def node_phi(a):
    return np.array([[float((M(v.real) ** 2 + M(v.imag) ** 2) / 2) for v in row] for row in a])


def v_chi(j):
    return mp.pi * M(DR) ** 2 * M(DX) / 3 if j == 0 else 2 * mp.pi * j * M(DR) ** 2 * M(DX)


def v_q(j):
    return mp.pi * (M(DR) / 2) ** 2 * M(DX) if j == 0 else 2 * mp.pi * j * M(DR) ** 2 * M(DX)


def test_p10_pass_a():
    o, rng = fresh(4)
    p = particles(rng)
    o.set_particles(**p)
    ex, er, btn, a = o.field("ex").copy(), o.field("er").copy(), o.field("btn").copy(), o.field("a").copy()
    o.pass_a()
    phi = node_phi(a)
    # centred differences of Phi at the nodes; Phi = 0 outside [0, Nx] and above Nr; 0 on the axis
    P = lambda i, j: M(phi[i, j]) if 0 <= i <= NX and 0 <= j <= NR else mp.mpf(0)  # noqa: E731
    gx = np.array([[float((P(i + 1, j) - P(i - 1, j)) / (2 * M(DX))) for j in range(NR + 1)] for i in range(NX + 1)])
    gr = np.array([[0.0 if j == 0 else float((P(i, j + 1) - P(i, j - 1)) / (2 * M(DR)))
                    for j in range(NR + 1)] for i in range(NX + 1)])
    chi = [[mp.mpf(0)] * (NR + 1) for _ in range(NX + 1)]
    hdt = M(DT) / 2
    mom = []
    for k in range(len(p["x"])):
        x, y, z = M(p["x"][k]), M(p["y"][k]), M(p["z"][k])
        r = mp.sqrt(y * y + z * z)
        c, s = (y / r, z / r) if r > 0 else (mp.mpf(1), mp.mpf(0))
        Ex = gather_hat(ex, x, r, 0.5, 0.0, False)
        Er = gather_hat(er, x, r, 0.0, 0.5, True)
        Bt = gather_hat(btn, x, r, 0.5, 0.5, True)
        ph = gather_hat(phi, x, r, 0.0, 0.0, False)
        Gx, Gr = gather_hat(gx, x, r, 0, 0, False), gather_hat(gr, x, r, 0, 0, False)
        E = mp.matrix([Ex, Er * c, Er * s])
        B = mp.matrix([0, -Bt * s, Bt * c])
        G = mp.matrix([Gx, Gr * c, Gr * s])
        pv = mp.matrix([M(p["px"][k]), M(p["py"][k]), M(p["pz"][k])])
        g0 = mp.sqrt(1 + (pv.T * pv)[0] + ph)
        pstar = pv + hdt * (Q * E - G / (2 * g0))
        gt = mp.sqrt(1 + (pstar.T * pstar)[0] + ph)
        for i in range(NX + 1):
            for j in range(NR + 1):
                sw = hat(x / M(DX) - i) * hat(r / M(DR) - j)
                if sw:
                    chi[i][j] += Q * Q * M(p["w"][k]) * sw / (gt * v_chi(j))
        F = Q * E - G / (2 * gt)
        pm = pv + hdt * F
        gm = mp.sqrt(1 + (pm.T * pm)[0] + ph)
        t = Q * B * hdt / gm
        sv = 2 * t / (1 + (t.T * t)[0])
        cross = lambda u, v: mp.matrix([u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]])  # noqa: E731
        pp = pm + cross(pm, t)
        pn = pm + cross(pp, sv) + hdt * F
        mom.append([float(pn[0]), float(pn[1]), float(pn[2])])
    mom = np.array(mom)
    close(np.stack([o.part("px"), o.part("py"), o.part("pz")], 1), mom)
    close(o.field("chi"), np.array([[float(v) for v in row] for row in chi]))


def test_p10_pass_b():
    o, rng = fresh(5)
    p = particles(rng)
    o.set_particles(**p)
    a, am = o.field("a").copy(), o.field("am").copy()
    o.pass_b()
    phih = (node_phi(a) + node_phi(am)) / 2          # (Phi^{n+1} + Phi^n)/2 at the nodes
    jx = [[mp.mpf(0)] * (NR + 1) for _ in range(NX)]
    jr = [[mp.mpf(0)] * NR for _ in range(NX + 1)]
    dq = [[mp.mpf(0)] * (NR + 1) for _ in range(NX + 1)]
    pos = []
    for k in range(len(p["x"])):
        x0, y0, z0 = M(p["x"][k]), M(p["y"][k]), M(p["z"][k])
        r0 = mp.sqrt(y0 * y0 + z0 * z0)
        pv = [M(p["px"][k]), M(p["py"][k]), M(p["pz"][k])]
        ph = gather_hat(phih, x0, r0, 0.0, 0.0, False)
        gb = mp.sqrt(1 + sum(v * v for v in pv) + ph)
        x1, y1, z1 = (x0 + M(DT) * pv[0] / gb, y0 + M(DT) * pv[1] / gb, z0 + M(DT) * pv[2] / gb)
        r1 = mp.sqrt(y1 * y1 + z1 * z1)
        pos.append([float(x1), float(y1), float(z1)])
        qw = Q * M(p["w"][k])
        S0x = [hat(x0 / M(DX) - i) for i in range(NX + 1)]
        S1x = [hat(x1 / M(DX) - i) for i in range(NX + 1)]
        S0r = [hat(r0 / M(DR) - j) for j in range(NR + 1)]
        S1r = [hat(r1 / M(DR) - j) for j in range(NR + 1)]
        for i in range(NX + 1):
            for j in range(NR + 1):
                dq[i][j] += qw * (S1x[i] * S1r[j] - S0x[i] * S0r[j])
        # Esirkepov weights and their prefix sums over the whole column / row
        for j in range(NR + 1):
            run = mp.mpf(0)
            for i in range(NX):
                run += (S1x[i] - S0x[i]) * (S0r[j] + (S1r[j] - S0r[j]) / 2)
                jx[i][j] += -qw / M(DT) * run * M(DX) / v_q(j)
        for i in range(NX + 1):
            run = mp.mpf(0)
            for j in range(NR):
                run += (S1r[j] - S0r[j]) * (S0x[i] + (S1x[i] - S0x[i]) / 2)
                jr[i][j] += -qw / M(DT) * run / (2 * mp.pi * (j + mp.mpf(1) / 2) * M(DR) * M(DX))
    close(np.stack([o.part("x"), o.part("y"), o.part("z")], 1), np.array(pos))
    close(o.field("jx"), np.array([[float(v) for v in row] for row in jx]))
    close(o.field("jr"), np.array([[float(v) for v in row] for row in jr]))
    close(o.field("dq"), np.array([[float(v) for v in row] for row in dq]))
