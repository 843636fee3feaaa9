"""Pins of the oracle's deposits, loading and Maxwell coupling.

P7  charge conservation: with the charge Q_ij = sum q w S_x S_r deposited directly (here, in
    numpy) at x^n and x^{n+1}, dQ/dt + (I_x(i+1/2)-I_x(i-1/2)) + (I_r(j+1/2)-I_r(j-1/2)) = 0
    at every node, I being the oracle's J times the face area; and the discrete Gauss law
    div E - rho stays constant over full steps (Maxwell's equations conserve it exactly
    only if the current is charge-conserving and uses the same volumes).
P9  uniform cold plasma at rest: chi = n0 on every off-axis node (Sec. 2: chi is the
    density over gamma), and on the axis the fixed ratio of the lattice's deposit to the
    axis volume pi dr^2 dx / 3 (3/8 over 1/3).
Loading: the lattice weights sum to n0 times the exact annulus volumes; ids are unique.
"""
import math

import numpy as np

from oracle.oracle import OSim, splitmix64


def deposit_charge(x, y, z, w, x0, dx, dr, nx, nr):
    """Direct linear-weight charge deposit q w S on the primal nodes (q = -1)."""
    Q = np.zeros((nx + 1, nr + 1))
    xn = (x - x0) / dx
    rn = np.sqrt(y * y + z * z) / dr
    i0 = np.floor(xn).astype(int)
    j0 = np.floor(rn).astype(int)
    fx, fr = xn - i0, rn - j0
    for di, wx in ((0, 1 - fx), (1, fx)):
        for dj, wr in ((0, 1 - fr), (1, fr)):
            np.add.at(Q, (i0 + di, j0 + dj), -w * wx * wr)
    return Q


def node_volume_q(nr, dx, dr):
    v = 2 * np.pi * np.arange(nr + 1) * dr * dr * dx
    v[0] = np.pi * dr * dr * dx / 4
    return v


def _random_plasma(rng, n, nx, nr, dx, dr, margin=3):
    x = rng.uniform(margin * dx, (nx - margin) * dx, n)
    r = np.concatenate([rng.uniform(0, 1.5 * dr, n // 4), rng.uniform(0, (nr - margin) * dr, n - n // 4)])
    th = rng.uniform(0, 2 * np.pi, n)
    p = 0.6 * rng.standard_normal((3, n))
    return dict(x=x, y=r * np.cos(th), z=r * np.sin(th), px=p[0], py=p[1], pz=p[2],
                w=rng.uniform(0.5, 1.5, n) * 1e-3)


def test_p7_continuity_node_by_node():
    nx, nr, dx, dr, dt = 24, 16, 0.7, 0.9, 0.5
    rng = np.random.default_rng(1)
    s = OSim(nx, nr, dx, dr, dt, moving_window=False)
    s.set_particles(**_random_plasma(rng, 3000, nx, nr, dx, dr))
    for _ in range(3):
        before = s.particles()
        q0 = deposit_charge(before["x"], before["y"], before["z"], before["w"], 0, dx, dr, nx, nr)
        s.pass_a()
        s.envelope()
        s.pass_b()
        after = s.particles()
        q1 = deposit_charge(after["x"], after["y"], after["z"], after["w"], 0, dx, dr, nx, nr)
        jx, jr = s.field("jx"), s.field("jr")
        area_x = node_volume_q(nr, dx, dr) / dx                   # (nr+1,)
        area_r = 2 * np.pi * (np.arange(nr) + 0.5) * dr * dx     # (nr,)
        ix = np.zeros((nx + 2, nr + 1))
        ix[1:nx + 1] = jx * area_x[None, :]
        ir = np.zeros((nx + 1, nr + 1))
        ir[:, 1:] = jr * area_r[None, :]
        ir_full = np.zeros((nx + 1, nr + 2))
        ir_full[:, 1:nr + 1] = jr * area_r[None, :]
        div = (ix[1:] - ix[:-1]) + (ir_full[:, 1:] - ir_full[:, :-1])
        res = (q1 - q0) / dt + div
        scale = np.abs(div).max()
        assert scale > 0
        assert np.abs(res).max() < 1e-12 * scale
        np.testing.assert_allclose(s.field("dq"), q1 - q0, rtol=0, atol=1e-12 * np.abs(q1 - q0).max())


def test_p7_gauss_law_constant_over_full_steps():
    nx, nr, dx, dr, dt = 24, 16, 0.7, 0.9, 0.5
    rng = np.random.default_rng(2)
    s = OSim(nx, nr, dx, dr, dt, moving_window=False)
    s.set_particles(**_random_plasma(rng, 3000, nx, nr, dx, dr, margin=6))
    s.field("a")[:] = 0.2
    s.field("am")[:] = 0.2
    vol = node_volume_q(nr, dx, dr)

    def gauss():
        ex, er = s.field("ex"), s.field("er")
        exp_ = np.zeros((nx + 2, nr + 1))
        exp_[1:nx + 1] = ex
        rh = (np.arange(nr) + 0.5) * dr
        flux = np.zeros((nx + 1, nr + 2))
        flux[:, 1:nr + 1] = 2 * np.pi * dx * rh[None, :] * er
        div = (exp_[1:] - exp_[:-1]) / dx + (flux[:, 1:] - flux[:, :-1]) / vol[None, :]
        p = s.particles()
        rho = deposit_charge(p["x"], p["y"], p["z"], p["w"], 0, dx, dr, nx, nr) / vol[None, :]
        return (div - rho)[1:nx, 0:nr]

    g0 = gauss()
    for _ in range(4):
        s.step(1)
        g = gauss()
        assert np.abs(g - g0).max() < 1e-11 * np.abs(g0).max()
    assert np.abs(s.field("ex")).max() > 0  # the plasma really moved and drove fields


def test_p9_uniform_cold_plasma_chi():
    nx, nr, dx, dr = 12, 10, 0.69, 1.5
    s = OSim(nx, nr, dx, dr, 0.552, moving_window=False)
    n0 = 0.0017
    s.load_plasma(n0, 0.0, 0.0, (2, 2, 4), 0)
    assert s.np == nx * nr * 16
    s.pass_a()
    chi = s.field("chi")
    np.testing.assert_allclose(chi[1:nx, 1:nr], n0, rtol=1e-13)
    np.testing.assert_allclose(chi[1:nx, 0], n0 * (3 / 8) / (1 / 3), rtol=1e-13)


def test_loading_weights_ids_and_azimuthal_lattice():
    nx, nr, dx, dr = 10, 8, 0.7, 1.2
    s = OSim(nx, nr, dx, dr, 0.5, moving_window=False)
    n0 = 0.003
    s.load_plasma(n0, 0.0, 0.0, (2, 2, 4), 9)
    p = s.particles()
    assert len(np.unique(p["id"])) == s.np == nx * nr * 16
    total = n0 * math.pi * (nr * dr) ** 2 * nx * dx
    assert abs(p["w"].sum() / total - 1) < 1e-13
    # four azimuthal samples per (x, r) lattice point, spaced exactly pi/2, offset from SplitMix64
    th = np.arctan2(p["z"], p["y"]).reshape(-1, 4)
    d = np.mod(np.diff(th, axis=1), 2 * np.pi)
    np.testing.assert_allclose(d, np.pi / 2, atol=1e-12)
    u = (splitmix64(9, 1) >> 11) * 2.0 ** -53      # cell 0 -> first output of the stream
    assert abs(np.mod(th[0, 0], 2 * np.pi) - 2 * np.pi * u / 4) < 1e-12


def test_splitmix64_reference_value():
    # first output of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    assert splitmix64(0, 1) == 0xE220A8397B1DCDAF


def test_ramp_profile_and_window_injection():
    nx, nr, dx, dr, dt = 16, 6, 0.7, 1.5, 0.56
    s = OSim(nx, nr, dx, dr, dt, moving_window=True)
    s.load_plasma(0.01, 2.0, 5.0, (2, 2, 4), 0)
    p = s.particles()
    xs = np.unique(p["x"])
    dens = {x: p["w"][p["x"] == x].sum() for x in xs}
    # weights follow the linear ramp: density ~ (x - x_start)/ramp inside it, zero before it
    assert min(xs) > 2.0
    ratios = [dens[x] / ((x - 2.0) / 5.0) for x in xs if x < 7.0]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)
    n0 = s.np
    s.step(3)  # time 1.68 = 2.4 dx: two shifts, two fresh columns at full density
    assert s.shift == 2
    assert (p["x"] >= 2 * dx).all()  # nothing crossed the back of the window
    assert s.np == n0 + 2 * nr * 16
