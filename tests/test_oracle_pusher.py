"""Pins of the oracle's gather + Cartesian projection + ponderomotive Boris push.

P3  static envelope, E = B = 0: the ponderomotive Lorentz factor sqrt(1 + p^2 + Phi) is a
    constant of motion of Eq. (EquationsOfMotion) with force -grad(Phi)/(2 gamma); the
    error after a full passage converges with the grid.
P4  plane pulse Phi(x - t), particle at rest: gamma - p_x = 1 along the motion, p_x = Phi/2
    at the peak, p -> 0 after the pulse.
P5  pure magnetic field conserves |p| to rounding (Boris rotation); the whole push commutes
    with a rotation about the axis (cylindrical symmetry, Sec. 2), which fixes the signs of
    the Cartesian projection that the printed component equations garble.
    Force directions follow the Lorentz force of an electron.
Linear fields are gathered exactly (linear shape), including the odd radial ghost of Er.
"""
import math

import numpy as np

from oracle.oracle import OSim


def _passage(dt, h):
    nx, nr = int(60 / h), int(20 / h)
    s = OSim(nx, nr, h, h, dt, moving_window=False)
    xc, sig, phi0 = 20.0, 4.0, 0.5
    xi = np.arange(nx + 1) * h
    rj = np.arange(nr + 1) * h
    amp = np.sqrt(2 * phi0 * np.exp(-((xi[:, None] - xc) ** 2 + rj[None, :] ** 2) / sig ** 2))
    s.field("a")[:] = amp
    s.field("am")[:] = amp
    s.set_particles(x=np.array([xc - 14.0]), y=np.array([2.0]), z=np.array([1.0]),
                    px=np.array([0.6]), py=np.array([0.05]), pz=np.array([0.0]), w=np.array([0.0]))
    g0 = math.sqrt(1 + 0.6 ** 2 + 0.05 ** 2)
    worst = 0.0
    for _ in range(int(round(80.0 / dt))):
        s.pass_a()
        x, y, z = s.part("x")[0], s.part("y")[0], s.part("z")[0]
        s.pass_b()
        p = np.array([s.part("px")[0], s.part("py")[0], s.part("pz")[0]])
        xm = 0.5 * (x + s.part("x")[0])
        ym = 0.5 * (y + s.part("y")[0])
        zm = 0.5 * (z + s.part("z")[0])
        phi = phi0 * math.exp(-((xm - xc) ** 2 + ym * ym + zm * zm) / sig ** 2)
        worst = max(worst, abs(math.sqrt(1 + p @ p + phi) / g0 - 1))
    # the particle was deflected by the bump: the invariant was exercised
    assert abs(s.part("py")[0]) > 0.3
    return worst


def test_p3_static_envelope_invariant_converges():
    e_coarse = _passage(0.04, 0.2)
    e_fine = _passage(0.04, 0.1)
    assert e_coarse < 1.2e-4
    assert e_coarse / e_fine > 2.5, (e_coarse, e_fine)


def _plane_pulse(dt, dx, a0=0.5, L=10.0):
    nx, nr, dr = int(250 / dx), 4, 1.0
    s = OSim(nx, nr, dx, dr, dt, moving_window=False)
    xi = np.arange(nx + 1) * dx
    xs, xp = 40.0, 100.0

    def env(t):
        return np.repeat((a0 * np.exp(-((xi - xs - t) / L) ** 2))[:, None], nr + 1, axis=1)

    s.set_particles(x=np.array([xp]), y=np.array([1.5]), z=np.array([0.0]), w=np.array([0.0]))
    inv, pxs = [], []
    for k in range(int((xp - xs + 4 * L + 20) / dt)):
        s.field("a")[:] = env(k * dt)
        s.field("am")[:] = env((k - 1) * dt)
        s.pass_a()
        s.field("a")[:] = env((k + 1) * dt)
        s.field("am")[:] = env(k * dt)
        x0 = s.part("x")[0]
        s.pass_b()
        px, py, pz = s.part("px")[0], s.part("py")[0], s.part("pz")[0]
        xm = 0.5 * (x0 + s.part("x")[0])
        phi = 0.5 * a0 ** 2 * math.exp(-2 * ((xm - xs - (k + 0.5) * dt) / L) ** 2)
        inv.append(math.sqrt(1 + px * px + py * py + pz * pz + phi) - px - 1)
        pxs.append(px)
    pfinal = np.array([s.part("px")[0], s.part("py")[0], s.part("pz")[0]])
    return max(np.abs(inv)), max(pxs) / (a0 ** 2 / 4) - 1, np.abs(pfinal).max()


def test_p4_plane_pulse_lightfront_invariant():
    inv1, peak1, pend1 = _plane_pulse(0.2, 0.5)
    inv2, peak2, pend2 = _plane_pulse(0.2, 0.25)
    assert inv1 < 2.5e-4 and inv2 < 6e-5
    assert inv1 / inv2 > 3.0
    assert abs(peak1) < 5e-3 and abs(peak2) < 1.5e-3
    assert pend1 < 1e-4 and pend2 < 1e-5


def _random_fields(s, rng, scale=0.05):
    for name in ("ex", "er", "bt"):
        f = s.field(name)
        f[:] = scale * rng.standard_normal(f.shape)
    s.field("btn")[:] = s.field("bt")
    a = 0.3 * (rng.standard_normal(s.field("a").shape) + 1j * rng.standard_normal(s.field("a").shape))
    s.field("a")[:] = a
    s.field("am")[:] = a


def test_p5_pure_magnetic_field_conserves_momentum_magnitude():
    rng = np.random.default_rng(5)
    s = OSim(32, 16, 1.0, 1.0, 0.5, moving_window=False)
    s.field("bt")[:] = 0.3 * rng.standard_normal(s.field("bt").shape)
    n = 64
    r = rng.uniform(0, 12, n)
    th = rng.uniform(0, 2 * np.pi, n)
    p = rng.standard_normal((3, n))
    s.set_particles(x=rng.uniform(8, 24, n), y=r * np.cos(th), z=r * np.sin(th),
                    px=p[0], py=p[1], pz=p[2], w=np.zeros(n))
    p0 = np.sqrt(p[0] ** 2 + p[1] ** 2 + p[2] ** 2)
    for _ in range(20):
        s.faraday()  # E = 0 keeps B constant and sets B^n = B
        s.pass_a()
        s.pass_b()
    pn = np.sqrt(s.part("px") ** 2 + s.part("py") ** 2 + s.part("pz") ** 2)
    assert np.max(np.abs(pn / p0 - 1)) < 1e-13


def test_p5_rotation_about_axis_commutes_with_push():
    rng = np.random.default_rng(7)
    n = 200
    x = rng.uniform(6, 26, n)
    r = rng.uniform(0, 12, n)
    th = rng.uniform(0, 2 * np.pi, n)
    p = 0.3 * rng.standard_normal((3, n))
    alpha = 0.731
    ca, sa = math.cos(alpha), math.sin(alpha)
    finals = []
    for rot in (False, True):
        s = OSim(32, 16, 1.0, 1.0, 0.5, moving_window=False)
        _random_fields(s, np.random.default_rng(11))
        y, z = r * np.cos(th), r * np.sin(th)
        py, pz = p[1], p[2]
        if rot:
            y, z = ca * y - sa * z, sa * y + ca * z
            py, pz = ca * p[1] - sa * p[2], sa * p[1] + ca * p[2]
        s.set_particles(x=x, y=y, z=z, px=p[0], py=py, pz=pz, w=np.ones(n) * 1e-3)
        for _ in range(3):
            s.pass_a()
            s.pass_b()
        st = s.particles()
        if rot:  # rotate back
            st["y"], st["z"] = ca * st["y"] + sa * st["z"], -sa * st["y"] + ca * st["z"]
            st["py"], st["pz"] = ca * st["py"] + sa * st["pz"], -sa * st["py"] + ca * st["pz"]
        finals.append(st)
    for k in ("x", "y", "z", "px", "py", "pz"):
        np.testing.assert_allclose(finals[0][k], finals[1][k], rtol=0, atol=1e-12)


def _one_kick(field, value, p=(0.0, 0.0, 0.0), y=3.0, z=0.0):
    s = OSim(16, 8, 1.0, 1.0, 0.5, moving_window=False)
    if field == "bt":
        s.field("btn")[:] = value
    elif field == "phi_r":  # Phi increasing with r
        rj = np.arange(9) * 1.0
        s.field("a")[:] = np.sqrt(2 * value * rj)[None, :]
    else:
        s.field(field)[:] = value
    s.set_particles(x=np.array([8.3]), y=np.array([y]), z=np.array([z]), px=np.array([p[0]]),
                    py=np.array([p[1]]), pz=np.array([p[2]]), w=np.array([0.0]))
    s.pass_a()
    return s.part("px")[0], s.part("py")[0], s.part("pz")[0]


def test_force_directions_of_an_electron():
    px, _, _ = _one_kick("ex", 0.1)
    assert px < 0                                  # F = qE, q = -1
    _, py, pz = _one_kick("er", 0.1)
    assert py < 0 and abs(pz) < 1e-15              # radial E>0 pulls the electron inward
    _, py, _ = _one_kick("bt", 0.2, p=(0.5, 0.0, 0.0))
    assert py > 0                                  # q v x B: +x motion in B_theta>0 pushes out
    _, py, _ = _one_kick("phi_r", 0.05)
    assert py < 0                                  # ponderomotive force points down grad(Phi)
    _, py, pz = _one_kick("er", 0.1, y=0.0, z=3.0)
    assert pz < 0 and abs(py) < 1e-15              # same physics at theta = pi/2


def test_linear_fields_gathered_exactly_with_odd_radial_ghost():
    dx, dr, dt = 0.8, 1.1, 0.5
    s = OSim(20, 12, dx, dr, dt, moving_window=False)
    xh = (np.arange(20) + 0.5) * dx
    rj = np.arange(13) * dr
    xn = np.arange(21) * dx
    rh = (np.arange(12) + 0.5) * dr
    s.field("ex")[:] = 0.01 + 0.002 * xh[:, None] - 0.003 * rj[None, :]
    s.field("er")[:] = (0.004 + 0.001 * xn[:, None]) * rh[None, :]   # odd in r, linear
    rng = np.random.default_rng(3)
    n = 100
    x = rng.uniform(2, 14, n)
    r = np.concatenate([rng.uniform(0, 0.5 * dr, 20), rng.uniform(0, 9, n - 20)])
    th = rng.uniform(0, 2 * np.pi, n)
    s.set_particles(x=x, y=r * np.cos(th), z=r * np.sin(th), w=np.zeros(n))
    s.pass_a()
    ex = 0.01 + 0.002 * x - 0.003 * r
    er = (0.004 + 0.001 * x) * r
    # E only: Boris with B = 0 gives p = q E dt exactly; er*cos etc. for the Cartesian part
    np.testing.assert_allclose(s.part("px"), -dt * ex, rtol=0, atol=1e-15)
    np.testing.assert_allclose(s.part("py"), -dt * er * np.cos(th), rtol=0, atol=1e-15)
    np.testing.assert_allclose(s.part("pz"), -dt * er * np.sin(th), rtol=0, atol=1e-15)


def test_uniform_ex_gives_exact_momentum_and_hyperbolic_motion():
    e0, dt = 0.05, 0.1
    s = OSim(400, 8, 0.5, 1.0, dt, moving_window=False)
    s.field("ex")[:] = e0
    x0 = 150.0
    s.set_particles(x=np.array([x0]), y=np.array([2.0]), z=np.array([0.0]), w=np.array([0.0]))
    nst = 1000
    for _ in range(nst):
        s.pass_a()
        s.pass_b()
    # leapfrog: p^{n+1/2} = -e0 (n+1) dt exactly
    assert abs(s.part("px")[0] + e0 * nst * dt) < 1e-12
    t = nst * dt
    x_exact = x0 - (math.sqrt(1 + (e0 * t) ** 2) - 1) / e0
    assert abs(s.part("x")[0] - x_exact) < 2e-3 * abs(x_exact - x0)
