"""Pins of the oracle's current filter (Sec. 4: an uncompensated binomial filter of 7 passes
applied against numerical Cherenkov radiation).

Reading: a pass replaces F_i by (F_{i-1} + 2 F_i + F_{i+1}) / 4 along x, F = 0 outside the
window, on Jx, Jr and the step's charge change.  Pinned by: the impulse response of 7 passes,
which must be the binomial coefficients C(14, k) / 2^14 (the expansion of ((1 + z)/2)^14);
the transfer function cos(kappa/2)^14 of a cosine away from the ends; the zero-outside
boundary (one pass of an edge impulse keeps 3/4 of it); mirror symmetry; and the continuity
equation, which the filtered current must keep with the identically filtered charge.
"""
import math

import numpy as np

from oracle.oracle import OSim

from test_oracle_deposit import _random_plasma, deposit_charge, node_volume_q

PASSES = 7


def test_impulse_response_is_binomial():
    o = OSim(48, 8, 0.69, 1.5, 0.5, False)
    o.set_filter(PASSES)
    for name, j in (("jx", 3), ("jr", 5), ("dq", 0)):
        f = o.field(name)
        f[:] = 0.0
        f[20, j] = 1.0
    o.filter()
    want = np.array([math.comb(2 * PASSES, k) for k in range(2 * PASSES + 1)]) / 2.0 ** (2 * PASSES)
    for name, j in (("jx", 3), ("jr", 5), ("dq", 0)):
        f = o.field(name)
        np.testing.assert_array_equal(f[20 - PASSES:21 + PASSES, j], want)   # exact (dyadic)
        assert np.count_nonzero(f) == 2 * PASSES + 1                         # x only, no radial spread


def test_cosine_transfer_function():
    nx, nr = 64, 6
    o = OSim(nx, nr, 0.69, 1.5, 0.5, False)
    o.set_filter(PASSES)
    for kappa in (0.3, 1.1, 2.5):
        f = o.field("jx")
        i = np.arange(nx)[:, None]
        f[:] = np.cos(kappa * i + 0.4) * np.ones((1, nr + 1))
        before = f.copy()
        o.filter()
        inner = slice(PASSES, nx - PASSES)
        gain = np.cos(kappa / 2) ** (2 * PASSES)
        np.testing.assert_allclose(o.field("jx")[inner], gain * before[inner], rtol=0, atol=1e-14)


def test_zero_outside_and_mirror_symmetry():
    o = OSim(16, 4, 0.69, 1.5, 0.5, False)
    o.set_filter(1)
    f = o.field("jx")
    f[:] = 0.0
    f[0, 2] = 1.0                      # an impulse on the first face
    o.filter()
    g = o.field("jx")
    assert g[0, 2] == 0.5 and g[1, 2] == 0.25 and g[:, 2].sum() == 0.75
    rng = np.random.default_rng(3)
    o.set_filter(PASSES)
    f = o.field("jr")
    v = rng.standard_normal(f.shape)
    f[:] = v
    o.filter()
    a = o.field("jr").copy()
    o.field("jr")[:] = v[::-1]
    o.filter()
    np.testing.assert_allclose(o.field("jr")[::-1], a, rtol=0, atol=1e-15)


def binomial_x(q):
    """7 passes as one convolution with C(14, k)/2^14 along x (zero extension)."""
    c = np.array([math.comb(2 * PASSES, k) for k in range(2 * PASSES + 1)]) / 2.0 ** (2 * PASSES)
    out = np.zeros_like(q)
    for j in range(q.shape[1]):
        out[:, j] = np.convolve(q[:, j], c, mode="same")
    return out


def test_filtered_current_keeps_continuity_with_filtered_charge():
    nx, nr, dx, dr, dt = 40, 12, 0.7, 0.9, 0.5
    rng = np.random.default_rng(4)
    s = OSim(nx, nr, dx, dr, dt, moving_window=False)
    s.set_filter(PASSES)
    s.set_particles(**_random_plasma(rng, 2000, nx, nr, dx, dr, margin=12))
    for _ in range(2):
        before = s.particles()
        q0 = deposit_charge(before["x"], before["y"], before["z"], before["w"], 0, dx, dr, nx, nr)
        s.pass_a()
        s.envelope()
        s.pass_b()
        s.filter()
        after = s.particles()
        q1 = deposit_charge(after["x"], after["y"], after["z"], after["w"], 0, dx, dr, nx, nr)
        dqf = binomial_x(q1 - q0)
        np.testing.assert_allclose(s.field("dq"), dqf, rtol=0, atol=1e-12 * np.abs(dqf).max())
        jx, jr = s.field("jx"), s.field("jr")
        area_x = node_volume_q(nr, dx, dr) / dx
        area_r = 2 * np.pi * (np.arange(nr) + 0.5) * dr * dx
        ix = np.zeros((nx + 2, nr + 1))
        ix[1:nx + 1] = jx * area_x[None, :]
        ir_full = np.zeros((nx + 1, nr + 2))
        ir_full[:, 1:nr + 1] = jr * area_r[None, :]
        div = (ix[1:] - ix[:-1]) + (ir_full[:, 1:] - ir_full[:, :-1])
        res = dqf / dt + div
        assert np.abs(div).max() > 0
        assert np.abs(res).max() < 1e-12 * np.abs(div).max()
        s.ampere()
        s.window()
