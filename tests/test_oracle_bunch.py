"""Pins of the oracle's initial fields for an externally injected relativistic bunch.

* the initial E satisfies the discrete Gauss law of the Yee grid node by node (the same
  divergence the Maxwell solver conserves, P7), to rounding;
* in the middle of a long uniform cylinder, E_r at r_{j+1/2} is the charge enclosed within
  that radius over 2 pi r dx (Gauss's law in integral form), and E_x vanishes;
* B_theta = beta E_r for the uniformly moving charge;
* the bunch and its fields, stepped with the oracle's own loop in vacuum, move together: after
  20 steps E_r is within 1 % of the initial-field solution for the moved bunch, while a bunch
  started from zero fields leaves an order-one transient.
"""
import numpy as np

from oracle.bunch import bunch_fields, node_charge
from oracle.oracle import OSim

from test_oracle_deposit import node_volume_q


def gauss_residual(ex, er, Q, nx, nr, dx, dr):
    vol = node_volume_q(nr, dx, dr)
    exp_ = np.zeros((nx + 2, nr + 1))
    exp_[1:nx + 1] = ex
    rh = (np.arange(nr) + 0.5) * dr
    flux = np.zeros((nx + 1, nr + 2))
    flux[:, 1:nr + 1] = 2 * np.pi * dx * rh[None, :] * er
    div = (exp_[1:] - exp_[:-1]) / dx + (flux[:, 1:] - flux[:, :-1]) / vol[None, :]
    return (div - Q / vol[None, :])[1:nx, 0:nr], np.abs(Q / vol[None, :]).max()


def gaussian_bunch(rng, n, xc, sx, sr, charge=1.0):
    x = rng.normal(xc, sx, n)
    y, z = rng.normal(0, sr, n), rng.normal(0, sr, n)
    w = np.full(n, charge / n)
    return x, y, z, w


def test_initial_field_satisfies_discrete_gauss_law():
    nx, nr, dx, dr, dt, gamma = 64, 32, 0.69, 1.5, 0.5, 200.0
    rng = np.random.default_rng(5)
    x, y, z, w = gaussian_bunch(rng, 20000, 22.0, 3.0, 4.0)
    ex, er, bt = bunch_fields(x, y, z, w, nx, nr, dx, dr, dt, gamma)
    Q = node_charge(x, y, z, w, nx, nr, dx, dr)
    res, scale = gauss_residual(ex, er, Q, nx, nr, dx, dr)
    assert np.abs(res).max() < 1e-11 * scale
    beta = np.sqrt(1 - 1 / gamma**2)
    # B_theta is beta E_r (of the field moved back by beta dt/2), i.e. between E_r's x nodes
    lo, hi = np.minimum(er[:-1], er[1:]), np.maximum(er[:-1], er[1:])
    assert np.all(bt >= beta * lo - 1e-15) and np.all(bt <= beta * hi + 1e-15)


def test_long_cylinder_matches_enclosed_charge():
    nx, nr, dx, dr, dt, gamma = 200, 24, 0.69, 1.5, 0.5, 1000.0
    a = 9.0
    # a regular lattice filling r < a for 10 < x < 128, uniform density
    xs = (np.arange(int(10 / dx * 4), int(128 / dx * 4)) + 0.5) * dx / 4
    rs = (np.arange(int(a / dr * 8)) + 0.5) * dr / 8
    th = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    X, Rr, T = np.meshgrid(xs, rs, th, indexing="ij")
    x, r, t = X.ravel(), Rr.ravel(), T.ravel()
    w = r * 1e-4                                  # uniform density: weight ~ r dr dtheta dx
    y, z = r * np.cos(t), r * np.sin(t)
    ex, er, bt = bunch_fields(x, y, z, w, nx, nr, dx, dr, dt, gamma)
    Q = node_charge(x, y, z, w, nx, nr, dx, dr)
    i = int(69 / dx)                              # the middle of the cylinder
    enclosed = np.cumsum(Q[i, :nr])               # charge within r_{j+1/2}
    rh = (np.arange(nr) + 0.5) * dr
    want = enclosed / (2 * np.pi * rh * dx)
    np.testing.assert_allclose(er[i], want, rtol=1e-6, atol=1e-9 * np.abs(want).max())
    assert np.abs(ex[i]).max() < 1e-6 * np.abs(er[i]).max()


def lattice_bunch(xc, sx, sr, dx, dr, charge, sub=4, nth=8):
    """A quiet (lattice-sampled) Gaussian bunch: no shot noise at the grid scale, whose
    fields would otherwise lag the particles at the Yee grid's slow Nyquist phase velocity."""
    xs = np.arange(xc - 4 * sx, xc + 4 * sx, dx / sub) + dx / (2 * sub)
    rs = (np.arange(int(4 * sr / dr * sub)) + 0.5) * dr / sub
    th = (np.arange(nth) + 0.5) * 2 * np.pi / nth
    X, Rr, T = np.meshgrid(xs, rs, th, indexing="ij")
    x, r, t = X.ravel(), Rr.ravel(), T.ravel()
    w = np.exp(-(x - xc) ** 2 / (2 * sx * sx) - r * r / (2 * sr * sr)) * r
    return x, r * np.cos(t), r * np.sin(t), w * charge / w.sum()


def _comoving_error(init_fields, steps=20):
    """max |E_r - E_r,static| / max |E_r,static| after `steps`, E_r,static being the
    initial-field solution for the bunch where it has moved to."""
    nx, nr, dx, dr, dt, gamma = 96, 24, 0.69, 1.5, 0.5, 100.0
    x, y, z, w = lattice_bunch(25.0, 4.0, 3.0, dx, dr, 0.05)
    beta = np.sqrt(1 - 1 / gamma**2)
    s = OSim(nx, nr, dx, dr, dt, moving_window=False)
    s.set_particles(x=x, y=y, z=z, px=np.full(len(x), gamma * beta), w=w)
    if init_fields:
        ex0, er0, bt0 = bunch_fields(x, y, z, w, nx, nr, dx, dr, dt, gamma)
        s.field("ex")[:] = ex0
        s.field("er")[:] = er0
        s.field("bt")[:] = bt0
    s.step(steps)
    p = s.particles()
    _, er1, _ = bunch_fields(p["x"], p["y"], p["z"], p["w"], nx, nr, dx, dr, dt, gamma)
    inner = slice(10, nx - 10)
    return np.abs(s.field("er")[inner] - er1[inner]).max() / np.abs(er1).max()


def test_bunch_and_fields_move_together():
    good = _comoving_error(True)
    bad = _comoving_error(False)
    assert good < 0.01, good
    assert bad > 0.5, bad
