"""Pins of the oracle's envelope solver (Eq. envelope_solver) to physics it must reproduce.

P1  vacuum diffraction of a focused Gaussian pulse against the Rayleigh law
    w(x) = w0 sqrt(1 + (x/xR)^2), xR = w0^2/2 (Sec. 4, first benchmark; the printed
    law is read with x/xR, the dimensionally correct paraxial form).
P2  uniform susceptibility: a spatially uniform envelope evolves as g^n, with g a root of
    the scheme's characteristic polynomial, and g -> exp(-i (sqrt(1+chi) - 1) dt), the
    plasma dispersion w^2 = 1 + n of the carrier, at second order in dt.
"""
import math

import numpy as np
import pytest

from oracle.oracle import OSim


def waist_second_moment(A, dr):
    r = np.arange(A.shape[1]) * dr
    vol = 2 * np.pi * r * dr
    vol[0] = np.pi * dr * dr / 4
    inten = np.abs(A) ** 2
    return math.sqrt(2 * (inten * r ** 2 * vol).sum() / (inten * vol).sum())


@pytest.mark.parametrize("dx,dr,nx,nr,nsteps", [(0.7, 1.5, 96, 48, 400)])
def test_p1_vacuum_diffraction_rayleigh(dx, dr, nx, nr, nsteps):
    w0, L = 15.0, 10.0
    dt = 0.8 * dx
    s = OSim(nx, nr, dx, dr, dt, moving_window=True)
    xc = nx * dx - 3 * L
    s.init_envelope(1.0, w0, L, xc, xc)
    xR = w0 * w0 / 2
    for k in range(nsteps):
        s.step(1)
        if (k + 1) % 50 == 0:
            t = (k + 1) * dt
            grow = math.sqrt(1 + (t / xR) ** 2)
            w = waist_second_moment(s.field("a"), dr)
            assert abs(w / (w0 * grow) - 1) < 0.015, (t, w, w0 * grow)
            amax = np.abs(s.field("a")[:, 0]).max()
            assert abs(amax * grow - 1) < 0.015, (t, amax, 1 / grow)
    # the beam really diffracted: the check above is not satisfied by a frozen profile
    assert waist_second_moment(s.field("a"), dr) > 2.0 * w0


def _uniform_run(dt, chi, nsteps, a_prev_factor):
    n = nsteps
    s = OSim(2 * n + 10, 2 * n + 10, 1.0, 1.0, dt, moving_window=False)
    s.field("a")[:] = 1.0
    s.field("am")[:] = a_prev_factor
    s.field("chi")[:] = chi
    for _ in range(n):
        s.envelope()
    # node farther than n cells from every Dirichlet boundary; row 0 is the axis
    return s.field("a")[n + 2, 0], s.field("a")[n + 2, 7]


def test_p2_uniform_chi_characteristic_root():
    dt, chi, n = 0.4, 0.05, 30
    roots = np.roots([1 - 1j * dt, -(2 - dt * dt * chi), 1 + 1j * dt])
    g = roots[np.argmin(np.abs(roots - 1))]
    assert abs(abs(g) - 1) < 1e-14  # neutrally stable branch
    axis, off = _uniform_run(dt, chi, n, 1 / g)
    assert abs(axis - g ** n) < 1e-12
    assert abs(off - g ** n) < 1e-12


def test_p2_uniform_chi_plasma_dispersion_second_order():
    chi, n = 0.05, 40
    delta = math.sqrt(1 + chi) - 1
    errs = []
    for dt in (0.4, 0.2, 0.1):
        gc = np.exp(-1j * delta * dt)
        axis, _ = _uniform_run(dt, chi, n, 1 / gc)
        phase = np.angle(axis) / n
        errs.append(abs(phase / (-delta * dt) - 1))
        assert abs(abs(axis) - 1) < 1e-6
    assert errs[0] < 5e-5
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
