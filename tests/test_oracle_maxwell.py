"""Pin of the oracle's m=0 Yee solver (Eq. MaxwellEqsCylindrical, FDTD of Sec. 3).

P8  TM_011 mode of a closed perfectly conducting cylinder: Ex = J0(k_perp r) cos(pi x/Lx),
    J0(k_perp r_max) = 0, angular frequency w^2 = k_perp^2 + (pi/Lx)^2.  The measured
    frequency converges to it at second order in the cell size, axis row included.
"""
import math

import numpy as np
import pytest

from oracle.oracle import OSim

special = pytest.importorskip("scipy.special")


def cavity_frequency_error(dx, dr, nx, nr, dt, periods=3):
    s = OSim(nx, nr, dx, dr, dt, moving_window=False)
    rmax, lx = nr * dr, nx * dx
    kperp = special.jn_zeros(0, 1)[0] / rmax
    kx = math.pi / lx
    w = math.sqrt(kperp ** 2 + kx ** 2)
    xh = (np.arange(nx) + 0.5) * dx
    rj = np.arange(nr + 1) * dr
    xn = np.arange(nx + 1) * dx
    rh = (np.arange(nr) + 0.5) * dr
    s.field("ex")[:] = np.outer(np.cos(kx * xh), special.j0(kperp * rj))
    s.field("ex")[:, nr] = 0.0
    # divergence-free companion: Er = (kx/kperp) J1(kperp r) sin(kx x)
    s.field("er")[:] = np.outer(np.sin(kx * xn), (kx / kperp) * special.j1(kperp * rh))
    nst = int(periods * 2 * math.pi / w / dt)
    rec = []
    for _ in range(nst):
        rec.append(s.field("ex")[0, 0])
        s.faraday()
        s.ampere()
    rec = np.array(rec)
    t = np.arange(nst) * dt
    zc = [t[k - 1] + dt * rec[k - 1] / (rec[k - 1] - rec[k])
          for k in range(1, nst) if rec[k - 1] * rec[k] < 0]
    assert len(zc) >= 4
    wnum = math.pi / np.diff(zc).mean()
    return wnum / w - 1


def test_p8_tm_cavity_mode_second_order():
    e1 = cavity_frequency_error(0.5, 0.5, 64, 40, 0.3)
    e2 = cavity_frequency_error(0.25, 0.25, 128, 80, 0.15)
    assert abs(e1) < 1e-4
    assert abs(e1 / e2) > 3.0, (e1, e2)
