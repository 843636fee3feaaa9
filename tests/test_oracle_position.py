"""Reading G24: the oracle keeps a particle's x as a lab cell index plus an in-cell offset and
takes the new radius as r^n plus the radial step (dy (y0 + y1) + dz (z0 + z1)) / (r0 + r1).

Both are rewritings of the plain position push of Eq. EquationsOfMotion (Sec. 3): x^{n+1} =
x^n + dt p_x / gbar in the lab frame and r^{n+1} = sqrt(y1^2 + z1^2).  Where the plain form is
well conditioned (displacements of a sizeable fraction of a cell, at shift 0, on a small
grid), the two must give the same positions and the same charge-conserving current to
rounding.  The reference here is that plain lab-frame evaluation, written in numpy with
hat-function shape factors over the whole grid (no cell bookkeeping at all), so a slip in
the oracle's cell/offset arithmetic (a lost carry, an offset taken from the wrong cell, a
wrong sign in the radial step) shows up as a difference far above 1e-14.
"""
import numpy as np

from oracle.oracle import OSim

NX, NR, DX, DR, DT = 8, 8, 0.69, 1.5, 0.5
TOL = 1e-14


def hat(u):
    return np.maximum(0.0, 1.0 - np.abs(u))


def lab_frame_pass_b(x0, y0, z0, px, py, pz, w):
    """One position push and Esirkepov current with Phi = 0, from lab-frame coordinates."""
    gb = np.sqrt(1.0 + px * px + py * py + pz * pz)
    x1, y1, z1 = x0 + DT * px / gb, y0 + DT * py / gb, z0 + DT * pz / gb
    r0, r1 = np.hypot(y0, z0), np.hypot(y1, z1)
    i = np.arange(NX + 1)
    j = np.arange(NR + 1)
    s0x, s1x = hat(x0[:, None] / DX - i), hat(x1[:, None] / DX - i)
    s0r, s1r = hat(r0[:, None] / DR - j), hat(r1[:, None] / DR - j)
    dsx, dsr = s1x - s0x, s1r - s0r
    qw = -w
    # Jx(i+1/2, j): prefix sum over i of DSx (S0r + DSr/2), over the ring area V_j / dx
    wx = dsx[:, :, None] * (s0r + 0.5 * dsr)[:, None, :]
    area = 2 * np.pi * j * DR * DR
    area[0] = np.pi * (DR / 2) ** 2
    jx = (-qw[:, None, None] / DT * np.cumsum(wx, axis=1)[:, :NX, :] / area).sum(0)
    # Jr(i, j+1/2): prefix sum over j of DSr (S0x + DSx/2), over 2 pi r_{j+1/2} dx
    wr = dsr[:, None, :] * (s0x + 0.5 * dsx)[:, :, None]
    face = 2 * np.pi * (j[:NR] + 0.5) * DR * DX
    jr = (-qw[:, None, None] / DT * np.cumsum(wr, axis=2)[:, :, :NR] / face).sum(0)
    return np.stack([x1, y1, z1], 1), jx, jr


def test_g24_cell_offset_push_equals_the_lab_frame_push():
    rng = np.random.default_rng(24)
    n = 400
    x = rng.uniform(1.2, NX - 1.2, n) * DX
    r = rng.uniform(0.3, NR - 1.3, n) * DR
    th = rng.uniform(0, 2 * np.pi, n)
    p = {"x": x, "y": r * np.cos(th), "z": r * np.sin(th), "px": rng.uniform(-0.9, 0.9, n),
         "py": rng.uniform(-0.9, 0.9, n), "pz": rng.uniform(-0.9, 0.9, n),
         "w": rng.uniform(0.5, 1.5, n)}
    o = OSim(NX, NR, DX, DR, DT, False)          # no laser: Phi = 0; shift 0
    o.set_particles(**p)
    o.pass_b()
    pos, jx, jr = lab_frame_pass_b(*(p[k] for k in ("x", "y", "z", "px", "py", "pz", "w")))
    got = np.stack([o.part("x"), o.part("y"), o.part("z")], 1)
    assert np.abs(got[:, 0] - pos[:, 0]).max() <= TOL * NX * DX
    assert np.abs(got[:, 1:] - pos[:, 1:]).max() <= TOL * NR * DR
    assert np.abs(o.field("jx") - jx).max() <= TOL * np.abs(jx).max()
    assert np.abs(o.field("jr") - jr).max() <= TOL * np.abs(jr).max()
    # the displacements are a sizeable part of a cell: the comparison is well conditioned
    assert np.abs(pos[:, 0] - x).mean() > 0.1 * DX


def test_g24_offset_carry_across_cell_faces():
    """Particles that start on a cell face (offset exactly 0) or cross one in either
    direction keep x = (cell + offset) dx equal to the lab-frame x^n + dt p_x / gbar."""
    xs = np.array([2.0, 3.0, 4.0, 5.0, 3.5, 4.999]) * DX
    pxs = np.array([0.0, -0.6, 0.6, -3.0, 3.0, 0.2])
    n = len(xs)
    p = {"x": xs, "y": np.full(n, 3.0 * DR), "z": np.zeros(n), "px": pxs, "py": np.zeros(n),
         "pz": np.zeros(n), "w": np.ones(n)}
    o = OSim(NX, NR, DX, DR, DT, False)
    o.set_particles(**p)
    o.pass_b()
    pos, _, _ = lab_frame_pass_b(*(p[k] for k in ("x", "y", "z", "px", "py", "pz", "w")))
    assert np.abs(o.part("x") - pos[:, 0]).max() <= TOL * NX * DX
    crossed = np.floor(pos[:, 0] / DX) != np.floor(xs / DX)
    assert crossed.any() and (~crossed).any()
