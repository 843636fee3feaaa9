"""Test-side glue: build the oracle and the CUDA simulation from one workload, move a state
between them, and compare states the way the parity bar is stated (normwise per field,
particles matched by id)."""
from __future__ import annotations

import numpy as np

from oracle.oracle import OSim

FIELDS = ("ex", "er", "bt", "a", "am", "chi", "jx", "jr")
PCOMP = ("x", "y", "z", "px", "py", "pz", "w")


def oracle_from(w, plasma=True, laser=True, moving=None, filter_passes=0):
    s = OSim(w.nx, w.nr, w.dx, w.dr, w.dt, w.moving_window if moving is None else moving)
    if filter_passes:
        s.set_filter(filter_passes)
    if laser:
        s.init_envelope(w.a0, w.w0, w.L, w.x_center, w.x_center)
    if plasma:
        s.load_plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed)
    return s


def gpu_from(w, precision="fp64", plasma=True, laser=True, moving=None, sort_every=None,
             track=False, capacity=None, filter_passes=0):
    from paper_1912_04674_gb300 import lpic as L
    g = L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, w.moving_window if moving is None else moving,
               sort_every or w.sort_every, track_continuity=track, filter_passes=filter_passes)
    la = L.Laser(w.a0, w.w0, w.L, w.x_center, w.x_center) if laser else None
    pl = L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed) if plasma else None
    if not plasma and capacity is None:
        capacity = 0
    return L.Simulation(g, la, pl, precision=precision, capacity=capacity)


def oracle_state_to_gpu(o: OSim, sim):
    sim.upload_counters(o.step_index, o.shift)
    for k in ("ex", "er", "bt", "a", "am"):
        sim.upload_field(k, o.field(k))
    p = o.particles()
    sim.upload_particles(p)


def gpu_state_to_oracle(sim, o: OSim):
    c = sim.counters()
    o.set_counters(c["step"], c["shift"])
    for k in ("ex", "er", "bt", "a", "am"):
        o.field(k)[:] = sim.field(k)
    o.set_particles(**sim.particles())


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max() if b.size else 0.0
    d = np.abs(a - b).max() if b.size else 0.0
    return d / scale if scale > 0 else d


def field_errors(o: OSim, sim, names=FIELDS):
    return {k: rel_err(sim.field(k), o.field(k)) for k in names}


def particle_errors(o: OSim, sim):
    po = o.particles()
    pg = sim.particles()
    io = np.argsort(po["id"])
    ig = np.argsort(pg["id"])
    assert len(io) == len(ig), (len(io), len(ig))
    assert np.array_equal(po["id"][io], pg["id"][ig])
    out = {}
    for k in PCOMP:
        a, b = pg[k][ig], po[k][io]
        if k in ("px", "py", "pz"):
            scale = max(np.abs(po["px"]).max(), np.abs(po["py"]).max(), np.abs(po["pz"]).max(), 1e-300)
        elif k == "x":
            scale = o.nx * o.dx
        elif k in ("y", "z"):
            scale = o.nr * o.dr
        else:
            scale = np.abs(b).max() if b.size else 1.0
        out[k] = np.abs(a - b).max() / scale if b.size else 0.0
    return out
