"""FP64 CUDA path against the FP64 oracle, through the C ABI, on the same seeded inputs.

Bar: after every compared step each field and each particle component agrees with the oracle
to 1e-10 relative in the max norm (atomic deposit order and FMA contraction are the only
differences; both are O(1e-16) per operation).  Particles are matched by id.
"""
import dataclasses
import math

import numpy as np
import pytest

from helpers import (field_errors, gpu_from, oracle_from, oracle_state_to_gpu, particle_errors,
                     rel_err)
from workloads import C1

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def assert_parity(o, sim, tol=TOL, names=None):
    fe = field_errors(o, sim) if names is None else field_errors(o, sim, names)
    pe = particle_errors(o, sim) if o.np else {}
    bad = {k: v for k, v in {**fe, **pe}.items() if not v <= tol}
    assert not bad, bad
    return fe, pe


def test_first_step_c1_full_size():
    o = oracle_from(C1)
    g = gpu_from(C1)
    assert g.counters()["alive"] == o.np == C1.particles
    assert_parity(o, g)           # initial lattice and envelope
    o.step(1)
    g.step(1)
    assert_parity(o, g)


def test_free_run_c1_forty_steps_with_sorting():
    w = dataclasses.replace(C1, sort_every=4)
    o = oracle_from(w)
    g = gpu_from(w)
    for n in (1, 9, 30):
        o.step(n)
        g.step(n)
        fe, pe = assert_parity(o, g, tol=1e-9)
    assert g.counters()["shift"] == o.shift > 0


def test_one_step_from_oracle_state_after_25_steps():
    o = oracle_from(C1)
    o.step(25)
    g = gpu_from(C1)
    oracle_state_to_gpu(o, g)
    assert_parity(o, g, names=("ex", "er", "bt", "a", "am"))
    for _ in range(2):
        o.step(1)
        g.step(1)
        assert_parity(o, g)


@pytest.mark.parametrize("nx,nr,ppc", [(37, 23, (2, 2, 4)), (50, 9, (1, 3, 2)), (129, 33, (3, 1, 1))])
def test_ragged_grids_moving_window_and_injection(nx, nr, ppc):
    w = dataclasses.replace(C1, name="ragged", nx=nx, nr=nr, ppc=ppc, a0=0.5, w0=8.0, L=6.0,
                            n0=0.01, ramp_cells=7, sort_every=3)
    o = oracle_from(w)
    g = gpu_from(w)
    for _ in range(4):
        o.step(3)
        g.step(3)
        assert_parity(o, g, tol=1e-9)
    assert o.shift >= 9


def test_vacuum_envelope_and_waist_no_particles():
    w = dataclasses.replace(C1, name="vacuum", nx=96, nr=48, w0=15.0, L=10.0, a0=1.0)
    o = oracle_from(w, plasma=False)
    g = gpu_from(w, plasma=False)
    o.step(60)
    g.step(60)
    assert_parity(o, g, names=("a", "am", "ex", "er", "bt"))
    A = o.field("a")
    r = np.arange(w.nr + 1) * w.dr
    v = r * w.dr
    v[0] = w.dr * w.dr / 8
    inten = np.abs(A) ** 2
    waist = np.sqrt(2 * (inten * r ** 2 * v).sum() / (inten * v).sum())
    assert abs(g.waist() / waist - 1) < 1e-12
    assert abs(g.a_abs_max() / np.abs(A).max() - 1) < 1e-12


def test_diagnostics_match_oracle_state():
    from paper_1912_04674_gb300 import lpic as L
    w = dataclasses.replace(C1, name="diag", nx=64, nr=32, a0=1.0, w0=12.0, L=8.0, n0=0.01)
    thr = 0.01
    o = oracle_from(w)
    gt = L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, w.sort_every, track_continuity=True,
                accel_px_min=thr)
    g = L.Simulation(gt, L.Laser(w.a0, w.w0, w.L, w.x_center, w.x_center),
                     L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed))
    o.step(40)
    g.step(40)
    assert rel_err(g.ex_axis(), o.field("ex")[:, 0]) < 1e-9
    c = g.counters()
    assert c["alive"] == o.np and c["step"] == 40 and c["shift"] == o.shift
    res = g.cont_residual()
    assert res < 1e-12, res
    # accelerated-electron statistics against numpy on the oracle state
    p = o.particles()
    sel = p["px"] > thr
    gam = np.sqrt(1 + p["px"] ** 2 + p["py"] ** 2 + p["pz"] ** 2) - 1
    cnt, sw, mean, rms = g.accel_energy()
    assert cnt == sel.sum() and cnt > 0
    ww = p["w"][sel]
    m = (ww * gam[sel]).sum() / ww.sum()
    assert abs(sw / ww.sum() - 1) < 1e-9
    assert abs(mean / m - 1) < 1e-8
    assert abs(rms - np.sqrt((ww * (gam[sel] - m) ** 2).sum() / ww.sum())) < 1e-8 * m


def test_errors_are_reported_not_faulted():
    from paper_1912_04674_gb300 import lpic as L
    w = dataclasses.replace(C1, nx=32, nr=16)
    g = L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, 4)
    with pytest.raises(L.LpicError) as e:          # capacity far too small for the lattice
        L.Simulation(g, None, L.Plasma(0.001), capacity=100)
    assert e.value.status == 4
    sim = L.Simulation(g, None, None, capacity=0)
    with pytest.raises(L.LpicError) as e:          # continuity tracking is off
        sim.cont_residual()
    assert e.value.status == 8
    with pytest.raises(L.LpicError) as e:          # wrong upload size
        sim.upload_field("ex", np.zeros((3, 3)))
    assert e.value.status == 1
    sim.step(3)                                    # vacuum, no particles: still runs
    assert sim.counters()["step"] == 3


def test_window_slide_relocation_matches_oracle():
    """A window of 20 cells shifted 64 times: the sliding live region reaches the end of
    its allocation and is copied back twice; the state must not notice."""
    w = dataclasses.replace(C1, name="reloc", nx=20, nr=12, ppc=(2, 2, 2), a0=0.6, w0=6.0,
                            L=3.0, n0=0.01, sort_every=7)
    o = oracle_from(w)
    g = gpu_from(w)
    for _ in range(8):
        o.step(10)
        g.step(10)
        assert_parity(o, g, tol=1e-9)
    assert o.shift >= 60


def test_async_wake_read_matches_the_synchronising_read():
    """lpic_diagnose_async: the wake enqueued after a step is the one lpic_diagnose returns
    for that step, whether the kernel writes it straight into page-locked host memory or it is
    copied through the staging area into pageable memory; a short buffer is refused."""
    import torch

    g = gpu_from(C1, precision="fp32")
    held = torch.zeros(C1.nx, dtype=torch.float64).pin_memory()
    pinned, pageable = held.numpy(), np.zeros(C1.nx)
    for _ in range(3):
        g.step(5)
        for buf in (pinned, pageable):
            g.ex_axis_async(buf)
            ev = torch.cuda.Event()
            ev.record(g.stream)
            ev.synchronize()
            np.testing.assert_array_equal(buf, g.ex_axis())
    assert np.abs(pinned).max() > 0
    with pytest.raises(Exception):
        g.ex_axis_async(np.zeros(3))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_non_finite_momentum_is_reported_by_the_next_call(precision):
    """A NaN momentum (planted through the upload path; every index the kernels derive from
    it is clamped into the grid) is pushed to a NaN position, which the position push latches
    on the device: the next call reports LPIC_ENONFINITE instead of running on silently."""
    from paper_1912_04674_gb300 import lpic as L
    w = dataclasses.replace(C1, name="nan", nx=32, nr=16, sort_every=4)
    g = gpu_from(w, precision=precision)
    g.step(2)
    assert g.counters()["step"] == 2
    p = g.particles()
    p["px"][len(p["px"]) // 2] = np.nan
    g.upload_particles(p)
    g.step(1)
    with pytest.raises(L.LpicError) as e:
        g.counters()
    assert e.value.status == 7


def test_full_c1_run_of_200_steps():
    """Config 1 in full (paper Sec. 4 linear-wake parameters): 200 steps of the 256 x 64,
    262,144-electron run with the moving window and the periodic sort, compared with the
    oracle every 10 steps; the bar holds at every comparison."""
    o = oracle_from(C1)
    g = gpu_from(C1)
    worst = {}
    for _ in range(C1.steps // 10):
        o.step(10)
        g.step(10)
        errs = {**field_errors(o, g), **particle_errors(o, g)}
        worst = {k: max(worst.get(k, 0.0), v) for k, v in errs.items()}
    assert o.step_index == g.counters()["step"] == C1.steps
    assert g.counters()["alive"] == o.np and o.shift == g.counters()["shift"] > 150
    bad = {k: v for k, v in worst.items() if not v <= TOL}
    assert not bad, (bad, worst)


def _exact_face_cells(dx, first, count):
    """Lab cells c >= first whose face x = c dx splits back into (c, offset 0) exactly."""
    out, c = [], first
    while len(out) < count:
        if math.floor((c * dx) / dx) == c and (c * dx) / dx - c == 0.0:
            out.append(c)
        c += 1
    return out


def _edge_particles(w, shift):
    """Hand-placed electrons on the branches of the locate / push / removal logic that a
    random lattice rarely reaches (ids 2^40 + k)."""
    dx, dr, nx, nr = w.dx, w.dr, w.nx, w.nr
    wt = 2e-3
    faces = _exact_face_cells(dx, shift + 12, 3)
    rmax = nr * dr
    rows = [
        # x (lab),                 y,          z,         px,   py,   pz
        ((shift + 20.3) * dx,      0.0,        0.0,       0.0,  0.0,  0.0),   # on the axis, at rest
        ((shift + 21.7) * dx,      0.0,        0.0,       0.2,  0.3, -0.1),   # on the axis, moving off it
        (faces[0] * dx,            2.3,        1.1,       0.0,  0.1,  0.0),   # on an x face (offset 0)
        (faces[1] * dx,            5 * dr,     0.0,       0.1,  0.0,  0.0),   # on an x and a radial face
        ((shift + 17.4) * dx,      0.0,        7 * dr,    0.0,  0.0, -0.2),   # on a radial face (r/dr = 7)
        ((shift + 25.5) * dx,      0.2,        0.05,     -0.1, -3.0, -1.0),   # crosses the axis this step
        ((shift + 26.5) * dx,     -0.05,       0.01,      0.0,  2.0,  0.0),   # crosses the axis the other way
        ((shift + 28.2) * dx,      rmax - 0.01, 0.0,      0.0,  1.0,  0.0),   # just below r_max, leaving
        ((shift + 29.2) * dx,      0.0,        rmax - 0.02, 0.0, 0.0, -0.5),  # just below r_max, staying
        (shift * dx,               3.0,        0.0,       0.0,  0.0,  0.0),   # on the back window edge
        ((shift + 0.02) * dx,      4.0,       -1.0,      -0.5,  0.0,  0.0),   # just inside it, moving back
        ((shift + nx - 0.02) * dx, 6.0,        0.0,       3.0,  0.0,  0.0),   # at the front, moving out
        (faces[2] * dx,            0.0,        0.0,      -0.4,  0.0,  0.0),   # on the axis and an x face
    ]
    a = np.array(rows, dtype=np.float64)
    n = len(rows)
    return {"x": a[:, 0], "y": a[:, 1], "z": a[:, 2], "px": a[:, 3], "py": a[:, 4], "pz": a[:, 5],
            "w": np.full(n, wt), "id": (np.uint64(1) << np.uint64(40)) + np.arange(n, dtype=np.uint64)}


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("fp32", 1e-3)])
def test_hand_placed_edge_particles_step_by_step(precision, tol):
    """Electrons exactly on the axis, on x and radial cell faces, crossing the axis, leaving
    at r_max, at the back edge while the window shifts and leaving at the front, added to a
    driven plasma: every field and particle component agrees with the oracle after each of
    eight steps (the same particles are removed on both sides)."""
    w = dataclasses.replace(C1, name="edges", nx=40, nr=16, a0=1.0, w0=8.0, L=5.0, n0=0.01,
                            sort_every=3)
    o = oracle_from(w)
    o.step(3)
    p = o.particles()
    e = _edge_particles(w, o.shift)
    both = {k: np.concatenate([p[k], e[k]]) for k in p}
    o.set_particles(**both)
    g = gpu_from(w, precision=precision)
    g.upload_counters(o.step_index, o.shift)
    for k in ("ex", "er", "bt", "a", "am"):
        g.upload_field(k, o.field(k))
    g.upload_particles(both)
    for step in range(8):
        o.step(1)
        g.step(1)
        fe, pe = field_errors(o, g), particle_errors(o, g)
        bad = {k: v for k, v in {**fe, **pe}.items() if not v <= tol}
        assert not bad, (step, bad)
    ids = set(o.part("id").tolist())
    gone = [k for k in range(len(e["x"])) if int(e["id"][k]) not in ids]
    assert {7, 9, 10} <= set(gone), gone        # the r_max and back-edge removals happened
    assert 8 not in gone and 0 not in gone


def test_upload_from_pinned_host_memory_matches_pageable():
    """Uploads from page-locked host memory are read by the conversion kernels in place (no
    staging); the state they leave must equal the staged upload of the same pageable data."""
    import torch

    w = dataclasses.replace(C1, name="pinned", nx=64, nr=32, a0=1.0, w0=10.0, L=6.0, n0=0.01)
    src = gpu_from(w)
    src.step(7)
    parts = src.particles()
    fields = {k: src.field(k) for k in ("ex", "er", "bt", "a", "am")}
    c = src.counters()
    raw = np.concatenate([parts[k] for k in ("x", "y", "z", "px", "py", "pz", "w")])
    pinned_raw = torch.from_numpy(raw).pin_memory()
    pinned_ids = torch.from_numpy(np.ascontiguousarray(parts["id"].view(np.int64))).pin_memory()
    pinned_f = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in fields.items()}
    a, b = gpu_from(w), gpu_from(w)
    for sim in (a, b):
        sim.upload_counters(c["step"], c["shift"])
    for k, v in fields.items():
        a.upload_field(k, v)                           # pageable: staged
        b.upload_field(k, pinned_f[k].numpy())         # page-locked: read in place
    a.upload_particles_raw(raw, parts["id"])
    b.upload_particles_raw(pinned_raw.numpy(), pinned_ids.numpy().view(np.uint64))
    for k in fields:
        np.testing.assert_array_equal(a.field(k), b.field(k))
    pa, pb = a.particles(), b.particles()
    for k in pa:
        np.testing.assert_array_equal(pa[k], pb[k])
    a.step(3)
    b.step(3)
    for k in ("ex", "a", "chi", "jx"):
        assert rel_err(b.field(k), a.field(k)) <= 1e-12
