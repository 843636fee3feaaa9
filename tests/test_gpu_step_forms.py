"""One lpic_step call of many steps, the same steps one call each, and the kernel-by-kernel
timing mode reach the same state.

lpic_step replays eight steps from one CUDA graph when none of them sorts or relocates the
window, one-step graphs otherwise, and plain launches with kernel timing on; the FP32 particle
passes hand the last slots of a launch out by ticket (at this size every slot: the launch has
more blocks than units).  The three forms differ only in the order of the FP64 atomic
additions (and, in FP32, in which block takes which slots), so their counters agree exactly,
FP64 states agree with each other and with the oracle at the multi-step parity bar (1e-10 and
1e-9; 6e-15 measured between forms), and FP32 states agree with each other at 1e-4: there the
atomic order's last-bit differences in the fields flip FP32 roundings of single particles,
which the following steps carry on (2.8e-6 measured, on chi, after 40 steps).  The grid
(Nx = 24: 29 live columns in 58) makes the window relocate within the 40 steps, and the sort
cadence of 11 leaves room for one eight-step replay after each sort, with single steps up to
the next.
"""
import dataclasses

import numpy as np
import pytest

from helpers import FIELDS, gpu_from, oracle_from, particle_errors, field_errors, rel_err
from workloads import C1

pytestmark = pytest.mark.gpu

W = dataclasses.replace(C1, name="forms", nx=24, nr=24, a0=0.8, w0=8.0, L=4.0, n0=0.01,
                        ramp_cells=4, sort_every=11)
STEPS = 40


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def _run(precision, form):
    sim = gpu_from(W, precision=precision)
    if form == "one_call":
        sim.step(STEPS)
    elif form == "per_step":
        for _ in range(STEPS):
            sim.step(1)
    else:
        sim.set_timing(True)
        sim.step(STEPS)
        sim.set_timing(False)
    return sim


def _same_particles(a, b, tol):
    pa, pb = a.particles(), b.particles()
    ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
    assert np.array_equal(pa["id"][ia], pb["id"][ib])
    for k in ("x", "y", "z", "px", "py", "pz", "w"):
        assert rel_err(pa[k][ia], pb[k][ib]) <= tol, k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_forms_agree(precision):
    sims = {f: _run(precision, f) for f in ("one_call", "per_step", "timed")}
    c = {f: s.counters() for f, s in sims.items()}
    assert c["one_call"]["step"] == STEPS
    assert c["one_call"]["shift"] > 29   # past one relocation of the live window
    for f in ("per_step", "timed"):
        for k in ("step", "shift", "alive"):
            assert c[f][k] == c["one_call"][k], (f, k)
    tol = 1e-10 if precision == "fp64" else 1e-4
    ref = sims["one_call"]
    for f in ("per_step", "timed"):
        for k in FIELDS:
            assert rel_err(sims[f].field(k), ref.field(k)) <= tol, (f, k)
        _same_particles(sims[f], ref, tol)
    if precision == "fp64":
        o = oracle_from(W)
        o.step(STEPS)
        errs = {**field_errors(o, ref), **particle_errors(o, ref)}
        bad = {k: v for k, v in errs.items() if not v <= 1e-9}
        assert not bad, bad
