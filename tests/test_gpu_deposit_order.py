"""The deposits do not depend on the order of the particles in memory.

The passes sum each warp's deposits per cell or node before the FP64 atomics: FP32 pass A
through warp-private node buckets covering the 31 cells from the warp's lowest cell, FP32 pass
B and the FP64 passes over runs of neighbouring lanes with equal cells.  Electrons outside a
warp's 31 cells deposit alone.  With the particle order shuffled at random (and a sort cadence longer
than the test, so that it stays shuffled) nearly every warp takes those single-electron paths.
Bars, for two steps from an oracle state: FP64 against the oracle at 1e-10, as for a sorted
state; FP32 shuffled and sorted against the oracle at the 1e-3 element-by-element bar of the
FP32 ragged-grid test, and against each other at 1e-4 of each field's scale.  That last bar
follows from the exact FP32 deposit (G18): each value is rounded once, to at most 2^-25 of the
largest value in its warp.  Sorted, a warp holds the electrons of a few neighbouring cells and
of similar weights; shuffled, a warp mixes electrons near the axis (weight proportional to r)
with electrons at the outer radius, so a near-axis value is rounded to 2^-25 of an outer
weight, and the axis row's small volume V_0 = pi (dr/2)^2 dx (1/380 of the outermost row's at
Nr = 48) scales that up in chi and Jx: about 64 values per node x 2^-25 x 380 / 16 values per
node at the maximum ~ 5e-5 of the field's scale (1.2e-5 measured for chi).
"""
import dataclasses

import numpy as np
import pytest

from helpers import field_errors, gpu_from, oracle_from, particle_errors, rel_err
from workloads import C1

pytestmark = pytest.mark.gpu

W = dataclasses.replace(C1, name="shuffled", nx=128, nr=48, a0=0.8, w0=12.0, L=8.0, n0=0.01,
                        ramp_cells=10, sort_every=1000)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def _load(sim, o, perm):
    sim.upload_counters(o.step_index, o.shift)
    for k in ("ex", "er", "bt", "a", "am"):
        sim.upload_field(k, o.field(k))
    p = o.particles()
    sim.upload_particles({k: np.asarray(v)[perm] for k, v in p.items()})


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shuffled_particles_deposit_like_sorted_ones(precision):
    o = oracle_from(W)
    o.step(6)
    n = o.np
    shuffled = np.random.default_rng(7).permutation(n)
    in_order = np.arange(n)
    a = gpu_from(W, precision=precision, sort_every=1000)
    b = gpu_from(W, precision=precision, sort_every=1000)
    _load(a, o, shuffled)
    _load(b, o, in_order)
    for _ in range(2):
        o.step(1)
        a.step(1)
        b.step(1)
    tol = 1e-10 if precision == "fp64" else 1e-3
    for sim in (a, b):
        errs = {**field_errors(o, sim), **particle_errors(o, sim)}
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, bad
    if precision == "fp32":
        for k in ("chi", "jx", "jr", "ex", "er", "bt", "a"):
            assert rel_err(a.field(k), b.field(k)) <= 1e-4, k
