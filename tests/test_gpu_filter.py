"""Binomial current filter (Sec. 4: 7 passes against numerical Cherenkov radiation) on the
GPU against the oracle with the same filter.

Bar: FP64, 1e-9 per field and particle component after each compared step, as for the
unfiltered parity runs of several steps (Bt measured against the scale at which rounding of
E enters it, see `check`); FP32_MIXED within 1e-3 of FP64 on
the wake; the continuity residual of the filtered current against the filtered charge at
rounding level; a batch with filtered and unfiltered simulations equal to their alone runs.
"""
import dataclasses

import numpy as np
import pytest

from helpers import field_errors, gpu_from, oracle_from, particle_errors, rel_err
from workloads import C1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def check(o, g, tol):
    """Per-field normwise errors; Bt against the larger of its own norm and dt |E| / dx, the
    scale at which rounding of E enters the Faraday update.  The filtered current is smooth
    along x, so the x-differences of E that make Bt cancel strongly in the first steps and
    Bt's own norm understates what rounding can reach."""
    fe = field_errors(o, g)
    e_scale = max(np.abs(o.field("ex")).max(), np.abs(o.field("er")).max())
    bt_scale = max(np.abs(o.field("bt")).max(), o.dt * e_scale / min(o.dx, o.dr))
    if bt_scale > 0:
        fe["bt"] = float(np.abs(g.field("bt") - o.field("bt")).max() / bt_scale)
    pe = particle_errors(o, g)
    bad = {k: v for k, v in {**fe, **pe}.items() if not v <= tol}
    assert not bad, bad


def test_filter_parity_c1_moving_window():
    w = dataclasses.replace(C1, a0=0.6, sort_every=7)
    o = oracle_from(w, filter_passes=7)
    g = gpu_from(w, filter_passes=7)
    for n in (1, 9, 20):
        o.step(n)
        g.step(n)
        check(o, g, 1e-9)
    assert o.shift > 0
    # the filter did act: J differs from an unfiltered run of the same state
    u = gpu_from(w)
    u.step(30)
    assert rel_err(u.field("jx"), g.field("jx")) > 1e-3


@pytest.mark.parametrize("nx,nr,passes", [(37, 23, 3), (129, 40, 16), (64, 31, 1)])
def test_filter_ragged_tiles(nx, nr, passes):
    w = dataclasses.replace(C1, name="ragged", nx=nx, nr=nr, a0=0.6, w0=8.0, L=6.0, n0=0.01,
                            ramp_cells=5, sort_every=3)
    o = oracle_from(w, filter_passes=passes)
    g = gpu_from(w, filter_passes=passes)
    for _ in range(3):
        o.step(4)
        g.step(4)
        check(o, g, 1e-9)


def test_filter_continuity_and_fp32():
    w = dataclasses.replace(C1, name="nl", nx=256, nr=64, a0=1.5, w0=12.0, L=8.0, n0=0.004,
                            sort_every=10)
    g64 = gpu_from(w, filter_passes=7, track=True)
    g32 = gpu_from(w, precision="fp32", filter_passes=7, track=True)
    worst = 0.0
    for _ in range(4):
        g64.step(25)
        g32.step(25)
        e64 = g64.ex_axis()
        worst = max(worst, float(np.linalg.norm(g32.ex_axis() - e64) / np.linalg.norm(e64)))
    assert worst < 1e-3, worst
    assert g64.cont_residual() < 1e-12
    assert g32.cont_residual() < 1e-5


def test_batch_with_filter_matches_alone():
    import torch

    from paper_1912_04674_gb300 import lpic as L
    base = dataclasses.replace(C1, a0=0.8, L=8.0, n0=0.004, sort_every=5)
    ws = [dataclasses.replace(base, name="f0", nx=96, nr=32, w0=10.0, seed=1),
          dataclasses.replace(base, name="f1", nx=160, nr=48, w0=14.0, seed=2)]
    passes = [7, 0]
    alone = []
    for w, p in zip(ws, passes):
        s = gpu_from(w, filter_passes=p)
        s.step(25)
        alone.append(s)
    mixed = [gpu_from(w, filter_passes=p) for w, p in zip(ws, passes)]
    b = L.Batch(mixed, torch.cuda.Stream())
    b.step([25, 25])
    b.close()
    for a, m in zip(alone, mixed):
        for f in ("ex", "er", "bt", "a", "jx", "jr"):
            assert rel_err(m.field(f), a.field(f)) < 1e-10, f
        assert a.counters() == m.counters()
