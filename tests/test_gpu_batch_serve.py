"""Batched and served forms: every simulation gives the same result when it runs alone and
when it runs inside a batch or a served mix of uneven simulations.

Bar: FP64, 1e-10 relative per field (only the order of the FP64 atomic additions differs);
FP32_MIXED, 1e-5 on the wake and peak |A| (the same kernels on the same inputs; atomic order
changes FP64 sums in their last bits, which FP32 fields can round differently).
"""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_from, rel_err
from workloads import C1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def small_jobs():
    base = dataclasses.replace(C1, a0=0.8, L=8.0, n0=0.004, sort_every=5)
    return [dataclasses.replace(base, name="j0", nx=96, nr=32, w0=10.0, seed=1),
            dataclasses.replace(base, name="j1", nx=160, nr=48, w0=14.0, seed=2, ramp_cells=20),
            dataclasses.replace(base, name="j2", nx=64, nr=40, w0=12.0, seed=3, a0=1.5)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_batch_matches_alone(precision, tol):
    import torch

    from paper_1912_04674_gb300 import lpic as L
    jobs = small_jobs()
    steps = [30, 45, 20]
    alone = []
    for w, n in zip(jobs, steps):
        s = gpu_from(w, precision=precision)
        s.step(n)
        alone.append(s)
    mixed = [gpu_from(w, precision=precision) for w in jobs]
    b = L.Batch(mixed, torch.cuda.Stream())
    b.step([10, 10, 10])          # all three together
    b.step([20, 35, 10])          # uneven: later launches run fewer simulations
    # one fused launch per phase (pass B of the untracked simulations only) per step; the
    # three simulations sort together every 5 steps in seven more fused launches
    assert b.launches() == 6 * 45 + 7 * (45 // 5)
    b.close()
    for a, m, n in zip(alone, mixed, steps):
        assert m.counters()["step"] == n
        for f in ("ex", "er", "bt", "a", "chi", "jx"):
            assert rel_err(m.field(f), a.field(f)) < tol, (f, rel_err(m.field(f), a.field(f)))
        assert a.counters() == m.counters()


def test_unfused_schedule_matches_alone():
    """packs = -1: every batch step replays each simulation's own step graph, in turn."""
    import torch

    from paper_1912_04674_gb300 import lpic as L
    jobs = small_jobs()
    steps = [30, 45, 20]
    alone = []
    for w, n in zip(jobs, steps):
        s = gpu_from(w, precision="fp32")
        s.step(n)
        alone.append(s)
    mixed = [gpu_from(w, precision="fp32") for w in jobs]
    b = L.Batch(mixed, torch.cuda.Stream())
    b.set_tuning(4096, -1)
    b.step(steps)
    assert b.launches() > 0
    b.close()
    for a, m, n in zip(alone, mixed, steps):
        assert m.counters()["step"] == n
        for f in ("ex", "er", "bt", "a", "chi", "jx"):
            assert rel_err(m.field(f), a.field(f)) < 1e-5, (f, rel_err(m.field(f), a.field(f)))
        assert a.counters() == m.counters()


def test_batch_interleaved_with_own_steps_matches_alone():
    """Batch steps and each simulation's own steps alternate on the same states (the host
    mirrors and the device state are the simulation's; the batch holds none of its own)."""
    import torch

    from paper_1912_04674_gb300 import lpic as L
    jobs = small_jobs()
    alone = []
    for w in jobs:
        s = gpu_from(w, precision="fp32")
        s.step(33)
        alone.append(s)
    mixed = [gpu_from(w, precision="fp32") for w in jobs]
    b = L.Batch(mixed, torch.cuda.Stream())
    b.step([6, 6, 6])
    for s, n in zip(mixed, (7, 11, 3)):
        s.step(n)
    b.step([12, 8, 16])
    for s, n in zip(mixed, (8, 8, 8)):
        s.step(n)
    b.close()
    for a, m in zip(alone, mixed):
        assert m.counters()["step"] == 33
        for f in ("ex", "er", "bt", "a", "chi", "jx"):
            assert rel_err(m.field(f), a.field(f)) < 1e-5, (f, rel_err(m.field(f), a.field(f)))
        assert a.counters() == m.counters()


def test_batch_larger_than_one_pack_matches_alone():
    """More simulations than one launch's parameter pack holds: the batch splits them into
    packs whose launch sequences run as parallel graph branches."""
    import torch

    from paper_1912_04674_gb300 import lpic as L
    base = dataclasses.replace(C1, a0=0.5, L=6.0, n0=0.004, sort_every=4, ppc=(1, 1, 2))
    ws = [dataclasses.replace(base, name=f"p{k}", nx=40 + 4 * (k % 7), nr=16 + 2 * (k % 5),
                              w0=6.0 + 0.1 * k, seed=k) for k in range(61)]
    steps = [12 + (k % 3) for k in range(61)]
    mixed = [gpu_from(w, precision="fp32") for w in ws]
    b = L.Batch(mixed, torch.cuda.Stream())
    with pytest.raises(L.LpicError):
        b.set_tuning(1000)                     # not a multiple of 256
    b.set_tuning(1024)                         # several items per simulation
    b.step([5] * len(ws))
    b.set_tuning(8192, 5)                      # re-planned between steps, five branches
    b.step([n - 5 for n in steps])
    b.close()
    for w, m, n in zip(ws, mixed, steps):
        a = gpu_from(w, precision="fp32")
        a.step(n)
        assert m.counters() == a.counters()
        assert rel_err(m.field("ex"), a.field("ex")) < 1e-5
        assert rel_err(m.field("a"), a.field("a")) < 1e-5


def test_served_mix_matches_alone_and_respects_budget():
    from paper_1912_04674_gb300 import serve
    jobs_w = small_jobs() + [dataclasses.replace(small_jobs()[1], name="j3", seed=9, a0=0.3)]
    steps = [40, 60, 30, 50]
    arrivals = [0.0, 0.0, 0.05, 0.1]
    fp = [serve.job_footprint(w, "fp32", 20) for w in jobs_w]
    budget = sum(sorted(fp)[-2:]) + 1024          # at most two (largest) jobs fit at once
    srv = serve.ScanServer(budget, precision="fp32", max_slots=8, chunk_steps=7)
    jobs = [serve.Job(w, n, t) for w, n, t in zip(jobs_w, steps, arrivals)]
    rep = srv.run(jobs)
    assert rep["jobs"] == 4 and rep["rejected"] == 0
    assert rep["max_concurrent"] <= 3 and rep["p99_s"] >= rep["p50_s"] > 0
    from paper_1912_04674_gb300 import autotune
    for j in jobs:
        w = j.workload
        s = serve.make_simulation(w, "fp32", autotune.sort_every_for(w.nx, w.nr, w.ppc, "fp32"))
        s.step(j.steps)
        assert rel_err(j.result["ex_axis"], s.ex_axis()) < 1e-5
        assert abs(j.result["a_abs_max"] / s.a_abs_max() - 1) < 1e-5
        assert j.result["counters"]["step"] == j.steps


def test_server_rejects_malformed_job_and_keeps_serving():
    from paper_1912_04674_gb300 import serve
    good = small_jobs()[0]
    bad = dataclasses.replace(good, name="bad", dt=1.0)      # violates the Yee limit
    srv = serve.ScanServer(1 << 34, precision="fp32", chunk_steps=5)
    rep = srv.run([serve.Job(good, 15, 0.0), serve.Job(bad, 15, 0.0)])
    assert rep["jobs"] == 1 and rep["rejected"] == 1
    assert "stability" in srv.rejected[0].result["error"]


def test_one_slot_server_retires_and_admits_in_turn():
    """With one slot every admission follows a retirement, so each new job must get a batch
    of its own (membership changes even when the host objects' storage is reused)."""
    from paper_1912_04674_gb300 import autotune, serve
    ws = small_jobs()
    srv = serve.ScanServer(1 << 34, precision="fp32", max_slots=1, chunk_steps=9)
    jobs = [serve.Job(w, 25 + 5 * k, 0.0) for k, w in enumerate(ws)]
    rep = srv.run(jobs)
    assert rep["jobs"] == 3 and rep["max_concurrent"] == 1
    for j in jobs:
        w = j.workload
        s = serve.make_simulation(w, "fp32", autotune.sort_every_for(w.nx, w.nr, w.ppc, "fp32"))
        s.step(j.steps)
        assert rel_err(j.result["ex_axis"], s.ex_axis()) < 1e-5
        assert j.result["counters"] == s.counters()
