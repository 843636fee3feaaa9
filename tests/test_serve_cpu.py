"""Host-side logic of the serving form (no GPU): admission order against the memory budget
and slots, rejection of malformed jobs, seeded Poisson arrivals."""
import dataclasses

import numpy as np
import pytest

from paper_1912_04674_gb300 import serve


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def test_admission_first_fit_within_budget_and_slots():
    assert serve.admit_order([10, 50, 20, 5], used=0, budget=40, running=0, slots=8) == [0, 2, 3]
    assert serve.admit_order([10, 10, 10], used=25, budget=40, running=0, slots=8) == [0]
    assert serve.admit_order([1, 1, 1, 1], used=0, budget=100, running=6, slots=8) == [0, 1]
    assert serve.admit_order([], used=0, budget=1, running=0, slots=1) == []


def test_malformed_jobs_are_rejected_with_a_reason():
    import workloads
    w = workloads.scan_jobs(1)[0]
    assert serve.validate(w) is None
    assert "stability" in serve.validate(dataclasses.replace(w, dt=1.0))
    assert serve.validate(dataclasses.replace(w, w0=float("nan"))) is not None
    assert serve.validate(dataclasses.replace(w, n0=-1.0)) is not None


def test_poisson_arrivals_are_seeded_and_have_the_rate():
    a = serve.poisson_jobs(400, 2.0, seed=7)
    b = serve.poisson_jobs(400, 2.0, seed=7)
    assert [j.arrival for j in a] == [j.arrival for j in b]
    t = np.array([j.arrival for j in a])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] / 2.0 - 1) < 0.15        # mean rate 2 jobs/s
    steps = np.array([j.steps for j in a])
    assert steps.min() >= 500 and steps.max() <= 3000


def test_negative_step_counts_are_rejected_before_admission():
    """A job with a negative or non-integer step count is rejected on its own; it never
    reaches the batch (where it would stop every job in flight)."""
    import workloads
    srv = object.__new__(serve.ScanServer)       # host bookkeeping only: no device stream
    srv.queue, srv.rejected, srv.running = [], [], []
    srv.used, srv.budget, srv.max_slots, srv.max_running = 0, 0, 4, 0
    srv.precision = "fp32"
    w = workloads.scan_jobs(1)[0]
    bad = [serve.Job(w, -5, 0.0, 0), serve.Job(w, 2.5, 0.0, 1)]
    srv.queue = list(bad)
    assert srv._admit(0.0) is False              # budget 0: nothing valid fits either
    assert [j.job_id for j in srv.rejected] == [0, 1]
    assert all("steps" in j.result["error"] for j in srv.rejected)
    assert srv.queue == [] and srv.running == []
