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
