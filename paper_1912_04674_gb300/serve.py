"""Continuous-batching server for parametric scans of the envelope PIC method.

Jobs (a0, density, waist, grid size, step count) arrive over time.  Each admitted job owns
its simulation state on the device until it finishes (fields and particles stay resident);
admission is by device-memory footprint (lpic_required_bytes) against a budget and by a
slot count.  All running jobs advance together through one lpic_batch (per step, one
fused launch per phase over every active simulation, replayed from a CUDA graph); jobs
that arrive while others run are admitted at the next step boundary, and finished jobs
retire there, freeing their memory for the queue.
The server records each job's time to result (completion minus arrival) and reports the
p50/p99 latency, jobs/hour and aggregate particle-steps/s.

The loop is single-threaded on the host; every step's work runs in the CUDA library.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import autotune
from . import lpic as L


@dataclass
class Job:
    workload: object                 # workloads.Workload (parameters only)
    steps: int
    arrival: float = 0.0             # seconds after the server's start
    job_id: int = -1
    # filled in by the server
    admitted: float | None = None
    finished: float | None = None
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


class _Running:
    def __init__(self, job: Job, sim: L.Simulation, nbytes: int):
        self.job, self.sim, self.nbytes = job, sim, nbytes
        self.remaining = job.steps
        self.particle_steps = 0.0


def job_footprint(w, precision: str, sort_every: int) -> int:
    g = L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, sort_every)
    gs = L.grid_struct(g, L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed))
    return L.lpic_required_bytes(gs, L.PRECISION[precision]) + 256


def make_simulation(w, precision: str, sort_every: int) -> L.Simulation:
    g = L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, sort_every)
    return L.Simulation(g, L.Laser(w.a0, w.w0, w.L, w.x_center, w.x_center),
                        L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed), precision=precision)


def admit_order(queue_bytes: list[int], used: int, budget: int, running: int,
                slots: int) -> list[int]:
    """Indices of queued jobs (in arrival order, footprints queue_bytes) admitted now:
    first-fit in arrival order against the free memory and the free slots, so a large job
    at the head does not block smaller ones behind it."""
    out = []
    for k, need in enumerate(queue_bytes):
        if running + len(out) >= slots:
            break
        if used + need <= budget:
            out.append(k)
            used += need
    return out


def validate(w) -> str | None:
    """Reason a job cannot run (None if it can)."""
    try:
        g = L.grid_struct(L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, 20))
        L.lpic_check_params(g, L.plasma_struct(L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed)))
        if not all(np.isfinite([w.a0, w.w0, w.L])) or w.w0 <= 0 or w.L <= 0:
            return "laser parameters must be finite with w0 > 0, L > 0"
    except L.LpicError as e:
        return str(e)
    return None


def collect_result(sim: L.Simulation) -> dict:
    return {"ex_axis": sim.ex_axis(), "a_abs_max": sim.a_abs_max(),
            "accel_energy": sim.accel_energy(), "counters": sim.counters()}


class ScanServer:
    def __init__(self, hbm_budget_bytes: int, precision: str = "fp32", max_slots: int = 64,
                 chunk_steps: int = 10, device: int = 0):
        import torch

        self.budget = int(hbm_budget_bytes)
        self.precision = precision
        self.max_slots = max_slots
        self.chunk = chunk_steps
        self.device = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(self.device)
        self.queue: list[Job] = []
        self.running: list[_Running] = []
        self.done: list[Job] = []
        self.used = 0
        self._batch = None
        self._batch_key = None
        self.t0 = None
        self.particle_steps = 0.0
        self.max_running = 0
        self.rejected: list[Job] = []
        self.launches = 0               # kernels enqueued by the batches

    # -- batch membership ----------------------------------------------------------------
    def _rebuild_batch(self):
        # membership by job id (unique per run); object ids can be reused after a retirement
        key = tuple(r.job.job_id for r in self.running)
        if key == self._batch_key:
            return
        if self._batch is not None:
            self.launches += self._batch.launches()
            self._batch.close()
            self._batch = None
        if self.running:
            self._batch = L.Batch([r.sim for r in self.running], self.stream)
            # a tuned work-item size if one was measured for this bucket (tuning itself
            # would advance the jobs past their step counts, so the server never tunes)
            total = sum(int(r.sim.gs.particle_capacity) for r in self.running)
            self._batch.set_tuning(*autotune.batch_tuning_for(total, len(self.running), self.precision))
        self._batch_key = key

    def _admit(self, now: float):
        ok = []
        for job in self.queue:
            why = validate(job.workload)
            if why is None and (not isinstance(job.steps, (int, np.integer)) or job.steps < 0):
                why = f"steps must be a non-negative integer (got {job.steps!r})"
            if why:
                job.result = {"error": why}
                job.finished = now
                self.rejected.append(job)
            else:
                ok.append(job)
        self.queue = ok
        plans = []
        for job in self.queue:
            w = job.workload
            k = autotune.sort_every_for(w.nx, w.nr, w.ppc, self.precision)
            plans.append((k, job_footprint(w, self.precision, k)))
        take = admit_order([b for _, b in plans], self.used, self.budget, len(self.running),
                           self.max_slots)
        for idx in take:
            job, (k, need) = self.queue[idx], plans[idx]
            try:
                sim = make_simulation(job.workload, self.precision, k)
            except L.LpicError as e:     # this job cannot be set up: reject it alone
                job.result = {"error": str(e)}
                job.finished = now
                self.rejected.append(job)
                continue
            job.admitted = now
            self.running.append(_Running(job, sim, need))
            self.used += need
        taken = set(take)
        self.queue = [j for n, j in enumerate(self.queue) if n not in taken]
        self.max_running = max(self.max_running, len(self.running))
        return bool(take)

    def _retire(self, now: float):
        keep = []
        for r in self.running:
            if r.remaining > 0:
                keep.append(r)
                continue
            try:
                r.job.result = collect_result(r.sim)
                self.done.append(r.job)
            except L.LpicError as e:     # a device-side error of this job only
                r.job.result = {"error": str(e)}
                self.rejected.append(r.job)
            r.job.finished = now
            r.sim.close()
            self.used -= r.nbytes
        changed = len(keep) != len(self.running)
        self.running = keep
        return changed

    # -- main loop -------------------------------------------------------------------------
    def run(self, jobs: list[Job], clock=time.perf_counter) -> dict:
        """Serve `jobs` (arrival times in seconds from now) until all are done."""
        import torch

        pending = sorted(jobs, key=lambda j: j.arrival)
        if len({j.job_id for j in pending}) != len(pending) or any(j.job_id < 0 for j in pending):
            for n, j in enumerate(pending):   # ids must be unique: they key the batch membership
                j.job_id = n
        self.t0 = clock()
        while pending or self.queue or self.running:
            now = clock() - self.t0
            while pending and pending[0].arrival <= now:
                self.queue.append(pending.pop(0))
            if self.queue:
                self._admit(now)
            if not self.running:
                if pending:  # idle until the next arrival
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.05)))
                    continue
                if self.queue:   # nothing runs and the head still does not fit: it never will
                    for job in self.queue:
                        job.result = {"error": "footprint exceeds the memory budget"}
                        job.finished = now
                        self.rejected.append(job)
                    self.queue = []
                break
            self._rebuild_batch()
            steps = [min(self.chunk, r.remaining) for r in self.running]
            self._batch.step(steps)
            self.stream.synchronize()
            for r, s in zip(self.running, steps):
                r.remaining -= s
                r.particle_steps += s * r.job.workload.particles
                self.particle_steps += s * r.job.workload.particles
            if any(r.remaining == 0 for r in self.running):
                # the contexts' own streams are ordered after the batch stream
                self._retire(clock() - self.t0)
        if self._batch is not None:
            self.launches += self._batch.launches()
            self._batch.close()
            self._batch = None
        torch.cuda.synchronize(self.device)
        return self.report(clock() - self.t0)

    def report(self, elapsed: float) -> dict:
        lat = np.array([j.latency for j in self.done if j.latency is not None])
        return {"jobs": len(self.done), "rejected": len(self.rejected), "elapsed_s": elapsed,
                "max_concurrent": self.max_running, "gpu_launches": self.launches,
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "jobs_per_hour": len(self.done) / elapsed * 3600.0 if elapsed > 0 else None,
                "particle_steps_per_s": self.particle_steps / elapsed if elapsed > 0 else None}


def poisson_jobs(n: int, rate_per_s: float, steps_range=(500, 3000), seed: int = 2,
                 job_seed: int = 1, nx_range=(256, 2048), nr_range=(64, 256)) -> list[Job]:
    """Jobs drawn as in the scan workload, with Poisson arrival times and uniform step counts."""
    import workloads
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    scans = workloads.scan_jobs(n, seed=job_seed, nx_range=nx_range, nr_range=nr_range)
    steps = rng.integers(steps_range[0], steps_range[1] + 1, n)
    return [Job(w, int(s), float(a), k) for k, (w, s, a) in enumerate(zip(scans, steps, t))]
