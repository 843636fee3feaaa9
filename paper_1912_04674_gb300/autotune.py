"""Autotuners for the sort cadence of a simulation shape and the work-item size of a batch.

The counting sort keeps particles ordered by cell so that warps gather from and deposit to
few cells; sorting too often wastes bandwidth, too rarely lets particles drift apart.  For a
shape (Nx, Nr, particles per cell, precision) the tuner times a short run of the real step
for each candidate cadence on the current GPU and keeps the fastest in a JSON cache beside
the built library.  Shapes are bucketed (Nx and Nr rounded to powers of two) so that a
parameter scan reuses a handful of measurements.

The fused particle passes of a batch walk items of a fixed number of particle slots; small
items balance the blocks, large ones cost less per item.  The batch tuner times real steps
of the batch itself (the simulations advance while it measures, so no work is wasted) for
each candidate item size and pack count, and the unfused schedule (each simulation's own
step graph on its own stream, which overlaps better when the simulations are large), and
keeps the fastest, cached per precision, sim count and total-capacity bucket.
"""
from __future__ import annotations

import json
import math
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "_build", "autotune.json")
CANDIDATES = (10, 20, 40, 60, 100)
DEFAULT = 20
TILE_CANDIDATES = (2048, 4096, 8192, 16384)
TILE_DEFAULT = 4096
PACK_CANDIDATES = (2, 4, 8, 16)
_lock = threading.Lock()


def _bucket(nx: int, nr: int, ppc: tuple, precision: str) -> str:
    b = lambda v: 2 ** round(math.log2(max(v, 1)))  # noqa: E731
    return f"{b(nx)}x{b(nr)}:{ppc[0]}x{ppc[1]}x{ppc[2]}:{precision}"


def _load() -> dict:
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def cached_sort_every(nx: int, nr: int, ppc: tuple, precision: str) -> int | None:
    return _load().get(_bucket(nx, nr, ppc, precision))


def tune_sort_every(workload, precision: str = "fp32", steps: int = 40,
                    candidates=CANDIDATES) -> int:
    """Measure each candidate cadence on `workload` (a workloads.Workload) and cache the best."""
    import dataclasses

    import torch

    from . import lpic as L

    key = _bucket(workload.nx, workload.nr, workload.ppc, precision)
    with _lock:
        hit = _load().get(key)
    if hit:
        return int(hit)
    best, best_ms = DEFAULT, float("inf")
    for k in candidates:
        w = dataclasses.replace(workload, sort_every=k)
        sim = L.Simulation(L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, k),
                           L.Laser(w.a0, w.w0, w.L, w.x_center, w.x_center),
                           L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed), precision=precision)
        sim.step(2 * k)  # let the particles drift as they do between sorts
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(steps, 2 * k)
        torch.cuda.synchronize()
        a.record(sim.stream)
        sim.step(n)
        b.record(sim.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        sim.close()
        if ms < best_ms:
            best, best_ms = k, ms
    with _lock:
        data = _load()
        data[key] = best
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        json.dump(data, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    return best


def sort_every_for(nx: int, nr: int, ppc: tuple, precision: str) -> int:
    """Cadence for a shape: the tuned value if one was measured for its bucket, else 20."""
    v = cached_sort_every(nx, nr, ppc, precision)
    return int(v) if v else DEFAULT


def _batch_bucket(total_capacity: int, n_sims: int, precision: str) -> str:
    b = lambda v: 2 ** round(math.log2(max(v, 1)))  # noqa: E731
    return f"batch:{b(total_capacity)}:{b(n_sims)}:{precision}"


def _time_batch(batch, steps: int) -> float:
    import torch

    n = len(batch.sims)
    batch.step([1] * n)  # records the graph for this setting outside the timed region
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(batch.stream)
    batch.step([steps] * n)
    b.record(batch.stream)
    b.synchronize()
    return a.elapsed_time(b) / steps


def tune_batch(batch, precision: str, steps: int = 4, tiles=TILE_CANDIDATES,
               packs=PACK_CANDIDATES) -> tuple[int, int]:
    """Pick the work-item size and the pack count of `batch` (an lpic.Batch) by timing
    `steps` real batch steps per candidate (item size first, then packs at the best size,
    then packs = -1: the simulations' own step graphs, unfused); sets the winner on the
    batch, caches it and returns (particles_per_item, packs); the measurements are left in
    batch.tuning_log.  Every simulation of the batch advances (1 + steps) steps per
    candidate."""
    total = sum(int(s.gs.particle_capacity) for s in batch.sims)
    key = _batch_bucket(total, len(batch.sims), precision)
    with _lock:
        hit = _load().get(key)
    if hit:
        batch.set_tuning(int(hit[0]), int(hit[1]))
        return int(hit[0]), int(hit[1])
    best, best_ms = (TILE_DEFAULT, 0), float("inf")
    batch.tuning_log = []
    for c in tiles:
        batch.set_tuning(c, 0)
        ms = _time_batch(batch, steps)
        batch.tuning_log.append((c, 0, ms))
        if ms < best_ms:
            best, best_ms = (c, 0), ms
    for p in tuple(packs) + (-1,):
        if p == 0 or p > len(batch.sims):
            continue
        batch.set_tuning(best[0], p)
        ms = _time_batch(batch, steps)
        batch.tuning_log.append((best[0], p, ms))
        if ms < best_ms:
            best, best_ms = (best[0], p), ms
    batch.set_tuning(*best)
    with _lock:
        data = _load()
        data[key] = list(best)
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        json.dump(data, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    return best


def batch_tuning_for(total_capacity: int, n_sims: int, precision: str) -> tuple[int, int]:
    """(particles_per_item, packs) for a batch: the tuned values for its bucket if measured."""
    v = _load().get(_batch_bucket(total_capacity, n_sims, precision))
    return (int(v[0]), int(v[1])) if v else (TILE_DEFAULT, 0)
