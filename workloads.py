"""Seeded synthetic workloads, shared by the tests, the smoke check and the benchmark.

Only parameters live here (grid, laser, plasma, seeds); no arithmetic of the method.  Both
the CUDA library and the CPU oracle generate the plasma lattice and the laser envelope
themselves from these numbers.  Shapes follow the paper's benchmarks (Sec. 4): Gaussian
envelopes, uniform or ramped plasma near 0.0017 n_c, dt = 0.8 dx, regular particles per cell.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    nr: int
    dx: float
    dr: float
    dt: float
    steps: int
    a0: float
    w0: float
    L: float
    n0: float
    ramp_cells: int = 0
    ppc: tuple = (2, 2, 4)
    seed: int = 0
    moving_window: bool = True
    sort_every: int = 20

    @property
    def x_center(self) -> float:
        """Pulse centre 3 L behind the window front; focus at the centre at t = 0."""
        return self.nx * self.dx - 3.0 * self.L

    @property
    def ramp_len(self) -> float:
        return self.ramp_cells * self.dx

    @property
    def particles(self) -> int:
        return self.nx * self.nr * self.ppc[0] * self.ppc[1] * self.ppc[2]


# Plain FP64 run: 256 x 64 cells, 262,144 electrons, linear regime.
C1 = Workload("c1_fp64_256x64", nx=256, nr=64, dx=0.69, dr=1.5, dt=0.8 * 0.69, steps=200,
              a0=0.1, w0=30.0, L=20.0, n0=0.0017)
# Single run FP32 vs FP64: 2048 x 256 cells, 8,388,608 electrons, 200-cell up-ramp at the
# back of the initial window, nonlinear driver.
# Sort cadence 60: measured at the developed wake (step 2600), the step time falls from
# 0.377 ms at k = 5 to 0.333 at k = 20 and 0.320 at k = 60 (0.319 at k = 100): background
# electrons keep their lab cells, so runs of equal cells survive many steps between sorts.
C2 = Workload("c2_2048x256_8.4M", nx=2048, nr=256, dx=0.69, dr=1.5, dt=0.8 * 0.69, steps=5000,
              a0=2.0, w0=60.0, L=25.0, n0=0.0017, ramp_cells=200, sort_every=60)
# Large single run: 8192 x 512 cells, 67,108,864 electrons.
C3 = Workload("c3_8192x512_67M", nx=8192, nr=512, dx=0.69, dr=1.5, dt=0.8 * 0.69, steps=10000,
              a0=3.0, w0=80.0, L=30.0, n0=0.001, sort_every=60)

ALL = {w.name: w for w in (C1, C2, C3)}


def scan_jobs(n: int = 64, seed: int = 1, nx_range=(256, 2048), nr_range=(64, 256)):
    """Parametric-scan jobs (batched and served forms): Nx, Nr uniform, a0 ~ U[0.5, 3],
    n0 log-uniform in [5e-4, 5e-3] n_c, w0 ~ U[30, 80], dr chosen so that r_max >= 3 w0."""
    import numpy as np

    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        nr = int(rng.integers(nr_range[0], nr_range[1] + 1))
        a0 = float(rng.uniform(0.5, 3.0))
        n0 = float(np.exp(rng.uniform(np.log(5e-4), np.log(5e-3))))
        w0 = float(rng.uniform(30.0, 80.0))
        dr = max(1.5, 3.0 * w0 / nr)
        jobs.append(Workload(f"scan{k}", nx=nx, nr=nr, dx=0.69, dr=dr, dt=0.8 * 0.69, steps=2000,
                             a0=a0, w0=w0, L=25.0, n0=n0, seed=k))
    return jobs
