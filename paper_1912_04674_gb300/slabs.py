"""x-slab decomposition of one simulation (Sec. 3: the envelope solver parallelises with the
strategies of a standard Yee scheme, sub-domains that exchange guard cells).

The window of Nx cells is cut into slabs along x.  Slab k owns the cells [b_k, b_{k+1}) and
holds, as one context of the library, the columns [b_k - halo, b_{k+1} + halo] clipped to the
window: its owned cells plus `halo` columns on each inner side.  Every slab computes its whole
local window each step (the halo columns redundantly, with wrong boundary values at its local
edges); then `lpic_slab_exchange` overwrites each halo with the owner's fields and electrons.
One step's phases reach at most 6 columns from a wrong boundary value, so with halo >= 8 the
owned columns come out exactly as a whole-window run computes them.  Only the front slab
injects plasma at the moving window's front; the slabs shift together (the library's window
rule counts the global shifts, see ``slab_x0``).

All slabs live on one device and share one stream here.  The exchange is a neighbour exchange
of whole columns and of the electrons in the halo cells; on several devices the same copies
would go through a peer copy into a local buffer first.  `plan_slabs` and `exchange_sets` are
the host-side bookkeeping (which columns and which electrons go where), also used by the
multi-process tests.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np

from . import lpic as L

STEP_REACH = 6        # columns one step's phases reach from a wrong boundary value
MIN_HALO = STEP_REACH + 2


@dataclass(frozen=True)
class Slab:
    index: int
    x0: int          # global window column of local column 0
    nx: int          # local cells
    own_lo: int      # owned global cells [own_lo, own_hi)
    own_hi: int
    front: bool      # holds the window front: the moving window injects plasma here


def min_halo(filter_passes: int = 0) -> int:
    return MIN_HALO + int(filter_passes)


def plan_slabs(nx: int, nslab: int, halo: int) -> list[Slab]:
    """Cut nx cells into nslab slabs of near-equal owned width, each with `halo` columns on
    its inner sides; every owned width must be at least 2*halo."""
    if nslab < 1 or halo < 1:
        raise ValueError("nslab >= 1 and halo >= 1 required")
    bounds = [round(k * nx / nslab) for k in range(nslab + 1)]
    slabs = []
    for k in range(nslab):
        a, b = bounds[k], bounds[k + 1]
        if b - a < 2 * halo:
            raise ValueError(f"slab {k} owns {b - a} cells, fewer than 2*halo = {2 * halo}")
        lo = a - halo if k > 0 else 0
        hi = b + halo if k < nslab - 1 else nx
        slabs.append(Slab(k, lo, hi - lo, a, b, k == nslab - 1))
    return slabs


def owned_nodes(sl: Slab, nx: int) -> tuple[int, int]:
    """Global node (or cell) columns a slab contributes to a whole-window array: its owned
    cells, and for the last slab also the final node column nx."""
    return sl.own_lo, (sl.own_hi + 1 if sl.own_hi == nx else sl.own_hi)


def exchange_sets(left: Slab, cells_left: np.ndarray, right: Slab, cells_right: np.ndarray, halo: int) -> dict:
    """The electron bookkeeping of one exchange at the boundary B between `left` and `right`,
    from the global cells of each slab's electrons: which each keeps (left: cells < B, right:
    cells >= B) and which each sends (right's cells in [B, B+halo) to left, left's cells in
    [B-halo, B) to right).  The CUDA exchange applies the same rules on the device."""
    B = right.own_lo
    assert B == left.own_hi and right.x0 == B - halo and left.x0 + left.nx == B + halo
    keep_l = cells_left < B
    keep_r = cells_right >= B
    send_r2l = keep_r & (cells_right < B + halo)
    send_l2r = keep_l & (cells_left >= B - halo)
    return {"keep_left": np.flatnonzero(keep_l), "keep_right": np.flatnonzero(keep_r),
            "right_to_left": np.flatnonzero(send_r2l), "left_to_right": np.flatnonzero(send_l2r)}


class SlabSimulation:
    """One simulation cut into x-slabs on one device (all slabs on one stream)."""

    def __init__(self, grid: L.Grid, laser: L.Laser | None, plasma: L.Plasma | None, nslab: int = 2,
                 halo: int | None = None, precision: str = "fp64", device: int = 0):
        import torch

        self.grid = grid
        self.halo = halo if halo is not None else min_halo(grid.filter_passes)
        if self.halo < min_halo(grid.filter_passes):
            raise ValueError(f"halo {self.halo} below the {min_halo(grid.filter_passes)} columns one step reaches")
        self.plan = plan_slabs(grid.nx, nslab, self.halo)
        self.stream = torch.cuda.Stream(torch.device("cuda", device))
        self.sims = []
        for sl in self.plan:
            g = dataclasses.replace(grid, nx=sl.nx, slab_x0=sl.x0, slab_front_interior=not sl.front)
            cap = L.lpic_particle_capacity(L.grid_struct(g), L.plasma_struct(plasma)) if plasma else 0
            if plasma:
                # every exchange removes the halo electrons (holes until the next sort) and
                # appends fresh copies: room for one halo of appends per inner side and step
                # between compactions, at up to twice the lattice density
                sides = (sl.index > 0) + (not sl.front)
                cap += (grid.sort_every + 2) * sides * 2 * self.halo * grid.nr * int(np.prod(plasma.ppc))
            sim = L.Simulation(g, None, None, precision=precision, device=device, stream=self.stream,
                               capacity=cap)
            sim.upload_counters(0, sl.x0)        # local column 0 is lab cell x0 at t = 0
            if laser is not None:
                L.lpic_init_envelope(sim.ctx, L.laser_struct(laser))
            if plasma is not None:
                L.lpic_load_plasma(sim.ctx, L.plasma_struct(plasma))
            self.sims.append(sim)

    def close(self):
        for s in self.sims:
            s.close()

    def step(self, n: int = 1):
        for _ in range(n):
            for s in self.sims:
                s.step(1)
            for k in range(len(self.sims) - 1):
                L.lpic_slab_exchange(self.sims[k].ctx, self.sims[k + 1].ctx, self.halo)

    # -- whole-window views ----------------------------------------------------------------------
    def counters(self) -> dict:
        c = self.sims[0].counters()
        return {"step": c["step"], "shift": c["shift"] - self.plan[0].x0}

    def field(self, name: str) -> np.ndarray:
        """A whole-window array (canonical layout) assembled from each slab's owned columns."""
        nx = self.grid.nx
        cells = name in ("ex", "bt", "jx")
        parts = []
        for sl, s in zip(self.plan, self.sims):
            lo, hi = (sl.own_lo, sl.own_hi) if cells else owned_nodes(sl, nx)
            parts.append(s.field(name)[lo - sl.x0:hi - sl.x0])
        return np.concatenate(parts, axis=0)

    def ex_axis(self) -> np.ndarray:
        return self.field("ex")[:, 0]

    def particles(self) -> dict:
        """The electrons of the whole window: each slab's electrons in the cells it owns."""
        shift = self.counters()["shift"]
        out = {k: [] for k in (*L.PART_COMPONENTS, "id")}
        for sl, s in zip(self.plan, self.sims):
            p = s.particles()
            cell = np.floor(p["x"] / self.grid.dx).astype(np.int64) - shift
            sel = (cell >= sl.own_lo) & (cell < sl.own_hi)
            for k in out:
                out[k].append(p[k][sel])
        return {k: np.concatenate(v) for k, v in out.items()}
