"""x-slab decomposition on one GPU against the whole-window FP64 oracle (Sec. 3: the solver
parallelises like a standard Yee scheme, by sub-domains exchanging guard cells).

Two and three slabs, all on one device and one stream, stepped through window shifts with
plasma injected at the front slab; after every step the whole-window fields assembled from the
slabs' owned columns and the electrons each slab owns agree with the oracle to 1e-10 (FP64;
electrons matched by id, each owned by exactly one slab)."""
import dataclasses

import numpy as np
import pytest

from helpers import field_errors, oracle_from, particle_errors
from workloads import C1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def slab_sim(w, nslab, precision="fp64", halo=None):
    from paper_1912_04674_gb300 import lpic as L
    from paper_1912_04674_gb300.slabs import SlabSimulation
    g = L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, w.moving_window, w.sort_every)
    return SlabSimulation(g, L.Laser(w.a0, w.w0, w.L, w.x_center, w.x_center),
                          L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed), nslab=nslab, halo=halo,
                          precision=precision)


W = dataclasses.replace(C1, name="slabs", nx=96, nr=24, a0=0.8, w0=8.0, L=5.0, n0=0.01, ramp_cells=12,
                        sort_every=5)


@pytest.mark.parametrize("nslab,precision,tol", [(2, "fp64", 1e-10), (3, "fp64", 1e-10), (2, "fp32", 1e-3)])
def test_slabs_equal_the_whole_window_oracle_every_step(nslab, precision, tol):
    o = oracle_from(W)
    s = slab_sim(W, nslab, precision)
    worst = {}
    for step in range(30):
        o.step(1)
        s.step(1)
        errs = {**field_errors(o, s), **particle_errors(o, s)}
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, (step, bad)
        worst = {k: max(worst.get(k, 0.0), v) for k, v in errs.items()}
    c = s.counters()
    assert c["step"] == o.step_index == 30 and c["shift"] == o.shift >= 20
    assert len(s.particles()["id"]) == o.np
    s.close()


def test_slab_exchange_refuses_mismatched_slabs():
    from paper_1912_04674_gb300 import lpic as L
    s = slab_sim(W, 2)
    a, b = s.sims
    with pytest.raises(L.LpicError) as e:
        L.lpic_slab_exchange(a.ctx, b.ctx, s.halo + 1)        # boundary does not match
    assert e.value.status == 1
    with pytest.raises(L.LpicError):
        L.lpic_slab_exchange(b.ctx, a.ctx, s.halo)            # wrong order
    a.step(1)                                                 # one slab a step ahead
    with pytest.raises(L.LpicError):
        L.lpic_slab_exchange(a.ctx, b.ctx, s.halo)
    s.close()
