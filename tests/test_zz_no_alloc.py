"""The allocation-free envelope statistics entry point, for callers that cannot call
cudaMalloc (their device memory all comes from a pool they were handed), checked against
lpic_diagnose's peak |A| and waist on the same envelope, on two calls in a row.

The test itself allocates its input and output with PyTorch: it stands in for the caller's
pool; the entry point under test allocates nothing.  Collected last on purpose."""
import dataclasses

import numpy as np
import pytest

from workloads import C1

pytestmark = pytest.mark.gpu
TOL = 1e-12   # same bar as the FP64 diagnostics tests


def test_envelope_stats_without_allocation_two_calls():
    import torch

    from paper_1912_04674_gb300 import build, lpic as L
    build.build()
    w = dataclasses.replace(C1, name="noalloc", nx=200, nr=60, a0=0.7, w0=20.0, L=12.0)
    sim = L.Simulation(L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, w.sort_every),
                       L.Laser(w.a0, w.w0, w.L, w.x_center, w.x_center),
                       L.Plasma(w.n0, 0.0, 0.0, w.ppc, w.seed), precision="fp64")
    dev = sim.device
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    for nsteps in (3, 40):           # two calls in a row, on different envelopes
        sim.step(nsteps)
        amax_ref, waist_ref = sim.a_abs_max(), sim.waist()
        a = torch.from_numpy(np.ascontiguousarray(sim.field("a")).view(np.float64).copy()).to(dev)
        torch.cuda.synchronize(dev)
        with torch.cuda.device(dev):
            L.lpic_envelope_stats_noalloc(a.data_ptr(), w.nx, w.nr, w.dr, out.data_ptr(),
                                          stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] / amax_ref - 1) < TOL, (got[0], amax_ref)
        assert abs(got[1] / waist_ref - 1) < TOL, (got[1], waist_ref)
        out.fill_(float("nan"))
    with pytest.raises(L.LpicError) as e:   # beyond the fixed scratch
        L.lpic_envelope_stats_noalloc(a.data_ptr(), 8191, 4096, w.dr, out.data_ptr(), stream.cuda_stream)
    assert e.value.status == 4
    sim.close()
