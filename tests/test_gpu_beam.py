"""Beam parameters of the injected electrons (Table BeamParams quantities, Sec. 4) from the
GPU diagnostic against the oracle's definitions, on the same uploaded particle set.

Bar: FP64, the integer-valued fields (counts, bins) exactly and the rest to 1e-10 (the
energies and bin decisions are evaluated without contraction on both sides, so only the
order of the weighted sums differs); FP32_MIXED (momenta stored in FP32) to 1e-4, counts to
a few electrons at bin and window edges.
"""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_from
from oracle.beam import FIELDS, beam_parameters
from workloads import C1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def synthetic_beam(rng, nx, nr, dx, dr):
    """A plasma at rest, a low-energy tail and a GeV-class bunch with a Gaussian spectrum."""
    n_bg, n_tail, n_b = 6000, 800, 3000
    x = rng.uniform(2 * dx, (nx - 2) * dx, n_bg + n_tail + n_b)
    r = rng.uniform(0, 0.8 * nr * dr, len(x))
    th = rng.uniform(0, 2 * np.pi, len(x))
    e = np.concatenate([rng.uniform(0, 0.01, n_bg), rng.uniform(15, 80, n_tail),
                        rng.normal(600.0, 12.0, n_b)])
    g = 1.0 + e
    pt = np.concatenate([np.zeros(n_bg), rng.normal(0, 0.5, n_tail), rng.normal(0, 2.0, n_b)])
    phi = rng.uniform(0, 2 * np.pi, len(x))
    py, pz = pt * np.cos(phi), pt * np.sin(phi)
    px = np.sqrt(np.maximum(g * g - 1.0 - py * py - pz * pz, 0.0))
    y, z = r * np.cos(th), r * np.sin(th)
    # a correlated transverse phase space for the bunch
    py[-n_b:] += 0.05 * y[-n_b:]
    w = rng.uniform(0.5, 1.5, len(x)) * 1e-3
    return dict(x=x, y=y, z=z, px=px, py=py, pz=pz, w=w)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_beam_parameters_match_oracle(precision):
    w = dataclasses.replace(C1, nx=96, nr=48)
    rng = np.random.default_rng(7)
    parts = synthetic_beam(rng, w.nx, w.nr, w.dx, w.dr)
    g = gpu_from(w, precision=precision, plasma=False, capacity=20000)
    g.upload_particles(parts)
    got = g.beam_parameters()
    src = g.particles() if precision == "fp32" else parts      # the values the GPU holds
    want = beam_parameters(src["px"], src["py"], src["pz"], src["y"], src["z"], src["w"])
    assert want["n_beam"] > 2000 and want["eps_mean"] > 0
    if precision == "fp64":
        for k in ("n_accel", "n_beam", "nbins"):
            assert got[k] == want[k], k
        for k in FIELDS:
            assert abs(got[k] - want[k]) <= 1e-10 * max(abs(want[k]), 1e-300), (k, got[k], want[k])
    else:
        assert got["n_accel"] == want["n_accel"] and got["nbins"] == want["nbins"]
        assert abs(got["n_beam"] - want["n_beam"]) <= 3
        for k in ("charge", "e_peak", "fwhm", "de_over_e", "eps_y", "eps_z", "e_mean", "e_max"):
            assert abs(got[k] / want[k] - 1) < 1e-4, (k, got[k], want[k])


def test_no_accelerated_electrons_gives_zeros():
    g = gpu_from(C1)
    b = g.beam_parameters()
    assert b["n_accel"] == 0 and b["charge"] == 0 and b["e_peak"] == 0 and b["nbins"] == 256
