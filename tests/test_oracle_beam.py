"""Pins of the oracle's beam parameters (Table BeamParams quantities, Sec. 4).

* emittance: a four-point beam (y = +-a, p_y = +-b, every combination, equal weights) has
  eps = a b exactly; a fully correlated beam (p_y = k y) has eps = 0; a linear symplectic map
  of the (y, p_y) plane (a shear p_y -> p_y + k y, a drift y -> y + L p_y) leaves eps unchanged;
* spectrum: a triangular spectrum sampled at the bin centres has its peak at the apex and a
  FWHM of half its base (linear interpolation is exact on a linear profile); a Gaussian
  spectrum gives FWHM = 2 sqrt(2 ln 2) sigma to within a bin; electrons outside 2 FWHM of the
  peak, and electrons below the p_x threshold, change nothing.
"""
import math

import numpy as np

from oracle.beam import beam_parameters, peak_and_fwhm


def beam_from_energy(e, rng):
    """Electrons moving along x with kinetic energy e (gamma - 1), tiny transverse momenta."""
    g = 1.0 + e
    px = np.sqrt(g * g - 1.0)
    n = len(e)
    return px, 1e-6 * rng.standard_normal(n), 1e-6 * rng.standard_normal(n)


def test_four_point_beam_emittance_exact():
    a, b = 3.0, 0.25
    y = np.array([a, a, -a, -a])
    py = np.array([b, -b, b, -b])
    px = np.full(4, 50.0)
    r = beam_parameters(px, py, py[::-1].copy(), y, y[::-1].copy(), np.ones(4), nbins=1)
    assert r["n_beam"] == 4
    assert abs(r["eps_y"] - a * b) < 1e-15 and abs(r["eps_z"] - a * b) < 1e-15


def test_correlated_beam_has_zero_emittance_and_symplectic_invariance():
    rng = np.random.default_rng(1)
    n = 4000
    y, z = rng.normal(0, 2.0, n), rng.normal(0, 1.5, n)
    py, pz = rng.normal(0, 0.3, n), rng.normal(0, 0.2, n)
    px = rng.normal(200.0, 1.0, n)
    w = rng.uniform(0.5, 1.5, n)
    corr = beam_parameters(px, 0.7 * y, -0.2 * z, y, z, w, nbins=64)
    assert corr["eps_y"] < 1e-12 * 2.0 * 0.7 * 2.0 and corr["eps_z"] < 1e-12
    base = beam_parameters(px, py, pz, y, z, w, nbins=64)
    shear = beam_parameters(px, py + 0.9 * y, pz, y, z, w, nbins=64)      # kick
    drift = beam_parameters(px, py, pz, y + 4.0 * py, z, w, nbins=64)     # drift
    for r in (shear, drift):
        assert abs(r["eps_y"] / base["eps_y"] - 1) < 1e-12
        assert r["n_beam"] == base["n_beam"]


def test_triangular_spectrum_peak_and_fwhm_exact():
    nbins, width = 40, 0.5
    centres = (np.arange(nbins) + 0.5) * width
    apex, half_base = centres[20], 6.0
    h = np.clip(1.0 - np.abs(centres - apex) / half_base, 0.0, None)
    e_peak, fwhm = peak_and_fwhm(h, width)
    assert e_peak == apex
    assert abs(fwhm - half_base) < 1e-12


def test_gaussian_spectrum_and_selection():
    rng = np.random.default_rng(2)
    sigma, e0 = 8.0, 300.0
    e = rng.normal(e0, sigma, 400000)
    px, py, pz = beam_from_energy(e, rng)
    y = rng.normal(0, 1.0, len(e))
    z = rng.normal(0, 1.0, len(e))
    w = np.ones(len(e))
    nb = 512        # ~13k electrons in the peak bin: the max-bin bias stays below 1 %
    r = beam_parameters(px, py, pz, y, z, w, nbins=nb)
    bin_w = r["e_max"] / nb
    assert abs(r["e_peak"] - e0) < 2 * bin_w + 0.05 * sigma
    assert abs(r["fwhm"] - 2 * math.sqrt(2 * math.log(2)) * sigma) < 0.05 * sigma
    # the beam is the core within +-FWHM: erf(FWHM/(sigma sqrt 2)) of the electrons
    frac = math.erf(2 * math.sqrt(2 * math.log(2)) / math.sqrt(2))
    assert abs(r["n_beam"] / len(e) - frac) < 0.01
    # a far low-energy tail and slow electrons do not change the beam
    e_tail = rng.uniform(20.0, 60.0, 5000)
    pxt, pyt, pzt = beam_from_energy(e_tail, rng)
    slow = np.full(100, 5.0)
    r2 = beam_parameters(np.concatenate([px, pxt, slow]), np.concatenate([py, pyt, np.zeros(100)]),
                         np.concatenate([pz, pzt, np.zeros(100)]),
                         np.concatenate([y, rng.normal(0, 1, 5000), np.zeros(100)]),
                         np.concatenate([z, rng.normal(0, 1, 5000), np.zeros(100)]),
                         np.ones(len(e) + 5100), nbins=nb)
    assert r2["n_accel"] == len(e) + 5000
    assert abs(r2["charge"] - r["charge"]) <= 0.002 * r["charge"]     # binning shifts a few
    assert abs(r2["e_peak"] - r["e_peak"]) < 3 * bin_w
