"""Beam parameters of the injected electrons (the quantities of the paper's Table BeamParams,
Sec. 4), computed in FP64 with numpy from a particle set.

TEST INFRASTRUCTURE ONLY: used by the test-suite and the benchmark's reference leg; it shares
nothing with the CUDA library.

Definitions (the table's caption fixes the quantities; the reading fixes the rest):
  * electrons: alive particles with p_x > px_min (the accelerated electrons);
  * energy: E = gamma - 1 = sqrt(1 + |p|^2) - 1 (m c^2 units), weight w (charge);
  * spectrum: the w-weighted histogram of E over [0, E_max] in `nbins` equal bins, E_max the
    largest selected energy;
  * E_peak: the centre of the first bin holding the largest weight;
  * FWHM: between the half-maximum crossings on either side of the peak, each located by
    linear interpolation between the centres of the last bin at or above half the peak and the
    first bin below it (the spectrum's end counts as zero);
  * the beam: electrons with |E - E_peak| <= FWHM (2 FWHM widths around the peak);
  * Q = sum of w over the beam; dE/E = rms spread of E over the beam / E_peak;
  * eps_n in each transverse plane u (y or z): sqrt(s_uu s_pp - s_up^2) with the w-weighted
    central second moments of u and p_u over the beam (units c/w0); eps_mean = their mean.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("n_accel", "n_beam", "charge", "e_peak", "fwhm", "de_over_e", "eps_y", "eps_z",
          "eps_mean", "e_mean", "e_max", "nbins")


def spectrum(e, w, nbins):
    e_max = float(e.max())
    edges_w = e_max / nbins if e_max > 0 else 1.0
    idx = np.minimum((e / edges_w).astype(np.int64), nbins - 1)
    h = np.zeros(nbins)
    np.add.at(h, idx, w)
    return h, edges_w


def peak_and_fwhm(h, width):
    """Peak bin centre and full width at half maximum of a histogram with bins of `width`."""
    k = int(np.argmax(h))
    half = 0.5 * h[k]
    centre = lambda b: (b + 0.5) * width  # noqa: E731

    def crossing(step):
        b = k
        while 0 <= b + step < len(h) and h[b + step] >= half:
            b += step
        nxt = b + step
        hn = h[nxt] if 0 <= nxt < len(h) else 0.0
        # linear interpolation between the centres of b (>= half) and nxt (< half)
        t = (h[b] - half) / (h[b] - hn) if h[b] != hn else 0.0
        return centre(b) + step * t * width

    return centre(k), crossing(1) - crossing(-1)


def beam_parameters(px, py, pz, y, z, w, px_min=10.0, nbins=256):
    px, py, pz, y, z, w = (np.asarray(a, dtype=np.float64) for a in (px, py, pz, y, z, w))
    sel = px > px_min
    out = dict.fromkeys(FIELDS, 0.0)
    out["nbins"] = float(nbins)
    out["n_accel"] = float(sel.sum())
    if not sel.any():
        return out
    e = np.sqrt(1.0 + px[sel] ** 2 + py[sel] ** 2 + pz[sel] ** 2) - 1.0
    ws, ys, zs, pys, pzs = w[sel], y[sel], z[sel], py[sel], pz[sel]
    h, width = spectrum(e, ws, nbins)
    e_peak, fwhm = peak_and_fwhm(h, width)
    beam = np.abs(e - e_peak) <= fwhm
    q = ws[beam].sum()
    out.update(e_peak=e_peak, fwhm=fwhm, e_max=float(e.max()), n_beam=float(beam.sum()), charge=q)
    if q <= 0:
        return out
    wb = ws[beam]

    def mean(a):
        return float((wb * a).sum() / q)

    eb = e[beam]
    out["e_mean"] = mean(eb)
    out["de_over_e"] = float(np.sqrt(max(mean(eb * eb) - mean(eb) ** 2, 0.0)) / e_peak)
    eps = []
    for u, pu in ((ys[beam], pys[beam]), (zs[beam], pzs[beam])):
        suu = mean(u * u) - mean(u) ** 2
        spp = mean(pu * pu) - mean(pu) ** 2
        sup = mean(u * pu) - mean(u) * mean(pu)
        eps.append(float(np.sqrt(max(suu * spp - sup * sup, 0.0))))
    out["eps_y"], out["eps_z"] = eps
    out["eps_mean"] = 0.5 * (eps[0] + eps[1])
    return out
