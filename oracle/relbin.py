"""Relative binning (heterodyned likelihood) -- the likelihood compression the paper names as
the remedy for bin saturation (Sec. 3.3, Sec. 5, Appendix C); the method is that of Zackay,
Dai & Venumadhav (2018) and Cornish's heterodyning (2010), restated here.  Test
infrastructure: the oracle of the relative-binning likelihood, plain FP64 numpy.

Around a fiducial waveform h0 (the template at theta0 continued above its cutoff, so that h0 is
smooth and non-zero over the whole band), a proposal's strain is h = h0 r with a ratio r(f) that
varies slowly.  Over coarse bins b = [e_b, e_{b+1}) of the frequency grid,
r(f) ~ r_b + r1_b (f - f_{e_b}) with r_b = r(f_{e_b}), r1_b = (r_{b+1} - r_b) / (f_{e_{b+1}} - f_{e_b}),
so with the summary data of each coarse bin and detector (w = 4 df / S_n)

  A0 = sum conj(d) h0 w,   A1 = sum conj(d) h0 w (f - f_e),
  B0 = sum |h0|^2 w,       B1 = sum |h0|^2 w (f - f_e),       B2 = sum |h0|^2 w (f - f_e)^2

the inner products are  <d|h>_b = Re(A0 r_b + A1 r1_b)  and
<h|h>_b = B0 |r_b|^2 + 2 B1 Re(conj(r_b) r1_b) + B2 |r1_b|^2.  The ratio needs the proposal's
strain only at the coarse-bin edges (~10^2 instead of ~10^4 bins).

The template's cutoff (f_ISCO for TaylorF2, Mf = 0.2 for the IMRPhenomD form) moves with the
proposal's mass and makes r discontinuous.  Coarse bins wholly below the proposal's cutoff use
the expansion (the edge values of r are taken from the continued template), except the last
coarse bin of the grid, whose right edge lies off the grid; from the first coarse bin that does
not qualify up to the cutoff, the active bins are summed exactly (that range holds the cutoff,
or it is the last coarse bin); the bins above the cutoff contribute nothing.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2509_04336_gb300.synth import frequencies

from . import likelihood as L

# Power laws of the PN phase whose largest differences set the bin widths (Zackay et al. 2018)
GAMMAS = (-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0)


def default_edges(f_min: float, df: float, n_bins: int, eps: float = 0.25) -> np.ndarray:
    """Coarse-bin edges (bin indices, ascending, first 0, last n_bins) such that the proxy for
    the largest phase difference any template can have from the fiducial,
    dpsi(f) = 2 pi sum_g sign(g) (f / f_g)^g with f_g = f_min (g < 0) or f_max (g > 0),
    changes by at most eps radians across a coarse bin (and a bin holds at least one grid bin)."""
    f = frequencies(f_min, df, n_bins)
    f_max = f[-1]
    dpsi = np.zeros(n_bins)
    for g in GAMMAS:
        dpsi += 2.0 * math.pi * math.copysign(1.0, g) * (f / (f_min if g < 0 else f_max)) ** g
    edges = [0]
    for k in range(1, n_bins):
        if abs(dpsi[k] - dpsi[edges[-1]]) > eps:
            edges.append(k)
    edges.append(n_bins)
    return np.array(edges, dtype=np.int64)


def edge_frequencies(event, edges) -> np.ndarray:
    """Frequency of each edge (the last edge, n_bins, lies one step above the grid)."""
    return event.f_min + event.df * np.asarray(edges, dtype=np.float64)


def summary_data(event, theta0, edges, waveform: int, table=None) -> dict:
    """Summary data of every coarse bin and detector around the fiducial theta0."""
    f = frequencies(event.f_min, event.df, event.n_bins)
    fe = edge_frequencies(event, edges)
    nb = len(edges) - 1
    nd = len(event.detectors)
    A0 = np.zeros((nd, nb), np.complex128)
    A1 = np.zeros((nd, nb), np.complex128)
    B0 = np.zeros((nd, nb))
    B1 = np.zeros((nd, nb))
    B2 = np.zeros((nd, nb))
    h0_edges = np.zeros((nd, nb + 1), np.complex128)
    dd = 0.0
    for i, d in enumerate(event.detectors):
        h0 = L.project(event, i, theta0, waveform, table, cutoff=False)
        h0_edges[i] = L.project(event, i, theta0, waveform, table, f=fe, cutoff=False)
        w = 4.0 * event.df / d.psd
        cd = np.conj(d.data) * h0 * w
        p0 = np.abs(h0) ** 2 * w
        for b in range(nb):
            s = slice(edges[b], edges[b + 1])
            x = f[s] - fe[b]
            A0[i, b] = np.sum(cd[s])
            A1[i, b] = np.sum(cd[s] * x)
            B0[i, b] = np.sum(p0[s])
            B1[i, b] = np.sum(p0[s] * x)
            B2[i, b] = np.sum(p0[s] * x * x)
        dd += L.inner(d.data, d.data, d.psd, event.df)
    return {"edges": np.asarray(edges), "fe": fe, "A0": A0, "A1": A1, "B0": B0, "B1": B1, "B2": B2,
            "h0_edges": h0_edges, "dd": dd, "theta0": np.array(theta0, dtype=np.float64)}


def active_bins(event, theta, waveform: int, table=None) -> int:
    """Number of grid bins below the template's cutoff (the template is zero from there on)."""
    f = frequencies(event.f_min, event.df, event.n_bins)
    hp, hc = L.polarizations(waveform, f, theta, table)
    on = (np.abs(hp) + np.abs(hc)) > 0.0
    n = int(np.sum(on))
    assert np.all(on[:n]) and not np.any(on[n:]), "the cutoff is a single frequency"
    return n


def n_expanded(edges, k_end: int, n_bins: int) -> int:
    """Number of leading coarse bins taken by the expansion: those wholly below the cutoff
    (right edge <= k_end) whose right edge is a grid bin (< n_bins)."""
    n = 0
    while n + 1 < len(edges) and edges[n + 1] <= k_end and edges[n + 1] < n_bins:
        n += 1
    return n


def log_likelihood(event, theta, sd: dict, waveform: int, use_ratio: bool = False, table=None) -> float:
    """ln L of theta from the summary data sd (the -1/2 <d - h|d - h> of the full likelihood,
    or the ratio form)."""
    edges, fe = sd["edges"], sd["fe"]
    nb = len(edges) - 1
    k_end = active_bins(event, theta, waveform, table)
    f = frequencies(event.f_min, event.df, event.n_bins)
    dh = 0.0
    hh = 0.0
    n_full = n_expanded(edges, k_end, event.n_bins)
    lo = int(edges[n_full])
    for i, d in enumerate(event.detectors):
        r = L.project(event, i, theta, waveform, table, f=fe[:n_full + 1], cutoff=False) / sd["h0_edges"][i][:n_full + 1]
        w = 4.0 * event.df / d.psd
        for b in range(n_full):
            r0 = r[b]
            r1 = (r[b + 1] - r[b]) / (fe[b + 1] - fe[b])
            dh += (sd["A0"][i, b] * r0 + sd["A1"][i, b] * r1).real
            hh += (sd["B0"][i, b] * abs(r0) ** 2 + 2.0 * sd["B1"][i, b] * (np.conj(r0) * r1).real
                   + sd["B2"][i, b] * abs(r1) ** 2)
        if lo < k_end:
            # from the first coarse bin not expanded up to the cutoff: exact over the active bins
            h = L.project(event, i, theta, waveform, table, f=f[lo:k_end])
            dh += float(np.sum((np.conj(d.data[lo:k_end]) * h).real * w[lo:k_end]))
            hh += float(np.sum(np.abs(h) ** 2 * w[lo:k_end]))
    if use_ratio:
        return dh - 0.5 * hh
    return -0.5 * (sd["dd"] - 2.0 * dh + hh)
