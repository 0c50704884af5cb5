"""Frequency-domain Gaussian-noise likelihood (Sec. 3.3, "standard frequency-domain
likelihood" over frequency bins and detectors, no heterodyning).

  <a|b> = 4 df Re sum_k conj(a_k) b_k / S_n(f_k)
  ln L(theta) = -1/2 sum_det <d - h_det(theta) | d - h_det(theta)>      (no normalisation)
  use_ratio:  ln Lambda = ln L + 1/2 sum_det <d|d>  (the likelihood ratio against noise)
  h_det(f) = (F+ h+(f) + Fx hx(f)) exp(-2 pi i f dt_det)
Sums run over every bin in FP64 (numpy's pairwise summation).
"""
import numpy as np

from paper_2509_04336_gb300.synth import TAYLORF2, PHENOMD_FORM, frequencies

from . import detector, taylorf2


def polarizations(waveform: int, f, theta, table=None, cutoff: bool = True):
    if waveform == TAYLORF2:
        return taylorf2.polarizations(f, theta, cutoff)
    if waveform == PHENOMD_FORM:
        from . import phenomd
        return phenomd.polarizations(f, theta, table, cutoff)
    raise ValueError(waveform)


def inner(a, b, psd, df) -> float:
    return float(4.0 * df * np.sum((np.conj(a) * b).real / psd))


def project(event, det_index: int, theta, waveform: int = TAYLORF2, table=None, f=None,
            cutoff: bool = True) -> np.ndarray:
    """Strain of the waveform seen by one detector of the event (at the event's bins, or at
    the frequencies f; cutoff=False continues the template above its cutoff)."""
    d = event.detectors[det_index]
    if f is None:
        f = frequencies(event.f_min, event.df, event.n_bins)
    hp, hc = polarizations(waveform, f, theta, table, cutoff)
    ra, dec, psi = float(theta[9]), float(theta[10]), float(theta[6])
    fp, fc = detector.antenna_pattern(d.x_arm, d.y_arm, ra, dec, psi, event.gmst)
    dt = detector.time_delay(d.vertex, ra, dec, event.gmst)
    return (fp * hp + fc * hc) * np.exp(-2j * np.pi * f * dt)


def log_likelihood(event, theta, waveform: int = TAYLORF2, use_ratio: bool = False, table=None) -> float:
    total = 0.0
    for i, d in enumerate(event.detectors):
        r = d.data - project(event, i, theta, waveform, table)
        total += inner(r, r, d.psd, event.df)
        if use_ratio:
            total -= inner(d.data, d.data, d.psd, event.df)
    return -0.5 * total


def log_likelihood_batch(event, thetas, waveform: int = TAYLORF2, use_ratio: bool = False, table=None) -> np.ndarray:
    return np.array([log_likelihood(event, th, waveform, use_ratio, table) for th in np.atleast_2d(thetas)])


def network_snr(event, theta, waveform: int = TAYLORF2, table=None) -> float:
    s = 0.0
    for i, d in enumerate(event.detectors):
        h = project(event, i, theta, waveform, table)
        s += inner(h, h, d.psd, event.df)
    return float(np.sqrt(s))
