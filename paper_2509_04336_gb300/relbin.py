"""Coarse-bin edges for the relative-binning likelihood (ns_relbin_set).

The rule of Zackay, Dai & Venumadhav (2018): a coarse bin ends where the largest phase
difference any template in the prior can have from the fiducial could have changed by eps
radians.  That difference is bounded by a sum of the phase's power laws f^g (g = -5/3, -2/3, 1,
5/3, 7/3), each normalised at the end of the band where it is largest:
dpsi(f) = 2 pi sum_g sign(g) (f / f_g)^g, f_g = f_min for g < 0 and f_max for g > 0.  dpsi
increases with f, so each edge is the first grid bin past the previous edge's dpsi + eps.
"""
from __future__ import annotations

import numpy as np

_POWERS = (-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0)


def coarse_edges(f_min: float, df: float, n_bins: int, eps: float = 0.25) -> np.ndarray:
    """int32 edges [n_coarse + 1]: 0, ..., n_bins (grid-bin indices, strictly increasing)."""
    f = f_min + df * np.arange(n_bins, dtype=np.float64)
    f_top = f[-1]
    dpsi = np.zeros(n_bins)
    for g in _POWERS:
        ref = f_min if g < 0 else f_top
        dpsi += np.sign(g) * 2.0 * np.pi * (f / ref) ** g
    edges = [0]
    while True:
        k = int(np.searchsorted(dpsi, dpsi[edges[-1]] + eps, side="right"))
        if k >= n_bins:
            break
        edges.append(max(k, edges[-1] + 1))
    edges.append(n_bins)
    return np.asarray(edges, dtype=np.int32)
