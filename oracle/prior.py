"""Unit-cube prior transforms (Sec. 3.4, Table 1; sampling in the unit hypercube, Sec. 3.1).

Each sampled parameter is an independent draw from a separable prior, mapped
from u in [0, 1] by its inverse CDF:
  uniform  on [a, b]:       x = a + u (b - a)
  power law (alpha != -1):  x = (a^(alpha+1) + u (b^(alpha+1) - a^(alpha+1)))^(1/(alpha+1))
  sine     on [a, b]:       x = arccos(cos a - u (cos a - cos b))
  cosine   on [a, b]:       x = arcsin(sin a + u (sin b - sin a))
  fixed:                    x = value (not sampled)
"""
import math

import numpy as np

from paper_2509_04336_gb300.synth import UNIFORM, POWERLAW, SINE, COSINE, FIXED


def sampled_indices(priors):
    """Physical-parameter indices of the sampled (non-fixed) dimensions, in order."""
    return [i for i, p in enumerate(priors) if p.kind != FIXED]


def periodic_mask(priors):
    return np.array([p.periodic for p in priors if p.kind != FIXED], dtype=bool)


def transform_one(u: float, p) -> float:
    if p.kind == UNIFORM:
        return p.lo + u * (p.hi - p.lo)
    if p.kind == POWERLAW:
        e = p.alpha + 1.0
        return (p.lo ** e + u * (p.hi ** e - p.lo ** e)) ** (1.0 / e)
    if p.kind == SINE:
        return math.acos(math.cos(p.lo) - u * (math.cos(p.lo) - math.cos(p.hi)))
    if p.kind == COSINE:
        return math.asin(math.sin(p.lo) + u * (math.sin(p.hi) - math.sin(p.lo)))
    raise ValueError("fixed parameters are not transformed")


def transform(u, priors) -> np.ndarray:
    """Map one unit-cube point u [D] to the physical parameter vector theta [11]."""
    theta = np.empty(len(priors), dtype=np.float64)
    d = 0
    for i, p in enumerate(priors):
        if p.kind == FIXED:
            theta[i] = p.value
        else:
            theta[i] = transform_one(float(u[d]), p)
            d += 1
    return theta


def transform_batch(U, priors) -> np.ndarray:
    U = np.atleast_2d(U)
    return np.stack([transform(u, priors) for u in U])


def log_prior_volume_density(theta, priors) -> float:
    """log pi(theta) of the separable prior (used only by checks of the transforms)."""
    lp = 0.0
    for i, p in enumerate(priors):
        x = theta[i]
        if p.kind == FIXED:
            continue
        if not (p.lo <= x <= p.hi):
            return -math.inf
        if p.kind == UNIFORM:
            lp += -math.log(p.hi - p.lo)
        elif p.kind == POWERLAW:
            e = p.alpha + 1.0
            lp += math.log(e * x ** p.alpha / (p.hi ** e - p.lo ** e))
        elif p.kind == SINE:
            lp += math.log(math.sin(x) / (math.cos(p.lo) - math.cos(p.hi)))
        elif p.kind == COSINE:
            lp += math.log(math.cos(x) / (math.sin(p.hi) - math.sin(p.lo)))
    return lp
