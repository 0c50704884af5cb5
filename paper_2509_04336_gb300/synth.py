"""Seeded synthetic inputs for the batched acceptance-walk nested sampler.

This module is the only code shared by the CUDA path's callers (bench, smoke)
and the CPU oracle.  It holds workload descriptions and seeded random draws and
none of the method's arithmetic: no waveform, no antenna pattern, no inner
product, no prior transform.  Where a workload needs a signal (an injection, a
target SNR) the caller passes in its own waveform and inner-product functions.

Workloads follow the paper's analyses (Sec. 4.1.1 4 s signal, Table 2; Sec. 4.4
8 s signal, Table 4; Table 1 priors) with the paper's O4 noise curves replaced
by the analytic PSD below and bilby's noise by seeded Gaussian draws.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Callable, Sequence

import numpy as np

# Physical parameter order used everywhere (theta vectors are length 11).
PARAM_NAMES = (
    "chirp_mass",          # detector-frame chirp mass [Msun]
    "mass_ratio",          # q = m2/m1 <= 1
    "chi_1",               # aligned spin of the heavier body
    "chi_2",               # aligned spin of the lighter body
    "luminosity_distance", # [Mpc]
    "theta_jn",            # inclination [rad]
    "psi",                 # polarisation angle [rad]
    "phase",               # coalescence (orbital) phase [rad]
    "geocent_time",        # coalescence time at the geocentre, relative to the segment reference [s]
    "ra",                  # right ascension [rad]
    "dec",                 # declination [rad]
)
N_PARAMS = len(PARAM_NAMES)

# Prior kinds (Table 1 of the paper plus a FIXED kind for parameters held at a value).
UNIFORM, POWERLAW, SINE, COSINE, FIXED = 0, 1, 2, 3, 4
KIND_NAMES = {UNIFORM: "uniform", POWERLAW: "powerlaw", SINE: "sine", COSINE: "cosine", FIXED: "fixed"}

TAYLORF2, PHENOMD_FORM = 0, 1
PREC_FP64, PREC_MIXED, PREC_MIXED_FF = 0, 1, 2
TERM_DLOGZ, TERM_FRAC_REMAINING = 0, 1

EARTH_RADIUS_M = 6.371e6           # spherical Earth used for detector vertices
GMST_RAD = 4.3                      # fixed Greenwich sidereal angle of every synthetic event

# (latitude deg, longitude deg, x-arm azimuth deg, y-arm azimuth deg); azimuths are
# measured clockwise from local North.  Approximate LIGO-Hanford, LIGO-Livingston
# and Virgo sites, rounded; the exact values are a choice of this workload.
DETECTOR_SITES = {
    "H": (46.455, -119.408, 324.0, 234.0),
    "L": (30.563, -90.774, 252.3, 162.3),
    "V": (43.631, 10.504, 19.4, 289.4),
}


@dataclass(frozen=True)
class PriorEntry:
    kind: int
    lo: float = 0.0
    hi: float = 1.0
    alpha: float = 0.0
    periodic: bool = False
    value: float = 0.0     # used when kind == FIXED


@dataclass
class Detector:
    name: str
    vertex: np.ndarray     # [3] metres, Earth-fixed frame
    x_arm: np.ndarray      # [3] unit vector
    y_arm: np.ndarray      # [3] unit vector
    psd: np.ndarray        # [n_bins] one-sided PSD [1/Hz]
    data: np.ndarray       # [n_bins] complex strain [1/Hz]


@dataclass
class Event:
    f_min: float
    df: float
    n_bins: int
    detectors: list
    gmst: float
    theta_inj: np.ndarray  # [11] injected physical parameters


@dataclass
class Workload:
    name: str
    detectors: Sequence[str]
    f_min: float
    f_max: float
    duration: float
    waveform: int
    injection: np.ndarray          # [11] before SNR rescaling
    snr: float                     # target network optimal SNR (d_L rescaled to reach it)
    noise: bool
    priors: list                   # [11] PriorEntry
    n_live: int
    num_delete: int
    naccept: int
    maxmcmc: int
    term_kind: int
    term_value: float
    seed: int
    precision: int = PREC_MIXED
    use_ratio: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def df(self) -> float:
        return 1.0 / self.duration

    @property
    def n_bins(self) -> int:
        return n_bins_for(self.f_min, self.f_max, self.df)

    @property
    def n_dim(self) -> int:
        return sum(1 for p in self.priors if p.kind != FIXED)


def n_bins_for(f_min: float, f_max: float, df: float) -> int:
    """Number of bins of the grid f_k = f_min + k df, k = 0.., inclusive of f_max."""
    return int(math.floor((f_max - f_min) / df + 1e-9)) + 1


def frequencies(f_min: float, df: float, n_bins: int) -> np.ndarray:
    return f_min + df * np.arange(n_bins, dtype=np.float64)


def detector_vectors(name: str):
    """Vertex and arm unit vectors (Earth-fixed, metres) of a named site."""
    lat, lon, az_x, az_y = (math.radians(v) for v in DETECTOR_SITES[name])
    vertex = EARTH_RADIUS_M * np.array([math.cos(lat) * math.cos(lon),
                                        math.cos(lat) * math.sin(lon),
                                        math.sin(lat)])
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.array([-math.sin(lat) * math.cos(lon), -math.sin(lat) * math.sin(lon), math.cos(lat)])
    x_arm = math.cos(az_x) * north + math.sin(az_x) * east
    y_arm = math.cos(az_y) * north + math.sin(az_y) * east
    return vertex, x_arm, y_arm


def analytic_psd(f: np.ndarray, s0: float = 1e-49, f0: float = 215.0) -> np.ndarray:
    """S_n(f) = S0 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)], x = f/f0."""
    x = np.asarray(f, dtype=np.float64) / f0
    return s0 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))


def gaussian_noise(psd: np.ndarray, df: float, seed: int, event: int, det: int) -> np.ndarray:
    """n_k = (N(0,1) + i N(0,1)) sqrt(S_n/(4 df)), so that E<n|n> = 2 per bin."""
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 1000 * event + det], dtype=np.uint64)))
    z = rng.standard_normal((2, psd.shape[0]))
    return (z[0] + 1j * z[1]) * np.sqrt(psd / (4.0 * df))


def uniform_unit_cube(n: int, dim: int, seed: int) -> np.ndarray:
    """Seeded unit-cube points (used for random prior draws in tests and benches)."""
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 777], dtype=np.uint64)))
    return rng.random((n, dim))


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

TABLE2_INJECTION = np.array([35.0, 0.90, 0.40, -0.30, 1000.0, 0.40, 2.66, 1.30, 0.0, 1.38, -1.21])
TABLE4_INJECTION = np.array([10.0, 0.70, -0.34, 0.01, 500.0, 1.30, 1.83, 5.21, 0.0, 1.07, -1.01])


def _standard_priors(mc, q, chi) -> list:
    """Table 1 priors with signal-dependent mass/spin ranges."""
    two_pi = 2.0 * math.pi
    return [
        PriorEntry(UNIFORM, mc[0], mc[1]),
        PriorEntry(UNIFORM, q[0], q[1]),
        PriorEntry(UNIFORM, chi[0], chi[1]),
        PriorEntry(UNIFORM, chi[0], chi[1]),
        PriorEntry(POWERLAW, 100.0, 5000.0, alpha=2.0),
        PriorEntry(SINE, 0.0, math.pi),
        PriorEntry(UNIFORM, 0.0, math.pi, periodic=True),
        PriorEntry(UNIFORM, 0.0, two_pi, periodic=True),
        PriorEntry(UNIFORM, -0.1, 0.1),
        PriorEntry(UNIFORM, 0.0, two_pi, periodic=True),
        PriorEntry(COSINE, -0.5 * math.pi, 0.5 * math.pi),
    ]


def workload(name: str) -> Workload:
    """Named synthetic workloads.

    four_param_2det_taylorf2   2 detectors, 20-512 Hz at 0.25 Hz (1969 bins), zero noise,
                               Mc=28 q=0.8 chi=(0.3,-0.2) at SNR 20, 4 sampled parameters,
                               100 live points, naccept 20, plain FP64.
    bbh11_3det_4s_taylorf2     3 detectors, 20-1024 Hz (4017 bins), seeded noise, Table 2
                               injection at SNR 39.6, 11 parameters, 1000 live points.
    bbh11_3det_8s_phenomd      3 detectors, 20-2048 Hz at 0.125 Hz (16,225 bins), Table 4
                               injection at SNR 30, IMRPhenomD-form waveform, 2000 live points.
    bbh11_3det_8s_phenomd_flow the same with 4000 live points (k = 2000), for flow proposals.
    """
    if name == "four_param_2det_taylorf2":
        inj = np.array([28.0, 0.8, 0.3, -0.2, 1000.0, 0.40, 2.66, 1.30, 0.0, 1.38, -1.21])
        pri = _standard_priors((20.0, 40.0), (0.125, 1.0), (-0.99, 0.99))
        # Every parameter but (Mc, q, chi1, chi2) is held at its injected value; the
        # distance entry is overwritten with the SNR-rescaled value in make_event.
        pri = pri[:4] + [PriorEntry(FIXED, value=float(inj[i])) for i in range(4, 11)]
        return Workload(name, ("H", "L"), 20.0, 512.0, 4.0, TAYLORF2, inj, 20.0, False, pri,
                        n_live=100, num_delete=50, naccept=20, maxmcmc=5000,
                        term_kind=TERM_DLOGZ, term_value=0.1, seed=0, precision=PREC_FP64)
    if name == "bbh11_3det_4s_taylorf2":
        pri = _standard_priors((25.0, 50.0), (0.25, 1.0), (-1.0, 1.0))
        return Workload(name, ("H", "L", "V"), 20.0, 1024.0, 4.0, TAYLORF2, TABLE2_INJECTION.copy(),
                        39.6, True, pri, n_live=1000, num_delete=500, naccept=60, maxmcmc=5000,
                        term_kind=TERM_DLOGZ, term_value=0.1, seed=1, precision=PREC_MIXED)
    if name == "bbh11_3det_8s_phenomd":
        pri = _standard_priors((10.0, 25.0), (0.25, 1.0), (-0.8, 0.8))
        return Workload(name, ("H", "L", "V"), 20.0, 2048.0, 8.0, PHENOMD_FORM, TABLE4_INJECTION.copy(),
                        30.0, True, pri, n_live=2000, num_delete=1000, naccept=60, maxmcmc=5000,
                        term_kind=TERM_DLOGZ, term_value=0.1, seed=2, precision=PREC_MIXED)
    if name == "bbh11_3det_8s_phenomd_flow":
        # the 8 s workload with 4000 live points, for the flow-proposal runs
        return replace(workload("bbh11_3det_8s_phenomd"), name=name, n_live=4000, num_delete=2000)
    raise KeyError(name)


def shrink(w: Workload, *, f_max: float | None = None, n_live: int | None = None,
           num_delete: int | None = None, naccept: int | None = None) -> Workload:
    """A smaller copy of a workload (fewer bins or live points) for quick checks."""
    kw = {}
    if f_max is not None:
        kw["f_max"] = f_max
    if n_live is not None:
        kw["n_live"] = n_live
        kw["num_delete"] = num_delete if num_delete is not None else n_live // 2
    elif num_delete is not None:
        kw["num_delete"] = num_delete
    if naccept is not None:
        kw["naccept"] = naccept
    return replace(w, **kw)


def make_event(w: Workload,
               project: Callable[[Event, int, np.ndarray], np.ndarray],
               inner: Callable[[np.ndarray, np.ndarray, np.ndarray, float], float],
               event_index: int = 0,
               injection: np.ndarray | None = None,
               snr: float | None = None,
               rescale: bool = True) -> Event:
    """Build one event: seeded noise plus an injected signal rescaled to the target SNR.

    `project(event, det, theta)` returns the detector strain of the caller's waveform
    model; `inner(a, b, psd, df)` the caller's noise-weighted inner product.  The
    distance of the injection is rescaled so that the network optimal SNR equals
    the target (the strain amplitude is inversely proportional to distance); with
    rescale=False the injection keeps its distance.
    """
    f = frequencies(w.f_min, w.df, w.n_bins)
    psd = analytic_psd(f)
    dets = []
    for i, name in enumerate(w.detectors):
        vertex, x_arm, y_arm = detector_vectors(name)
        dets.append(Detector(name, vertex, x_arm, y_arm, psd.copy(), np.zeros(w.n_bins, np.complex128)))
    theta = np.array(w.injection if injection is None else injection, dtype=np.float64).copy()
    ev = Event(w.f_min, w.df, w.n_bins, dets, GMST_RAD, theta)
    target = w.snr if snr is None else snr
    snr2 = 0.0
    for i, d in enumerate(dets):
        h = project(ev, i, theta)
        snr2 += inner(h, h, d.psd, w.df)
    if rescale:
        theta[4] *= math.sqrt(snr2) / target
    ev.theta_inj = theta
    for i, d in enumerate(dets):
        h = project(ev, i, theta)
        n = gaussian_noise(d.psd, w.df, w.seed, event_index, i) if w.noise else 0.0
        d.data = h + n
    return ev


def priors_with_injection(w: Workload, ev: Event) -> list:
    """The workload priors with FIXED entries set from the (rescaled) injection."""
    out = []
    for i, p in enumerate(w.priors):
        out.append(replace(p, value=float(ev.theta_inj[i])) if p.kind == FIXED else p)
    return out


def injection_set(n: int = 96, seed: int = 500, base: str = "four_param_2det_taylorf2", n_live: int = 300,
                  naccept: int = 30, snr: float = 15.0, precision: int = PREC_MIXED_FF) -> list:
    """Seeded injection study on synthetic data (the paper's PP test, Sec. 4.2, with a new set).

    Injection e takes the base workload and redraws every sampled parameter from its own prior
    (so that the true values follow the prior the sampler uses), keeps the fixed ones, adds
    seeded noise (seed `seed` + e) and rescales the distance to network SNR `snr`.
    """
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 5555], dtype=np.uint64)))
    w0 = workload(base)
    out = []
    for e in range(n):
        inj = w0.injection.copy()
        for i, p in enumerate(w0.priors):
            if p.kind == UNIFORM:
                inj[i] = rng.uniform(p.lo, p.hi)
            elif p.kind != FIXED:
                raise ValueError("injection_set draws uniform priors only")
        out.append(replace(w0, name=f"injection_{e}", injection=inj, snr=snr, noise=True, seed=seed + e,
                           n_live=n_live, num_delete=n_live // 2, naccept=naccept, precision=precision))
    return out


def batched_workloads(n_events: int = 64, seed: int = 100, waveform: int = PHENOMD_FORM,
                      precision: int = PREC_MIXED_FF) -> list:
    """Seeded population of independent events sampled together in one launch.

    Event e: Mc ~ U[10, 60] Msun, q ~ U[0.25, 1], spins ~ U[-0.8, 0.8], the other parameters
    from the Table 1 priors; target network SNR ~ U[12, 40]; duration 4, 8 or 16 s, the
    smallest exceeding the Newtonian chirp time from 20 Hz plus 2 s, except that the first
    three quarters of the events are stratified over the three durations so that each
    appears at least n_events/4 times (20-1024 Hz at 4 s, 20-2048 Hz at 8 and 16 s: 4017,
    16,225 and 32,449 bins); n_live ~ U{500, 600, ..., 2000}, num_delete = n_live / 2;
    priors Mc +- 25 % around the injection, q [0.25, 1], spins [-0.8, 0.8]; noise seed `seed` + e.
    """
    rng = np.random.Generator(np.random.Philox(key=np.array([seed, 4444], dtype=np.uint64)))
    out = []
    tsun = 4.925490947641267e-06
    for e in range(n_events):
        mc = rng.uniform(10.0, 60.0)
        q = rng.uniform(0.25, 1.0)
        chi = rng.uniform(-0.8, 0.8, size=2)
        u = rng.random(7)
        inj = np.array([mc, q, chi[0], chi[1], 1000.0, math.acos(1 - 2 * u[0]), math.pi * u[1],
                        2 * math.pi * u[2], -0.1 + 0.2 * u[3], 2 * math.pi * u[4], math.asin(2 * u[5] - 1)])
        snr = rng.uniform(12.0, 40.0)
        # Newtonian chirp time from 20 Hz (seconds)
        tau0 = 5.0 / 256.0 * (math.pi * 20.0) ** (-8.0 / 3.0) * (mc * tsun) ** (-5.0 / 3.0)
        natural = next((d for d in (4.0, 8.0, 16.0) if d > tau0 + 2.0), 16.0)
        strata = (4.0, 8.0, 16.0)
        duration = strata[e % 3] if e < (3 * n_events) // 4 else natural
        f_max = 1024.0 if duration == 4.0 else 2048.0
        n_live = int(rng.integers(5, 21)) * 100
        pri = _standard_priors((0.75 * mc, 1.25 * mc), (0.25, 1.0), (-0.8, 0.8))
        w = Workload(f"batched_{e}", ("H", "L", "V"), 20.0, f_max, duration, waveform, inj, snr, True, pri,
                     n_live=n_live, num_delete=n_live // 2, naccept=60, maxmcmc=5000,
                     term_kind=TERM_DLOGZ, term_value=0.1, seed=seed + e, precision=precision)
        out.append(w)
    return out
