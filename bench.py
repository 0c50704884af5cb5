"""Benchmark of the batched acceptance-walk nested sampler on GB300.

A step is one batch of the sampler over one event: deletion of the k lowest live points,
evidence update, k parallel DE acceptance walks (every walk step a full GW likelihood),
insertion and walk-length retune -- every row of the hot path.  Workload: 11-parameter
aligned-spin BBH, 3 detectors, 4 s at 20-1024 Hz (4017 bins), TaylorF2, seeded coloured
Gaussian noise from the analytic PSD, Table 2 injection at network SNR 39.6, 1000 live
points, k = 500, naccept 60; mixed precision, with the plain FP64 walk timed beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank samples its own independently seeded event (weak scaling, no
collective on the data path).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2509_04336_gb300 import synth  # noqa: E402

WORKLOAD = "bbh11_3det_4s_taylorf2"
METRIC = "wall-time to logZ (|Δ|≤0.1 vs FP64 oracle); lnL evals/s vs plain FP64 walk"
UNIT = "lnL evals/s"
# The method's own work per useful (walker, active bin) -- a bin of a likelihood call the chain
# uses, not of a speculative proposal dropped after an earlier acceptance -- counted from the
# formulas with an FMA as 2 flops, whatever precision carries it:
#   TaylorF2: phase over the 8-function basis and its 2 log-type terms (25), per detector the
#   time shift and range reduction (4), the amplitude (10), per detector the complex projection
#   (6) and the compensated data-term update (12): 25 + 10 + 3 * (4 + 6 + 12) = 101 flops, and
#   one sincos per detector (2 SFU ops each: 6).
#   IMRPhenomD form (merger-ringdown bins, most of the band): 3 basis terms (6), the arctangent
#   term (~20), the amplitude shape (~12), per detector time shift (4), projection (6), data
#   term (12) and template-power update (6): 38 + 3 * 28 = 122 flops, and 6 SFU ops.
ALG_FLOPS_PER_WALKER_BIN = {synth.TAYLORF2: 101.0, synth.PHENOMD_FORM: 122.0}
ALG_SFU_PER_WALKER_BIN = 6.0
# FP32 flops the float-float walk executes per evaluated (walker, bin), speculative proposals
# included (the float-float emulation of the phase and sincospi's polynomial counted):
#   TaylorF2: phase over 8 basis terms as float-float (14 each), reduction (2), per detector the
#   exact time-shift reduction (9), sincospi (20), complex multiply-accumulate (6), two Kahan
#   updates (8): 114 + 3 * 43 = 243.  IMRPhenomD form: 3 basis terms (42), arctangent (~20),
#   reduction (2), amplitude shape (~12), per detector 43 + template power (6): 76 + 3 * 49 = 223.
EXEC_FP32_FLOPS_PER_WALKER_BIN = {synth.TAYLORF2: 199.0, synth.PHENOMD_FORM: 179.0}
# Plain FP64 walk: the same formula count carried in FP64 (its FP64 sincos not counted).
FP64_ALG_FLOPS_PER_WALKER_BIN = {synth.TAYLORF2: 101.0, synth.PHENOMD_FORM: 122.0}
FP32_PEAK_TFLOPS = 80.5      # GB300 FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 1.259     # GB300 FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz
# DRAM bytes (read + write) of one walk launch, from one ncu capture of the current kernel
# (walk_kernel_ff<3, WF>, batch 10 of the 4 s TaylorF2 workload and batch 3 of the 8 s
# IMRPhenomD one); None for workloads without a capture of the current kernel.
NCU_WALK_TRAFFIC_BYTES = {"bbh11_3det_4s_taylorf2": 239360 + 0, "bbh11_3det_8s_phenomd": 1354240 + 156672}
# Workloads measured beside the headline in the default run (their own roofline, baseline, e2e).
EXTRA_WORKLOADS = ("bbh11_3det_8s_phenomd", "batched64")


def rank_info():
    from paper_2509_04336_gb300 import shard
    return shard.rank_info()


# ---------------------------------------------------------------- event synthesis
def library_event(w: synth.Workload, seed_offset: int, device: int):
    """Event with its injection made by the library's own waveform (ns_waveform)."""
    from dataclasses import replace

    from paper_2509_04336_gb300 import gwns

    w = replace(w, seed=w.seed + seed_offset)
    f = synth.frequencies(w.f_min, w.df, w.n_bins)
    psd = synth.analytic_psd(f)
    dets = []
    for name in w.detectors:
        v, x, y = synth.detector_vectors(name)
        dets.append(synth.Detector(name, v, x, y, psd.copy(), np.zeros(w.n_bins, np.complex128)))
    ev = synth.Event(w.f_min, w.df, w.n_bins, dets, synth.GMST_RAD, w.injection.copy())
    tmp = replace(w, n_live=8, num_delete=4)
    cfg = gwns.make_config(tmp, synth.priors_with_injection(tmp, ev), precision=synth.PREC_FP64)
    h = gwns.ns_init([cfg], [ev], device)
    try:
        def strain(theta):
            hr = np.zeros((1, len(dets), w.n_bins))
            hi = np.zeros_like(hr)
            gwns.ns_waveform(h, 0, np.ascontiguousarray(theta[None, :]), hr, hi)
            return hr[0] + 1j * hi[0]
        theta = w.injection.copy()
        hs = strain(theta)
        snr = math.sqrt(sum(4 * w.df * np.sum(np.abs(hs[i]) ** 2 / psd) for i in range(len(dets))))
        theta[4] *= snr / w.snr
        hs = strain(theta)
    finally:
        gwns.ns_free(h)
    for i, d in enumerate(dets):
        d.data = hs[i] + (synth.gaussian_noise(psd, w.df, w.seed, 0, i) if w.noise else 0.0)
    ev.theta_inj = theta
    return w, ev


def build_events(name: str, rank: int, device: int):
    """Workloads and library-made events of a named bench workload."""
    from paper_2509_04336_gb300 import shard
    if name == "batched64":
        ws = shard.rank_population(64, rank)
        out = [library_event(w, 0, device) for w in ws]
        return [w for w, _ in out], [e for _, e in out]
    w, ev = library_event(synth.workload(name), shard.single_event_seed_offset(rank), device)
    return [w], [ev]


WORKLOAD_DESCRIPTIONS = {
    "four_param_2det_taylorf2": "four_param_2det_taylorf2: 2 detectors, 1969 bins (4 s, 20-512 Hz), TaylorF2, 4 params "
                                "(Mc, q, chi1, chi2), n_live 100, num_delete 50, naccept 20, SNR 20, zero noise",
    "bbh11_3det_4s_taylorf2": "bbh11_3det_4s_taylorf2: 3 detectors, 4017 bins (4 s, 20-1024 Hz), TaylorF2, 11 params, "
                              "n_live 1000, num_delete 500, naccept 60, SNR 39.6, seeded noise",
    "bbh11_3det_8s_phenomd": "bbh11_3det_8s_phenomd: 3 detectors, 16,225 bins (8 s, 20-2048 Hz), IMRPhenomD form, "
                             "11 params, n_live 2000, num_delete 1000, naccept 60, SNR 30, seeded noise",
    "batched64": "batched64: 64 events in one handle, IMRPhenomD form, 3 detectors, 4/8/16 s "
                 "(4017/16,225/32,449 bins), Mc U[10,60], SNR U[12,40], n_live U{500..2000}, num_delete n_live/2",
    "bbh11_3det_8s_phenomd_flow": "bbh11_3det_8s_phenomd_flow: 3 detectors, 16,225 bins (8 s, 20-2048 Hz), "
                                  "IMRPhenomD form, 11 params, n_live 4000, num_delete 2000, naccept 60, SNR 30, "
                                  "seeded noise; DE + flow proposals (8 coupling layers, hidden 128, bf16 tensor "
                                  "cores), flow retrained on the survivors every batch (50 Adam steps, lr 3e-3)",
}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- oracle timing
def oracle_walk_rate(w: synth.Workload, ev: synth.Event, budget_s: float, walkers: int = 4, steps: int = 8,
                     max_rounds: int | None = None, round0: int = 0):
    """lnL evals/s of the oracle's acceptance walk on this workload (single thread).  Rounds
    round0, round0 + 1, ... are the walk's iteration counters, so processes given different
    round0 walk different chains."""
    from oracle import likelihood as L, prior as P, walk

    pri = synth.priors_with_injection(w, ev)
    ll = lambda u: L.log_likelihood(ev, P.transform(u, pri), w.waveform, w.use_ratio)
    surv = synth.uniform_unit_cube(64, w.n_dim, 99)
    lnl_s = np.array([ll(x) for x in surv])
    star = float(np.quantile(lnl_s, 0.5))
    idx = np.where(lnl_s > star)[0][:walkers]
    n_like, t0, rounds = 0, time.perf_counter(), 0
    while True:
        _, _, _, nl, _ = walk.acceptance_walk(ll, surv[idx], lnl_s[idx], star, surv, steps,
                                              P.periodic_mask(pri), (w.seed, 0), round0 + rounds)
        n_like += int(nl.sum())
        rounds += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_rounds is not None and rounds >= max_rounds):
            break
    return n_like / el, {"evals": n_like, "seconds": el, "rounds": rounds,
                         "sample": f"{walkers} walkers x {steps} DE steps per round, {rounds} rounds, "
                                   f"{w.n_bins} bins x {len(w.detectors)} detectors"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(procs: int):
    """A process pool for the oracle, started with spawn (never forked from a process that
    holds a CUDA context)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(procs)


def oracle_walk_rate_all_cores(w: synth.Workload, ev: synth.Event, budget_s: float, pool=None, procs=None):
    """lnL evals/s of the oracle's acceptance walk on every host core: one process per core,
    each walking its own chains (different Philox iteration counters) for budget_s seconds;
    rate = all processes' likelihood calls / the longest process time."""
    procs = procs or host_cores()
    own = pool is None
    pool = oracle_pool(procs) if own else pool
    try:
        res = pool.starmap(oracle_walk_rate, [(w, ev, budget_s, 4, 8, None, 1000 * (i + 1)) for i in range(procs)])
    finally:
        if own:
            pool.close()
            pool.join()
    evals = sum(r[1]["evals"] for r in res)
    secs = max(r[1]["seconds"] for r in res)
    rounds = sum(r[1]["rounds"] for r in res)
    return evals / secs, {"evals": evals, "seconds": secs, "processes": procs,
                          "sample": f"{procs} processes x (4 walkers x 8 DE steps per round), {rounds} rounds "
                                    f"in all, {w.n_bins} bins x {len(w.detectors)} detectors"}


def cpu_baseline(w: synth.Workload, ev: synth.Event, seconds: float, pool, procs: int):
    """The oracle as it stands on the host: all cores (the reported value) and one core."""
    rate_all, info_all = oracle_walk_rate_all_cores(w, ev, seconds, pool, procs)
    rate_1, info_1 = oracle_walk_rate(w, ev, budget_s=max(1.0, seconds / 2))
    return {"value": rate_all, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": info_all["sample"],
            "single_core": {"value": rate_1, "unit": UNIT, "cores": 1, "sample": info_1["sample"]}}


def oracle_relbin_rate(w: synth.Workload, ev: synth.Event, edges, budget_s: float, max_evals: int | None = None):
    """ln L evals/s of the oracle's relative-binning likelihood (single thread) on prior draws,
    after its summary data (not timed) around the injection."""
    from oracle import prior as P, relbin as RB

    pri = synth.priors_with_injection(w, ev)
    sd = RB.summary_data(ev, ev.theta_inj, edges, w.waveform)
    pts = synth.uniform_unit_cube(256, w.n_dim, 98)
    n, t0 = 0, time.perf_counter()
    while True:
        RB.log_likelihood(ev, P.transform(pts[n % 256], pri), sd, w.waveform, w.use_ratio)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_evals is not None and n >= max_evals):
            break
    return n / el, {"evals": n, "seconds": el,
                    "sample": f"{n} relative-binning ln L evaluations at prior draws, {len(edges) - 1} coarse bins, "
                              f"{w.n_bins} bins x {len(w.detectors)} detectors"}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    w = synth.workload(WORKLOAD)
    from oracle import likelihood as L
    ev = synth.make_event(w, L.project, L.inner)
    procs = host_cores()
    pool = oracle_pool(procs)
    try:
        pool.starmap(oracle_walk_rate, [(w, ev, 0.0, 1, 1, 1, 0)] * procs)   # start-up, untimed
        n_total, t_total = 0, 0.0
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.starmap(oracle_walk_rate, [(w, ev, 0.0, 4, 8, 1, 1000 * (p + 1) + i) for p in range(procs)])
            el = time.perf_counter() - t0
            if i >= args.warmup:
                n_total += sum(r[1]["evals"] for r in res)
                t_total += el
    finally:
        pool.close()
        pool.join()
    value = n_total / t_total
    sample = f"per step: {procs} processes x (4 walkers x 8 DE steps of the oracle), {WORKLOAD} event"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESCRIPTIONS[WORKLOAD], "precision": "FP64 (the oracle, numpy, CPU)",
                       "step": "a bounded sample of the workload's walk on every host core", "events_per_rank": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours
def run_to_logz(gwns, w, ev, precision, device, relbin_edges=None, **cfg_kw):
    """Wall time from ns_init (host inputs) to ns_evidence of one event sampled to its stopping
    rule, with the evidence it returns and the posterior's effective sample size
    (Kish: 1 / sum w_i^2 of the normalised weights of the dead and final live points).
    relbin_edges: coarse-bin edges of the relative-binning likelihood around the injection
    (its setup, ns_relbin_set, inside the timed region)."""
    import torch
    cfg = gwns.make_config(w, synth.priors_with_injection(w, ev), precision=precision, **cfg_kw)
    keep = gwns.make_event(ev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = gwns.ns_init([cfg], [keep[0]], device)
    try:
        if relbin_edges is not None:
            gwns.ns_relbin_set(h, 0, relbin_edges, ev.theta_inj)
        done, batches, steps = False, 0, []
        while not done and batches < 4000:
            _, prog = gwns.ns_step(h, 8)
            batches += 8
            done = bool(prog[0]["done"])
            steps.append(prog[0]["n_steps"])
        lz, lz_err, _, n_like = gwns.ns_evidence(h, 0)
        seconds = time.perf_counter() - t0
        _, lw = gwns.ns_posterior(h, 0)
    finally:
        gwns.ns_free(h)
    wgt = np.exp(lw - np.max(lw))
    wgt /= wgt.sum()
    ess = float(1.0 / np.sum(wgt * wgt))
    return {"seconds": seconds, "log_z": lz, "log_z_err": lz_err, "n_like": int(n_like),
            "iterations": int(prog[0]["iterations"]), "done": done, "posterior_ess": ess,
            "lnl_evals_per_ess": int(n_like) / ess, "walk_length_every_8_batches": steps}


def flow_to_logz(gwns, w, ev, device, p_flows=(0.0, 0.5, 0.9), weights=(1.0,)):
    """The learned-proposal configuration's metrics: time to ln Z and likelihood calls per
    effective posterior sample, for the DE walk (p_flow 0) and the DE + flow walk at each
    weight of an accepted flow step in the walk-length retune (keys "p_flow" for weight 1,
    "p_flow@w" otherwise), each run from ns_init to its stopping rule in the float-float mode."""
    out = {}
    for pf in p_flows:
        for wt in (weights if pf > 0.0 else (1.0,)):
            kw = {} if pf == 0.0 else {"p_flow": pf, "flow_layers": 8, "flow_accept_weight": wt}
            key = str(pf) if wt == 1.0 else f"{pf}@w{wt:g}"
            out[key] = run_to_logz(gwns, w, ev, synth.PREC_MIXED_FF, device, **kw)
    return out


def time_to_logz(gwns, device):
    """The metric's first half: wall time to ln Z, the evidence within 0.1 of the FP64 reference.

    4-parameter configuration (2 detectors, 1969 bins, zero noise, 100 live points, seed 0):
    the oracle's own run on the same seed is stored in tests/golden/logz_oracle.json (written by
    tests/golden/make_logz_golden.py, which calls only oracle/); the library's FP64 walk
    reproduces that chain (tests/test_gpu_walk.py), the float-float mode follows it up to
    decisions within its lnL tolerance of L*.  11-parameter headline configuration: the
    reference is the library's plain FP64 walk on the same data; the oracle itself would take
    days at this size.  Events are made with the library's waveform.
    """
    out = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "logz_oracle.json")) as f:
        golden_all = json.load(f)
    golden = golden_all["four_param_2det_taylorf2"]
    w4, ev4 = library_event(synth.workload("four_param_2det_taylorf2"), 0, device)
    for tag, prec in (("fp64", synth.PREC_FP64), ("float_float", synth.PREC_MIXED_FF)):
        r = run_to_logz(gwns, w4, ev4, prec, device)
        d = abs(r["log_z"] - golden["log_z"])
        out["four_param_2det_taylorf2_" + tag] = dict(r, reference="oracle (FP64 CPU, 1 core), same seed",
                                                      reference_log_z=golden["log_z"],
                                                      reference_seconds=golden["seconds"],
                                                      abs_delta=d, within_0_1=d <= 0.1)
    w11, ev11 = library_event(synth.workload(WORKLOAD), 0, device)
    r = run_to_logz(gwns, w11, ev11, synth.PREC_MIXED_FF, device)
    ref = run_to_logz(gwns, w11, ev11, synth.PREC_FP64, device)
    d = abs(r["log_z"] - ref["log_z"])
    out[WORKLOAD + "_float_float"] = dict(r, reference="plain FP64 walk on the GPU, same seed and data",
                                          reference_log_z=ref["log_z"], reference_seconds=ref["seconds"],
                                          abs_delta=d, within_0_1=d <= 0.1)
    anchor = golden_all.get(WORKLOAD)
    if anchor is not None:
        # the oracle's own run of this configuration (all host cores, same seed)
        d64 = abs(ref["log_z"] - anchor["log_z"])
        out[WORKLOAD + "_fp64"] = dict(ref, reference="oracle (FP64 CPU), same seed", reference_log_z=anchor["log_z"],
                                       reference_seconds=anchor["seconds"],
                                       reference_processes=anchor.get("processes", 1), abs_delta=d64,
                                       within_0_1=d64 <= 0.1)
    return out


def lnl_precision(gwns, w, ev, local, n=256):
    """Worst ln L error of the mixed modes on the injection and n prior draws (the FP64 handle's
    initial live points), measured against the FP64 mode, which the likelihood parity tests hold
    within 1e-10 relative of the oracle's ln L.  Relative errors are taken against
    max(|ln L|, SNR^2 / 2), the zero-noise floor of ln L near the truth."""
    hs = {}
    try:
        for p in (synth.PREC_FP64, synth.PREC_MIXED, synth.PREC_MIXED_FF):
            hs[p] = gwns.ns_init([gwns.make_config(w, synth.priors_with_injection(w, ev), precision=p)], [ev], local)
        th, _ = gwns.ns_posterior(hs[synth.PREC_FP64], 0, cap=n)
        th = np.ascontiguousarray(np.vstack([ev.theta_inj, th]))
        lnl = {}
        for p, h in hs.items():
            lnl[p] = np.zeros(th.shape[0])
            gwns.ns_likelihood_batch(h, 0, th, lnl[p])
        ref = lnl[synth.PREC_FP64]
        scale = np.maximum(np.abs(ref), 0.5 * w.snr ** 2)
        out = {"points": int(th.shape[0]), "reference": "FP64 mode (within 1e-10 relative of the oracle)"}
        for p, key in ((synth.PREC_MIXED, "mixed_fp64_phase"), (synth.PREC_MIXED_FF, "float_float")):
            err = np.abs(lnl[p] - ref)
            out[key] = {"max_abs": float(np.max(err)), "max_rel": float(np.max(err / scale))}
        return out
    finally:
        for h in hs.values():
            gwns.ns_free(h)


def measure_workload(gwns, name, steps, warmup, rank, world, local, dist, flush, sample_clocks=True, p_flow=None,
                     with_fp64=True, cpu_seconds=10.0, pool=None, procs=1):
    """One workload's line: the float-float walk timed over `steps` sampler batches after
    `warmup` (lnL evals/s, CUDA events on the library's stream, L2 flushed between batches),
    the FP64-phase and plain FP64 walks beside it, the walk's roofline on the method's own work,
    the end-to-end figure through the public API with host buffers and the oracle baseline."""
    import torch

    def barrier():
        if dist is not None:
            dist.barrier()

    def reduce(x, op):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=op)
        return float(t.item())

    MAX = dist.ReduceOp.MAX if dist else None
    SUM = dist.ReduceOp.SUM if dist else None
    ws, evs = build_events(name, rank, local)
    w, ev = ws[0], evs[0]
    ne = len(evs)
    flow_run = name.endswith("_flow")

    def configs(precision, pf=None):
        if flow_run and pf is None:
            pf = p_flow
        kw = {} if pf is None else {"p_flow": pf, "flow_layers": 8}
        return [gwns.make_config(wi, synth.priors_with_injection(wi, ei), precision=precision, **kw)
                for wi, ei in zip(ws, evs)]

    def total(progress):
        keys = ("n_like", "n_bins", "n_spec")
        out = {k: sum(p[k] for p in progress) for k in keys}
        out.update({k: progress[0][k] for k in ("walk_ms", "kernel_launches", "spec_depth", "n_steps", "mean_accept")})
        return out

    def timed_steps(precision, clocks_on=False, pf=None):
        h = gwns.ns_init(configs(precision, pf), evs, local)
        accepted = 0.0
        try:
            for _ in range(warmup):
                gwns.ns_step(h, 1, ne)
            _, p0 = gwns.ns_step(h, 0, ne)
            p0 = total(p0)
            ms = 0.0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            clocks = ClockSampler(local) if clocks_on else None
            barrier()
            torch.cuda.synchronize()
            if clocks:
                clocks.__enter__()
            for _ in range(steps):
                flush.zero_()                      # L2 flushed between steps (outside the events)
                torch.cuda.synchronize()
                e0.record()
                _, p = gwns.ns_step(h, 1, ne)      # synchronous: returns when the batch is done
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                accepted += sum(pi["mean_accept"] * wi.num_delete for pi, wi in zip(p, ws))
            if clocks:
                clocks.__exit__()
            torch.cuda.synchronize()
            barrier()
            p1 = total(p)
            return {"ms": ms, "evals": p1["n_like"] - p0["n_like"], "bins": p1["n_bins"] - p0["n_bins"],
                    "walk_ms": p1["walk_ms"] - p0["walk_ms"], "spec": p1["n_spec"] - p0["n_spec"],
                    "launches": p1["kernel_launches"] - p0["kernel_launches"], "progress": p1,
                    "accepted": accepted, "clocks": clocks.summary() if clocks else None}
        finally:
            gwns.ns_free(h)

    def rate(r):
        t = reduce(r["ms"], MAX)
        return reduce(float(r["evals"]), SUM) / (t * 1e-3), t

    mixed = timed_steps(synth.PREC_MIXED_FF, clocks_on=sample_clocks)
    value, t_max = rate(mixed)
    sweep = mixed64 = plain = None
    if flow_run:
        # the plain FP64 walk at 4000 live points takes seconds a batch: the flow line compares
        # proposals instead, every arm in the float-float mode
        sweep = {}
        for pf in (0.0, 0.5, 0.9):
            r = mixed if pf == p_flow else timed_steps(synth.PREC_MIXED_FF, pf=pf)
            sweep[str(pf)] = {"lnl_evals_per_s": r["evals"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / steps,
                              "accepted_steps_per_s": r["accepted"] / (r["ms"] * 1e-3),
                              "accepted_per_lnl_call": r["accepted"] / max(r["evals"], 1),
                              "walk_ms_per_step": r["walk_ms"] / steps}
    elif with_fp64:
        mixed64 = timed_steps(synth.PREC_MIXED)
        plain = timed_steps(synth.PREC_FP64)

    # end to end through the public API with host buffers: init (host data upload and the
    # initial live points), K batches, evidence read back
    cfgs = configs(synth.PREC_MIXED_FF)
    keep = [gwns.make_event(e) for e in evs]
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h = gwns.ns_init(cfgs, [k[0] for k in keep], local)
    try:
        for _ in range(steps):
            gwns.ns_step(h, 1, ne)
        evid = [gwns.ns_evidence(h, e) for e in range(ne)]
        _, pe = gwns.ns_step(h, 0, ne)
    finally:
        gwns.ns_free(h)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = reduce(e0.elapsed_time(e1), MAX)
    e2e_evals = reduce(float(sum(x[3] for x in evid)), SUM)
    h2d = sum(len(e.detectors) * e.n_bins * 3 * 8 for e in evs) / steps
    d2h = (288 * ne + sum(2 * p["iterations"] * wi.num_delete * 8 + wi.n_live * 8 + 200 * 8
                          for p, wi in zip(pe, ws))) / steps
    if rank != 0:
        return None

    wf = w.waveform
    kname = f"walk_kernel_ff<{len(ev.detectors)},{wf}>"
    # roofline of the dominant kernel (the walk) on the method's own work: useful (walker,
    # active bin) pairs x the formula count, over the walk's event-timed duration
    useful = float(mixed["bins"])
    evaluated = useful * mixed["spec"] / max(mixed["evals"], 1)
    walk_s = mixed["walk_ms"] * 1e-3
    achieved = useful * ALG_FLOPS_PER_WALKER_BIN[wf] / walk_s / 1e12
    roof = {"bound": "alu", "pipe": "fp32", "kernel": kname + " (float-float phase)",
            "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
            "traffic": NCU_WALK_TRAFFIC_BYTES.get(name), "avg_launch_ms": mixed["walk_ms"] / steps,
            "counted": f"{ALG_FLOPS_PER_WALKER_BIN[wf]:.0f} flops per useful (walker, active bin) "
                       f"(speculative proposals dropped after an acceptance not counted), FMA = 2",
            "useful_walker_bins_per_launch": useful / steps,
            "sfu": {"achieved_tops": useful * ALG_SFU_PER_WALKER_BIN / walk_s / 1e12,
                    "per_walker_bin": ALG_SFU_PER_WALKER_BIN},
            "executed_fp32": {"achieved": evaluated * EXEC_FP32_FLOPS_PER_WALKER_BIN[wf] / walk_s / 1e12,
                              "frac": evaluated * EXEC_FP32_FLOPS_PER_WALKER_BIN[wf] / walk_s / 1e12
                              / FP32_PEAK_TFLOPS,
                              "counted": f"{EXEC_FP32_FLOPS_PER_WALKER_BIN[wf]:.0f} FP32 flops per evaluated "
                                         "(walker, bin), speculative proposals and the float-float emulation "
                                         "included"},
            "peak_source": "derived: GB300 FP32, 152 SMs x 128 lanes x 2 flop x 2.07 GHz (an FMA "
                           "microbenchmark measured 74.7)"}
    out = {
        "value": value, "unit": UNIT, "ms_per_step": t_max / steps, "steps": steps, "warmup": warmup,
        "config": {"workload": WORKLOAD_DESCRIPTIONS[name],
                   "precision": "mixed: FP32 sums, float-float phase, FP64 per-walker constants and lnL assembly",
                   "step": "one sampler batch (select, walk, insert)",
                   "l2": "flushed (256 MB write) between timed steps", "events_per_rank": ne},
        "p_flow": p_flow if flow_run else None, "p_flow_sweep": sweep,
        "speculative_evals_per_eval": mixed["spec"] / max(mixed["evals"], 1),
        "spec_depth": mixed["progress"]["spec_depth"],
        "mean_walk_steps": mixed["progress"]["n_steps"], "mean_accept": mixed["progress"]["mean_accept"],
        "active_bins_per_eval": mixed["bins"] / max(mixed["evals"], 1),
        "e2e": {"value": e2e_evals / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": steps, "log_z": evid[0][0], "log_z_err": evid[0][1]},
        "gpu_launches": int(mixed["launches"]),
        "roofline": roof,
        "clocks": mixed["clocks"],
    }
    if plain is not None:
        vp, tp = rate(plain)
        vm, tm = rate(mixed64)
        ach64 = plain["bins"] * FP64_ALG_FLOPS_PER_WALKER_BIN[wf] / (plain["walk_ms"] * 1e-3) / 1e12
        out["plain_fp64"] = {"value": vp, "unit": UNIT, "ms_per_step": tp / steps,
                             "roofline": {"bound": "alu", "pipe": "fp64", "kernel": f"walk_kernel<0,{len(ev.detectors)},{wf}>",
                                          "achieved": ach64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                          "frac": ach64 / FP64_PEAK_TFLOPS,
                                          "avg_launch_ms": plain["walk_ms"] / steps,
                                          "counted": f"{FP64_ALG_FLOPS_PER_WALKER_BIN[wf]:.0f} FP64 flops per useful "
                                                     "(walker, active bin), FP64 sincos not counted",
                                          "peak_source": "derived: GB300 FP64, 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz"},
                             "spec_depth": plain["progress"]["spec_depth"]}
        out["mixed_fp64_phase"] = {"value": vm, "unit": UNIT, "ms_per_step": tm / steps}
        out["mixed_over_plain"] = value / vp
    out["lnl_err_vs_fp64"] = lnl_precision(gwns, w, ev, local)
    if pool is not None:
        out["cpu_baseline"] = cpu_baseline(w, ev, cpu_seconds, pool, procs)
    return out


def run_ours(args):
    import torch

    from paper_2509_04336_gb300 import build, gwns

    rank, world, local = rank_info()
    dist = None
    procs = host_cores()
    # the oracle's process pool starts (spawn) before any CUDA work of this process
    pool = oracle_pool(procs) if rank == 0 else None
    try:
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        torch.cuda.set_device(local)
        if rank == 0:
            build.build()
        if dist is not None:
            dist.barrier()
        gwns.load()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        head = measure_workload(gwns, args.workload, args.steps, args.warmup, rank, world, local, dist, flush,
                                p_flow=args.p_flow, cpu_seconds=args.cpu_seconds, pool=pool, procs=procs)
        extra = {}
        if args.workload == WORKLOAD and not args.headline_only:
            # the other configurations' lines, on fewer batches (the plain FP64 walk takes seconds
            # a batch there)
            xs, xw = max(3, min(args.steps, 5)), 3
            for name in EXTRA_WORKLOADS:
                # the 64-event population's plain FP64 walk takes ~35 s a batch: its FP64 arms are
                # left to --workload batched64
                extra[name] = measure_workload(gwns, name, xs, xw, rank, world, local, dist, flush,
                                               sample_clocks=False, cpu_seconds=args.cpu_seconds / 2,
                                               pool=pool, procs=procs, with_fp64=name != "batched64")
        if rank != 0:
            return 0
        to_logz = time_to_logz(gwns, local) if args.workload == WORKLOAD else None
        if args.workload.endswith("_flow") and args.to_logz:
            ws, evs = build_events(args.workload, 0, local)
            to_logz = flow_to_logz(gwns, ws[0], evs[0], local,
                                   weights=tuple(float(x) for x in args.flow_weights.split(",")))
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    clocks = head.pop("clocks") or {}
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic"}
    for k in ("config", "plain_fp64", "mixed_fp64_phase", "mixed_over_plain", "p_flow", "p_flow_sweep",
              "speculative_evals_per_eval", "spec_depth", "mean_walk_steps", "mean_accept", "active_bins_per_eval",
              "e2e", "gpu_launches", "roofline", "lnl_err_vs_fp64", "cpu_baseline"):
        if k in head:
            line[k] = head[k]
    line["clocks"] = {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                      "reasons": clocks.get("reasons", [])}
    line["time_to_logz"] = to_logz
    for name, x in extra.items():
        x.pop("clocks", None)
        line[name] = x
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_logz_seeds(args):
    """The metric's ln Z condition over many seeds: the headline configuration run to its
    stopping rule in the float-float mode and with the plain FP64 walk on N independent noise
    realisations and sampler seeds; the mean and standard error of ln Z(float-float) - ln Z(FP64)."""
    import torch

    from paper_2509_04336_gb300 import build, gwns

    rank, world, local = rank_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    build.build()
    gwns.load()
    from dataclasses import replace
    runs = []
    for sd in range(args.logz_seeds):
        w, ev = library_event(synth.workload(args.workload), sd, local)
        w = replace(w, seed=synth.workload(args.workload).seed + sd)
        ff = run_to_logz(gwns, w, ev, synth.PREC_MIXED_FF, local)
        fp = run_to_logz(gwns, w, ev, synth.PREC_FP64, local)
        runs.append({"seed_offset": sd, "log_z_ff": ff["log_z"], "log_z_fp64": fp["log_z"],
                     "log_z_err_fp64": fp["log_z_err"], "delta": ff["log_z"] - fp["log_z"],
                     "seconds_ff": ff["seconds"], "seconds_fp64": fp["seconds"],
                     "n_like_ff": ff["n_like"], "n_like_fp64": fp["n_like"]})
        print(json.dumps(runs[-1]), file=sys.stderr, flush=True)
    d = np.array([r["delta"] for r in runs])
    line = {"metric": "ln Z(float-float) - ln Z(plain FP64 walk), each run to its stopping rule",
            "workload": WORKLOAD_DESCRIPTIONS[args.workload], "seeds": len(runs),
            "mean_delta": float(d.mean()), "std_delta": float(d.std(ddof=1)) if d.size > 1 else None,
            "stderr_mean_delta": float(d.std(ddof=1) / math.sqrt(d.size)) if d.size > 1 else None,
            "mean_abs_delta": float(np.abs(d).mean()),
            "mean_log_z_err": float(np.mean([r["log_z_err_fp64"] for r in runs])),
            "mean_seconds_ff": float(np.mean([r["seconds_ff"] for r in runs])),
            "mean_seconds_fp64": float(np.mean([r["seconds_fp64"] for r in runs])), "runs": runs}
    print(json.dumps(line))
    return 0


def run_hrss(args):
    """HRSS line: the sampler with hit-and-run slice sampling as its inner kernel against the DE
    walk on --workload, both in the float-float mode: lnL evals/s over K batches after W warm-up
    batches (L2 flushed between them), then each run from ns_init to its stopping rule (wall time
    to ln Z, likelihood calls per effective posterior sample)."""
    import torch

    from paper_2509_04336_gb300 import build, gwns

    rank, world, local = rank_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    build.build()
    gwns.load()
    w, ev = library_event(synth.workload(args.workload), 0, local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    arms = {}
    kinds = (("de", {}), ("hrss", {"hrss_moves": args.hrss_moves}))
    with ClockSampler(local) as clocks:
        for tag, kw in kinds:
            h = gwns.ns_init([gwns.make_config(w, synth.priors_with_injection(w, ev), precision=synth.PREC_MIXED_FF,
                                               **kw)], [ev], local)
            try:
                for _ in range(args.warmup):
                    gwns.ns_step(h, 1)
                _, p0 = gwns.ns_step(h, 0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ms = 0.0
                for _ in range(args.steps):
                    flush.zero_()
                    torch.cuda.synchronize()
                    e0.record()
                    _, p = gwns.ns_step(h, 1)
                    e1.record()
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                evals = p[0]["n_like"] - p0[0]["n_like"]
                arms[tag] = {"lnl_evals_per_s": evals / (ms * 1e-3), "ms_per_step": ms / args.steps,
                             "walk_ms_per_step": (p[0]["walk_ms"] - p0[0]["walk_ms"]) / args.steps,
                             "steps_per_walker": p[0]["n_steps"], "mean_accept": p[0]["mean_accept"],
                             "lnl_calls_per_walker_batch": evals / args.steps / w.num_delete}
            finally:
                gwns.ns_free(h)
    for tag, kw in kinds:
        arms[tag]["to_logz"] = run_to_logz(gwns, w, ev, synth.PREC_MIXED_FF, local, **kw)
    ck = clocks.summary()
    de, hr = arms["de"]["to_logz"], arms["hrss"]["to_logz"]
    line = {
        "metric": "HRSS inner kernel: wall time to ln Z and lnL calls per effective sample against the DE walk",
        "value": hr["seconds"], "unit": "s to ln Z", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCRIPTIONS[args.workload], "precision": "float-float phase (mode 2)",
                   "hrss_moves": args.hrss_moves or 2 * w.n_dim, "l2": "flushed (256 MB write) between timed steps"},
        "de": arms["de"], "hrss": arms["hrss"],
        "time_to_logz_ratio_hrss_over_de": hr["seconds"] / de["seconds"],
        "lnl_calls_per_ess_ratio_hrss_over_de": hr["lnl_evals_per_ess"] / de["lnl_evals_per_ess"],
        "delta_log_z": hr["log_z"] - de["log_z"],
        "combined_log_z_err": math.hypot(hr["log_z_err"], de["log_z_err"]),
        "clocks": {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons", [])},
    }
    print(json.dumps(line))
    return 0


def run_logz_convergence(args):
    """ln Z of the headline configuration against the inner kernel's decorrelation: the DE walk
    with naccept and maxmcmc scaled up, and HRSS with more moves a batch, each on N seeds (noise
    realisation and sampler seed), float-float mode; mean ln Z and its standard error per arm, and
    every run's ln Z minus the same seed's reference arm (DE, naccept 60, maxmcmc 5000)."""
    import torch

    from dataclasses import replace

    from paper_2509_04336_gb300 import build, gwns

    rank, world, local = rank_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    build.build()
    gwns.load()
    base = synth.workload(args.workload)
    arms = [("de_60_5000", {}, {}), ("de_120_20000", {"naccept": 120, "maxmcmc": 20000}, {}),
            ("de_240_50000", {"naccept": 240, "maxmcmc": 50000}, {}),
            ("hrss_22", {}, {"hrss_moves": 22}), ("hrss_66", {}, {"hrss_moves": 66}),
            ("hrss_198", {}, {"hrss_moves": 198})]
    if args.workload.endswith("_flow"):
        # the learned proposal at the default walk settings against longer DE walks and HRSS
        arms = [("de_60_5000", {}, {}), ("de_240_50000", {"naccept": 240, "maxmcmc": 50000}, {}),
                ("flow_0.5", {}, {"p_flow": 0.5, "flow_layers": 8}),
                ("flow_0.9", {}, {"p_flow": 0.9, "flow_layers": 8}), ("hrss_198", {}, {"hrss_moves": 198})]
        # and at each weight of an accepted flow step in the walk-length retune (--flow-weights)
        for wt in (float(x) for x in args.flow_weights.split(",")):
            if wt != 1.0:
                arms += [(f"flow_{pf}_w{wt:g}", {}, {"p_flow": pf, "flow_layers": 8, "flow_accept_weight": wt})
                         for pf in (0.5, 0.9)]
    out = {a[0]: [] for a in arms}
    for sd in range(args.logz_seeds):
        w0, ev = library_event(base, sd, local)
        w0 = replace(w0, seed=base.seed + sd)
        edges = gwns.ns_relbin_edges(ev.f_min, ev.df, ev.n_bins, args.relbin) if args.relbin > 0.0 else None
        for tag, wk, ck in arms:
            r = run_to_logz(gwns, replace(w0, **wk), ev, synth.PREC_MIXED_FF, local, relbin_edges=edges, **ck)
            out[tag].append(r)
            print(json.dumps({"seed": sd, "arm": tag, "log_z": r["log_z"], "log_z_err": r["log_z_err"],
                              "seconds": r["seconds"], "n_like": r["n_like"], "iterations": r["iterations"],
                              "walk_length_every_8_batches": r["walk_length_every_8_batches"]}),
                  file=sys.stderr, flush=True)
    ref = np.array([r["log_z"] for r in out["de_60_5000"]])
    summary = {}
    for tag, _, _ in arms:
        lz = np.array([r["log_z"] for r in out[tag]])
        d = lz - ref
        n = lz.size
        summary[tag] = {"mean_log_z": float(lz.mean()), "mean_delta_vs_de_60_5000": float(d.mean()),
                        "stderr_delta": float(d.std(ddof=1) / math.sqrt(n)) if n > 1 else None,
                        "mean_log_z_err": float(np.mean([r["log_z_err"] for r in out[tag]])),
                        "mean_seconds": float(np.mean([r["seconds"] for r in out[tag]])),
                        "mean_n_like": float(np.mean([r["n_like"] for r in out[tag]])),
                        "mean_lnl_evals_per_ess": float(np.mean([r["lnl_evals_per_ess"] for r in out[tag]]))}
    print(json.dumps({"metric": "ln Z against the inner kernel's decorrelation (float-float mode)",
                      "workload": WORKLOAD_DESCRIPTIONS[args.workload], "seeds": args.logz_seeds,
                      "relbin_eps_rad": args.relbin or None, "arms": summary}))
    return 0


def run_batched_logz(args):
    """The batched form's wall time to ln Z against the plain FP64 walk at the same accuracy: the
    first N events of the 64-event population (n_live reduced to --batched-n-live, num_delete
    half of it, maxmcmc to --batched-maxmcmc, in every arm, so that the plain FP64 arm ends in
    minutes), each sampled to its stopping rule
    (1) all in one handle, float-float mode, (2) one handle at a time, float-float mode, and
    (3) all in one handle with the plain FP64 walk; every event's ln Z in (1) against (3), over
    the two runs' errors."""
    import torch

    from dataclasses import replace

    from paper_2509_04336_gb300 import build, gwns

    rank, world, local = rank_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    build.build()
    gwns.load()
    n, nl, mm = args.batched_logz, args.batched_n_live, args.batched_maxmcmc
    ws, evs = build_events("batched64", 0, local)
    ws = [replace(w, n_live=nl, num_delete=nl // 2, maxmcmc=mm) for w in ws[:n]]
    evs = evs[:n]

    def one_handle(precision):
        cfgs = [gwns.make_config(w, synth.priors_with_injection(w, ev), precision=precision)
                for w, ev in zip(ws, evs)]
        keep = [gwns.make_event(ev) for ev in evs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = gwns.ns_init(cfgs, [k[0] for k in keep], local)
        try:
            done, batches = False, 0
            while not done and batches < 4000:
                _, prog = gwns.ns_step(h, 8, n)
                batches += 8
                done = all(p["done"] for p in prog)
            out = [gwns.ns_evidence(h, e) for e in range(n)]
            seconds = time.perf_counter() - t0
        finally:
            gwns.ns_free(h)
        return {"seconds": seconds, "log_z": [o[0] for o in out], "log_z_err": [o[1] for o in out],
                "n_like": int(sum(o[3] for o in out)), "iterations": [int(p["iterations"]) for p in prog]}

    batched = one_handle(synth.PREC_MIXED_FF)
    seq = [run_to_logz(gwns, w, ev, synth.PREC_MIXED_FF, local) for w, ev in zip(ws, evs)]
    plain = one_handle(synth.PREC_FP64)
    d = np.array(batched["log_z"]) - np.array(plain["log_z"])
    sd = np.hypot(np.array(batched["log_z_err"]), np.array(plain["log_z_err"]))
    print(json.dumps({
        "metric": "wall time to ln Z of N events: batched float-float, one at a time, batched plain FP64",
        "workload": f"the first {n} events of batched64 ({WORKLOAD_DESCRIPTIONS['batched64']}), n_live {nl}, "
                    f"num_delete {nl // 2}, maxmcmc {mm} (every arm)",
        "bins": [int(ev.n_bins) for ev in evs],
        "batched_float_float": batched,
        "one_at_a_time_float_float": {"seconds": sum(r["seconds"] for r in seq), "log_z": [r["log_z"] for r in seq],
                                      "n_like": int(sum(r["n_like"] for r in seq))},
        "batched_plain_fp64": plain,
        "speedup_batched_ff_over_plain_fp64": plain["seconds"] / batched["seconds"],
        "speedup_batched_ff_over_one_at_a_time": sum(r["seconds"] for r in seq) / batched["seconds"],
        "delta_log_z_ff_minus_fp64": d.tolist(), "delta_over_error": (d / sd).tolist(),
        "mean_delta": float(d.mean()), "stderr_mean_delta": float(d.std(ddof=1) / math.sqrt(n)) if n > 1 else None}))
    return 0


def run_profile_case(args):
    """A small case for profilers: N batches of the bench workload, no timing."""
    from paper_2509_04336_gb300 import build, gwns
    import torch
    build.build()
    gwns.load()
    torch.cuda.set_device(0)
    ws, evs = build_events(args.workload, 0, 0)
    kw = {"p_flow": args.p_flow, "flow_layers": 8} if args.workload.endswith("_flow") else {}
    if args.hrss:
        kw["hrss_moves"] = args.hrss_moves
    cfgs = [gwns.make_config(w, synth.priors_with_injection(w, e), precision=args.precision, **kw)
            for w, e in zip(ws, evs)]
    h = gwns.ns_init(cfgs, evs)
    try:
        if args.relbin > 0.0:
            for e, ev in enumerate(evs):
                gwns.ns_relbin_set(h, e, gwns.ns_relbin_edges(ev.f_min, ev.df, ev.n_bins, args.relbin), ev.theta_inj)
        for _ in range(args.profile_batches):
            _, p = gwns.ns_step(h, 1, len(evs))
        print(json.dumps(p[0]))
    finally:
        gwns.ns_free(h)
    return 0


def run_relbin(args):
    """Relative-binning line: the float-float walk on the full likelihood and on the
    relative-binning likelihood (coarse bins of eps radians), each timed over K sampler
    batches after W warm-up batches (lnL evals/s, L2 flushed between batches), then each run
    from ns_init to its stopping rule (wall time to ln Z and the evidence)."""
    import torch

    from paper_2509_04336_gb300 import build, gwns

    rank, world, local = rank_info()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    build.build()
    gwns.load()
    w, ev = library_event(synth.workload(args.workload), 0, local)
    edges = gwns.ns_relbin_edges(ev.f_min, ev.df, ev.n_bins, args.relbin)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    arms = {}
    with ClockSampler(local) as clocks:
        for tag, ed in (("full", None), ("relbin", edges)):
            h = gwns.ns_init([gwns.make_config(w, synth.priors_with_injection(w, ev),
                                               precision=synth.PREC_MIXED_FF)], [ev], local)
            try:
                if ed is not None:
                    gwns.ns_relbin_set(h, 0, ed, ev.theta_inj)
                for _ in range(args.warmup):
                    gwns.ns_step(h, 1)
                _, p0 = gwns.ns_step(h, 0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ms = 0.0
                for _ in range(args.steps):
                    flush.zero_()
                    torch.cuda.synchronize()
                    e0.record()
                    _, p = gwns.ns_step(h, 1)
                    e1.record()
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                evals = p[0]["n_like"] - p0[0]["n_like"]
                arms[tag] = {"lnl_evals_per_s": evals / (ms * 1e-3), "ms_per_step": ms / args.steps,
                             "_bins": p[0]["n_bins"] - p0[0]["n_bins"], "_spec": p[0]["n_spec"] - p0[0]["n_spec"],
                             "_evals": evals, "_walk_ms": p[0]["walk_ms"] - p0[0]["walk_ms"],
                             "walk_ms_per_step": (p[0]["walk_ms"] - p0[0]["walk_ms"]) / args.steps,
                             "spec_depth": p[0]["spec_depth"], "mean_walk_steps": p[0]["n_steps"],
                             # grid bins an evaluation touched: active bins (full), or edges plus
                             # the exact range (relative binning)
                             "bins_per_eval": (p[0]["n_bins"] - p0[0]["n_bins"]) / max(evals, 1)}
            finally:
                gwns.ns_free(h)
    for tag, ed in (("full", None), ("relbin", edges)):
        arms[tag]["to_logz"] = run_to_logz(gwns, w, ev, synth.PREC_MIXED_FF, local, relbin_edges=ed)
    ck = clocks.summary()
    # roofline of the walk on the relative-binning path: the per-bin FP32 count of the waveform
    # for every grid bin an evaluation touched (edges and exact range), speculative ones included
    rb = arms["relbin"]
    flops_bin = ALG_FLOPS_PER_WALKER_BIN[w.waveform]
    touched = rb["_bins"]
    achieved = touched * flops_bin / (rb["_walk_ms"] * 1e-3) / 1e12
    for a in arms.values():
        for key in ("_bins", "_spec", "_evals", "_walk_ms"):
            a.pop(key)
    cpu_rate, cpu_info = oracle_relbin_rate(w, ev, edges, args.cpu_seconds)
    line = {
        "metric": "relative-binning likelihood: lnL evals/s and wall time to ln Z against the full likelihood",
        "value": arms["relbin"]["lnl_evals_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": arms["relbin"]["ms_per_step"], "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCRIPTIONS[args.workload], "relbin_eps_rad": args.relbin,
                   "coarse_bins": int(len(edges) - 1), "fiducial": "the injection",
                   "precision": "float-float phase (mode 2)", "l2": "flushed (256 MB write) between timed steps"},
        "full": arms["full"], "relbin": arms["relbin"],
        "speedup_evals": arms["relbin"]["lnl_evals_per_s"] / arms["full"]["lnl_evals_per_s"],
        "speedup_to_logz": arms["full"]["to_logz"]["seconds"] / arms["relbin"]["to_logz"]["seconds"],
        "abs_delta_log_z": abs(arms["full"]["to_logz"]["log_z"] - arms["relbin"]["to_logz"]["log_z"]),
        "roofline": {"bound": "alu", "pipe": "fp32",
                     "kernel": f"walk_kernel_ff<3,{w.waveform}> (relative-binning path)",
                     "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "counted": f"{flops_bin:.0f} flops (the full path's per-bin formula count) for every grid "
                                "bin a used evaluation touched (edges, exact range); speculative proposals and the "
                                "per-proposal constants are not counted"},
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cpu_info["sample"]},
        "clocks": {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons", [])},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="seconds of oracle work per process behind each cpu_baseline")
    ap.add_argument("--headline-only", action="store_true",
                    help="measure only the headline workload (no 8 s and 64-event lines)")
    ap.add_argument("--profile-batches", type=int, default=0,
                    help="run this many batches of the workload without timing (a small case for ncu)")
    ap.add_argument("--precision", type=int, default=synth.PREC_MIXED_FF)
    ap.add_argument("--p-flow", type=float, default=0.5, help="flow-step probability of the *_flow workloads")
    ap.add_argument("--to-logz", action="store_true",
                    help="*_flow workloads: also run p_flow 0, 0.5, 0.9 to their stopping rule (minutes)")
    ap.add_argument("--flow-weights", default="1",
                    help="--to-logz and --logz-convergence on *_flow workloads: comma-separated weights of "
                         "an accepted flow step in the walk-length retune; the flow arms run at each")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_DESCRIPTIONS),
                    help="bench workload (the default is the headline line)")
    ap.add_argument("--relbin", type=float, default=0.0,
                    help="eps [rad] > 0: the relative-binning line (full vs relative-binning likelihood) "
                         "on --workload instead of the headline line")
    ap.add_argument("--hrss", action="store_true",
                    help="the HRSS line (slice-sampling inner kernel against the DE walk) on --workload instead")
    ap.add_argument("--hrss-moves", type=int, default=0, help="HRSS moves per walker and batch (0: 2 D)")
    ap.add_argument("--logz-convergence", action="store_true",
                    help="with --logz-seeds N: ln Z of DE walks with longer walks and of HRSS with more moves")
    ap.add_argument("--batched-logz", type=int, default=0,
                    help="N > 0: wall time to ln Z of the first N events of batched64, batched and one at a "
                         "time in float-float and batched in plain FP64, instead")
    ap.add_argument("--batched-n-live", type=int, default=250, help="--batched-logz: live points per event")
    ap.add_argument("--batched-maxmcmc", type=int, default=5000, help="--batched-logz: walk-length cap")
    ap.add_argument("--logz-seeds", type=int, default=0,
                    help="N > 0: run --workload to ln Z in float-float and plain FP64 on N seeds instead")
    args = ap.parse_args()
    if args.profile_batches > 0:
        return run_profile_case(args)
    if args.logz_seeds > 0:
        return run_logz_convergence(args) if args.logz_convergence else run_logz_seeds(args)
    if args.batched_logz > 0:
        return run_batched_logz(args)
    if args.hrss:
        if args.workload == "batched64" or args.workload.endswith("_flow"):
            ap.error("--hrss runs a single-event DE workload")
        return run_hrss(args)
    if args.relbin > 0.0:
        if args.workload == "batched64":
            ap.error("--relbin runs a single-event workload")
        if args.warmup < 3:
            ap.error("--warmup must be >= 3")
        return run_relbin(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
