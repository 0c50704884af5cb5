"""Writes tests/golden/logz_oracle.json: the oracle's evidence for workloads that the GPU
sampler tests and the bench compare against (too slow to recompute inside them).

Calls only oracle/ and the seeded input generators:

    python tests/golden/make_logz_golden.py                          # the 4-parameter workload
    python tests/golden/make_logz_golden.py --workload bbh11_3det_4s_taylorf2 --procs 7

--procs spreads each batch's walks over a process pool (walker ranges; the chains are those
of the one-process run).  Entries of other workloads already in the file are kept.
"""
import argparse
import functools
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from oracle import likelihood as L, nested, prior as P  # noqa: E402
from _util import event, priors  # noqa: E402

OUT = os.path.join(HERE, "logz_oracle.json")


def _loglike(x, ev, pri, waveform, use_ratio):
    return L.log_likelihood(ev, P.transform(x, pri), waveform, use_ratio)


def run(name, procs, max_iter, n_live=None):
    w, ev = event(name, n_live=n_live)
    pri = priors(w, ev)
    ll = functools.partial(_loglike, ev=ev, pri=pri, waveform=w.waveform, use_ratio=w.use_ratio)
    t0 = time.time()

    def progress(st):
        it, n_steps, acc, calls, lstar, lz = st
        print(f"[{name}] batch {it}: n_steps {n_steps} mean_accept {acc:.2f} calls {calls} "
              f"lnL* {lstar:.4f} logZ {lz:.4f}  t={time.time() - t0:.0f}s", file=sys.stderr, flush=True)

    pool = mp.get_context("spawn").Pool(procs) if procs > 1 else None
    try:
        r = nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc, P.periodic_mask(pri),
                              (w.seed, 0), max_iter=max_iter, walk_pool=pool, walk_chunks=4 * procs,
                              progress=progress)
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    src = f"oracle.nested.run_nested, DE walk, seed (w.seed, 0), max_iter {max_iter}"
    if procs > 1:
        src += f", walks spread over {procs} processes"
    if n_live is not None:
        src += f", n_live {n_live}"
    return {"log_z": r.log_z, "log_z_err": r.log_z_err, "info_h": r.info_h, "n_iter": r.n_iter,
            "n_like": r.n_like, "seconds": round(time.time() - t0, 1), "processes": procs, "source": src}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="four_param_2det_taylorf2")
    ap.add_argument("--procs", type=int, default=1)
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--n-live", type=int, default=None)
    a = ap.parse_args()
    res = run(a.workload, a.procs, a.max_iter, a.n_live)
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    key = a.workload if a.n_live is None else f"{a.workload}@n_live={a.n_live}"
    out[key] = res
    with open(OUT, "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
