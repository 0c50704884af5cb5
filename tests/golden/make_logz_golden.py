"""Writes tests/golden/logz_oracle.json: the oracle's evidence for the small workloads that the
GPU sampler tests compare against statistically (too slow to recompute inside the tests).

Calls only oracle/ and the seeded input generators:  python tests/golden/make_logz_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from oracle import likelihood as L, nested, prior as P  # noqa: E402
from _util import event, priors  # noqa: E402

WORKLOADS = ("four_param_2det_taylorf2",)


def main():
    out = {}
    for name in WORKLOADS:
        w, ev = event(name)
        pri = priors(w, ev)
        ll = lambda x: L.log_likelihood(ev, P.transform(x, pri), w.waveform, w.use_ratio)
        t0 = time.time()
        r = nested.run_nested(ll, w.n_dim, w.n_live, w.num_delete, w.naccept, w.maxmcmc, P.periodic_mask(pri),
                              (w.seed, 0), max_iter=400)
        out[name] = {"log_z": r.log_z, "log_z_err": r.log_z_err, "info_h": r.info_h, "n_iter": r.n_iter,
                     "n_like": r.n_like, "seconds": round(time.time() - t0, 1),
                     "source": "oracle.nested.run_nested, DE walk, seed (w.seed, 0), max_iter 400"}
    with open(os.path.join(HERE, "logz_oracle.json"), "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
