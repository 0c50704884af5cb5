"""The host-side pieces of bench.py that run without a GPU: the oracle timings behind the
cpu_baseline fields and the clock summary parser."""
import os
import sys


sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

from _util import event  # noqa: E402


def test_oracle_walk_rate_counts_calls():
    w, ev = event("four_param_2det_taylorf2", f_max=64.0)
    rate, info = bench.oracle_walk_rate(w, ev, budget_s=60.0, walkers=2, steps=3, max_rounds=1)
    assert info["rounds"] == 1 and 0 < info["evals"] <= 2 * 3
    assert rate > 0 and abs(rate - info["evals"] / info["seconds"]) < 1e-9 * rate


def test_oracle_relbin_rate_counts_evaluations():
    from oracle import relbin
    w, ev = event("four_param_2det_taylorf2", f_max=64.0)
    edges = relbin.default_edges(ev.f_min, ev.df, ev.n_bins, 0.25)
    rate, info = bench.oracle_relbin_rate(w, ev, edges, budget_s=60.0, max_evals=3)
    assert info["evals"] == 3 and rate > 0
    assert f"{len(edges) - 1} coarse bins" in info["sample"]


def test_clock_summary_reads_the_sampled_reasons(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    with open(c.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)
