"""The paper's experiments on this GPU (Sections IV and V).

Experiment 1 (Section IV-A): for each input instance -- the number of trial
DMs, every power of two from 2 to 4096, DM_0 = 0 and step 0.25 -- time every
meaningful configuration of the kernel's parameters and keep the one with
the highest GFLOP/s (one add per channel per output sample, the paper's
flop count, Section IV: "20 MFLOP per DM" for Apertif).

Experiment 2 (Section IV-B, V-B): performance of the tuned instances, the
"signal-to-noise ratio" of each optimum (its distance from the mean GFLOP/s
of all configurations in standard deviations), Chebyshev's bound 1/k^2 on the
chance of picking a configuration that far from the mean, and the real-time
check: one second of data (S = samples per second) dedispersed in under one
second.

Experiment 3 (Section IV-C, V-C): the same with every trial DM equal to 0, so
there are no delays ("perfect data reuse").

Discussion (Section V-D): the best fixed configuration, i.e. the one that
maximises the sum of GFLOP/s over all instances, and the speedup of the tuned
optimum over it for each instance.

Here a configuration is a compiled kernel variant (kind, DMs and samples per
thread, warps along DM and time) at a fixed staging per setup: Apertif 16
channels per stage, LOFAR 4 (a LOFAR DM step moves the lowest channel by ~900
samples, so each trial of a tile stages its own window per channel, and a
chunk holds at most 32 windows; with every DM 0, 16 as for Apertif), 2
stages, with the launch order of the
setup's tiles (LOFAR: time tiles fastest, which keeps its rows in L2); the
variants that do not fit an instance are not meaningful for it. Inputs are
seeded N(0,1) noise (performance does not depend on the values).

    python -m paper_1601_05052_gb300.experiments --setup apertif [--dm0]
    python -m paper_1601_05052_gb300.experiments --setup all --markdown
"""
import argparse
import json
import statistics
import sys

import torch

from . import Plan, variants

SETUPS = {
    # Section IV: 20 000 samples/s, 1024 channels of 0.29 MHz from 1420 MHz
    "apertif": dict(n_chan=1024, f_lo=1420.0, chan_width=300.0 / 1024, t_samp=1 / 20000,
                    n_out=20000, chans_per_stage=16, order="dm"),
    # Section IV: 200 000 samples/s, 32 channels of ~0.19 MHz from 138 MHz
    "lofar": dict(n_chan=32, f_lo=138.0, chan_width=0.1953125, t_samp=1 / 200000,
                  n_out=200000, chans_per_stage=4, order="time"),
}
DDM = 0.25


def _plan(name, n_dm, dm0_only):
    s = SETUPS[name]
    freqs = [s["f_lo"] + c * s["chan_width"] for c in range(s["n_chan"])]
    dms = [0.0 if dm0_only else i * DDM for i in range(n_dm)]
    return Plan(freqs, freqs[-1], s["t_samp"], dms, s["n_out"], batch=1)


def _configs(name, dm0_only=False):
    cch = 16 if dm0_only else SETUPS[name]["chans_per_stage"]
    return [v for v in variants() if v["chans_per_stage"] == cch and v["stages"] == 2]


def _time_ms(plan, x, w, o, reps=3):
    plan.execute(x, w, o)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.execute(x, w, o)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


def run(name, dm0_only=False, instances=None, log=sys.stderr):
    instances = instances or [2 ** k for k in range(1, 13)]
    configs = _configs(name, dm0_only)
    key = lambda v: tuple(v.values())
    table = {}  # instance -> {config key: GFLOP/s}
    rows = []
    for n_dm in instances:
        plan = _plan(name, n_dm, dm0_only)
        g = torch.Generator(device="cuda")
        g.manual_seed(n_dm)
        x = torch.randn(plan.in_shape, generator=g, device="cuda")
        w = torch.ones(plan.n_chan, device="cuda")
        o = torch.empty(plan.out_shape, device="cuda")
        flop = float(plan.n_dm) * plan.n_out * plan.n_chan
        perf = {}
        for v in configs:
            try:
                plan.variant = v
            except Exception:
                continue  # not meaningful for this instance
            plan.launch_order = SETUPS[name]["order"]
            perf[key(v)] = flop / (_time_ms(plan, x, w, o) * 1e6)
        table[n_dm] = perf
        vals = list(perf.values())
        best = max(perf, key=perf.get)
        mean = statistics.fmean(vals)
        sd = statistics.stdev(vals) if len(vals) > 1 else 0.0
        snr = (perf[best] - mean) / sd if sd > 0 else 0.0
        t_best = flop / (perf[best] * 1e9)
        rows.append({"n_dm": n_dm, "configs": len(vals), "best": dict(zip(configs[0].keys(), best)),
                     "best_gflops": perf[best], "mean_gflops": mean, "std_gflops": sd,
                     "snr": snr, "chebyshev": (1.0 / snr ** 2) if snr > 1 else 1.0,
                     "seconds_per_second_of_data": t_best, "real_time": t_best < 1.0})
        if log is not None:
            print("%s%s D=%d: best %.1f GFLOP/s (%s), mean %.1f, sd %.1f, SNR %.2f"
                  % (name, " DM0" if dm0_only else "", n_dm, perf[best], best, mean, sd, snr),
                  file=log, flush=True)
        del x, o
        plan.close()
    # the best fixed configuration: meaningful everywhere, largest summed GFLOP/s
    common = set.intersection(*[set(p) for p in table.values()])
    fixed = max(common, key=lambda k: sum(table[n][k] for n in table)) if common else None
    for r in rows:
        if fixed is not None:
            f = table[r["n_dm"]][fixed]
            r["fixed_gflops"] = f
            r["speedup_tuned_over_fixed"] = r["best_gflops"] / f
    return {"setup": name, "dm0_only": dm0_only,
            "fixed": dict(zip(configs[0].keys(), fixed)) if fixed else None, "instances": rows}


def markdown(results):
    """One table row per instance from the results of run() for the four
    experiments (Apertif and LOFAR, each with real DMs and with DM = 0)."""
    by = {(r["setup"], r["dm0_only"]): {i["n_dm"]: i for i in r["instances"]} for r in results}
    ap = by.get(("apertif", False), {})
    cols = [("apertif", True), ("lofar", False), ("lofar", True)]
    lines = ["| D | Apertif best GFLOP/s | mean | SNR | Chebyshev | tuned / fixed | "
             "Apertif DM=0 best | LOFAR best | LOFAR DM=0 best |",
             "|---|---|---|---|---|---|---|---|---|"]
    ns = sorted(set().union(*[set(v) for v in by.values()])) if by else []
    for n in ns:
        a = ap.get(n)
        cells = [str(n)]
        if a:
            cells += ["%.0f" % a["best_gflops"], "%.0f" % a["mean_gflops"], "%.2f" % a["snr"],
                      "%.2f" % a["chebyshev"],
                      "%.2f" % a["speedup_tuned_over_fixed"] if "speedup_tuned_over_fixed" in a
                      else "-"]
        else:
            cells += ["-"] * 5
        for key in cols:
            i = by.get(key, {}).get(n)
            cells.append("%.0f" % i["best_gflops"] if i else "-")
        lines.append("| " + " | ".join(cells) + " |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--setup", choices=sorted(SETUPS) + ["all"], default="apertif")
    ap.add_argument("--dm0", action="store_true", help="every trial DM = 0 (Section IV-C)")
    ap.add_argument("--max-log2-dm", type=int, default=12)
    ap.add_argument("--markdown", action="store_true",
                    help="print the results as one markdown table (with --setup all)")
    a = ap.parse_args(argv)
    instances = [2 ** k for k in range(1, a.max_log2_dm + 1)]
    if a.setup == "all":
        res = [run(name, dm0, instances) for name in ("apertif", "lofar") for dm0 in (False, True)]
    else:
        res = [run(a.setup, a.dm0, instances)]
    print(json.dumps(res if len(res) > 1 else res[0]))
    if a.markdown:
        print(markdown(res))


if __name__ == "__main__":
    main()
