#!/usr/bin/env python3
"""Throughput benchmark of brute-force dedispersion on GB300.

One step = one forward dedispersion of the survey-scale workload (1 beam,
1024 channels over 1420-1720 MHz, 50 us sampling, 2048 trial DMs 0-511.75,
20000 output samples, FP32 input, unit weights, 10 injected pulses) through
the C ABI's dd_execute. Prints ONE JSON line (rank 0).

  value     DM-trial*samples/s over the whole job (beams are independent:
            every rank dedisperses its own beam, weak scaling)
  e2e       the same metric through dd_execute_host: pinned host input ->
            device -> kernel -> host output, every step
  roofline  the forward kernel's algorithmic adds (B*D*S*C) per second
            against the FP32 ALU peak: with ~150 adds per compulsory HBM byte
            the brute-force method is bound by arithmetic, not HBM; the HBM
            fraction is reported beside it
  extras    8-bit / FP16 batched forms of the uneven-beam workload against
            plain FP32 launches of the same workload (default and per-plan
            tuned), the survey workload in 16-bit and 8-bit input, the
            64-channel workload and its 8/16-bit forms as graph-replayed
            microsecond launches (L2-resident) beside the FP64 oracle, the
            96-beam and HBM-bound FP32 points, and the differentiable
            workload's forward, adjoint and forward+backward

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the paper publishes no code to run).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DM-trial·samples/s"
# Sources that define the timed forward kernel; the DRAM traffic recorded in
# profiles/ is only reported while they are unchanged.
KERNEL_SOURCES = ["paper_1601_05052_gb300/csrc/dd_fwd_tile.cuh",
                  "paper_1601_05052_gb300/csrc/dd_fwd.cu",
                  "paper_1601_05052_gb300/csrc/dd_ptx.cuh",
                  "paper_1601_05052_gb300/csrc/dd_plan.cpp",
                  "paper_1601_05052_gb300/csrc/dd_kinds.h"]
TRAFFIC_PROFILE = "profiles/fwd_survey_f32.md"
UNIT = "DM-trial·samples/s"
WORKLOAD = "apertif_survey"
L2_FLUSH_BYTES = 256 << 20


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["uneven_u8", "uneven_f16", "uneven_f32", "f32_96beams",
                                       "f32_hbm_bound", "survey_precisions", "differentiable",
                                       "small_graph", "lofar"],
                    help="run one secondary workload alone (for profiling its kernels)")
    ap.add_argument("--no-tune", action="store_true",
                    help="with --only: keep the plans' starting variants (the built-in default, "
                         "or the DD_TUNE_CACHE entry an earlier tuned run recorded)")
    ap.add_argument("--variant", default=None,
                    help="with --only uneven_*/f32_96beams: JSON forward variant to use instead "
                         "of tuning (e.g. one a tuned run printed)")
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16", "u8"], default=None,
                    help="with --only survey_precisions: that input type alone")
    ap.add_argument("--launch-order", choices=["dm", "time"], default=None,
                    help="with --only lofar: the tiles' launch order (default: the tuned one)")
    ap.add_argument("--n-out", type=int, default=None,
                    help="with --only lofar: output samples (default: the full 200000)")
    ap.add_argument("--tune-ms", type=int, default=0,
                    help="auto-tune the forward variant for this budget first (0 = no)")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _recorded(variant, text=None):
    """The committed ncu summary of the forward kernel (or `text`), or None
    if the kernel sources or the variant changed since it was captured."""
    if text is None:
        try:
            text = open(os.path.join(ROOT, TRAFFIC_PROFILE)).read()
        except OSError:
            return None
    m_hash = re.search(r"kernel source hash: ([0-9a-f]{16})", text)
    m_var = re.search(r"variant: (\{[^}]*\})", text)
    if not (m_hash and m_var) or m_hash.group(1) != kernel_hash():
        return None
    if json.loads(m_var.group(1)) != variant:
        return None
    return text


def recorded_traffic(variant, text=None):
    """DRAM bytes per launch of the forward kernel from the committed ncu
    summary (or `text`), or None if the kernel sources or the variant changed
    since."""
    text = _recorded(variant, text)
    if text is None:
        return None
    m_rd = re.search(r"dram__bytes_read\.sum: ([0-9.]+) MB", text)
    m_wr = re.search(r"dram__bytes_write\.sum: ([0-9.]+) MB", text)
    if not (m_rd and m_wr):
        return None
    return (float(m_rd.group(1)) + float(m_wr.group(1))) * 1e6


def recorded_wavefronts(variant, text=None):
    """Shared-memory wavefronts per launch of the forward kernel from the
    committed ncu summary (or `text`), or None as for recorded_traffic."""
    text = _recorded(variant, text)
    if text is None:
        return None
    m = re.search(r"shared-memory wavefronts per launch: ([0-9]+)", text)
    return int(m.group(1)) if m else None


def _smem_roofline(variant, ms, n_sm, peaks):
    """The shared-memory pipe, which binds the survey kernel: the recorded
    wavefronts per launch (128 bytes each) over this run's launch time,
    against one wavefront per SM per clock."""
    wf = recorded_wavefronts(variant)
    peak = n_sm * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9
    if wf is None:
        return {"wavefronts": None, "peak_gbs": peak, "frac": None}
    gbs = wf * 128 / (ms * 1e-3) / 1e9
    return {"wavefronts": wf, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
            "note": "wavefronts per launch from ncu (%s); the floor at frac 1 is %.3f ms"
                    % (TRAFFIC_PROFILE, wf * 128 / peak / 1e6)}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                   "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows
                                   if r[3].replace(".", "").isdigit()) if rows else None}


# ---------------------------------------------------------------- helpers

def _setup_inputs(s, shifts, seed, dtype="f32", n_pulses=10):
    import synth
    pulses = synth.pulse_plan(s, seed, n_per_beam=n_pulses)
    return synth.make_input(s.with_(dtype=dtype), shifts, seed=seed, pulses=pulses,
                            pad_value={"u8": np.uint8(0), "bf16": np.uint16(0)}.get(dtype, 0))


def _time_steps(fn, steps, warmup, flush, torch):
    """Per-step CUDA-event times (ms) of fn() on the current stream, with the
    L2 flushed (a 256 MB write) before every step, outside the events; flush
    None: no flush (only for inputs larger than L2)."""
    for _ in range(warmup):
        if flush is not None:
            flush.zero_()
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for e0, e1 in ev:
        if flush is not None:
            flush.zero_()
        e0.record()
        fn()
        e1.record()
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def _cpu_baseline(x, w, shifts, s, target_s=12.0):
    """The FP64 oracle on the first n trial DMs (all channels, all samples),
    n doubled until one run takes >= target_s or covers every trial."""
    import oracle
    n = 4
    while True:
        t0 = time.perf_counter()
        oracle.forward(x, w, shifts[:n], s.n_out)
        dt = time.perf_counter() - t0
        if dt >= target_s or n >= s.n_dm:
            break
        n = min(s.n_dm, n * 2 if dt < target_s / 4 else max(n + 1, int(n * target_s / dt)))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * s.n_out * s.batch / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle (C, OpenMP over outputs) on trial DMs [0, %d) of %d, all %d "
                      "channels and %d samples, one beam: %.1f s" % (n, s.n_dm, s.n_chan,
                                                                   s.n_out, dt)}


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import synth
    s = synth.setup(WORKLOAD)
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    x = _setup_inputs(s, sh, seed=2)
    w = np.ones(s.n_chan, np.float32)
    budget = 150.0 / max(1, args.steps + args.warmup)  # seconds per step
    n = 1
    while n < s.n_dm:
        t0 = time.perf_counter()
        oracle.forward(x, w, sh[:n], s.n_out)
        if time.perf_counter() - t0 > budget / 2:
            break
        n *= 2
    for _ in range(args.warmup):
        oracle.forward(x, w, sh[:n], s.n_out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forward(x, w, sh[:n], s.n_out)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    v = n * s.n_out / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "survey scale, 1 beam x 1024 ch x 2048 DM x 20000 samples "
                                   "(sampled: trial DMs [0, %d))" % n},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "FP64 oracle on trial DMs [0, %d) of %d per step" % (n, s.n_dm)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def _rand_input(torch, g, p, seed, dtype):
    g.manual_seed(seed)
    xf = torch.randn(p.in_shape, generator=g, device="cuda", dtype=torch.float32)
    if dtype == "u8":
        return (128.0 + 16.0 * xf).round_().clamp_(0, 255).to(torch.uint8)
    return xf.to({"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype])


def _case_uneven(torch, flush, n_rep, dtypes=("u8", "f16", "f32"), tune=True, variant=None):
    """Uneven-beam batch: 96 x (64 ch) + 32 x (256 ch, low frequency); 8-bit
    and FP16 as one graph-captured persistent launch (batch-tuned), FP32 as
    plain launches, once in each plan's default variant and once with each
    plan tuned on its own (the like-for-like comparison: tuned against
    tuned)."""
    import synth
    from paper_1601_05052_gb300 import Batch, Plan
    g = torch.Generator(device="cuda")
    hi, lo = synth.setup("lband64_x96_u8"), synth.setup("lowfreq256_u8")
    units = hi.batch * hi.n_dm * hi.n_out + lo.batch * lo.n_dm * lo.n_out
    res, used = {}, {}
    for dtype in dtypes:
        plans = [Plan.from_setup(s, dtype=dtype) for s in (hi, lo)]
        xs = [_rand_input(torch, g, p, 40 + i, dtype) for i, p in enumerate(plans)]
        ws = [torch.ones(p.n_chan, dtype=p.w_dtype, device="cuda") for p in plans]
        outs = [torch.empty(p.out_shape, dtype=p.out_dtype, device="cuda") for p in plans]
        if dtype == "f32":  # the plain form: one dd_execute launch per setup
            fn = lambda: [p.execute(x, w, o) for p, x, w, o in zip(plans, xs, ws, outs)]
            used["f32_default"] = [p.variant for p in plans]
            res["f32_default"] = units / (statistics.median(
                _time_steps(fn, n_rep, 2, flush, torch)) * 1e-3)
            if not tune:
                res[dtype] = res["f32_default"]
                used[dtype] = used["f32_default"]
                continue
            for p in plans:
                p.tune(budget_ms=8000)
            used[dtype] = [p.variant for p in plans]
        else:
            bt = Batch(plans)
            if variant:
                bt.variant = variant
            elif tune:
                bt.tune(budget_ms=15000)
            fn = lambda bt=bt: bt.execute(xs, ws, outs)
            used[dtype] = bt.plan_variants
        t = statistics.median(_time_steps(fn, n_rep, 2, flush, torch))
        res[dtype] = units / (t * 1e-3)
        del xs, outs
        torch.cuda.empty_cache()
    out = {"workload": "96 beams x (64 ch, 64 DM, 4096 samples) + 32 beams x (256 ch 120-180 "
                       "MHz, 2000 DM, 10000 samples)", "unit": UNIT, "variants": used}
    for dtype in dtypes:
        out["plain_f32_tuned_launches" if dtype == "f32" else "batched_%s_graph" % dtype] = \
            res[dtype]
    if "f32" in res:
        out["plain_f32_default_launches"] = res["f32_default"]
        for dtype in dtypes:
            if dtype != "f32":
                out["speedup_%s_vs_f32" % dtype] = res[dtype] / res["f32"]
                out["speedup_%s_vs_f32_default" % dtype] = res[dtype] / res["f32_default"]
    return out


def _case_small_graph(torch, n_rep, per_graph=200, tune=True):
    """The 64-channel, 64-trial, 4096-sample workload in FP32 (unit weights)
    and its 8-bit / FP16 / BF16 forms (weights U(0.5, 1.5), 5 % masked, Q8
    integers for 8-bit input): a microsecond-scale launch, so `per_graph`
    launches are captured in one CUDA graph and each step replays it. The
    1.1 MB input and 1 MB output stay in L2 across launches (L2-resident, no
    flush). Beside it, the FP64 oracle on the same input."""
    import oracle
    import synth
    from paper_1601_05052_gb300 import Plan
    out = {"workload": "64 ch (1400-1500 MHz, 64 us) x 64 DM (0-31.5) x 4096 samples, 1 beam",
           "unit": UNIT, "launches_per_graph": per_graph,
           "l2": "L2-resident (input and output stay in L2 across the replayed launches)"}
    for dtype in ("f32", "u8", "f16", "bf16"):
        s = synth.setup("lband64" if dtype == "f32" else "lband64_" + dtype)
        sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
        pulses = synth.pulse_plan(s, 1, fixed=(40, 1000, 5.0))
        x = synth.make_input(s, sh, seed=1 if dtype == "f32" else 3, pulses=pulses,
                             pad_value={"u8": np.uint8(0), "bf16": np.uint16(0)}.get(dtype, 0))
        w = synth.make_weights(s.n_chan, 3, "ones" if dtype == "f32" else "uniform")
        if dtype == "u8":
            w = synth.quantize_weights_q8(w)
        p = Plan.from_setup(s)
        if tune:
            p.tune(budget_ms=3000)
        xt = torch.from_numpy(x)
        if dtype == "bf16":
            xt = xt.view(torch.bfloat16)
        xd = xt.cuda()
        wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
        od = torch.empty(p.out_shape, dtype=p.out_dtype, device="cuda")
        p.execute(xd, wd, od)  # first launch outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(per_graph):
                p.execute(xd, wd, od)
        t = statistics.median(_time_steps(graph.replay, n_rep, 3, None, torch)) / per_graph
        t0 = time.perf_counter()
        if dtype == "u8":
            oracle.forward_u8(x, w, sh, s.n_out)
        else:
            oracle.forward(x, w, sh, s.n_out, dtype=dtype)
        t_or = time.perf_counter() - t0
        units = s.batch * s.n_dm * s.n_out
        out[dtype] = {"value": units / (t * 1e-3), "us_per_launch": t * 1e3,
                      "variant": p.variant, "oracle_ms": t_or * 1e3,
                      "oracle_value": units / t_or}
        del graph
    return out


def _case_96beams(torch, flush, n_rep, peaks, tune=True, variant=None, name="lband64_x96"):
    """A 64-channel setup over many beams in FP32: the benchmark's 96-beam
    point (where HBM could bind), or the 4-trial, 384-beam point where it
    does."""
    import synth
    from paper_1601_05052_gb300 import Plan
    g = torch.Generator(device="cuda")
    s = synth.setup(name)
    p = Plan.from_setup(s)
    if variant:
        p.variant = variant
    elif tune:
        p.tune(budget_ms=8000)
    x = _rand_input(torch, g, p, 7, "f32")
    w = torch.ones(p.n_chan, device="cuda")
    o = torch.empty(p.out_shape, device="cuda")
    # Inputs larger than the flush buffer (twice L2) need no flush; the flush
    # write would leave L2 full of dirty lines that the timed kernel then
    # writes back, charging it traffic that is not its own.
    big = x.numel() * 4 > L2_FLUSH_BYTES
    t = statistics.median(_time_steps(lambda: p.execute(x, w, o), n_rep, 2,
                                      None if big else flush, torch))
    comp = (x.numel() * 4 + o.numel() * 4) / (t * 1e-3) / 1e9
    return {"value": s.batch * s.n_dm * s.n_out / (t * 1e-3), "unit": UNIT, "ms": t,
            "variant": p.variant, "effective_hbm_gbs": comp, "hbm_frac": comp / peaks["hbm_gbs"],
            "l2": "input larger than L2, no flush" if big else "flushed before every step"}


def _case_differentiable(torch, flush, n_rep, tune=True):
    """16 beams x 512 ch x 1024 DM x 8192: forward, adjoint alone (grad_in and
    grad_w of a full cotangent) and forward + backward of a windowed loss."""
    import synth
    from paper_1601_05052_gb300 import Plan, dedisperse
    g = torch.Generator(device="cuda")
    s = synth.setup("diff16_512ch")
    p = Plan.from_setup(s)
    rep_adj = None
    if tune:
        p.tune(budget_ms=8000)
        rep_adj = p.tune_adjoint(budget_ms=8000)
    x = _rand_input(torch, g, p, 9, "f32").requires_grad_(True)
    w = torch.ones(p.n_chan, device="cuda", requires_grad=True)
    gout = torch.randn(p.out_shape, generator=g, device="cuda")

    def fwd_bwd():
        y = dedisperse(p, x, w)
        (y[:, 256:768, 2048:6144] ** 2).sum().backward()

    tf = statistics.median(_time_steps(lambda: p.execute(x.detach(), w.detach()), n_rep, 2, flush,
                                       torch))
    ta = statistics.median(_time_steps(lambda: p.adjoint(gout, w.detach(), x.detach()), n_rep, 2,
                                       flush, torch))
    tb = statistics.median(_time_steps(fwd_bwd, n_rep, 2, flush, torch))
    units = s.batch * s.n_dm * s.n_out
    return {"forward": units / (tf * 1e-3), "forward_backward": units / (tb * 1e-3), "unit": UNIT,
            "forward_ms": tf, "adjoint_ms": ta, "forward_backward_ms": tb,
            "variant": p.variant, "adjoint_variant": rep_adj["best"] if rep_adj else None}


def _case_survey_precisions(torch, flush, n_rep, f32_ms=None,
                            dtypes=("f32", "f16", "bf16", "u8")):
    """The survey workload (1 beam x 1024 ch x 2048 DM x 20000) with 16-bit
    and 8-bit input against FP32, each in its default variant."""
    import synth
    from paper_1601_05052_gb300 import Plan
    g = torch.Generator(device="cuda")
    s = synth.setup(WORKLOAD)
    units = s.batch * s.n_dm * s.n_out
    out = {"workload": "survey scale, default variant per input type", "unit": UNIT}
    for dtype in dtypes:
        if dtype == "f32" and f32_ms is not None:
            out["f32"] = units / (f32_ms * 1e-3)
            continue
        p = Plan.from_setup(s, dtype=dtype)
        x = _rand_input(torch, g, p, 11, dtype)
        w = (torch.full((p.n_chan,), 256, dtype=torch.int32, device="cuda") if dtype == "u8"
             else torch.ones(p.n_chan, device="cuda"))
        o = torch.empty(p.out_shape, dtype=p.out_dtype, device="cuda")
        t = statistics.median(_time_steps(lambda: p.execute(x, w, o), n_rep, 2, flush, torch))
        out[dtype] = units / (t * 1e-3)
        out[dtype + "_variant"] = p.variant
        del x, o
        p.close()
    for dtype in dtypes:
        if dtype != "f32" and "f32" in out:
            out["speedup_%s_vs_f32" % dtype] = out[dtype] / out["f32"]
    return out


def _case_lofar(torch, n_rep, peaks, tune=True, variant=None, n_out=None, order=None):
    """The paper's LOFAR instance (Section IV): 32 channels of 0.195 MHz from
    138 MHz, 5 us sampling, 2048 trial DMs 0-511.75, 200000 samples (1 s),
    FP32, unit weights. One DM step moves the lowest channel by ~900
    samples, so a trial's input window is shared with almost no other trial
    (the paper's low-reuse regime). The 260 MB input is larger than L2: no
    flush."""
    import synth
    from paper_1601_05052_gb300 import Plan
    g = torch.Generator(device="cuda")
    s = synth.setup("lofar")
    if n_out:  # a shorter observation (smaller captures for profiling)
        s = s.with_(n_out=n_out)
    p = Plan.from_setup(s)
    if variant:
        p.variant = variant
    elif tune:
        p.tune(budget_ms=8000)
    if order:
        p.launch_order = order
    x = _rand_input(torch, g, p, 13, "f32")
    w = torch.ones(p.n_chan, device="cuda")
    o = torch.empty(p.out_shape, device="cuda")
    by_order = {}
    chosen = p.launch_order
    for order in (chosen, "time" if chosen == "dm" else "dm"):
        p.launch_order = order
        by_order[order] = statistics.median(
            _time_steps(lambda: p.execute(x, w, o), n_rep, 2, None, torch))
    p.launch_order = chosen
    t = by_order[chosen]
    adds = s.batch * s.n_dm * s.n_out * s.n_chan
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    alu_peak = n_sm * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    comp = (x.numel() * 4 + o.numel() * 4) / (t * 1e-3)
    return {"workload": "LOFAR: 32 ch (138-144.25 MHz, 5 us) x 2048 DM (0-511.75) x %d "
                        "samples, FP32" % s.n_out, "unit": UNIT,
            "value": s.batch * s.n_dm * s.n_out / (t * 1e-3), "ms": t, "variant": p.variant,
            "launch_order": chosen, "ms_by_launch_order": by_order,
            "gflops": adds / (t * 1e-3) / 1e9, "alu_frac": adds / (t * 1e-3) / alu_peak,
            "effective_hbm_gbs": comp / 1e9, "hbm_frac": comp / 1e9 / peaks["hbm_gbs"],
            "l2": "input larger than L2, no flush"}


# The HBM-bound point runs this variant (the tuner's usual pick there), so
# that its DRAM counters in profiles/fwd_hbm_bound_4dm_f32.md belong to the
# kernel it times.
HBM_BOUND_VARIANT = {"kind": 0, "dm_per_thread": 4, "samples_per_thread": 8, "warps_dm": 1,
                     "warps_time": 8, "chans_per_stage": 4, "stages": 3}


def _extras(torch, flush, peaks, steps, f32_ms=None):
    """Secondary measurement points (rank 0, one GPU)."""
    n_rep = max(3, min(20, steps // 10))
    return {"uneven_beams": _case_uneven(torch, flush, n_rep),
            "survey_precisions": _case_survey_precisions(torch, flush, n_rep, f32_ms),
            "small_graph_64ch": _case_small_graph(torch, n_rep),
            "lofar_f32": _case_lofar(torch, n_rep, peaks),
            "f32_96beams_64ch": _case_96beams(torch, flush, n_rep, peaks),
            "f32_hbm_bound_4dm_384beams": _case_96beams(torch, flush, n_rep, peaks,
                                                        variant=HBM_BOUND_VARIANT,
                                                        name="lband64_4dm_x384"),
            "differentiable_16beams": _case_differentiable(torch, flush, n_rep)}


def run_only(args):
    """One secondary workload by itself (its own timed loop, args.steps
    repetitions): a short command line for profiling that row's kernels."""
    import torch
    torch.cuda.set_device(0)
    peaks, _ = _peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    n = max(1, args.steps)
    tune = not args.no_tune
    variant = json.loads(args.variant) if args.variant else None
    if args.only.startswith("uneven_"):
        out = _case_uneven(torch, flush, n, dtypes=(args.only.split("_", 1)[1],), tune=tune,
                           variant=variant)
    elif args.only == "f32_96beams":
        out = _case_96beams(torch, flush, n, peaks, tune=tune, variant=variant)
    elif args.only == "f32_hbm_bound":
        out = _case_96beams(torch, flush, n, peaks, tune=tune,
                            variant=variant or HBM_BOUND_VARIANT,
                            name="lband64_4dm_x384")
    elif args.only == "small_graph":
        out = _case_small_graph(torch, n, tune=tune)
    elif args.only == "lofar":
        out = _case_lofar(torch, n, peaks, tune=tune, variant=variant, n_out=args.n_out,
                          order=args.launch_order)
    elif args.only == "survey_precisions":
        out = _case_survey_precisions(torch, flush, n,
                                      dtypes=(args.dtype,) if args.dtype else
                                      ("f32", "f16", "bf16", "u8"))
    else:
        out = _case_differentiable(torch, flush, n, tune=tune)
    print(json.dumps({"case": args.only, "steps": n, **out}), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    import synth
    from paper_1601_05052_gb300 import Plan
    from paper_1601_05052_gb300.shard import max_over_ranks

    peaks, peaks_kind = _peaks()
    s = synth.setup(WORKLOAD)
    plan = Plan.from_setup(s)
    tune_rep = plan.tune(budget_ms=args.tune_ms) if args.tune_ms > 0 else None
    sh = plan.shifts()
    x_host = _setup_inputs(s, sh, seed=2 + rank)
    w_host = np.ones(s.n_chan, np.float32)
    x = torch.from_numpy(x_host).cuda()
    w = torch.from_numpy(w_host).cuda()
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    uuid = getattr(props, "uuid", None)
    uuid = ("GPU-" + str(uuid)) if uuid is not None and not str(uuid).startswith("GPU-") else uuid

    step = lambda: plan.execute(x, w, out)
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(uuid)
    clk.start()
    times = _time_steps(step, args.steps, 0, flush, torch)
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    # a step lasts as long as the slowest rank's
    total_ms = max_over_ranks(float(sum(times)), device="cuda")
    ms = total_ms / args.steps
    units = s.batch * s.n_dm * s.n_out
    value = world * units / (ms * 1e-3)

    # parity spot check of what was timed (sampled against nothing but itself
    # is meaningless: the oracle parity lives in tests/; here only sanity)
    plan.check_device()

    # roofline of the forward kernel: one FP32 FMA per channel per output
    ops = s.batch * s.n_dm * s.n_out * s.n_chan
    n_sm = props.multi_processor_count
    alu_peak = n_sm * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = ops / (ms * 1e-3) / 1e12
    comp_bytes = x.numel() * 4 + out.numel() * 4
    eff_gbs = comp_bytes / (ms * 1e-3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "survey scale: 1 beam x 1024 ch (1420-1720 MHz) x 2048 trial "
                                   "DMs (0-511.75) x 20000 samples, FP32, unit weights, "
                                   "10 pulses; per rank",
                       "beams_per_rank": s.batch, "n_chan": s.n_chan, "n_dm": s.n_dm,
                       "n_out": s.n_out, "input_len": plan.input_len,
                       "l2": "flushed before every step (256 MB write outside the timed events)",
                       "variant": plan.variant},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": achieved / alu_peak,
                         "traffic": recorded_traffic(plan.variant),
                         "traffic_note": "DRAM bytes per launch (ncu, %s); compulsory %d"
                                         % (TRAFFIC_PROFILE, comp_bytes),
                         "peak_kind": "derived: %d SMs x 128 FP32 lanes x %.0f MHz (%s max clock)"
                                      % (n_sm, peaks.get("sm_max_mhz", 2070.0), peaks_kind),
                         "op": "one FP32 add/FMA per channel per output (the paper's flop)",
                         # the packed f32x2 adds the kernel issues double the lanes' rate
                         "peak_f32x2": 2 * alu_peak, "frac_f32x2": achieved / (2 * alu_peak),
                         "hbm": {"effective_gbs": eff_gbs, "peak_gbs": peaks["hbm_gbs"],
                                 "frac": eff_gbs / peaks["hbm_gbs"],
                                 "compulsory_bytes": comp_bytes},
                         "smem": _smem_roofline(plan.variant, ms, n_sm, peaks)},
            "gpu_launches": args.steps,
            "clocks": clocks,
            # Section V-B's real-time check: seconds of observation per beam
            # (S samples of t_samp) against the seconds one GPU spends on them
            "real_time": {"seconds_of_data": s.n_out * s.t_samp,
                          "seconds_to_dedisperse": ms * 1e-3 / s.batch,
                          "factor": s.n_out * s.t_samp / (ms * 1e-3 / s.batch)},
            # the paper's flop count: one add per channel per output (Section IV)
            "paper_gflops": ops / (ms * 1e-3) / 1e9}
    if tune_rep:
        line["tune"] = tune_rep

    if rank == 0:
        # end to end through the C ABI with pinned host buffers
        hx = torch.from_numpy(x_host).pin_memory()
        hw = torch.from_numpy(w_host).pin_memory()
        hout = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
        n_e2e = max(3, min(args.steps, 20))
        plan.execute_host(hx, hw, hout)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            plan.execute_host(hx, hw, hout)
        dt = (time.perf_counter() - t0) / n_e2e
        line["e2e"] = {"value": world * units / dt, "unit": UNIT,
                       "h2d_bytes_per_step": hx.numel() * 4 + hw.numel() * 4,
                       "d2h_bytes_per_step": hout.numel() * 4, "ms_per_step": dt * 1e3}
        line["paper_context"] = {"hd7970_2000dm_apertif_s": 0.106,
                                 "hd7970_dm_trial_samples_per_s": 2000 * 20000 / 0.106,
                                 "note": "AMD HD7970, OpenCL FP32, 2000 DMs (not 2048): context"}
        if world == 1 and not args.no_extras:
            line["extras"] = _extras(torch, flush, peaks, args.steps, f32_ms=ms)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline(x_host, w_host, sh.astype(np.int64), s)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
