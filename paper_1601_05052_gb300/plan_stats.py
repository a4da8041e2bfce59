"""Host-side statistics of a delay table that decide which forward kernel
kind pays for it (plan arithmetic only; no GPU and no kernel involved).

* Shared delays: the fraction of adjacent trial pairs (d, d + 1) whose delay
  in a channel is equal. The lane-strided kind 5 reuses the loaded operands
  for such a pair.
* Delay patterns: within a DM tile of `dt` trials and a group of `group`
  adjacent channels (reference = the group's last channel), the number of
  distinct relative patterns rho(d) = (shift[d][c] - shift[d][ref])_c. The
  sub-band kinds build one partial series per pattern.
* Shared-memory words per tile of `dt` trials by `ts` samples: one word per
  channel-add for the lane-strided kind, against, for the sub-band form, one
  word per group-add in the trial loop plus, per pattern p with base delays
  in [bmin_p, bmax_p], (bmax_p - bmin_p + ts) series elements that each cost
  `group` loads and one store to build.

    python -m paper_1601_05052_gb300.plan_stats --setup apertif --dt 64 --ts 256
"""
import argparse
import json

import numpy as np

SETUPS = {
    # name: (channels, lowest frequency MHz, channel width MHz, t_samp s, DM step)
    "apertif": (1024, 1420.0, 300.0 / 1024, 50e-6, 0.25),
    "lband64": (64, 1400.0, 100.0 / 64, 64e-6, 0.5),
    "lowfreq256": (256, 120.0, 60.0 / 256, 204.8e-6, 0.05),
    "diff512": (512, 1250.0, 300.0 / 512, 100e-6, 0.25),
    "lofar": (32, 138.0, 0.1953125, 5e-6, 0.25),
}


def setup_shifts(name, n_dm):
    """The Eq. 1 delay table of a named band-edge setup (reference = top channel)."""
    from . import compute_shifts
    c, f0, df, ts, ddm = SETUPS[name]
    freqs = f0 + np.arange(c) * df
    return compute_shifts(freqs, freqs[-1], ts, np.arange(n_dm) * ddm).astype(np.int64)


def shared_adjacent_delays(shifts):
    """Fraction of adjacent trial pairs whose delay in a channel is equal."""
    sh = np.asarray(shifts)
    return float((sh[1:] == sh[:-1]).mean()) if sh.shape[0] > 1 else 0.0


def delay_patterns(shifts, dt, group=4):
    """Per (DM tile, channel group): number of distinct relative patterns and
    the sum over patterns of the base-delay spans (bmax - bmin)."""
    sh = np.asarray(shifts)
    D, C = sh.shape
    n_dt, n_g = (D + dt - 1) // dt, (C + group - 1) // group
    count = np.zeros((n_dt, n_g), np.int64)
    span = np.zeros((n_dt, n_g), np.int64)
    for k in range(n_dt):
        tile = sh[k * dt:(k + 1) * dt]
        for g in range(n_g):
            cols = tile[:, g * group:(g + 1) * group]
            base = cols[:, -1]
            rel = cols - base[:, None]
            pats = {}
            for r, b in zip(map(tuple, rel), base):
                lo, hi = pats.get(r, (b, b))
                pats[r] = (min(lo, b), max(hi, b))
            count[k, g] = len(pats)
            span[k, g] = sum(hi - lo for lo, hi in pats.values())
    return count, span


def shared_words(shifts, dt, ts, group=4):
    """Shared-memory words of one pass over all DM tiles (per time tile of ts
    samples): (lane-strided words, sub-band words, their ratio)."""
    sh = np.asarray(shifts)
    D, C = sh.shape
    count, span = delay_patterns(sh, dt, group)
    lane = float(D) * ts * C
    trials = float(D) * ts * count.shape[1]
    build = float(((span + count * ts) * (group + 1)).sum())
    return lane, trials + build, lane / (trials + build)


def report(shifts, dt, ts, group=4):
    count, _ = delay_patterns(shifts, dt, group)
    lane, sub, ratio = shared_words(shifts, dt, ts, group)
    return {"n_dm": int(np.asarray(shifts).shape[0]), "n_chan": int(np.asarray(shifts).shape[1]),
            "dm_tile": dt, "time_tile": ts, "group": group,
            "shared_adjacent_delays": shared_adjacent_delays(shifts),
            "patterns_mean": float(count.mean()), "patterns_max": int(count.max()),
            "lane_strided_words": lane, "subband_words": sub,
            "words_ratio_lane_over_subband": ratio}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--setup", default="apertif", choices=sorted(SETUPS))
    ap.add_argument("--n-dm", type=int, default=2048)
    ap.add_argument("--dt", type=int, default=64)
    ap.add_argument("--ts", type=int, default=256)
    ap.add_argument("--group", type=int, default=4)
    a = ap.parse_args(argv)
    print(json.dumps(report(setup_shifts(a.setup, a.n_dm), a.dt, a.ts, a.group)))


if __name__ == "__main__":
    main()
