"""Ensembles of the paper's Cahn-Hilliard campaign (Secs. 4.1-4.3, Tables 3-5) on the GPU.

M runs of one domain size L at gamma = 0.01, dt = 0.0012, dx = 2 pi / 256, stepped to
t = 100 with beta sampled every 10 steps into the series rings; then, on the device, the
moments across the runs per sample time, the window mean of mu_1 over [20, 100] (the
paper's beta_0 estimate) and over the later windows [40, 100], [60, 100], [80, 100], k of
the least-squares line mu_2 = k t on [20, 100], and the per-run time averages of beta.

Starts: "asymmetric" (Sec. 4.1-4.2, Table 4): C = 0.5 + 0.1 (r - 1), r uniform on [0, 1)
per point, drawn on the host; "symmetric" (Sec. 4.3, Table 5): a mixture of mean zero,
C = 0.1 (2u - 1) from the library's own counter-based start with C0 = 0.

    python -m paper_1911_03386_gb300.campaign --L 2pi --M 1024 --precision fp32 --start asymmetric
"""
import argparse
import json
import math
import time

import numpy as np

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl

L_NAMES = {"2pi": 2 * math.pi, "4pi": 4 * math.pi, "8pi": 8 * math.pi, "16pi": 16 * math.pi}


LATE_WINDOWS = [(40.0, 100.0), (60.0, 100.0), (80.0, 100.0)]


def run(L, M, precision, preset=wl.CAMPAIGN, seed=wl.BASE_SEED, T=None, stream=None, start="asymmetric"):
    """Run one ensemble; returns a dict of throughput and statistics."""
    if start not in ("asymmetric", "symmetric"):
        raise ValueError("start must be 'asymmetric' or 'symmetric'")
    T = preset["T"] if T is None else T
    n = int(round(L / preset["dx"]))
    steps = int(round(T / preset["dt"]))
    every = preset["every"]
    t1, t2 = preset["window"]
    c0 = 0.45 if start == "asymmetric" else 0.0
    descs = [dict(nx=n, ny=n, L=L, gamma=preset["gamma"], dt=preset["dt"], C0=c0, seed=seed,
                  counter_base=k * n * n) for k in range(M)]
    with ch.Ensemble.batch(descs, precision) as e:
        if stream is not None:
            e.set_stream(stream)
        if start == "asymmetric":
            for k in range(M):
                e.set_field(k, wl.asymmetric_field(n, seed, k))
        e.set_sampling(every, t1, steps // every + 1)
        e.synchronize()
        t0 = time.perf_counter()
        e.step(steps)
        e.synchronize()
        wall = time.perf_counter() - t0
        mom = e.moments()
        b0, k, nw, nf = e.trend(t1, t2, t1, t2)
        late = {"%g-%g" % w: e.trend(w[0], w[1], t1, t2)[0] for w in LATE_WINDOWS if w[1] <= T}
        avg, cnt = e.beta_avg()
        tuning = e.tuning()
    fin = np.isfinite(avg)
    return {"L": L, "n": n, "M": M, "start": start, "precision": "fp64" if precision == ch.CH_FP64 else "fp32",
            "steps": steps, "beta0_window_mean_mu1_late": late,
            "t_end": steps * preset["dt"], "run_s": wall, "grid_point_steps_per_s": M * n * n * steps / wall,
            "s": preset["gamma"] * preset["dt"] / (L / n) ** 4, "samples": int(mom.shape[0]),
            "beta0_window_mean_mu1": b0, "k_fit_mu2": k, "window": [t1, t2], "window_samples": nw,
            "runs_counted_last_sample": int(mom[-1, 1]) if mom.shape[0] else 0,
            "mu1_last": float(mom[-1, 2]) if mom.shape[0] else None,
            "mu2_last": float(mom[-1, 3]) if mom.shape[0] else None,
            "beta_avg_mean": float(np.mean(avg[fin])) if fin.any() else None,
            "beta_avg_se": float(np.std(avg[fin], ddof=1) / math.sqrt(fin.sum())) if fin.sum() > 1 else None,
            "runs_finite": int(fin.sum()), "tuning": tuning}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", default="2pi", choices=sorted(L_NAMES))
    ap.add_argument("--M", type=int, default=wl.CAMPAIGN["M"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--T", type=float, default=wl.CAMPAIGN["T"])
    ap.add_argument("--start", default="asymmetric", choices=["asymmetric", "symmetric"])
    args = ap.parse_args()
    prec = ch.CH_FP64 if args.precision == "fp64" else ch.CH_FP32
    out = run(L_NAMES[args.L], args.M, prec, T=args.T, start=args.start)
    table = wl.CAMPAIGN["table4" if args.start == "asymmetric" else "table5"]
    if args.L in table:
        out["paper_table"] = dict(zip(["beta0", "k"], table[args.L]))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
