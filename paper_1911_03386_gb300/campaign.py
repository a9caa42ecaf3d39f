"""Ensembles of the paper's Cahn-Hilliard campaign (Sec. 4.1-4.2, Tables 3-4) on the GPU.

M runs of one domain size L at gamma = 0.01, dt = 0.0012, dx = 2 pi / 256 from the
asymmetric start C = 0.5 + 0.1 (r - 1), stepped to t = 100 with beta sampled every 10
steps into the series rings; then, on the device, the moments across the runs per sample
time, the window mean of mu_1 over [20, 100] (the paper's beta_0 estimate), k of the
least-squares line mu_2 = k t on the same window, and the per-run time averages of beta.

    python -m paper_1911_03386_gb300.campaign --L 2pi --M 1024 --precision fp32
"""
import argparse
import json
import math
import time

import numpy as np

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl

L_NAMES = {"2pi": 2 * math.pi, "4pi": 4 * math.pi, "8pi": 8 * math.pi, "16pi": 16 * math.pi}


def run(L, M, precision, preset=wl.CAMPAIGN, seed=wl.BASE_SEED, T=None, stream=None):
    """Run one ensemble; returns a dict of throughput and statistics."""
    T = preset["T"] if T is None else T
    n = int(round(L / preset["dx"]))
    steps = int(round(T / preset["dt"]))
    every = preset["every"]
    t1, t2 = preset["window"]
    descs = [dict(nx=n, ny=n, L=L, gamma=preset["gamma"], dt=preset["dt"], C0=0.45, seed=seed,
                  counter_base=k * n * n) for k in range(M)]
    with ch.Ensemble.batch(descs, precision) as e:
        if stream is not None:
            e.set_stream(stream)
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
        avg, cnt = e.beta_avg()
        tuning = e.tuning()
    fin = np.isfinite(avg)
    return {"L": L, "n": n, "M": M, "precision": "fp64" if precision == ch.CH_FP64 else "fp32", "steps": steps,
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
    args = ap.parse_args()
    prec = ch.CH_FP64 if args.precision == "fp64" else ch.CH_FP32
    out = run(L_NAMES[args.L], args.M, prec, T=args.T)
    out["paper_table4"] = dict(zip(["beta0", "k"], wl.CAMPAIGN["table4"][args.L]))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
