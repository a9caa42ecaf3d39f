"""Model 1 ensembles of the paper (Secs. 2-3, Tables 1-2) on the GPU.

For each population size N: M = 100 populations of N droplets with radii uniform on
[0, 1), integrated to t = 40 by `ch_droplets_run` (Dormand-Prince 5(4), eps = 1e-3),
beta sampled every 0.1; then, on the device (`ch_stats_moments`, `ch_stats_trend`), the
moments of beta across the populations per sample time (Sec. 3.3 Eqs. (41a,b)), the
window mean of mu_1 over [20, 40] (Eq. (42)) and k of mu_2 = k t over [0, 40].

    python -m paper_1911_03386_gb300.droplets --N 512 1024
"""
import argparse
import json
import time

import numpy as np

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl


def run(N, preset=wl.DROPLETS, M=None, T=None, seed=wl.BASE_SEED):
    import torch

    M = preset["M"] if M is None else M
    T = preset["T"] if T is None else T
    ts = np.round(np.arange(0.0, T + 0.5 * preset["sample_dt"], preset["sample_dt"]), 12)
    R0 = wl.droplet_radii(M, N, seed)
    t0 = time.perf_counter()
    R, ser, steps = ch.ch_droplets_run(R0, T, ts, rtol=preset["rtol"], atol=preset["atol"], h0=preset["h0"],
                                       eps=preset["eps"])
    wall = time.perf_counter() - t0
    beta = torch.from_numpy(np.ascontiguousarray(ser[:, :, 3])).cuda()
    tt = torch.from_numpy(np.ascontiguousarray(ts)).cuda()
    mom = torch.empty((ts.size, ch.CH_MOMENTS), dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    ch.ch_stats_moments(tt.data_ptr(), beta.data_ptr(), M, ts.size, ts.size, mom.data_ptr())
    (w1, w2), (f1, f2) = preset["window"], preset["fit"]
    ch.ch_stats_trend(mom.data_ptr(), ts.size, w1, w2, f1, f2, out.data_ptr())
    torch.cuda.synchronize()
    tr = out.cpu().numpy()
    m = mom.cpu().numpy()
    return {"N": N, "M": M, "T": T, "wall_s": wall, "steps_accepted_mean": float(steps[:, 0].mean()),
            "steps_rejected_mean": float(steps[:, 1].mean()), "live_at_T_mean": float(ser[:, -1, 4].mean()),
            "beta0_window_mean_mu1": float(tr[0]), "window": [w1, w2], "k_fit_mu2": float(tr[1]), "fit": [f1, f2],
            "mu1_at_T": float(m[-1, 2]), "mu2_at_T": float(m[-1, 3]),
            "paper_table2": dict(zip(["beta0", "k"], preset["table2"].get(N, (None, None))))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, nargs="+", default=[512, 1024])
    ap.add_argument("--M", type=int, default=wl.DROPLETS["M"])
    ap.add_argument("--T", type=float, default=wl.DROPLETS["T"])
    args = ap.parse_args()
    for n in args.N:
        print(json.dumps(run(n, M=args.M, T=args.T)), flush=True)


if __name__ == "__main__":
    main()
