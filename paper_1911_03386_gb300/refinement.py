"""Grid-refinement study of Appendix A on the GPU path.

The same single-droplet start (`workloads.droplet_field`) is run to the final time T on
grids of n = 128, 256, ... points per axis with dt = 0.1 dx (rounded so every grid ends at
T), in FP64.  E_n, the mean L1 distance between the n-grid field restricted by 2 x 2
block means and the n/2-grid field, is computed on the device
(`ch_ensemble_refinement_error`); log2(E_n / E_2n) is the observed order of convergence.
Each grid is one handle; only two are alive at a time.  A single grid fills the GPU only
with the launch shapes that split its lines (the fused segment forms up to n = 1024), so
each grid's shape is chosen by the autotuner on that grid before its run (tune=False keeps
the library's default, the split form with one thread per line).

    python -m paper_1911_03386_gb300.refinement --nmax 4096
"""
import argparse
import json
import math
import time

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl


def run_grid(n, preset=wl.REFINEMENT, torch=None, tune=True):
    """A handle holding the droplet run on the n-grid after its steps; (handle, info)."""
    steps, dt = wl.refinement_steps(n, preset)
    tuning = None
    if tune:
        from paper_1911_03386_gb300 import autotune
        desc = dict(nx=n, ny=n, L=preset["L"], gamma=preset["gamma"], dt=dt, C0=0.0, seed=wl.BASE_SEED)
        tuning, _ = autotune.tune([desc], ch.CH_FP64, steps=16)
    e = ch.Ensemble.create(n, n, preset["L"], preset["gamma"], dt, [0.0], wl.BASE_SEED, ch.CH_FP64)
    try:
        if tuning:
            e.set_tuning(**tuning)
        e.set_field(0, wl.droplet_field(n, preset["L"], preset["gamma"]))
        e.set_sampling(max(1, steps), 0.0, 0)  # no samples needed beyond the start
        t0 = time.perf_counter()
        e.step(steps)
        e.synchronize()
        wall = time.perf_counter() - t0
        F, D, _ = e.observables()  # of the field at T
    except Exception:
        e.close()
        raise
    return e, {"n": n, "steps": steps, "dt": dt, "s": preset["gamma"] * dt / (preset["L"] / n) ** 4,
               "run_s": wall, "grid_point_steps_per_s": n * n * steps / max(wall, 1e-12),
               "F_T": float(F[0]), "dFdt_T": float(D[0]), "tuning": e.tuning()}


def study(sizes=None, preset=wl.REFINEMENT, tune=True):
    """Rows {n, steps, dt, E_n (against n/2), order log2(E_n / E_2n)} for sizes[1:]."""
    sizes = list(preset["sizes"] if sizes is None else sizes)
    rows = []
    prev, prev_info = run_grid(sizes[0], preset, tune=tune)
    try:
        for n in sizes[1:]:
            cur, info = run_grid(n, preset, tune=tune)
            info["E_n"] = ch.ch_ensemble_refinement_error(cur.h, 0, prev.h, 0)
            prev.close()
            prev, prev_info = cur, info
            rows.append(info)
    finally:
        prev.close()
    for a, b in zip(rows, rows[1:]):
        a["order"] = math.log2(a["E_n"] / b["E_n"]) if a["E_n"] > 0 and b["E_n"] > 0 else None
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nmin", type=int, default=128)
    ap.add_argument("--nmax", type=int, default=2048)
    ap.add_argument("--T", type=float, default=wl.REFINEMENT["T"], help="final time (the study's is 10)")
    ap.add_argument("--no-tune", action="store_true", help="the library's default launch shapes")
    args = ap.parse_args()
    preset = dict(wl.REFINEMENT, T=args.T)
    sizes = [n for n in preset["sizes"] if args.nmin <= n <= args.nmax]
    print(json.dumps(study(sizes, preset, tune=not args.no_tune)), flush=True)


if __name__ == "__main__":
    main()
