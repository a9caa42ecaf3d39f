#!/usr/bin/env python
"""Benchmark of the GB300 Cahn-Hilliard ensemble engine (one JSON line on rank 0).

Workload (default): an ensemble of 256 independent periodic runs on 256x256 grids,
gamma = 0.005, dt = 1e-3, 20 000 steps (t = 20), members 0-127 at C0 = 0 and 128-255 at
C0 = 0.4, uniform noise +-0.1, F / dF/dt / beta sampled every 100 steps and beta averaged
over t >= 4, FP64.  One benchmark "step" is one sampling interval: 100 time steps of
every member (stencil + row sweep, column sweep + update) including the sample.  The
default --steps 200 therefore times the whole 20 000-step horizon.

Reported:
  value          grid-point-steps/s of the FP64 path, device-timed (CUDA events on the
                 engine's stream), inputs resident in HBM; max over ranks for N > 1.
  e2e            the same metric through the C ABI with host buffers: the initial fields
                 are uploaded from page-locked host memory and every step ends with a
                 device-to-host read of F, dF/dt, beta (ch_observables).
  fp32           the FP32 form on the same workload (throughput, <beta> against FP64).
  roofline       the dominant kernel against its bound (FP64 pipe for the FP64 path).
  ensemble_stats moments, histograms and trend statistics of beta across runs: kernel
                 times on a paper-size synthetic ensemble and the workload's own values.
  droplets       Model 1: 100 droplet populations of 512 to t = 40 (adaptive Dormand-Prince
                 on the GPU) and their Table 2 statistics.
  refinement     the Appendix-A grid-refinement study (E_n and observed order) up to
                 --refinement-nmax points per axis.
  cpu_baseline   the FP64 CPU oracle timed on this host's cores (bounded sample).
  --impl reference  times the oracle alone (the reference arm), same metric and config.
"""
import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CH grid-point-steps/s per GB300 (FP32 vs FP64 path); served p50/p99 latency"
UNIT = "grid-point-steps/s"
STEPS_PER_BENCH_STEP = 100
FP64_PIPE_PEAK = 1.25e12  # FLOP/s: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal; replaced by the measured rate)


def _hbm_peak():
    """Measured HBM copy bandwidth (B/s) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]) * 1e9, "measured hbm_gbs (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6.8e12, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


HBM_PEAK, HBM_PEAK_SOURCE = _hbm_peak()
# Algorithmic work per grid point of one time step, per kernel (flop, field words moved):
#   stencil  mu (9) + R' (6) flop; read C, write R'
#   rowsweep forward/backward row recurrences (8); read R', write W
#   rows     (fused) stencil + row recurrences (23); read C, write W
#   cols     column recurrences (8) + update (2); read W, read C, write C
#   resident (cluster-resident FP32 form) the whole step on chip: mu (9) + R' (6) + row
#            recurrences (8) + column recurrences (8) + update (2) flop; the field crosses HBM
#            once per launch (read and written: 2 words per point per launch, not per step)
KERNEL_WORK = {"stencil": (15.0, 2), "rowsweep": (8.0, 2), "rows": (23.0, 2), "cols": (10.0, 3), "resident": (33.0, 0)}
# The same work in FP64 pipe operations (an ADD or MUL takes a pipe slot like an FMA):
#   stencil  mu 6 (3 FMA, 1 MUL, 2 ADD) + R' 4 (2 FMA, 2 ADD); rowsweep 4 (2 FMA per
#   recurrence); cols 5 (4 FMA + the update FMA)
KERNEL_OPS = {"stencil": 10.0, "rowsweep": 4.0, "rows": 14.0, "cols": 5.0}


# ------------------------------------------------------------------------------------------
# CPU oracle legs (spawn pool, created before any CUDA call)
# ------------------------------------------------------------------------------------------
def _oracle_worker(args):
    nx, ny, L, gamma, dt, C0, seed, base, nsteps, field = args
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle.oracle import get
    orc = get()
    C = orc.initial_field(nx, ny, C0, seed, base) if field is None else np.array(field)
    t = time.perf_counter()
    for _ in range(nsteps):
        orc.step(C, L, gamma, dt)
    return time.perf_counter() - t, C


def make_pool(cores):
    from oracle import build as obuild
    obuild.build()
    return mp.get_context("spawn").Pool(cores)


def oracle_sample(pool, p, cores, nsteps, fields=None):
    """Run `cores` members of the workload for nsteps each, one per process."""
    from paper_1911_03386_gb300 import workloads as wl
    jobs = []
    for k in range(cores):
        mk = (k * len(p["C0"])) // cores
        jobs.append((p["nx"], p["ny"], p["L"], p["gamma"], p["dt"], p["C0"][mk], wl.BASE_SEED,
                     mk * p["nx"] * p["ny"], nsteps, None if fields is None else fields[k]))
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    pts = cores * p["nx"] * p["ny"] * nsteps
    return pts, wall, [r[1] for r in res]


def cpu_baseline(pool, p, cores, target_s=12.0):
    pts1, wall1, _ = oracle_sample(pool, p, cores, 2)          # calibration
    per_step = wall1 / 2
    nsteps = max(2, int(target_s / max(per_step, 1e-6)))
    pts, wall, _ = oracle_sample(pool, p, cores, nsteps)
    out = {"value": pts / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d members x %d steps of %dx%d (one member per process, FP64, single-threaded C "
                     "oracle), %.1f s wall" % (cores, nsteps, p["nx"], p["ny"], wall)}
    # the 64^2 single-run workload in full (2000 steps, one core)
    from paper_1911_03386_gb300 import workloads as wl
    s = wl.SINGLE_64
    job = (s["nx"], s["ny"], s["L"], s["gamma"], s["dt"], s["C0"][0], wl.BASE_SEED, 0, s["steps"], None)
    w = pool.apply(_oracle_worker, (job,))[0]
    out["single_64_full"] = {"workload": s["name"], "time_steps": s["steps"], "wall_s": w, "cores": 1,
                             "value": s["nx"] * s["ny"] * s["steps"] / w, "unit": UNIT}
    return out


# ------------------------------------------------------------------------------------------
# Helpers
# ------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to $CH_CLOCK_LOG_DIR when set (kept beside the run's outputs),
        # else to a temporary file; the JSON line carries their summary either way
        log_dir = os.environ.get("CH_CLOCK_LOG_DIR")
        self.path = (os.path.join(log_dir, "clocks_rank%d.csv" % index) if log_dir and os.path.isdir(log_dir)
                     else os.path.join(tempfile.gettempdir(), "ch_clocks_%d_%d.csv" % (os.getpid(), index)))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() in ("active", "0x1", "1")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


def finite_or_none(x):
    """Strict JSON: non-finite floats (e.g. the beta average of a run that ends before its
    window opens) become null."""
    if isinstance(x, float):
        return x if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: finite_or_none(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [finite_or_none(v) for v in x]
    return x


STEP_SOURCES = ("ch_api.cu", "ch_internal.h", "ch_kernels.cu")  # the step's kernels and launch shapes


def kernel_source_hash():
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1911_03386_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu table (profiles/traffic.txt),
    if it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            lines = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    src = kernel_source_hash()
    for ln in lines:
        parts = [x.strip() for x in ln.split("|")]
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[3] == src:
            return int(parts[2])
    return None


def kernel_name(phase, t, elt, nx=256):
    """Kernel that runs a phase under tuning t (member 0's kernel classes)."""
    ty = "double" if elt == 8 else "float"
    if phase == "resident":
        return "res_kernel<%d, %d, false, false>" % (nx, t.get("resident_rows") or 32)
    if phase == "stencil":
        return "stencil_kernel<%s>" % ty
    if phase == "rowsweep":
        return ("rowstream_kernel<%s>" if t["stream"] else "rowsweep_kernel<%s>") % ty
    if phase == "rows":
        if t["row_seg"] in (16, 32):
            return "rows_seg_kernel<%s, %d, %s>" % (ty, t["row_seg"], "true" if t["persist"] & 2 else "false")
        return "rowsT_kernel<%s>" % ty if t["row_seg"] == 1 else "rows_kernel<%s, false>" % ty
    if t["col_seg"] in (16, 32):
        return "colseg_kernel<%s, %d>" % (ty, t["col_seg"])
    if t["split"] and t["stream"]:
        return "colstream_kernel<%s>" % ty
    return "cols_kernel<%s, %s>" % (ty, "true" if t["persist"] & 1 else "false")


def workload_config(p, prec_name):
    return {"workload": p["name"], "members": len(p["C0"]), "nx": p["nx"], "ny": p["ny"], "L": "2*pi",
            "gamma": p["gamma"], "dt": p["dt"], "time_steps": p["steps"], "C0": "half 0.0, half 0.4",
            "time_steps_per_bench_step": STEPS_PER_BENCH_STEP, "sample_every": p["every"], "beta_window_t1": p["t1"],
            "precision": prec_name,
            "l2": "inputs larger than L2: field %d MiB + row-solve scratch %d MiB (FP64) > 126 MiB L2" % (
                len(p["C0"]) * p["nx"] * p["ny"] * 8 >> 20, len(p["C0"]) * p["nx"] * p["ny"] * 8 >> 20)}


# ------------------------------------------------------------------------------------------
# GPU legs
# ------------------------------------------------------------------------------------------
def run_gpu_leg(ch, torch, p, prec, K, W, rank, world, dist, profile_kernels=True):
    """Device-timed run of K bench steps after W warm-up steps; returns a dict."""
    from paper_1911_03386_gb300 import replicas
    from paper_1911_03386_gb300 import workloads as wl
    npts = len(p["C0"]) * p["nx"] * p["ny"]
    # replica r: its own members, disjoint counter ranges of the same SplitMix64 stream
    descs = [dict(nx=p["nx"], ny=p["ny"], L=p["L"], gamma=p["gamma"], dt=p["dt"], C0=c0, seed=wl.BASE_SEED,
                  counter_base=replicas.member_counter_base(rank, len(p["C0"]), p["nx"] * p["ny"]) + k * p["nx"] * p["ny"])
             for k, c0 in enumerate(p["C0"])]
    e = ch.Ensemble.batch(descs, prec)
    stream = torch.cuda.Stream()
    e.set_stream(stream.cuda_stream)
    e.set_sampling(p["every"], p["t1"], capacity=0)
    for _ in range(W):
        e.step(STEPS_PER_BENCH_STEP)
    e.synchronize()
    e.reset()  # the timed region covers steps 0 .. K*100 of the workload
    e.set_sampling(p["every"], p["t1"], capacity=0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(K):
            e.step(STEPS_PER_BENCH_STEP)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    avg, cnt = e.beta_avg()
    out = {"ms": ms, "pts": npts * K * STEPS_PER_BENCH_STEP, "clocks": clk.summary(), "beta_avg": avg,
           }
    out["tuning"] = e.tuning()
    out["launches"] = K * STEPS_PER_BENCH_STEP * (3 if out["tuning"]["split"] else 2)
    if profile_kernels and out["tuning"]["resident"] == 1:
        # The cluster-resident form runs a sampling interval (100 steps) as one launch of its
        # kernel: events around each launch, over 4 intervals after the timed region.
        out["launches"] = K
        reps = 4
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        evs[0].record(stream)
        for r in range(reps):
            e.step(STEPS_PER_BENCH_STEP)
            evs[r + 1].record(stream)
        torch.cuda.synchronize()
        out["kernels"] = {"resident": sum(evs[r].elapsed_time(evs[r + 1]) for r in range(reps)) / reps /
                          STEPS_PER_BENCH_STEP}
        out["resident_launch_ms"] = evs[0].elapsed_time(evs[reps]) / reps
    elif profile_kernels:
        # Per-kernel durations: events around each phase launch on the engine's stream,
        # over 2 sampling intervals of the same state after the timed region.
        split = out["tuning"]["split"]
        names = ["stencil", "rowsweep", "cols"] if split else ["rows", None, "cols"]
        reps = 2 * STEPS_PER_BENCH_STEP
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4 * reps)]
        for r in range(reps):
            for ph in range(3):
                evs[4 * r + ph].record(stream)
                e.launch_phase(ph)
            evs[4 * r + 3].record(stream)
        torch.cuda.synchronize()
        out["kernels"] = {}
        for ph, name in enumerate(names):
            if name is None:
                continue
            out["kernels"][name] = sum(evs[4 * r + ph].elapsed_time(evs[4 * r + ph + 1]) for r in range(reps)) / reps
    e.close()
    return out


def run_descs_leg(ch, torch, descs, prec, nsteps, every, t1, warm=300, tuning=None):
    """Device-timed run of an uneven batch (member descriptors) for nsteps time steps after
    `warm` untimed ones (then reset): grid-point-steps/s, per-member window averages."""
    e = ch.Ensemble.batch(descs, prec)
    if tuning:
        e.set_tuning(**tuning)
    stream = torch.cuda.Stream()
    e.set_stream(stream.cuda_stream)
    e.set_sampling(every, t1, capacity=0)
    e.step(warm)
    e.synchronize()
    e.reset()
    e.set_sampling(every, t1, capacity=0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    e.step(nsteps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    avg, cnt = e.beta_avg()
    pts = sum(d["nx"] * d["ny"] for d in descs) * nsteps
    out = {"value": pts / (ms * 1e-3), "unit": UNIT, "ms_per_time_step": ms / nsteps, "time_steps": nsteps,
           "tuning": e.tuning(), "beta_avg": avg}
    e.close()
    return out


def run_stats_leg(ch, torch, p, prec, nsteps=2000, every=10):
    """Ensemble statistics of beta (Sec. 3.3 Eqs. (41a,b), (42); Sec. 1 Eq. (7)).
    (a) The statistics kernels timed with CUDA events on a synthetic beta ensemble of the
        paper's Sec. 4.2 size (1024 runs; 32768 sample times, about t = 100 at dt = 0.0012
        sampled every 2-3 steps): 256 MiB of beta, above the L2.
    (b) The statistics of the workload's own ensemble over its first nsteps time steps,
        sampled every `every` steps, per initial mean C0: mu_1 and mu_2 at the last sample,
        the window mean of mu_1 over the second half and k of mu_2 = k t."""
    import numpy as np
    from paper_1911_03386_gb300 import workloads as wl
    M, T, nb = 1024, 32768, 100
    t, beta = wl.beta_ensemble(M, T, seed=wl.BASE_SEED + 77, t_end=100.0, diverged=8)
    tb = torch.from_numpy(t).cuda()
    bb = torch.from_numpy(beta).cuda()
    mom = torch.empty((T, ch.CH_MOMENTS), dtype=torch.float64, device="cuda")
    hist = torch.empty((T, nb + 2), dtype=torch.int64, device="cuda")
    tr = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    calls = {
        "moments": lambda: ch.ch_stats_moments(tb.data_ptr(), bb.data_ptr(), M, T, T, mom.data_ptr(), st.cuda_stream),
        "histogram": lambda: ch.ch_stats_histogram(bb.data_ptr(), M, T, T, 0.0, 0.6, nb, hist.data_ptr(),
                                                   st.cuda_stream),
        "trend": lambda: ch.ch_stats_trend(mom.data_ptr(), T, 20.0, 100.0, 20.0, 100.0, tr.data_ptr(), st.cuda_stream),
    }
    dense = {"members": M, "samples": T, "bins": nb, "beta_bytes": M * T * 8}
    for name, fn in calls.items():
        for _ in range(3):
            fn()
        reps = 10
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        dense[name + "_ms"] = ms
        if name != "trend":
            # algorithmic bytes: beta read once (plus t and the output rows)
            byts = M * T * 8 + (T * 8 * (1 + ch.CH_MOMENTS) if name == "moments" else T * (nb + 2) * 8)
            dense[name + "_gbs"] = byts / (ms * 1e-3) / 1e9
            dense[name + "_frac_of_measured_hbm"] = byts / (ms * 1e-3) / HBM_PEAK
    tv = tr.cpu().numpy()
    dense["synthetic_beta0_window_20_100"] = float(tv[0])
    dense["synthetic_k_fit_20_100"] = float(tv[1])
    dense["synthetic_law"] = "beta0 = 0.28, mu_2 = 0.0056 t (the generator's parameters)"
    del tb, bb, mom, hist

    descs = [dict(nx=p["nx"], ny=p["ny"], L=p["L"], gamma=p["gamma"], dt=p["dt"], C0=c0, seed=wl.BASE_SEED,
                  counter_base=k * p["nx"] * p["ny"]) for k, c0 in enumerate(p["C0"])]
    own = {"time_steps": nsteps, "sample_every": every}
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_sampling(every, 0.0, nsteps // every + 1)
        e.step(nsteps)
        e.synchronize()
        t_end = nsteps * p["dt"]
        for c0 in sorted(set(p["C0"])):
            members = [k for k, c in enumerate(p["C0"]) if c == c0]
            t0 = time.perf_counter()
            m = e.moments(members=members)
            wall = time.perf_counter() - t0
            b0, k, nw, nf = e.trend(0.5 * t_end, t_end, 0.0, t_end, members=members)
            own["C0=%g" % c0] = {"members": len(members), "samples": int(m.shape[0]), "mu1_last": float(m[-1, 2]),
                                 "mu2_last": float(m[-1, 3]), "mu3_last": float(m[-1, 4]),
                                 "mu4_last": float(m[-1, 5]),
                                 "beta0_window": float(b0), "window": [0.5 * t_end, t_end], "k_fit": float(k),
                                 "fit_window": [0.0, t_end], "moments_call_wall_ms": 1e3 * wall}
    return {"dense_synthetic": dense, "workload_ensemble": own}


def run_e2e_leg(ch, torch, p, prec, K, rank, dist):
    """End to end through the C ABI with host buffers (see module docstring)."""
    import numpy as np
    from paper_1911_03386_gb300 import replicas
    from paper_1911_03386_gb300 import workloads as wl
    m = len(p["C0"])
    npts = m * p["nx"] * p["ny"]
    descs = [dict(nx=p["nx"], ny=p["ny"], L=p["L"], gamma=p["gamma"], dt=p["dt"], C0=c0, seed=wl.BASE_SEED,
                  counter_base=replicas.member_counter_base(rank, m, p["nx"] * p["ny"]) + k * p["nx"] * p["ny"])
             for k, c0 in enumerate(p["C0"])]
    e = ch.Ensemble.batch(descs, prec)
    e.set_sampling(p["every"], p["t1"], capacity=0)
    # the job's input: every member's initial field, in page-locked host memory
    host_in = torch.empty(npts, dtype=torch.float64).pin_memory()
    e.get_fields_ptr(host_in.data_ptr())
    e.reset()
    e.set_sampling(p["every"], p["t1"], capacity=0)
    F = np.empty(m)
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e.set_fields_ptr(host_in.data_ptr())
    for _ in range(K):
        e.step(STEPS_PER_BENCH_STEP)
        F, D, B = e.observables()
    avg, cnt = e.beta_avg()
    t1 = time.perf_counter()
    if dist:
        torch.distributed.barrier()
    e.close()
    return {"s": t1 - t0, "pts": npts * K * STEPS_PER_BENCH_STEP, "h2d": npts * 8 / K, "d2h": 3 * m * 8}


def run_serving_leg(ch, torch, n_requests, rate, seed, precision, budget_bytes=8 << 30, keep=False):
    """Poisson stream of single-run requests through one server; latencies are the
    library's submit-to-result times (keep=True also returns each request's result)."""
    import numpy as np
    from paper_1911_03386_gb300 import workloads as wl
    reqs = wl.request_stream(count=n_requests, rate=rate, seed=seed)
    lat, ids, results = [], [], []
    with ch.Server(budget_bytes, precision, max_members=4096) as srv:
        t0 = time.perf_counter()
        for r in reqs:
            delay = r["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(nx=r["nx"], ny=r["ny"], L=r["L"], gamma=r["gamma"], dt=r["dt"], C0=r["C0"],
                                  seed=r["seed"], nsteps=r["steps"]))
        t_sub = time.perf_counter() - t0
        for i in ids:
            res = srv.wait(i, 3600.0)
            lat.append(res["t_total_s"])
            results.append(res)
        wall = time.perf_counter() - t0
        st = srv.stats()
    work = sum(r["nx"] * r["ny"] * r["steps"] for r in reqs)
    span = max(reqs[-1]["arrival"], 1e-9)
    cap = st["grid_point_steps"] / max(st["busy_s"], 1e-9)
    lat = np.array(lat)
    out = {"requests": n_requests, "rate_per_s": rate, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "max_s": float(lat.max()),
            "throughput": work / wall, "capacity": cap, "offered": work / span, "rho": (work / span) / cap,
            "max_running": st["max_running"], "submit_span_s": t_sub, "wall_s": wall, "unit": UNIT}
    if keep:
        out["results"] = results
    return out


def run_peak_leg(ch, torch):
    """FMA throughput of the FP64 and FP32 pipes (ch_fma_peak), CUDA-event timed on one
    stream over about a second of work each, with the SM clock sampled meanwhile: the
    denominators of the FP64 path's "alu" roofline and of the on-chip FP32 kernels."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    out = {"sms": sms}
    for prec, name, iters in ((ch.CH_FP64, "fp64", 400), (ch.CH_FP32, "fp32", 20000)):
        blocks, threads, reps = 2 * sms, 1024, 40
        for _ in range(2):
            ch.ch_fma_peak(prec, blocks, threads, iters, sink.data_ptr(), st.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            a.record(st)
            flops = 0.0
            for _ in range(reps):
                flops += ch.ch_fma_peak(prec, blocks, threads, iters, sink.data_ptr(), st.cuda_stream)
            b.record(st)
            torch.cuda.synchronize()
        s_ = a.elapsed_time(b) * 1e-3
        c = clk.summary()
        rate = flops / s_
        r = {"flops_per_s": rate, "tflops": rate / 1e12, "seconds": s_, "clocks": c}
        if c.get("sm_mhz"):
            # FMAs per SM per clock at the sampled median clock (2 flop per FMA)
            r["fma_per_sm_per_clk"] = rate / 2 / (sms * c["sm_mhz"] * 1e6)
            r["at_max_clock_tflops"] = rate / 1e12 * c["sm_max_mhz"] / c["sm_mhz"]
        out[name] = r
    return out


def run_beta_check(ch, torch, p):
    """<beta> acceptance of the FP32 form on the workload itself: the whole horizon (20 000
    steps, t = 20) in FP64 and FP32 from the same start, the window average of beta per
    run (t >= t1), then per C0 group the mean and standard error over the runs and
    whether |mean_32 - mean_64| <= SE_64 (within one standard error)."""
    from paper_1911_03386_gb300 import workloads as wl
    descs = [dict(nx=p["nx"], ny=p["ny"], L=p["L"], gamma=p["gamma"], dt=p["dt"], C0=c0, seed=wl.BASE_SEED,
                  counter_base=k * p["nx"] * p["ny"]) for k, c0 in enumerate(p["C0"])]
    labels = list(p["C0"])
    res = {"workload": p["name"], "time_steps": p["steps"], "sample_every": p["every"], "window_t1": p["t1"],
           "window": [p["t1"], p["steps"] * p["dt"]]}
    stats = {}
    for prec, name in ((ch.CH_FP64, "fp64"), (ch.CH_FP32, "fp32")):
        stream = torch.cuda.Stream()
        with ch.Ensemble.batch(descs, prec) as e:
            e.set_stream(stream.cuda_stream)
            e.set_sampling(p["every"], p["t1"], capacity=0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            e.step(p["steps"])
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            avg, cnt = e.beta_avg()
        stats[name] = replicas_stats(avg, labels)
        res[name] = {"seconds": ms * 1e-3, "value": len(descs) * p["nx"] * p["ny"] * p["steps"] / (ms * 1e-3),
                     "unit": UNIT, "samples_in_window": int(min(cnt)), "beta_avg": stats[name]}
    res["within_one_se"] = {k: abs(stats["fp32"][k]["mean"] - stats["fp64"][k]["mean"]) <= stats["fp64"][k]["se"]
                            for k in stats["fp64"]}
    res["diff_in_se"] = {k: abs(stats["fp32"][k]["mean"] - stats["fp64"][k]["mean"]) / stats["fp64"][k]["se"]
                         for k in stats["fp64"]}
    return res


def replicas_stats(values, labels):
    """Mean, standard error and count of the window-averaged beta per initial mean C0."""
    from paper_1911_03386_gb300 import replicas
    return {"C0=%g" % k: v for k, v in replicas.ensemble_stats(values, labels).items()}


def value_estimate(res):
    """Grid-point-steps/s of one device-timed leg."""
    return res["pts"] / (res["ms"] * 1e-3)


# Cases for profiler captures (one kernel, few launches, a few hundred MB at most), stepped
# 200 times to leave the start transient, then one more sampling interval of 100 steps
# (steps 200 and 300 are sample steps; step 250 is not).  The suffixes 64 and 32 are the
# precision (resident32: FP32 and 32 members):
#   resident32  FP32, cluster-resident form, 32 members of the 256 x 256 ensemble (one wave
#               of clusters): one res_kernel launch per 100 steps
#   stream64    FP64 split form, the whole 256-member ensemble (256 MB, above the L2):
#               stencil_kernel, rowstream_kernel, colstream_kernel per step
#   segment32   FP32 with the resident form off, the whole ensemble (134 MB):
#               rows_seg_kernel, colseg_kernel per step
# name: (precision, ch_tuning.resident, members, workload)
KERNEL_CASES = {"resident32": ("fp32", 0, 32, "ensemble"), "stream64": ("fp64", -1, 256, "ensemble"),
                "segment32": ("fp32", -1, 256, "ensemble"), "long16": ("fp32", -1, 16, "long")}


def kernel_case(name):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03386_gb300 as ch
    from paper_1911_03386_gb300 import workloads as wl
    prec, res, members, work = KERNEL_CASES[name]
    p = wl.ENSEMBLE_256 if work == "ensemble" else wl.LONG_1024
    stride = len(p["C0"]) // members
    descs = [dict(nx=p["nx"], ny=p["ny"], L=p["L"], gamma=p["gamma"], dt=p["dt"], C0=p["C0"][stride * k],
                  seed=wl.BASE_SEED, counter_base=k * p["nx"] * p["ny"]) for k in range(members)]
    with ch.Ensemble.batch(descs, ch.CH_FP32 if prec == "fp32" else ch.CH_FP64) as e:
        e.set_tuning(resident=res)
        stream = torch.cuda.Stream()
        e.set_stream(stream.cuda_stream)
        # sampling every 100 steps; the 1024^2 workload averages over the last 80 % of its horizon
        e.set_sampling(p.get("every", 100), p.get("t1", 0.2 * p["steps"] * p["dt"]), capacity=0)
        e.step(200)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e.step(STEPS_PER_BENCH_STEP)
        b.record(stream)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": name, "members": len(descs), "time_steps": STEPS_PER_BENCH_STEP,
                          "ms": a.elapsed_time(b), "tuning": e.tuning()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="bench steps (100 time steps each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=120)
    ap.add_argument("--serving-full", action="store_true",
                    help="serving legs of 1000 requests each: the workload's 50/s, the highest rate at which "
                         "the measured load stays below 0.8 of capacity, and 200 requests FP32 vs FP64 "
                         "(several minutes of GPU time)")
    ap.add_argument("--no-batches", action="store_true", help="skip the uneven-batch and 1024^2 legs")
    ap.add_argument("--no-stats", action="store_true", help="skip the ensemble-statistics leg")
    ap.add_argument("--campaign", action="store_true",
                    help="also run the paper's L = 2 pi campaign ensemble (1024 x 256^2 to t = 100, FP32; "
                         "about 75 s of GPU time) and report its Table 4 statistics")
    ap.add_argument("--no-droplets", action="store_true",
                    help="skip the Model 1 leg (100 populations of 512 droplets to t = 40, about 10 s)")
    ap.add_argument("--refinement-nmax", type=int, default=1024,
                    help="largest grid of the Appendix-A refinement study leg (0: skip)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA-throughput measurement")
    ap.add_argument("--no-beta-check", action="store_true",
                    help="skip the whole-horizon <beta> check of the FP32 form against FP64 (about 20 s)")
    ap.add_argument("--long-beta", action="store_true",
                    help="also run the 32 x 1024^2 coarsening ensemble over its whole horizon in both precisions "
                         "and compare <beta> (minutes of GPU time)")
    ap.add_argument("--kernel-case", choices=sorted(KERNEL_CASES),
                    help="run one small profiling case (for ncu) and exit; see kernel_case()")
    args = ap.parse_args()
    if args.kernel_case:
        kernel_case(args.kernel_case)
        return
    K, W = args.steps, args.warmup
    if W < 3:
        raise SystemExit("--warmup must be >= 3")

    from paper_1911_03386_gb300 import workloads as wl
    p = wl.ENSEMBLE_256
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1

    if args.impl == "reference":
        # The reference arm: the FP64 CPU oracle as it stands, on the host cores, rank 0 only.
        if rank != 0:
            return
        pool = make_pool(cores)
        fields = None
        for _ in range(W):
            _, _, fields = oracle_sample(pool, p, cores, 1, fields)
        tot_pts, tot_s = 0, 0.0
        ref_steps = 2
        for _ in range(K):
            pts, wall, fields = oracle_sample(pool, p, cores, ref_steps, fields)
            tot_pts += pts
            tot_s += wall
        pool.close()
        v = tot_pts / tot_s
        line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K, "warmup": W,
                "ms_per_step": 1e3 * tot_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": workload_config(p, "fp64"), "impl": "reference",
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": "per step: %d members x %d time steps of %dx%d, one member per process"
                                           % (cores, ref_steps, p["nx"], p["ny"])},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(finite_or_none(line), allow_nan=False), flush=True)
        return

    pool = make_pool(cores) if (rank == 0 and world == 1 and not args.no_cpu) else None

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03386_gb300 as ch

    dist = world > 1
    torch.cuda.set_device(local_rank)
    if dist:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    r64 = run_gpu_leg(ch, torch, p, ch.CH_FP64, K, W, rank, world, dist)
    r32 = None if args.no_fp32 else run_gpu_leg(ch, torch, p, ch.CH_FP32, K, W, rank, world, dist)
    e2e = None if args.no_e2e else run_e2e_leg(ch, torch, p, ch.CH_FP64, K, rank, dist)
    peaks = None if args.no_peaks else run_peak_leg(ch, torch)
    beta_check = None if (args.no_beta_check or rank != 0) else run_beta_check(ch, torch, p)
    serving = None
    if not args.no_serving and rank == 0:
        # the serving workload's own rate, then a rate the measured capacity sustains
        nreq = 1000 if args.serving_full else args.serving_requests
        at_rate = run_serving_leg(ch, torch, nreq, wl.SERVING["rate"], wl.BASE_SEED, ch.CH_FP32)
        # mean work of a request from the generator itself (not from one leg's sample)
        probe = wl.request_stream(count=20000, rate=1.0, seed=wl.BASE_SEED + 99)
        mean_work = sum(r["nx"] * r["ny"] * r["steps"] for r in probe) / len(probe)
        # a steady leg: a rate below capacity (busy-time throughput of the loaded leg); with
        # the full legs, lowered until the measured load is at most 0.8
        frac = 0.7 if args.serving_full else 0.5
        steady_rate = frac * at_rate["capacity"] / mean_work
        steady = run_serving_leg(ch, torch, nreq, steady_rate, wl.BASE_SEED + 1, ch.CH_FP32)
        tries = 0
        while args.serving_full and steady["rho"] > 0.8 and tries < 4:
            steady_rate *= 0.75 / steady["rho"]
            steady = run_serving_leg(ch, torch, nreq, steady_rate, wl.BASE_SEED + 1, ch.CH_FP32)
            tries += 1
        # the served FP32 form against the plain FP64 GPU path: the same requests at a rate
        # the FP64 ensemble throughput sustains, with paired <beta> differences
        ncmp = 200 if args.serving_full else max(10, nreq // 3)
        cmp_rate = 0.5 * value_estimate(r64) / mean_work
        c32 = run_serving_leg(ch, torch, ncmp, cmp_rate, wl.BASE_SEED + 2, ch.CH_FP32, keep=True)
        c64 = run_serving_leg(ch, torch, ncmp, cmp_rate, wl.BASE_SEED + 2, ch.CH_FP64, keep=True)
        import numpy as np
        creqs = wl.request_stream(count=ncmp, rate=cmp_rate, seed=wl.BASE_SEED + 2)
        pairs = [(a["beta_avg"], b["beta_avg"], r["nx"]) for a, b, r in zip(c32.pop("results"), c64.pop("results"), creqs)
                 if math.isfinite(a["beta_avg"]) and math.isfinite(b["beta_avg"])]
        # relative difference for every request; absolute difference for the well-resolved
        # sizes (n <= 256): at finer grids the factorised scheme damps the grid-scale modes of
        # the initial noise by only ~1/(4s) per step, and they dominate dF/dt and beta
        rel = np.array([abs(x - y) / max(abs(y), 1e-300) for x, y, _ in pairs])
        d = np.array([x - y for x, y, n in pairs if n <= 256])
        serving = {"workload": wl.SERVING["name"], "precision": "fp32",
                   "sample": "%d requests per leg (n in {64..1024}^2, horizons U[1000, 50000], C0 ~ U[0, 0.5])"
                             % nreq, "mean_work_per_request": mean_work, "at_workload_rate": at_rate,
                   "workload_rate_over_capacity": at_rate["rho"] > 1.0, "steady": steady,
                   "fp32_vs_fp64_same_requests": {
                       "requests": ncmp, "rate_per_s": cmp_rate, "fp32": c32, "fp64": c64,
                       "p99_ratio_fp64_over_fp32": c64["p99_s"] / c32["p99_s"],
                       "beta_avg_rel_diff_max": float(rel.max()) if rel.size else None,
                       "beta_avg_rel_diff_median": float(np.median(rel)) if rel.size else None,
                       "beta_avg_diff_mean_n_le_256": float(d.mean()) if d.size else None,
                       "beta_avg_diff_max_abs_n_le_256": float(np.abs(d).max()) if d.size else None}}

    batches = None
    if not args.no_batches and rank == 0:
        # the uneven batch (its whole 2000-step horizon) and the 32 x 1024^2 ensemble (the
        # first 1000 of its 200 000 steps), both precisions, default kernel classes
        import numpy as np
        ub = wl.UNEVEN
        udescs = wl.uneven_members()
        lb = wl.LONG_1024
        ldescs = [dict(nx=lb["nx"], ny=lb["ny"], L=lb["L"], gamma=lb["gamma"], dt=lb["dt"], C0=c0, seed=wl.BASE_SEED,
                       counter_base=k * lb["nx"] * lb["ny"]) for k, c0 in enumerate(lb["C0"])]
        batches = {}
        for name, descs, nsteps, every, t1 in [(ub["name"], udescs, ub["steps"], 100, 0.4),
                                               (lb["name"], ldescs, 1000, 100, 0.1)]:
            legs = {}
            for prec, pname in ((ch.CH_FP32, "fp32"), (ch.CH_FP64, "fp64")):
                # FP64 uneven batch: the fused segment forms (its few lines per size do not
                # fill the GPU with the split form's thread-per-line streams)
                tk = {"split": 0} if (prec == ch.CH_FP64 and descs is udescs) else None
                r = run_descs_leg(ch, torch, descs, prec, nsteps, every, t1, tuning=tk)
                r.pop("beta_avg")
                legs[pname] = r
            legs["fp32_speedup"] = legs["fp32"]["value"] / legs["fp64"]["value"]
            if descs is udescs:
                # the same batch with the autotuner's choice of shape per precision
                from paper_1911_03386_gb300 import autotune
                for prec, pname in ((ch.CH_FP32, "fp32"), (ch.CH_FP64, "fp64")):
                    best, table = autotune.tune(descs, prec)
                    r = run_descs_leg(ch, torch, descs, prec, nsteps, every, t1, tuning=best)
                    r.pop("beta_avg")
                    r["candidates"] = len(table)
                    legs[pname + "_autotuned"] = r
            batches[name] = legs
        if args.long_beta:
            # <beta> over the whole horizon, t in [20, 100] (the paper's window), FP32 vs FP64
            long = {}
            for prec, pname in ((ch.CH_FP32, "fp32"), (ch.CH_FP64, "fp64")):
                r = run_descs_leg(ch, torch, ldescs, prec, lb["steps"], 100, 20.0, warm=100)
                labels = [d["C0"] for d in ldescs]
                st = replicas_stats(r.pop("beta_avg"), labels)
                long[pname] = dict(r, beta_avg=st)
            long["within_one_se"] = {k: abs(long["fp32"]["beta_avg"][k]["mean"] - long["fp64"]["beta_avg"][k]["mean"])
                                     <= long["fp64"]["beta_avg"][k]["se"] for k in long["fp64"]["beta_avg"]}
            batches[lb["name"] + "/whole-horizon"] = long

    stats = None
    if not args.no_stats and rank == 0:
        stats = run_stats_leg(ch, torch, p, ch.CH_FP64)
    refine = None
    if args.refinement_nmax >= 128 and rank == 0:
        # Appendix A: E_n between the n- and n/2-grids of a single-droplet run to T = 10,
        # dt = 0.1 dx, FP64 (the paper's table runs n = 128 ... 8192)
        from paper_1911_03386_gb300 import refinement
        sizes = [n for n in wl.REFINEMENT["sizes"] if n <= args.refinement_nmax]
        refine = {"workload": wl.REFINEMENT["name"], "gamma": wl.REFINEMENT["gamma"], "T": wl.REFINEMENT["T"],
                  "dt": "0.1 dx", "precision": "fp64", "rows": refinement.study(sizes)}

    drops = None
    if not args.no_droplets and rank == 0:
        # Model 1 (Secs. 2-3): Table 1's M = 100 populations, N = 512, t to 40, with the
        # window mean of mu_1 over [20, 40] and k of mu_2 = k t over [0, 40] (Table 2)
        from paper_1911_03386_gb300 import droplets
        drops = droplets.run(512)
    camp = None
    if args.campaign and rank == 0:
        from paper_1911_03386_gb300 import campaign
        camp = campaign.run(2 * math.pi, wl.CAMPAIGN["M"], ch.CH_FP32)
        camp["paper_table"] = dict(zip(["beta0", "k"], wl.CAMPAIGN["table4"]["2pi"]))

    from paper_1911_03386_gb300 import replicas
    tdist = torch.distributed if dist else None

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, tdist, device="cuda")

    def gather_avg(avg):
        return replicas.gather_members(avg, tdist, device="cuda")

    ms64 = max_over_ranks(r64["ms"])
    total_pts = r64["pts"] * world
    value = total_pts / (ms64 * 1e-3)
    avg64 = gather_avg(r64["beta_avg"])
    fp32 = None
    if r32 is not None:
        ms32 = max_over_ranks(r32["ms"])
        avg32 = gather_avg(r32["beta_avg"])
        fp32 = {"value": r32["pts"] * world / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32 / K,
                "speedup_vs_fp64": ms64 / ms32}
    e2e_line = None
    if e2e is not None:
        s = max_over_ranks(e2e["s"])
        e2e_line = {"value": e2e["pts"] * world / s, "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                    "d2h_bytes_per_step": e2e["d2h"]}

    cpu = cpu_baseline(pool, p, cores) if pool is not None else None
    if pool is not None:
        pool.close()
    if rank != 0:
        return

    import numpy as np

    def beta_stats(avg):
        m = len(p["C0"])
        labels = [p["C0"][k % m] for k in range(len(avg))]
        return {"C0=%g" % c0: v for c0, v in replicas.ensemble_stats(avg, labels).items()}

    npts = len(p["C0"]) * p["nx"] * p["ny"]

    def kernel_roofline(res, bound, elt):
        ks = res["kernels"]
        dom = max(ks, key=ks.get)
        flops, words = KERNEL_WORK[dom]
        tname = kernel_name(dom, res["tuning"], elt, p["nx"])
        if dom == "resident":
            return resident_roofline(res, tname, ks[dom], elt)
        per_launch = {k: {"ms": v, "achieved_tflops": KERNEL_WORK[k][0] * npts / (v * 1e-3) / 1e12,
                          "achieved_gbs": KERNEL_WORK[k][1] * elt * npts / (v * 1e-3) / 1e9} for k, v in ks.items()}
        step_ms = sum(ks.values())
        if bound == "alu":
            # the FP64 pipe issues an ADD or MUL in a slot an FMA would take: achieved is
            # counted in FMA-equivalent flops (2 per pipe operation) against the measured FMA
            # rate, i.e. the fraction of pipe slots the kernel's minimal operations fill; the
            # plain flop count and its fraction are given beside it
            ach = 2.0 * KERNEL_OPS[dom] * npts / (ks[dom] * 1e-3)
            ach_flop = flops * npts / (ks[dom] * 1e-3)
            # peak from the unit counts and the clock sampled during the timed region: 152 SMs x
            # 2 FP64 pipe operations per clock x 2 flop; the FMA probe's measured rate beside it
            sms = peaks["sms"] if peaks is not None else 152
            mhz = (res.get("clocks") or {}).get("sm_mhz") or 2070.0
            pk = sms * 2 * 2 * mhz * 1e6
            rl = {"bound": "alu", "kernel": tname, "achieved": ach / 1e12, "peak": pk / 1e12,
                  "unit": "TFLOP/s (FMA-equivalent: 2 x FP64 pipe operations)", "frac": ach / pk,
                  "peak_source": "derived: %d SMs x 2 FP64 pipe operations per clock x 2 flop x %.0f MHz "
                                 "(median SM clock of the timed region)" % (sms, mhz),
                  "pipe_ops_per_point": KERNEL_OPS[dom], "achieved_flop_tflops": ach_flop / 1e12,
                  "frac_flop": ach_flop / pk}
            if peaks is not None:
                rl["probe_fma_tflops"] = peaks["fp64"]["tflops"]
                rl["frac_of_probe"] = ach / peaks["fp64"]["flops_per_s"]
        else:
            ach = words * elt * npts / (ks[dom] * 1e-3)
            rl = {"bound": "hbm", "kernel": tname, "achieved": ach / 1e9, "peak": HBM_PEAK / 1e9, "unit": "GB/s",
                  "frac": ach / HBM_PEAK, "peak_source": HBM_PEAK_SOURCE}
        rl["traffic"] = ncu_traffic(tname, p["name"])
        rl["algorithmic_per_point"] = {"flop": flops, "bytes": words * elt}
        rl["per_kernel"] = per_launch
        rl["step_ms_sum_of_kernels"] = step_ms
        # the whole step against the HBM bound of any factorised ADI step: 2 reads + 2 writes
        # of a field word per point (16 B FP32, 32 B FP64)
        rl["fused_step_hbm"] = {"step_ms": step_ms, "algorithmic_bytes_per_point": 4 * elt,
                                "achieved_gbs": 4 * elt * npts / (step_ms * 1e-3) / 1e9,
                                "frac": 4 * elt * npts / (step_ms * 1e-3) / HBM_PEAK, "peak_gbs": HBM_PEAK / 1e9,
                                "peak_source": HBM_PEAK_SOURCE}
        return rl

    def resident_roofline(res, tname, step_ms, elt):
        # The cluster-resident kernel keeps the field on chip: its bound is the SM (FP32
        # issue and shared-memory latency), so it is stated against the measured FP32 FMA
        # rate with its minimal 33 flop per point and step.  Beside it: the HBM rate a
        # streaming step would need for the same throughput at the 16 B per point minimum
        # of any factorised ADI step, and the traffic it actually needs (one read and one
        # write of the field per launch of 100 steps).
        flops = KERNEL_WORK["resident"][0]
        ach = flops * npts / (step_ms * 1e-3)
        sms = peaks["sms"] if peaks is not None else 152
        mhz = (res.get("clocks") or {}).get("sm_mhz") or 2070.0
        pk = sms * 128 * 2 * mhz * 1e6  # 128 FP32 FMA lanes per SM
        rl = {"bound": "alu", "kernel": tname, "achieved": ach / 1e12, "peak": pk / 1e12,
              "unit": "TFLOP/s", "frac": ach / pk,
              "peak_source": "derived: %d SMs x 128 FP32 FMA per clock x 2 flop x %.0f MHz; FMA probe measured %s"
                             % (sms, mhz, "%.1f TFLOP/s" % peaks["fp32"]["tflops"] if peaks is not None else "-"),
              "traffic": ncu_traffic(tname, p["name"]), "traffic_per": "launch of 100 steps",
              "algorithmic_per_point": {"flop": flops, "bytes_per_launch": 2 * elt},
              "step_ms": step_ms, "launch_ms": res.get("resident_launch_ms"),
              "hbm_needed_per_launch_gbs": 2 * elt * npts / (res["resident_launch_ms"] * 1e-3) / 1e9}
        rl["fused_step_hbm"] = {"step_ms": step_ms, "algorithmic_bytes_per_point": 4 * elt,
                                "equivalent_gbs": 4 * elt * npts / (step_ms * 1e-3) / 1e9,
                                "frac": 4 * elt * npts / (step_ms * 1e-3) / HBM_PEAK, "peak_gbs": HBM_PEAK / 1e9,
                                "peak_source": HBM_PEAK_SOURCE,
                                "note": "equivalent rate: the resident form moves the field through HBM once per "
                                        "launch, not per step"}
        return rl

    roofline = kernel_roofline(r64, "alu", 8)
    roofline["tuning"] = r64["tuning"]
    if fp32 is not None:
        fp32["roofline"] = kernel_roofline(r32, "hbm", 4)
        fp32["roofline"]["tuning"] = r32["tuning"]
        s64, s32 = beta_stats(avg64), beta_stats(avg32)
        fp32["beta_avg_vs_fp64"] = {k: {"fp32": s32[k]["mean"], "fp64": s64[k]["mean"], "se_fp64": s64[k]["se"],
                                        "within_one_se": abs(s32[k]["mean"] - s64[k]["mean"]) <= s64[k]["se"]}
                                    for k in s64}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms64 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config(p, "fp64"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e_line,
            "gpu_launches": r64["launches"], "clocks": r64["clocks"], "fp32": fp32,
            "beta_avg": beta_stats(avg64), "serving": serving, "batches": batches, "ensemble_stats": stats,
            "refinement": refine, "campaign": camp, "droplets": drops, "peaks": peaks, "beta_check": beta_check,
            "kernel_source": kernel_source_hash()}
    print(json.dumps(finite_or_none(line), allow_nan=False), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
