"""Autotuner of the kernels' launch shapes (ch_tuning) for a grid size and precision.

The three phases of a step are separate kernels, so each kernel's shape is tuned on its
own: a candidate's phase time is measured with CUDA events around ch_launch_phase on the
handle's stream (warm, after a few untimed launches), on a synthetic ensemble of the
given grid size holding about `points` grid points.  The best shape per kernel is
combined into one ch_tuning.  Results can be cached in a JSON file keyed by grid size,
precision and device name.
"""
import json
import os

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl


def _candidates(precision):
    """(split, phase, fields) candidates per kernel."""
    out = []
    for threads in (128, 256, 512):
        for rb in (2, 4, 8, 16, 32):
            out.append((1, 0, dict(rows_band=rb, threads=threads)))
    for sb in (8, 16, 32, 64, 128):
        out.append((1, 1, dict(sweep_band=sb, stream=0)))
    out.append((1, 1, dict(stream=1)))
    out.append((1, 2, dict(stream=1)))
    for threads in (128, 256):
        for rb in (8, 16, 32, 64):
            for rp in (1, 2, 4, 8):
                if rb * rp <= threads:
                    out.append((0, 0, dict(rows_band=rb, rows_p=rp, threads=threads)))
    for threads in (128, 256, 512):
        for cb in (8, 16, 32, 64):
            for cp in (1, 2, 4, 8):
                for persist in (0, 1):
                    if cb * cp <= threads:
                        out.append((-1, 2, dict(cols_panel=cb, cols_p=cp, threads=threads, stream=0, persist=persist)))
    return out


def _time_phase(torch, e, stream, phase, reps):
    for _ in range(3):
        for ph in range(3):
            e.launch_phase(ph)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    for r in range(reps):
        for ph in range(3):
            if ph == phase:
                evs[2 * r].record(stream)
            e.launch_phase(ph)
            if ph == phase:
                evs[2 * r + 1].record(stream)
    torch.cuda.synchronize()
    return sorted(evs[2 * r].elapsed_time(evs[2 * r + 1]) for r in range(reps))[reps // 2]


def tune(nx, ny, precision, points=1 << 24, reps=20, verbose=False):
    """Best ch_tuning fields for nx x ny members in `precision`; returns (tuning, table)."""
    import torch

    m = max(1, points // (nx * ny))
    C0 = [0.0 if k % 2 == 0 else 0.4 for k in range(m)]
    stream = torch.cuda.Stream()
    table = []
    with ch.Ensemble.create(nx, ny, wl.TWO_PI, 0.005, 1e-3, C0, wl.BASE_SEED, precision) as e:
        e.set_stream(stream.cuda_stream)
        e.set_sampling(100, 0.0, 0)
        for split, phase, fields in _candidates(precision):
            kw = dict(fields)
            kw["split"] = split if split >= 0 else (1 if precision == ch.CH_FP64 else 0)
            try:
                e.set_tuning(**kw)
            except ch.ChError:
                continue
            ms = _time_phase(torch, e, stream, phase, reps)
            table.append(dict(split=kw["split"], phase=phase, ms=ms, **fields))
            if verbose:
                print(kw, phase, "%.4f ms" % ms, flush=True)
    best = {}
    for split in (0, 1):
        row = [t for t in table if t["split"] == split and t["phase"] == 0]
        sw = [t for t in table if t["split"] == 1 and t["phase"] == 1]
        if not row:
            continue
        r0 = min(row, key=lambda t: t["ms"])
        tot = r0["ms"]
        sel = dict(split=split, rows_band=r0["rows_band"], rows_p=r0.get("rows_p", 0), threads=r0["threads"])
        if split:
            s1 = min(sw, key=lambda t: t["ms"])
            tot += s1["ms"]
            if s1.get("stream"):
                sel["stream"] = 1
            else:
                sel["sweep_band"] = s1["sweep_band"]
                sel["stream"] = 0
        best[split] = (tot, sel)
    split, (tot, sel) = min(best.items(), key=lambda kv: kv[1][0])
    # column kernel: streaming (split form only) or shared-memory panels with the stencil's thread count
    cols = [t for t in table if t["phase"] == 2 and not t.get("stream")]
    same = [t for t in cols if t["threads"] == sel["threads"]] or cols
    c2 = min(same, key=lambda t: t["ms"])
    cms = c2["ms"]
    streamed = [t for t in table if t["phase"] == 2 and t.get("stream")]
    if split and sel.get("stream") and streamed and streamed[0]["ms"] < cms:
        cms = streamed[0]["ms"]
    else:
        if split and sel.get("stream"):
            # streaming rows with panel columns is not a shape; compare the two whole options
            s_panel = min([t for t in table if t["phase"] == 1 and not t.get("stream")], key=lambda t: t["ms"])
            sel.update(stream=0, sweep_band=s_panel["sweep_band"])
            tot += s_panel["ms"] - min(t["ms"] for t in table if t["phase"] == 1)
        sel.update(cols_panel=c2["cols_panel"], cols_p=c2["cols_p"], persist=c2.get("persist", 0))
    return sel, dict(table=table, step_ms=tot + cms, members=m)


def cached(path, nx, ny, precision):
    """Tuning stored for (nx, ny, precision, device) in the JSON file at path, or None."""
    import torch

    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    return data.get("%dx%d|%d|%s" % (nx, ny, precision, torch.cuda.get_device_name()))


def store(path, nx, ny, precision, tuning):
    import torch

    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data["%dx%d|%d|%s" % (nx, ny, precision, torch.cuda.get_device_name())] = tuning
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
