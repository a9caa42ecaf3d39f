"""Autotuner of a batch's launch shapes (ch_tuning).

Kernel classes are chosen per member by the library (segment, chunked, panel or streaming
forms, see include/ch.h); what remains to tune per batch is the step form, band heights,
CTA sizes and which classes are allowed.  Each candidate tuning is applied to the batch
and the whole step is timed with CUDA events around graph-replayed ch_step calls on the
handle's stream (after untimed warm-up steps); the fastest candidate wins.  The batch is
the caller's (member descriptors), so uneven batches are tuned as they run.  Results can
be cached in a JSON file keyed by the batch's sizes, precision and device name.
"""
import json
import os

import paper_1911_03386_gb300 as ch


def candidates(precision):
    """Candidate tunings (dicts of ch_tuning fields) for a precision."""
    out = []
    if precision == ch.CH_FP32:
        # members that fit the cluster-resident form use it in all of these (resident = 0);
        # the shapes vary the tiled kernels of the others, and the last two turn it off
        for row_seg in (0, -1):
            for band in (8, 16, 32):
                for threads in (128, 256):
                    for col_seg in (0, -1):
                        out.append(dict(split=0, row_seg=row_seg, rows_band=band, threads=threads, col_seg=col_seg))
        out.append(dict(split=0, resident=-1))
        out.append(dict(split=0, rows_band=8, threads=128, resident=-1))
    else:
        out.append(dict(split=1, stream=1))
        for band in (8, 16):
            out.append(dict(split=1, stream=1, rows_band=band))
        for row_seg in (0, -1):
            for col_seg in (0, -1):
                out.append(dict(split=0, row_seg=row_seg, col_seg=col_seg))
    return out


def time_step(torch, e, stream, warm=8, steps=32):
    """Milliseconds per time step of the handle's current tuning (graph replay)."""
    e.step(warm)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    e.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def tune(descs, precision, cands=None, steps=32, verbose=False):
    """Fastest tuning for the batch `descs` (member descriptors of ch_create_batch);
    returns (tuning dict, table of (tuning, ms per step))."""
    import torch

    cands = candidates(precision) if cands is None else cands
    stream = torch.cuda.Stream()
    table = []
    with ch.Ensemble.batch(descs, precision) as e:
        e.set_stream(stream.cuda_stream)
        e.set_sampling(100, 0.0, 0)
        for t in cands:
            try:
                e.set_tuning(**t)
            except ch.ChError:
                continue  # a shape the batch does not admit
            e.reset()
            e.set_sampling(100, 0.0, 0)
            ms = time_step(torch, e, stream, steps=steps)
            table.append((dict(t), ms))
            if verbose:
                print(t, "%.4f ms" % ms, flush=True)
    if not table:
        raise RuntimeError("no candidate tuning applies to this batch")
    best = min(table, key=lambda r: r[1])[0]
    return best, table


def batch_key(descs, precision):
    import torch

    sizes = sorted({(d["nx"], d["ny"]) for d in descs})
    return "%s|%d|%d|%s" % (",".join("%dx%d" % s for s in sizes), len(descs), precision,
                            torch.cuda.get_device_name())


def cached(path, descs, precision):
    """Tuning stored for this batch signature in the JSON file at path, or None."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    return data.get(batch_key(descs, precision))


def store(path, descs, precision, tuning):
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data[batch_key(descs, precision)] = tuning
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
