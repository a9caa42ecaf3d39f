"""The autotuner (paper_1911_03386_gb300/autotune.py) on an uneven batch: every candidate
it times is a valid shape, the winner is the fastest of its table, and the batch stepped
with the winner still matches the oracle."""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import autotune
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def batch():
    out, base = [], 0
    for k, (nx, ny, c0) in enumerate([(64, 64, 0.0), (128, 32, 0.2), (96, 80, 0.4), (32, 128, 0.1)]):
        out.append(dict(nx=nx, ny=ny, L=TWO_PI, gamma=0.005, dt=1e-3, C0=c0, seed=91, counter_base=base))
        base += nx * ny
    return out


@pytest.mark.parametrize("prec", [ch.CH_FP32, ch.CH_FP64])
def test_tuner_picks_fastest_valid_shape(prec, tmp_path):
    descs = batch()
    cands = autotune.candidates(prec)[:6] + [dict(split=0, row_seg=16)]  # the last one does not fit 96
    best, table = autotune.tune(descs, prec, cands=cands, steps=8)
    assert len(table) == len(cands) - 1
    assert best == min(table, key=lambda r: r[1])[0]
    path = str(tmp_path / "tune.json")
    autotune.store(path, descs, prec, best)
    assert autotune.cached(path, descs, prec) == best
    orc = get_oracle()
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_tuning(**best)
        e.step(30)
        for k, d in enumerate(descs):
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], 30)
            assert np.max(np.abs(e.field(k) - ref.C)) <= (1e-12 if prec == ch.CH_FP64 else 1e-4)
