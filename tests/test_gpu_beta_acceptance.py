"""The FP32 form against the FP64 path on the ensemble mean of the time-averaged beta.

The dynamics are chaotic, so FP32 and FP64 runs from the same start part ways over long
horizons and their fields are not compared there; what must agree is the ensemble
statistic the paper reports: the window average of beta per run (Sec. 3.3 Eq. (42),
applied per run as in Sec. 4.2, Table 4), averaged over the runs of each initial mean
C0.  Acceptance: |mean_32 - mean_64| <= SE_64 = s_64 / sqrt(M) per C0 group, with s_64
the sample standard deviation of the FP64 runs' values (the reading of "within one
standard error").  Workload: the 256 x 256^2 ensemble's parameters (gamma = 0.005,
dt = 1e-3, C0 = 0 and 0.4, window t >= 4) on 64 x 64 grids, 64 runs per group, its whole
20 000-step horizon.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import replicas
from paper_1911_03386_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def window_betas(descs, prec, steps, every, t1):
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_sampling(every, t1, capacity=0)
        e.step(steps)
        avg, cnt = e.beta_avg()
    return np.asarray(avg), np.asarray(cnt)


def test_fp32_beta_average_within_one_standard_error_of_fp64():
    p = wl.ENSEMBLE_256
    n, per_group, steps = 64, 64, p["steps"]
    c0s = [0.0] * per_group + [0.4] * per_group
    descs = [dict(nx=n, ny=n, L=p["L"], gamma=p["gamma"], dt=p["dt"], C0=c0, seed=wl.BASE_SEED,
                  counter_base=k * n * n) for k, c0 in enumerate(c0s)]
    b64, c64 = window_betas(descs, ch.CH_FP64, steps, p["every"], p["t1"])
    b32, c32 = window_betas(descs, ch.CH_FP32, steps, p["every"], p["t1"])
    # every run sampled the whole window (t = 4 ... 19.9, every 100 steps)
    assert np.all(c64 == c32) and c64.min() >= (steps - int(round(p["t1"] / p["dt"]))) // p["every"] - 1
    assert np.all(np.isfinite(b64)) and np.all(np.isfinite(b32))
    s64 = replicas.ensemble_stats(b64, c0s)
    s32 = replicas.ensemble_stats(b32, c0s)
    for c0 in sorted(set(c0s)):
        d = abs(s32[c0]["mean"] - s64[c0]["mean"])
        print("C0 = %g: FP32 %.5f +- %.5f, FP64 %.5f +- %.5f, |diff| %.2e = %.3f SE" % (
            c0, s32[c0]["mean"], s32[c0]["se"], s64[c0]["mean"], s64[c0]["se"], d, d / s64[c0]["se"]))
        assert s64[c0]["n"] == per_group
        assert d <= s64[c0]["se"], (c0, d, s64[c0]["se"])
