"""The paper-campaign driver (asymmetric start set from the host, sampled run, on-device
statistics) on small ensembles, against the oracle."""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import campaign
from paper_1911_03386_gb300 import workloads as wl
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu

# the campaign's gamma, dt and start on 32^2 grids (dx = 2 pi / 32), 50 steps
SMALL = dict(wl.CAMPAIGN, dx=2 * math.pi / 32, T=0.06, every=5, window=(0.0, 0.06))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("prec,tol", [(ch.CH_FP64, 1e-12), (ch.CH_FP32, 1e-4)])
def test_host_start_runs_match_oracle(prec, tol):
    orc = get_oracle()
    n, M, L = 32, 3, 2 * math.pi
    steps = int(round(SMALL["T"] / SMALL["dt"]))
    descs = [dict(nx=n, ny=n, L=L, gamma=SMALL["gamma"], dt=SMALL["dt"], C0=0.45, seed=wl.BASE_SEED,
                  counter_base=k * n * n) for k in range(M)]
    with ch.Ensemble.batch(descs, prec) as e:
        for k in range(M):
            e.set_field(k, wl.asymmetric_field(n, wl.BASE_SEED, k))
        e.set_sampling(5, 0.0, 64)
        e.step(steps)
        for k in range(M):
            C0 = wl.asymmetric_field(n, wl.BASE_SEED, k)
            assert abs(C0.mean() - 0.45) < 0.01 and C0.min() >= 0.4 and C0.max() < 0.5
            ref = orc.run(C0, L, SMALL["gamma"], SMALL["dt"], steps, every=5)
            assert np.max(np.abs(e.field(k) - ref.C)) <= tol


@pytest.mark.parametrize("start", ["asymmetric", "symmetric"])
def test_campaign_driver_small(start):
    out = campaign.run(2 * math.pi, 6, ch.CH_FP64, preset=SMALL, start=start)
    assert out["n"] == 32 and out["steps"] == 50 and out["samples"] == 10 and out["start"] == start
    assert out["runs_finite"] == 6 and out["runs_counted_last_sample"] == 6
    assert math.isfinite(out["beta0_window_mean_mu1"]) and math.isfinite(out["k_fit_mu2"])


def test_symmetric_start_is_the_library_start_about_zero():
    # Sec. 4.3's symmetric mixture: mean zero, the device start C = 0.1 (2u - 1); runs match
    # the oracle from the oracle's own start
    orc = get_oracle()
    n, M, L = 32, 2, 2 * math.pi
    steps = int(round(SMALL["T"] / SMALL["dt"]))
    descs = [dict(nx=n, ny=n, L=L, gamma=SMALL["gamma"], dt=SMALL["dt"], C0=0.0, seed=wl.BASE_SEED,
                  counter_base=k * n * n) for k in range(M)]
    with ch.Ensemble.batch(descs, ch.CH_FP64) as e:
        for k in range(M):
            start = orc.initial_field(n, n, 0.0, wl.BASE_SEED, k * n * n)
            assert abs(start.mean()) < 0.01 and np.max(np.abs(start)) <= 0.1
            assert np.array_equal(e.field(k), start)
        e.step(steps)
        for k in range(M):
            ref = orc.run(orc.initial_field(n, n, 0.0, wl.BASE_SEED, k * n * n), L, SMALL["gamma"], SMALL["dt"], steps)
            assert np.max(np.abs(e.field(k) - ref.C)) <= 1e-12
