"""Serving (ch_server_*): continuous batching of single-run requests on the GPU.

Checks that a served run equals the oracle's run of the same request, that a run's
result is identical alone and in a mix of other runs admitted before and after it,
that admission respects the HBM budget, that a short request submitted while a long
one runs finishes first, and the error paths (unknown ids, timeouts, bad requests).
"""
import math
import time

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def req(nx, ny, nsteps, C0=0.0, seed=11, gamma=0.005, dt=1e-3, L=TWO_PI, every=10, t1=-1.0, field=True):
    out = np.zeros(nx * ny) if field else None
    return dict(nx=nx, ny=ny, L=L, gamma=gamma, dt=dt, C0=C0, seed=seed, nsteps=nsteps, every=every, t1=t1,
                field_out=out)


def test_served_runs_match_oracle():
    orc = get_oracle()
    reqs = [req(32, 32, 80, C0=0.0, seed=1), req(48, 40, 120, C0=0.4, seed=2, gamma=0.01),
            req(64, 64, 50, C0=0.2, seed=3), req(5, 7, 30, C0=0.1, seed=4, gamma=0.02)]
    with ch.Server(64 << 20, ch.CH_FP64, max_members=8) as s:
        ids = [s.submit(**r) for r in reqs]
        res = [s.wait(i, 120.0) for i in ids]
    for r, out in zip(reqs, res):
        C0 = orc.initial_field(r["nx"], r["ny"], r["C0"], r["seed"], 0)
        t1 = 0.2 * r["nsteps"] * r["dt"]
        ref = orc.run(C0, r["L"], r["gamma"], r["dt"], r["nsteps"], every=r["every"], t1=t1)
        got = r["field_out"].reshape(r["ny"], r["nx"])
        assert np.max(np.abs(got - ref.C)) <= 1e-12
        Fo, Do = orc.field_observables(ref.C, r["L"], r["gamma"])
        assert out["steps"] == r["nsteps"]
        assert abs(out["F"] - Fo) <= 1e-11 * abs(Fo)
        assert abs(out["dFdt"] - Do) <= 1e-9 * abs(Do)
        assert out["beta_count"] == ref.beta_count
        assert abs(out["beta_avg"] - ref.beta_avg) <= 1e-9 * abs(ref.beta_avg)
        assert out["t_total_s"] >= out["t_run_s"] > 0


@pytest.mark.parametrize("prec", [ch.CH_FP32, ch.CH_FP64])
def test_result_same_alone_and_in_mix(prec):
    target = req(96, 64, 300, C0=0.3, seed=77)
    with ch.Server(256 << 20, prec) as s:
        alone = s.wait(s.submit(**target), 120.0)
    field_alone = target["field_out"].copy()
    target["field_out"][:] = 0
    others_before = [req(n, n, k, C0=0.1 * (n % 5), seed=n + k) for n, k in [(128, 500), (32, 40), (64, 260)]]
    others_after = [req(n, m, k, seed=3 * n) for n, m, k in [(256, 256, 200), (40, 72, 120), (17, 33, 90)]]
    with ch.Server(256 << 20, prec) as s:
        ids = [s.submit(**r) for r in others_before]
        time.sleep(0.05)
        tid = s.submit(**target)
        ids += [s.submit(**r) for r in others_after]
        mixed = s.wait(tid, 120.0)
        for i in ids:
            s.wait(i, 120.0)
        assert s.stats()["max_running"] >= 2
    assert np.array_equal(field_alone, target["field_out"])
    for k in ("F", "dFdt", "beta", "beta_avg", "beta_count", "steps"):
        assert alone[k] == mixed[k], k


def test_fp32_compensated_run_served_equals_ensemble():
    # s_x = 21.5 > 16: the served FP32 run keeps hi + lo in two arena blocks
    r = req(64, 48, 150, C0=0.3, seed=5, gamma=0.5, dt=4e-3, L=TWO_PI)
    with ch.Server(16 << 20, ch.CH_FP32) as s:
        res = s.wait(s.submit(**r), 120.0)
    with ch.Ensemble.create(64, 48, TWO_PI, 0.5, 4e-3, [0.3], 5, ch.CH_FP32) as e:
        e.set_tuning(split=0)
        e.set_sampling(10, 0.2 * 150 * 4e-3, 0)
        e.step(150)
        field = e.field(0)
        F, D, B = e.observables()
        avg, cnt = e.beta_avg()
    assert np.array_equal(r["field_out"].reshape(48, 64), field)
    assert res["F"] == F[0] and res["beta_avg"] == avg[0]


def test_admission_respects_hbm_budget():
    # FP32: a 128x128 run needs 2 x 64 KiB (field + scratch); the budget fits one at a time
    budget = 2 * 128 * 128 * 4 + 4096
    with ch.Server(budget, ch.CH_FP32) as s:
        ids = [s.submit(**req(128, 128, 60, seed=k, field=False)) for k in range(3)]
        for i in ids:
            s.wait(i, 120.0)
        st = s.stats()
        assert st["completed"] == 3 and st["max_running"] == 1
        assert st["arena_peak_bytes"] <= st["arena_bytes"]
        with pytest.raises(ch.ChError) as e:
            s.submit(**req(256, 256, 10, field=False))
        assert e.value.code == ch.CH_ENOMEM


def test_short_request_overtakes_long_one():
    with ch.Server(256 << 20, ch.CH_FP32) as s:
        long_id = s.submit(**req(256, 256, 3000, field=False))
        time.sleep(0.02)
        short_id = s.submit(**req(64, 64, 100, field=False))
        short = s.wait(short_id, 120.0)
        assert s.poll(long_id) is None  # still running when the short one is done
        long_ = s.wait(long_id, 120.0)
        assert short["t_total_s"] < long_["t_total_s"]
        assert s.stats()["max_running"] == 2


def test_server_error_paths():
    with ch.Server(32 << 20, ch.CH_FP32) as s:
        with pytest.raises(ch.ChError) as e:
            s.poll(12345)
        assert e.value.code == ch.CH_ENOTFOUND
        with pytest.raises(ch.ChError) as e:
            s.submit(**req(4, 16, 10, field=False))
        assert e.value.code == ch.CH_EINVAL
        with pytest.raises(ch.ChError) as e:
            s.submit(**req(16, 16, 0, field=False))
        assert e.value.code == ch.CH_EINVAL
        rid = s.submit(**req(256, 256, 5000, field=False))
        with pytest.raises(ch.ChError) as e:
            s.wait(rid, 0.001)
        assert e.value.code == ch.CH_ETIMEOUT
    # destroying a server with work in flight returns promptly


def test_diverging_run_is_reported():
    with ch.Server(32 << 20, ch.CH_FP64) as s:
        # dt far beyond the scheme's stability limit for this gamma: the run blows up
        rid = s.submit(**req(32, 32, 400, C0=0.0, gamma=0.01, dt=1.0, field=False))
        with pytest.raises(ch.ChError) as e:
            s.wait(rid, 120.0)
        assert e.value.code == ch.CH_ENONFINITE
