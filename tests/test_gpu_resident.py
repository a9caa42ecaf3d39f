"""The cluster-resident form of the FP32 step against the oracle and the tiled kernels.

FP32 members with nx = 128 or 256 and ny = 32 Q (Q = 1 .. 8) are stepped by a cluster
of Q CTAs that keep the field in shared memory for a launch of many steps (row
recurrences as segment scans, column recurrences joined through distributed shared
memory, halo rows exchanged between neighbouring CTAs).  Checks: fields and sampled
observables against the FP64 oracle (the FP32 bars of the other FP32 tests), every
cluster size and both row widths, compensated members (s > 16), a launch chunk boundary,
horizons that end inside a launch, observables of the current field, and agreement with
the tiled kernels (resident = -1) to FP32 rounding.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu

TWO_PI = 2 * math.pi
SEED = wl.BASE_SEED


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def orc():
    return get_oracle()


# every cluster size Q = ny / 32 from 1 to 8, both row widths, s from 0.05 to 36 (the last
# two members are compensated pairs, s > 16)
MEMBERS = [
    dict(nx=256, ny=256, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.4),
    dict(nx=128, ny=128, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0),
    dict(nx=256, ny=32, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.2),
    dict(nx=128, ny=64, L=3.0, gamma=0.004, dt=2e-3, C0=-0.3),
    dict(nx=256, ny=96, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.1),
    dict(nx=128, ny=160, L=4.0, gamma=0.01, dt=1e-3, C0=0.3),
    dict(nx=256, ny=192, L=TWO_PI, gamma=0.004, dt=1e-3, C0=0.0),
    dict(nx=128, ny=224, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.25),
    dict(nx=256, ny=256, L=TWO_PI, gamma=0.01, dt=1.2e-3, C0=0.45),   # s = 33: compensated
    dict(nx=128, ny=96, L=2.0, gamma=0.01, dt=1e-3, C0=0.0),          # s = 36: compensated
]


def descs_of(members):
    out, base = [], 0
    for k, d in enumerate(members):
        out.append(dict(d, seed=SEED + k, counter_base=base))
        base += d["nx"] * d["ny"]
    return out


def s_max(d):
    return max(d["gamma"] * d["dt"] / (d["L"] / d["nx"]) ** 4, d["gamma"] * d["dt"] / (d["L"] / d["ny"]) ** 4)


def test_members_run_resident():
    with ch.Ensemble.batch(descs_of(MEMBERS), ch.CH_FP32) as e:
        assert e.tuning()["resident"] == 1
    with ch.Ensemble.batch(descs_of(MEMBERS[8:9]), ch.CH_FP32) as e:
        assert e.tuning()["resident"] == -1  # compensated 256-wide: tiled unless asked
        e.set_tuning(resident=1)
        assert e.tuning()["resident"] == 1
    with ch.Ensemble.batch(descs_of(MEMBERS), ch.CH_FP64) as e:
        assert e.tuning()["resident"] == -1  # FP32 only


@pytest.mark.parametrize("rows", [32, 64])
def test_resident_members_match_oracle(orc, rows):
    # rows = 64: the 256-column members with ny a multiple of 64 run in CTAs of 64 rows
    descs = descs_of(MEMBERS)
    nsteps, every = 120, 20
    with ch.Ensemble.batch(descs, ch.CH_FP32) as e:
        e.set_tuning(resident=1, resident_rows=rows)  # every member, compensated 256-wide ones included
        assert e.tuning()["resident_rows"] == rows
        e.set_sampling(every, 0.0, capacity=16)
        e.step(nsteps)
        F, D, B = e.observables()
        for k, d in enumerate(descs):
            start = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(start, d["L"], d["gamma"], d["dt"], nsteps, every=every)
            got = e.field(k)
            err = np.max(np.abs(got - ref.C))
            # the FP32 bar, or where s is large the FP32 solve's conditioning: up to 2 u
            # (1 + 16 s) of a step's size per step, the first step being the largest
            one = start.copy()
            orc.step(one, d["L"], d["gamma"], d["dt"])
            bound = max(1e-4, nsteps * 2 * 2.0 ** -24 * (1 + 16 * s_max(d)) * np.max(np.abs(one - start)))
            assert err <= bound, (k, d, err, bound)
            ser = e.series(k, 16)
            assert ser.shape[0] == ref.series.shape[0] == nsteps // every
            assert np.array_equal(ser[:, 0], ref.series[:, 0])  # sample times bit-exact
            np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-5)
            np.testing.assert_allclose(ser[:, 2], ref.series[:, 2], rtol=1e-3)
            # observables of the current field: the FP64 functional of the stored field
            Fo, Do = orc.field_observables(got, d["L"], d["gamma"])
            assert abs(F[k] - Fo) <= 1e-11 * abs(Fo), (k, F[k], Fo)
            assert abs(D[k] - Do) <= 1e-9 * abs(Do), (k, D[k], Do)
            assert e.step_index(k) == nsteps


def test_resident_agrees_with_tiled_kernels(orc):
    descs = descs_of(MEMBERS)
    nsteps = 60
    fields = {}
    for res, rows in ((1, 32), (1, 64), (-1, 0)):
        with ch.Ensemble.batch(descs, ch.CH_FP32) as e:
            e.set_tuning(resident=res, resident_rows=rows)
            assert e.tuning()["resident"] == res
            e.set_sampling(10, 0.0, capacity=8)
            e.step(nsteps)
            fields[rows] = [(e.field(k), e.series(k, 8)) for k in range(len(descs))]
    for k, d in enumerate(descs):
        (a, sa), (a64, sa64), (b, sb) = fields[32][k], fields[64][k], fields[0][k]
        # two FP32 evaluations of the same steps, each within 2 u (1 + 16 s) of the step's
        # size per step (the solve's conditioning; the first step is the largest) plus the
        # rounding of the stored field: their difference is within twice that
        start = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
        one = start.copy()
        orc.step(one, d["L"], d["gamma"], d["dt"])
        bound = 2 * (nsteps * 2 * 2.0 ** -24 * (1 + 16 * s_max(d)) * np.max(np.abs(one - start)) + 2.0 ** -24)
        assert np.max(np.abs(a - b)) <= bound, (k, np.max(np.abs(a - b)), bound)
        assert np.max(np.abs(a64 - b)) <= bound, (k, np.max(np.abs(a64 - b)), bound)
        np.testing.assert_allclose(sa[:, 1:], sb[:, 1:], rtol=1e-4)
        np.testing.assert_allclose(sa64[:, 1:], sb[:, 1:], rtol=1e-4)


def test_resident_launch_chunks_and_horizons(orc):
    # 4100 steps cross the 4096-step launch chunk; the sampled times stay on schedule
    d = [dict(nx=128, ny=32, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.0),
         dict(nx=256, ny=64, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.4)]
    descs = descs_of(d)
    nsteps = 4100
    with ch.Ensemble.batch(descs, ch.CH_FP32) as e:
        e.set_sampling(100, 1.0, capacity=64)
        e.step(nsteps)
        avg, cnt = e.beta_avg()
        for k, dd in enumerate(descs):
            assert e.step_index(k) == nsteps
            ser = e.series(k, 64)
            assert ser.shape[0] == 41
            np.testing.assert_array_equal(ser[:, 0], np.arange(41) * 100 * dd["dt"])
            assert cnt[k] == 41 - 10  # samples with t >= 1
            assert math.isfinite(avg[k])
    # the same first member against the oracle over the first 300 steps
    with ch.Ensemble.batch(descs[:1], ch.CH_FP32) as e:
        e.step(300)
        start = orc.initial_field(128, 32, 0.0, descs[0]["seed"], 0)
        ref = orc.run(start, descs[0]["L"], descs[0]["gamma"], descs[0]["dt"], 300)
        assert np.max(np.abs(e.field(0) - ref.C)) <= 1e-4


def test_resident_serving_horizons_and_mix():
    # resident-size requests through a server: horizons ending inside a launch, and the
    # same request alone and in a mix gives the same result bit for bit
    reqs = [dict(nx=256, ny=256, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.3, seed=11, nsteps=137),
            dict(nx=128, ny=128, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.1, seed=12, nsteps=61),
            dict(nx=512, ny=512, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.2, seed=13, nsteps=40),
            dict(nx=128, ny=64, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0, seed=14, nsteps=200)]
    alone, fa = [], []
    for r in reqs:
        f = np.zeros(r["nx"] * r["ny"])
        with ch.Server(256 << 20, ch.CH_FP32) as s:
            alone.append(s.wait(s.submit(**r, field_out=f), 120.0))
        fa.append(f)
    fb = [np.zeros(r["nx"] * r["ny"]) for r in reqs]
    with ch.Server(256 << 20, ch.CH_FP32) as s:
        ids = [s.submit(**r, field_out=f) for r, f in zip(reqs, fb)]
        mixed = [s.wait(i, 120.0) for i in ids]
        assert s.stats()["max_running"] >= 2
    for r, a, b, x, y in zip(reqs, alone, mixed, fa, fb):
        assert a["steps"] == r["nsteps"] == b["steps"]
        for k in ("F", "dFdt", "beta", "beta_avg", "beta_count"):
            assert a[k] == b[k] or (math.isnan(a[k]) and math.isnan(b[k])), k
        assert np.array_equal(x, y) and np.all(np.isfinite(x))
