"""GPU path (libch through its C ABI) against the FP64 CPU oracle.

Tolerances: FP64 fields within 1e-11 of the oracle after 1000 steps of the 64x64
workload (single run, gamma = 0.01, dt = 1e-3, C0 = 0); single steps within a
round-off bound; the FP32 form within 1e-4 over 200 steps.  Integer-exact parts (the
initial field in FP64, step counters, sample times) are compared bit for bit.
"""
import math
import os

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


def ens(nx, ny, C0, gamma=0.01, dt=1e-3, L=TWO_PI, prec=ch.CH_FP64, seed=SEED):
    return ch.Ensemble.create(nx, ny, L, gamma, dt, C0, seed, prec)


# ------------------------------------------------------------------------------------------
# Initial field
# ------------------------------------------------------------------------------------------
def test_initial_field_bit_exact(orc):
    nx, ny, C0 = 37, 23, [0.0, 0.4, -0.2]
    with ens(nx, ny, C0) as e:
        for k, c0 in enumerate(C0):
            ref = orc.initial_field(nx, ny, c0, SEED, k * nx * ny)
            assert np.array_equal(e.field(k), ref)
    with ens(nx, ny, C0, prec=ch.CH_FP32) as e:
        for k, c0 in enumerate(C0):
            ref = orc.initial_field(nx, ny, c0, SEED, k * nx * ny).astype(np.float32).astype(np.float64)
            assert np.array_equal(e.field(k), ref)


# ------------------------------------------------------------------------------------------
# One step: the row kernel (stencil + row solve) and the column kernel on their own
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(48, 40), (64, 64), (5, 7), (33, 130)])
def test_single_step_rows_and_columns(orc, nx, ny):
    L, gamma, dt = TWO_PI, 0.01, 1e-3
    C = np.ascontiguousarray(wl.random_field(ny, nx, 11, amplitude=0.8, mean=0.1))
    hx, hy = L / nx, L / ny
    mu, R = orc.rhs(C, hx, hy, gamma, dt)
    sx = gamma * dt / hx ** 4
    W_ref = np.stack([orc.penta_solve(sx, R[j]) for j in range(ny)])
    C_ref = C.copy()
    orc.step(C_ref, L, gamma, dt)
    with ens(nx, ny, [0.0], gamma, dt, L) as e:
        e.set_field(0, C)
        W = e.row_solve(0)
        assert np.array_equal(e.field(0), C) and e.step_index(0) == 0
        e.step(1)
        C1 = e.field(0)
    scaleW = np.max(np.abs(W_ref))
    assert np.max(np.abs(W - W_ref)) <= 1e-12 * scale_or_one(scaleW)
    # column kernel alone: the oracle's column solve applied to the GPU's own W
    sy = gamma * dt / hy ** 4
    dC_from_W = np.stack([orc.penta_solve(sy, W[:, i]) for i in range(nx)], axis=1)
    assert np.max(np.abs((C1 - C) - dC_from_W)) <= 1e-12 * scale_or_one(np.max(np.abs(dC_from_W)))
    assert np.max(np.abs(C1 - C_ref)) <= 1e-13


def scale_or_one(x):
    return x if x > 0 else 1.0


# ------------------------------------------------------------------------------------------
# The 64x64 workload: 1000 steps in FP64 against the oracle
# ------------------------------------------------------------------------------------------
def test_parity_single_64_fp64_1000_steps(orc):
    p = wl.SINGLE_64
    nsteps, every = 1000, 10
    C0 = orc.initial_field(p["nx"], p["ny"], 0.0, SEED, 0)
    ref = orc.run(C0, p["L"], p["gamma"], p["dt"], nsteps, every=every, t1=0.5)
    with ens(p["nx"], p["ny"], [0.0], p["gamma"], p["dt"], p["L"]) as e:
        e.set_sampling(every, 0.5, capacity=nsteps // every + 1)
        e.step(nsteps)
        C = e.field(0)
        ser = e.series(0, 1000)
        avg, cnt = e.beta_avg()
        assert e.step_index(0) == nsteps
    err = np.max(np.abs(C - ref.C))
    print("max|dC| after %d steps: %.3e" % (nsteps, err))
    assert err <= 1e-11
    assert ser.shape == ref.series.shape
    assert np.array_equal(ser[:, 0], ref.series[:, 0])  # sample times bit-exact
    np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-11)
    np.testing.assert_allclose(ser[:, 2], ref.series[:, 2], rtol=1e-9)
    np.testing.assert_allclose(ser[1:, 3], ref.series[1:, 3], rtol=1e-9)
    assert ser[0, 3] == 0.0
    assert cnt[0] == ref.beta_count
    assert abs(avg[0] - ref.beta_avg) <= 1e-9 * abs(ref.beta_avg)


# ------------------------------------------------------------------------------------------
# Linear amplification of single Fourier modes on a non-square grid (closed form)
# ------------------------------------------------------------------------------------------
def test_fourier_mode_amplification_gpu():
    nx, ny, L, gamma, dt, C0, eps, nsteps = 48, 40, TWO_PI, 0.01, 1e-3, 0.3, 1e-6, 25
    hx, hy = L / nx, L / ny
    X, Y = np.meshgrid(np.arange(nx) * hx, np.arange(ny) * hy)
    sigma, d = gamma * dt, 3 * C0 * C0 - 1
    with ens(nx, ny, [0.0], gamma, dt, L) as e:
        for kx, ky in [(1, 0), (0, 3), (2, 5), (11, 7), (24, 20), (4, 19)]:
            phi = np.cos(kx * X + ky * Y)
            e.set_field(0, C0 + eps * phi)
            e.step(nsteps)
            amp = np.sum((e.field(0) - C0) * phi) / np.sum(phi * phi)
            ax = 4 / hx ** 2 * math.sin(math.pi * kx / nx) ** 2
            ay = 4 / hy ** 2 * math.sin(math.pi * ky / ny) ** 2
            A = ax + ay
            G = 1 - dt * (A * d + gamma * A * A) / ((1 + sigma * ax * ax) * (1 + sigma * ay * ay))
            want = eps * G ** nsteps
            # modes that decay below the spacing of doubles near C0 are not representable
            assert abs(amp - want) <= 1e-7 * abs(want) + 1e-15, (kx, ky, amp, want)


# ------------------------------------------------------------------------------------------
# Uneven batch: every member against its own oracle run (small, ragged, large s)
# ------------------------------------------------------------------------------------------
UNEVEN_SMALL = [
    dict(nx=5, ny=5, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.0),
    dict(nx=7, ny=9, L=1.0, gamma=0.002, dt=1e-3, C0=0.3),      # s large: pre-roll longer than the line
    dict(nx=33, ny=17, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.4),
    dict(nx=64, ny=48, L=TWO_PI, gamma=0.005, dt=1e-3, C0=-0.2),
    dict(nx=100, ny=37, L=4.0, gamma=0.02, dt=5e-4, C0=0.1),
    dict(nx=16, ny=130, L=TWO_PI, gamma=0.005, dt=2e-3, C0=0.0),
]


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
def test_uneven_batch_members_match_oracle(orc, prec):
    descs = []
    base = 0
    for k, d in enumerate(UNEVEN_SMALL):
        dd = dict(d, seed=SEED + k, counter_base=base)
        base += d["nx"] * d["ny"]
        descs.append(dd)
    nsteps = 60
    with ch.Ensemble.batch(descs, prec) as e:
        e.step(nsteps)
        for k, d in enumerate(descs):
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps)
            err = np.max(np.abs(e.field(k) - ref.C))
            tol = 1e-12 if prec == ch.CH_FP64 else 1e-4
            assert err <= tol, (k, d, err)


# ------------------------------------------------------------------------------------------
# FP32 form against the FP64 oracle
# ------------------------------------------------------------------------------------------
def test_fp32_form_200_steps(orc):
    p = wl.SINGLE_64
    C0 = orc.initial_field(p["nx"], p["ny"], 0.0, SEED, 0)
    ref = orc.run(C0, p["L"], p["gamma"], p["dt"], 200)
    with ens(p["nx"], p["ny"], [0.0], p["gamma"], p["dt"], p["L"], prec=ch.CH_FP32) as e:
        e.step(200)
        err = np.max(np.abs(e.field(0) - ref.C))
    print("FP32 max|dC| after 200 steps: %.3e" % err)
    assert err <= 1e-4


# ------------------------------------------------------------------------------------------
# FP32 form at large s: the field is kept as the pair hi + lo (compensated update) for
# members with max(s_x, s_y) > 16; the pair holds the FP64 initial field to ~2^-48
# ------------------------------------------------------------------------------------------
COMP = dict(nx=64, ny=48, L=TWO_PI, gamma=0.5, dt=4e-3)  # s_x = 21.5 > 16, dt < 0.7 gamma


def test_fp32_compensated_initial_field_and_round_trip(orc):
    d = COMP
    with ens(d["nx"], d["ny"], [0.2, -0.1], d["gamma"], d["dt"], d["L"], prec=ch.CH_FP32) as e:
        for k, c0 in enumerate([0.2, -0.1]):
            ref = orc.initial_field(d["nx"], d["ny"], c0, SEED, k * d["nx"] * d["ny"])
            got = e.field(k)
            assert np.max(np.abs(got - ref)) <= 2.0 ** -46 * np.max(np.abs(ref))  # plain FP32: 2^-24
            assert not np.array_equal(got, ref.astype(np.float32).astype(np.float64))
        x = np.ascontiguousarray(wl.random_field(d["ny"], d["nx"], 3, amplitude=0.7, mean=0.05))
        e.set_field(1, x)
        assert np.max(np.abs(e.field(1) - x)) <= 2.0 ** -46
    # below the threshold the FP32 field is plain FP32
    with ens(d["nx"], d["ny"], [0.2], 0.01, 1e-3, d["L"], prec=ch.CH_FP32) as e:
        ref = orc.initial_field(d["nx"], d["ny"], 0.2, SEED, 0)
        assert np.array_equal(e.field(0), ref.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("tuning", [dict(), dict(split=0, col_seg=-1), dict(split=1, stream=1)],
                         ids=["segment", "panels", "streaming"])
def test_fp32_compensated_run_matches_oracle(orc, tuning):
    d = COMP
    C0 = orc.initial_field(d["nx"], d["ny"], 0.3, SEED, 0)
    nsteps = 200
    ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps, every=20)
    with ens(d["nx"], d["ny"], [0.3], d["gamma"], d["dt"], d["L"], prec=ch.CH_FP32) as e:
        e.set_tuning(**tuning)
        e.set_sampling(20, 0.0, capacity=16)
        e.step(nsteps)
        err = np.max(np.abs(e.field(0) - ref.C))
        ser = e.series(0, 16)
    assert err <= 1e-4, err
    np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-5)
    np.testing.assert_allclose(ser[:, 2], ref.series[:, 2], rtol=1e-3)


def test_fp32_compensated_checkpoint(tmp_path):
    d = COMP
    path = str(tmp_path / "ck32.bin")
    with ens(d["nx"], d["ny"], [0.0, 0.3], d["gamma"], d["dt"], d["L"], prec=ch.CH_FP32) as e:
        e.step(30)
        e.save(path)
        e.step(20)
        a = [e.field(k) for k in range(2)]
        e.load(path)
        e.step(20)
        for k in range(2):
            assert np.array_equal(a[k], e.field(k))


# ------------------------------------------------------------------------------------------
# Observables on their own; non-finite detection
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
def test_observables_of_current_field(orc, prec):
    nx, ny, L, gamma, dt = 40, 56, 3.0, 0.02, 1e-3
    with ens(nx, ny, [0.1, -0.3], gamma, dt, L, prec=prec) as e:
        e.step(37)
        F, D, B = e.observables()
        for k in range(2):
            C = e.field(k)
            Fo, Do = orc.field_observables(C, L, gamma)
            t = 37 * dt
            # FP64 reductions of the FP64 functional of the stored field in both forms
            rt = 1e-11
            assert abs(F[k] - Fo) <= 1e-12 * abs(Fo)
            assert abs(D[k] - Do) <= rt * abs(Do)
            assert abs(B[k] - (-(t / Fo) * Do)) <= rt * abs(B[k])


def test_nonfinite_run_is_reported():
    with ens(16, 16, [0.0]) as e:
        e.set_field(0, np.full((16, 16), 1e120) * np.cos(np.arange(256)).reshape(16, 16))
        e.step(3)
        with pytest.raises(ch.ChError) as exc:
            e.observables()
        assert exc.value.code == ch.CH_ENONFINITE


# ------------------------------------------------------------------------------------------
# Determinism, graph replay, alone vs in the mix, reset, checkpoint/resume
# ------------------------------------------------------------------------------------------
def test_graph_replay_equals_single_launches():
    with ens(64, 48, [0.0, 0.4]) as a, ens(64, 48, [0.0, 0.4]) as b:
        a.step(16 * 3 + 5)
        for _ in range(16 * 3 + 5):
            b.step(1)
        for k in range(2):
            assert np.array_equal(a.field(k), b.field(k))


def test_member_alone_equals_member_in_mix():
    d = dict(nx=64, ny=64, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.4, seed=77, counter_base=0)
    others = [dict(nx=n, ny=n, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0, seed=5 + n, counter_base=0)
              for n in (32, 128, 17)]
    with ch.Ensemble.batch([d]) as alone, ch.Ensemble.batch(others[:2] + [d] + others[2:]) as mix:
        alone.step(120)
        mix.step(120)
        assert np.array_equal(alone.field(0), mix.field(2))


def test_reset_reproduces_run():
    with ens(32, 32, [0.2]) as e:
        e.step(40)
        a = e.field(0)
        e.reset()
        assert e.step_index(0) == 0
        e.step(40)
        assert np.array_equal(a, e.field(0))


def test_checkpoint_resume_bit_exact(tmp_path):
    path = str(tmp_path / "ck.bin")
    with ens(32, 40, [0.0, 0.3]) as e:
        e.set_sampling(5, 0.01, capacity=64)
        e.step(30)
        e.save(path)
        e.step(25)
        a = [e.field(k) for k in range(2)]
        sa = e.series(1, 64)
        e.load(path)
        assert e.step_index(1) == 30
        e.step(25)
        for k in range(2):
            assert np.array_equal(a[k], e.field(k))
        assert np.array_equal(sa, e.series(1, 64))


def test_zero_steps_and_argument_errors():
    with ens(8, 8, [0.0]) as e:
        before = e.field(0)
        e.step(0)
        assert np.array_equal(before, e.field(0))
        with pytest.raises(ch.ChError):
            e.step(-1)
        with pytest.raises(ch.ChError):
            e.field(3)
        with pytest.raises(ch.ChError):
            e.set_field(0, np.full((8, 8), np.nan))
        with pytest.raises(ch.ChError):
            e.set_sampling(0)


def test_runs_on_a_torch_stream():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    with ens(32, 32, [0.0]) as a, ens(32, 32, [0.0]) as b:
        b.set_stream(s.cuda_stream)
        a.step(40)
        b.step(40)
        b.synchronize()
        assert np.array_equal(a.field(0), b.field(0))


# ------------------------------------------------------------------------------------------
# Full-size workloads in the benchmark's launch configuration, sampled members
# ------------------------------------------------------------------------------------------
def test_ensemble_256_full_size_sampled_members(orc):
    p = wl.ENSEMBLE_256
    nsteps = 200
    with ens(p["nx"], p["ny"], p["C0"], p["gamma"], p["dt"], p["L"]) as e:
        e.set_sampling(p["every"], p["t1"], capacity=4)
        e.step(nsteps)
        F, D, B = e.observables()
        for k in (0, 200):
            C0 = orc.initial_field(p["nx"], p["ny"], p["C0"][k], SEED, k * p["nx"] * p["ny"])
            ref = orc.run(C0, p["L"], p["gamma"], p["dt"], nsteps)
            err = np.max(np.abs(e.field(k) - ref.C))
            print("member %d max|dC| %.3e" % (k, err))
            assert err <= 1e-11
            Fo, Do = orc.field_observables(ref.C, p["L"], p["gamma"])
            assert abs(F[k] - Fo) <= 1e-11 * abs(Fo)
        # properties of every member: mass conserved, F decreased
        for k in range(0, 256, 51):
            C = e.field(k)
            C0 = orc.initial_field(p["nx"], p["ny"], p["C0"][k], SEED, k * p["nx"] * p["ny"])
            assert abs(C.sum() - C0.sum()) <= 1e-9


def test_ensemble_256_fp32_full_size_sampled_members(orc):
    # the FP32 leg of the benchmark: default kernel classes (the cluster-resident form)
    p = wl.ENSEMBLE_256
    nsteps = 200
    with ens(p["nx"], p["ny"], p["C0"], p["gamma"], p["dt"], p["L"], prec=ch.CH_FP32) as e:
        t = e.tuning()
        assert t["resident"] == 1
        e.set_sampling(p["every"], p["t1"], capacity=4)
        e.step(nsteps)
        F, D, B = e.observables()
        s = p["gamma"] * p["dt"] / (p["L"] / p["nx"]) ** 4
        for k in (3, 255):
            C0 = orc.initial_field(p["nx"], p["ny"], p["C0"][k], SEED, k * p["nx"] * p["ny"])
            C1 = C0.copy()
            orc.step(C1, p["L"], p["gamma"], p["dt"])
            ref = orc.run(C0, p["L"], p["gamma"], p["dt"], nsteps)
            # at s = 13.8 the FP32 step's error is up to 2 u (1 + 16 s) of the step (see
            # test_fp32_single_step_error_grows_with_s); bound: that of the first (largest)
            # step, accumulated over the run
            bound = nsteps * 2 * 2.0 ** -24 * (1 + 16 * s) * np.max(np.abs(C1 - C0))
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= bound, (err, bound)
            Fo, Do = orc.field_observables(ref.C, p["L"], p["gamma"])
            assert abs(F[k] - Fo) <= 1e-5 * abs(Fo)


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
def test_uneven_full_size_sampled_members(orc, prec):
    # 64 x 128^2 + 32 x 256^2 + 8 x 512^2 in one batch (the benchmark's uneven leg)
    descs = wl.uneven_members()
    nsteps = 20
    with ch.Ensemble.batch(descs, prec) as e:
        if prec == ch.CH_FP64:
            e.set_tuning(split=0)  # the fused segment forms the benchmark uses for this batch
        e.step(nsteps)
        for k in (0, 95, 103):  # a 128^2, a 256^2 and a 512^2 member (FP32: compensated, s = 220)
            d = descs[k]
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps)
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= (1e-12 if prec == ch.CH_FP64 else 1e-4), (k, err)


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
def test_long_1024_full_size_sampled_members(orc, prec):
    # 32 x 1024^2, gamma 0.0025, dt 5e-4 (s = 882): two members against the oracle
    lb = wl.LONG_1024
    descs = [dict(nx=lb["nx"], ny=lb["ny"], L=lb["L"], gamma=lb["gamma"], dt=lb["dt"], C0=c0, seed=SEED,
                  counter_base=k * lb["nx"] * lb["ny"]) for k, c0 in enumerate(lb["C0"])]
    nsteps = 10
    with ch.Ensemble.batch(descs, prec) as e:
        e.step(nsteps)
        for k in (0, 31):
            d = descs[k]
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps)
            err = np.max(np.abs(e.field(k) - ref.C))
            # FP64: single-step round-off times cond(I + s D^4) <= 1 + 16 s per direction
            assert err <= (1e-10 if prec == ch.CH_FP64 else 1e-4), (k, err)


# ------------------------------------------------------------------------------------------
# Every launch shape gives the oracle's result (tuning changes only the round-off order)
# ------------------------------------------------------------------------------------------
TUNINGS = [
    dict(split=0), dict(split=1), dict(split=1, rows_band=3, sweep_band=5, cols_panel=7, cols_p=1),
    dict(split=0, rows_band=8, rows_p=4, cols_panel=16, cols_p=4, threads=128),
    dict(split=1, rows_band=32, sweep_band=64, cols_panel=64, cols_p=2, threads=512),
    dict(split=0, rows_band=2, rows_p=1, cols_panel=8, cols_p=8, threads=64),
    dict(split=1, stream=1), dict(split=1, stream=1, rows_band=4, threads=128),
    dict(split=1, stream=0, sweep_band=32, cols_panel=32, cols_p=1),
    dict(split=0, persist=1, cols_panel=8, cols_p=2, threads=128), dict(split=0, persist=0, rows_p=1, cols_p=1),
    dict(split=1, stream=0, persist=1, cols_panel=16, cols_p=1, threads=256),
    dict(split=0, rows_band=64, rows_p=2, cols_panel=32, cols_p=4, threads=128),
]


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
@pytest.mark.parametrize("tuning", TUNINGS, ids=[str(i) for i in range(len(TUNINGS))])
def test_every_tuning_matches_oracle(orc, prec, tuning):
    descs = []
    base = 0
    extra = [dict(nx=96, ny=80, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.2),
             dict(nx=8, ny=100, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.1),
             dict(nx=100, ny=12, L=TWO_PI, gamma=0.005, dt=1e-3, C0=-0.1)]
    for k, d in enumerate(UNEVEN_SMALL[:4] + extra):
        descs.append(dict(d, seed=SEED + 7 * k, counter_base=base))
        base += d["nx"] * d["ny"]
    nsteps = 40
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_tuning(**tuning)
        e.set_sampling(10, 0.0, capacity=8)
        e.step(nsteps)
        F, D, B = e.observables()
        for k, d in enumerate(descs):
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps, every=10)
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= (1e-12 if prec == ch.CH_FP64 else 1e-4), (k, err)
            ser = e.series(k, 8)
            np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-11 if prec == ch.CH_FP64 else 1e-5)


# Members whose rows split into a power of two <= 32 of segments (16 or 32 points): the
# segment form of the fused row sweep, incl. one lane per row (nx = S), a long pre-roll
# (K > nx), ragged bands and groups that share a warp.
SEG_MEMBERS = [
    dict(nx=16, ny=9, L=1.0, gamma=0.002, dt=1e-3, C0=0.3),       # G = 1 (S = 16); s large
    dict(nx=32, ny=37, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.4),
    dict(nx=64, ny=48, L=TWO_PI, gamma=0.005, dt=1e-3, C0=-0.2),
    dict(nx=128, ny=20, L=4.0, gamma=0.02, dt=5e-4, C0=0.1),
    dict(nx=256, ny=7, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0),
    dict(nx=512, ny=12, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.25),  # s = 220, G = 32 (S = 16)
]
SEG_TUNINGS = [dict(split=0, row_seg=0), dict(split=0, row_seg=16, rows_band=3, threads=64),
               dict(split=0, row_seg=32, rows_band=16, threads=256, persist=0),
               dict(split=0, row_seg=16, rows_band=1, threads=512, cols_panel=8, cols_p=2, persist=2),
               dict(split=0, row_seg=16, rows_band=5, threads=128, persist=3),
               dict(split=0, row_seg=1), dict(split=0, row_seg=1, col_seg=-1, threads=64),
               dict(split=1, row_seg=16), dict(split=1, stream=0, row_seg=32, threads=128)]


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
@pytest.mark.parametrize("tuning", SEG_TUNINGS, ids=[str(i) for i in range(len(SEG_TUNINGS))])
def test_segment_row_sweep_matches_oracle(orc, prec, tuning):
    descs, base = [], 0
    members = SEG_MEMBERS if tuning.get("row_seg") in (0, 16) else SEG_MEMBERS[1:]  # nx = 16 < S, not 32 nw
    for k, d in enumerate(members):
        descs.append(dict(d, seed=SEED + 11 * k, counter_base=base))
        base += d["nx"] * d["ny"]
    nsteps = 40
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_tuning(**tuning)
        t = e.tuning()
        assert t["row_seg"] == (tuning["row_seg"] or 16)
        e.set_sampling(10, 0.0, capacity=8)
        # the row phase alone: W of the segment sweep against the oracle's row solves
        for k, d in enumerate(descs):
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            hx, hy = d["L"] / d["nx"], d["L"] / d["ny"]
            _, R = orc.rhs(C0, hx, hy, d["gamma"], d["dt"])
            sx = d["gamma"] * d["dt"] / hx ** 4
            Wref = np.stack([orc.penta_solve(sx, R[j]) for j in range(d["ny"])])
            Wgot = e.row_solve(k)
            # ||A^-1|| <= 1: rounding of R (relative to its largest value) bounds the error
            tol = 1e-13 if prec == ch.CH_FP64 else 2e-6
            assert np.max(np.abs(Wgot - Wref)) <= tol * np.max(np.abs(R)), k
        e.step(nsteps)
        for k, d in enumerate(descs):
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps, every=10)
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= (1e-12 if prec == ch.CH_FP64 else 1e-4), (k, err)
            ser = e.series(k, 8)
            np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-11 if prec == ch.CH_FP64 else 1e-5)
            np.testing.assert_allclose(ser[:, 2], ref.series[:, 2], rtol=1e-9 if prec == ch.CH_FP64 else 1e-3)


# Members whose columns split into a power of two of 16- or 32-row segments: the segment
# form of the column kernel, incl. one segment per column (ny = S), partial column tiles
# (nx not a multiple of 32), several panels per CTA and s large.
COLSEG_MEMBERS = [
    dict(nx=33, ny=32, L=1.0, gamma=0.002, dt=1e-3, C0=0.3),
    dict(nx=100, ny=64, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.4),
    dict(nx=7, ny=128, L=TWO_PI, gamma=0.005, dt=1e-3, C0=-0.2),
    dict(nx=64, ny=256, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0),
    dict(nx=48, ny=16, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.1),   # S = 32 does not fit
]
COLSEG_TUNINGS = [dict(split=0, col_seg=16), dict(split=0, col_seg=16, row_seg=-1, threads=128),
                  dict(split=1, stream=1, col_seg=16), dict(split=0, col_seg=32)]


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
@pytest.mark.parametrize("tuning", COLSEG_TUNINGS, ids=[str(i) for i in range(len(COLSEG_TUNINGS))])
def test_segment_column_kernel_matches_oracle(orc, prec, tuning):
    members = COLSEG_MEMBERS if tuning["col_seg"] == 16 else COLSEG_MEMBERS[:4]
    descs, base = [], 0
    for k, d in enumerate(members):
        descs.append(dict(d, seed=SEED + 13 * k, counter_base=base))
        base += d["nx"] * d["ny"]
    nsteps = 40
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_tuning(**tuning)
        assert e.tuning()["col_seg"] == tuning["col_seg"]
        e.set_sampling(10, 0.0, capacity=8)
        e.step(nsteps)
        for k, d in enumerate(descs):
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps, every=10)
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= (1e-12 if prec == ch.CH_FP64 else 1e-4), (k, err)
            ser = e.series(k, 8)
            np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-11 if prec == ch.CH_FP64 else 1e-5)
            assert e.step_index(k) == nsteps


def test_segment_column_selection_and_errors():
    d = dict(L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0, seed=1)
    with ch.Ensemble.batch([dict(d, nx=64, ny=64, counter_base=0), dict(d, nx=32, ny=1024, counter_base=4096)],
                           ch.CH_FP32) as e:
        assert e.tuning()["col_seg"] == 32  # 1024 = 32 x 32
        e.set_tuning(col_seg=16)  # 1024 / 16 = 64 segments: over a CTA pair
        assert e.tuning()["col_seg"] == 16
        e.step(2)
        with pytest.raises(ch.ChError) as err:
            e.set_tuning(col_seg=8)  # S is 16 or 32
        assert err.value.code == ch.CH_EINVAL
    with ch.Ensemble.batch([dict(d, nx=64, ny=1024, counter_base=0)], ch.CH_FP64) as e:
        assert e.tuning()["col_seg"] == -1  # FP64 default: streaming columns
        e.set_tuning(split=0)
        assert e.tuning()["col_seg"] == 32  # 32 segments of doubles: over a CTA pair
        with pytest.raises(ch.ChError):
            e.set_tuning(col_seg=16)  # 64 segments of doubles: above the pair limit of 32
        e.set_tuning(split=1, col_seg=-1)
    with ens(64, 100, [0.0], prec=ch.CH_FP32) as e:
        assert e.tuning()["col_seg"] == -1  # 100 rows: no power of two of segments


@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
def test_segment_columns_over_cta_pairs_match_oracle(orc, prec):
    # columns taller than one CTA holds: FP64 1024 rows (32 segments of 32), FP32 2048 rows
    # (64 segments), split over the two CTAs of a cluster; a short member beside them
    ny = 1024 if prec == ch.CH_FP64 else 2048
    # L = 8 pi (FP64) / 16 pi (FP32) keeps s_y moderate (14 and 3.5) for the FP32 bound
    d = dict(L=4 * TWO_PI if prec == ch.CH_FP64 else 8 * TWO_PI, gamma=0.005, dt=1e-3, seed=SEED)
    descs = [dict(d, nx=40, ny=ny, C0=0.2, counter_base=0), dict(d, nx=33, ny=ny, C0=-0.1, counter_base=40 * ny),
             dict(d, nx=64, ny=64, C0=0.3, counter_base=73 * ny)]
    nsteps = 6
    with ch.Ensemble.batch(descs, prec) as e:
        e.set_tuning(split=0, col_seg=32)
        e.set_sampling(3, 0.0, capacity=4)
        e.step(nsteps)
        for k, dd in enumerate(descs):
            C0 = orc.initial_field(dd["nx"], dd["ny"], dd["C0"], dd["seed"], dd["counter_base"])
            ref = orc.run(C0, dd["L"], dd["gamma"], dd["dt"], nsteps, every=3)
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= (1e-10 if prec == ch.CH_FP64 else 1e-4), (k, err)
            np.testing.assert_allclose(e.series(k, 4)[:, 1], ref.series[:, 1],
                                       rtol=1e-11 if prec == ch.CH_FP64 else 1e-5)


def test_segment_form_selection_and_errors():
    with ch.Ensemble.batch([dict(nx=64, ny=16, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0, seed=1, counter_base=0),
                            dict(nx=1024, ny=8, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.0, seed=1,
                                 counter_base=1024)], ch.CH_FP32) as e:
        # classes are per member: member 0 (nx = 64) takes the segment form with S = 16,
        # member 1 (1024 = 32 x 32) S = 32
        assert e.tuning()["row_seg"] == 16
        with pytest.raises(ch.ChError) as err:
            e.set_tuning(row_seg=16)  # forced for every member: 1024 / 16 = 64 lanes is too many
        assert err.value.code == ch.CH_EINVAL
        with pytest.raises(ch.ChError):
            e.set_tuning(row_seg=1)  # 1024 = 32 x 32 warps: more than 16
        assert e.tuning()["row_seg"] == 16
        e.set_tuning(row_seg=32)
        assert e.tuning()["row_seg"] == 32
        with pytest.raises(ch.ChError):
            e.set_tuning(row_seg=8)
        e.set_tuning(row_seg=-1)
        assert e.tuning()["row_seg"] == -1
    with ens(100, 16, [0.0], prec=ch.CH_FP32) as e:
        assert e.tuning()["row_seg"] == -1  # 100 is no power of two of segments: chunked sweep
    with ens(64, 16, [0.0]) as e:
        assert e.tuning()["row_seg"] == 0  # FP64 default: split form


def test_tuning_round_trip_and_errors():
    with ens(64, 48, [0.0]) as e:
        e.set_tuning(split=1, rows_band=8, sweep_band=16, cols_panel=16, cols_p=1, threads=128, stream=0)
        t = e.tuning()
        assert t["split"] == 1 and t["rows_band"] == 8 and t["sweep_band"] == 16 and t["cols_panel"] == 16
        assert t["stream"] == 0 and t["threads"] == 128
        with pytest.raises(ch.ChError):
            e.set_tuning(cols_panel=64, cols_p=16, threads=128)
        with pytest.raises(ch.ChError):
            e.set_tuning(threads=100)
        assert e.tuning()["rows_band"] == 8  # a rejected request keeps the shape in effect
        ch.ch_set_tuning(e.h)  # defaults
        e.step(3)


# ------------------------------------------------------------------------------------------
# FP32 form at large s: one step from a random field against the oracle.  The factorised
# solve's condition number is 1 + 16 s per direction, so the FP32 step's error relative to
# the step grows like the unit round-off times s (both column kernels)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [256, 512, 1024])
@pytest.mark.parametrize("col_seg", [-1, 0])
def test_fp32_single_step_error_grows_with_s(orc, n, col_seg):
    L, gamma, dt = TWO_PI, 0.005, 1e-3
    h = L / n
    s = gamma * dt / h ** 4
    # the FP32 form holds the field rounded to FP32: the oracle steps the same values
    C = np.ascontiguousarray(wl.random_field(n, n, 7, amplitude=0.1, mean=0.3)).astype(np.float32).astype(np.float64)
    ref = C.copy()
    orc.step(ref, L, gamma, dt)
    dref = ref - C
    with ens(n, n, [0.0], gamma, dt, L, prec=ch.CH_FP32) as e:
        e.set_tuning(split=0, col_seg=col_seg)
        e.set_field(0, C)
        e.step(1)
        got = e.field(0)
    err = np.max(np.abs((got - C) - dref))
    # solve: 2 u (1 + 16 s) of the step; storing C + dC in FP32: u max|C|
    bound = 2 * 2.0 ** -24 * (1 + 16 * s) * np.max(np.abs(dref)) + 2.0 ** -24 * np.max(np.abs(ref))
    assert err <= bound, (err, bound)


# ------------------------------------------------------------------------------------------
# The factorised scheme at fine grids: grid-scale diagonal modes decay only by ~1/(4s)
# per step (s = gamma dt / h^4), the closed-form amplification factor of the scheme
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [ch.CH_FP64, ch.CH_FP32])
def test_fine_grid_nyquist_mode_decays_as_the_scheme_says(prec):
    n, L, gamma, dt, C0, eps, nsteps = 1024, TWO_PI, 0.005, 1e-3, 0.3, 0.05, 20
    h = L / n
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    phi = np.where((i + j) % 2 == 0, 1.0, -1.0)  # cos(pi i + pi j): the diagonal Nyquist mode
    sigma, d = gamma * dt, 3 * C0 * C0 - 1
    a = 4 / h ** 2
    A = 2 * a
    G = 1 - dt * (A * d + gamma * A * A) / (1 + sigma * a * a) ** 2
    assert 1 - G < 1e-4  # s = 3520: the mode barely decays
    with ens(n, n, [0.0], gamma, dt, L, prec=prec) as e:
        e.set_field(0, C0 + eps * phi)
        e.step(nsteps)
        got = e.field(0)
    amp = np.sum((got - C0) * phi) / phi.size
    # phi^2 = 1 and phi^3 = phi: the mode's amplitude follows a scalar recursion exactly
    want = eps
    for _ in range(nsteps):
        want -= dt * (A * (d * want + want ** 3) + gamma * A * A * want) / (1 + sigma * a * a) ** 2
    tol = 1e-11 if prec == ch.CH_FP64 else 2e-5
    assert abs(amp - want) <= tol * abs(want), (amp, want)
    assert abs(eps - amp) > 0.5 * abs(eps - want)  # the decay itself, not only the amplitude
    # away from the mode: rounding in R', which the operator passes to the smooth modes with
    # gain up to (1 + 16 s)^2 ~ 3e9 relative to this one; the oracle's own deviation here
    # is 7e-13 (FP64).  FP32: once rounding breaks the pattern's symmetry, the rounding of
    # R' (unit round-off of its largest value, |R'| = 8 |mu_1|, mu_1 = 8 gamma eps / h^2)
    # reaches the smooth modes with gain up to dt / h^2 per step: a worst-case bound.
    if prec == ch.CH_FP64:
        bound = 2e-12
    else:
        bound = nsteps * (dt / h ** 2) * 2.0 ** -24 * 8 * (8 * gamma * eps / h ** 2)
    assert np.max(np.abs(got - C0 - amp * phi)) <= bound


# ------------------------------------------------------------------------------------------
# FP64 split form: rows too long for a shared-memory band run the stencil in blocks of
# rows x 256 columns (stencil_block_kernel)
# ------------------------------------------------------------------------------------------
# h_x = 0.1 on the long members (s_x = 0.1, 0.05): the standard FP64 bars apply
LONG_ROWS = [dict(nx=4096, ny=24, L=409.6, gamma=0.01, dt=1e-3, C0=0.1),
             dict(nx=8192, ny=10, L=819.2, gamma=0.005, dt=1e-3, C0=-0.2),
             dict(nx=1000, ny=17, L=100.0, gamma=0.01, dt=1e-3, C0=0.3),    # ragged last block
             dict(nx=64, ny=64, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.0)]     # whole rows, same launch
# the same width on [0, 2 pi): s_x = 1.8e6, where the bars follow from the conditioning
LONG_ROWS_STIFF = [dict(nx=4096, ny=24, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.1),
                   dict(nx=64, ny=64, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.0)]


@pytest.mark.parametrize("members", [LONG_ROWS, LONG_ROWS_STIFF], ids=["moderate_s", "stiff"])
def test_long_rows_match_oracle(orc, members):
    descs, base = [], 0
    for k, d in enumerate(members):
        descs.append(dict(d, seed=SEED + 11 * k, counter_base=base))
        base += d["nx"] * d["ny"]
    nsteps = 12
    with ch.Ensemble.batch(descs, ch.CH_FP64) as e:
        assert e.tuning()["split"] == 1
        e.set_sampling(4, 0.0, capacity=8)
        e.step(nsteps)
        F, D, _ = e.observables()  # of the current fields (observe mode of both stencil forms)
        for k, d in enumerate(descs):
            Fo, Do = orc.field_observables(e.field(k), d["L"], d["gamma"])
            assert abs(F[k] - Fo) <= 1e-12 * abs(Fo), (k, F[k], Fo)
            if d["gamma"] * d["dt"] / min(d["L"] / d["nx"], d["L"] / d["ny"]) ** 4 < 1e3:
                assert abs(D[k] - Do) <= 1e-9 * abs(Do), (k, D[k], Do)
            C0 = orc.initial_field(d["nx"], d["ny"], d["C0"], d["seed"], d["counter_base"])
            ref = orc.run(C0, d["L"], d["gamma"], d["dt"], nsteps, every=4)
            # round-off bound: each side's step is backward stable for the factorised
            # operator, whose condition number is at most 1 + 16 s per axis, so a step adds
            # at most ~2 u (1 + 16 s_max) max|dC| (s_x = 1.8e6 for the 4096-wide member)
            s_max = d["gamma"] * d["dt"] / min(d["L"] / d["nx"], d["L"] / d["ny"]) ** 4
            C, inc = C0.copy(), 0.0
            for _ in range(nsteps):
                prev = C.copy()
                orc.step(C, d["L"], d["gamma"], d["dt"])
                inc += np.max(np.abs(C - prev))
            tol = max(1e-12, 2 * 2 * 2.0 ** -53 * (1 + 16 * s_max) * inc)
            err = np.max(np.abs(e.field(k) - ref.C))
            assert err <= tol, (k, err, tol)
            if s_max < 1e3:
                assert err <= 1e-12, (k, err)
            ser = e.series(k, 8)
            assert np.array_equal(ser[:, 0], ref.series[:, 0])
            np.testing.assert_allclose(ser[:, 1], ref.series[:, 1], rtol=1e-11)
            if s_max < 1e3:
                # dF/dt = -h^2 sum |D+ mu|^2 with mu containing gamma lap_h C: at s_x ~ 1e6 the
                # field's round-off above reaches it amplified by gamma / h^2, so only the
                # moderate-s members are held to the 1e-9 series bar
                np.testing.assert_allclose(ser[:, 2], ref.series[:, 2], rtol=1e-9)


def test_stencil_blocks_equal_whole_rows():
    """A band taller than the shared memory holds for whole rows switches the member to the
    block stencil; mu and R' are formed in the same operation order, so the fields equal the
    whole-row kernel's bit for bit (observables: the same sums grouped by block)."""
    d = dict(nx=512, ny=70, L=TWO_PI, gamma=0.01, dt=1e-3, C0=0.2, seed=SEED, counter_base=0)
    out = []
    for band in (16, 64):  # 16: whole rows fit (155 KB); 64: block form
        with ch.Ensemble.batch([d], ch.CH_FP64) as e:
            e.set_tuning(split=1, rows_band=band)
            e.set_sampling(5, 0.0, capacity=8)
            e.step(30)
            out.append((e.field(0), e.series(0, 8), e.observables()))
    assert np.array_equal(out[0][0], out[1][0])
    for q in range(2):
        np.testing.assert_allclose(out[1][2][q], out[0][2][q], rtol=1e-12)
    np.testing.assert_allclose(out[1][1][:, 1], out[0][1][:, 1], rtol=1e-13)
    np.testing.assert_allclose(out[1][1][:, 2], out[0][1][:, 2], rtol=1e-12)
