"""Ensemble statistics of beta on the GPU (ch_stats_* and ch_ensemble_*) against the oracle.

The statistics are those of Sec. 3.3 Eqs. (41a,b) and (42) (moments across the runs per
sample time, the window mean of mu_1, the slope k of mu_2 = k t) and the histogram form
of p_beta(b, t), Sec. 1 Eq. (7).

Bars.  On the same inputs: histogram counts and value counts bit for bit (both sides
take the bin decision with the same FP64 division); moments within the rounding bound
of two FP64 summation orders (derived per sample below).  Over a run's own series (GPU
run against oracle run, each from its own fields): moments and trend within the bound
that the FP64 beta agreement implies, histogram counts equal except for values within
that agreement of a bin edge.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
SEED = wl.BASE_SEED


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def orc():
    return get_oracle()


@pytest.fixture(scope="module")
def torch():
    import torch

    assert torch.cuda.is_available()
    return torch


def dev(torch, a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dtype)


def gpu_moments(torch, t, beta, ld=None):
    M, T = beta.shape
    ld = T if ld is None else ld
    b = np.full((M, ld), 7.0)
    b[:, :T] = beta
    tb, bb = dev(torch, t), dev(torch, b)
    out = torch.full((max(T, 1), ch.CH_MOMENTS), -1.0, dtype=torch.float64, device="cuda")
    ch.ch_stats_moments(tb.data_ptr(), bb.data_ptr(), M, T, ld, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()[:T]


def gpu_histogram(torch, beta, lo, hi, nbins):
    M, T = beta.shape
    bb = dev(torch, beta)
    out = torch.full((max(T, 1), nbins + 2), -1, dtype=torch.int64, device="cuda")
    ch.ch_stats_histogram(bb.data_ptr(), M, T, T, lo, hi, nbins, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()[:T]


def moment_tolerance(beta, ref):
    """Per sample and p = 1..4, twice the bound on one side's rounding error.  With c finite
    values, the mean carries at most delta = (c + 1) u max|beta|; each (beta - mean)^p term
    then moves by p |d|^(p-1) delta + (p + 1) u |d|^p, and a sum of c terms adds c u times
    the sum of magnitudes."""
    T = beta.shape[1]
    tol = np.zeros((T, 5))
    for s in range(T):
        v = beta[:, s][np.isfinite(beta[:, s])]
        c = v.size
        if c == 0:
            continue
        d = np.abs(v - ref[s, 1])
        delta = (c + 1) * U * np.max(np.abs(v))
        tol[s, 1] = 2 * delta
        for p in (2, 3, 4):
            A = np.mean(d ** p)
            B = np.mean((d + delta) ** (p - 1))
            tol[s, p] = 2 * ((c + p + 2) * U * A + p * delta * B) + 1e-300
    return tol


def check_moments(got, t, ref, tol):
    T = ref.shape[0]
    assert got.shape == (T, ch.CH_MOMENTS)
    assert np.array_equal(got[:, 0], t)
    assert np.array_equal(got[:, 1], ref[:, 0])
    for s in range(T):
        if ref[s, 0] == 0:
            assert np.all(np.isnan(got[s, 2:]))
            continue
        for p in range(1, 5):
            err = abs(got[s, p + 1] - ref[s, p])
            assert err <= tol[s, p], "sample %d mu_%d: %r vs %r (tol %g)" % (s, p, got[s, p + 1], ref[s, p], tol[s, p])


# ------------------------------------------------------------------------------------------
# Dense forms on seeded synthetic ensembles (the same inputs on both sides)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("M,T", [(1003, 777), (1, 5), (8, 32), (257, 33), (4096, 64)])
def test_dense_moments_match_oracle(torch, orc, M, T):
    t, beta = wl.beta_ensemble(M, T, seed=SEED + M, diverged=min(5, M - 1))
    if T > 3 and M > 2:
        beta[0, 1] = np.inf
        beta[1, 1] = -np.inf
        beta[:, 3] = np.nan  # every run diverged at one sample
    ref = orc.beta_moments(beta)
    got = gpu_moments(torch, t, beta, ld=T + 3)
    check_moments(got, t, ref, moment_tolerance(beta, ref))
    if M == 1:
        assert np.all(got[:, 3:] == 0.0)


def test_dense_moments_shift_and_scale(torch):
    """An affine map a beta + c moves mu_1 to a mu_1 + c and scales mu_p by a^p (to
    rounding): a structural check independent of the oracle."""
    t, beta = wl.beta_ensemble(300, 70, seed=SEED + 5)
    a, c = -0.5, 0.125  # exact in binary: the mapped inputs carry no extra rounding
    g0 = gpu_moments(torch, t, beta)
    g1 = gpu_moments(torch, t, a * beta + c)
    assert np.allclose(g1[:, 2], a * g0[:, 2] + c, rtol=0, atol=1e-14)
    for p in (2, 3, 4):
        assert np.allclose(g1[:, p + 1], a ** p * g0[:, p + 1], rtol=1e-12, atol=1e-15 * np.max(np.abs(g0[:, 3])) ** (p / 2))


def test_dense_empty_and_errors(torch):
    out = torch.zeros((1, ch.CH_MOMENTS), dtype=torch.float64, device="cuda")
    b = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    ch.ch_stats_moments(b.data_ptr(), b.data_ptr(), 4, 0, 4, out.data_ptr())  # no samples: nothing to do
    for args in [(4, 5, 4), (0, 4, 4), (4, -1, 4)]:  # ld < samples, no members, negative samples
        with pytest.raises(ch.ChError):
            ch.ch_stats_moments(b.data_ptr(), b.data_ptr(), *args, out.data_ptr())
    h = torch.zeros((4, 10), dtype=torch.int64, device="cuda")
    for lo, hi, nb in [(1.0, 1.0, 8), (0.0, math.inf, 8), (0.0, 1.0, 0), (0.0, 1.0, ch.CH_MAX_BINS + 1)]:
        with pytest.raises(ch.ChError):
            ch.ch_stats_histogram(b.data_ptr(), 4, 4, 4, lo, hi, nb, h.data_ptr())


@pytest.mark.parametrize("M,T,lo,hi,nbins", [(1003, 777, 0.1, 0.47, 50), (64, 40, -0.2, 0.9, ch.CH_MAX_BINS),
                                             (31, 97, 0.25, 0.3125, 1)])
def test_dense_histogram_bit_exact(torch, orc, M, T, lo, hi, nbins):
    t, beta = wl.beta_ensemble(M, T, seed=SEED + 11, diverged=3)
    w = (hi - lo) / nbins
    beta[:5, 2] = lo + w * np.arange(5)  # on (rounded) edges
    beta[5, 2], beta[6, 2] = lo, hi
    beta[7, 2] = np.inf
    ref = orc.beta_histogram(beta, lo, hi, nbins)
    got = gpu_histogram(torch, beta, lo, hi, nbins)
    assert np.array_equal(got, ref)
    assert np.array_equal(got.sum(axis=1), np.isfinite(beta).sum(axis=0))


def test_dense_trend_matches_oracle(torch, orc):
    """Trend statistics of a moments table built by the oracle from a synthetic ensemble
    whose spread grows like sqrt(k t) (so mu_2 ~ k t): same table on both sides."""
    t, beta = wl.beta_ensemble(512, 1001, seed=SEED + 21, t_end=100.0, k=0.0056)
    ref = orc.beta_moments(beta)
    table = np.zeros((t.size, ch.CH_MOMENTS))
    table[:, 0] = t
    table[:, 1:] = ref
    mt = dev(torch, table)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for (t1, t2, tf1, tf2) in [(20.0, 40.0, 0.0, 40.0), (20.0, 100.0, 20.0, 100.0), (19.95, 40.05, 0.0, 100.0),
                               (200.0, 300.0, 200.0, 300.0)]:
        ch.ch_stats_trend(mt.data_ptr(), t.size, t1, t2, tf1, tf2, out.data_ptr())
        torch.cuda.synchronize()
        g = out.cpu().numpy()
        want = orc.beta_trend(t, ref[:, 1], ref[:, 2], t1, t2, tf1, tf2)
        assert g[2] == want[2] and g[3] == want[3]
        if want[2] < 2:
            assert np.isnan(g[0]) and np.isnan(g[1])
            continue
        n = t.size
        assert abs(g[0] - want[0]) <= 4 * n * U * np.max(np.abs(ref[:, 1]))
        assert abs(g[1] - want[1]) <= 4 * n * U * abs(want[1])
    # the synthetic spread grows like k t with k = 0.0056: the fit finds it to sampling error
    ch.ch_stats_trend(mt.data_ptr(), t.size, 20.0, 40.0, 0.0, 100.0, out.data_ptr())
    torch.cuda.synchronize()
    assert abs(out.cpu().numpy()[1] - 0.0056) < 0.0056 * 0.1


# ------------------------------------------------------------------------------------------
# Over an ensemble's own series (ring buffers of the handle)
# ------------------------------------------------------------------------------------------
NX, NY, L, GAMMA, DT = 32, 32, 2 * math.pi, 0.02, 2e-3
C0S = [0.0, 0.1, -0.1, 0.2, 0.0, 0.3, -0.2, 0.05, 0.0, 0.15, -0.05, 0.25]
EVERY, STEPS, CAP = 5, 300, 40


@pytest.fixture(scope="module")
def runs(orc):
    """Oracle series of every member (all samples) and the GPU handle after the same steps."""
    series = []
    for k, c0 in enumerate(C0S):
        C = orc.initial_field(NX, NY, c0, SEED, k * NX * NY)
        series.append(orc.run(C, L, GAMMA, DT, STEPS, every=EVERY).series)
    return np.stack(series)  # (M, samples, 4)


def beta_tolerance(beta):
    """Agreement of the FP64 GPU beta with the oracle's after a few hundred steps (the
    FP64 field bar is 1e-11 after 1000 steps; beta carries its relative error, scaled
    by t / F and dF/dt): a priori 1e-9 relative to the largest |beta|."""
    return 1e-9 * max(np.max(np.abs(beta[np.isfinite(beta)])), 1e-3)


def perturbed_moment_tolerance(beta, ref, eps):
    """Moments of values each within eps of the oracle's: the mean moves by <= eps, each
    deviation d by <= 2 eps, so mu_p by <= p (2 eps) mean((|d| + 2 eps)^(p-1)); plus
    the rounding bound of moment_tolerance."""
    tol = moment_tolerance(beta, ref)
    for s in range(beta.shape[1]):
        v = beta[:, s][np.isfinite(beta[:, s])]
        if v.size == 0:
            continue
        d = np.abs(v - ref[s, 1])
        tol[s, 1] += eps
        for p in (2, 3, 4):
            tol[s, p] += p * 2 * eps * np.mean((d + 2 * eps) ** (p - 1))
    return tol


def held_window(total):
    """Sample numbers the ring still holds after `total` samples."""
    return max(0, total - CAP), total


def test_ensemble_statistics_match_oracle_runs(orc, runs):
    total = runs.shape[1]
    a, b = held_window(total)
    assert a > 0, "the ring must have wrapped"
    beta = runs[:, a:b, 3]
    t = runs[0, a:b, 0]
    eps = beta_tolerance(beta)
    with ch.Ensemble.create(NX, NY, L, GAMMA, DT, C0S, SEED, ch.CH_FP64) as e:
        e.set_sampling(EVERY, 0.0, CAP)
        e.step(STEPS)
        got = e.moments()
        ref = orc.beta_moments(beta)
        assert np.array_equal(got[:, 0], t)  # sample times bit for bit
        check_moments(got, t, ref, perturbed_moment_tolerance(beta, ref, eps))

        # a subset of members, in a given order
        sub = [7, 0, 3, 11]
        got_s = e.moments(members=sub)
        ref_s = orc.beta_moments(beta[sub])
        check_moments(got_s, t, ref_s, perturbed_moment_tolerance(beta[sub], ref_s, eps))

        # histogram: counts equal except for values within eps of an edge
        lo, hi, nb = float(np.min(beta[:, 1:])), float(np.max(beta)) * 0.9, 16
        gh = e.histogram(lo, hi, nb)
        rh = orc.beta_histogram(beta, lo, hi, nb)
        edges = lo + (hi - lo) / nb * np.arange(nb + 1)
        for s in range(beta.shape[1]):
            near = int(np.sum(np.min(np.abs(beta[:, s][:, None] - edges[None, :]), axis=1) <= 2 * eps))
            assert gh[s].sum() == rh[s].sum() == len(C0S)
            assert np.abs(gh[s] - rh[s]).sum() <= 2 * near, (s, gh[s], rh[s])

        # trend statistics
        tr = e.trend(t[5], t[-5], t[0], t[-1])
        want = orc.beta_trend(t, ref[:, 1], ref[:, 2], t[5], t[-5], t[0], t[-1])
        assert tr[2] == want[2] and tr[3] == want[3]
        tol1 = eps + 8 * len(t) * U * np.max(np.abs(ref[:, 1]))
        tol = perturbed_moment_tolerance(beta, ref, eps)
        assert abs(tr[0] - want[0]) <= tol1 + np.max(tol[:, 1])
        assert abs(tr[1] - want[1]) <= np.sum(t * tol[:, 2]) / np.sum(t * t) + 8 * len(t) * U * abs(want[1])


def test_ensemble_and_dense_forms_agree_bit_for_bit(torch):
    """The ring view and the dense view of the same samples run the same reductions in the
    same order: equal results to the bit (GPU series read back through ch_series)."""
    with ch.Ensemble.create(NX, NY, L, GAMMA, DT, C0S, SEED, ch.CH_FP64) as e:
        e.set_sampling(EVERY, 0.0, CAP)
        e.step(STEPS)
        ser = np.stack([e.series(k, CAP) for k in range(len(C0S))])
        got = e.moments()
        dense = gpu_moments(torch, ser[0, :, 0], ser[:, :, 3])
        assert np.array_equal(got, dense)
        gh = e.histogram(0.0, 0.5, 32)
        assert np.array_equal(gh, gpu_histogram(torch, ser[:, :, 3], 0.0, 0.5, 32))


def test_ensemble_fp32_statistics_consistent(torch):
    with ch.Ensemble.create(NX, NY, L, GAMMA, DT, C0S, SEED, ch.CH_FP32) as e:
        e.set_sampling(EVERY, 0.0, 1000)
        e.step(STEPS)
        ser = np.stack([e.series(k, 1000) for k in range(len(C0S))])
        got = e.moments()
        assert got.shape[0] == ser.shape[1] == STEPS // EVERY
        assert np.array_equal(got, gpu_moments(torch, ser[0, :, 0], ser[:, :, 3]))


def test_ensemble_statistics_edge_cases():
    with ch.Ensemble.create(NX, NY, L, GAMMA, DT, [0.0, 0.1], SEED, ch.CH_FP64) as e:
        with pytest.raises(ch.ChError):
            e.moments()  # no series kept
        e.set_sampling(EVERY, 0.0, 16)
        assert e.moments().shape == (0, ch.CH_MOMENTS)  # nothing sampled yet
        assert e.histogram(0.0, 1.0, 4).shape == (0, 6)
        m0, k0, nw, nf = e.trend(0.0, 1.0, 0.0, 1.0)
        assert nw == 0 and nf == 0 and math.isnan(m0) and math.isnan(k0)
        e.step(1)
        one = e.moments()
        assert one.shape == (1, ch.CH_MOMENTS) and one[0, 0] == 0.0 and one[0, 1] == 2
        assert one[0, 2] == 0.0 and one[0, 3] == 0.0  # beta = 0 at t = 0 for every run
        with pytest.raises(ch.ChError):
            e.moments(members=[0, 2])
        with pytest.raises(ch.ChError):
            e.moments(members=[])
        with pytest.raises(ch.ChError):
            e.histogram(1.0, 0.0, 4)
    descs = [dict(nx=32, ny=32, L=L, gamma=GAMMA, dt=DT, C0=0.0, seed=SEED, counter_base=0),
             dict(nx=32, ny=32, L=L, gamma=GAMMA, dt=2 * DT, C0=0.0, seed=SEED, counter_base=1024)]
    with ch.Ensemble.batch(descs, ch.CH_FP64) as e:
        e.set_sampling(EVERY, 0.0, 16)
        e.step(20)
        with pytest.raises(ch.ChError):
            e.moments()  # sampled at different times
        assert e.moments(members=[1]).shape == (4, ch.CH_MOMENTS)
