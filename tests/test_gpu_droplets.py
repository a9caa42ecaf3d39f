"""Model 1 droplet ensembles on the GPU (ch_droplets_run) against the oracle.

Bars.  Fixed steps: the same Dormand-Prince arithmetic on both sides, so radii and
samples agree to rounding (1e-12 relative) while no droplet goes extinct.  Adaptive steps:
the step sequence is not reproducible across summation orders -- near an extinction the
right-hand side -1/R^2 magnifies rounding, and the oracle itself takes 7841 instead of
7810 steps when h0 moves by one ulp -- so the adaptive runs are held to the integration
error the oracle shows at the same tolerance: four times its distance from a run at a
thousand times tighter tolerance, per population; live droplet counts agree exactly and
step counts within 5 %.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def orc():
    return get_oracle()


@pytest.mark.parametrize("M,N", [(3, 37), (2, 1), (1, 1500), (2, 3000)])  # 3000: global working arrays
def test_fixed_steps_match_oracle(orc, M, N):
    rng = np.random.default_rng(N)
    R0 = 0.5 + 0.5 * rng.random((M, N))  # no extinction before t = 0.05
    ts = np.linspace(0.0, 0.05, 6)
    R, ser, steps = ch.ch_droplets_run(R0, 0.05, ts, rtol=0.0, h0=1e-3)
    for m in range(M):
        Ro, so, acc, rej = orc.drop_run(R0[m], 0.05, ts, rtol=0.0, h0=1e-3)
        np.testing.assert_allclose(R[m], Ro, rtol=1e-12, atol=0)
        np.testing.assert_allclose(ser[m][:, :3], so[:, :3], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(ser[m][1:, 3], so[1:, 3], rtol=1e-10, atol=1e-14)
        assert np.array_equal(ser[m][:, 4], so[:, 4])
        assert steps[m, 0] == acc and steps[m, 1] == rej == 0 and steps[m, 2] == 0


def test_adaptive_with_extinctions_matches_oracle(orc):
    M, N = 4, 64
    R0 = wl.droplet_radii(M, N, seed=wl.BASE_SEED + 1)
    ts = np.linspace(0.0, 1.0, 11)
    R, ser, steps = ch.ch_droplets_run(R0, 1.0, ts, rtol=1e-6, atol=1e-9, h0=1e-6, eps=1e-3)
    for m in range(M):
        Ro, so, acc, rej = orc.drop_run(R0[m], 1.0, ts, rtol=1e-6, atol=1e-9, h0=1e-6, eps=1e-3)
        Rt, st, _, _ = orc.drop_run(R0[m], 1.0, ts, rtol=1e-9, atol=1e-12, h0=1e-6, eps=1e-3)
        assert steps[m, 2] == 0
        assert abs(steps[m, 0] - acc) <= 0.05 * acc and abs(steps[m, 1] - rej) <= 0.05 * rej, (steps[m], acc, rej)
        assert np.array_equal(ser[m][:, 4], so[:, 4])  # live droplets
        assert so[-1, 4] < N  # droplets went extinct on the way
        live = (Ro > 0) & (R[m] > 0)
        assert np.array_equal(Ro > 0, R[m] > 0)
        tol_r = 4 * np.max(np.abs(Ro - Rt)[live])
        assert np.max(np.abs(R[m] - Ro)[live]) <= tol_r
        tol_s = 4 * np.max(np.abs(so[:, 1:3] - st[:, 1:3]), axis=0)[None, :] + 1e-12 * np.abs(so[:, 1:3])
        assert np.all(np.abs(ser[m][:, 1:3] - so[:, 1:3]) <= tol_s), (ser[m][:, 1:3], so[:, 1:3])


def test_volume_is_conserved_and_F_decreases():
    """sum R^3 over live droplets is an invariant of Eqs. (13)-(14) up to the volume of the
    droplets that died (each at most (eps + R at death)^3); F decreases."""
    R0 = wl.droplet_radii(8, 512, seed=wl.BASE_SEED + 2)
    ts = np.linspace(0.0, 2.0, 21)
    R, ser, steps = ch.ch_droplets_run(R0, 2.0, ts, rtol=1e-8, atol=1e-11, h0=1e-6, eps=1e-3)
    for m in range(8):
        v0 = np.sum(R0[m] ** 3)
        live = R[m][R[m] > 0]
        dead = np.sum(R[m] <= 0)
        assert abs(np.sum(live ** 3) - v0) <= 1e-5 * v0 + dead * 1e-6
        assert np.all(np.diff(ser[m][:, 1]) <= 0)
        assert np.all(ser[m][:, 2] <= 0)


def test_errors_and_limits():
    R0 = np.full((2, 4), 0.5)
    with pytest.raises(ch.ChError):
        ch.ch_droplets_run(R0, 1.0, [0.5, 0.2])  # decreasing sample times
    with pytest.raises(ch.ChError):
        ch.ch_droplets_run(R0, -1.0, [])
    with pytest.raises(ch.ChError):
        ch.ch_droplets_run(R0, 1.0, [], h0=0.0)
    with pytest.raises(ch.ChError):
        ch.ch_droplets_run(wl.droplet_radii(1, 64), 1.0, [], max_steps=10)  # step limit
    R, ser, steps = ch.ch_droplets_run(R0, 0.0, [0.0, 1.0])
    assert steps[0, 0] == 0 and ser[0, 0, 0] == 0.0 and np.isnan(ser[0, 1, 0])
    # equal radii: u = 1/R, every droplet is stationary
    R, ser, steps = ch.ch_droplets_run(R0, 3.0, [3.0], rtol=1e-8)
    assert np.max(np.abs(R - 0.5)) <= 1e-13 and ser[0, 0, 2] == pytest.approx(0.0, abs=1e-10)
