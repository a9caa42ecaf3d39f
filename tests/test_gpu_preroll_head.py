"""FP32 heads of the FP64 streaming sweeps' pre-rolls (ch_tuning.preroll_head) on the GPU.

The head changes only rounding below the FP64 pre-roll's own tolerance: runs with and
without it agree to FP64 round-off, both match the oracle, including a grid whose
pre-roll (and head) wraps the line several times, and a NaN still reaches the
observables through a head.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu

SEED = wl.BASE_SEED


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def run(nx, ny, L, C0, nsteps, head, gamma=0.005, dt=1e-3):
    with ch.Ensemble.create(nx, ny, L, gamma, dt, C0, SEED, ch.CH_FP64) as e:
        e.set_tuning(preroll_head=head)
        assert e.tuning()["preroll_head"] == head and e.tuning()["stream"] == 1
        e.step(nsteps)
        return [e.field(k) for k in range(len(C0))]


def test_ensemble_size_members_with_and_without_head():
    # 256 x 256 over [0, 2 pi)^2: K = 110 with a 32-point FP32 head in the row sweeps
    K, head = ch.ch_preroll_head(0.005 * 1e-3 / (2 * math.pi / 256) ** 4)
    assert head == 32
    # Rounding differences grow with the spinodal instability, at most like exp(t / (4 gamma))
    # (the linear growth rate k^2 (1 - gamma k^2) peaks at 1 / (4 gamma) = 50): by 1.6 over
    # 10 steps, by 150 over 100.
    C0 = [0.0, 0.4, 0.0, 0.4]
    for nsteps, tol in ((10, 1e-14), (100, 1e-12)):
        on = run(256, 256, 2 * math.pi, C0, nsteps, 0)
        off = run(256, 256, 2 * math.pi, C0, nsteps, -1)
        for a, b in zip(on, off):
            assert np.max(np.abs(a - b)) <= tol


@pytest.mark.parametrize("nx,ny", [(32, 32), (48, 40), (256, 24)])
def test_heads_match_oracle(nx, ny):
    # the row spacing of the 256^2 ensemble on smaller domains: K = 110 (head 32) wraps
    # rows of 32 and 48 points several times
    orc = get_oracle()
    L = nx * 2 * math.pi / 256  # hx of the ensemble; hy = L / ny
    nsteps = 60
    C0 = [0.0, 0.3]
    on = run(nx, ny, L, C0, nsteps, 0)
    for k, c0 in enumerate(C0):
        ref = orc.run(orc.initial_field(nx, ny, c0, SEED, k * nx * ny), L, 0.005, 1e-3, nsteps)
        assert np.max(np.abs(on[k] - ref.C)) <= 1e-12


def test_nan_passes_through_a_head():
    with ch.Ensemble.create(256, 256, 2 * math.pi, 0.005, 1e-3, [0.0, 0.4], SEED, ch.CH_FP64) as e:
        assert ch.ch_preroll_head(0.005 * 1e-3 / (2 * math.pi / 256) ** 4)[1] > 0
        e.set_sampling(1, 0.0, capacity=4)
        e.step(2)
        ch.ch_set_fault("nan:1")
        try:
            e.step(2)
        finally:
            ch.ch_set_fault(None)
        with pytest.raises(ch.ChError) as err:
            e.observables()
        assert err.value.code == ch.CH_ENONFINITE
        assert np.all(np.isfinite(e.field(0)))
        assert not np.all(np.isfinite(e.field(1)))


def test_preroll_head_argument_errors():
    with ch.Ensemble.create(64, 64, 2 * math.pi, 0.005, 1e-3, [0.0], SEED, ch.CH_FP64) as e:
        for bad in (1, -2):
            with pytest.raises(ch.ChError):
                e.set_tuning(preroll_head=bad)
        assert e.tuning()["preroll_head"] == 0
