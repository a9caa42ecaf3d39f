"""Grid-refinement error of Appendix A on the GPU (ch_refinement_error and
ch_ensemble_refinement_error) against the oracle, and the droplet runs of the study.

Bars: on the same fields every restricted difference is formed in the same operation
order on both sides, so E differs only by the summation order (bound N u E for N
non-negative terms, doubled); over runs, E differs by at most the largest field
difference of the two grids, and the FP64 fields are held to 1e-10 of the oracle's
after the study's ~500-1000 steps.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import refinement
from paper_1911_03386_gb300 import workloads as wl
from oracle.oracle import get as get_oracle

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def gpu_refinement(torch, fine, coarse):
    ny, nx = fine.shape
    f = torch.from_numpy(np.ascontiguousarray(fine)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(coarse)).cuda()
    out = torch.full((1 + ny // 2,), -1.0, dtype=torch.float64, device="cuda")
    ch.ch_refinement_error(f.data_ptr(), c.data_ptr(), nx, ny, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("nx,ny", [(64, 48), (2, 2), (4096, 6), (10, 2048), (514, 130)])
def test_dense_refinement_error_matches_oracle(torch, orc, nx, ny):
    rng = np.random.default_rng(nx * 7919 + ny)
    coarse = rng.standard_normal((ny // 2, nx // 2))
    fine = np.kron(coarse, np.ones((2, 2))) + 0.01 * rng.standard_normal((ny, nx))
    got = gpu_refinement(torch, fine, coarse)
    want = orc.refinement_error(fine, coarse)
    n = (nx // 2) * (ny // 2)
    assert abs(got[0] - want) <= 2 * n * U * want
    for j in range(ny // 2):  # row means: the definition on the two fine rows of coarse row j
        wj = orc.refinement_error(fine[2 * j:2 * j + 2], coarse[j:j + 1])
        assert abs(got[1 + j] - wj) <= 2 * (nx // 2) * U * wj


def test_dense_refinement_errors(torch):
    f = torch.zeros(16, dtype=torch.float64, device="cuda")
    for nx, ny in [(3, 4), (4, 3), (0, 4), (4, 0)]:
        with pytest.raises(ch.ChError):
            ch.ch_refinement_error(f.data_ptr(), f.data_ptr(), nx, ny, f.data_ptr())


# The study's start and rules at sizes the oracle runs in seconds; dt = 0.01 dx to T = 0.5
# keeps dt/gamma <= 0.4 on the 16-grid (the study's dt = 0.1 dx would be unstable there).
SMALL = dict(wl.REFINEMENT, cfl=0.01, T=0.5)


def oracle_droplet_run(orc, n, preset=SMALL):
    steps, dt = wl.refinement_steps(n, preset)
    C = wl.droplet_field(n, preset["L"], preset["gamma"])
    res = orc.run(C, preset["L"], preset["gamma"], dt, steps, every=steps)
    return res.C


@pytest.mark.parametrize("n", [32, 64])
def test_droplet_runs_and_refinement_error_match_oracle(orc, n):
    """The study's runs on the n- and n/2-grids (GPU, FP64) against the oracle's runs of the
    same start, and E_n from the GPU fields against E_n from the oracle fields."""
    fine_ref = oracle_droplet_run(orc, n)
    coarse_ref = oracle_droplet_run(orc, n // 2)
    e_ref = orc.refinement_error(fine_ref, coarse_ref)
    fe, finfo = refinement.run_grid(n, SMALL)
    ce, cinfo = refinement.run_grid(n // 2, SMALL)
    try:
        df = np.max(np.abs(fe.field(0) - fine_ref))
        dc = np.max(np.abs(ce.field(0) - coarse_ref))
        assert df <= 1e-10 and dc <= 1e-10, (df, dc)
        e = ch.ch_ensemble_refinement_error(fe.h, 0, ce.h, 0)
        assert abs(e - e_ref) <= df + dc + 4 * (n // 2) ** 2 * U * e_ref
        assert finfo["steps"] == wl.refinement_steps(n, SMALL)[0]
    finally:
        fe.close()
        ce.close()


def test_ensemble_refinement_error_checks():
    with ch.Ensemble.create(16, 16, 2 * math.pi, 0.01, 1e-3, [0.0], wl.BASE_SEED, ch.CH_FP64) as a, \
            ch.Ensemble.create(8, 8, 2 * math.pi, 0.01, 1e-3, [0.0, 0.1], wl.BASE_SEED, ch.CH_FP64) as b, \
            ch.Ensemble.create(10, 8, 2 * math.pi, 0.01, 1e-3, [0.0], wl.BASE_SEED, ch.CH_FP64) as c, \
            ch.Ensemble.create(8, 8, 2 * math.pi, 0.01, 1e-3, [0.0], wl.BASE_SEED, ch.CH_FP32) as d:
        e = ch.ch_ensemble_refinement_error(a.h, 0, b.h, 1)
        want = get_oracle().refinement_error(a.field(0), b.field(1))
        assert abs(e - want) <= 1e-15 * want
        for args in [(a.h, 0, c.h, 0), (a.h, 1, b.h, 0), (a.h, 0, b.h, 2), (a.h, 0, d.h, 0), (b.h, 0, a.h, 0)]:
            with pytest.raises(ch.ChError):
                ch.ch_ensemble_refinement_error(*args)


def test_small_study_converges():
    """The study on n = 128 ... 1024: E_n decreases with n (the scheme converges under the
    study's joint refinement dt = 0.1 dx)."""
    rows = refinement.study([128, 256, 512, 1024])
    es = [r["E_n"] for r in rows]
    assert all(math.isfinite(x) and x > 0 for x in es)
    assert es[-1] < es[-2]


def test_tuned_grid_equals_default_shapes():
    """The study's autotuned launch shape (a single grid: usually the fused segment forms)
    and the library's default (split form, one thread per line) give the same field to
    FP64 rounding, and so the same E_n."""
    n = 256
    a, ia = refinement.run_grid(n, SMALL, tune=True)
    b, ib = refinement.run_grid(n, SMALL, tune=False)
    c, _ = refinement.run_grid(n // 2, SMALL, tune=False)
    try:
        assert ib["tuning"]["split"] == 1
        fa, fb = a.field(0), b.field(0)
        assert np.max(np.abs(fa - fb)) <= 1e-12 * max(1.0, np.max(np.abs(fb)))
        ea = ch.ch_ensemble_refinement_error(a.h, 0, c.h, 0)
        eb = ch.ch_ensemble_refinement_error(b.h, 0, c.h, 0)
        assert abs(ea - eb) <= 1e-9 * eb
    finally:
        a.close()
        b.close()
        c.close()
