"""Host-side checks of the seeded input recipes (no GPU): shapes, determinism, the
structure they claim, and the stability reading that fixes the refinement study's
coarsest grid."""
import math

import numpy as np

from paper_1911_03386_gb300 import workloads as wl


def test_beta_ensemble_structure():
    t, beta = wl.beta_ensemble(4000, 51, seed=3, t_end=100.0, beta0=0.28, k=0.0056, diverged=7)
    assert t.shape == (51,) and beta.shape == (4000, 51) and t[0] == 0.0 and t[-1] == 100.0
    assert np.array_equal(beta, wl.beta_ensemble(4000, 51, seed=3, t_end=100.0, beta0=0.28, k=0.0056,
                                                 diverged=7)[1], equal_nan=True)
    assert np.all(np.isnan(beta[-7:, 25:])) and np.all(np.isfinite(beta[:-7]))
    live = beta[:-7]
    assert np.all(live[:, 0] == 0.28)  # no spread at t = 0
    # mean beta0 and variance k t (to sampling error), positive skew
    var = live[:, 1:].var(axis=0)
    assert np.max(np.abs(live[:, 1:].mean(axis=0) - 0.28) / np.sqrt(var / live.shape[0])) < 5
    assert abs(np.polyfit(t[1:], var, 1)[0] - 0.0056) < 0.0056 * 0.1
    assert np.mean(((live[:, -1] - live[:, -1].mean()) ** 3)) > 0


def test_droplet_field_and_steps():
    n = 64
    C = wl.droplet_field(n)
    assert C.shape == (n, n) and np.all(np.abs(C) <= 1)
    # symmetric under the box's reflections about its centre lines (cell-centred samples)
    for X in (C[::-1, :], C[:, ::-1], C.T):
        np.testing.assert_allclose(C, X, rtol=0, atol=1e-12)
    assert C[n // 2, n // 2] > 0.99 and C[0, 0] < -0.99  # outside the droplet at the centre, inside at the corner
    for n in wl.REFINEMENT["sizes"]:
        steps, dt = wl.refinement_steps(n)
        assert abs(steps * dt - wl.REFINEMENT["T"]) < 1e-12
        assert abs(dt / (0.1 * wl.REFINEMENT["L"] / n) - 1) < 1.0 / steps + 1e-12


def _min_amplification(n, dt, gamma, d=2.0, L=2 * math.pi):
    """Smallest linear amplification factor of the factorised scheme over the grid modes
    of an n x n grid, about a state with 3 C^2 - 1 = d (C = +-1: d = 2)."""
    h = L / n
    k = np.arange(n)
    a = 4.0 / h ** 2 * np.sin(math.pi * k / n) ** 2
    ax, ay = np.meshgrid(a, a)
    A = ax + ay
    s = gamma * dt
    G = 1.0 - dt * (A * d + gamma * A * A) / ((1.0 + s * ax * ax) * (1.0 + s * ay * ay))
    return G.min()


def test_refinement_grids_start_where_the_scheme_is_stable():
    """With dt = 0.1 dx the 64-grid has a mode with G < -1 about C = +-1 (the run diverges);
    every grid of the study (128 and up) stays within [-1, 1]."""
    g = wl.REFINEMENT["gamma"]
    assert _min_amplification(64, wl.refinement_steps(64)[1], g) < -1.1
    for n in wl.REFINEMENT["sizes"][:4]:
        assert _min_amplification(n, wl.refinement_steps(n)[1], g) > -1.0


def test_campaign_and_droplet_starts():
    C = wl.asymmetric_field(128, 5, 3)
    assert C.shape == (128, 128) and C.min() >= 0.4 and C.max() < 0.5 and abs(C.mean() - 0.45) < 0.002
    assert not np.array_equal(C, wl.asymmetric_field(128, 5, 4))
    R = wl.droplet_radii(10, 300)
    assert R.shape == (10, 300) and R.min() >= 0 and R.max() < 1
    assert np.array_equal(R, wl.droplet_radii(10, 300))
    n = int(round(wl.CAMPAIGN["Ls"][0] / wl.CAMPAIGN["dx"]))
    assert n == 256
