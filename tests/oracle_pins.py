"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each pin takes an `Oracle` instance and raises AssertionError on a mismatch.  None of them
retypes the oracle's own formula: they use published generator outputs, closed forms
(Fourier symbols, exact sums of cos^k), dense brute force with a library solver,
conservation, energy decay and the continuum interface energy.  The pin tests run them
on the oracle; the mutation test runs them on deliberately broken builds and requires
every break to be caught.
"""
import ctypes
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TWO_PI = 2.0 * math.pi


def _golden_splitmix():
    vals = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 16))
    return vals


def _symbol(k_index, n, h):
    """Eigenvalue of minus the periodic second difference for mode k: (4/h^2) sin^2(theta/2)."""
    theta = TWO_PI * k_index / n
    return 4.0 / (h * h) * math.sin(theta / 2.0) ** 2


# ------------------------------------------------------------------------------------------
# Random numbers and the initial field
# ------------------------------------------------------------------------------------------
def pin_splitmix_golden(orc):
    for k, v in enumerate(_golden_splitmix()):
        got = orc.splitmix64(0, k)
        assert got == v, "splitmix64(0,%d) = %#x, published %#x" % (k, got, v)


def pin_uniform_exact(orc):
    for k, v in enumerate(_golden_splitmix()):
        want = float(v >> 11) / 9007199254740992.0
        assert orc.uniform(0, k) == want


def pin_initial_field(orc):
    gold = _golden_splitmix()
    nx, ny, C0 = 7, 5, 0.3
    C = orc.initial_field(nx, ny, C0, 0, 0)
    for k in range(3):
        u = float(gold[k] >> 11) / 9007199254740992.0
        assert C[0, k] == C0 + 0.1 * (2.0 * u - 1.0), "IC point %d" % k
    # draw k = base + j*nx + i: row-major, x fastest, counter shifted by the base
    C2 = orc.initial_field(nx, ny, C0, 0, 3)
    assert np.array_equal(C2.ravel()[:-3], C.ravel()[3:])
    assert np.all(np.abs(C - C0) <= 0.1)
    big = orc.initial_field(128, 128, -0.2, 12345, 0)
    assert abs(big.mean() + 0.2) < 4 * 0.1 / math.sqrt(3 * 128 * 128)
    assert abs(big.std() - 0.1 / math.sqrt(3)) < 2e-3


# ------------------------------------------------------------------------------------------
# Stencils: exact Fourier symbols, the nonlinear term in closed form
# ------------------------------------------------------------------------------------------
def pin_laplacian_symbol(orc):
    nx, ny, L = 12, 10, TWO_PI
    hx, hy = L / nx, L / ny
    x = np.arange(nx) * hx
    y = np.arange(ny) * hy
    X, Y = np.meshgrid(x, y)
    for kx, ky in [(1, 0), (0, 1), (2, 3), (5, 4), (6, 5)]:
        v = np.cos(kx * X + ky * Y + 0.37)
        lam = _symbol(kx, nx, hx) + _symbol(ky, ny, hy)
        got = orc.laplacian(v, hx, hy)
        assert np.max(np.abs(got + lam * v)) <= 1e-12 * max(1.0, lam), (kx, ky)


def pin_rhs_constant(orc):
    C = np.full((9, 11), 0.37)
    mu, R = orc.rhs(C, 0.5, 0.4, 0.01, 1e-3)
    assert np.all(R == 0.0)
    assert np.allclose(mu, 0.37 ** 3 - 0.37, rtol=0, atol=1e-15)


def _rhs_single_axis_case(orc, axis):
    # C = a cos(k x) along one axis: C^3 - C = (3a^3/4 - a) cos(k x) + (a^3/4) cos(3 k x),
    # every cos(m k x) is an eigenfunction of lap_h with eigenvalue -symbol(m k).
    n_along, n_across, L, gamma, dt, a, k = 16, 6, TWO_PI, 0.013, 2e-3, 0.7, 1
    h = L / n_along
    s = np.arange(n_along) * h
    c1 = np.cos(k * s)
    c3 = np.cos(3 * k * s)
    line = a * c1
    if axis == 0:  # variation along x
        C = np.tile(line, (n_across, 1))
        hx, hy = h, L / n_across
    else:
        C = np.tile(line[:, None], (1, n_across))
        hx, hy = L / n_across, h
    l1, l3 = _symbol(k, n_along, h), _symbol(3 * k, n_along, h)
    mu_line = (0.75 * a ** 3 - a + gamma * a * l1) * c1 + 0.25 * a ** 3 * c3
    R_line = -dt * ((0.75 * a ** 3 - a + gamma * a * l1) * l1 * c1 + 0.25 * a ** 3 * l3 * c3)
    mu, R = orc.rhs(C, hx, hy, gamma, dt)
    mu_want = np.tile(mu_line, (n_across, 1)) if axis == 0 else np.tile(mu_line[:, None], (1, n_across))
    R_want = np.tile(R_line, (n_across, 1)) if axis == 0 else np.tile(R_line[:, None], (1, n_across))
    assert np.max(np.abs(mu - mu_want)) < 1e-12
    assert np.max(np.abs(R - R_want)) < 1e-12 * max(1.0, np.max(np.abs(R_want)))


def pin_rhs_nonlinear_x(orc):
    _rhs_single_axis_case(orc, 0)


def pin_rhs_nonlinear_y(orc):
    _rhs_single_axis_case(orc, 1)


# ------------------------------------------------------------------------------------------
# Cyclic pentadiagonal solve
# ------------------------------------------------------------------------------------------
def _dense_cyclic(n, s):
    P = np.roll(np.eye(n), 1, axis=1)
    P2 = P @ P
    return (1 + 6 * s) * np.eye(n) - 4 * s * (P + P.T) + s * (P2 + P2.T)


def pin_penta_dense_lu(orc):
    rng = np.random.default_rng(7)
    for n in range(5, 17):
        for s in [1e-3, 0.107, 1.0, 13.8, 880.0, 1e4]:
            A = _dense_cyclic(n, s)
            r = rng.standard_normal(n)
            ref = np.linalg.solve(A, r)
            got = orc.penta_solve(s, r)
            tol = 64 * np.finfo(float).eps * (1 + 16 * s) * max(1.0, np.max(np.abs(ref)))
            assert np.max(np.abs(got - ref)) <= tol, (n, s, np.max(np.abs(got - ref)), tol)


def pin_penta_eigenvectors(orc):
    for n in [5, 7, 16, 64]:
        for s in [0.3, 3.7, 500.0]:
            i = np.arange(n)
            for k in range(n):
                theta = TWO_PI * k / n
                r = np.cos(theta * i + 0.3)
                want = r / (1.0 + s * (2.0 - 2.0 * math.cos(theta)) ** 2)
                got = orc.penta_solve(s, r)
                assert np.max(np.abs(got - want)) < 1e-13 * (1 + 16 * s), (n, s, k)


def pin_penta_constant(orc):
    for n in [5, 6, 33]:
        for s in [0.01, 10.0, 1e4]:
            got = orc.penta_solve(s, np.full(n, -1.25))
            assert np.max(np.abs(got + 1.25)) < 1e-14 * (1 + 16 * s)


# ------------------------------------------------------------------------------------------
# Full step: linear amplification of a single Fourier mode, conservation, energy
# ------------------------------------------------------------------------------------------
def pin_mode_amplification(orc):
    nx, ny, L, gamma, dt, C0, eps, nsteps = 16, 12, TWO_PI, 0.01, 1e-3, 0.3, 1e-6, 20
    hx, hy = L / nx, L / ny
    X, Y = np.meshgrid(np.arange(nx) * hx, np.arange(ny) * hy)
    sigma = gamma * dt
    d = 3 * C0 * C0 - 1
    for kx, ky in [(1, 0), (0, 2), (2, 1), (3, 3), (7, 5)]:
        phi = np.cos(kx * X + ky * Y)
        C = C0 + eps * phi
        for _ in range(nsteps):
            orc.step(C, L, gamma, dt)
        amp = np.sum((C - C0) * phi) / np.sum(phi * phi)
        ax, ay = _symbol(kx, nx, hx), _symbol(ky, ny, hy)
        A = ax + ay
        G = 1 - dt * (A * d + gamma * A * A) / ((1 + sigma * ax * ax) * (1 + sigma * ay * ay))
        want = eps * G ** nsteps
        assert abs(amp - want) <= 1e-7 * abs(want), (kx, ky, amp, want)


def pin_nyquist_mode_exact(orc):
    # The checkerboard (-1)^(i+j) is closed under the step, nonlinear term included:
    # phi^2 = 1 is constant (the Laplacian removes it) and phi^3 = phi.  So its amplitude
    # follows a scalar recursion exactly, here at s = gamma dt / h^4 of order 10^3, where the
    # factorised operator damps the mode by only about 1 / (4 s) per step.
    nx, ny, L, gamma, dt, C0, eps, nsteps = 96, 80, 0.6, 0.005, 1e-3, 0.3, 0.05, 12
    hx, hy = L / nx, L / ny
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.where((i + j) % 2 == 0, 1.0, -1.0)
    C = C0 + eps * phi
    for _ in range(nsteps):
        orc.step(C, L, gamma, dt)
    amp = np.sum((C - C0) * phi) / phi.size
    sigma, ax, ay = gamma * dt, 4 / hx ** 2, 4 / hy ** 2
    A, d = ax + ay, 3 * C0 * C0 - 1
    assert sigma * ax * ax / 16 > 1e3  # s_x
    x = eps
    for _ in range(nsteps):
        x -= dt * (A * (d * x + x ** 3) + gamma * A * A * x) / ((1 + sigma * ax * ax) * (1 + sigma * ay * ay))
    assert 0 < 1 - x / eps < 1e-2
    assert abs(amp - x) <= 1e-12 * abs(x), (amp, x)
    assert np.max(np.abs(C - C0 - amp * phi)) <= 1e-12


def pin_mass_conservation(orc):
    C = orc.initial_field(40, 24, 0.2, 99, 0)
    m0 = C.sum()
    for _ in range(100):
        orc.step(C, TWO_PI, 0.01, 1e-3)
    bound = 50 * C.size * np.finfo(float).eps * np.max(np.abs(C)) * math.sqrt(100)
    assert abs(C.sum() - m0) <= bound, (C.sum() - m0, bound)


def pin_energy_monotone(orc):
    C = orc.initial_field(32, 32, 0.0, 5, 0)
    Fs = []
    for _ in range(300):
        F, _ = orc.step(C, TWO_PI, 0.01, 1e-5, with_obs=True)
        Fs.append(F)
    Fs = np.array(Fs)
    assert np.all(np.diff(Fs) <= 1e-13 * Fs[:-1]), np.max(np.diff(Fs))
    assert Fs[-1] < Fs[0]


def pin_dFdt_is_time_derivative(orc):
    # Semi-discrete identity: the rate of change of F_h along the scheme equals dFdt_h as
    # dt -> 0, to first order in dt.
    n, L, gamma = 32, TWO_PI, 0.05
    h = L / n
    X, Y = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    base = 0.4 * np.cos(X) + 0.3 * np.sin(2 * Y) + 0.2 * np.cos(X + Y) + 0.1
    errs = []
    for dt in [2e-6, 1e-6]:
        C = base.copy()
        F0, D0 = orc.step(C, L, gamma, dt, with_obs=True)
        F1, _ = orc.field_observables(C, L, gamma)
        errs.append(abs((F1 - F0) / dt - D0) / abs(D0))
    assert errs[1] < 1e-4, errs
    assert 0.35 < errs[1] / errs[0] < 0.65, errs  # first order in dt


def pin_constant_field_observables(orc):
    C0, L, gamma = 0.3, 1.7, 0.02
    C = np.full((9, 12), C0)
    F, D = orc.field_observables(C, L, gamma)
    assert abs(F - 0.25 * (C0 * C0 - 1) ** 2 * L * L) <= 1e-14 * F
    assert D == 0.0
    assert orc.beta(3.0, F, D) == 0.0


def pin_single_mode_energy(orc):
    # C = C0 + a cos(theta i) along x: exact sums sum cos = 0, cos^2 = n/2, cos^3 = 0,
    # cos^4 = 3n/8 (4k not a multiple of n), sum (c_{i+1}-c_i)^2 = n (1 - cos theta).
    nx, ny, L, gamma, C0, a, k = 16, 7, 3.0, 0.02, 0.25, 0.6, 1
    hx, hy = L / nx, L / ny
    theta = TWO_PI * k / nx
    line = C0 + a * np.cos(theta * np.arange(nx))
    C = np.tile(line, (ny, 1))
    p, q, r = C0 * C0 - 1, 2 * C0 * a, a * a
    bulk = nx * p * p + (q * q + 2 * p * r) * nx / 2 + r * r * 3 * nx / 8
    grad = (a * a / (hx * hx)) * nx * (1 - math.cos(theta))
    want = hx * hy * ny * (0.25 * bulk + 0.5 * gamma * grad)
    F, _ = orc.field_observables(C, L, gamma)
    assert abs(F - want) <= 1e-13 * abs(want), (F, want)


def pin_interface_energy(orc):
    # Two flat interfaces relaxed to equilibrium: F -> 2 L (2 sqrt(2)/3) sqrt(gamma), the
    # interface energy of the 1/4 (C^2-1)^2 + gamma/2 |grad C|^2 functional; O(h^2) error.
    nx, ny, L, gamma, dt = 256, 6, TWO_PI, 0.01, 1e-3
    x = np.arange(nx) * (L / nx)
    w = math.sqrt(2 * gamma)
    line = np.tanh((np.abs(x - L / 2) - L / 4) / (1.5 * w))
    C = np.ascontiguousarray(np.tile(line, (ny, 1)))
    for _ in range(600):
        orc.step(C, L, gamma, dt)
    F, D = orc.field_observables(C, L, gamma)
    want = 2 * L * (2 * math.sqrt(2) / 3) * math.sqrt(gamma)
    assert abs(F - want) <= 5e-3 * want, (F, want)
    assert -5e-3 < D <= 0.0, D  # relaxing towards equilibrium


def pin_run_sampling(orc):
    L, gamma, dt, every = TWO_PI, 0.01, 1e-3, 5
    C = orc.initial_field(16, 12, 0.1, 3, 0)
    t1 = 20 * dt
    res = orc.run(C, L, gamma, dt, 37, every=every, t1=t1)
    # samples at n = 0, 5, ..., 35 from C^n before the update
    assert res.series.shape[0] == 8
    ref = C.copy()
    betas_in_window = []
    for n in range(37):
        if n % every == 0:
            F, D = orc.field_observables(ref, L, gamma)
            row = res.series[n // every]
            assert row[0] == n * dt
            assert abs(row[1] - F) <= 1e-13 * abs(F) and abs(row[2] - D) <= 1e-12 * abs(D) + 1e-14
            t = n * dt
            b = -t * D / F
            assert abs(row[3] - b) <= 1e-12 * abs(b) + 1e-15
            if t >= t1:
                betas_in_window.append(row[3])
        orc.step(ref, L, gamma, dt)
    assert res.series[0, 3] == 0.0
    assert np.array_equal(ref, res.C)
    assert res.beta_count == len(betas_in_window) == 4
    assert abs(res.beta_sum - sum(betas_in_window)) <= 1e-14 * abs(res.beta_sum)


# ------------------------------------------------------------------------------------------
# Ensemble statistics of beta (Sec. 3.3 Eqs. (41a,b), (42); Sec. 1 Eq. (7))
# ------------------------------------------------------------------------------------------
def pin_moments_discrete_uniform(orc):
    """Values 1..M: mean (M+1)/2, central moments (M^2-1)/12, 0, (M^2-1)(3M^2-7)/240;
    an affine map a x + c maps mu_1 to a mu_1 + c and mu_p to a^p mu_p."""
    M = 11
    x = np.arange(1, M + 1, dtype=np.float64)
    a, c = -2.0, 0.5
    beta = np.stack([x, a * x + c, x[::-1]], axis=1)  # (M, 3): member j, sample s
    m = orc.beta_moments(beta)
    mu1, mu2, mu3, mu4 = (M + 1) / 2.0, (M * M - 1) / 12.0, 0.0, (M * M - 1) * (3.0 * M * M - 7.0) / 240.0
    for s, (scale, shift) in enumerate([(1.0, 0.0), (a, c), (1.0, 0.0)]):
        assert m[s, 0] == M
        assert abs(m[s, 1] - (scale * mu1 + shift)) <= 1e-14 * abs(scale * mu1 + shift)
        assert abs(m[s, 2] - scale ** 2 * mu2) <= 1e-13 * scale ** 2 * mu2
        assert abs(m[s, 3] - scale ** 3 * mu3) <= 1e-12 * abs(scale) ** 3 * mu2 ** 1.5
        assert abs(m[s, 4] - scale ** 4 * mu4) <= 1e-13 * scale ** 4 * mu4


def pin_moments_two_point(orc):
    """A two-point law (value c with weight 1-p, c+d with weight p) has central moments
    p(1-p) d^2, p(1-p)(1-2p) d^3, p(1-p)(1-3p+3p^2) d^4 (the skew's sign follows p < 1/2)."""
    c, d = 0.25, 2.0
    for ones, zeros in [(1, 3), (3, 1), (2, 6)]:
        col = np.array([c + d] * ones + [c] * zeros)
        p = ones / float(ones + zeros)
        m = orc.beta_moments(col[:, None])
        q = p * (1.0 - p)
        want = [ones + zeros, c + p * d, q * d ** 2, q * (1.0 - 2.0 * p) * d ** 3,
                q * (1.0 - 3.0 * p + 3.0 * p * p) * d ** 4]
        for k in range(5):
            assert abs(m[0, k] - want[k]) <= 1e-14 * max(1.0, abs(want[k])), (ones, zeros, k, m[0], want)


def pin_moments_library_with_nonfinite(orc):
    """Random ensembles against scipy.stats.moment (central moments, 1/M normalisation) on
    the finite values; NaN and infinite entries (diverged runs) are left out and counted."""
    from scipy import stats
    rng = np.random.default_rng(7)
    M, T = 37, 9
    beta = 0.3 + rng.standard_normal((M, T)) * np.linspace(0.01, 0.2, T) + 0.05 * rng.exponential(size=(M, T))
    beta[3, 2] = np.nan
    beta[5, 2] = np.inf
    beta[:, 7] = np.nan  # every run diverged at this sample
    m = orc.beta_moments(beta)
    for s in range(T):
        v = beta[:, s][np.isfinite(beta[:, s])]
        assert m[s, 0] == v.size
        if v.size == 0:
            assert np.all(np.isnan(m[s, 1:]))
            continue
        assert abs(m[s, 1] - v.mean()) <= 1e-14
        for p in (2, 3, 4):
            want = float(stats.moment(v, moment=p))
            assert abs(m[s, p] - want) <= 1e-12 * np.mean(np.abs(v - v.mean()) ** p) + 1e-300, (s, p)


def pin_histogram_brute_force(orc):
    """Bins of dyadic width (edges exact in binary) against comparison with the edges:
    value b falls in bin k when lo + k w <= b < lo + (k+1) w; b < lo and b >= hi in the
    two outer counters; values on an edge go to the bin above; non-finite ones nowhere."""
    lo, hi, nb = -0.5, 1.5, 16
    w = (hi - lo) / nb
    rng = np.random.default_rng(3)
    M, T = 53, 4
    beta = rng.uniform(-1.0, 2.0, size=(M, T))
    edges = lo + w * np.arange(nb + 1)
    beta[:8, 0] = edges[:8]          # exactly on lower edges
    beta[8, 0] = hi                  # exactly at hi: overflow
    beta[9, 0] = lo                  # exactly at lo: first bin
    beta[10:14, 1] = edges[1:5] + 0.5 * w   # bin centres
    beta[14, 1] = np.nan
    beta[15, 1] = -np.inf
    beta[16, 1] = np.inf
    h = orc.beta_histogram(beta, lo, hi, nb)
    assert h.shape == (T, nb + 2)
    for s in range(T):
        want = np.zeros(nb + 2, dtype=np.int64)
        for b in beta[:, s]:
            if not np.isfinite(b):
                continue
            if b < lo:
                want[0] += 1
            elif b >= hi:
                want[nb + 1] += 1
            else:
                k = [i for i in range(nb) if edges[i] <= b < edges[i + 1]]
                assert len(k) == 1
                want[k[0] + 1] += 1
        assert np.array_equal(h[s], want), (s, h[s], want)
    assert h[1].sum() == M - 3


def pin_trend_closed_forms(orc):
    """Trapezoid window mean: exact for mu_1 linear in t; for mu_1 = t^2 on a uniform grid
    of step h it exceeds the exact mean (t1^2 + t1 t2 + t2^2)/3 by h^2/6; the mean of a
    constant is that constant also when the window extends beyond the samples.  Least
    squares through the origin: k = 0.3 for mu_2 = 0.3 t; k = 3n(n+1)/(2(2n+1)) for
    mu_2 = t^2 on t = 1..n (sum t^3 / sum t^2)."""
    h = 0.25
    t = np.arange(0, 41) * h            # 0 .. 10
    t1, t2 = 2.0, 7.0
    mean_lin, _, nw, _ = orc.beta_trend(t, 0.2 + 0.05 * t, 0 * t, t1, t2, 0.0, 10.0)
    assert nw == 21
    assert abs(mean_lin - (0.2 + 0.05 * (t1 + t2) / 2.0)) <= 1e-15
    mean_sq, _, _, _ = orc.beta_trend(t, t * t, 0 * t, t1, t2, 0.0, 10.0)
    assert abs(mean_sq - ((t1 * t1 + t1 * t2 + t2 * t2) / 3.0 + h * h / 6.0)) <= 1e-13
    mean_c, _, nw, _ = orc.beta_trend(t, np.full_like(t, 0.28), 0 * t, -3.0, 2.1, 0.0, 10.0)
    assert nw == 9 and mean_c == 0.28
    _, k, _, nf = orc.beta_trend(t, 0 * t, 0.3 * t, t1, t2, 2.0, 7.0)
    assert nf == 21 and abs(k - 0.3) <= 1e-15
    n = 40
    tt = np.arange(1, n + 1, dtype=np.float64)
    _, k, _, nf = orc.beta_trend(tt, 0 * tt, tt * tt, 0.0, 1.0, 1.0, float(n))
    assert nf == n and abs(k - 3.0 * n * (n + 1) / (2.0 * (2 * n + 1))) <= 1e-13 * k
    mean_none, k_none, nw, nf = orc.beta_trend(t, t, t, 20.0, 30.0, 20.0, 30.0)
    assert nw == 0 and nf == 0 and np.isnan(mean_none) and np.isnan(k_none)


# ------------------------------------------------------------------------------------------
# Grid-refinement error (Appendix A)
# ------------------------------------------------------------------------------------------
def _cell_centres(n, L):
    return (np.arange(n) + 0.5) * (L / n)


def pin_refinement_prolongation_and_linear(orc):
    """A fine field that repeats every coarse value over its 2 x 2 block, and a linear
    function sampled at cell centres (whose 2 x 2 means are its values at the coarse
    centres), restrict exactly: E = 0 to rounding.  Odd sizes are rejected (NaN)."""
    rng = np.random.default_rng(5)
    coarse = rng.standard_normal((9, 14))
    fine = np.kron(coarse, np.ones((2, 2)))
    assert orc.refinement_error(fine, coarse) <= 4e-16 * np.max(np.abs(coarse))
    L = 2.0 * math.pi
    xf, yf = _cell_centres(28, L), _cell_centres(18, L)
    xc, yc = _cell_centres(14, L), _cell_centres(9, L)
    lin = lambda x, y: 0.3 + 0.7 * x[None, :] - 0.2 * y[:, None]
    assert orc.refinement_error(lin(xf, yf), lin(xc, yc)) <= 1e-14
    dp = ctypes.POINTER(ctypes.c_double)
    assert math.isnan(orc._L.or_refinement_error(7, 4, fine.ctypes.data_as(dp), coarse.ctypes.data_as(dp)))


def pin_refinement_fourier_mode(orc):
    """cos(kx) cos(ly) on cell-centred grids: the mean of a 2 x 2 block of the fine samples
    is the coarse sample times cos(k h_x/2) cos(l h_y/2) (h the fine spacings), so
    E = (1 - cos(k h_x/2) cos(l h_y/2)) * mean_i |cos(k x_i)| * mean_j |cos(l y_j)| over
    the coarse points.  A restriction off by one point or a wrong normalisation fails."""
    L = 2.0 * math.pi
    for (nx, ny, k, l) in [(24, 16, 3, 2), (40, 40, 5, 1), (12, 20, 1, 4)]:
        xf, yf = _cell_centres(nx, L), _cell_centres(ny, L)
        xc, yc = _cell_centres(nx // 2, L), _cell_centres(ny // 2, L)
        fine = np.cos(l * yf)[:, None] * np.cos(k * xf)[None, :]
        coarse = np.cos(l * yc)[:, None] * np.cos(k * xc)[None, :]
        hx, hy = L / nx, L / ny
        want = (1.0 - math.cos(k * hx / 2) * math.cos(l * hy / 2)) * np.mean(np.abs(np.cos(k * xc))) * \
            np.mean(np.abs(np.cos(l * yc)))
        got = orc.refinement_error(fine, coarse)
        assert abs(got - want) <= 1e-13 * want + 1e-16, (nx, ny, k, l, got, want)


# ------------------------------------------------------------------------------------------
# Model 1 droplet populations and the Dormand-Prince integrator
# ------------------------------------------------------------------------------------------
def pin_dp_quadrature_orders(orc):
    """For y' = t^p the fifth-order solution is the method's quadrature: exact for p <= 4
    (the order conditions sum b c^k = 1/(k+1), k <= 4) and wrong at p = 5, its error
    scaling like h^6; the embedded fourth-order solution is exact for p <= 3, so the error
    estimate vanishes there and scales like h^5 at p = 4."""
    t0 = 0.3
    for p in range(5):
        for h in (0.7, 0.35):
            v, e = orc.dp_poly_step(p, t0, 0.0, h)
            want = ((t0 + h) ** (p + 1) - t0 ** (p + 1)) / (p + 1)
            assert abs(v - want) <= 1e-15 * max(1.0, abs(want)), (p, h, v, want)
            if p <= 3:
                assert abs(e) <= 1e-15, (p, e)
    e1 = orc.dp_poly_step(4, 0.0, 0.0, 0.2)[1]
    e2 = orc.dp_poly_step(4, 0.0, 0.0, 0.1)[1]
    assert e1 != 0.0 and abs(e1 / e2 - 32.0) < 1e-9
    d1 = orc.dp_poly_step(5, 0.0, 0.0, 0.2)[0] - 0.2 ** 6 / 6
    d2 = orc.dp_poly_step(5, 0.0, 0.0, 0.1)[0] - 0.1 ** 6 / 6
    assert d1 != 0.0 and abs(d1 / d2 - 64.0) < 1e-6


def pin_dp_linear_stability(orc):
    """On y' = lam y one step multiplies y by the method's stability function, for the
    Dormand-Prince pair R(z) = sum_{k <= 5} z^k / k! + z^6 / 600 (z = lam h); the error
    estimate behaves like z^5."""
    for lam, h in [(1.0, 0.5), (-3.0, 0.1), (-20.0, 0.1), (2.0, 0.01)]:
        z = lam * h
        R = sum(z ** k / math.factorial(k) for k in range(6)) + z ** 6 / 600.0
        v, _ = orc.dp_lin_step(lam, 1.0, h)
        assert abs(v - R) <= 4e-16 * max(1.0, abs(R)), (lam, h, v, R)
    e1 = orc.dp_lin_step(-1.0, 1.0, 0.04)[1]
    e2 = orc.dp_lin_step(-1.0, 1.0, 0.02)[1]
    assert e1 != 0.0 and abs(e1 / e2 - 32.0) < 1.0


def pin_drop_single_and_invariants(orc):
    """One droplet is stationary (u = 1/R balances the curvature term).  Along a stretch
    with no extinction the flow conserves the total volume sum R^3 (3 sum R^2 dR/dt =
    3 sum (u R - 1) = 0 by the definition of u) and F decreases."""
    R, ser, acc, rej = orc.drop_run([0.37], 5.0, [0.0, 5.0], rtol=1e-10, atol=1e-12)
    assert abs(R[0] - 0.37) <= 1e-13
    R0 = np.array([0.6, 0.7, 0.8, 0.95, 1.0])
    R, ser, acc, rej = orc.drop_run(R0, 0.05, np.linspace(0, 0.05, 6), rtol=1e-11, atol=1e-13)
    assert np.all(ser[:, 4] == 5)
    assert abs(np.sum(R ** 3) - np.sum(R0 ** 3)) <= 1e-10
    assert np.all(np.diff(ser[:, 1]) < 0)


def pin_drop_observables_identity(orc):
    """dF/dt of Eq. (33) equals -sum 1/R + u N over the live droplets (expand the square
    and use u sum R = N); dead droplets (R <= 0) count in neither F nor dF/dt."""
    rng = np.random.default_rng(9)
    R = rng.uniform(0.05, 1.0, 40)
    R[[3, 17]] = [-1e-3, 0.0]
    live = R[R > 0]
    u = live.size / live.sum()
    F, D, A = orc.drop_observables(R)
    assert A == live.size
    assert abs(F - 0.5 * np.sum(live ** 2)) <= 1e-14 * F
    assert abs(D - (-np.sum(1.0 / live) + u * live.size)) <= 1e-12 * abs(D)


def pin_drop_dFdt_is_derivative(orc):
    """The sampled dF/dt is the time derivative of the sampled F: central differences of
    F at spacing delta agree to O(delta^2) (tight tolerances, no extinction)."""
    R0 = np.array([0.5, 0.65, 0.8, 0.9, 1.0, 1.1])
    d = 1e-3
    ts = np.array([0.02 - d, 0.02, 0.02 + d])
    _, ser, _, _ = orc.drop_run(R0, 0.03, ts, rtol=1e-12, atol=1e-14)
    fd = (ser[2, 1] - ser[0, 1]) / (2 * d)
    assert abs(fd - ser[1, 2]) <= 1e-4 * abs(ser[1, 2]), (fd, ser[1, 2])
    assert abs(ser[1, 3] - (-(0.02 / ser[1, 1]) * ser[1, 2])) <= 1e-15 * abs(ser[1, 3])


def pin_drop_convergence_order(orc):
    """Fixed steps (rtol <= 0) converge at fifth order or better on a smooth stretch (no
    extinction before t = 0.1): halving h from 0.025 divides the error by more than 2^4.5
    (measured 44; a tableau that loses an order condition drops to 16 or below)."""
    R0 = np.array([0.6, 0.8, 1.0])
    ref = orc.drop_run(R0, 0.1, [], rtol=0.0, h0=0.1 / 1024)[0]
    errs = [np.max(np.abs(orc.drop_run(R0, 0.1, [], rtol=0.0, h0=0.1 / m)[0] - ref)) for m in (4, 8)]
    assert errs[0] / errs[1] > 2.0 ** 4.5 and errs[1] < 1e-9, errs


def pin_drop_extinction(orc):
    """A droplet much smaller than the others vanishes after about R^3/3 (dR/dt ~ -1/R^2),
    then sits at or just below -eps, out of the live count; the adaptive integrator with
    tight tolerances agrees with fine fixed steps."""
    R0 = np.array([0.05, 1.0])
    R, ser, _, _ = orc.drop_run(R0, 2e-4, [1e-5, 2e-4], rtol=1e-9, atol=1e-12, h0=1e-7, eps=1e-3)
    assert ser[0, 4] == 2 and ser[1, 4] == 1
    assert -2e-3 < R[0] <= -1e-3
    R1 = np.array([0.6, 0.8, 1.0])
    a = orc.drop_run(R1, 0.1, [], rtol=1e-11, atol=1e-13)[0]
    b = orc.drop_run(R1, 0.1, [], rtol=0.0, h0=0.1 / 256)[0]
    assert np.max(np.abs(a - b)) <= 1e-10


ALL_PINS = [
    pin_splitmix_golden,
    pin_uniform_exact,
    pin_initial_field,
    pin_laplacian_symbol,
    pin_rhs_constant,
    pin_rhs_nonlinear_x,
    pin_rhs_nonlinear_y,
    pin_penta_dense_lu,
    pin_penta_eigenvectors,
    pin_penta_constant,
    pin_mode_amplification,
    pin_nyquist_mode_exact,
    pin_mass_conservation,
    pin_energy_monotone,
    pin_dFdt_is_time_derivative,
    pin_constant_field_observables,
    pin_single_mode_energy,
    pin_interface_energy,
    pin_run_sampling,
    pin_moments_discrete_uniform,
    pin_moments_two_point,
    pin_moments_library_with_nonfinite,
    pin_histogram_brute_force,
    pin_trend_closed_forms,
    pin_refinement_prolongation_and_linear,
    pin_refinement_fourier_mode,
    pin_dp_quadrature_orders,
    pin_dp_linear_stability,
    pin_drop_single_and_invariants,
    pin_drop_observables_identity,
    pin_drop_dFdt_is_derivative,
    pin_drop_convergence_order,
    pin_drop_extinction,
]
