"""Seeded synthetic workloads: member lists, C0 values and request streams.

Pure input generation, shared by the tests, the benchmark and the oracle runs; it holds
none of the method's arithmetic (the initial fields themselves are drawn inside the
library and inside the oracle, each from its own SplitMix64).  The shapes follow the
paper's workload (Sec. 4.1: ensembles of M runs of one size, uniform random initial
noise about a mean concentration, symmetric and asymmetric mixtures) at the sizes of the
five workloads below.
"""
import math

import numpy as np

BASE_SEED = 1911033860
TWO_PI = 2.0 * math.pi

# Workload presets (L = 2 pi everywhere; gamma, dt, sizes and horizons per preset).
SINGLE_64 = dict(name="single-64x64-fp64", nx=64, ny=64, L=TWO_PI, gamma=0.01, dt=1e-3, steps=2000,
                 C0=[0.0], every=1)
ENSEMBLE_256 = dict(name="ensemble-256x(256x256)-fp64", nx=256, ny=256, L=TWO_PI, gamma=0.005, dt=1e-3,
                    steps=20000, C0=[0.0] * 128 + [0.4] * 128, every=100, t1=4.0)
UNEVEN = dict(name="uneven-64x128^2+32x256^2+8x512^2", gamma=0.005, dt=1e-3, L=TWO_PI, steps=2000,
              groups=[(64, 128), (32, 256), (8, 512)], C0_cycle=[0.0, 0.2, 0.4])
SERVING = dict(name="serving-poisson-50/s", rate=50.0, requests=2000, sizes=[64, 128, 256, 512, 1024],
               horizon=(1000, 50000), C0=(0.0, 0.5), gamma=0.005, dt=1e-3, L=TWO_PI)
LONG_1024 = dict(name="long-32x(1024x1024)", nx=1024, ny=1024, L=TWO_PI, gamma=0.0025, dt=5e-4,
                 steps=200000, C0=[0.0] * 16 + [0.3] * 16)


def uneven_members(preset=UNEVEN, seed=BASE_SEED):
    """Member descriptors (dicts for ch_create_batch) of the uneven batch, in group order.

    Every member draws from one SplitMix64 stream (`seed`) at its own counter range.
    """
    out = []
    base = 0
    k = 0
    for count, n in preset["groups"]:
        for _ in range(count):
            out.append(dict(nx=n, ny=n, L=preset["L"], gamma=preset["gamma"], dt=preset["dt"],
                            C0=preset["C0_cycle"][k % len(preset["C0_cycle"])], seed=seed, counter_base=base))
            base += n * n
            k += 1
    return out


def request_stream(preset=SERVING, seed=BASE_SEED, count=None, rate=None):
    """Poisson arrivals of single-run requests: list of dicts with arrival time (s), size,
    horizon (steps), C0 and a per-request seed."""
    rng = np.random.default_rng(seed)
    n = count if count is not None else preset["requests"]
    lam = rate if rate is not None else preset["rate"]
    gaps = rng.exponential(1.0 / lam, size=n)
    t = np.cumsum(gaps) - gaps[0]
    sizes = rng.choice(preset["sizes"], size=n)
    lo, hi = preset["horizon"]
    horizons = rng.integers(lo, hi + 1, size=n)
    c0 = rng.uniform(preset["C0"][0], preset["C0"][1], size=n)
    seeds = rng.integers(1, 2 ** 63 - 1, size=n, dtype=np.int64)
    return [dict(arrival=float(t[i]), nx=int(sizes[i]), ny=int(sizes[i]), steps=int(horizons[i]), C0=float(c0[i]),
                 seed=int(seeds[i]), L=preset["L"], gamma=preset["gamma"], dt=preset["dt"]) for i in range(n)]


def random_field(ny, nx, seed, amplitude=0.1, mean=0.0):
    """A seeded i.i.d. uniform test field (numpy generator), for tests that set fields."""
    rng = np.random.default_rng(seed)
    return mean + amplitude * (2.0 * rng.random((ny, nx)) - 1.0)


def beta_ensemble(members, samples, seed=BASE_SEED, t_end=100.0, beta0=0.28, k=0.0056, diverged=0):
    """A seeded synthetic ensemble of beta series with the structure the paper reports
    (Secs. 3.3, 4.2): every run fluctuates about a common beta0, the spread grows like
    sqrt(k t) and the law has a positive tail.  Returns (t, beta): t of shape (samples,)
    from 0 to t_end, beta of shape (members, samples).  The last `diverged` runs turn NaN
    half way (runs whose F or dF/dt stopped being finite).  Inputs for the statistics
    tests; a stand-in for the paper's runs, not a model of them."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, t_end, samples)
    g = rng.standard_normal((members, samples))
    e = rng.exponential(size=(members, samples))
    z = (g + 0.5 * (e - 1.0)) / math.sqrt(1.25)
    beta = beta0 + np.sqrt(k * t)[None, :] * z
    if diverged:
        beta[members - diverged:, samples // 2:] = np.nan
    return t, beta


# Appendix A grid-refinement study: [0, 2 pi]^2, gamma = 0.01, final time T = 10,
# dt = 0.1 dx per grid, a single-droplet start; E_n compares the n-grid with the n/2-grid.
# The grids start at 128: with dt = 0.1 dx the 64-grid has dt/gamma = 0.98, and the
# scheme's amplification factor about C = +-1 then reaches -1.14 for some modes (the run
# diverges); at 128 (dt/gamma = 0.49) every mode stays within [-0.78, 1].
REFINEMENT = dict(name="appendix-A refinement study", L=TWO_PI, gamma=0.01, T=10.0, cfl=0.1,
                  sizes=[128, 256, 512, 1024, 2048, 4096, 8192])


def droplet_field(n, L=TWO_PI, gamma=0.01):
    """The single-droplet start of the refinement study on an n x n grid (row-major (y, x)):
    C = tanh((r - L/2) / sqrt(2 gamma)), r the periodic distance of the cell centre
    ((i + 1/2) L/n, (j + 1/2) L/n) from the origin.  tanh(d / sqrt(2 gamma)) is the
    equilibrium profile across a flat interface of the free energy 1/4 (C^2 - 1)^2 +
    gamma/2 |grad C|^2, so the start is smooth on every grid of the study."""
    h = L / n
    x = (np.arange(n) + 0.5) * h
    d = np.minimum(x, L - x)
    r = np.sqrt(d[None, :] ** 2 + d[:, None] ** 2)
    return np.tanh((r - 0.5 * L) / math.sqrt(2.0 * gamma))


def refinement_steps(n, preset=REFINEMENT):
    """(steps, dt) of the n-grid: dt nominally cfl * dx, rounded so that every grid ends
    exactly at T."""
    dx = preset["L"] / n
    steps = max(1, int(round(preset["T"] / (preset["cfl"] * dx))))
    return steps, preset["T"] / steps


# The paper's Cahn-Hilliard campaign (Sec. 4.1-4.2, Tables 3-4): M = 1024 runs per domain
# size L, gamma = 0.01, dt = 0.0012, dx = 2 pi / 256 (Sec. 4.1's resolution; Table 3's
# caption says 2 pi / 512), t up to 100, asymmetric mixtures; Table 4 reports the window
# mean of mu_1 over [20, 100] and k of mu_2 = k t fitted on the same window.
CAMPAIGN = dict(name="paper-campaign-asymmetric", gamma=0.01, dt=0.0012, dx=TWO_PI / 256, T=100.0,
                Ls=[TWO_PI, 2 * TWO_PI, 4 * TWO_PI, 8 * TWO_PI], M=1024, every=10, window=(20.0, 100.0),
                table4={"2pi": (0.33, 0.036), "4pi": (0.28, 0.0056), "8pi": (0.28, 0.0013), "16pi": (0.28, 0.00031)},
                # Sec. 4.3, Table 5 (symmetric mixtures; the paper discards L = 2 pi)
                table5={"4pi": (0.356, 0.0011), "8pi": (0.346, 0.00025), "16pi": (0.346, 0.00062)})


def asymmetric_field(n, seed, member):
    """Sec. 4.1's asymmetric start on an n x n grid: C = 0.5 + 0.1 (r - 1), r i.i.d. uniform
    on [0, 1) (numpy's generator, one stream per (seed, member))."""
    rng = np.random.default_rng([seed, member])
    return 0.5 + 0.1 * (rng.random((n, n)) - 1.0)


# Model 1 (Secs. 2-3): ensembles of M = 100 droplet populations of N droplets each, radii
# drawn uniformly from [0, 1) (Eq. (38)), N = 512 ... 8192 (Table 1), t up to 40, eps = 1e-3.
DROPLETS = dict(name="model1-droplet-ensembles", M=100, Ns=[512, 1024, 2048, 4096, 8192], T=40.0, eps=1e-3,
                rtol=1e-6, atol=1e-9, h0=1e-6, sample_dt=0.1, window=(20.0, 40.0), fit=(0.0, 40.0),
                table2={512: (0.24, 0.0075), 1024: (0.2613, 0.0036), 2048: (0.2833, 0.0017),
                        4096: (0.2908, 8.6e-4), 8192: (0.2995, 4.5e-4)})


def droplet_radii(M, N, seed=BASE_SEED):
    """Initial radii of M populations of N droplets, i.i.d. uniform on [0, 1): (M, N)."""
    return np.random.default_rng([seed, N]).random((M, N))
