"""ctypes wrapper around oracle/ch_oracle.c (plain FP64 reference, one thread).

TEST INFRASTRUCTURE ONLY.  Every method forwards to the C oracle; the scheme it follows
(Sec. 1 Eqs. (3), (4), (6); Sec. 3.3 Eq. (42); Sec. 4.1 of the paper) is stated in
ch_oracle.c.  No code is shared with the CUDA library.  `Oracle(path)` can load another
build of the same source (the pin tests load deliberately mutated builds to show that
the pins catch mistakes).
"""
import ctypes
import numpy as np

from . import build as _build

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i, _d, _u64, _i64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64

_SIGS = {
    "or_splitmix64": (_u64, [_u64, _u64]),
    "or_uniform": (_d, [_u64, _u64]),
    "or_initial_field": (None, [_i, _i, _d, _u64, _u64, _dp]),
    "or_laplacian": (None, [_i, _i, _d, _d, _dp, _dp]),
    "or_rhs": (None, [_i, _i, _d, _d, _d, _d, _dp, _dp, _dp]),
    "or_cyclic_penta_solve": (_i, [_i, _d, _dp, _dp]),
    "or_observables": (None, [_i, _i, _d, _d, _d, _dp, _dp, _dp, _dp]),
    "or_beta": (_d, [_d, _d, _d]),
    "or_step": (_i, [_i, _i, _d, _d, _d, _dp, _dp]),
    "or_field_observables": (_i, [_i, _i, _d, _d, _dp, _dp, _dp]),
    "or_run": (_i, [_i, _i, _d, _d, _d, _dp, _i64, _i64, _i, _d, _dp, _i64, _i64p, _dp, _i64p]),
    "or_beta_moments": (None, [_i64, _i64, _i64, _dp, _dp]),
    "or_beta_histogram": (_i, [_i64, _i64, _i64, _dp, _d, _d, _i, _i64p]),
    "or_beta_trend": (None, [_i64, _dp, _dp, _dp, _d, _d, _d, _d, _dp]),
    "or_refinement_error": (_d, [_i, _i, _dp, _dp]),
    "or_drop_observables": (None, [_i, _dp, _dp, _dp, _dp]),
    "or_drop_run": (_i, [_i, _dp, _d, _i, _dp, _d, _d, _d, _d, _i64, _dp, _i64p]),
    "or_dp_poly_step": (_d, [_i, _d, _d, _d, _dp]),
    "or_dp_lin_step": (_d, [_d, _d, _d, _dp]),
}


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class RunResult:
    def __init__(self, C, series, beta_sum, beta_count):
        self.C = C
        self.series = series  # (nsamples, 4): t, F, dFdt, beta
        self.beta_sum = beta_sum
        self.beta_count = beta_count

    @property
    def beta_avg(self):
        return self.beta_sum / self.beta_count if self.beta_count else float("nan")


class Oracle:
    def __init__(self, path=None):
        L = ctypes.CDLL(path or _build.build())
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        self._L = L

    def splitmix64(self, seed, k):
        return int(self._L.or_splitmix64(seed, k))

    def uniform(self, seed, k):
        return float(self._L.or_uniform(seed, k))

    def initial_field(self, nx, ny, C0, seed, counter_base=0):
        """C = C0 + 0.1(2u-1) on an ny x nx grid (row-major, x fastest)."""
        C = np.empty((ny, nx), dtype=np.float64)
        self._L.or_initial_field(nx, ny, C0, seed, counter_base, _ptr(C))
        return C

    def laplacian(self, v, hx, hy):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty_like(v)
        ny, nx = v.shape
        self._L.or_laplacian(nx, ny, hx, hy, _ptr(v), _ptr(out))
        return out

    def rhs(self, C, hx, hy, gamma, dt):
        """(mu, R): mu = C^3 - C - gamma lap_h C, R = dt lap_h mu."""
        C = np.ascontiguousarray(C, dtype=np.float64)
        ny, nx = C.shape
        mu = np.empty_like(C)
        R = np.empty_like(C)
        self._L.or_rhs(nx, ny, hx, hy, gamma, dt, _ptr(C), _ptr(mu), _ptr(R))
        return mu, R

    def penta_solve(self, s, r):
        """x with (I + s D^4) x = r on a periodic line (cyclic pentadiagonal)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        x = np.empty_like(r)
        rc = self._L.or_cyclic_penta_solve(r.shape[0], s, _ptr(r), _ptr(x))
        if rc != 0:
            raise ValueError("or_cyclic_penta_solve rc=%d" % rc)
        return x

    def observables(self, C, mu, hx, hy, gamma):
        C = np.ascontiguousarray(C, dtype=np.float64)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        ny, nx = C.shape
        F, D = _d(), _d()
        self._L.or_observables(nx, ny, hx, hy, gamma, _ptr(C), _ptr(mu), ctypes.byref(F), ctypes.byref(D))
        return F.value, D.value

    def field_observables(self, C, L, gamma):
        C = np.ascontiguousarray(C, dtype=np.float64)
        ny, nx = C.shape
        F, D = _d(), _d()
        rc = self._L.or_field_observables(nx, ny, L, gamma, _ptr(C), ctypes.byref(F), ctypes.byref(D))
        if rc != 0:
            raise ValueError("or_field_observables rc=%d" % rc)
        return F.value, D.value

    def beta(self, t, F, dFdt):
        return float(self._L.or_beta(t, F, dFdt))

    def step(self, C, L, gamma, dt, with_obs=False):
        """One step in place on the (ny, nx) float64 array C; returns (F, dFdt) of C^n if asked."""
        assert C.dtype == np.float64 and C.flags["C_CONTIGUOUS"]
        ny, nx = C.shape
        obs = np.zeros(2)
        rc = self._L.or_step(nx, ny, L, gamma, dt, _ptr(C), _ptr(obs) if with_obs else None)
        if rc != 0:
            raise ValueError("or_step rc=%d" % rc)
        return (obs[0], obs[1]) if with_obs else None

    def run(self, C, L, gamma, dt, nsteps, every=1, t1=0.0, n0=0):
        """Advance a copy of C by nsteps steps from step index n0, sampling every `every` steps."""
        C = np.array(C, dtype=np.float64, order="C", copy=True)
        ny, nx = C.shape
        nmax = max(1, (nsteps + every - 1) // every + 1)
        series = np.zeros((nmax, 4))
        ns, bsum, bcnt = _i64(0), _d(0.0), _i64(0)
        rc = self._L.or_run(nx, ny, L, gamma, dt, _ptr(C), n0, nsteps, every, t1, _ptr(series), nmax,
                            ctypes.byref(ns), ctypes.byref(bsum), ctypes.byref(bcnt))
        if rc != 0:
            raise ValueError("or_run rc=%d" % rc)
        return RunResult(C, series[: ns.value].copy(), bsum.value, bcnt.value)

    # ---- ensemble statistics of beta (Sec. 3.3 Eqs. (41a,b), (42); Sec. 1 Eq. (7)) ----
    def beta_moments(self, beta):
        """beta: (M, T) array, run j's beta at sample s.  Returns (T, 5): count of finite
        values, mu_1, mu_2, mu_3, mu_4 per sample."""
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        M, T = beta.shape
        out = np.zeros((T, 5))
        if T > 0:
            self._L.or_beta_moments(M, T, T, _ptr(beta), _ptr(out))
        return out

    def beta_histogram(self, beta, lo, hi, nbins):
        """Counts (T, nbins + 2): below lo, nbins bins of width (hi - lo) / nbins, at or above hi."""
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        M, T = beta.shape
        out = np.zeros((T, nbins + 2), dtype=np.int64)
        rc = self._L.or_beta_histogram(M, T, T, _ptr(beta), lo, hi, nbins, out.ctypes.data_as(_i64p))
        if rc != 0:
            raise ValueError("or_beta_histogram rc=%d" % rc)
        return out

    def beta_trend(self, t, mu1, mu2, t1, t2, tf1, tf2):
        """(window mean of mu_1 over [t1, t2], k of mu_2 = k t over [tf1, tf2], samples in
        each window)."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        mu1 = np.ascontiguousarray(mu1, dtype=np.float64)
        mu2 = np.ascontiguousarray(mu2, dtype=np.float64)
        assert t.shape == mu1.shape == mu2.shape
        out = np.zeros(4)
        self._L.or_beta_trend(t.size, _ptr(t), _ptr(mu1), _ptr(mu2), t1, t2, tf1, tf2, _ptr(out))
        return out[0], out[1], int(out[2]), int(out[3])

    # ---- grid-refinement error (Appendix A) ----
    def refinement_error(self, fine, coarse):
        """E_n between a (ny, nx) fine field and its (ny/2, nx/2) coarse counterpart."""
        fine = np.ascontiguousarray(fine, dtype=np.float64)
        coarse = np.ascontiguousarray(coarse, dtype=np.float64)
        ny, nx = fine.shape
        assert coarse.shape == (ny // 2, nx // 2)
        return float(self._L.or_refinement_error(nx, ny, _ptr(fine), _ptr(coarse)))

    # ---- Model 1 droplet populations (Secs. 2-3) ----
    def drop_observables(self, R):
        """(F, dF/dt, droplets with R > 0) of radii R (Eqs. (31), (33))."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        F, D, A = _d(), _d(), _d()
        self._L.or_drop_observables(R.size, _ptr(R), ctypes.byref(F), ctypes.byref(D), ctypes.byref(A))
        return F.value, D.value, int(A.value)

    def drop_run(self, R0, t_end, ts, rtol=1e-6, atol=1e-9, h0=1e-4, eps=1e-3, max_steps=10 ** 7):
        """Integrate one population from R0 to t_end; returns (R(t_end), samples (len(ts), 5):
        t, F, dF/dt, beta, alive; accepted steps, rejected steps)."""
        R = np.array(R0, dtype=np.float64, order="C", copy=True)
        ts = np.ascontiguousarray(ts, dtype=np.float64)
        series = np.full((max(ts.size, 1), 5), np.nan)
        stats = np.zeros(2, dtype=np.int64)
        rc = self._L.or_drop_run(R.size, _ptr(R), t_end, ts.size, _ptr(ts), rtol, atol, h0, eps, max_steps,
                                 _ptr(series), stats.ctypes.data_as(_i64p))
        if rc != 0:
            raise ValueError("or_drop_run rc=%d" % rc)
        return R, series[: ts.size], int(stats[0]), int(stats[1])

    def dp_poly_step(self, p, t, y, h):
        """One Dormand-Prince step of y' = t^p: (fifth-order value, fifth - fourth)."""
        e = _d()
        v = self._L.or_dp_poly_step(p, t, y, h, ctypes.byref(e))
        return v, e.value

    def dp_lin_step(self, lam, y, h):
        """One Dormand-Prince step of y' = lam y: (fifth-order value, fifth - fourth)."""
        e = _d()
        v = self._L.or_dp_lin_step(lam, y, h, ctypes.byref(e))
        return v, e.value


_default = None


def get():
    """The oracle built from oracle/ch_oracle.c (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
