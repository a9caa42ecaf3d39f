"""Python binding of libch (include/ch.h): argument marshalling only.

Every call forwards to the C ABI of the in-tree CUDA library
paper_1911_03386_gb300/_build/libch.so; every step of the Cahn-Hilliard path runs in its
sm_103a kernels.  There is no CPU fallback: if the library is missing or cannot be
loaded, `lib()` raises.  The names follow the C ABI (ch_create_ensemble, ch_step, ...);
`Ensemble` is a small convenience holder of a handle.
"""
import ctypes
import os

import numpy as np

__all__ = [
    "CH_OK", "CH_PENDING", "CH_EINVAL", "CH_ENOMEM", "CH_ECUDA", "CH_ENONFINITE", "CH_ETIMEOUT",
    "CH_EBUSY", "CH_ENOTFOUND", "CH_FP64", "CH_FP32", "ChError", "MemberDesc", "lib", "lib_path",
    "ch_create_ensemble", "ch_create_batch", "ch_destroy", "ch_set_stream", "ch_set_sampling",
    "ch_step", "ch_synchronize", "ch_observables", "ch_beta_avg", "ch_series", "ch_get_field",
    "ch_set_field", "ch_set_fields", "ch_get_fields", "ch_launch_phase", "ch_set_tuning", "ch_get_tuning", "Tuning",
    "ch_get_step", "ch_reset", "ch_num_members", "ch_member_shape",
    "ch_debug_row_solve", "ch_save", "ch_load", "ch_penta_factor", "ch_preroll_head", "ch_seg_tables", "ch_step_field_noalloc", "ch_last_error", "ch_version",
    "CH_MOMENTS", "CH_MAX_BINS", "ch_stats_moments", "ch_stats_histogram", "ch_stats_trend", "ch_ensemble_moments",
    "ch_ensemble_histogram", "ch_ensemble_trend", "ch_refinement_error", "ch_ensemble_refinement_error",
    "ch_droplets_run",
    "Ensemble", "Server", "Request", "Result", "ServerStats", "ch_server_create", "ch_submit", "ch_poll",
    "ch_server_wait", "ch_server_stats", "ch_server_destroy",
]

CH_OK, CH_PENDING = 0, 1
CH_EINVAL, CH_ENOMEM, CH_ECUDA, CH_ENONFINITE, CH_ETIMEOUT, CH_EBUSY, CH_ENOTFOUND = -1, -2, -3, -4, -5, -6, -7
CH_FP64, CH_FP32 = 0, 1
CH_MOMENTS, CH_MAX_BINS = 6, 1024

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "_build", "libch.so")


class ChError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libch error %d: %s" % (code, msg))
        self.code = code


class MemberDesc(ctypes.Structure):
    """ch_member_desc: one run of an uneven batch."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("L", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dt", ctypes.c_double), ("C0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("counter_base", ctypes.c_uint64)]


class Request(ctypes.Structure):
    """ch_request: one single-run request to a server."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("L", ctypes.c_double), ("gamma", ctypes.c_double),
                ("dt", ctypes.c_double), ("C0", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("nsteps", ctypes.c_int64), ("every", ctypes.c_int), ("t1", ctypes.c_double),
                ("field_out", ctypes.POINTER(ctypes.c_double))]


class Result(ctypes.Structure):
    """ch_result: outcome of a served run."""
    _fields_ = [("steps", ctypes.c_int64), ("F", ctypes.c_double), ("dFdt", ctypes.c_double),
                ("beta", ctypes.c_double), ("beta_avg", ctypes.c_double), ("beta_count", ctypes.c_int64),
                ("nonfinite", ctypes.c_int), ("t_queued_s", ctypes.c_double), ("t_run_s", ctypes.c_double),
                ("t_total_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("running", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("max_running", ctypes.c_int64), ("member_steps", ctypes.c_int64),
                ("grid_point_steps", ctypes.c_int64), ("chunks", ctypes.c_int64), ("busy_s", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("arena_bytes", ctypes.c_size_t), ("arena_peak_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    """ch_tuning: launch shape of a handle's kernels (fields <= 0 / split -1: default)."""
    _fields_ = [("split", ctypes.c_int), ("rows_band", ctypes.c_int), ("rows_p", ctypes.c_int),
                ("sweep_band", ctypes.c_int), ("cols_panel", ctypes.c_int), ("cols_p", ctypes.c_int),
                ("threads", ctypes.c_int), ("stream", ctypes.c_int), ("persist", ctypes.c_int),
                ("row_seg", ctypes.c_int), ("col_seg", ctypes.c_int), ("resident", ctypes.c_int),
                ("resident_rows", ctypes.c_int), ("preroll_head", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_c_int, _c_dbl, _c_i64, _c_u64, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "ch_create_ensemble": (_c_int, [_c_int, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_int, _dp, _c_u64, _c_int,
                                    ctypes.POINTER(_vp)]),
    "ch_create_batch": (_c_int, [_c_int, ctypes.POINTER(MemberDesc), _c_int, ctypes.POINTER(_vp)]),
    "ch_destroy": (None, [_vp]),
    "ch_set_stream": (_c_int, [_vp, _vp]),
    "ch_set_sampling": (_c_int, [_vp, _c_int, _c_dbl, _c_i64]),
    "ch_step": (_c_int, [_vp, _c_i64]),
    "ch_synchronize": (_c_int, [_vp]),
    "ch_observables": (_c_int, [_vp, _dp, _dp, _dp]),
    "ch_beta_avg": (_c_int, [_vp, _dp, _i64p]),
    "ch_series": (_c_int, [_vp, _c_int, _dp, _c_i64, _i64p]),
    "ch_get_field": (_c_int, [_vp, _c_int, _dp]),
    "ch_set_field": (_c_int, [_vp, _c_int, _dp]),
    "ch_get_step": (_c_int, [_vp, _c_int, _i64p]),
    "ch_set_fields": (_c_int, [_vp, _vp]),
    "ch_get_fields": (_c_int, [_vp, _vp]),
    "ch_launch_phase": (_c_int, [_vp, _c_int]),
    "ch_set_tuning": (_c_int, [_vp, ctypes.POINTER(Tuning)]),
    "ch_get_tuning": (_c_int, [_vp, ctypes.POINTER(Tuning)]),
    "ch_reset": (_c_int, [_vp]),
    "ch_num_members": (_c_int, [_vp, _ip]),
    "ch_member_shape": (_c_int, [_vp, _c_int, _ip, _ip]),
    "ch_debug_row_solve": (_c_int, [_vp, _c_int, _dp]),
    "ch_save": (_c_int, [_vp, ctypes.c_char_p]),
    "ch_load": (_c_int, [_vp, ctypes.c_char_p]),
    "ch_penta_factor": (_c_int, [_c_dbl, _c_int, _dp, _dp, _dp, _ip]),
    "ch_preroll_head": (_c_int, [_c_dbl, _ip, _ip]),
    "ch_seg_tables": (_c_int, [_c_dbl, _c_int, _c_int, _dp]),
    "ch_step_field_noalloc": (_c_int, [_vp, _c_int, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_i64, _vp]),
    "ch_stats_moments": (_c_int, [_vp, _vp, _c_i64, _c_i64, _c_i64, _vp, _vp]),
    "ch_stats_histogram": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_dbl, _c_dbl, _c_int, _vp, _vp]),
    "ch_stats_trend": (_c_int, [_vp, _c_i64, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _vp, _vp]),
    "ch_ensemble_moments": (_c_int, [_vp, _ip, _c_int, _dp, _c_i64, _i64p]),
    "ch_ensemble_histogram": (_c_int, [_vp, _ip, _c_int, _c_dbl, _c_dbl, _c_int, _i64p, _c_i64, _i64p]),
    "ch_ensemble_trend": (_c_int, [_vp, _ip, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _dp]),
    "ch_refinement_error": (_c_int, [_vp, _vp, _c_int, _c_int, _vp, _vp]),
    "ch_ensemble_refinement_error": (_c_int, [_vp, _c_int, _vp, _c_int, _dp]),
    "ch_droplets_run": (_c_int, [_c_int, _c_int, _dp, _c_dbl, _c_int, _dp, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_i64,
                                 _dp, _i64p, _vp]),
    "ch_server_create": (_c_int, [ctypes.c_size_t, _c_int, _c_int, ctypes.POINTER(_vp)]),
    "ch_submit": (_c_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "ch_poll": (_c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "ch_server_wait": (_c_int, [_vp, ctypes.c_uint64, _c_dbl, ctypes.POINTER(Result)]),
    "ch_server_stats": (_c_int, [_vp, ctypes.POINTER(ServerStats)]),
    "ch_server_destroy": (None, [_vp]),
    "ch_fma_peak": (_c_int, [_c_int, _c_int, _c_int, _c_i64, _vp, _vp, _dp]),
    "ch_set_fault": (_c_int, [ctypes.c_char_p]),
    "ch_last_error": (ctypes.c_char_p, []),
    "ch_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libch (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise RuntimeError("libch.so is not built (%s); run __graft_entry__.build()" % lib_path)
        L = ctypes.CDLL(lib_path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, ok=(CH_OK,)):
    if rc not in ok:
        raise ChError(rc, lib().ch_last_error().decode())
    return rc


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp)


def ch_last_error():
    return lib().ch_last_error().decode()


def ch_version():
    return lib().ch_version().decode()


def ch_penta_factor(s, precision=CH_FP64):
    """(c, p1, p2, K) of I + s D^4 = c Q Q^T (host computation, no GPU)."""
    c, p1, p2, K = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().ch_penta_factor(s, precision, ctypes.byref(c), ctypes.byref(p1), ctypes.byref(p2), ctypes.byref(K)))
    return c.value, p1.value, p2.value, K.value


def ch_preroll_head(s):
    """(K, head) of the FP64 pre-roll of I + s D^4: its length and the leading points the
    FP64 streaming sweeps run in FP32 (host computation, no GPU)."""
    K, head = ctypes.c_int(), ctypes.c_int()
    _check(lib().ch_preroll_head(s, ctypes.byref(K), ctypes.byref(head)))
    return K.value, head.value


def ch_seg_tables(s, seg, groups):
    """Scan tables of the segment row sweep (host computation, no GPU): dict with
    A (5 x 2 x 2, M^(seg 2^d)), B (32 x 2 x 2, M^(seg l)) and P (2 x 2, (I - M^n)^-1)."""
    out = np.zeros(152)
    _check(lib().ch_seg_tables(s, seg, groups, _ptr(out)))
    return {"A": out[:20].reshape(5, 2, 2), "B": out[20:148].reshape(32, 2, 2), "P": out[148:].reshape(2, 2)}


def ch_step_field_noalloc(C_ptr, nx, ny, L, gamma, dt, nsteps, stream_ptr=None):
    """Advance a caller-owned FP64 device field (address C_ptr) by nsteps steps without
    allocating anything (scratch in a static 8 MiB device array; nx*ny <= 1048576)."""
    _check(lib().ch_step_field_noalloc(C_ptr, nx, ny, L, gamma, dt, nsteps, stream_ptr or None))


def ch_set_fault(spec):
    """Arm one host-side fault ("alloc[:N]", "nan[:member]", "timeout[:ms]"; None disarms)."""
    _check(lib().ch_set_fault(None if spec is None else spec.encode()))


def ch_fma_peak(precision, blocks, threads, iters, sink_ptr, stream_ptr=None):
    """Enqueue the FMA-throughput kernel (see include/ch.h); returns the flops it performs."""
    flops = ctypes.c_double()
    _check(lib().ch_fma_peak(precision, blocks, threads, iters, sink_ptr, stream_ptr or None, ctypes.byref(flops)))
    return flops.value


def ch_create_ensemble(nx, ny, L, gamma, dt, C0, seed, precision=CH_FP64):
    C0 = _f64(C0).ravel()
    h = _vp()
    _check(lib().ch_create_ensemble(nx, ny, L, gamma, dt, C0.size, _ptr(C0), seed, precision, ctypes.byref(h)))
    return h.value


def ch_create_batch(descs, precision=CH_FP64):
    arr = (MemberDesc * len(descs))()
    for k, d in enumerate(descs):
        arr[k] = d if isinstance(d, MemberDesc) else MemberDesc(**d)
    h = _vp()
    _check(lib().ch_create_batch(len(descs), arr, precision, ctypes.byref(h)))
    return h.value


def ch_destroy(h):
    lib().ch_destroy(h)


def ch_set_stream(h, stream_ptr):
    _check(lib().ch_set_stream(h, stream_ptr or None))


def ch_set_sampling(h, every, t1=0.0, capacity=0):
    _check(lib().ch_set_sampling(h, every, t1, capacity))


def ch_step(h, nsteps):
    _check(lib().ch_step(h, nsteps))


def ch_synchronize(h):
    _check(lib().ch_synchronize(h))


def ch_num_members(h):
    m = ctypes.c_int()
    _check(lib().ch_num_members(h, ctypes.byref(m)))
    return m.value


def ch_member_shape(h, member):
    nx, ny = ctypes.c_int(), ctypes.c_int()
    _check(lib().ch_member_shape(h, member, ctypes.byref(nx), ctypes.byref(ny)))
    return nx.value, ny.value


def ch_observables(h):
    """(F, dFdt, beta) arrays of the current fields."""
    m = ch_num_members(h)
    F, D, B = np.empty(m), np.empty(m), np.empty(m)
    _check(lib().ch_observables(h, _ptr(F), _ptr(D), _ptr(B)))
    return F, D, B


def ch_beta_avg(h):
    m = ch_num_members(h)
    avg = np.empty(m)
    cnt = np.empty(m, dtype=np.int64)
    _check(lib().ch_beta_avg(h, _ptr(avg), cnt.ctypes.data_as(_i64p)))
    return avg, cnt


def ch_series(h, member, cap):
    out = np.zeros((max(cap, 1), 4))
    n = ctypes.c_int64()
    _check(lib().ch_series(h, member, _ptr(out), cap, ctypes.byref(n)))
    return out[: n.value].copy()


# ---- ensemble statistics of beta (dense forms: device pointers as ints) ----
def ch_stats_moments(t_ptr, beta_ptr, members, samples, ld, out_ptr, stream_ptr=None):
    _check(lib().ch_stats_moments(t_ptr, beta_ptr, members, samples, ld, out_ptr, stream_ptr))


def ch_stats_histogram(beta_ptr, members, samples, ld, lo, hi, nbins, out_ptr, stream_ptr=None):
    _check(lib().ch_stats_histogram(beta_ptr, members, samples, ld, lo, hi, nbins, out_ptr, stream_ptr))


def ch_stats_trend(moments_ptr, samples, t1, t2, tf1, tf2, out_ptr, stream_ptr=None):
    _check(lib().ch_stats_trend(moments_ptr, samples, t1, t2, tf1, tf2, out_ptr, stream_ptr))


def _member_list(members):
    if members is None:
        return None, 0, None
    arr = np.ascontiguousarray(members, dtype=np.int32)
    return arr.ctypes.data_as(_ip), arr.size, arr


def ch_ensemble_moments(h, members=None, cap=None):
    """(T, CH_MOMENTS) table: t, count, mu_1 .. mu_4 per sample time."""
    mp, cnt, keep = _member_list(members)
    if cap is None:
        cap = 1 << 20
    out = np.zeros((max(cap, 1), CH_MOMENTS))
    n = ctypes.c_int64()
    _check(lib().ch_ensemble_moments(h, mp, cnt, _ptr(out), cap, ctypes.byref(n)))
    return out[: n.value].copy()


def ch_ensemble_histogram(h, lo, hi, nbins, members=None, cap=None):
    """(T, nbins + 2) int64 counts: below lo, the bins, past the last bin."""
    mp, cnt, keep = _member_list(members)
    if cap is None:
        cap = 1 << 16
    out = np.zeros((max(cap, 1), nbins + 2), dtype=np.int64)
    n = ctypes.c_int64()
    _check(lib().ch_ensemble_histogram(h, mp, cnt, lo, hi, nbins, out.ctypes.data_as(_i64p), cap, ctypes.byref(n)))
    return out[: n.value].copy()


def ch_ensemble_trend(h, t1, t2, tf1, tf2, members=None):
    """(window mean of mu_1, k of mu_2 = k t, samples in the window, samples in the fit)."""
    mp, cnt, keep = _member_list(members)
    out = np.zeros(4)
    _check(lib().ch_ensemble_trend(h, mp, cnt, t1, t2, tf1, tf2, _ptr(out)))
    return out[0], out[1], int(out[2]), int(out[3])


def ch_refinement_error(fine_ptr, coarse_ptr, nx, ny, out_ptr, stream_ptr=None):
    """Appendix A's E between device fields (fine nx x ny, coarse nx/2 x ny/2); out gets
    1 + ny/2 doubles."""
    _check(lib().ch_refinement_error(fine_ptr, coarse_ptr, nx, ny, out_ptr, stream_ptr))


def ch_ensemble_refinement_error(fine_h, fine_member, coarse_h, coarse_member):
    out = ctypes.c_double()
    _check(lib().ch_ensemble_refinement_error(fine_h, fine_member, coarse_h, coarse_member, ctypes.byref(out)))
    return out.value


def ch_droplets_run(R0, t_end, t_samples, rtol=1e-6, atol=1e-9, h0=1e-6, eps=1e-3, max_steps=10 ** 9,
                    stream_ptr=None):
    """Model 1 populations R0 (M, N) to t_end on the GPU: (R(t_end) (M, N), samples
    (M, len(t_samples), 5): t, F, dF/dt, beta, live droplets; steps (M, 3))."""
    R = np.array(R0, dtype=np.float64, order="C", copy=True)
    if R.ndim != 2:
        raise ValueError("R0 must be (M, N)")
    M, N = R.shape
    ts = np.ascontiguousarray(t_samples, dtype=np.float64)
    series = np.zeros((M, max(ts.size, 1), 5))
    steps = np.zeros((M, 3), dtype=np.int64)
    _check(lib().ch_droplets_run(M, N, _ptr(R), t_end, ts.size, _ptr(ts), rtol, atol, h0, eps, max_steps,
                                 _ptr(series), steps.ctypes.data_as(_i64p), stream_ptr))
    return R, series[:, : ts.size].copy(), steps


def ch_get_field(h, member):
    nx, ny = ch_member_shape(h, member)
    out = np.empty((ny, nx))
    _check(lib().ch_get_field(h, member, _ptr(out)))
    return out


def ch_set_field(h, member, field):
    nx, ny = ch_member_shape(h, member)
    f = _f64(field, nx * ny)
    _check(lib().ch_set_field(h, member, _ptr(f)))


def ch_get_step(h, member=0):
    n = ctypes.c_int64()
    _check(lib().ch_get_step(h, member, ctypes.byref(n)))
    return n.value


def ch_set_fields(h, ptr):
    """All members' fields from host memory at address ptr (FP64, member order)."""
    _check(lib().ch_set_fields(h, ptr))


def ch_get_fields(h, ptr):
    _check(lib().ch_get_fields(h, ptr))


def ch_launch_phase(h, phase):
    _check(lib().ch_launch_phase(h, phase))


def ch_set_tuning(h, split=-1, rows_band=0, rows_p=0, sweep_band=0, cols_panel=0, cols_p=0, threads=0, stream=-1,
                  persist=-1, row_seg=0, col_seg=0, resident=0, resident_rows=0, preroll_head=0):
    t = Tuning(split, rows_band, rows_p, sweep_band, cols_panel, cols_p, threads, stream, persist, row_seg, col_seg,
               resident, resident_rows, preroll_head)
    _check(lib().ch_set_tuning(h, ctypes.byref(t)))


def ch_get_tuning(h):
    t = Tuning()
    _check(lib().ch_get_tuning(h, ctypes.byref(t)))
    return t.as_dict()


def ch_reset(h):
    _check(lib().ch_reset(h))


def ch_debug_row_solve(h, member):
    """W = (I + s D_x^4)^-1 dt lap_h mu of member's current field (no state change)."""
    nx, ny = ch_member_shape(h, member)
    out = np.empty((ny, nx))
    _check(lib().ch_debug_row_solve(h, member, _ptr(out)))
    return out


def ch_save(h, path):
    _check(lib().ch_save(h, os.fsencode(path)))


def ch_load(h, path):
    _check(lib().ch_load(h, os.fsencode(path)))


def ch_server_create(hbm_budget_bytes, precision=CH_FP32, max_members=4096):
    s = _vp()
    _check(lib().ch_server_create(hbm_budget_bytes, precision, max_members, ctypes.byref(s)))
    return s.value


def ch_submit(s, nx, ny, L, gamma, dt, C0, seed, nsteps, every=0, t1=-1.0, field_out=None):
    """Queue a run; field_out (optional float64 numpy array of ny*nx) receives the final field."""
    fo = None
    if field_out is not None:
        assert field_out.dtype == np.float64 and field_out.flags["C_CONTIGUOUS"] and field_out.size == nx * ny
        fo = _ptr(field_out)
    r = Request(nx, ny, L, gamma, dt, C0, seed, nsteps, every, t1, fo)
    rid = ctypes.c_uint64()
    _check(lib().ch_submit(s, ctypes.byref(r), ctypes.byref(rid)))
    return rid.value


def ch_poll(s, rid):
    """None while pending, else the result dict (raises on a failed run)."""
    res = Result()
    rc = lib().ch_poll(s, rid, ctypes.byref(res))
    if rc == CH_PENDING:
        return None
    _check(rc)
    return res.as_dict()


def ch_server_wait(s, rid, timeout_s):
    res = Result()
    _check(lib().ch_server_wait(s, rid, timeout_s, ctypes.byref(res)))
    return res.as_dict()


def ch_server_stats(s):
    st = ServerStats()
    _check(lib().ch_server_stats(s, ctypes.byref(st)))
    return st.as_dict()


def ch_server_destroy(s):
    lib().ch_server_destroy(s)


class Server:
    """Owns one libch server; methods forward to the ch_server_* functions."""

    def __init__(self, hbm_budget_bytes, precision=CH_FP32, max_members=4096):
        self.s = ch_server_create(hbm_budget_bytes, precision, max_members)

    def submit(self, **req):
        return ch_submit(self.s, **req)

    def poll(self, rid):
        return ch_poll(self.s, rid)

    def wait(self, rid, timeout_s=600.0):
        return ch_server_wait(self.s, rid, timeout_s)

    def stats(self):
        return ch_server_stats(self.s)

    def close(self):
        if self.s:
            ch_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Owns one libch handle; methods forward to the ch_* functions above."""

    def __init__(self, handle):
        self.h = handle

    @classmethod
    def create(cls, nx, ny, L, gamma, dt, C0, seed, precision=CH_FP64):
        return cls(ch_create_ensemble(nx, ny, L, gamma, dt, C0, seed, precision))

    @classmethod
    def batch(cls, descs, precision=CH_FP64):
        return cls(ch_create_batch(descs, precision))

    def close(self):
        if self.h:
            ch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def m(self):
        return ch_num_members(self.h)

    def step(self, n):
        ch_step(self.h, n)

    def synchronize(self):
        ch_synchronize(self.h)

    def set_sampling(self, every, t1=0.0, capacity=0):
        ch_set_sampling(self.h, every, t1, capacity)

    def observables(self):
        return ch_observables(self.h)

    def beta_avg(self):
        return ch_beta_avg(self.h)

    def series(self, member, cap):
        return ch_series(self.h, member, cap)

    def moments(self, members=None, cap=None):
        return ch_ensemble_moments(self.h, members, cap)

    def histogram(self, lo, hi, nbins, members=None, cap=None):
        return ch_ensemble_histogram(self.h, lo, hi, nbins, members, cap)

    def trend(self, t1, t2, tf1, tf2, members=None):
        return ch_ensemble_trend(self.h, t1, t2, tf1, tf2, members)

    def field(self, member):
        return ch_get_field(self.h, member)

    def set_field(self, member, field):
        ch_set_field(self.h, member, field)

    def set_fields_ptr(self, ptr):
        ch_set_fields(self.h, ptr)

    def get_fields_ptr(self, ptr):
        ch_get_fields(self.h, ptr)

    def launch_phase(self, phase):
        ch_launch_phase(self.h, phase)

    def set_tuning(self, **kw):
        ch_set_tuning(self.h, **kw)

    def tuning(self):
        return ch_get_tuning(self.h)

    def step_index(self, member=0):
        return ch_get_step(self.h, member)

    def reset(self):
        ch_reset(self.h)

    def row_solve(self, member):
        return ch_debug_row_solve(self.h, member)

    def set_stream(self, stream_ptr):
        ch_set_stream(self.h, stream_ptr)

    def save(self, path):
        ch_save(self.h, path)

    def load(self, path):
        ch_load(self.h, path)
