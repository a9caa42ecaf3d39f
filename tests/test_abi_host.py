"""CPU checks of the C ABI: exported symbols, argument validation, host-side constants.

No test here launches GPU work: the factorisation query and argument checks return
before any CUDA call.
"""
import os
import re

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import _build
from oracle.oracle import get as get_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?[\s\*])?(ch_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_header_declares_the_core_boundary():
    names = header_functions()
    for required in ["ch_create_ensemble", "ch_step", "ch_observables", "ch_create_batch", "ch_destroy"]:
        assert required in names


def test_library_exports_every_header_symbol():
    L = ch.lib()
    names = header_functions()
    assert names
    for n in names:
        assert hasattr(L, n), "libch.so does not export %s" % n
        assert n in ch._SIGS, "binding lacks %s" % n


def test_version_and_error_paths():
    assert "sm_103a" in ch.ch_version()
    with pytest.raises(ch.ChError) as e:
        ch.ch_create_ensemble(4, 16, 1.0, 0.01, 1e-3, [0.0], 1)
    assert e.value.code == ch.CH_EINVAL
    for bad in [dict(L=0.0), dict(gamma=-1.0), dict(dt=float("nan"))]:
        kw = dict(nx=8, ny=8, L=1.0, gamma=0.01, dt=1e-3)
        kw.update(bad)
        with pytest.raises(ch.ChError) as e:
            ch.ch_create_ensemble(kw["nx"], kw["ny"], kw["L"], kw["gamma"], kw["dt"], [0.0], 1)
        assert e.value.code == ch.CH_EINVAL
    with pytest.raises(ch.ChError):
        ch.ch_create_ensemble(8, 8, 1.0, 0.01, 1e-3, [float("inf")], 1)
    with pytest.raises(ch.ChError):
        ch.ch_create_ensemble(8, 8, 1.0, 0.01, 1e-3, [0.0], 1, precision=7)
    with pytest.raises(ch.ChError):
        ch.ch_penta_factor(-1.0)
    assert "must" in ch.ch_last_error() or "s" in ch.ch_last_error()


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(ch, "_lib", None)
    monkeypatch.setattr(ch, "lib_path", "/nonexistent/libch.so")
    with pytest.raises(RuntimeError):
        ch.lib()


def _dense(n, s):
    P = np.roll(np.eye(n), 1, axis=1)
    P2 = P @ P
    return (1 + 6 * s) * np.eye(n) - 4 * s * (P + P.T) + s * (P2 + P2.T)


@pytest.mark.parametrize("s", [1e-6, 1e-3, 0.107, 1.0, 13.8, 880.0, 1e4, 1e6])
def test_factor_reconstructs_operator(s):
    c, p1, p2, K = ch.ch_penta_factor(s)
    n = 12
    P = np.roll(np.eye(n), 1, axis=1)  # (P y)_i = y_{i-1}... as a circulant shift
    Q = np.eye(n) - p1 * P.T - p2 * (P.T @ P.T)
    A = c * Q @ Q.T
    assert np.max(np.abs(A - _dense(n, s))) <= 1e-13 * (1 + 16 * s)
    assert 0 < -p2 < 1 and K > 0
    _, _, _, K32 = ch.ch_penta_factor(s, ch.CH_FP32)
    assert K32 < K


def preroll_solve_model(r, c, p1, p2, K, chunks):
    """numpy model of the sweep the kernels run: chunked, pre-rolled forward then backward
    recurrences, then division by c.  Test helper only."""
    n = r.size
    bounds = np.linspace(0, n, chunks + 1).astype(int)
    y = np.zeros(n)
    for a, b in zip(bounds[:-1], bounds[1:]):
        y1 = y2 = 0.0
        for q in range(K):
            k = (a - K + q) % n
            yy = r[k] + p1 * y1 + p2 * y2
            y2, y1 = y1, yy
        for i in range(a, b):
            yy = r[i] + p1 * y1 + p2 * y2
            y[i] = yy
            y2, y1 = y1, yy
    x = np.zeros(n)
    for a, b in zip(bounds[:-1], bounds[1:]):
        x1 = x2 = 0.0
        for q in range(K):
            k = (b - 1 + K - q) % n
            xx = y[k] + p1 * x1 + p2 * x2
            x2, x1 = x1, xx
        for i in range(b - 1, a - 1, -1):
            xx = y[i] + p1 * x1 + p2 * x2
            x[i] = xx
            x2, x1 = x1, xx
    return x / c


@pytest.mark.parametrize("n,s,chunks", [(5, 0.3, 1), (7, 13.8, 1), (16, 880.0, 2), (64, 0.107, 4),
                                        (100, 13.8, 3), (256, 13.8, 1), (300, 1e4, 5)])
def test_preroll_sweep_matches_oracle(n, s, chunks):
    orc = get_oracle()
    c, p1, p2, K = ch.ch_penta_factor(s)
    rng = np.random.default_rng(n)
    r = rng.standard_normal(n)
    ref = orc.penta_solve(s, r)
    got = preroll_solve_model(r, c, p1, p2, K, chunks)
    assert np.max(np.abs(got - ref)) <= 1e-13 * (1 + 16 * s) * np.max(np.abs(ref))


def seg_solve_model(r, c, p1, p2, seg, tabs):
    """numpy model of the segment form of the row sweep: per segment a pass from a zero
    state, the Kogge-Stone scan of the end states with the library's tables, the periodic
    start state and a second pass; forward then backward, then division by c.  Test helper
    only."""
    n = r.size
    G = n // seg
    A, B, P = tabs["A"], tabs["B"], tabs["P"]

    def one(v):
        segs = v.reshape(G, seg)
        e = np.zeros((G, 2))
        for l in range(G):
            a = b = 0.0
            for u in range(seg):
                a, b = segs[l, u] + p1 * a + p2 * b, a
            e[l] = (a, b)
        Y, d = e.copy(), 0
        while (1 << d) < G:
            Y = np.array([Y[l] + (A[d] @ Y[l - (1 << d)] if l >= (1 << d) else 0) for l in range(G)])
            d += 1
        x0 = P @ Y[G - 1]
        out = np.empty((G, seg))
        for l in range(G):
            a, b = B[l] @ x0 + (Y[l - 1] if l else 0)
            for u in range(seg):
                a, b = segs[l, u] + p1 * a + p2 * b, a
                out[l, u] = a
        return out.reshape(n)

    y = one(r)
    return one(y[::-1])[::-1] / c


@pytest.mark.parametrize("n,s,seg", [(16, 0.3, 16), (64, 0.107, 16), (64, 13.8, 32), (256, 13.8, 16),
                                     (512, 220.0, 16), (1024, 3527.0, 32), (32, 5.0, 16)])
def test_segment_sweep_matches_oracle(n, s, seg):
    orc = get_oracle()
    c, p1, p2, _ = ch.ch_penta_factor(s)
    tabs = ch.ch_seg_tables(s, seg, n // seg)
    rng = np.random.default_rng(n + seg)
    r = rng.standard_normal(n)
    ref = orc.penta_solve(s, r)
    got = seg_solve_model(r, c, p1, p2, seg, tabs)
    assert np.max(np.abs(got - ref)) <= 1e-13 * (1 + 16 * s) * np.max(np.abs(ref))


def test_segment_tables_are_matrix_powers():
    # independent of the library's products: powers of the companion matrix by numpy
    s, seg, G = 13.8, 16, 8
    _, p1, p2, _ = ch.ch_penta_factor(s)
    M = np.array([[p1, p2], [1.0, 0.0]])
    t = ch.ch_seg_tables(s, seg, G)
    MS = np.linalg.matrix_power(M, seg)
    for d in range(3):
        assert np.allclose(t["A"][d], np.linalg.matrix_power(MS, 1 << d), rtol=1e-12, atol=1e-15)
    assert not t["A"][3].any() and not t["A"][4].any()
    for l in range(G):
        assert np.allclose(t["B"][l], np.linalg.matrix_power(MS, l), rtol=1e-12, atol=1e-15)
    assert not t["B"][G:].any()
    assert np.allclose(t["P"] @ (np.eye(2) - np.linalg.matrix_power(M, seg * G)), np.eye(2), atol=1e-12)
    for bad in [(s, 16, 3), (s, 0, 4), (s, 16, 64), (-1.0, 16, 4)]:
        with pytest.raises(ch.ChError) as e:
            ch.ch_seg_tables(*bad)
        assert e.value.code == ch.CH_EINVAL


def test_fault_specs_parse_without_gpu_work():
    # arming and disarming touch only host state
    for spec in ["alloc", "alloc:3", "nan", "nan:2", "timeout", "timeout:10", "none", ""]:
        ch.ch_set_fault(spec)
    ch.ch_set_fault(None)
    for bad in ["alloc:0", "alloc:-1", "nan:x", "boom", "timeout:", "alloc:2x"]:
        with pytest.raises(ch.ChError) as e:
            ch.ch_set_fault(bad)
        assert e.value.code == ch.CH_EINVAL
        assert "ch_set_fault" in ch.ch_last_error()
    ch.ch_set_fault(None)
