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
