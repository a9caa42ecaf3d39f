"""FP32 heads of the FP64 pre-rolls (ch_preroll_head, ch_tuning.preroll_head), host side.

The FP64 streaming sweeps start each periodic recurrence y_i = r_i + p1 y_{i-1} +
p2 y_{i-2} (the spectral factor of I + s D^4, Sec. 4.1's pentadiagonal solves) from a
state pre-rolled over the K points before the line; the first `head` of those points run
in FP32.  Here the split is emulated on the CPU (FP32 head with the kernels' truncating
binary64 -> binary32 conversion and single-rounding FMAs, FP64 tail) and its start state
compared with the periodic one computed in extended precision: the head must add nothing
visible to the FP64 pre-roll's own error, while a head 32 points longer must.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def f32_trunc(x):
    """binary64 -> binary32 keeping the top 23 fraction bits (exponent rebiased by 896)."""
    b = np.asarray(x, np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    mag, sign = hi & np.uint32(0x7FFFFFFF), hi & np.uint32(0x80000000)
    body = ((mag - np.uint32(896 << 20)) << np.uint32(3)) | (lo >> np.uint32(29))
    bits = np.where(mag < np.uint32(897 << 20), sign,
                    np.where(mag >= np.uint32(1151 << 20), sign | np.uint32(0x7F800000), sign | body))
    return bits.astype(np.uint32).view(np.float32)


def fmaf(a, b, c):
    # the product of two FP32 values is exact in FP64; one rounding to FP32 after the sum
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def start_state(r, p1, p2, K, head):
    """State (y_{-1}, y_{-2}) after pre-rolling over positions -K .. -1 (mod n), the first
    `head` of them in FP32."""
    n = len(r)
    f1 = f2 = np.float32(0)
    q1, q2 = np.float32(p1), np.float32(p2)
    rf = f32_trunc(r)
    for q in range(head):
        y = fmaf(q1, f1, fmaf(q2, f2, rf[(q - K) % n]))
        f2, f1 = f1, y
    y1, y2 = float(f1), float(f2)
    for q in range(head, K):
        y = p1 * y1 + (p2 * y2 + r[(q - K) % n])
        y2, y1 = y1, y
    return np.array([y1, y2])


def periodic_state(r, p1, p2, K):
    """The periodic solution's state at the line start, in extended precision (a pre-roll
    of 8K points: the truncation is ||M^8K||, far below any rounding here)."""
    n = len(r)
    P1, P2 = np.longdouble(p1), np.longdouble(p2)
    y1 = y2 = np.longdouble(0)
    for q in range(8 * K):
        y = P1 * y1 + P2 * y2 + np.longdouble(r[(q - 8 * K) % n])
        y2, y1 = y1, y
    return np.array([y1, y2])


def s_of(n, L=2 * math.pi, gamma=0.005, dt=1e-3):
    return gamma * dt / (L / n) ** 4


@pytest.mark.parametrize("s", [s_of(32), s_of(64), s_of(128), s_of(256), s_of(512), s_of(1024), 1e-3, 1.0])
def test_head_is_a_multiple_of_16_within_the_preroll(s):
    K, head = ch.ch_preroll_head(s)
    assert K == ch.ch_penta_factor(s, ch.CH_FP64)[3]
    assert head % 16 == 0 and 0 <= head <= K


def test_ensemble_preroll_has_a_head():
    # 256 x 256 over [0, 2 pi)^2, gamma 0.005, dt 1e-3: s = 13.8, K = 110
    K, head = ch.ch_preroll_head(s_of(256))
    assert K == 110 and head == 32


@pytest.mark.parametrize("n,s", [(256, s_of(256)), (32, s_of(256)), (256, s_of(128)), (1024, s_of(1024))])
def test_head_adds_nothing_visible_to_the_fp64_preroll(n, s):
    _, p1, p2, K = ch.ch_penta_factor(s, ch.CH_FP64)
    _, head = ch.ch_preroll_head(s)
    rng = np.random.default_rng(n + int(s))
    r = rng.uniform(-1.0, 1.0, n)
    exact = periodic_state(r, p1, p2, K)
    err64 = np.max(np.abs(start_state(r, p1, p2, K, 0) - exact))
    err_split = np.max(np.abs(start_state(r, p1, p2, K, head) - exact))
    R = np.max(np.abs(r))
    assert err_split <= err64 + 1e-16 * R
    # the FP32 part alone is far from FP64 accuracy: the tail is what makes the state exact
    err32 = np.max(np.abs(start_state(r, p1, p2, K, K) - exact))
    assert err32 > 1e4 * max(err64, 1e-17 * R)


@pytest.mark.parametrize("s", [s_of(256), s_of(128)])
def test_a_longer_head_would_show(s):
    # 32 more FP32 points leave the FP32 rounding too little FP64 damping: visible errors
    n = 256
    _, p1, p2, K = ch.ch_penta_factor(s, ch.CH_FP64)
    _, head = ch.ch_preroll_head(s)
    r = np.random.default_rng(7).uniform(-1.0, 1.0, n)
    exact = periodic_state(r, p1, p2, K)
    err_split = np.max(np.abs(start_state(r, p1, p2, K, head) - exact))
    err_long = np.max(np.abs(start_state(r, p1, p2, K, min(K, head + 32)) - exact))
    assert err_long > 10 * err_split


def test_f32_trunc_fields():
    x = np.array([1.0, -2.5, 3.0e-40, -1e-300, 1e39, np.inf, 0.0, 1.0 + 2.0 ** -30, math.pi])
    y = f32_trunc(x)
    assert y[0] == 1.0 and y[1] == -2.5
    assert y[2] == 0.0 and y[3] == 0.0 and np.signbit(y[3])
    assert np.isinf(y[4]) and np.isinf(y[5]) and y[6] == 0.0
    assert y[7] == 1.0  # truncated, not rounded
    assert abs(float(y[8]) - math.pi) < 2.0 ** -23 * math.pi and float(y[8]) <= math.pi


def test_tuning_field_validated():
    # preroll_head takes -1 or 0; checked before any device work (no handle needed for the
    # struct layout: the binding's Tuning mirrors ch_tuning field for field)
    names = [f for f, _ in ch.Tuning._fields_]
    assert names[-1] == "preroll_head"
