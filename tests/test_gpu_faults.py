"""Host-side fault injection (ch_set_fault): the library's error paths under failures made
on the host, never on the device.

- an allocation that reports failure: the call returns CH_ENOMEM with a message, leaves no
  handle, and every byte it had allocated is released (device free memory unchanged);
- a NaN written into a member's field: that member's observables report CH_ENONFINITE, the
  others stay finite, and the handle stays usable;
- a stalled serving worker: a short wait returns CH_ETIMEOUT, a later one the result.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch

pytestmark = pytest.mark.gpu

TWO_PI = 2 * math.pi


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(autouse=True)
def disarm():
    ch.ch_set_fault(None)
    yield
    ch.ch_set_fault(None)


def free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def create(prec=ch.CH_FP64, nx=64, ny=48):
    return ch.Ensemble.create(nx, ny, TWO_PI, 0.01, 1e-3, [0.0, 0.3], 7, prec)


# create_common allocates 7 device buffers, then the tile tables 6 more: fail each in turn
@pytest.mark.parametrize("n", [1, 2, 4, 7, 8, 10, 13])
def test_failed_allocation_during_create_leaks_nothing(n):
    torch = pytest.importorskip("torch")
    with create():  # context, module and the allocator's pools already in place
        pass
    free0 = free_bytes(torch)
    ch.ch_set_fault("alloc:%d" % n)
    with pytest.raises(ch.ChError) as e:
        create()
    assert e.value.code == ch.CH_ENOMEM
    assert "memory" in str(e.value).lower() or "alloc" in str(e.value).lower()
    assert free_bytes(torch) == free0
    with create() as h:  # the fault fired once: the next creation succeeds
        h.step(3)


def test_failed_allocation_in_sampling_leaves_the_handle_usable():
    with create() as h:
        ch.ch_set_fault("alloc")
        with pytest.raises(ch.ChError) as e:
            h.set_sampling(5, 0.0, capacity=32)
        assert e.value.code == ch.CH_ENOMEM
        h.set_sampling(5, 0.0, capacity=32)
        h.step(20)
        assert h.series(0, 32).shape[0] == 4


def test_failed_allocation_in_server_create():
    torch = pytest.importorskip("torch")
    with ch.Server(16 << 20, ch.CH_FP32):
        pass
    free0 = free_bytes(torch)
    ch.ch_set_fault("alloc:3")
    with pytest.raises(ch.ChError) as e:
        ch.Server(16 << 20, ch.CH_FP32)
    assert e.value.code == ch.CH_ENOMEM
    assert free_bytes(torch) == free0


@pytest.mark.parametrize("prec,nx,ny", [(ch.CH_FP64, 64, 48), (ch.CH_FP32, 128, 64), (ch.CH_FP32, 40, 56)])
def test_injected_nan_is_reported_for_its_member(prec, nx, ny):
    # (FP32 128 x 64 runs in the cluster-resident form, 40 x 56 in the tiled kernels)
    with create(prec, nx, ny) as h:
        h.set_sampling(1, 0.0, capacity=8)
        h.step(2)
        ch.ch_set_fault("nan:1")
        h.step(3)
        with pytest.raises(ch.ChError) as e:
            h.observables()
        assert e.value.code == ch.CH_ENONFINITE
        assert "not finite" in ch.ch_last_error()
        s0, s1 = h.series(0, 8), h.series(1, 8)
        assert np.all(np.isfinite(s0[:, 1:3]))
        assert not np.all(np.isfinite(s1[-1, 1:3]))
        assert np.all(np.isfinite(h.field(0)))
        h.step(1)  # still usable


def test_injected_stall_times_out_a_short_wait():
    with ch.Server(64 << 20, ch.CH_FP32) as s:
        ch.ch_set_fault("timeout:1500")
        rid = s.submit(nx=64, ny=64, L=TWO_PI, gamma=0.005, dt=1e-3, C0=0.2, seed=3, nsteps=200)
        with pytest.raises(ch.ChError) as e:
            s.wait(rid, 0.2)
        assert e.value.code == ch.CH_ETIMEOUT
        res = s.wait(rid, 60.0)
        assert res["steps"] == 200 and math.isfinite(res["F"])


@pytest.mark.parametrize("n", [9, 11, 14])
def test_failed_allocation_in_server_tiles_leaks_nothing(n):
    # the server's tile tables are allocated after its buffers: fail one of them
    torch = pytest.importorskip("torch")
    with ch.Server(16 << 20, ch.CH_FP32):
        pass
    free0 = free_bytes(torch)
    ch.ch_set_fault("alloc:%d" % n)
    try:
        ch.Server(16 << 20, ch.CH_FP32).close()
    except ch.ChError as e:
        assert e.code == ch.CH_ENOMEM
    ch.ch_set_fault(None)
    assert free_bytes(torch) == free0
