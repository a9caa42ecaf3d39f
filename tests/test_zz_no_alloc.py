"""The allocation-free step (ch_step_field_noalloc) against the handle API's step and the oracle.

Callers that cannot allocate device memory -- frameworks that own all device memory
through their own pool, real-time loops that forbid allocation after start-up -- pass
their own device field and get the same step as ch_create_ensemble + ch_step, with the
scratch in a static device array.  Two calls in a row (different grids and parameters)
must each match the handle path; this also checks that the shared scratch carries
nothing from one call into the next.  The file is named to be collected last.
"""
import math

import numpy as np
import pytest

import paper_1911_03386_gb300 as ch
from paper_1911_03386_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def handle_result(field, L, gamma, dt, nsteps):
    ny, nx = field.shape
    with ch.Ensemble.create(nx, ny, L, gamma, dt, [0.0], 1, ch.CH_FP64) as e:
        # the allocation-free step runs every pre-roll point in FP64: so does this handle,
        # and the two round alike
        e.set_tuning(preroll_head=-1)
        e.set_field(0, field)
        e.step(nsteps)
        return e.field(0)


def noalloc_result(torch, field, L, gamma, dt, nsteps, stream):
    ny, nx = field.shape
    C = torch.tensor(field, dtype=torch.float64, device="cuda").contiguous()
    torch.cuda.synchronize()
    ch.ch_step_field_noalloc(C.data_ptr(), nx, ny, L, gamma, dt, nsteps, stream.cuda_stream)
    stream.synchronize()
    return C.cpu().numpy()


def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    cases = [
        (wl.random_field(48, 64, 3, amplitude=0.5, mean=0.1), 2 * math.pi, 0.01, 1e-3, 30),
        (wl.random_field(56, 40, 4, amplitude=0.3, mean=-0.2), 3.0, 0.005, 2e-3, 25),
    ]
    stream = torch.cuda.Stream()
    for field, L, gamma, dt, nsteps in cases:
        want = handle_result(field, L, gamma, dt, nsteps)
        got = noalloc_result(torch, field, L, gamma, dt, nsteps, stream)
        assert np.max(np.abs(got - want)) <= 1e-13, np.max(np.abs(got - want))


# Grids for the oracle comparison: a 64 x 48 field, and two tiny grids whose pre-roll is
# longer than the line, so the recurrences wrap around it (at L = 0.2 on 9 x 7, s = 41
# and the pre-roll runs 144 points over a 9-point row).
ORACLE_CASES = [
    (64, 48, 2 * math.pi, 0.01, 1e-3, 0.1, 100),
    (7, 9, 1.0, 0.002, 1e-3, 0.3, 60),
    (9, 7, 0.2, 0.01, 1e-3, -0.2, 60),
]


@pytest.mark.parametrize("nx,ny,L,gamma,dt,c0,nsteps", ORACLE_CASES)
def test_noalloc_step_matches_oracle(nx, ny, L, gamma, dt, c0, nsteps):
    torch = pytest.importorskip("torch")
    from oracle.oracle import get as get_oracle

    orc = get_oracle()
    start = orc.initial_field(nx, ny, c0, wl.BASE_SEED, 0)
    want = orc.run(start, L, gamma, dt, nsteps).C
    got = noalloc_result(torch, start, L, gamma, dt, nsteps, torch.cuda.Stream())
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - want)) <= 1e-12, np.max(np.abs(got - want))


def test_noalloc_largest_grid_and_no_allocation():
    # 1024 x 1024 is the largest grid the scratch holds; its rows and columns are too long
    # for the default band and panel, so the launch shapes shrink to fit shared memory
    torch = pytest.importorskip("torch")
    n, L, gamma, dt, nsteps = 1024, 2 * math.pi, 0.01, 1e-3, 3
    field = wl.random_field(n, n, 11, amplitude=0.4, mean=0.1)
    want = handle_result(field, L, gamma, dt, nsteps)
    stream = torch.cuda.Stream()
    C = torch.tensor(field, dtype=torch.float64, device="cuda").contiguous()
    first = C.clone()
    torch.cuda.synchronize()
    ch.ch_step_field_noalloc(C.data_ptr(), n, n, L, gamma, dt, nsteps, stream.cuda_stream)
    stream.synchronize()
    got = C.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want))), np.max(np.abs(got - want))
    # a second call allocates no device memory (the first one has loaded the kernels)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ch.ch_step_field_noalloc(first.data_ptr(), n, n, L, gamma, dt, nsteps, stream.cuda_stream)
    stream.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert np.array_equal(first.cpu().numpy(), got)


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    C = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ch.ChError) as e:
        ch.ch_step_field_noalloc(C.data_ptr(), 2048, 1024, 1.0, 0.01, 1e-3, 1)
    assert e.value.code == ch.CH_EINVAL
    assert "1048576" in str(e.value)
