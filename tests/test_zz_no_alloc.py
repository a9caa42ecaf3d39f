"""The allocation-free step (ch_step_field_noalloc) against the handle API's step.

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
        e.set_field(0, field)
        e.step(nsteps)
        return e.field(0)


def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    cases = [
        (wl.random_field(48, 64, 3, amplitude=0.5, mean=0.1), 2 * math.pi, 0.01, 1e-3, 30),
        (wl.random_field(56, 40, 4, amplitude=0.3, mean=-0.2), 3.0, 0.005, 2e-3, 25),
    ]
    stream = torch.cuda.Stream()
    for field, L, gamma, dt, nsteps in cases:
        ny, nx = field.shape
        want = handle_result(field, L, gamma, dt, nsteps)
        C = torch.tensor(field, dtype=torch.float64, device="cuda").contiguous()
        torch.cuda.synchronize()
        ch.ch_step_field_noalloc(C.data_ptr(), nx, ny, L, gamma, dt, nsteps, stream.cuda_stream)
        stream.synchronize()
        got = C.cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-13, np.max(np.abs(got - want))


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    C = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ch.ChError) as e:
        ch.ch_step_field_noalloc(C.data_ptr(), 2048, 1024, 1.0, 0.01, 1e-3, 1)
    assert e.value.code == ch.CH_EINVAL
    assert "1048576" in str(e.value)
