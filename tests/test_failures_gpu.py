"""Host-visible failures on the GPU path, made without faulting the GPU: a
device allocation that cannot succeed, non-finite objectives, and calls in
the wrong order. Each must return a status and leave the library usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu

HYPER = dict(synth.DEFAULT_HYPER)


def small_solve_works():
    shape = (6, 7, 9)
    vol = synth.make_volume(shape, blobs=3, radius=2, seed=91)
    s = spg.SPG(dict(shape=shape, **HYPER))
    s.set_data(0, vol.b, vol.w)
    s.reweight()
    s.iterate(4)
    x = s.get_x(0).cpu().numpy()
    s.close()
    ref = oracle.solve(vol.b, vol.w, oracle.Params(shape, **HYPER), 1, 4)
    return np.linalg.norm(x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


def test_out_of_memory_is_reported_and_released():
    """5000^3 float32 needs 500 GB per array, more than the GPU holds: the
    first iterate allocation fails, spg_create returns SPG_ENOMEM, frees what
    it had allocated, and the library keeps working."""
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(spg.SPGError) as e:
        spg.SPG(dict(shape=(5000, 5000, 5000), **HYPER))
    assert e.value.status == spg.SPG_ENOMEM
    assert "alloc" in str(e.value)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (64 << 20)  # nothing large left behind
    assert small_solve_works()


def test_out_of_memory_in_a_batch():
    """The second volume of a batch makes the allocation impossible."""
    with pytest.raises(spg.SPGError) as e:
        spg.SPG([dict(shape=(8, 8, 8), **HYPER), dict(shape=(4800, 4800, 4800), **HYPER)])
    assert e.value.status == spg.SPG_ENOMEM
    assert small_solve_works()


def test_non_finite_objective_is_flagged():
    """Huge data overflow the float32 objective sums: the step records a
    non-finite history entry and the API reports SPG_ENONFINITE; a new
    context is unaffected."""
    shape = (8, 8, 16)
    b = np.full(shape, 3e37, np.float32)
    w = np.full(shape, 1e30, np.float32)
    s = spg.SPG(dict(shape=shape, **HYPER))
    s.set_data(0, b, w)
    s.reweight()
    with pytest.raises(spg.SPGError) as e:
        s.iterate(2)
        s.objective(0)
    assert e.value.status == spg.SPG_ENONFINITE
    s.close()
    assert small_solve_works()


def test_calls_in_the_wrong_order():
    shape = (4, 4, 4)
    s = spg.SPG(dict(shape=shape, **HYPER))
    for call in (lambda: s.reweight(), lambda: s.iterate(1), lambda: s.certificate(0)):
        with pytest.raises(spg.SPGError) as e:
            call()
        assert e.value.status == spg.SPG_ENOTREADY
    s.close()
    assert small_solve_works()
