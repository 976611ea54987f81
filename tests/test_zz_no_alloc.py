"""The allocation-free objective entry point agrees with spg_objective and
with the FP64 oracle.

Some callers cannot allocate device memory themselves: code whose device
memory is owned entirely by another pool (a framework's caching allocator,
a fixed arena), or latency-critical paths where the implicit device
synchronisation of cudaMalloc is not acceptable. spg_objective_noalloc serves
them with a fixed scratch area inside the library. These tests call it
through the C ABI twice in a row (the scratch is shared and keeps the
previous call's contents), compare each result with the context-based
spg_objective and with the oracle on the same inputs, and call it from a
second CUDA context made current with the driver API, where the scratch
array has another device address. The file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu

SHAPE = (37, 45, 70)


def _case(seed):
    """Inputs at a non-zero iterate with non-uniform weights, and the
    objective spg_objective reports for them."""
    hyper = dict(synth.DEFAULT_HYPER)
    vol = synth.make_volume(SHAPE, blobs=20, radius=9, seed=seed)
    s = spg.SPG(dict(shape=SHAPE, **hyper))
    s.set_data(0, vol.b, vol.w)
    s.reweight()
    s.iterate(15)
    s.reweight()  # weights from a non-zero iterate
    want = s.objective(0)
    sv = spg.parse_state(s.get_state(), [SHAPE])["volumes"][0]
    s.close()
    arrs = {k: np.ascontiguousarray(v, dtype=np.float32)
            for k, v in dict(x=sv["x"], b=vol.b, w=vol.w, om1=sv["om1"], omtv=sv["omtv"]).items()}
    p = oracle.Params(SHAPE, **hyper)
    ref = oracle.objective(arrs["x"], arrs["b"], arrs["w"], arrs["om1"], arrs["omtv"], p)
    return hyper, arrs, want, ref


def _call(lib, hyper, ptrs, out_ptr, stream):
    return lib.spg_objective_noalloc(SHAPE[2], SHAPE[1], SHAPE[0], ctypes.c_float(hyper["lambda_l1"]),
                                     ctypes.c_float(hyper["lambda_tv"]), ctypes.c_float(hyper["mu"]),
                                     *[ctypes.c_void_p(q) for q in ptrs], ctypes.c_void_p(out_ptr),
                                     ctypes.c_void_p(stream))


def test_objective_noalloc_matches_objective_and_oracle_twice():
    lib = spg.load()
    results = []
    for seed in (11, 12):
        hyper, arrs, want, ref = _case(seed)
        dev = {k: torch.from_numpy(v).cuda() for k, v in arrs.items()}
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        ptrs = [dev[k].data_ptr() for k in ("x", "b", "w", "om1", "omtv")]
        st = _call(lib, hyper, ptrs, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == spg.SPG_OK, lib.spg_noalloc_last_error()
        assert lib.spg_noalloc_last_error() == b"no error"
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-6)
        np.testing.assert_allclose(got, ref, rtol=1e-6)
        results.append(got)
    assert not np.allclose(results[0], results[1])


def test_objective_noalloc_in_a_second_driver_context():
    """A context created with the driver API and made current (as a host
    application that manages its own contexts does): the entry point looks up
    the scratch array's address in that context, and afterwards still the
    right one in the primary context."""
    lib = spg.load()
    hyper, arrs, want, ref = _case(13)
    torch.cuda.synchronize()
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    ctx = ctypes.c_void_p()
    assert cu.cuCtxCreate_v4(ctypes.byref(ctx), None, 0, dev) == 0  # pushed: current on this thread
    got = []
    try:
        bufs = {}
        try:
            for k, v in list(arrs.items()) + [("out", np.zeros(4))]:
                ptr = ctypes.c_uint64()
                assert cu.cuMemAlloc_v2(ctypes.byref(ptr), ctypes.c_size_t(v.nbytes)) == 0
                bufs[k] = ptr
                assert cu.cuMemcpyHtoD_v2(ptr, v.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(v.nbytes)) == 0
            ptrs = [bufs[k].value for k in ("x", "b", "w", "om1", "omtv")]
            for _ in range(2):
                host = np.full(4, np.nan)
                assert cu.cuMemcpyHtoD_v2(bufs["out"], host.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(32)) == 0
                st = _call(lib, hyper, ptrs, bufs["out"].value, 0)
                assert st == spg.SPG_OK, lib.spg_noalloc_last_error()
                assert cu.cuCtxSynchronize() == 0
                assert cu.cuMemcpyDtoH_v2(host.ctypes.data_as(ctypes.c_void_p), bufs["out"], ctypes.c_size_t(32)) == 0
                got.append(host.copy())
        finally:
            for ptr in bufs.values():
                cu.cuMemFree_v2(ptr)
    finally:
        popped = ctypes.c_void_p()
        assert cu.cuCtxPopCurrent_v2(ctypes.byref(popped)) == 0
        assert cu.cuCtxDestroy_v2(ctx) == 0
    for g in got:
        np.testing.assert_allclose(g, want, rtol=1e-6)
        np.testing.assert_allclose(g, ref, rtol=1e-6)
    # back in the primary context
    devt = {k: torch.from_numpy(v).cuda() for k, v in arrs.items()}
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    st = _call(lib, hyper, [devt[k].data_ptr() for k in ("x", "b", "w", "om1", "omtv")], out.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
    assert st == spg.SPG_OK, lib.spg_noalloc_last_error()
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-6)


def test_objective_noalloc_rejects_too_many_planes():
    lib = spg.load()
    dummy = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.spg_objective_noalloc(1, 1, 4097, ctypes.c_float(0.05), ctypes.c_float(0.1), ctypes.c_float(1e-3),
                                   p, p, p, p, p, ctypes.c_void_p(out.data_ptr()), None)
    assert st == spg.SPG_EINVAL
    assert b"4096" in lib.spg_noalloc_last_error()
