"""The allocation-free objective entry point agrees with spg_objective.

Some callers cannot allocate device memory themselves: code whose device
memory is owned entirely by another pool (a framework's caching allocator,
a fixed arena), or latency-critical paths where the implicit device
synchronisation of cudaMalloc is not acceptable. spg_objective_noalloc serves
them with a fixed scratch area inside the library. This test calls it through
the C ABI twice in a row (the scratch is shared and keeps the previous call's
contents) and compares each result with the context-based spg_objective on
the same inputs. It lives in its own file so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu


def test_objective_noalloc_matches_objective_twice():
    lib = spg.load()
    shape = (37, 45, 70)
    hyper = dict(synth.DEFAULT_HYPER)
    results = []
    for seed in (11, 12):
        vol = synth.make_volume(shape, blobs=20, radius=9, seed=seed)
        s = spg.SPG(dict(shape=shape, **hyper))
        s.set_data(0, vol.b, vol.w)
        s.reweight()
        s.iterate(15)
        s.reweight()  # weights from a non-zero iterate
        want = s.objective(0)
        sv = spg.parse_state(s.get_state(), [shape])["volumes"][0]
        s.close()
        dev = {k: torch.from_numpy(np.array(v, dtype=np.float32)).cuda()
               for k, v in dict(x=sv["x"], om1=sv["om1"], omtv=sv["omtv"], b=vol.b, w=vol.w).items()}
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        p = [ctypes.c_void_p(dev[k].data_ptr()) for k in ("x", "b", "w", "om1", "omtv")]
        st = lib.spg_objective_noalloc(shape[2], shape[1], shape[0], ctypes.c_float(hyper["lambda_l1"]),
                                       ctypes.c_float(hyper["lambda_tv"]), ctypes.c_float(hyper["mu"]), *p,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == spg.SPG_OK, lib.spg_noalloc_last_error()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-6)
        results.append(got)
    assert not np.allclose(results[0], results[1])


def test_objective_noalloc_rejects_too_many_planes():
    lib = spg.load()
    dummy = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.spg_objective_noalloc(1, 1, 4097, ctypes.c_float(0.05), ctypes.c_float(0.1), ctypes.c_float(1e-3),
                                   p, p, p, p, p, ctypes.c_void_p(out.data_ptr()), None)
    assert st == spg.SPG_EINVAL
    assert b"4096" in lib.spg_noalloc_last_error()
