"""GPU Fourier shell correlation (Eq. 30) against the numpy oracle, and the
gold-standard half-map check (Sec. 2.3) on synthetic half-maps."""
import numpy as np
import pytest
import torch

from oracle import fsc as ofsc
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [16, 33, 64])
def test_fsc_matches_oracle(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n)).astype(np.float32)
    b = (a + 0.7 * rng.standard_normal((n, n, n))).astype(np.float32)
    got, cnt = spg.spg_fsc(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    want, wcnt = ofsc.fsc(a, b)
    np.testing.assert_array_equal(cnt, wcnt)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6)


def test_fsc_host_inputs_and_identity():
    a = synth.random_volume((24, 24, 24), 5).astype(np.float32)
    got, _ = spg.spg_fsc(a, a)
    np.testing.assert_allclose(got, 1.0, atol=1e-6)


def test_half_maps_regularised_vs_raw():
    """Two half-maps with independent noise, each solved independently in one
    batched context (3 rounds x 100): the FSC between the solutions stays
    above the FSC between the raw data maps at mid frequencies, and the GPU
    FSC matches the oracle on both pairs."""
    n = 64
    h1, h2 = synth.make_half_maps((n, n, n), blobs=40, radius=24, seed=123)
    hyper = dict(synth.DEFAULT_HYPER)
    s = spg.SPG([dict(shape=(n, n, n), **hyper)] * 2)
    s.set_data(0, h1.b, h1.w)
    s.set_data(1, h2.b, h2.w)
    s.solve(3, 100)
    x1, x2 = s.get_x(0), s.get_x(1)
    s.close()
    raw, _ = spg.spg_fsc(h1.b, h2.b)
    sol, _ = spg.spg_fsc(x1, x2)
    np.testing.assert_allclose(sol, ofsc.fsc(x1.cpu().numpy(), x2.cpu().numpy())[0], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(raw, ofsc.fsc(h1.b, h2.b)[0], rtol=1e-5, atol=1e-6)
    kr, ks = ofsc.resolution_shell(raw), ofsc.resolution_shell(sol)
    print(f"half-maps 64^3: FSC=0.143 at shell {kr} (raw) vs {ks} (regularised)")
    mid = slice(4, n // 4)
    assert sol[mid].mean() > raw[mid].mean()


def test_fsc_repeats_within_rounding():
    """Shell sums are accumulated with shared-memory double atomics, so their
    order, and the last bits of the result, can change between runs; two runs
    on the same maps agree far below the float32 inputs' precision."""
    rng = np.random.default_rng(9)
    n = 48
    a = torch.from_numpy(rng.standard_normal((n, n, n)).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal((n, n, n)).astype(np.float32)).cuda()
    f1, c1 = spg.spg_fsc(a, b)
    f2, c2 = spg.spg_fsc(a, b)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_allclose(f1, f2, rtol=0, atol=1e-12)
