"""Fourier-domain data term (Eq. 31) on the GPU against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fourier
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu

HYPER = dict(synth.DEFAULT_HYPER)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def gpu_fourier_solve(fv, hyper, rounds, iters, **kw):
    shape = fv.phantom.shape
    s = spg.SPG(dict(shape=shape, **hyper), **kw)
    s.set_data_fourier(0, synth.half_spectrum(fv.y).astype(np.complex64),
                       synth.half_spectrum(fv.N).astype(np.float32))
    s.solve(rounds, iters)
    x = s.get_x(0).cpu().numpy()
    obj = s.objective(0)
    hist = s.history(0)
    s.close()
    return x, obj, hist


# power-of-two nz take the own transform along z (32; long lines with
# narrower tiles: 1024 with 8 columns per CTA, 2048 with 4, 4096 with 2);
# other nz the 3-D library transforms around the spectrum pass (24, 17, 28,
# 1, and 5000 beyond the own transform's range)
@pytest.mark.parametrize("shape", [(24, 28, 30), (32, 32, 32), (17, 40, 25), (28, 12, 16), (1, 24, 30),
                                   (1024, 6, 8), (2048, 4, 4), (4096, 2, 4), (5000, 2, 2)])
def test_fourier_solve_matches_oracle(shape):
    fv = synth.make_fourier_volume(shape, blobs=12, radius=6, seed=sum(shape))
    hyper = dict(HYPER, mu=0.02)
    x, obj, hist = gpu_fourier_solve(fv, hyper, 2, 40)
    p = oracle.Params(shape, **hyper)
    xr, hr, rr = fourier.solve(fv.y, fv.N, p, 2, 40)
    err = rel_l2(x, xr)
    print(f"fourier {shape}: rel-L2 {err:.3e}")
    assert err <= 1e-5
    # l1 and TV columns of the history (its data column is 0 in this mode)
    np.testing.assert_allclose(hist[:, 2:4], np.concatenate([hr[0, :, 1:3], hr[1, :, 1:3]]), rtol=1e-5)


@pytest.mark.parametrize("shape", [(128, 24, 30), (256, 12, 20), (512, 40, 120), (512, 6, 4)])
def test_fourier_register_resident_z_transform(shape):
    """Lengths 128 .. 512 along z (16 columns per tile in the
    register-resident kernel): one tile, several rows of tiles (512 x 40 x
    120: 153 tiles) and a ragged last tile (18 columns); one round against
    the oracle."""
    fv = synth.make_fourier_volume(shape, blobs=12, radius=6, seed=sum(shape))
    hyper = dict(HYPER, mu=0.02)
    x, obj, hist = gpu_fourier_solve(fv, hyper, 1, 15)
    p = oracle.Params(shape, **hyper)
    xr, hr, rr = fourier.solve(fv.y, fv.N, p, 1, 15)
    err = rel_l2(x, xr)
    print(f"fourier z length {shape[0]} {shape}: rel-L2 {err:.3e}")
    assert err <= 1e-5


def test_fourier_objective_value():
    shape = (20, 22, 24)
    fv = synth.make_fourier_volume(shape, blobs=8, radius=5, seed=61)
    hyper = dict(HYPER, mu=0.02)
    s = spg.SPG(dict(shape=shape, **hyper))
    s.set_data_fourier(0, synth.half_spectrum(fv.y).astype(np.complex64), synth.half_spectrum(fv.N).astype(np.float32))
    rng = np.random.default_rng(62)
    x0 = (0.3 * rng.standard_normal(shape)).astype(np.float32)
    s.set_x(0, x0)
    s.reweight()
    obj = s.objective(0)
    s.close()
    p = oracle.Params(shape, **hyper)
    om1, omtv, _ = oracle.reweight(x0, p)
    want = fourier.objective(x0.astype(np.float64), fv.y, fv.N, om1, omtv, p)
    np.testing.assert_allclose(obj, want, rtol=1e-6)


def test_constant_weight_matches_real_space_solve():
    """N = w0 and y = sqrt(w0) A b: the Fourier-form solve equals the
    real-space solve with w = w0 (different code paths on the GPU)."""
    shape = (32, 32, 32)
    vol = synth.make_volume(shape, blobs=10, radius=8, seed=63)
    w0 = 2.0
    fv = synth.FourierVolume(y=np.sqrt(w0) * np.fft.fftn(vol.b.astype(np.float64), norm="ortho"),
                             N=np.full(shape, w0), phantom=vol.phantom)
    hyper = dict(HYPER, mu=0.02)
    xf, _, _ = gpu_fourier_solve(fv, hyper, 2, 50)
    s = spg.SPG(dict(shape=shape, **hyper))
    s.set_data(0, vol.b, np.full(shape, w0, np.float32))
    s.solve(2, 50)
    xr = s.get_x(0).cpu().numpy()
    s.close()
    assert rel_l2(xf, xr.astype(np.float64)) <= 1e-5


def test_fourier_param_scales():
    """Sec. 2.5 scales with the Fourier-domain term: RMS(A^H D y) by
    Parseval from the spectrum, and mean / max / min of N over the full
    spectrum, against the real-space c of the oracle."""
    shape = (16, 20, 24)
    fv = synth.make_fourier_volume(shape, blobs=8, radius=5, seed=64)
    s = spg.SPG(dict(shape=shape, **HYPER))
    s.set_data_fourier(0, synth.half_spectrum(fv.y).astype(np.complex64), synth.half_spectrum(fv.N).astype(np.float32))
    sc = s.param_scales(0)
    s.close()
    got = [sc["rms_wb"], sc["mean_w"], sc["max_w"], sc["min_w"]]
    c = fourier.data_parts(fv.y, fv.N)
    want = [np.sqrt(np.mean(c * c)), fv.N.mean(), fv.N.max(), fv.N.min()]
    np.testing.assert_allclose(got, want, rtol=2e-5)


@pytest.mark.parametrize("shape", [(20, 24, 28), (128, 20, 22), (16, 128, 128)])
def test_fourier_anchor_matches_oracle(shape):
    """The implicit-gradient term gamma |x - a|^2 with the Fourier-domain data
    term (Eq. 31): the spectrum pass uses N + 2 gamma and the anchor's
    transform; iterate and data-plus-anchor value against the oracle, on the
    library's 3-D transforms (nz = 20) and on the TMA-fed z pass (nz = 128,
    with narrow and with square 128 x 128 planes)."""
    fv = synth.make_fourier_volume(shape, blobs=10, radius=5, seed=65)
    hyper = dict(HYPER, mu=0.02)
    anchor = (0.2 * np.random.default_rng(66).standard_normal(shape)).astype(np.float32)
    gamma = 0.3 * float(fv.N.mean())
    s = spg.SPG(dict(shape=shape, **hyper))
    s.set_data_fourier(0, synth.half_spectrum(fv.y).astype(np.complex64), synth.half_spectrum(fv.N).astype(np.float32))
    s.set_anchor(0, gamma, anchor)
    s.solve(2, 40)
    x = s.get_x(0).cpu().numpy().astype(np.float64)
    obj = s.objective(0)
    st = s.round_stats(0)
    s.close()
    p = oracle.Params(shape, **hyper, gamma=gamma, anchor=anchor.astype(np.float64))
    xr, hr, rr = fourier.solve(fv.y, fv.N, p, 2, 40, with_hist=False)
    err = rel_l2(x, xr)
    print(f"fourier + anchor {shape}: rel-L2 {err:.3e}")
    assert err <= 1e-5
    np.testing.assert_allclose(st[4], rr[1, 4], rtol=1e-6)  # L of round 2 includes 2 gamma
    want = fourier.data_value(x, fv.y, fv.N) + gamma * float(((x - anchor) ** 2).sum())
    np.testing.assert_allclose(obj[0], want, rtol=1e-5)


@pytest.mark.parametrize("shape", [(16, 18, 20), (16, 40, 128)])
def test_fourier_checkpoint_resume_bitwise(shape):
    """State saved in the middle of a Fourier-domain round and restored gives
    the same iterates bit for bit: the extrapolated point is formed from the
    restored x_k and d_k exactly as before (by a separate pass ahead of the
    library's transforms, x = 20; inside the own row pass, x = 128)."""
    fv = synth.make_fourier_volume(shape, blobs=6, radius=4, seed=67)
    hyper = dict(HYPER, mu=0.02)
    s = spg.SPG(dict(shape=shape, **hyper))
    s.set_data_fourier(0, synth.half_spectrum(fv.y).astype(np.complex64), synth.half_spectrum(fv.N).astype(np.float32))
    s.reweight()
    s.iterate(23)
    blob = s.get_state()
    s.iterate(17)
    x1 = s.get_x(0).cpu().numpy()
    s.set_state(blob)
    s.iterate(17)
    x2 = s.get_x(0).cpu().numpy()
    s.close()
    np.testing.assert_array_equal(x1, x2)



# square power-of-two planes (128, 256, 512; the benchmark's planes are 512 x
# 512) with power-of-two nz: per-plane 2-D transforms around the own z pass
@pytest.mark.parametrize("shape", [(16, 128, 128), (128, 128, 128), (8, 256, 256), (32, 256, 256), (8, 512, 512)])
def test_fourier_square_planes_match_oracle(shape):
    fv = synth.make_fourier_volume(shape, blobs=12, radius=6, seed=sum(shape) + 1)
    hyper = dict(HYPER, mu=0.02)
    x, obj, hist = gpu_fourier_solve(fv, hyper, 2, 15)
    p = oracle.Params(shape, **hyper)
    xr, hr, rr = fourier.solve(fv.y, fv.N, p, 2, 15)
    err = rel_l2(x, xr)
    print(f"fourier square planes {shape}: rel-L2 {err:.3e}")
    assert err <= 1e-5
    np.testing.assert_allclose(hist[:, 2:4], np.concatenate([hr[0, :, 1:3], hr[1, :, 1:3]]), rtol=1e-5)


@pytest.mark.parametrize("shape", [(16, 128, 128), (8, 40, 256), (8, 512, 512), (8, 24, 1024)])
def test_row_pass_equals_library_transforms(shape, monkeypatch):
    """The own row pass (power-of-two nx, the spectrum held kx-major between
    it and the transform along y) against the library's per-plane 2-D
    transforms (SPG_ROW_PASS=0) on the same solve: the same arithmetic up to
    the transforms' rounding; ny not a multiple of the rows per CTA (40)
    leaves a ragged last group of rows."""
    fv = synth.make_fourier_volume(shape, blobs=12, radius=min(shape) / 3, seed=sum(shape) + 2)
    hyper = dict(HYPER, mu=0.02)
    x_own, _, h_own = gpu_fourier_solve(fv, hyper, 1, 20)
    monkeypatch.setenv("SPG_ROW_PASS", "0")
    x_lib, _, h_lib = gpu_fourier_solve(fv, hyper, 1, 20)
    err = rel_l2(x_own, x_lib)
    print(f"row pass vs library in-plane transforms {shape}: rel-L2 {err:.3e}")
    assert err <= 1e-6
    np.testing.assert_allclose(h_own[:, 2:4], h_lib[:, 2:4], rtol=1e-6)
