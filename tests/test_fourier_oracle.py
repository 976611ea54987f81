"""Pins of the Fourier-domain (Eq. 31) oracle. No GPU."""
import numpy as np
import pytest

import oracle
from oracle import fourier
from paper_1905_13408_gb300 import synth


@pytest.mark.parametrize("gamma", [0.0, 0.7])
def test_constant_weight_reduces_to_the_real_space_solve(gamma):
    """With N = w0 everywhere and y = sqrt(w0) A b, 1/2 |y - D A x|^2 equals
    1/2 w0 |x - b|^2 (A unitary), so the Fourier-form solve must reproduce the
    pinned real-space oracle exactly (up to FFT rounding), also with the
    implicit-gradient term gamma |x - a|^2 (two implementations of it)."""
    shape = (10, 12, 14)
    vol = synth.make_volume(shape, blobs=6, radius=3, seed=51)
    w0 = 2.5
    N = np.full(shape, w0)
    b = vol.b.astype(np.float64)
    y = np.sqrt(w0) * np.fft.fftn(b, norm="ortho")
    anchor = np.random.default_rng(50).standard_normal(shape) * 0.3
    p = oracle.Params(shape, mu=0.02, gamma=gamma, anchor=anchor if gamma > 0 else None)
    xf, hf, rf = fourier.solve(y, N, p, 2, 30)
    ref = oracle.solve(b, np.full(shape, w0), p, 2, 30)
    np.testing.assert_allclose(xf, ref.x, atol=1e-11)
    np.testing.assert_allclose(hf, ref.hist, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(rf, ref.rstats, rtol=1e-12)


def test_data_gradient_is_the_derivative_of_the_data_term():
    shape = (8, 9, 10)
    fv = synth.make_fourier_volume(shape, blobs=5, radius=2.5, seed=52)
    c = fourier.data_parts(fv.y, fv.N)
    rng = np.random.default_rng(53)
    x = rng.standard_normal(shape) * 0.2
    g = fourier.grad_data(x, fv.N, c)
    h = 1e-4  # the data term is quadratic: central differences are exact up to rounding
    for v in rng.choice(x.size, 12, replace=False):
        e = np.zeros(x.size)
        e[v] = h
        e = e.reshape(shape)
        fd = (fourier.data_value(x + e, fv.y, fv.N) - fourier.data_value(x - e, fv.y, fv.N)) / (2 * h)
        assert g.ravel()[v] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_generated_data_is_hermitian():
    fv = synth.make_fourier_volume((8, 10, 12), blobs=4, radius=2, seed=54)
    flip = np.conj(np.roll(np.flip(fv.y), 1, axis=(0, 1, 2)))
    np.testing.assert_allclose(fv.y, flip, atol=1e-12)
    np.testing.assert_allclose(fv.N, np.roll(np.flip(fv.N), 1, axis=(0, 1, 2)), atol=1e-15)
    c_full = np.fft.ifftn(np.sqrt(fv.N) * fv.y, norm="ortho")
    assert np.abs(c_full.imag).max() < 1e-12 * np.abs(c_full.real).max()


def test_fourier_solve_decreases_objective_with_plain_steps():
    shape = (12, 12, 12)
    fv = synth.make_fourier_volume(shape, blobs=6, radius=3, seed=55)
    p = oracle.Params(shape, mu=0.01, momentum="ista")
    _, h, _ = fourier.solve(fv.y, fv.N, p, 1, 60)
    tot = h[0, :, 3]
    assert np.all(np.diff(tot) <= 1e-10 * np.abs(tot[1:]))
