"""The index scheme of the register-resident transform along z (the fused
z pass of the Fourier-domain term), emulated in numpy for every power-of-two
length 8 .. 4096: thread t keeps the values at positions t + i n/8 (slot i);
a radix-8 Stockham stage of span Ns twiddles slot r by w^(r k n/(8 Ns))
(k = t mod Ns), takes the 8-point DFT, and its output q belongs at
(t - k) 8 + k + q Ns, read back in slot order through the exchange; the last
stage (span n/8, or a radix-2/4 stage of span n/R on butterflies t + m n/8)
stays in the slots. The emulation must equal the DFT of numpy (forward) and
n times its inverse (inverse). No GPU."""
import numpy as np
import pytest


def dft_small(v, sign):
    R = v.shape[-1]
    k = np.arange(R)
    W = np.exp(sign * 2j * np.pi * np.outer(k, k) / R)
    return v @ W.T


def transform(x, sign):
    n = x.size
    log2n = n.bit_length() - 1
    T, ns8, rem = n // 8, log2n // 3, log2n % 3
    w = np.exp(sign * 2j * np.pi * np.arange(n) / n)
    t = np.arange(T)
    v = np.stack([x[t + i * T] for i in range(8)], axis=1)  # v[t, slot]
    for s in range(ns8):
        Ns = 8 ** s
        k = t % Ns
        step = n // (8 * Ns)
        v = v * w[(np.arange(8)[None, :] * k[:, None] * step) % n]
        v = dft_small(v, sign)
        if s < ns8 - 1 or rem:
            buf = np.empty(n, dtype=complex)
            base = (t - k) * 8 + k
            for q in range(8):
                buf[base + q * Ns] = v[:, q]
            v = np.stack([buf[t + i * T] for i in range(8)], axis=1)
    if rem:
        R = 1 << rem
        per = 8 // R  # butterflies t + m T per thread, m < per; slots m + r per
        for m in range(per):
            jp = t + m * T
            slots = [m + r * per for r in range(R)]
            a = v[:, slots] * w[(np.arange(R)[None, :] * jp[:, None]) % n]
            v[:, slots] = dft_small(a, sign)
    out = np.empty(n, dtype=complex)
    for i in range(8):
        out[t + i * T] = v[:, i]
    return out


@pytest.mark.parametrize("log2n", range(3, 13))
def test_register_resident_scheme_is_the_dft(log2n):
    n = 1 << log2n
    rng = np.random.default_rng(log2n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    tol = 1e-12 * np.sqrt(n) * np.abs(x).sum()
    assert np.abs(transform(x, -1) - np.fft.fft(x)).max() <= tol
    assert np.abs(transform(x, +1) - n * np.fft.ifft(x)).max() <= tol


def test_exchange_positions_are_a_permutation():
    """Every exchange writes each of the n positions exactly once."""
    for log2n in range(3, 13):
        n = 1 << log2n
        T, ns8, rem = n // 8, log2n // 3, log2n % 3
        t = np.arange(T)
        for s in range(ns8 if rem else ns8 - 1):
            Ns = 8 ** s
            k = t % Ns
            pos = ((t - k) * 8 + k)[:, None] + np.arange(8)[None, :] * Ns
            assert np.array_equal(np.sort(pos.ravel()), np.arange(n))
