"""Fourier shell correlation (Sec. 2.3, Eq. 30), plain numpy.

TEST INFRASTRUCTURE ONLY (tests import it; the CUDA library does not).

FSC(k) = sum_{|k'| = k} F(k') G*(k') / sqrt(sum |F(k')|^2 sum |G(k')|^2),
over the full 3-D spectrum of two real cubic maps; the shell of a frequency
index (h, k, l) (numpy.fft.fftfreq order times n) is the nearest integer to
sqrt(h^2 + k^2 + l^2); shells 0 .. n/2 are reported. The real part of the
numerator is kept (the imaginary parts cancel between k' and -k' for real maps).
"""
import numpy as np


def shells(n):
    f = np.fft.fftfreq(n) * n
    r = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    return np.rint(r).astype(np.int64)


def fsc(a, b):
    """(fsc, counts) for shells 0 .. n/2 of two real n^3 maps."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    assert a.shape == (n, n, n) and b.shape == a.shape
    F = np.fft.fftn(a)
    G = np.fft.fftn(b)
    s = shells(n).ravel()
    keep = s <= n // 2
    s = s[keep]
    num = np.bincount(s, weights=(F * np.conj(G)).real.ravel()[keep], minlength=n // 2 + 1)
    d1 = np.bincount(s, weights=(np.abs(F) ** 2).ravel()[keep], minlength=n // 2 + 1)
    d2 = np.bincount(s, weights=(np.abs(G) ** 2).ravel()[keep], minlength=n // 2 + 1)
    cnt = np.bincount(s, minlength=n // 2 + 1).astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        out = num / np.sqrt(d1 * d2)
    return out, cnt


def resolution_shell(curve, threshold=0.143):
    """First shell (>= 1) where the FSC drops below the threshold (Sec. 2.3)."""
    for k in range(1, len(curve)):
        if curve[k] < threshold:
            return k
    return len(curve)
