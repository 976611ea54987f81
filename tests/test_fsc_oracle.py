"""Pins of the numpy FSC oracle (Sec. 2.3, Eq. 30). No GPU."""
import math

import numpy as np

from oracle import fsc as ofsc
from paper_1905_13408_gb300 import synth


def test_self_correlation_is_one_and_sign_flip_is_minus_one():
    a = synth.random_volume((16, 16, 16), 1)
    c, cnt = ofsc.fsc(a, a)
    np.testing.assert_allclose(c, 1.0, atol=1e-12)
    c, _ = ofsc.fsc(a, -a)
    np.testing.assert_allclose(c, -1.0, atol=1e-12)
    c, _ = ofsc.fsc(a, 3.5 * a)
    np.testing.assert_allclose(c, 1.0, atol=1e-12)


def test_shell_counts_are_lattice_point_counts():
    """Shell 0 holds one frequency, shell 1 the 6 axis neighbours plus the
    12 points at distance sqrt(2) (round(1.414) = 1)."""
    _, cnt = ofsc.fsc(np.ones((8, 8, 8)), np.ones((8, 8, 8)))
    assert cnt[0] == 1
    assert cnt[1] == 6 + 12
    assert cnt.sum() == (ofsc.shells(8) <= 4).sum()


def test_shifted_delta_closed_form():
    """a = delta at the origin, b = delta one voxel along x: F = 1 and
    G = exp(-2 pi i h / n), so FSC(shell) = mean over the shell of cos(2 pi h / n)."""
    n = 8
    a = np.zeros((n, n, n))
    b = np.zeros((n, n, n))
    a[0, 0, 0] = 1.0
    b[0, 0, 1] = 1.0
    c, _ = ofsc.fsc(a, b)
    f = np.fft.fftfreq(n) * n
    H = np.broadcast_to(f[None, None, :], (n, n, n))
    s = ofsc.shells(n)
    for k in range(n // 2 + 1):
        sel = s == k
        want = np.mean([math.cos(2 * math.pi * h / n) for h in H[sel]])
        assert abs(c[k] - want) < 1e-12


def test_independent_noise_is_uncorrelated():
    """Two independent white-noise maps: |FSC| ~ 1/sqrt(shell count)."""
    a = synth.random_volume((32, 32, 32), 2)
    b = synth.random_volume((32, 32, 32), 3)
    c, cnt = ofsc.fsc(a, b)
    z = np.abs(c[2:]) * np.sqrt(cnt[2:] / 2)
    assert np.all(z < 5)


def test_resolution_shell_is_the_first_crossing_after_the_origin():
    """The 0.143 criterion (Sec. 2.3): the first shell k >= 1 whose FSC is
    below the threshold; shell 0 (the mean) never decides it, and a curve
    that stays above it reports one past the last shell."""
    assert ofsc.resolution_shell(np.array([1.0, 0.95, 0.6, 0.2, 0.1, 0.05])) == 4
    assert ofsc.resolution_shell(np.array([0.0, 0.9, 0.3, 0.1])) == 3
    assert ofsc.resolution_shell(np.array([1.0, 0.9, 0.8]), threshold=0.5) == 3
    assert ofsc.resolution_shell(np.array([1.0, 0.9, 0.8]), threshold=0.85) == 2
