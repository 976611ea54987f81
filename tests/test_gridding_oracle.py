"""Pins of the kernel-regression back-projection oracle (Sec. 2.2). No GPU."""
import math

import numpy as np
import pytest

from oracle import gridding
from paper_1905_13408_gb300 import synth


def _single(n, kx, ky, rot, value=1.0 + 2.0j, c=1.0):
    X = np.zeros((1, n, n), dtype=np.complex128)
    C = np.zeros((1, n, n))
    X[0, ky % n, kx % n] = value
    C[0, ky % n, kx % n] = c
    return X, C, rot[None]


def test_gauss_weights_of_a_grid_aligned_sample():
    """Eq. 26-27 with h = 2: a sample on a grid point spreads exp(-d^2/2) to its
    27 neighbours (1, e^-1/2, e^-1, e^-3/2)."""
    n = 16
    X, C, R = _single(n, 3, 2, np.eye(3), value=2.0, c=1.0)
    num, N = gridding.grid(X, C, R, n, "gauss", 2.0)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                d2 = dx * dx + dy * dy + dz * dz
                assert abs(N[dz % n, 2 + dy, 3 + dx] - math.exp(-d2 / 2)) < 1e-15
                assert abs(num[dz % n, 2 + dy, 3 + dx] - 2.0 * math.exp(-d2 / 2)) < 1e-15
    assert np.count_nonzero(N) == 27


def test_trilinear_exact_on_grid_and_at_cell_centre():
    n = 16
    X, C, R = _single(n, -3, 4, np.eye(3), value=1.5 - 1j, c=0.5)
    num, N = gridding.grid(X, C, R, n, "trilinear")
    assert np.count_nonzero(N) == 1 and N[0, 4, n - 3] == 0.25
    assert num[0, 4, n - 3] == 0.5 * (1.5 - 1j)
    # a rotation by 45 degrees about z moves (kx, ky) = (2, 0) to (sqrt 2, sqrt 2, 0)
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
    X, C, R = _single(n, 2, 0, Rz, value=1.0, c=1.0)
    _, N = gridding.grid(X, C, R, n, "trilinear")
    assert abs(N.sum() - 1.0) < 1e-14  # trilinear weights partition unity


@pytest.mark.parametrize("posterior", [False, True])
def test_gridded_value_minimises_the_local_least_squares(posterior):
    """Eq. 26 vs Eq. 28: at a grid point the closed form num/N equals the
    brute-force minimiser of sum_i P_i sum_j K_j |X_ij - CTF_ij V|^2 over the
    samples that reach it (P_i the posterior weight of image-pose pair i, or
    1 for known poses)."""
    n = 12
    pd = synth.make_projection_data(n, blobs=4, radius=2.0, n_images=5, seed=71, noise_sd=0.5)
    pw = np.random.default_rng(70).uniform(0.05, 1.0, 5) if posterior else None
    num, N = gridding.grid(pd.X, pd.ctf, pd.rot, n, "gauss", 2.0, pw=pw)
    # recompute the normal equations point by point from the individual contributions
    f = np.fft.fftfreq(n) * n
    KY, KX = np.meshgrid(f, f, indexing="ij")
    keep = (KX * KX + KY * KY) <= (n / 2 - 2) ** 2
    target = (0, 1, 2)  # grid point (kz, ky, kx) = (0, 1, 2)
    rows, rhs = [], []
    for i in range(pd.X.shape[0]):
        p = pd.rot[i][:, 0][None, :] * KX[keep][:, None] + pd.rot[i][:, 1][None, :] * KY[keep][:, None]
        g = np.array([target[2], target[1], target[0]], dtype=float)
        d = p - g
        near = np.all(np.abs(np.rint(p) - g) <= 1, axis=1)
        K = np.exp(-(d * d).sum(1) / 2.0)
        sw = np.sqrt(K[near] * (1.0 if pw is None else pw[i]))
        rows.append(sw * pd.ctf[i][keep][near])
        rhs.append(sw * pd.X[i][keep][near])
    A = np.concatenate(rows)[:, None].astype(np.complex128)
    bvec = np.concatenate(rhs)
    v, *_ = np.linalg.lstsq(A, bvec, rcond=None)
    assert abs(num[target] / N[target] - v[0]) < 1e-12 * max(1.0, abs(v[0]))


def test_back_projection_is_hermitian():
    """Real images give a Hermitian gridded spectrum: num(-n) = conj num(n)."""
    n = 14
    pd = synth.make_projection_data(n, blobs=3, radius=2.0, n_images=4, seed=72)  # even box
    num, N = gridding.grid(pd.X, pd.ctf, pd.rot, n, "gauss", 2.0)
    flip = lambda a: np.roll(np.flip(a), 1, axis=(0, 1, 2))
    np.testing.assert_allclose(num, np.conj(flip(num)), atol=1e-10)
    np.testing.assert_allclose(N, flip(N), atol=1e-12)


def test_noiseless_slices_recover_the_transform():
    """Noiseless images with CTF = 1 sample the phantom's transform; where 150
    slices cross (|k| <= 8) the gridded num/N follows the 3-D DFT of the
    rendered phantom (origin at the box centre): within 6 % with the
    trilinear kernel, and with the wider Gaussian kernel of Sec. 2.2 (h = 2),
    which also smooths (Eq. 29), at a correlation above 0.99."""
    n = 32  # blob tails must vanish at the volume edge for the DFT to match the analytic transform
    pd = synth.make_projection_data(n, blobs=6, radius=3.0, n_images=150, seed=73, noise_sd=0.0)
    pd.X /= pd.ctf
    pd.ctf[:] = 1.0
    F = np.fft.fftn(np.fft.ifftshift(pd.phantom.astype(np.float64)))
    f = np.fft.fftfreq(n) * n
    r = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    for kernel, min_corr, max_rel in (("trilinear", 0.999, 0.06), ("gauss", 0.99, None)):
        num, N = gridding.grid(pd.X, pd.ctf, pd.rot, n, kernel, 2.0)
        sel = (r <= 8) & (N > 0)
        g, t = num[sel] / N[sel], F[sel]
        corr = np.real(np.vdot(t, g)) / np.linalg.norm(t) / np.linalg.norm(g)
        assert corr > min_corr, kernel
        if max_rel is not None:
            assert np.abs(g - t).max() / np.abs(F).max() < max_rel


def test_fourier_term_is_fitted_by_the_phantom():
    """Eq. 31 from gridded images: with y, N' from to_fourier_term, the phantom
    itself (a volume with its origin at array index 0, as the unitary DFT A
    takes it) nearly zeroes the residual y - sqrt(N') A x wherever slices cross
    (|k| <= 8), with the images' own CTF, while the zero volume leaves all of
    y. A dropped (-1)^k centring sign, a missing voxel-count factor in N' or a
    missing square root each leave a residual of the order of y itself."""
    n = 32
    pd = synth.make_projection_data(n, blobs=6, radius=3.0, n_images=150, seed=74, noise_sd=0.0)
    num, N = gridding.grid(pd.X, pd.ctf, pd.rot, n, "trilinear")
    y, Nq = gridding.to_fourier_term(num, N)
    f = np.fft.fftfreq(n) * n
    r = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    sel = (r <= 8) & (N > 0)
    Ax = np.fft.fftn(pd.phantom.astype(np.float64), norm="ortho")
    res = y - np.sqrt(Nq) * Ax
    assert np.linalg.norm(res[sel]) < 0.05 * np.linalg.norm(y[sel])
    assert np.all(y[N == 0] == 0)
