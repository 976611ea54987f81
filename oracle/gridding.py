"""Kernel-regression back-projection (Sec. 2.2, Eq. 24-28), plain numpy.

TEST INFRASTRUCTURE ONLY.

Image coefficient X_j at 2-D frequency index (kx, ky) of image i lands at the
3-D position p = R_i (kx, ky, 0) (Eq. 24). For every grid point n near p,
with kernel weight K (Eq. 26/27),
    num(n) += K CTF_j X_j,     N(n) += K CTF_j^2,
so that the gridded value num/N minimises sum_j K |X_j - CTF_j V_n|^2 (Eq. 28).
Each image is one image-pose pair; with posterior weights P (Eq. 26-28) its
contributions are multiplied by P (known poses: P = 1). Kernels:
  "gauss":     K = exp(-|p - n|^2 / h), n = round(p) + {-1, 0, 1}^3 (Sec. 2.2, h = 2)
  "trilinear": K = prod_a (1 - |p_a - n_a|), n the 8 corners of p's cell.
Only coefficients with kx^2 + ky^2 <= (n/2 - 2)^2 are used. Grid indices wrap
modulo n (fftfreq order, array axes [kz][ky][kx]). Image spectra take the
real-space origin at the box centre (n even), so the gridded spectrum is that
of the centred volume.
"""
import itertools

import numpy as np


def grid(X, ctf, rot, n, kernel="gauss", h=2.0, pw=None):
    """(num, N) full spectra (complex128, float64) [n][n][n]; pw: posterior
    weight of each image-pose pair (None: 1)."""
    num = np.zeros(n * n * n, dtype=np.complex128)
    N = np.zeros(n * n * n)
    f = np.fft.fftfreq(n) * n
    KY, KX = np.meshgrid(f, f, indexing="ij")
    keep = (KX * KX + KY * KY) <= (n / 2 - 2) ** 2
    kx, ky = KX[keep], KY[keep]
    for i in range(X.shape[0]):
        p = rot[i][:, 0][None, :] * kx[:, None] + rot[i][:, 1][None, :] * ky[:, None]   # (x, y, z)
        xv = X[i][keep]
        cv = ctf[i][keep]
        P = 1.0 if pw is None else float(pw[i])
        if kernel == "gauss":
            base = np.rint(p)
            offs = itertools.product((-1, 0, 1), repeat=3)
        else:
            base = np.floor(p)
            offs = itertools.product((0, 1), repeat=3)
        for o in offs:
            g = base + np.array(o)[None, :]
            d = p - g
            if kernel == "gauss":
                K = np.exp(-(d * d).sum(1) / h)
            else:
                K = np.prod(1.0 - np.abs(d), axis=1)
            gi = np.mod(g.astype(np.int64), n)
            flat = (gi[:, 2] * n + gi[:, 1]) * n + gi[:, 0]
            np.add.at(num, flat, P * K * cv * xv)
            np.add.at(N, flat, P * K * cv * cv)
    return num.reshape(n, n, n), N.reshape(n, n, n)


def to_fourier_term(num, N):
    """(y, N') of the Eq. 31 data term 1/2 |y - sqrt(N') A x|^2 with A the
    unitary DFT of a volume whose origin is at index 0: the images sample the
    unnormalised transform of the centred volume, which for even n is
    (-1)^(kx+ky+kz) times the uncentred one, so N' = V N and
    y = (-1)^(kx+ky+kz) num / sqrt(N) (0 where N = 0)."""
    n = num.shape[0]
    V = float(num.size)
    i = np.arange(n)
    sign = (-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :])
    with np.errstate(invalid="ignore", divide="ignore"):
        y = np.where(N > 0, sign * num / np.sqrt(np.where(N > 0, N, 1.0)), 0.0)
    return y, V * N
