"""FP64 oracle of the solve with the Fourier-domain data term of Eq. 31.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU leg import it).

Round objective (Sec. 2.5, Eq. 31, minimised; A the unitary 3-D DFT, D = diag
sqrt(N)):
    F(x) = 1/2 |y - D A x|^2 + lambda_l1 sum om1 |x| + lambda_tv sum omtv h_mu(Dx)
The data gradient is A^H D (D A x - y) = ifft(N fft(x)) - c with
c = A^H(D y) (numpy's unnormalised-forward / normalised-inverse pair makes
A^H N A = ifftn(N fftn(.))). The TV gradient, the soft-threshold, the weights
and the extrapolation are the real-space oracle's (spg_oracle.c, Eq. 11-21);
this module only replaces the data term and its Lipschitz constant (max N).
"""
import numpy as np

import oracle


def data_parts(y, N):
    """c = A^H(sqrt(N) y) (real) for a Hermitian y."""
    return np.fft.ifftn(np.sqrt(N) * y, norm="ortho").real


def grad_data(x, N, c):
    return np.fft.ifftn(N * np.fft.fftn(x)).real - c


def data_value(x, y, N):
    r = y - np.sqrt(N) * np.fft.fftn(x, norm="ortho")
    return 0.5 * float((np.abs(r) ** 2).sum())


def objective(x, y, N, om1, omtv, p):
    """{data, l1, tv, total}; with p.gamma > 0 the data part includes the
    implicit-gradient term gamma |x - anchor|^2 of Eq. 31 (the real-space
    oracle's objective with w = 0 is exactly that term)."""
    o = oracle.objective(x, np.zeros(x.shape), np.zeros(x.shape), om1, omtv, p)
    d = data_value(x, y, N) + (o[0] if p.gamma > 0 else 0.0)
    return np.array([d, o[1], o[2], d + o[1] + o[2]])


def solve(y, N, p, rounds, iters, x0=None, with_hist=True):
    """Reweighted FISTA solve of the Eq. 31 objective (same schedule as
    oracle.solve), with the gamma |x - anchor|^2 term when p.gamma > 0:
    returns (x, hist[rounds, iters, 4], rstats[rounds, 6])."""
    shape = tuple(p.shape)
    x = np.zeros(shape) if x0 is None else np.array(x0, dtype=np.float64)
    c = data_parts(y, N)
    hist = np.zeros((rounds, iters, 4))
    rst = np.zeros((rounds, 6))
    beta = oracle.beta_table(iters, p.momentum)
    for r in range(rounds):
        om1, omtv, st = oracle.reweight(x, p)
        L = float(N.max()) + 12.0 * p.lambda_tv * st[0] / p.mu + (2.0 * p.gamma if p.gamma > 0 else 0.0)
        tau = 1.0 / L
        rst[r, :4] = st
        rst[r, 4:] = (L, tau)
        xp = x.copy()
        for k in range(iters):
            if with_hist:
                hist[r, k] = objective(x, y, N, om1, omtv, p)
            yk = x + beta[k] * (x - xp)
            g = grad_data(yk, N, c) + p.lambda_tv * oracle.tv_grad(yk, omtv, p)
            if p.gamma > 0:  # implicit-gradient term of Eq. 22 / Eq. 31
                g = g + 2.0 * p.gamma * (yk - p.anchor)
            z = yk - tau * g
            t = tau * p.lambda_l1 * om1
            xn = np.sign(z) * np.maximum(np.abs(z) - t, 0.0)
            xp, x = x, xn
    return x, hist, rst
