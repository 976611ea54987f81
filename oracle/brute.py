"""Independent slow solvers for tiny volumes, used to pin the FP64 oracle.

TEST INFRASTRUCTURE ONLY (tests import it; nothing else does).

Everything here is built differently from ``spg_oracle.c`` so that a mistake
there does not repeat here:

* the difference operator D (Eq. 12, backward differences, zero on the first
  plane of each axis) is assembled as a sparse matrix from Kronecker products
  of 1-D difference matrices, instead of index loops;
* the minimiser of the round objective (Eq. 11/31 with the smoothed TV of
  Eq. 14) is found by generic methods that know nothing of the proximal
  update of Eq. 20-21: SciPy's L-BFGS-B on the exact split ``x = p - n``
  (``p, n >= 0``), and a long-run subgradient method with diminishing steps;
* the 1-D total-variation special case is solved by Newton's method with a
  banded (tridiagonal) Hessian.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def diff1d(n):
    """n x n backward-difference matrix with a zero first row."""
    main = np.ones(n)
    main[0] = 0.0
    off = -np.ones(n - 1)
    return sp.diags([main, off], [0, -1], shape=(n, n), format="csr")


def d_matrix(shape):
    """Stacked [D_x; D_y; D_z] (3n x n) for a [nz, ny, nx] volume, x fastest."""
    nz, ny, nx = shape
    Iz, Iy, Ix = sp.identity(nz), sp.identity(ny), sp.identity(nx)
    dx = sp.kron(sp.kron(Iz, Iy), diff1d(nx))
    dy = sp.kron(sp.kron(Iz, diff1d(ny)), Ix)
    dz = sp.kron(sp.kron(diff1d(nz), Iy), Ix)
    return sp.vstack([dx, dy, dz]).tocsr()


def huber_vec(g3, mu):
    """Smoothed norm of each column of a (3, n) array and its gradient."""
    s = np.sqrt((g3 * g3).sum(axis=0))
    val = np.where(s <= mu, s * s / (2 * mu), s - mu / 2)
    grad = g3 / np.maximum(mu, s)[None, :]
    return val, grad


class Problem:
    """Round objective F(x) on a tiny volume, from the sparse D above."""

    def __init__(self, b, w, om1, omtv, lambda_l1, lambda_tv, mu):
        self.shape = b.shape
        self.n = b.size
        self.b = b.ravel().astype(np.float64)
        self.w = w.ravel().astype(np.float64)
        self.om1 = np.ones(self.n) if om1 is None else om1.ravel().astype(np.float64)
        self.omtv = np.ones(self.n) if omtv is None else omtv.ravel().astype(np.float64)
        self.l1, self.tv, self.mu = float(lambda_l1), float(lambda_tv), float(mu)
        self.D = d_matrix(self.shape)

    def smooth(self, x):
        g3 = (self.D @ x).reshape(3, self.n)
        hv, hg = huber_vec(g3, self.mu)
        r = x - self.b
        f = 0.5 * (self.w * r * r).sum() + self.tv * (self.omtv * hv).sum()
        grad = self.w * r + self.tv * (self.D.T @ (self.omtv[None, :] * hg).ravel())
        return f, grad

    def parts(self, x):
        """(data, l1, tv) of the round objective (Eq. 11 with the data term of
        Eq. 28/31 and the smoothed norm of Eq. 14), each with its lambda, each
        summed on its own: a dot product of the weights with the per-voxel
        terms, with |Dx| taken from the sparse D above."""
        x = np.asarray(x, dtype=np.float64).ravel()
        g3 = (self.D @ x).reshape(3, self.n)
        hv, _ = huber_vec(g3, self.mu)
        r = x - self.b
        return (0.5 * np.dot(self.w, r * r),
                self.l1 * np.dot(self.om1, np.abs(x)),
                self.tv * np.dot(self.omtv, hv))

    def F(self, x):
        x = np.asarray(x, dtype=np.float64).ravel()
        f, _ = self.smooth(x)
        return f + self.l1 * (self.om1 * np.abs(x)).sum()

    def lbfgs(self, tol=1e-14, maxiter=200000):
        """Minimise F with L-BFGS-B over the split x = p - n, p, n >= 0."""
        from scipy.optimize import minimize
        n = self.n
        c = self.l1 * self.om1

        def fun(v):
            p, q = v[:n], v[n:]
            f, g = self.smooth(p - q)
            return f + (c * (p + q)).sum(), np.concatenate([g + c, -g + c])

        x0 = np.concatenate([np.maximum(self.b, 0), np.maximum(-self.b, 0)])
        res = minimize(fun, x0, jac=True, method="L-BFGS-B", bounds=[(0, None)] * (2 * n),
                       options=dict(maxiter=maxiter, maxfun=maxiter, ftol=tol, gtol=1e-13,
                                    maxcor=50))
        x = res.x[:n] - res.x[n:]
        return x.reshape(self.shape), self.F(x)

    def subgradient(self, iters=200000, x0=None):
        """Long-run subgradient method, minimum-norm subgradient, step 1/(m (k+1)) clipped at 1/L."""
        x = np.zeros(self.n) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
        m = self.w.min()
        L = self.w.max() + 12 * self.tv * self.omtv.max() / self.mu
        best_x, best_f = x.copy(), self.F(x)
        c = self.l1 * self.om1
        for k in range(iters):
            _, g = self.smooth(x)
            # minimum-norm element of the subdifferential of the weighted l1 term
            sg = np.where(x > 0, g + c, np.where(x < 0, g - c, np.sign(g) * np.maximum(np.abs(g) - c, 0)))
            step = min(1.0 / L, 1.0 / (m * (k + 1)))
            x = x - step * sg
            f = self.F(x)
            if f < best_f:
                best_f, best_x = f, x.copy()
        return best_x.reshape(self.shape), best_f

    def kkt_residual(self, x):
        """max violation of 0 in grad f + lambda_l1 om1 d|x| (elementwise)."""
        x = np.asarray(x, dtype=np.float64).ravel()
        _, g = self.smooth(x)
        c = self.l1 * self.om1
        nz = x != 0
        r = np.zeros(self.n)
        r[nz] = np.abs(g[nz] + c[nz] * np.sign(x[nz]))
        r[~nz] = np.maximum(np.abs(g[~nz]) - c[~nz], 0.0)
        return r.max()


def tv1d_newton(b, w, omtv, lambda_tv, mu, iters=200, tol=1e-15):
    """Minimise 1/2 sum w (x-b)^2 + lambda_tv sum omtv h_mu(x_i - x_{i-1}) in 1-D
    (i >= 1; h_mu the scalar Huber of Eq. 14) by damped Newton with a tridiagonal Hessian."""
    from scipy.linalg import solve_banded
    b = np.asarray(b, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    om = np.ones_like(b) if omtv is None else np.asarray(omtv, dtype=np.float64)
    n = b.size

    def obj(x):
        d = np.diff(x)
        h = np.where(np.abs(d) <= mu, d * d / (2 * mu), np.abs(d) - mu / 2)
        return 0.5 * (w * (x - b) ** 2).sum() + lambda_tv * (om[1:] * h).sum()

    x = b.copy()
    for _ in range(iters):
        d = np.diff(x)
        hp = d / np.maximum(mu, np.abs(d))
        hpp = np.where(np.abs(d) <= mu, 1.0 / mu, 0.0)
        g = w * (x - b)
        tvg = lambda_tv * om[1:] * hp
        g[1:] += tvg
        g[:-1] -= tvg
        c = lambda_tv * om[1:] * hpp
        diag = w.copy()
        diag[1:] += c
        diag[:-1] += c
        ab = np.zeros((3, n))
        ab[0, 1:] = -c
        ab[1] = diag
        ab[2, :-1] = -c
        dx = solve_banded((1, 1), ab, -g)
        f0, t = obj(x), 1.0
        while t > 1e-12:
            if obj(x + t * dx) <= f0 + 1e-4 * t * (g @ dx):
                break
            t *= 0.5
        x = x + t * dx
        if np.abs(t * dx).max() < tol * max(1.0, np.abs(x).max()):
            break
    return x
