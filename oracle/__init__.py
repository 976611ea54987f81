"""FP64 CPU oracle of the reweighted smoothing-proximal-gradient solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
and by the benchmark's CPU-baseline leg. The CUDA library and its Python
binding never import it.

Thin ctypes wrapper over ``spg_oracle.c`` (plain C, double precision). All
arrays are float64 numpy arrays of shape [nz, ny, nx] (x fastest). The
definitions each function follows are written at the top of ``spg_oracle.c``
(Eq. 11, 12, 14, 16, 17, 20, 21 and 31 of the paper).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spg_oracle.c")
_LIB = os.path.join(_HERE, "libspg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (portable flags, OpenMP over z-planes)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _P(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lambda_l1", ctypes.c_double), ("lambda_tv", ctypes.c_double),
                ("mu", ctypes.c_double), ("eps", ctypes.c_double), ("eps_tv", ctypes.c_double),
                ("momentum", ctypes.c_int), ("restart", ctypes.c_int), ("gamma", ctypes.c_double),
                ("anchor", ctypes.c_void_p), ("forward", ctypes.c_int), ("periodic", ctypes.c_int),
                ("post_div", ctypes.c_int)]


@dataclass
class Params:
    shape: tuple            # (nz, ny, nx)
    lambda_l1: float = 0.05
    lambda_tv: float = 0.1
    mu: float = 1e-3
    eps: float = 1e-3
    eps_tv: float = 1e-3
    momentum: str = "fista"  # "fista" or "ista"
    restart: bool = False    # gradient restart of the extrapolation
    gamma: float = 0.0       # implicit-gradient term gamma |x - anchor|^2 (Eq. 22)
    anchor: np.ndarray = None
    # alternative readings (the adopted ones are the defaults): Eq. 12's
    # backward differences or forward ones; differences vanishing at the
    # volume's edge (Neumann) or wrapping around it (periodic); the TV weight
    # inside the divergence, D^T(omtv grad h), or after it as Eq. 20 prints it
    difference: str = "backward"   # "backward" | "forward"
    boundary: str = "neumann"      # "neumann" | "periodic"
    tv_weight: str = "inside"      # "inside" | "post_div"

    def adopted_readings(self):
        return (self.difference, self.boundary, self.tv_weight) == ("backward", "neumann", "inside")

    def c(self):
        nz, ny, nx = self.shape
        if self.gamma > 0:
            self._anchor = np.ascontiguousarray(self.anchor, dtype=np.float64)
            assert self._anchor.shape == tuple(self.shape)
            ptr = self._anchor.ctypes.data
        else:
            ptr = None
        assert self.difference in ("backward", "forward") and self.boundary in ("neumann", "periodic")
        assert self.tv_weight in ("inside", "post_div")
        return _P(nx, ny, nz, self.lambda_l1, self.lambda_tv, self.mu, self.eps, self.eps_tv,
                  0 if self.momentum == "fista" else 1, 1 if self.restart else 0, self.gamma, ptr,
                  int(self.difference == "forward"), int(self.boundary == "periodic"),
                  int(self.tv_weight == "post_div"))


_D = ctypes.POINTER(ctypes.c_double)


def _bind(path):
    lib = ctypes.CDLL(path)
    PP = ctypes.POINTER(_P)
    sig = {
        "orc_soft": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
        "orc_huber": (ctypes.c_double, [ctypes.c_double] * 4),
        "orc_huber_grad": (None, [ctypes.c_double] * 4 + [_D]),
        "orc_grad": (None, [PP, _D, _D]),
        "orc_div": (None, [PP, _D, _D]),
        "orc_tv_grad": (None, [PP, _D, _D, _D]),
        "orc_grad_f": (None, [PP, _D, _D, _D, _D, _D]),
        "orc_objective": (None, [PP, _D, _D, _D, _D, _D, _D]),
        "orc_reweight": (None, [PP, _D, _D, _D, _D]),
        "orc_lipschitz": (ctypes.c_double, [PP, _D, ctypes.c_double]),
        "orc_beta_table": (None, [ctypes.c_int, ctypes.c_int, _D]),
        "orc_step": (None, [PP, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D]),
        "orc_solve": (ctypes.c_int, [PP, _D, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]),
        "orc_unrolled": (None, [PP, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D]),
        "orc_certificate": (ctypes.c_double, [PP, _D, _D, ctypes.c_double, _D, _D, _D]),
        "orc_unrolled_counts": (None, [PP, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D,
                                       ctypes.POINTER(ctypes.c_longlong)]),
        "orc_unrolled_active": (ctypes.c_longlong, [PP, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D]),
        "orc_step_sampled": (None, [PP, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D,
                                    ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _D]),
        "orc_backward": (ctypes.c_int, [PP, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D,
                                        _D, _D, _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


@contextlib.contextmanager
def using_library(path):
    """Temporarily route every wrapper call to another build of the oracle
    (used by the tests that plant mistakes in a copy of the source)."""
    global _lib
    _load()
    old = _lib
    _lib = _bind(path)
    try:
        yield
    finally:
        _lib = old


def _a(x, shape=None):
    """Contiguous float64 view (copy if needed) and its pointer."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        assert a.shape == tuple(shape), (a.shape, shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _opt(a, shape):
    return None if a is None else _a(a, shape)


# ---------- closed forms ----------

def soft(z, t):
    return _load().orc_soft(float(z), float(t))


def huber(z, mu):
    return _load().orc_huber(float(z[0]), float(z[1]), float(z[2]), float(mu))


def huber_grad(z, mu):
    out = np.zeros(3)
    _load().orc_huber_grad(float(z[0]), float(z[1]), float(z[2]), float(mu), _ptr(out))
    return out


# ---------- operators ----------

def grad(x, p: Params = None):
    x = _a(x)
    p = p or Params(x.shape)
    g = np.empty((3,) + x.shape)
    _load().orc_grad(ctypes.byref(p.c()), _ptr(x), _ptr(g))
    return g


def div(u, p: Params = None):
    u = _a(u)
    p = p or Params(u.shape[1:])
    out = np.empty(u.shape[1:])
    _load().orc_div(ctypes.byref(p.c()), _ptr(u), _ptr(out))
    return out


def tv_grad(x, omtv, p: Params):
    x = _a(x, p.shape)
    om = _opt(omtv, p.shape)
    out = np.empty(p.shape)
    _load().orc_tv_grad(ctypes.byref(p.c()), _ptr(x), _ptr(om), _ptr(out))
    return out


def grad_f(x, b, w, omtv, p: Params):
    x, b, w = _a(x, p.shape), _a(b, p.shape), _a(w, p.shape)
    om = _opt(omtv, p.shape)
    out = np.empty(p.shape)
    _load().orc_grad_f(ctypes.byref(p.c()), _ptr(x), _ptr(b), _ptr(w), _ptr(om), _ptr(out))
    return out


def objective(x, b, w, om1, omtv, p: Params):
    """(data, l1, tv, total) of the round objective at x."""
    x, b, w = _a(x, p.shape), _a(b, p.shape), _a(w, p.shape)
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    out = np.zeros(4)
    _load().orc_objective(ctypes.byref(p.c()), _ptr(x), _ptr(b), _ptr(w), _ptr(o1), _ptr(ot), _ptr(out))
    return out


def reweight(x, p: Params):
    """(om1, omtv, stats) with stats = (max omtv, nnz, sum om1, sum omtv)."""
    x = _a(x, p.shape)
    om1, omtv, st = np.empty(p.shape), np.empty(p.shape), np.zeros(4)
    _load().orc_reweight(ctypes.byref(p.c()), _ptr(x), _ptr(om1), _ptr(omtv), _ptr(st))
    return om1, omtv, st


def lipschitz(w, max_omtv, p: Params):
    w = _a(w, p.shape)
    return _load().orc_lipschitz(ctypes.byref(p.c()), _ptr(w), float(max_omtv))


def beta_table(iters, momentum="fista"):
    out = np.zeros(max(iters, 1))
    _load().orc_beta_table(0 if momentum == "fista" else 1, int(iters), _ptr(out))
    return out[:iters]


def step(xk, xkm1, beta, tau, b, w, om1, omtv, p: Params):
    xk, xkm1, b, w = (_a(a, p.shape) for a in (xk, xkm1, b, w))
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    out = np.empty(p.shape)
    _load().orc_step(ctypes.byref(p.c()), _ptr(xk), _ptr(xkm1), float(beta), float(tau), _ptr(b),
                     _ptr(w), _ptr(o1), _ptr(ot), _ptr(out))
    return out


def step_sampled(xk, xkm1, beta, tau, b, w, om1, omtv, p: Params, idx):
    """x_{k+1} at flat voxel indices ``idx``, each evaluated around that voxel
    (adopted readings only)."""
    if not p.adopted_readings():
        raise ValueError("step_sampled implements the adopted readings only")
    xk, xkm1, b, w = (_a(a, p.shape) for a in (xk, xkm1, b, w))
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.shape[0])
    _load().orc_step_sampled(ctypes.byref(p.c()), _ptr(xk), _ptr(xkm1), float(beta), float(tau),
                             _ptr(b), _ptr(w), _ptr(o1), _ptr(ot), idx.shape[0],
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(out))
    return out


@dataclass
class SolveResult:
    x: np.ndarray
    hist: np.ndarray     # [rounds, iters, 4]: F(x_k) = (data, l1, tv, total) before step k
    rstats: np.ndarray   # [rounds, 6]: max omtv, nnz, sum om1, sum omtv, L, tau
    om1: np.ndarray
    omtv: np.ndarray


def solve(b, w, p: Params, rounds, iters, x0=None, with_hist=True):
    b, w = _a(b, p.shape), _a(w, p.shape)
    x = np.zeros(p.shape) if x0 is None else _a(x0, p.shape).copy()
    hist = np.zeros((rounds, iters, 4)) if with_hist else None
    rst = np.zeros((rounds, 6))
    om1, omtv = np.empty(p.shape), np.empty(p.shape)
    rc = _load().orc_solve(ctypes.byref(p.c()), _ptr(b), _ptr(w), int(rounds), int(iters), _ptr(x),
                           _ptr(hist), _ptr(rst), _ptr(om1), _ptr(omtv))
    if rc != 0:
        raise MemoryError("oracle solve: allocation failed")
    return SolveResult(x=x, hist=hist, rstats=rst, om1=om1, omtv=omtv)


def unrolled(b, w, om1, omtv, tau, iters, x0, p: Params):
    b, w, x0 = _a(b, p.shape), _a(w, p.shape), _a(x0, p.shape)
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    out = np.empty(p.shape)
    _load().orc_unrolled(ctypes.byref(p.c()), _ptr(b), _ptr(w), _ptr(o1), _ptr(ot), float(tau),
                         int(iters), _ptr(x0), _ptr(out))
    return out


def unrolled_active(b, w, om1, omtv, tau, iters, x0, p: Params):
    """(x_K, number of voxel-steps where the soft-threshold passed)."""
    b, w, x0 = _a(b, p.shape), _a(w, p.shape), _a(x0, p.shape)
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    out = np.empty(p.shape)
    n = _load().orc_unrolled_active(ctypes.byref(p.c()), _ptr(b), _ptr(w), _ptr(o1), _ptr(ot), float(tau),
                                    int(iters), _ptr(x0), _ptr(out))
    return out, int(n)


def unrolled_counts(b, w, om1, omtv, tau, iters, x0, p: Params):
    """(x_K, (soft-threshold passes, voxel-steps on the quadratic branch of the
    smoothed norm)): the two kinds of kink of the unrolled map."""
    b, w, x0 = _a(b, p.shape), _a(w, p.shape), _a(x0, p.shape)
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    out = np.empty(p.shape)
    cnt = (ctypes.c_longlong * 2)()
    _load().orc_unrolled_counts(ctypes.byref(p.c()), _ptr(b), _ptr(w), _ptr(o1), _ptr(ot), float(tau),
                                int(iters), _ptr(x0), _ptr(out), cnt)
    return out, (int(cnt[0]), int(cnt[1]))


def certificate(y, xplus, tau, b, w, omtv, p: Params):
    y, xplus, b, w = (_a(a, p.shape) for a in (y, xplus, b, w))
    ot = _opt(omtv, p.shape)
    return _load().orc_certificate(ctypes.byref(p.c()), _ptr(y), _ptr(xplus), float(tau), _ptr(b),
                                   _ptr(w), _ptr(ot))


def backward(b, w, om1, omtv, tau, iters, x0, gK, p: Params):
    """(dL/db, dL/dw, (dL/dlambda_l1, dL/dlambda_tv)) through `iters` steps
    (adopted readings only)."""
    if not p.adopted_readings():
        raise ValueError("backward implements the adopted readings only")
    b, w, x0, gK = (_a(a, p.shape) for a in (b, w, x0, gK))
    o1, ot = _opt(om1, p.shape), _opt(omtv, p.shape)
    gb, gw, gs = np.empty(p.shape), np.empty(p.shape), np.zeros(2)
    rc = _load().orc_backward(ctypes.byref(p.c()), _ptr(b), _ptr(w), _ptr(o1), _ptr(ot), float(tau),
                              int(iters), _ptr(x0), _ptr(gK), _ptr(gb), _ptr(gw), _ptr(gs))
    if rc != 0:
        raise MemoryError("oracle backward: allocation failed")
    return gb, gw, gs
