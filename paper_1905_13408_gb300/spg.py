"""Python binding of ``libspg.so`` (include/spg.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
The module-level functions carry the C names (``spg_create``, ``spg_set_data``,
``spg_reweight``, ``spg_iterate``, ...); :class:`SPG` wraps a context for
convenience and :class:`UnrolledSPG` exposes the hand-written adjoint through
``torch.autograd.Function``.

Arrays may be CUDA tensors, CPU tensors or numpy arrays (C-contiguous,
[nz, ny, nx]); the library copies through unified addressing. There is no
fallback: if the library cannot be loaded, or no CUDA device is usable, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspg.so")

SPG_OK, SPG_EINVAL, SPG_ENOMEM, SPG_ECUDA, SPG_ENOTREADY, SPG_ENONFINITE, SPG_ETIMEOUT, SPG_ECHECK = \
    0, -1, -2, -3, -4, -5, -6, -7
SPG_F32, SPG_BF16 = 0, 1
SPG_FISTA, SPG_ISTA = 0, 1
SPG_STORE_DELTA, SPG_STORE_PREV = 0, 1
TILES = {"auto": 0, "128x8": 1, "128x4": 2, "64x8": 3, "64x4": 4, "128x7": 6, "128x15": 7, "64x7": 8,
         "128x7s4": 9}

_STATUS_NAMES = {0: "SPG_OK", -1: "SPG_EINVAL", -2: "SPG_ENOMEM", -3: "SPG_ECUDA", -4: "SPG_ENOTREADY",
                 -5: "SPG_ENONFINITE", -6: "SPG_ETIMEOUT", -7: "SPG_ECHECK"}

# Every entry point declared in include/spg.h.
EXPORTS = ["spg_create", "spg_create_batch", "spg_set_data", "spg_set_x", "spg_get_x", "spg_reweight",
           "spg_iterate", "spg_objective", "spg_history", "spg_round_stats", "spg_certificate", "spg_counters",
           "spg_get_state", "spg_set_state", "spg_backward", "spg_unrolled", "spg_probe_timeout",
           "spg_autotune", "spg_launch_count", "spg_plan_info", "spg_last_error", "spg_destroy",
           "spg_objective_noalloc", "spg_noalloc_last_error", "spg_set_anchor", "spg_param_scales",
           "spg_fsc", "spg_fsc_last_error", "spg_set_data_fourier", "spg_backproject",
           "spg_backproject_last_error", "spg_grid_create", "spg_grid_add", "spg_grid_finish", "spg_grid_reset",
           "spg_grid_count", "spg_grid_last_error", "spg_grid_destroy", "spg_set_halo", "spg_step_bound",
           "spg_set_step_bound", "spg_get_planes", "spg_set_planes", "spg_set_lambdas"]


class SPGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class VolumeParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lambda_l1", ctypes.c_float), ("lambda_tv", ctypes.c_float), ("mu", ctypes.c_float),
                ("eps", ctypes.c_float), ("eps_tv", ctypes.c_float)]


SPG_READ_FORWARD, SPG_READ_PERIODIC, SPG_READ_POST_DIV = 1, 2, 4


def readings_flags(difference="backward", boundary="neumann", tv_weight="inside"):
    """SPG_READ_* flags of a choice of readings (0: the adopted ones)."""
    if difference not in ("backward", "forward") or boundary not in ("neumann", "periodic") \
            or tv_weight not in ("inside", "post_div"):
        raise ValueError("difference: backward|forward, boundary: neumann|periodic, tv_weight: inside|post_div")
    return ((SPG_READ_FORWARD if difference == "forward" else 0) | (SPG_READ_PERIODIC if boundary == "periodic" else 0)
            | (SPG_READ_POST_DIV if tv_weight == "post_div" else 0))


class Options(ctypes.Structure):
    _fields_ = [("data_dtype", ctypes.c_int), ("momentum", ctypes.c_int), ("hist_every", ctypes.c_int),
                ("hist_capacity", ctypes.c_int), ("max_iters_per_round", ctypes.c_int), ("tile", ctypes.c_int),
                ("zchunk", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("iterate_storage", ctypes.c_int),
                ("restart", ctypes.c_int), ("readings", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load():
    """Load libspg.so (building it first if it is missing or stale). With
    SPG_CHECKED=1 in the environment the checked build (device-side index
    checks of the fused step, failures reported as SPG_ECHECK) is built and
    loaded instead."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        checked = os.environ.get("SPG_CHECKED", "0") == "1"
        path = _build.build(checked=checked)
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; the solver has no CPU path")
        lib = ctypes.CDLL(path)
        P, V, I, LL, D = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "spg_create": (I, [ctypes.POINTER(VolumeParams), ctypes.POINTER(Options), P, PP]),
            "spg_create_batch": (I, [I, ctypes.POINTER(VolumeParams), ctypes.POINTER(Options), P, PP]),
            "spg_set_data": (I, [P, I, V, V, I]),
            "spg_set_x": (I, [P, I, V]),
            "spg_get_x": (I, [P, I, V]),
            "spg_reweight": (I, [P]),
            "spg_iterate": (I, [P, I]),
            "spg_objective": (I, [P, I, ctypes.POINTER(D)]),
            "spg_history": (I, [P, I, ctypes.POINTER(D), I, ctypes.POINTER(I)]),
            "spg_round_stats": (I, [P, I, ctypes.POINTER(D)]),
            "spg_certificate": (I, [P, I, ctypes.POINTER(D)]),
            "spg_counters": (I, [P, ctypes.POINTER(LL), ctypes.POINTER(I)]),
            "spg_get_state": (I, [P, V, ctypes.POINTER(ctypes.c_size_t)]),
            "spg_set_state": (I, [P, V, ctypes.c_size_t]),
            "spg_backward": (I, [P, I, V, V, V, ctypes.POINTER(D), I]),
            "spg_unrolled": (I, [P, I, V]),
            "spg_probe_timeout": (I, [P, LL]),
            "spg_autotune": (I, [P, I, ctypes.POINTER(I)]),
            "spg_launch_count": (LL, [P]),
            "spg_plan_info": (I, [P, ctypes.POINTER(I)]),
            "spg_last_error": (ctypes.c_char_p, [P]),
            "spg_destroy": (None, [P]),
            "spg_objective_noalloc": (I, [I, I, I, ctypes.c_float, ctypes.c_float, ctypes.c_float, V, V, V, V, V,
                                          V, P]),
            "spg_noalloc_last_error": (ctypes.c_char_p, []),
            "spg_set_anchor": (I, [P, I, ctypes.c_float, V]),
            "spg_fsc": (I, [I, V, V, I, ctypes.POINTER(D), ctypes.POINTER(D), P]),
            "spg_fsc_last_error": (ctypes.c_char_p, []),
            "spg_set_data_fourier": (I, [P, I, V, V]),
            "spg_backproject": (I, [I, I, V, V, V, V, I, ctypes.c_float, V, V, P]),
            "spg_backproject_last_error": (ctypes.c_char_p, []),
            "spg_grid_create": (I, [I, I, ctypes.c_float, P, PP]),
            "spg_grid_add": (I, [P, I, V, V, V, V]),
            "spg_grid_finish": (I, [P, V, V]),
            "spg_grid_reset": (I, [P]),
            "spg_grid_count": (LL, [P]),
            "spg_grid_last_error": (ctypes.c_char_p, [P]),
            "spg_grid_destroy": (None, [P]),
            "spg_param_scales": (I, [P, I, ctypes.POINTER(D)]),
            "spg_set_halo": (I, [P, I, I, I]),
            "spg_step_bound": (I, [P, I, ctypes.POINTER(D)]),
            "spg_set_step_bound": (I, [P, I, D, D]),
            "spg_get_planes": (I, [P, I, I, I, V, V]),
            "spg_set_planes": (I, [P, I, I, I, V, V]),
            "spg_set_lambdas": (I, [P, I, ctypes.c_float, ctypes.c_float]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status, handle=None):
    if status != SPG_OK:
        msg = load().spg_last_error(handle)
        raise SPGError(status, msg.decode() if msg else "")


def _ptr(a, dtype="f32"):
    """(pointer, keepalive) of a contiguous tensor / array of the given dtype."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float32 if dtype == "f32" else torch.bfloat16
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    a = np.asarray(a)
    if dtype == "f32":
        if a.dtype != np.float32:
            raise TypeError(f"expected float32, got {a.dtype}")
    elif a.dtype not in (np.uint16, np.int16):
        raise TypeError("bfloat16 numpy data must be passed as uint16 bit patterns")
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), a


# ---------- C-named functions (handles are ctypes.c_void_p) ----------

def spg_create_batch(params, options=None, stream=None):
    arr = (VolumeParams * len(params))(*params)
    h = ctypes.c_void_p()
    opt = ctypes.byref(options) if options is not None else None
    _check(load().spg_create_batch(len(params), arr, opt, ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def spg_create(params, options=None, stream=None):
    return spg_create_batch([params], options, stream)


def spg_set_data(h, vol, b, w, dtype=SPG_F32):
    dt = "f32" if dtype == SPG_F32 else "bf16"
    pb, kb = _ptr(b, dt)
    pw, kw = _ptr(w, dt)
    _check(load().spg_set_data(h, vol, pb, pw, dtype), h)


def spg_set_anchor(h, vol, gamma, x_anchor):
    pa, ka = _ptr(x_anchor)
    _check(load().spg_set_anchor(h, vol, float(gamma), pa), h)


def spg_param_scales(h, vol=0):
    out = (ctypes.c_double * 4)()
    _check(load().spg_param_scales(h, vol, out), h)
    return dict(zip(["rms_wb", "mean_w", "max_w", "min_w"], out[:]))


def spg_fsc(a, b, stream=None):
    """(fsc, counts) for shells 0 .. n/2 of two n^3 float32 maps (Eq. 30)."""
    n = int(a.shape[0])
    pa, ka = _ptr(a)
    pb, kb = _ptr(b)
    m = n // 2 + 1
    fsc = np.zeros(m)
    cnt = np.zeros(m)
    st = load().spg_fsc(n, pa, pb, m, fsc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(stream or 0))
    if st != SPG_OK:
        raise SPGError(st, load().spg_fsc_last_error().decode())
    return fsc, cnt


def _ptr_complex64(a):
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.complex64 or not a.is_contiguous():
            raise TypeError("expected a contiguous complex64 tensor")
        return ctypes.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a, dtype=np.complex64)
    return ctypes.c_void_p(a.ctypes.data), a


def spg_set_data_fourier(h, vol, y_half, N_half):
    """Fourier-domain data term (Eq. 31): y_half complex64 and N_half float32,
    both [nz, ny, nx//2 + 1] (the real-to-complex half spectrum)."""
    py, ky = _ptr_complex64(y_half)
    pn, kn = _ptr(N_half)
    _check(load().spg_set_data_fourier(h, vol, py, pn), h)


def _grid_inputs(rot, X, ctf, pw):
    """Marshal (rot, X, ctf, pw) to pointers; numpy arrays become contiguous
    float32 / complex64 host arrays, torch tensors are passed as they are."""
    import torch
    keep = []

    def f32(a):
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise TypeError("expected a contiguous float32 tensor")
            keep.append(a)
            return ctypes.c_void_p(a.data_ptr())
        a = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(a)
        return ctypes.c_void_p(a.ctypes.data)

    pX, kX = _ptr_complex64(X)
    keep.append(kX)
    ptrs = (f32(rot), pX, f32(ctf), ctypes.c_void_p(0) if pw is None else f32(pw))
    return ptrs, keep


class Grid:
    """Streaming kernel-regression back-projection (Sec. 2.2, Eq. 24-28):
    add batches of image-pose pairs, then finish into the (y_half, N_half)
    of the Fourier-domain data term."""

    def __init__(self, n, kernel="gauss", h=2.0, stream=None):
        self.n = int(n)
        out = ctypes.c_void_p()
        st = load().spg_grid_create(self.n, 0 if kernel == "gauss" else 1, float(h), ctypes.c_void_p(stream or 0),
                                    ctypes.byref(out))
        if st != SPG_OK:
            raise SPGError(st, load().spg_grid_last_error(None).decode())
        self.handle = out
        self._keep = []

    def _check(self, st):
        if st != SPG_OK:
            raise SPGError(st, load().spg_grid_last_error(self.handle).decode())

    def add(self, rot, X, ctf, pw=None):
        """rot [m, 3, 3], X [m, n, n] complex, ctf [m, n, n], pw [m] or None
        (numpy arrays are staged through host memory; CUDA tensors are read
        in place and kept alive until finish)."""
        m = int(np.shape(rot)[0])
        (pr, pX, pc, pp), keep = _grid_inputs(rot, X, ctf, pw)
        self._check(load().spg_grid_add(self.handle, m, pr, pX, pc, pp))
        self._keep.extend(keep)

    def finish(self):
        """(y_half complex64, N_half float32) CUDA tensors [n, n, n/2+1]."""
        import torch
        n = self.n
        y = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
        N = torch.empty((n, n, n // 2 + 1), dtype=torch.float32, device="cuda")
        self._check(load().spg_grid_finish(self.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(N.data_ptr())))
        self._keep = []
        return y, N

    def reset(self):
        self._check(load().spg_grid_reset(self.handle))

    def count(self):
        return int(load().spg_grid_count(self.handle))

    def close(self):
        if self.handle:
            load().spg_grid_destroy(self.handle)
            self.handle = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spg_backproject(rot, X, ctf, pw=None, kernel="gauss", h=2.0, stream=None):
    """(y_half complex64, N_half float32) on the GPU of m n x n images
    (rot [m, 3, 3], X [m, n, n] complex, ctf [m, n, n], optional posterior
    weights pw [m]); kernel "gauss" or "trilinear" (Sec. 2.2)."""
    import torch
    m, n = int(np.shape(rot)[0]), int(X.shape[-1])
    (pr, pX, pc, pp), keep = _grid_inputs(rot, X, ctf, pw)
    y = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    N = torch.empty((n, n, n // 2 + 1), dtype=torch.float32, device="cuda")
    st = load().spg_backproject(n, m, pr, pX, pc, pp, 0 if kernel == "gauss" else 1, float(h),
                                ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(N.data_ptr()),
                                ctypes.c_void_p(stream or 0))
    if st != SPG_OK:
        raise SPGError(st, load().spg_backproject_last_error().decode())
    return y, N


def spg_set_x(h, vol, x):
    px, kx = _ptr(x)
    _check(load().spg_set_x(h, vol, px), h)


def spg_get_x(h, vol, out):
    px, kx = _ptr(out)
    _check(load().spg_get_x(h, vol, px), h)
    return out


def spg_reweight(h):
    _check(load().spg_reweight(h), h)


def spg_iterate(h, k):
    _check(load().spg_iterate(h, int(k)), h)


def spg_objective(h, vol=0):
    out = (ctypes.c_double * 4)()
    _check(load().spg_objective(h, vol, out), h)
    return np.array(out[:])


def spg_history(h, vol=0, max_entries=8192):
    n = ctypes.c_int()
    buf = np.zeros((max_entries, 5))
    _check(load().spg_history(h, vol, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), max_entries,
                              ctypes.byref(n)), h)
    return buf[:n.value].copy()


def spg_round_stats(h, vol=0):
    out = (ctypes.c_double * 6)()
    _check(load().spg_round_stats(h, vol, out), h)
    return np.array(out[:])


def spg_set_halo(h, vol, lo, hi):
    _check(load().spg_set_halo(h, int(vol), int(lo), int(hi)), h)


def spg_step_bound(h, vol=0):
    out = (ctypes.c_double * 2)()
    _check(load().spg_step_bound(h, int(vol), out), h)
    return float(out[0]), float(out[1])


def spg_set_step_bound(h, vol, max_w, max_omtv):
    _check(load().spg_set_step_bound(h, int(vol), float(max_w), float(max_omtv)), h)


def spg_set_lambdas(h, vol, lambda_l1, lambda_tv):
    _check(load().spg_set_lambdas(h, int(vol), float(lambda_l1), float(lambda_tv)), h)


def _opt_ptr(a):
    return (None, None) if a is None else _ptr(a)


def spg_get_planes(h, vol, z0, n, x, pair):
    px, kx = _opt_ptr(x)
    pp, kp = _opt_ptr(pair)
    _check(load().spg_get_planes(h, int(vol), int(z0), int(n), px, pp), h)


def spg_set_planes(h, vol, z0, n, x, pair):
    px, kx = _opt_ptr(x)
    pp, kp = _opt_ptr(pair)
    _check(load().spg_set_planes(h, int(vol), int(z0), int(n), px, pp), h)


def spg_certificate(h, vol=0):
    out = ctypes.c_double()
    _check(load().spg_certificate(h, vol, ctypes.byref(out)), h)
    return out.value


def spg_counters(h):
    kt, kr = ctypes.c_longlong(), ctypes.c_int()
    _check(load().spg_counters(h, ctypes.byref(kt), ctypes.byref(kr)), h)
    return kt.value, kr.value


def spg_get_state(h):
    n = ctypes.c_size_t()
    _check(load().spg_get_state(h, None, ctypes.byref(n)), h)
    buf = ctypes.create_string_buffer(n.value)
    _check(load().spg_get_state(h, buf, ctypes.byref(n)), h)
    return buf.raw


STATE_HEADER_BYTES = 48


def parse_state(blob, shapes):
    """Split a state blob (spg_get_state) into per-volume numpy views:
    dicts with x, x_prev (float64, exact), om1, omtv (float32 [nz, ny, nx]),
    tau and stats; with increment storage also d (float32)."""
    hdr = np.frombuffer(blob, dtype=np.int32, count=12, offset=0)
    k_round = int(hdr[4])
    storage = int(hdr[10])
    k_total = int(np.frombuffer(blob, dtype=np.int64, count=1, offset=24)[0])
    off = STATE_HEADER_BYTES
    vols = []
    for sh in shapes:
        n = int(np.prod(sh))
        arr = np.frombuffer(blob, dtype=np.float32, count=4 * n, offset=off).reshape(4, *sh)
        off += 16 * n
        tau = float(np.frombuffer(blob, dtype=np.float32, count=1, offset=off)[0])
        beta_last = float(np.frombuffer(blob, dtype=np.float32, count=1, offset=off + 4)[0])
        kmom = int(np.frombuffer(blob, dtype=np.int32, count=1, offset=off + 8)[0])
        off += 16
        stats = np.frombuffer(blob, dtype=np.float64, count=6, offset=off).copy() if off % 8 == 0 else \
            np.frombuffer(bytes(blob[off:off + 48]), dtype=np.float64).copy()
        off += 48
        v = dict(x=arr[0], om1=arr[2], omtv=arr[3], tau=tau, stats=stats, beta_last=beta_last, kmom=kmom)
        if storage == SPG_STORE_DELTA:
            v["d"] = arr[1]
            # the difference of two float32 values is exact in float64 here
            v["x_prev"] = arr[0].astype(np.float64) - arr[1].astype(np.float64)
        else:
            v["x_prev"] = arr[1]
        vols.append(v)
    return dict(k_round=k_round, k_total=k_total, storage=storage, volumes=vols)


def spg_set_state(h, blob):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().spg_set_state(h, buf, len(blob)), h)


def spg_backward(h, K, gx, gb, gw, ckpt_every=10):
    px, kx = _ptr(gx)
    pb, kb = _ptr(gb)
    pw, kw = _ptr(gw)
    gs = (ctypes.c_double * 2)()
    _check(load().spg_backward(h, int(K), px, pb, pw, gs, int(ckpt_every)), h)
    return np.array(gs[:])


def spg_unrolled(h, K, out):
    px, kx = _ptr(out)
    _check(load().spg_unrolled(h, int(K), px), h)
    return out


def spg_probe_timeout(h, timeout_ns):
    return load().spg_probe_timeout(h, int(timeout_ns))


def spg_autotune(h, trial_iters=10):
    info = (ctypes.c_int * 6)()
    _check(load().spg_autotune(h, int(trial_iters), info), h)
    return dict(zip(["tile_x", "tile_y", "zchunk", "items", "grid", "ctas_per_sm"], info[:]))


def spg_launch_count(h):
    return int(load().spg_launch_count(h))


def spg_plan_info(h):
    info = (ctypes.c_int * 6)()
    _check(load().spg_plan_info(h, info), h)
    return dict(zip(["tile_x", "tile_y", "zchunk", "items", "grid", "ctas_per_sm"], info[:]))


def spg_last_error(h=None):
    m = load().spg_last_error(h)
    return m.decode() if m else ""


def spg_destroy(h):
    if h:
        load().spg_destroy(h)


# ---------- convenience wrapper ----------

def volume_params(shape, lambda_l1=0.05, lambda_tv=0.1, mu=1e-3, eps=1e-3, eps_tv=None):
    nz, ny, nx = shape
    return VolumeParams(nx, ny, nz, lambda_l1, lambda_tv, mu, eps, eps if eps_tv is None else eps_tv)


class SPG:
    """A solver context over one or more volumes (one fused launch per iteration)."""

    def __init__(self, volumes, data_dtype="f32", momentum="fista", hist_every=1, hist_capacity=4096,
                 max_iters=100000, tile="auto", zchunk=0, ctas_per_sm=0, storage="delta", restart=False,
                 stream=None, difference="backward", boundary="neumann", tv_weight="inside"):
        if isinstance(volumes, dict):
            volumes = [volumes]
        self.shapes = [tuple(v["shape"]) for v in volumes]
        params = [volume_params(v["shape"], **{k: v[k] for k in v if k != "shape"}) for v in volumes]
        opt = Options(SPG_F32 if data_dtype == "f32" else SPG_BF16, SPG_FISTA if momentum == "fista" else SPG_ISTA,
                      hist_every, hist_capacity, max_iters, TILES[tile] if isinstance(tile, str) else int(tile),
                      zchunk, ctas_per_sm, SPG_STORE_DELTA if storage == "delta" else SPG_STORE_PREV,
                      1 if restart else 0, readings_flags(difference, boundary, tv_weight))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.handle = spg_create_batch(params, opt, stream)

    @property
    def nvol(self):
        return len(self.shapes)

    def set_data(self, vol, b, w, dtype=SPG_F32):
        spg_set_data(self.handle, vol, b, w, dtype)

    def set_x(self, vol, x):
        spg_set_x(self.handle, vol, x)

    def set_lambdas(self, vol, lambda_l1, lambda_tv):
        spg_set_lambdas(self.handle, vol, lambda_l1, lambda_tv)

    def set_data_fourier(self, vol, y_half, N_half):
        spg_set_data_fourier(self.handle, vol, y_half, N_half)

    def set_anchor(self, vol, gamma, x_anchor):
        spg_set_anchor(self.handle, vol, gamma, x_anchor)

    def param_scales(self, vol=0):
        return spg_param_scales(self.handle, vol)

    def get_x(self, vol=0, out=None):
        import torch
        if out is None:
            out = torch.empty(self.shapes[vol], dtype=torch.float32, device="cuda")
        spg_get_x(self.handle, vol, out)
        return out

    def reweight(self):
        spg_reweight(self.handle)

    def iterate(self, k):
        spg_iterate(self.handle, k)

    def objective(self, vol=0):
        return spg_objective(self.handle, vol)

    def history(self, vol=0):
        return spg_history(self.handle, vol)

    def round_stats(self, vol=0):
        return spg_round_stats(self.handle, vol)

    def certificate(self, vol=0):
        return spg_certificate(self.handle, vol)

    def set_halo(self, vol, lo, hi):
        spg_set_halo(self.handle, vol, lo, hi)

    def step_bound(self, vol=0):
        return spg_step_bound(self.handle, vol)

    def set_step_bound(self, vol, max_w, max_omtv):
        spg_set_step_bound(self.handle, vol, max_w, max_omtv)

    def get_planes(self, vol, z0, n):
        """(x, pair) planes [z0, z0 + n) of the current iterate pair, as CUDA tensors."""
        import torch
        nz, ny, nx = self.shapes[vol]
        x = torch.empty((n, ny, nx), dtype=torch.float32, device="cuda")
        p = torch.empty_like(x)
        spg_get_planes(self.handle, vol, z0, n, x, p)
        return x, p

    def set_planes(self, vol, z0, x, pair):
        spg_set_planes(self.handle, vol, z0, x.shape[0], x.contiguous(), pair.contiguous())

    def counters(self):
        return spg_counters(self.handle)

    def get_state(self):
        return spg_get_state(self.handle)

    def set_state(self, blob):
        spg_set_state(self.handle, blob)

    def launch_count(self):
        return spg_launch_count(self.handle)

    def plan_info(self):
        return spg_plan_info(self.handle)

    def autotune(self, trial_iters=10):
        return spg_autotune(self.handle, trial_iters)

    def solve(self, rounds, iters):
        for _ in range(rounds):
            self.reweight()
            self.iterate(iters)

    def close(self):
        if getattr(self, "handle", None):
            spg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# Idle contexts of UnrolledSPG, by (shape, mu, eps, eps_tv, momentum, device,
# stream). A forward takes one (or creates one) and re-sets its weights and
# data; its backward hands it back. A loop of forward/backward calls thus
# creates one context, whose workspace the later calls reuse. At most two
# idle contexts are kept per key.
_UNROLLED_POOL = {}
_UNROLLED_LOCK = threading.Lock()


def _unrolled_ctx(b, w, lambda_l1, lambda_tv, mu, eps, eps_tv, momentum):
    import torch
    stream = torch.cuda.current_stream(b.device).cuda_stream
    key = (tuple(b.shape), float(mu), float(eps), float(eps_tv), momentum, b.device.index, stream)
    with _UNROLLED_LOCK:
        idle = _UNROLLED_POOL.get(key)
        s = idle.pop() if idle else None
    if s is None:
        p = dict(shape=tuple(b.shape), lambda_l1=float(lambda_l1), lambda_tv=float(lambda_tv), mu=mu, eps=eps,
                 eps_tv=eps_tv)
        s = SPG(p, momentum=momentum, hist_every=1 << 30, stream=stream)
    else:
        s.set_lambdas(0, lambda_l1, lambda_tv)
    s.pool_key = key
    # the context's own iterate stays x_0 = 0: spg_unrolled and spg_backward
    # work on copies
    s.set_data(0, b.detach().contiguous(), w.detach().contiguous())
    s.reweight()  # from x_0 = 0: om1 = omtv = 1, tau = 1/L
    return s


def _unrolled_release(s):
    with _UNROLLED_LOCK:
        idle = _UNROLLED_POOL.setdefault(s.pool_key, [])
        if len(idle) < 2:
            idle.append(s)
            return
    s.close()


class UnrolledSPG:
    """x_K of K iterations of one round from x_0 = 0 (weights 1, tau fixed),
    differentiable w.r.t. b, w, lambda_l1 and lambda_tv through the
    hand-written adjoint with checkpoints every ``ckpt_every`` iterations."""

    @staticmethod
    def apply(b, w, lambda_l1, lambda_tv, K, mu=1e-3, eps=1e-3, eps_tv=1e-3, momentum="fista", ckpt_every=10):
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(fctx, b_, w_, l1_, tv_):
                s = _unrolled_ctx(b_, w_, l1_, tv_, mu, eps, eps_tv, momentum)
                out = torch.empty_like(b_)
                spg_unrolled(s.handle, K, out)
                fctx.solver = s
                fctx.scalar_like = (l1_, tv_)
                return out

            @staticmethod
            def backward(fctx, gx):
                s = fctx.solver
                if s is None:
                    raise RuntimeError("UnrolledSPG: one backward per forward")
                fctx.solver = None
                gb = torch.empty_like(gx)
                gw = torch.empty_like(gx)
                try:
                    gs = spg_backward(s.handle, K, gx.contiguous(), gb, gw, ckpt_every)
                except BaseException:
                    s.close()
                    raise
                _unrolled_release(s)
                l1_, tv_ = fctx.scalar_like
                return (gb, gw, torch.tensor(gs[0], dtype=l1_.dtype, device=l1_.device),
                        torch.tensor(gs[1], dtype=tv_.dtype, device=tv_.device))

        l1 = lambda_l1 if isinstance(lambda_l1, torch.Tensor) else torch.tensor(float(lambda_l1))
        tv = lambda_tv if isinstance(lambda_tv, torch.Tensor) else torch.tensor(float(lambda_tv))
        return _F.apply(b, w, l1, tv)
