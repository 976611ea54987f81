"""The pins of the numpy oracles catch plausible mistakes in them.

Each case plants one mistake (a wrong constant, sign, index order or
dropped factor) in a copy of oracle/gridding.py, oracle/fourier.py or
oracle/fsc.py, loads the copy as a module, points the pin module at it and
runs that module's pins: at least one must fail. No GPU is involved.
"""
import importlib
import inspect
import types

import numpy as np
import pytest

import test_fourier_oracle
import test_fsc_oracle
import test_gridding_oracle

MUTATIONS = {
    "oracle.gridding": (test_gridding_oracle, "gridding", {
        "Gaussian kernel with exponent over 2h": ("K = np.exp(-(d * d).sum(1) / h)",
                                                  "K = np.exp(-(d * d).sum(1) / (2.0 * h))"),
        "trilinear weight |d| instead of 1 - |d|": ("K = np.prod(1.0 - np.abs(d), axis=1)",
                                                    "K = np.prod(np.abs(d), axis=1)"),
        "trilinear cell from the nearest point": ("base = np.floor(p)", "base = np.rint(p)"),
        "Gaussian neighbourhood around floor(p)": ("base = np.rint(p)", "base = np.floor(p)"),
        "grid index with x and z transposed": ("flat = (gi[:, 2] * n + gi[:, 1]) * n + gi[:, 0]",
                                               "flat = (gi[:, 0] * n + gi[:, 1]) * n + gi[:, 2]"),
        "N without the squared CTF": ("np.add.at(N, flat, P * K * cv * cv)", "np.add.at(N, flat, P * K * cv)"),
        "numerator without the CTF": ("np.add.at(num, flat, P * K * cv * xv)", "np.add.at(num, flat, P * K * xv)"),
        "slice plane from the rotation's rows": (
            "p = rot[i][:, 0][None, :] * kx[:, None] + rot[i][:, 1][None, :] * ky[:, None]",
            "p = rot[i][0, :][None, :] * kx[:, None] + rot[i][1, :][None, :] * ky[:, None]"),
        "posterior weight only on the numerator": ("np.add.at(N, flat, P * K * cv * cv)",
                                                   "np.add.at(N, flat, K * cv * cv)"),
        "Fourier term without the centring sign": ("sign * num / np.sqrt", "num / np.sqrt"),
        "Fourier term without the voxel count": ("return y, V * N", "return y, N"),
        "Fourier term divides by N, not sqrt(N)": ("sign * num / np.sqrt(np.where(N > 0, N, 1.0))",
                                                   "sign * num / np.where(N > 0, N, 1.0)"),
    }),
    "oracle.fourier": (test_fourier_oracle, "fourier", {
        "data gradient with the wrong sign on c": ("np.fft.ifftn(N * np.fft.fftn(x)).real - c",
                                                   "np.fft.ifftn(N * np.fft.fftn(x)).real + c"),
        "c without the square root of N": ("np.fft.ifftn(np.sqrt(N) * y, norm=\"ortho\")",
                                           "np.fft.ifftn(N * y, norm=\"ortho\")"),
        "data gradient with a unitary forward transform": ("np.fft.ifftn(N * np.fft.fftn(x)).real",
                                                           "np.fft.ifftn(N * np.fft.fftn(x, norm=\"ortho\")).real"),
        "data value without the 1/2": ("return 0.5 * float((np.abs(r) ** 2).sum())",
                                       "return float((np.abs(r) ** 2).sum())"),
        "Lipschitz bound without max N": ("L = float(N.max()) + 12.0", "L = 12.0"),
        "gamma term without its factor 2": ("g = g + 2.0 * p.gamma * (yk - p.anchor)",
                                            "g = g + p.gamma * (yk - p.anchor)"),
        "objective without the gamma term": ("(o[0] if p.gamma > 0 else 0.0)", "0.0"),
        "extrapolation with the wrong sign": ("yk = x + beta[k] * (x - xp)", "yk = x - beta[k] * (x - xp)"),
        "soft-threshold without the l1 weight": ("t = tau * p.lambda_l1 * om1", "t = tau * p.lambda_l1"),
    }),
    "oracle.fsc": (test_fsc_oracle, "ofsc", {
        "shell by floor instead of nearest integer": ("return np.rint(r).astype(np.int64)",
                                                      "return np.floor(r).astype(np.int64)"),
        "denominator without the square root": ("out = num / np.sqrt(d1 * d2)", "out = num / (d1 * d2)"),
        "cross term without the conjugate": ("(F * np.conj(G)).real", "(F * G).real"),
        "frequencies as fractions of the box": ("f = np.fft.fftfreq(n) * n", "f = np.fft.fftfreq(n)"),
        "imaginary part of the cross term": ("(F * np.conj(G)).real", "(F * np.conj(G)).imag"),
        "resolution read from shell 0 on": ("for k in range(1, len(curve)):", "for k in range(len(curve)):"),
        "resolution at the first shell above the threshold": ("if curve[k] < threshold:", "if curve[k] > threshold:"),
    }),
}

CASES = [(mod, name) for mod, (_, _, muts) in MUTATIONS.items() for name in muts]


def _mutant(modname, old, new):
    mod = importlib.import_module(modname)
    src = inspect.getsource(mod)
    if old is not None:
        assert old in src, f"anchor of the mutation not found in {modname}"
        src = src.replace(old, new)
    m = types.ModuleType(modname)
    m.__file__ = mod.__file__
    exec(compile(src, mod.__file__, "exec"), m.__dict__)
    return m


def _pins(pinmod):
    """(name, zero-argument callable) for every test function of the pin
    module, one per parameter combination of its parametrize marks."""
    out = []
    for name, fn in vars(pinmod).items():
        if not (name.startswith("test_") and callable(fn)):
            continue
        combos = [{}]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [s.strip() for s in mark.args[0].split(",")]
            vals = [v if len(names) > 1 else (v,) for v in mark.args[1]]
            combos = [dict(c, **dict(zip(names, v))) for c in combos for v in vals]
        for kw in combos:
            out.append((f"{name}{kw or ''}", lambda fn=fn, kw=kw: fn(**kw)))
    return out


@pytest.mark.parametrize("modname", list(MUTATIONS))
def test_pins_pass_on_the_unmodified_oracle(modname, monkeypatch):
    pinmod, attr, _ = MUTATIONS[modname]
    monkeypatch.setattr(pinmod, attr, _mutant(modname, None, None))
    for name, run in _pins(pinmod):
        run()


@pytest.mark.parametrize("modname,mutation", CASES)
def test_a_pin_catches_the_mutation(modname, mutation, monkeypatch):
    pinmod, attr, muts = MUTATIONS[modname]
    old, new = muts[mutation]
    monkeypatch.setattr(pinmod, attr, _mutant(modname, old, new))
    caught = []
    for name, run in _pins(pinmod):
        try:
            with np.errstate(all="ignore"):  # a division by zero is one way a mistake shows
                run()
        except Exception as e:  # an assertion, or the mutant breaking the pin's arithmetic
            caught.append(f"{name}: {type(e).__name__}")
    assert caught, f"no pin of {pinmod.__name__} caught: {mutation}"

