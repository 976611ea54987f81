"""GPU kernel-regression back-projection (Sec. 2.2) against the numpy oracle,
and the full M-step pipeline: images -> back-projection -> Fourier-domain
reweighted solve (Eq. 31)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fourier, gridding
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu


def _inputs(n, m, seed, noise_sd=1.0):
    pd = synth.make_projection_data(n, blobs=10, radius=n / 6, n_images=m, seed=seed, noise_sd=noise_sd)
    rot = pd.rot.astype(np.float32)
    X = pd.X.astype(np.complex64)
    ctf = pd.ctf.astype(np.float32)
    return pd, rot, X, ctf


@pytest.mark.parametrize("kernel,posterior", [("gauss", False), ("trilinear", False), ("gauss", True)])
def test_backprojection_matches_oracle(kernel, posterior):
    """(y, N') at 24^3 from 30 image-pose pairs, against the FP64 oracle."""
    n, m = 24, 30
    pd, rot, X, ctf = _inputs(n, m, 81)
    pw = np.random.default_rng(80).uniform(0.0, 1.0, m).astype(np.float32) if posterior else None
    y, N = spg.spg_backproject(rot, X, ctf, pw=pw, kernel=kernel, h=2.0)
    num, Nf = gridding.grid(X.astype(np.complex128), ctf.astype(np.float64), rot.astype(np.float64), n, kernel, 2.0,
                            pw=None if pw is None else pw.astype(np.float64))
    yr, Nr = gridding.to_fourier_term(num, Nf)
    yr, Nr = synth.half_spectrum(yr), synth.half_spectrum(Nr)
    np.testing.assert_allclose(N.cpu().numpy(), Nr, rtol=1e-6, atol=1e-6 * Nr.max())
    np.testing.assert_allclose(y.cpu().numpy(), yr, rtol=1e-5, atol=1e-6 * np.abs(yr).max())


def test_images_to_regularised_map():
    """Back-project 120 images of a 32^3 phantom (Gaussian kernel, h = 2),
    then run the reweighted Fourier-domain solve: the GPU pipeline matches the
    oracle pipeline, and the regularised map correlates with the phantom."""
    n, m = 32, 120
    pd, rot, X, ctf = _inputs(n, m, 82, noise_sd=2.0)
    y, N = spg.spg_backproject(rot, X, ctf, kernel="gauss", h=2.0)
    hyper = dict(synth.DEFAULT_HYPER, mu=0.02, lambda_l1=0.02, lambda_tv=0.05)
    s = spg.SPG(dict(shape=(n, n, n), **hyper))
    s.set_data_fourier(0, y, N)
    s.solve(2, 60)
    x = s.get_x(0).cpu().numpy().astype(np.float64)
    s.close()
    num, Nf = gridding.grid(X.astype(np.complex128), ctf.astype(np.float64), rot.astype(np.float64), n, "gauss", 2.0)
    yr, Nr = gridding.to_fourier_term(num, Nf)
    xr, _, _ = fourier.solve(yr, Nr, oracle.Params((n, n, n), **hyper), 2, 60, with_hist=False)
    err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
    ph = pd.phantom.astype(np.float64)
    corr = float(((x - x.mean()) * (ph - ph.mean())).sum() / np.linalg.norm(x - x.mean()) / np.linalg.norm(ph - ph.mean()))
    print(f"pipeline 32^3, 120 images: rel-L2 vs oracle {err:.2e}, correlation with phantom {corr:.3f}")
    assert err <= 1e-5
    assert corr > 0.8


def test_streaming_accumulator():
    """Batches added to one accumulator (host arrays, CUDA tensors, a finish
    in between) equal the one-shot back-projection; reset empties it."""
    n, m = 20, 24
    pd, rot, X, ctf = _inputs(n, m, 83)
    pw = np.random.default_rng(84).uniform(0.2, 1.0, m).astype(np.float32)
    y1, N1 = spg.spg_backproject(rot, X, ctf, pw=pw)
    g = spg.Grid(n)
    g.add(rot[:10], X[:10], ctf[:10], pw[:10])
    g.finish()  # the sums stay
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g.add(d(rot[10:17]), d(X[10:17]), d(ctf[10:17]), d(pw[10:17]))
    g.add(rot[17:], X[17:], ctf[17:], pw[17:])
    assert g.count() == m
    y2, N2 = g.finish()
    torch.testing.assert_close(N2, N1, rtol=1e-6, atol=1e-6 * float(N1.max()))
    torch.testing.assert_close(y2, y1, rtol=1e-5, atol=1e-6 * float(y1.abs().max()))
    g.reset()
    assert g.count() == 0
    y3, N3 = g.finish()
    assert float(N3.abs().max()) == 0.0 and float(y3.abs().max()) == 0.0
    g.close()


def test_backprojection_repeats_within_rounding():
    """The accumulator takes FP64 global atomics in an order that can change
    between runs, so the double sums differ in their last bits; the outputs
    (y, N') are float32, rounded from those sums (y through num / sqrt(N)),
    so a value near a rounding boundary can land one or two float32 ulps
    apart. Two back-projections of the same images: every value within 4e-7
    relative, and almost all bitwise equal."""
    n, m = 24, 40
    pd, rot, X, ctf = _inputs(n, m, 83)
    y1, N1 = spg.spg_backproject(rot, X, ctf)
    y2, N2 = spg.spg_backproject(rot, X, ctf)
    for a, b in ((y1, y2), (N1, N2)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=4e-7, atol=1e-9 * np.abs(a).max())
        assert np.mean(a != b) < 0.02
