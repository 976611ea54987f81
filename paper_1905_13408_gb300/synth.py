"""Seeded synthetic inputs for the regularized real-space refinement solve.

This module draws the data volume ``b``, the weight volume ``w`` and the
ground-truth phantom that both the CUDA path and the FP64 oracle consume. It
holds none of the solver's arithmetic: it only renders a density, a smooth
positive weight field and noise.

Model (stand-in for the paper's back-projected cryo-EM maps, Sec. 2.2 Eq. 28,
where ``b`` is the kernel-regression numerator divided by ``N(n)`` and ``w`` is
``N(n)``):

* phantom: isotropic Gaussian blobs ``A exp(-|p-c|^2 / (2 s^2))`` truncated at
  ``5 s``, with ``s ~ U(1.5, 3)`` voxels, ``A ~ U(0.5, 1)`` and centres uniform
  inside a ball of radius ``R`` about the volume centre ``(n-1)/2``
  (radius ``R U^(1/3)``, isotropic direction);
* weight: ``w = exp(0.5 g)`` where ``g`` is white noise smoothed by a periodic
  Gaussian of ``sigma = 4`` voxels (FFT) and re-normalised to unit variance.
  An uneven ``w`` models uneven angular coverage (Sec. 1);
* data: ``b = phantom + N(0, 0.3^2) / sqrt(w)``.

Draw order from ``numpy.random.default_rng(seed)``: centres, sigmas,
amplitudes, field noise, data noise.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# The named workloads: (edge, blobs, ball radius, rounds, iterations, seed).
WORKLOADS = {
    "vol64": dict(n=64, blobs=40, radius=24.0, rounds=3, iters=200, seed=1000),
    "vol256": dict(n=256, blobs=1600, radius=100.0, rounds=3, iters=300, seed=1001),
    "vol512": dict(n=512, blobs=12800, radius=200.0, rounds=3, iters=None, seed=1002),
    "vol128_adjoint": dict(n=128, blobs=200, radius=50.0, rounds=1, iters=50, seed=1004),
}

# Hyper-parameters shared by the workloads (lambda_l1, lambda_tv, mu, eps).
DEFAULT_HYPER = dict(lambda_l1=0.05, lambda_tv=0.1, mu=1e-3, eps=1e-3, eps_tv=1e-3)

# Batched workload: 6 volumes each of 96^3, 128^3, 192^3, 256^3 with their own
# seeds; blob count and ball radius scale with the edge like the single-volume
# workloads (1600 blobs in radius 100 at 256^3).
BATCH_EDGES = [96] * 6 + [128] * 6 + [192] * 6 + [256] * 6


@dataclass
class Volume:
    b: np.ndarray        # float32 [nz][ny][nx]
    w: np.ndarray        # float32 [nz][ny][nx], strictly positive
    phantom: np.ndarray  # float32 [nz][ny][nx]


def _phantom(shape, centres, sigmas, amps):
    nz, ny, nx = shape
    vol = np.zeros(shape, dtype=np.float64)
    for (cz, cy, cx), s, a in zip(centres, sigmas, amps):
        r = 5.0 * s
        z0, z1 = max(0, int(np.ceil(cz - r))), min(nz - 1, int(np.floor(cz + r)))
        y0, y1 = max(0, int(np.ceil(cy - r))), min(ny - 1, int(np.floor(cy + r)))
        x0, x1 = max(0, int(np.ceil(cx - r))), min(nx - 1, int(np.floor(cx + r)))
        if z0 > z1 or y0 > y1 or x0 > x1:
            continue
        dz = (np.arange(z0, z1 + 1) - cz)[:, None, None]
        dy = (np.arange(y0, y1 + 1) - cy)[None, :, None]
        dx = (np.arange(x0, x1 + 1) - cx)[None, None, :]
        d2 = dz * dz + dy * dy + dx * dx
        blob = a * np.exp(-d2 / (2.0 * s * s))
        blob[d2 > r * r] = 0.0
        vol[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] += blob
    return vol


def _smooth_field(noise, sigma):
    """Periodic Gaussian smoothing through the FFT, then unit variance."""
    try:
        import scipy.fft as sfft
        fwd, inv = (lambda a: sfft.rfftn(a, workers=-1)), (lambda a, s: sfft.irfftn(a, s=s, workers=-1))
    except ImportError:  # pragma: no cover - numpy fallback keeps the generator usable
        fwd, inv = np.fft.rfftn, (lambda a, s: np.fft.irfftn(a, s=s))
    shape = noise.shape
    f = fwd(noise)
    kz = np.fft.fftfreq(shape[0])[:, None, None]
    ky = np.fft.fftfreq(shape[1])[None, :, None]
    kx = np.fft.rfftfreq(shape[2])[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    f *= np.exp(-2.0 * (np.pi ** 2) * (sigma ** 2) * k2)
    g = inv(f, shape)
    g -= g.mean()
    g /= g.std()
    return g


def make_volume(shape, blobs, radius, seed, noise_sd=0.3, field_sigma=4.0):
    """Render one seeded (b, w, phantom) triple of the given [nz, ny, nx] shape."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed)
    centre = np.array([(s - 1) / 2.0 for s in shape])
    dirs = rng.standard_normal((blobs, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = radius * rng.random(blobs) ** (1.0 / 3.0)
    centres = centre[None, :] + dirs * rad[:, None]
    sigmas = rng.uniform(1.5, 3.0, blobs)
    amps = rng.uniform(0.5, 1.0, blobs)
    field_noise = rng.standard_normal(shape)
    data_noise = rng.standard_normal(shape)
    phantom = _phantom(shape, centres, sigmas, amps)
    g = _smooth_field(field_noise, field_sigma)
    w = np.exp(0.5 * g)
    b = phantom + noise_sd * data_noise / np.sqrt(w)
    return Volume(b=b.astype(np.float32), w=w.astype(np.float32),
                  phantom=phantom.astype(np.float32))


def workload(name):
    """(Volume, hyper-parameters, rounds, iterations) of a named workload."""
    spec = WORKLOADS[name]
    n = spec["n"]
    vol = make_volume((n, n, n), spec["blobs"], spec["radius"], spec["seed"])
    return vol, dict(DEFAULT_HYPER), spec["rounds"], spec["iters"]


def batch_workload(first_seed=2000):
    """The 24-volume batch: list of (Volume, hyper-parameters)."""
    out = []
    rng = np.random.default_rng(first_seed - 1)
    lam_tv = rng.uniform(0.05, 0.2, len(BATCH_EDGES))
    for j, n in enumerate(BATCH_EDGES):
        scale = n / 256.0
        blobs = max(1, int(round(1600 * scale ** 3)))
        vol = make_volume((n, n, n), blobs, 100.0 * scale, first_seed + j)
        hyper = dict(DEFAULT_HYPER)
        hyper["lambda_tv"] = float(lam_tv[j])
        out.append((vol, hyper))
    return out


def random_volume(shape, seed, positive=False, scale=1.0):
    """Plain seeded random field, used for operator identities and odd shapes."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) * scale
    if positive:
        a = np.exp(0.5 * a)
    return a


def make_half_maps(shape, blobs, radius, seed, noise_sd=0.3, field_sigma=4.0):
    """Two data volumes of the same phantom and weight with independent noise,
    the synthetic stand-in for the gold-standard half-map split (Sec. 2.3):
    (Volume, Volume), the second drawing its data noise from seed + 500000."""
    v1 = make_volume(shape, blobs, radius, seed, noise_sd, field_sigma)
    rng = np.random.default_rng(seed + 500000)
    noise = rng.standard_normal(tuple(int(s) for s in shape))
    b2 = v1.phantom.astype(np.float64) + noise_sd * noise / np.sqrt(v1.w.astype(np.float64))
    v2 = Volume(b=b2.astype(np.float32), w=v1.w.copy(), phantom=v1.phantom.copy())
    return v1, v2


@dataclass
class FourierVolume:
    y: np.ndarray        # complex128 full spectrum [nz][ny][nx], Hermitian
    N: np.ndarray        # float64 full spectrum, positive, N(-k) = N(k)
    phantom: np.ndarray  # float32 [nz][ny][nx]


def fourier_weight(shape, scale=4.0, falloff=0.15, floor=0.05):
    """A positive, centro-symmetric N(k) that falls off with resolution and
    favours directions near the z axis (uneven angular coverage, Sec. 1)."""
    kz = np.fft.fftfreq(shape[0])[:, None, None]
    ky = np.fft.fftfreq(shape[1])[None, :, None]
    kx = np.fft.fftfreq(shape[2])[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    cos_z = np.abs(kz) / np.sqrt(np.where(k2 > 0, k2, 1.0))
    return scale * np.exp(-k2 / (2 * falloff ** 2)) * (0.25 + 0.75 * cos_z) + floor


def make_fourier_volume(shape, blobs, radius, seed, noise_sd=0.3):
    """Fourier-space data of Eq. 31: y = sqrt(N) A(phantom) + noise_sd A(e),
    A the unitary DFT and e real white noise, so y is Hermitian."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed)
    centre = np.array([(s - 1) / 2.0 for s in shape])
    dirs = rng.standard_normal((blobs, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = radius * rng.random(blobs) ** (1.0 / 3.0)
    centres = centre[None, :] + dirs * rad[:, None]
    sigmas = rng.uniform(1.5, 3.0, blobs)
    amps = rng.uniform(0.5, 1.0, blobs)
    noise = rng.standard_normal(shape)
    phantom = _phantom(shape, centres, sigmas, amps)
    N = fourier_weight(shape)
    y = np.sqrt(N) * np.fft.fftn(phantom, norm="ortho") + noise_sd * np.fft.fftn(noise, norm="ortho")
    return FourierVolume(y=y, N=N, phantom=phantom.astype(np.float32))


def half_spectrum(a):
    """The real-to-complex half of a full spectrum (last axis 0 .. nx/2)."""
    return np.ascontiguousarray(a[..., : a.shape[-1] // 2 + 1])


@dataclass
class ProjectionData:
    rot: np.ndarray      # float64 [m][3][3]; column 0 and 1 map the image axes (kx, ky) to 3-D (x, y, z)
    X: np.ndarray        # complex128 [m][n][n] image spectra [ky][kx], fftfreq order, Hermitian per image
    ctf: np.ndarray      # float64 [m][n][n] contrast transfer functions (real, centro-symmetric)
    phantom: np.ndarray  # float32 [n][n][n]


def random_rotations(m, rng):
    """m uniformly distributed rotations (unit quaternions)."""
    q = rng.standard_normal((m, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def make_projection_data(n, blobs, radius, n_images, seed, noise_sd=1.0):
    """Spectra of n x n projection images of a Gaussian-blob phantom (n even):
    by the projection-slice relation (Sec. 2, Eq. 1 and Eq. 24) image i
    samples the phantom's 3-D transform on the central plane R_i (kx, ky, 0);
    the blobs' transform is analytic, so the samples are exact at off-grid
    positions. Transforms take the real-space origin at the box centre
    (voxel n/2 on every axis), as cryo-EM images do, so they vary smoothly
    between grid points. Each image is multiplied by its own CTF (a
    defocus-like oscillation) and receives the 2-D transform of real white
    noise."""
    assert n % 2 == 0, "projection data need an even box"
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    centre = np.array([(n - 1) / 2.0] * 3)
    dirs = rng.standard_normal((blobs, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = radius * rng.random(blobs) ** (1.0 / 3.0)
    centres = centre[None, :] + dirs * rad[:, None]   # (z, y, x) voxel coordinates
    sigmas = rng.uniform(1.5, 3.0, blobs)
    amps = rng.uniform(0.5, 1.0, blobs)
    phantom = _phantom(shape, centres, sigmas, amps)
    rot = random_rotations(n_images, rng)
    defocus = rng.uniform(0.5, 1.5, n_images)
    f = np.fft.fftfreq(n) * n
    KY, KX = np.meshgrid(f, f, indexing="ij")
    cxyz = centres[:, ::-1] - n / 2.0                  # (x, y, z) about the box centre
    X = np.empty((n_images, n, n), dtype=np.complex128)
    ctf = np.empty((n_images, n, n))
    s2 = (KX * KX + KY * KY) / (n * n)
    for i in range(n_images):
        q = rot[i][:, 0][None, None, :] * KX[..., None] + rot[i][:, 1][None, None, :] * KY[..., None]
        qq = (q * q).sum(-1) / (n * n)
        phase = np.einsum("abk,ck->abc", q, cxyz) / n  # [ky][kx][blob]
        amp = amps * (2 * np.pi * sigmas ** 2) ** 1.5
        F = (amp[None, None, :] * np.exp(-2 * np.pi ** 2 * sigmas[None, None, :] ** 2 * qq[..., None])
             * np.exp(-2j * np.pi * phase)).sum(-1)
        ctf[i] = np.sin(0.5 + 30.0 * defocus[i] * s2)
        X[i] = ctf[i] * F + noise_sd * np.fft.fft2(rng.standard_normal((n, n)))
    return ProjectionData(rot=rot, X=X, ctf=ctf, phantom=phantom.astype(np.float32))
