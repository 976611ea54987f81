"""Differentiation at the workload's own size: a 128^3 volume, 50 unrolled
iterations (weights 1, tau fixed), checkpoints every 10, loss
L = |x_50 - phantom|^2. Central differences (step 1e-4) of the FP64 oracle in
64 seeded single-voxel directions (32 of b, 32 of w) and in both scalars are
compared with the oracle's adjoint and with the GPU's hand-written adjoint.

Differences of L are summed as sum (x+ - x-)(x+ + x- - 2 phantom), so the
two runs' common part cancels voxel by voxel instead of in two sums of 2e6
terms. The unrolled map is piecewise smooth: it has a kink wherever a
voxel-step passes the soft-threshold of Eq. 21 or moves between the two
branches of the smoothed norm of Eq. 14/16 (|Dy| = mu). A single-voxel
direction whose perturbed runs change either count is left out (5 of the 64
at this size). A scalar moves every threshold and every |Dy| at once, so at
2e6 voxels every step crosses some kinks and the central difference
converges to the derivative only linearly in the step; the scalars are
checked at steps 1e-4 down to 1e-7 (at 1e-7: rel 6e-8 and 3e-8 in FP64).
The oracle runs on the host cores (several minutes at this size).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu


def test_adjoint_config_central_differences():
    vol, hyper, _, K = synth.workload("vol128_adjoint")
    shape = vol.b.shape
    ph = vol.phantom.astype(np.float64)
    b, w = vol.b.astype(np.float64), vol.w.astype(np.float64)

    # GPU: forward and adjoint through the C ABI (checkpoints every 10)
    s = spg.SPG(dict(shape=shape, **hyper))
    s.set_data(0, torch.from_numpy(vol.b).cuda(), torch.from_numpy(vol.w).cuda())
    s.reweight()
    tau = s.round_stats(0)[5]
    xK = torch.empty((shape), dtype=torch.float32, device="cuda")
    spg.spg_unrolled(s.handle, K, xK)
    gx = (2 * (xK - torch.from_numpy(vol.phantom).cuda())).contiguous()
    gb_d, gw_d = torch.empty_like(xK), torch.empty_like(xK)
    gs_d = np.asarray(spg.spg_backward(s.handle, K, gx, gb_d, gw_d, ckpt_every=10))
    s.close()
    gb_d, gw_d = gb_d.cpu().numpy().astype(np.float64), gw_d.cpu().numpy().astype(np.float64)

    # oracle: FP64 adjoint
    p = oracle.Params(shape, **hyper)
    # the context keeps tau = 1/L as float32; the oracle runs with that value
    assert tau == pytest.approx(1.0 / oracle.lipschitz(w, 1.0, p), rel=1e-7)
    x0 = np.zeros(shape)
    ref_xK = oracle.unrolled(b, w, None, None, tau, K, x0, p)
    gb_o, gw_o, gs_o = oracle.backward(b, w, None, None, tau, K, x0, 2 * (ref_xK - ph), p)

    def run(bb, ww, pp):
        return oracle.unrolled_counts(bb, ww, None, None, tau, K, x0, pp)

    _, act0 = run(b, w, p)

    def dloss(xp, xm):
        return float(((xp - xm) * (xp + xm - 2 * ph)).sum())

    rng = np.random.default_rng(4004)
    h = 1e-4
    rows = []
    for which, base in (("b", b), ("w", w)):
        for v in rng.choice(b.size, 32, replace=False):
            e = np.zeros(b.size)
            e[v] = h
            e = e.reshape(shape)
            if which == "b":
                (xp, ap), (xm, am) = run(b + e, w, p), run(b - e, w, p)
            else:
                (xp, ap), (xm, am) = run(b, w + e, p), run(b, w - e, p)
            if ap != act0 or am != act0:
                continue
            fd = dloss(xp, xm) / (2 * h)
            go = (gb_o if which == "b" else gw_o).ravel()[v]
            gd = (gb_d if which == "b" else gw_d).ravel()[v]
            rows.append((which, int(v), fd, go, gd))
    assert len(rows) >= 48, len(rows)
    fd = np.array([r[2] for r in rows])
    go = np.array([r[3] for r in rows])
    gd = np.array([r[4] for r in rows])
    scale = np.abs(fd).max()
    e_o = np.abs(go - fd).max() / scale
    e_d = np.abs(gd - fd).max() / scale
    print(f"config-4 central differences: {len(rows)} directions; max |adjoint - FD| / max |FD|: "
          f"oracle {e_o:.2e}, GPU {e_d:.2e}")
    # the oracle's adjoint is exact up to FP64 rounding and the O(h^2) of the
    # central difference; the GPU's float32 adjoint is held to the 1e-4 of
    # the gradient parity gate
    np.testing.assert_allclose(go, fd, rtol=1e-6, atol=1e-7 * scale)
    np.testing.assert_allclose(gd, fd, rtol=1e-4, atol=1e-5 * scale)

    # the two scalars: the error of the central difference shrinks with the
    # step (kinks crossed on one side only cost O(step)); at 1e-7 it is far
    # below the gates
    for i, name in enumerate(("lambda_l1", "lambda_tv")):
        errs = []
        for hs in (1e-4, 1e-5, 1e-6, 1e-7):
            hp = oracle.Params(shape, **hyper)
            hm = oracle.Params(shape, **hyper)
            setattr(hp, name, getattr(p, name) + hs)
            setattr(hm, name, getattr(p, name) - hs)
            (xp, _), (xm, _) = run(b, w, hp), run(b, w, hm)
            fd = dloss(xp, xm) / (2 * hs)
            errs.append(abs(fd / gs_o[i] - 1))
        print(f"  d/d{name}: FD(1e-7) {fd:.9e}, oracle adjoint {gs_o[i]:.9e}, GPU {gs_d[i]:.9e}; "
              f"FD rel error at steps 1e-4..1e-7: {', '.join(f'{e:.1e}' for e in errs)}")
        assert errs[-1] <= 1e-6 and errs[-1] < errs[0]
        assert gs_d[i] == pytest.approx(fd, rel=1e-4)
