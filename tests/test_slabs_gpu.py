"""z-slab decomposition on one GPU: one volume cut into 2 or 3 slabs, one
context per slab, halo planes exchanged by device copies after every
iteration and one step size agreed after every re-weighting (the pattern of
a run over several GPUs, each holding one slab). The iterates are bitwise
those of one context holding the whole volume, and match the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_13408_gb300 import slabs, spg, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nslabs,storage", [(2, "delta"), (3, "delta"), (2, "prev")])
def test_slabs_equal_whole_volume(nslabs, storage):
    shape = (40, 45, 70)
    vol = synth.make_volume(shape, blobs=30, radius=12, seed=91)
    hyper = dict(synth.DEFAULT_HYPER)
    rounds, iters = 2, 30
    ss = slabs.SlabSolver(shape, hyper, nslabs, storage=storage)
    ss.set_data(vol.b, vol.w)
    ss.solve(rounds, iters)
    xs, hs, st = ss.get_x(), ss.history(), ss.round_stats()
    ss.close()
    s = spg.SPG(dict(shape=shape, **hyper), storage=storage)
    s.set_data(0, torch.from_numpy(vol.b).cuda(), torch.from_numpy(vol.w).cuda())
    taus = []
    for _ in range(rounds):
        s.reweight()
        taus.append(s.round_stats(0)[5])
        s.iterate(iters)
    x1, h1 = s.get_x(0).cpu().numpy(), s.history(0)
    s.close()
    np.testing.assert_array_equal(xs, x1)
    assert all(r[5] == taus[-1] for r in st)  # every slab took the whole volume's step of the last round
    assert hs.shape == h1.shape
    np.testing.assert_array_equal(hs[:, 0], h1[:, 0])
    np.testing.assert_allclose(hs[:, 1:], h1[:, 1:], rtol=1e-8)
    ref = oracle.solve(vol.b, vol.w, oracle.Params(shape, **hyper), rounds, iters)
    err = np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x)
    print(f"{nslabs} slabs ({storage}): bitwise equal to the whole volume; oracle rel-L2 {err:.2e}")
    assert err <= 1e-5
    np.testing.assert_allclose(hs[:, 4], ref.hist.reshape(-1, 4)[:, 3], rtol=1e-6)


def test_halo_and_plane_copies_validate_arguments():
    s = spg.SPG(dict(shape=(3, 8, 8), **synth.DEFAULT_HYPER))
    with pytest.raises(spg.SPGError):
        s.set_halo(0, 1, 1 + 1)
    s.set_halo(0, 1, 1)  # one interior plane left
    with pytest.raises(spg.SPGError):
        s.set_halo(0, 2, 0)
    with pytest.raises(spg.SPGError):
        s.get_planes(0, 2, 2)  # planes 2..3 of 3
    with pytest.raises(spg.SPGError):
        s.step_bound(0)  # before spg_reweight
    s.close()
