"""Alternative readings of the paper on the GPU (the plain two-pass path)
against the FP64 oracle run with the same readings."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu

HYPER = dict(synth.DEFAULT_HYPER, mu=0.02)
CASES = [("forward", "neumann", "inside"), ("backward", "periodic", "inside"), ("backward", "neumann", "post_div"),
         ("forward", "periodic", "post_div")]


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("storage", ["delta", "prev"])
@pytest.mark.parametrize("difference,boundary,tv_weight", CASES)
def test_readings_match_oracle(difference, boundary, tv_weight, storage):
    shape = (19, 26, 37)
    vol = synth.make_volume(shape, blobs=12, radius=6, seed=41)
    rd = dict(difference=difference, boundary=boundary, tv_weight=tv_weight)
    s = spg.SPG(dict(shape=shape, **HYPER), storage=storage, **rd)
    s.set_data(0, torch.from_numpy(vol.b).cuda(), torch.from_numpy(vol.w).cuda())
    stats = []
    for _ in range(2):
        s.reweight()
        stats.append(s.round_stats(0))
        s.iterate(30)
    x = s.get_x(0).cpu().numpy()
    hist = s.history(0)
    obj = s.objective(0)
    s.close()
    ref = oracle.solve(vol.b, vol.w, oracle.Params(shape, **HYPER, **rd), 2, 30)
    err = rel_l2(x, ref.x)
    print(f"{rd} {storage}: rel-L2 {err:.2e}")
    assert err <= 1e-6
    np.testing.assert_allclose(hist[:, 4], ref.hist.reshape(-1, 4)[:, 3], rtol=1e-6)
    np.testing.assert_allclose(np.array(stats)[:, :4], ref.rstats[:, :4], rtol=1e-6)
    p = oracle.Params(shape, **HYPER, **rd)
    want = oracle.objective(x.astype(np.float64), vol.b, vol.w, ref.om1, ref.omtv, p)
    np.testing.assert_allclose(obj[3], want[3], rtol=2e-6)


def test_readings_batch_and_graph():
    """A batch of two volumes under periodic forward differences, run long
    enough for the captured graph: each volume matches its own oracle solve."""
    shapes = [(16, 20, 24), (24, 16, 20)]
    vols = [synth.make_volume(sh, blobs=8, radius=5, seed=42 + j) for j, sh in enumerate(shapes)]
    rd = dict(difference="forward", boundary="periodic", tv_weight="inside")
    s = spg.SPG([dict(shape=sh, **HYPER) for sh in shapes], **rd)
    for j, v in enumerate(vols):
        s.set_data(j, torch.from_numpy(v.b).cuda(), torch.from_numpy(v.w).cuda())
    s.reweight()
    s.iterate(45)
    xs = [s.get_x(j).cpu().numpy() for j in range(2)]
    s.close()
    for sh, v, x in zip(shapes, vols, xs):
        ref = oracle.solve(v.b, v.w, oracle.Params(sh, **HYPER, **rd), 1, 45, with_hist=False)
        assert rel_l2(x, ref.x) <= 1e-6


def test_readings_restrictions():
    shape = (8, 8, 8)
    with pytest.raises(spg.SPGError):
        spg.SPG(dict(shape=shape, **HYPER), data_dtype="bf16", boundary="periodic")
    with pytest.raises(spg.SPGError):
        spg.SPG(dict(shape=shape, **HYPER), restart=True, difference="forward")
    vol = synth.make_volume(shape, blobs=2, radius=2, seed=43)
    s = spg.SPG(dict(shape=shape, **HYPER), tv_weight="post_div")
    s.set_data(0, torch.from_numpy(vol.b).cuda(), torch.from_numpy(vol.w).cuda())
    s.reweight()
    s.iterate(2)
    with pytest.raises(spg.SPGError):
        s.certificate(0)
    s.close()
