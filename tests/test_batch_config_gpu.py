"""The batched workload at its own sizes: 24 volumes (6 each of 96^3, 128^3,
192^3, 256^3, each from its own seed, lambda_tv ~ U(0.05, 0.2)) advanced
together by one fused launch per iteration with the autotuned plan, over the
full 3 rounds x 200 iterations. The first volume of each size is compared
with its own FP64 oracle solve: the iterate to rel-L2 <= 1e-5 and every
recorded objective to rel 1e-6 (the single-volume gates). The oracle runs on
the host cores (about a minute and a half for the four volumes).
"""
import numpy as np
import pytest

import oracle
from paper_1905_13408_gb300 import spg, synth

pytestmark = pytest.mark.gpu


def test_batch24_full_schedule_against_oracle():
    vols = synth.batch_workload()
    shapes = [v.b.shape for v, _ in vols]
    s = spg.SPG([dict(shape=sh, **h) for sh, (_, h) in zip(shapes, vols)], hist_capacity=1024)
    for i, (v, _) in enumerate(vols):
        s.set_data(i, v.b, v.w)
    s.reweight()
    plan = s.autotune(10)
    assert plan["items"] >= len(vols)
    s.solve(3, 200)
    picks = [shapes.index(sh) for sh in sorted(set(shapes))]  # first volume of each size
    xs = {j: s.get_x(j).cpu().numpy() for j in picks}
    hists = {j: s.history(j) for j in picks}
    s.close()
    for j in picks:
        v, h = vols[j]
        ref = oracle.solve(v.b, v.w, oracle.Params(shapes[j], **h), 3, 200)
        err = np.linalg.norm(xs[j] - ref.x) / np.linalg.norm(ref.x)
        herr = np.abs(hists[j][:, 4] / ref.hist.reshape(-1, 4)[:, 3] - 1).max()
        print(f"batch24 volume {j} {shapes[j]} lambda_tv {h['lambda_tv']:.4f}: rel-L2 {err:.2e}, "
              f"objective history max rel {herr:.2e}; plan {plan}")
        assert err <= 1e-5
        assert len(hists[j]) == 600
        np.testing.assert_allclose(hists[j][:, 4], ref.hist.reshape(-1, 4)[:, 3], rtol=1e-6)
