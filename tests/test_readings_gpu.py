"""Alternative readings of the paper on the GPU against the FP64 oracle run
with the same readings: forward differences alone on the fused path (over
volumes with every axis reversed), the other combinations on the plain
one-kernel step."""
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
        spg.SPG(dict(shape=shape, **HYPER), restart=True, difference="forward", tv_weight="post_div")
    vol = synth.make_volume(shape, blobs=2, radius=2, seed=43)
    s = spg.SPG(dict(shape=shape, **HYPER), tv_weight="post_div")
    s.set_data(0, torch.from_numpy(vol.b).cuda(), torch.from_numpy(vol.w).cuda())
    s.reweight()
    s.iterate(2)
    with pytest.raises(spg.SPGError):
        s.certificate(0)
    s.close()


FWD = dict(difference="forward", boundary="neumann", tv_weight="inside")


def reverse(a):
    return np.ascontiguousarray(np.asarray(a)[..., ::-1, ::-1, ::-1])


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("data_dtype,restart,storage", [("f32", False, "delta"), ("bf16", False, "delta"),
                                                        ("f32", True, "prev"), ("bf16", True, "delta")])
def test_forward_differences_on_the_fused_path(data_dtype, restart, storage):
    """Forward differences with a Neumann edge run the fused kernels on the
    axis-reversed volume (D_f = -R D_b R): with BF16 data, gradient restart
    and both iterate storages, which the plain path does not offer, the
    solve matches the oracle's forward-difference solve to the FP32 gate.
    An odd voxel count leaves a middle voxel that the reversal keeps."""
    shape = (19, 27, 45)
    vol = synth.make_volume(shape, blobs=12, radius=6, seed=45)
    hyper = dict(HYPER, mu=0.05) if restart else HYPER
    s = spg.SPG(dict(shape=shape, **hyper), data_dtype=data_dtype, restart=restart, storage=storage, **FWD)
    s.set_data(0, torch.from_numpy(vol.b).cuda(), torch.from_numpy(vol.w).cuda())
    stats = []
    for _ in range(2):
        s.reweight()
        stats.append(s.round_stats(0))
        s.iterate(120 if restart else 40)
    x = s.get_x(0).cpu().numpy()
    hist = s.history(0)
    s.close()
    b, w = (bf16_round(vol.b), bf16_round(vol.w)) if data_dtype == "bf16" else (vol.b, vol.w)
    p = oracle.Params(shape, restart=restart, **hyper, **FWD)
    ref = oracle.solve(b, w, p, 2, 120 if restart else 40)
    err = rel_l2(x, ref.x)
    print(f"forward on the fused path {data_dtype} restart={restart} {storage}: rel-L2 {err:.2e}")
    assert err <= 1e-5
    np.testing.assert_allclose(hist[:, 4], ref.hist.reshape(-1, 4)[:, 3], rtol=1e-6)
    np.testing.assert_allclose(np.array(stats)[:, :4], ref.rstats[:, :4], rtol=1e-6)
    if restart:
        plain = oracle.solve(b, w, oracle.Params(shape, **hyper, **FWD), 2, 120, with_hist=False)
        assert rel_l2(plain.x, ref.x) > 1e-4  # the restarts did change the trajectory


def test_forward_differences_batch_autotune_and_state():
    """An uneven batch under forward differences, autotuned, run through the
    captured graph, checkpointed and resumed in a fresh context: each volume
    matches its own oracle solve, and the state blob holds the volumes in
    their own orientation."""
    shapes = [(16, 20, 24), (23, 17, 31)]
    vols = [synth.make_volume(sh, blobs=8, radius=5, seed=46 + j) for j, sh in enumerate(shapes)]
    params = [dict(shape=sh, **HYPER) for sh in shapes]
    s = spg.SPG(params, **FWD)
    for j, v in enumerate(vols):
        s.set_data(j, torch.from_numpy(v.b).cuda(), torch.from_numpy(v.w).cuda())
    s.reweight()
    s.autotune(trial_iters=4)  # restores the iterates and counters after its trials
    s.iterate(25)
    blob = s.get_state()
    s.close()
    st = spg.parse_state(blob, shapes)["volumes"]
    r = spg.SPG(params, **FWD)
    for j, v in enumerate(vols):
        r.set_data(j, torch.from_numpy(v.b).cuda(), torch.from_numpy(v.w).cuda())
    r.set_state(blob)
    r.iterate(20)
    xs = [r.get_x(j).cpu().numpy() for j in range(2)]
    r.close()
    for sh, v, x, sv in zip(shapes, vols, xs, st):
        p = oracle.Params(sh, **HYPER, **FWD)
        mid = oracle.solve(v.b, v.w, p, 1, 25, with_hist=False)
        assert rel_l2(sv["x"], mid.x) <= 1e-6
        np.testing.assert_allclose(sv["omtv"], mid.omtv, rtol=2e-6)
        ref = oracle.solve(v.b, v.w, p, 1, 45, with_hist=False)
        assert rel_l2(x, ref.x) <= 1e-6


def test_forward_differences_certificate_and_adjoint():
    """The certificate and the adjoint under forward differences: the
    certificate against the oracle's with the forward reading; the gradients
    of K unrolled steps against the oracle's adjoint of the reversed problem
    reversed back (the oracle's adjoint takes the adopted reading)."""
    shape = (12, 14, 21)
    vol = synth.make_volume(shape, blobs=6, radius=4, seed=47)
    hyper = dict(HYPER, mu=0.02)
    p = oracle.Params(shape, **hyper, **FWD)
    s = spg.SPG(dict(shape=shape, **hyper), **FWD)
    s.set_data(0, vol.b, vol.w)
    s.reweight()
    s.iterate(30)
    blob = s.get_state()
    s.iterate(1)
    cert = s.certificate(0)
    x1 = s.get_x(0).cpu().numpy()
    s.close()
    sv = spg.parse_state(blob, [shape])["volumes"][0]
    xk, xkm1, omtv = (sv[k].astype(np.float64) for k in ("x", "x_prev", "omtv"))
    beta = float(np.float32(oracle.beta_table(31)[30]))
    want = oracle.certificate(xk + beta * (xk - xkm1), x1, sv["tau"], vol.b, vol.w, omtv, p)
    np.testing.assert_allclose(cert, want, rtol=1e-3)

    K = 12
    b = torch.from_numpy(vol.b).cuda()
    w = torch.from_numpy(vol.w).cuda()
    s = spg.SPG(dict(shape=shape, **hyper), **FWD)
    s.set_data(0, b, w)
    s.reweight()
    tau = s.round_stats(0)[5]
    xK = torch.empty_like(b)
    spg.spg_unrolled(s.handle, K, xK)
    gx = 2 * (xK - torch.from_numpy(vol.phantom).cuda())
    gb = torch.empty_like(b)
    gw = torch.empty_like(b)
    gs = spg.spg_backward(s.handle, K, gx.contiguous(), gb, gw, ckpt_every=5)
    s.close()
    x0 = np.zeros(shape)
    ref_xK = oracle.unrolled(vol.b, vol.w, None, None, tau, K, x0, p)
    assert rel_l2(xK.cpu().numpy(), ref_xK) <= 1e-6
    gK = 2 * (ref_xK - vol.phantom)
    pb = oracle.Params(shape, **hyper)
    rb, rw, rs = oracle.backward(reverse(vol.b), reverse(vol.w), None, None, tau, K, x0, reverse(gK), pb)
    assert rel_l2(gb.cpu().numpy(), reverse(rb)) <= 1e-4
    assert rel_l2(gw.cpu().numpy(), reverse(rw)) <= 1e-4
    np.testing.assert_allclose(gs, rs, rtol=1e-4)
