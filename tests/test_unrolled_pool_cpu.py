"""Host logic of UnrolledSPG's context reuse, on CPU with a stand-in solver
(no GPU, no library calls): a backward hands its context back, the next
forward of the same shape, smoothing, epsilons, momentum, device and stream
takes it and re-sets the weights and the data on it, other keys get their
own context, at most two idle contexts are kept per key, and a second
backward of one forward is refused."""
import types

import pytest
import torch

from paper_1905_13408_gb300 import spg


class FakeSolver:
    made = []

    def __init__(self, params, momentum="fista", hist_every=1, stream=None):
        self.params = params
        self.momentum = momentum
        self.stream = stream
        self.handle = object()
        self.calls = []
        self.closed = False
        FakeSolver.made.append(self)

    def set_lambdas(self, vol, l1, tv):
        self.calls.append(("set_lambdas", vol, float(l1), float(tv)))

    def set_data(self, vol, b, w):
        self.calls.append(("set_data", vol, float(b.sum()), float(w.sum())))

    def reweight(self):
        self.calls.append(("reweight",))

    def close(self):
        self.closed = True
        self.handle = None


@pytest.fixture
def fake(monkeypatch):
    FakeSolver.made = []
    monkeypatch.setattr(spg, "SPG", FakeSolver)
    monkeypatch.setattr(spg, "_UNROLLED_POOL", {})
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: types.SimpleNamespace(cuda_stream=7))

    def unrolled(h, K, out):
        out.fill_(float(K))

    def backward(h, K, gx, gb, gw, ckpt_every=10):
        gb.copy_(gx)
        gw.copy_(-gx)
        return [1.0, 2.0]

    monkeypatch.setattr(spg, "spg_unrolled", unrolled)
    monkeypatch.setattr(spg, "spg_backward", backward)
    return FakeSolver


def _call(shape, l1, tv, mu=1e-3, seed=0):
    g = torch.Generator().manual_seed(seed)
    b = torch.rand(shape, generator=g).requires_grad_(True)
    w = torch.rand(shape, generator=g).requires_grad_(True)
    x = spg.UnrolledSPG.apply(b, w, l1, tv, 5, mu=mu)
    return b, w, x


def test_backward_hands_the_context_back_and_the_next_forward_reuses_it(fake):
    b, w, x = _call((2, 3, 4), 0.05, 0.1)
    assert len(fake.made) == 1
    first = fake.made[0]
    assert first.params["lambda_l1"] == pytest.approx(0.05) and first.params["lambda_tv"] == pytest.approx(0.1)
    assert [c[0] for c in first.calls] == ["set_data", "reweight"]
    x.sum().backward()
    assert torch.equal(b.grad, torch.ones_like(b)) and torch.equal(w.grad, -torch.ones_like(w))
    assert not first.closed
    # same key: the idle context is taken, its weights re-set before data and re-weighting
    _, _, x2 = _call((2, 3, 4), 0.07, 0.2, seed=1)
    assert len(fake.made) == 1
    assert [c[0] for c in first.calls[2:]] == ["set_lambdas", "set_data", "reweight"]
    assert first.calls[2] == ("set_lambdas", 0, pytest.approx(0.07), pytest.approx(0.2))
    x2.sum().backward()
    # another shape or another smoothing: a context of its own
    _call((2, 3, 5), 0.05, 0.1)
    _call((2, 3, 4), 0.05, 0.1, mu=2e-3)
    assert len(fake.made) == 3


def test_two_idle_contexts_kept_per_key(fake):
    outs = [_call((3, 3, 3), 0.05, 0.1, seed=i) for i in range(3)]  # three forwards in flight: three contexts
    assert len(fake.made) == 3
    for _, _, x in outs:
        x.sum().backward()
    assert [s.closed for s in fake.made] == [False, False, True]
    assert len(spg._UNROLLED_POOL[next(iter(spg._UNROLLED_POOL))]) == 2


def test_second_backward_of_one_forward_is_refused(fake):
    b, w, x = _call((2, 2, 2), 0.05, 0.1)
    loss = x.sum()
    loss.backward(retain_graph=True)
    with pytest.raises(RuntimeError, match="one backward per forward"):
        loss.backward()
