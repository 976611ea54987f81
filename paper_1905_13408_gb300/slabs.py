"""z-slab decomposition of one volume over several solver contexts.

The fused step of a plane z reads the planes z - 1 and z + 1 (the backward
differences of Eq. 12 and the divergence of Eq. 17), so a volume cut into
slabs of consecutive planes needs, per slab, one halo plane on each side
that faces another slab. This module holds the bookkeeping of that cut
(which planes each slab owns, which planes go where after every iteration,
how the per-slab sums combine) as plain functions, and `SlabSolver`, which
drives one context per slab on the current GPU: the halo planes travel by
device copies and the sums are combined on the host, where a run over
several GPUs would use send/receive and an all-reduce. The contexts mark
their halo planes (spg_set_halo), so each one's objective history and
re-weighting statistics cover its own planes only; after each re-weighting
all slabs take one step size from the maxima over all slabs
(spg_step_bound / spg_set_step_bound). The slabs together then compute
bitwise the iterates of one context holding the whole volume.

No counterpart in the paper, whose solver runs on one GPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Slab:
    begin: int      # first plane the slab owns (global index)
    end: int        # one past its last plane
    lo: int         # 1 if the slab holds the plane below `begin` as a halo
    hi: int         # 1 if it holds the plane at `end` as a halo

    @property
    def ext_begin(self):
        return self.begin - self.lo

    @property
    def ext_end(self):
        return self.end + self.hi

    @property
    def ext_nz(self):
        return self.ext_end - self.ext_begin


def slab_ranges(nz, nslabs):
    """Cut planes [0, nz) into `nslabs` slabs of consecutive planes, sizes
    differing by at most one, each with a halo plane on every side that
    faces another slab."""
    if not 1 <= nslabs <= nz:
        raise ValueError("need 1 <= nslabs <= nz")
    bounds = [nz * i // nslabs for i in range(nslabs + 1)]
    return [Slab(bounds[i], bounds[i + 1], 1 if i > 0 else 0, 1 if i < nslabs - 1 else 0) for i in range(nslabs)]


def halo_exchanges(slabs):
    """Plane copies that refresh every halo after an iteration:
    (source slab, source local plane, destination slab, destination local
    plane). Sources are owned planes and destinations halo planes, so the
    copies may run in any order."""
    out = []
    for i in range(len(slabs) - 1):
        a, b = slabs[i], slabs[i + 1]
        out.append((i, a.end - 1 - a.ext_begin, i + 1, 0))                        # a's top plane -> b's lower halo
        out.append((i + 1, b.begin - b.ext_begin, i, a.ext_end - 1 - a.ext_begin))  # b's bottom plane -> a's upper halo
    return out


def common_step_bound(bounds):
    """The maxima (max w, max omtv) over all slabs from each slab's own."""
    bounds = np.asarray(bounds, dtype=np.float64)
    return float(bounds[:, 0].max()), float(bounds[:, 1].max())


def combine_histories(histories):
    """One objective history from the slabs' own: the same step counter, the
    data, l1, TV and total columns summed."""
    n = min(len(h) for h in histories)
    hs = [np.asarray(h[-n:], dtype=np.float64) for h in histories]
    for h in hs[1:]:
        if not np.array_equal(h[:, 0], hs[0][:, 0]):
            raise ValueError("slab histories are not aligned")
    out = hs[0].copy()
    for h in hs[1:]:
        out[:, 1:] += h[:, 1:]
    return out


def extended(a, slab):
    """The planes of a [nz][ny][nx] array that a slab's context holds."""
    return a[slab.ext_begin:slab.ext_end]


class SlabSolver:
    """One [nz][ny][nx] volume solved by `nslabs` contexts on the current GPU
    (one per slab), with the halo exchange after every iteration."""

    def __init__(self, shape, hyper, nslabs, **ctx_kw):
        from . import spg
        self.shape = tuple(shape)
        self.slabs = slab_ranges(self.shape[0], nslabs)
        self.plan = halo_exchanges(self.slabs)
        self.ctxs = []
        for sl in self.slabs:
            c = spg.SPG(dict(shape=(sl.ext_nz,) + self.shape[1:], **hyper), **ctx_kw)
            c.set_halo(0, sl.lo, sl.hi)
            self.ctxs.append(c)

    def set_data(self, b, w):
        import torch
        for sl, c in zip(self.slabs, self.ctxs):
            c.set_data(0, *(torch.as_tensor(np.ascontiguousarray(extended(np.asarray(a), sl)), device="cuda")
                            for a in (b, w)))

    def exchange(self):
        for src, sz, dst, dz in self.plan:
            x, p = self.ctxs[src].get_planes(0, sz, 1)
            self.ctxs[dst].set_planes(0, dz, x, p)

    def reweight(self):
        for c in self.ctxs:
            c.reweight()
        mw, mo = common_step_bound([c.step_bound(0) for c in self.ctxs])
        for c in self.ctxs:
            c.set_step_bound(0, mw, mo)

    def iterate(self, k):
        for _ in range(k):
            for c in self.ctxs:
                c.iterate(1)
            self.exchange()

    def solve(self, rounds, iters):
        for _ in range(rounds):
            self.reweight()
            self.iterate(iters)

    def history(self):
        return combine_histories([c.history(0) for c in self.ctxs])

    def round_stats(self):
        return [c.round_stats(0) for c in self.ctxs]

    def get_x(self):
        parts = []
        for sl, c in zip(self.slabs, self.ctxs):
            x = c.get_x(0).cpu().numpy()
            parts.append(x[sl.lo:sl.lo + (sl.end - sl.begin)])
        return np.concatenate(parts, axis=0)

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []
