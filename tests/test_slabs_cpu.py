"""Bookkeeping of the z-slab decomposition (paper_1905_13408_gb300/slabs.py)
on CPU: the cut, the halo exchange plan, and the exchange plus the
all-reduce of the objective between gloo ranks (world sizes 2 and 3), each
rank holding its slab of one volume. No GPU is involved."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1905_13408_gb300 import slabs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("nz,n", [(2, 2), (7, 2), (7, 3), (40, 3), (41, 4), (5, 5), (9, 1)])
def test_slab_ranges_partition_the_planes(nz, n):
    sl = slabs.slab_ranges(nz, n)
    assert len(sl) == n and sl[0].begin == 0 and sl[-1].end == nz
    for a, b in zip(sl, sl[1:]):
        assert a.end == b.begin and a.hi == 1 and b.lo == 1
    assert sl[0].lo == 0 and sl[-1].hi == 0
    sizes = [s.end - s.begin for s in sl]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    for s in sl:
        assert 0 <= s.ext_begin < s.ext_end <= nz and s.ext_nz == s.end - s.begin + s.lo + s.hi


@pytest.mark.parametrize("nz,n", [(7, 2), (40, 3), (41, 4), (5, 5)])
def test_halo_exchanges_copy_owned_planes_onto_halos(nz, n):
    sl = slabs.slab_ranges(nz, n)
    plan = slabs.halo_exchanges(sl)
    assert len(plan) == 2 * (n - 1)
    halos = set()
    for src, sz, dst, dz in plan:
        g_src, g_dst = sl[src].ext_begin + sz, sl[dst].ext_begin + dz
        assert g_src == g_dst                                   # the same global plane
        assert sl[src].begin <= g_src < sl[src].end             # owned by the source
        assert not (sl[dst].begin <= g_dst < sl[dst].end)       # a halo of the destination
        assert abs(src - dst) == 1
        halos.add((dst, dz))
    expect = {(i, 0) for i, s in enumerate(sl) if s.lo} | {(i, s.ext_nz - 1) for i, s in enumerate(sl) if s.hi}
    assert halos == expect


def test_combine_histories_sums_the_slabs():
    h1 = np.array([[3, 1.0, 2.0, 3.0, 6.0], [4, 0.5, 1.0, 1.5, 3.0]])
    h2 = np.array([[3, 10.0, 20.0, 30.0, 60.0], [4, 5.0, 10.0, 15.0, 30.0]])
    np.testing.assert_array_equal(slabs.combine_histories([h1, h2]),
                                  [[3, 11, 22, 33, 66], [4, 5.5, 11, 16.5, 33]])
    with pytest.raises(ValueError):
        slabs.combine_histories([h1, h2[::-1]])
    assert slabs.common_step_bound([(2.0, 0.5), (3.0, 0.25)]) == (3.0, 0.5)


def slab_objective(x, b, w, om1, omtv, lam1, lamtv, mu, sl):
    """(data, l1, tv) over the planes a slab owns, from its extended arrays;
    the z-difference of its first plane reads the halo below (none for the
    first slab: the volume's edge, Eq. 12)."""
    own = slice(sl.lo, sl.lo + sl.end - sl.begin)
    d = np.zeros((3,) + x.shape)
    d[0][:, :, 1:] = x[:, :, 1:] - x[:, :, :-1]
    d[1][:, 1:, :] = x[:, 1:, :] - x[:, :-1, :]
    d[2][1:] = x[1:] - x[:-1]
    s = np.sqrt((d * d).sum(axis=0))
    h = np.where(s <= mu, s * s / (2 * mu), s - mu / 2)
    return (0.5 * (w[own] * (x[own] - b[own]) ** 2).sum(), lam1 * (om1[own] * np.abs(x[own])).sum(),
            lamtv * (omtv[own] * h[own]).sum())


def full_volume(shape):
    rng = np.random.default_rng(77)
    x = rng.standard_normal(shape) * 10 ** rng.uniform(-3.5, 0, shape)
    return (x, rng.standard_normal(shape), rng.uniform(0.3, 3, shape), rng.uniform(0.05, 1, shape),
            rng.uniform(0.05, 1, shape))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, shape, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1905_13408_gb300 import slabs as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sl = S.slab_ranges(shape[0], world)
        me = sl[rank]
        full = full_volume(shape)
        ext = [np.ascontiguousarray(S.extended(a, me)) for a in full]
        x = ext[0]
        if me.lo:
            x[0] = np.nan          # the halos start stale: the exchange must fill them
        if me.hi:
            x[-1] = np.nan
        reqs, recv = [], []
        for src, sz, dst, dz in S.halo_exchanges(sl):
            if src == rank:
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(x[sz])), dst))
            if dst == rank:
                buf = torch.empty(shape[1:], dtype=torch.float64)
                reqs.append(dist.irecv(buf, src))
                recv.append((dz, buf))
        for r in reqs:
            r.wait()
        for dz, buf in recv:
            x[dz] = buf.numpy()
        halos_ok = bool(np.array_equal(x, S.extended(full[0], me)))
        parts = torch.tensor(slab_objective(x, *ext[1:], 0.07, 0.13, 1e-3, me), dtype=torch.float64)
        dist.all_reduce(parts)
        q.put((rank, halos_ok, parts.numpy().tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_halo_exchange_and_objective_allreduce(world):
    """Ranks exchange halo planes by send/receive as the plan says, then
    all-reduce the per-slab objective sums: every halo holds its neighbour's
    plane, and the reduced sums equal the oracle's objective of the whole
    volume."""
    import oracle
    oracle.build()
    shape = (11, 6, 7)
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shape, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    x, b, w, om1, omtv = full_volume(shape)
    want = oracle.objective(x, b, w, om1, omtv, oracle.Params(shape, lambda_l1=0.07, lambda_tv=0.13, mu=1e-3))
    for rank, halos_ok, parts in out:
        assert halos_ok, rank
        np.testing.assert_allclose(parts, want[:3], rtol=1e-12)
