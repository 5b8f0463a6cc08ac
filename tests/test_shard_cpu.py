"""Host side of the key-window split (CPU): equal-work cuts, and the gather of
the windows over a gloo process group (world size 2 and 3).

A CPU rank cannot run the library, so each rank's window is cut from the
oracle's product by key (the Kronecker code of Sec. 2, computed here from the
product's box): the test checks the orchestration (cuts, ordering, gather of
uneven and empty parts), while the GPU tests check the windows themselves.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1004_4548_gb300 import shard
from workloads import random_poly


def _codes(exps, omin, w):
    c = np.concatenate([[1], np.cumprod(w[:-1])]).astype(np.int64)
    return ((exps.astype(np.int64) - omin[:, None]) * c[:, None]).sum(axis=0)


def _product():
    f = random_poly(3, 150, [-3, 0, -2], [4, 5, 3], 41)
    g = random_poly(3, 120, [-3, 0, -2], [4, 5, 3], 42)
    r = oracle.poly_mul(f, g)
    omin = (f.exps.min(axis=1) + g.exps.min(axis=1)).astype(np.int64)
    w = (f.exps.max(axis=1) + g.exps.max(axis=1)).astype(np.int64) - omin + 1
    keys = _codes(r.exps, omin, w)
    return r, keys, int(np.prod(w))


def test_cuts_from_hist():
    cuts = shard.cuts_from_hist(np.ones(1000), 10_000, 4)
    assert cuts == [0, 2500, 5000, 7500, 10_000]
    h = np.zeros(64)
    h[10] = 5.0
    cuts = shard.cuts_from_hist(h, 6400, 3)
    assert cuts[0] == 0 and cuts[-1] == 6400 and cuts == sorted(cuts)
    assert all(c == 1100 for c in cuts[1:-1])   # all the work in one slice: the other windows are empty
    cuts = shard.cuts_from_hist(np.zeros(16), 100, 4)
    assert cuts == [0, 25, 50, 75, 100]
    rng = np.random.default_rng(3)
    h = rng.integers(0, 50, 4096).astype(np.float64)
    cuts = shard.cuts_from_hist(h, 1 << 40, 8)
    mass = [h[(c0 * 4096) >> 40:(c1 * 4096) >> 40].sum() for c0, c1 in zip(cuts, cuts[1:])]
    assert max(mass) <= h.sum() / 8 + h.max() + 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, forced_cuts, q):
    import torch
    import torch.distributed as dist
    os.environ["GLOO_SOCKET_IFNAME"] = os.environ.get("GLOO_SOCKET_IFNAME", "lo")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        r, keys, krange = _product()
        if forced_cuts is None:
            nb = 256
            hist = np.bincount((keys * nb) // krange, minlength=nb)
            cuts = shard.cuts_from_hist(hist, krange, world)
        else:
            cuts = forced_cuts
        sel = (keys >= cuts[rank]) & (keys < cuts[rank + 1])
        part = (torch.from_numpy(np.ascontiguousarray(r.exps[:, sel])),
                torch.from_numpy(np.ascontiguousarray(r.coef[sel])))
        ex, cf = shard.gather_parts(part)
        ok = np.array_equal(ex.numpy(), r.exps) and np.array_equal(cf.numpy(), r.coef)
        q.put((rank, ok, int(sel.sum()), cuts))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,forced", [(2, False), (3, False), (3, True)])
def test_gather_of_windows_over_gloo(world, forced):
    import multiprocessing as mp
    r, keys, krange = _product()
    forced_cuts = [0, int(keys[len(keys) // 3]), int(keys[len(keys) // 3]), krange] if forced else None
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, world, port, forced_cuts, q)) for k in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(ok for _, ok, _, _ in out), out
    assert sum(n for _, _, n, _ in out) == r.coef.shape[0]
    if forced:
        assert out[1][2] == 0   # the empty window contributes nothing and breaks nothing


def _mixed_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["GLOO_SOCKET_IFNAME"] = os.environ.get("GLOO_SOCKET_IFNAME", "lo")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        sizes = [5, 0, 3][:world]

        def part_of(r):
            k = sizes[r]
            base = 100 * r
            return (torch.arange(2 * k, dtype=torch.int32).reshape(2, k) + base,       # exponents
                    torch.arange(3 * k, dtype=torch.int32).reshape(3, k) - base,       # trig multipliers
                    (torch.arange(k, dtype=torch.int64) % 2).to(torch.uint8),          # kinds: odd byte counts
                    torch.arange(k, dtype=torch.float64) * 0.5 + r)                   # coefficients
        got = shard.gather_parts(part_of(rank))
        want = [torch.cat(x, dim=-1) for x in zip(*(part_of(r) for r in range(world)))]
        q.put((rank, all(torch.equal(a, b) and a.dtype == b.dtype for a, b in zip(got, want))))
    finally:
        dist.destroy_process_group()


def test_gather_of_mixed_fields_over_gloo():
    """Poisson-like parts (int32 rows, uint8 kinds, float64 coefficients; one
    rank empty): the packed gather restores every field in rank order."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_mixed_rank, args=(k, 3, port, q)) for k in range(3)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(3)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok in out), out
