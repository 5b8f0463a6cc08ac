"""One product split by output key windows, across calls or across GPUs.

The output keys of a product (Kronecker codes, or the Poisson keys) are
ordered like its terms, and the term pairs landing in disjoint key windows
are disjoint (Sec. 4 argues this for output intervals in the multicore
setting).  So a product splits into windows [cut_r, cut_{r+1}) that are
computed independently, each by one library call with a key window in its
options, and the windows' sorted terms concatenated in window order are the
whole product.  No accumulation crosses windows: the only exchange is the
final gather.

* ``split_points``: cuts of equal work from the library's sampled work
  histogram (``kron_split_hist``), identical on every rank for the same
  inputs.
* ``mul_window``: one window of the product.
* ``gather_parts``: all-gather of the windows' terms over a
  ``torch.distributed`` process group (NCCL between GPUs; gloo on CPU).
* ``sharded_mul``: rank r of a group computes window r and (optionally)
  gathers the whole product.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def cuts_from_hist(hist, krange: int, nparts: int) -> list[int]:
    """Window boundaries 0 = c_0 <= c_1 <= ... <= c_nparts = krange splitting the
    histogram's mass (over nbins equal slices of [0, krange)) into equal parts."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    h = np.asarray(hist, dtype=np.float64)
    nb = h.shape[0]
    c = np.cumsum(h)
    total = c[-1] if nb else 0.0
    cuts = [0]
    for q in range(1, nparts):
        if total <= 0:
            cut = (q * krange) // nparts
        else:
            b = int(np.searchsorted(c, q * total / nparts, side="left"))
            cut = ((b + 1) * krange) // nb   # the end of the slice where the quantile falls
        cuts.append(min(max(cut, cuts[-1]), krange))
    cuts.append(krange)
    return cuts


def split_points(f, g, nparts: int, ctx=None, nbins: int = 65536, nsamples: int = 1 << 22,
                 seed: int = 1, **opts) -> list[int]:
    """Equal-work key windows of f * g (the same on every rank)."""
    hist, krange = B.kron_split_hist(f, g, nbins=nbins, nsamples=nsamples, seed=seed, ctx=ctx, **opts)
    return cuts_from_hist(hist, krange, nparts)


def mul_window(f, g, lo: int, hi: int, ctx=None, **opts):
    """Terms of f * g with keys in [lo, hi): (exps, coef) for polynomials,
    (exps, trig, kind, coef) for Poisson series, as torch tensors."""
    opts = dict(opts)
    opts.pop("code_lo", None)
    opts.pop("code_hi", None)
    if hi <= lo:   # an empty window
        hi = lo = max(lo, 0)
        if hasattr(f, "trig"):
            return B.poisson_mul(f, g, ctx=ctx, code_lo=1, code_hi=1, **opts)[:4]
        ex, cf, _, _ = B.poly_mul(f.exps, f.coef, g.exps, g.coef, ctx=ctx, code_lo=1, code_hi=1, **opts)
        return ex, cf
    if hasattr(f, "trig"):
        return B.poisson_mul(f, g, ctx=ctx, code_lo=int(lo), code_hi=int(hi), **opts)[:4]
    ex, cf, _, _ = B.poly_mul(f.exps, f.coef, g.exps, g.coef, ctx=ctx, code_lo=int(lo), code_hi=int(hi),
                              **opts)
    return ex, cf


def gather_parts(part, group=None):
    """Concatenate every rank's part (tensors whose last axis is the term axis)
    in rank order; every rank receives the whole.  The fields of a part are
    packed into one byte buffer (each field padded to 8 bytes), so the gather
    is one all_gather of the term counts and one of the packed buffers.  Works
    with any backend that supports all_gather of int64 and uint8 tensors on
    the part's device."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = part[-1].device
    n = int(part[-1].shape[-1])
    mine = torch.tensor([n], dtype=torch.int64, device=dev)
    sizes_t = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes_t, mine, group=group)
    sizes = [int(x.item()) for x in sizes_t]

    def field_bytes(a, k):
        rows = 1
        for d in a.shape[:-1]:
            rows *= int(d)
        b = rows * k * a.element_size()
        return b, (b + 7) // 8 * 8

    def packed(k):
        return sum(field_bytes(a, k)[1] for a in part)

    m = max(8, max(packed(k) for k in sizes))
    buf = torch.zeros(m, dtype=torch.uint8, device=dev)
    o = 0
    for a in part:
        b, pb = field_bytes(a, n)
        if b:
            buf[o:o + b] = a.contiguous().view(-1).view(torch.uint8)
        o += pb
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    pieces = [[] for _ in part]
    for rb, k in zip(bufs, sizes):
        o = 0
        for q, a in enumerate(part):
            b, pb = field_bytes(a, k)
            pieces[q].append(rb[o:o + b].view(a.dtype).reshape(tuple(a.shape[:-1]) + (k,)))
            o += pb
    return tuple(torch.cat(p, dim=-1) for p in pieces)


def sharded_mul(f, g, group=None, ctx=None, gather: bool = True, **opts):
    """Rank r of `group` computes key window r of f * g (windows of equal
    sampled work); with gather, every rank returns the whole product, else
    (cuts, its own window's terms)."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    cuts = split_points(f, g, world, ctx=ctx, **opts)
    part = mul_window(f, g, cuts[rank], cuts[rank + 1], ctx=ctx, **opts)
    if not gather:
        return cuts, part
    return gather_parts(part, group)
