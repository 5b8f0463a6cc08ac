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
    in rank order; every rank receives the whole.  Works with any backend that
    supports all_gather for the part's device and dtypes."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = part[-1].device
    n = int(part[-1].shape[-1])
    mine = torch.tensor([n], dtype=torch.int64, device=dev)
    sizes_t = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes_t, mine, group=group)
    sizes = [int(x.item()) for x in sizes_t]
    m = max(1, max(sizes))
    out = []
    for a in part:
        pad = torch.zeros(tuple(a.shape[:-1]) + (m,), dtype=a.dtype, device=dev)
        pad[..., :n] = a
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad, group=group)
        out.append(torch.cat([b[..., :k] for b, k in zip(bufs, sizes)], dim=-1))
    return tuple(out)


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
