"""Autotuner for the per-product knobs: dense or hash path, dense block size,
hash load factor.

The paper picks the algorithm from the densities of the factors (Sec. 3.2)
without a threshold; here the choice is measured.  Products are grouped into
shape classes by kind (polynomial / Poisson series), the magnitude of the
term-product count and, for polynomials, the ratio of the code range W to the
term-product count.  For every class of the uneven batch, the class's
products (up to `per_class` of them) are multiplied as one batch
(kron_mul_batch, the way the options are used), once with the library's own
choices and once per candidate configuration (wall time around the call,
median of three after a warm-up).  A class gets a table entry only when a
candidate beats the library's choices by more than `margin`; every other
class keeps them.  opts_for() looks a product's class up in the table.

  python -m paper_1004_4548_gb300.autotune --out tuned.json [--products 4096]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuned.json")

# dense block sizes: a batch's dense products share one launch whose shared
# memory per CTA is set by its largest block, so larger blocks would lower the
# occupancy of every product in the batch
DENSE_S = (2048, 4096, 8192)
HASH_ALPHA = (0.3, 0.5, 0.7)

_table_cache: dict | None = None


def _np(a):
    return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)


def features(f, g) -> dict:
    """Shape features of the product f * g (host-side, from the exponent ranges)."""
    poisson = hasattr(f, "trig")
    nf, ng = int(f.coef.shape[0]), int(g.coef.shape[0])
    pairs = max(1, nf * ng)
    fe, ge = _np(f.exps), _np(g.exps)
    W = 1.0
    if fe.shape[0] > 0 and nf > 0 and ng > 0:
        w = (fe.max(axis=1).astype(np.int64) + ge.max(axis=1)) - (fe.min(axis=1).astype(np.int64) + ge.min(axis=1)) + 1
        W = float(np.prod(w.astype(np.float64)))
    if poisson and nf > 0 and ng > 0:
        R = np.abs(_np(f.trig)).max(axis=1).astype(np.int64) + np.abs(_np(g.trig)).max(axis=1)
        W *= float(np.prod((2 * R + 1).astype(np.float64)))
    return {"poisson": poisson, "pairs": pairs, "W": W}


def class_key(feat: dict) -> str:
    p = int(round(math.log2(feat["pairs"])))
    if feat["poisson"]:
        return f"pois|p{p}"
    d = int(round(math.log2(max(feat["W"], 1.0) / feat["pairs"])))
    d = max(-10, min(14, d))
    return f"poly|p{p}|d{d}"


def candidates(feat: dict) -> list[dict]:
    out = [{"path": 2, "load_factor": a} for a in HASH_ALPHA]
    if not feat["poisson"] and feat["W"] * 8 <= 4e9:
        out = [{"path": 1, "block_slots": s} for s in DENSE_S] + out
    return out


def load_table(path: str = TABLE) -> dict:
    global _table_cache
    if _table_cache is None:
        try:
            with open(path) as fh:
                _table_cache = json.load(fh).get("classes", {})
        except (OSError, ValueError):
            _table_cache = {}
    return _table_cache


def opts_for(f, g, table: dict | None = None) -> dict:
    """Tuned kr_opts fields for f * g ({} when its class was never tuned)."""
    t = load_table() if table is None else table
    feat = features(f, g)
    key = class_key(feat)
    o = t.get(key)
    if o is None:
        return {}
    o = dict(o)
    if o.get("path") == 1 and (feat["poisson"] or feat["W"] * 8 > 4e9):
        return {}
    return o


def _time_batch(kron, ctx, pairs, o, reps=3):
    import torch
    opts = [dict(o) for _ in pairs]
    ts = []
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        kron.kron_mul_batch(pairs, ctx=ctx, opts=opts)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    return float(np.median(ts[1:]))


def tune(products: int = 4096, per_class: int = 16, seed_base: int = 5000, margin: float = 0.03) -> dict:
    import torch
    import paper_1004_4548_gb300 as kron
    from workloads import PSeries, Poly, batch_mix
    ctx = kron.context()
    mix = batch_mix(products, seed_base=seed_base)

    def dev(p):
        if isinstance(p, PSeries):
            return PSeries(*(torch.from_numpy(x).cuda() for x in (p.exps, p.trig, p.kind, p.coef)))
        return Poly(torch.from_numpy(p.exps).cuda(), torch.from_numpy(p.coef).cuda())

    classes: dict[str, list] = {}
    for f, g in mix:
        feat = features(f, g)
        classes.setdefault(class_key(feat), []).append((f, g, feat))
    table, report = {}, {}
    for key, items in sorted(classes.items()):
        sample = [(dev(f), dev(g)) for f, g, _ in items[:per_class]]
        t_def = _time_batch(kron, ctx, sample, {})
        best, best_t = None, t_def
        for o in candidates(items[0][2]):
            t = _time_batch(kron, ctx, sample, o)
            if t < best_t and t < t_def * (1.0 - margin):
                best, best_t = o, t
        if best is not None:
            table[key] = best
        report[key] = {"n": len(items), "sampled": len(sample), "best": best, "ms": best_t * 1e3,
                       "default_ms": t_def * 1e3}
        del sample
        ctx.trim()
    return {"classes": table, "report": report,
            "candidates": {"dense_block_slots": DENSE_S, "hash_load_factor": HASH_ALPHA},
            "sample": f"{products} products of the uneven batch, seeds {seed_base}+k; per class up to "
                      f"{per_class} products as one batch; entries only where a candidate beats the "
                      f"library's choices by more than {margin:.0%}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--products", type=int, default=4096)
    ap.add_argument("--per-class", type=int, default=16)
    ap.add_argument("--margin", type=float, default=0.03)
    a = ap.parse_args()
    res = tune(a.products, a.per_class, margin=a.margin)
    with open(a.out, "w") as fh:
        json.dump(res, fh, indent=1, sort_keys=True)
    print(f"{len(res['classes'])} of {len(res['report'])} classes take tuned options -> {a.out}")


if __name__ == "__main__":
    main()
