"""Helpers shared by the GPU parity tests: run the library on numpy inputs and
compare with the oracle term by term."""
from __future__ import annotations

import numpy as np


def to_np(t):
    if t is None:
        return None
    if hasattr(t, "detach"):
        return t.detach().cpu().numpy()
    return np.asarray(t)


def poly_keys(exps: np.ndarray) -> np.ndarray:
    """Rows (one per term) comparable in the canonical order (last variable most significant)."""
    return np.ascontiguousarray(exps.T)


def assert_poly_equal(gexps, gcoef, r, what=""):
    """Bit-exact comparison of a polynomial product with the oracle result r."""
    gexps, gcoef = to_np(gexps), to_np(gcoef)
    assert gexps.shape == r.exps.shape, f"{what}: {gexps.shape[1]} terms vs oracle {r.exps.shape[1]}"
    if not np.array_equal(gexps, r.exps):
        bad = np.nonzero((gexps != r.exps).any(axis=0))[0]
        raise AssertionError(f"{what}: exponents differ at {bad.size} terms, first {bad[:5]}")
    if not np.array_equal(gcoef, r.coef):
        bad = np.nonzero(gcoef != r.coef)[0]
        raise AssertionError(f"{what}: coefficients differ at {bad.size} terms, first {bad[:5]}: "
                             f"{gcoef[bad[:3]]} vs {r.coef[bad[:3]]}")


def assert_poly_close(gexps, gcoef, r, rel=1e-12, what=""):
    """float64 polynomial product: same support up to exact zeros, |diff| <= rel * mass."""
    gexps, gcoef = to_np(gexps), to_np(gcoef)
    _assert_keyed_close(poly_keys(gexps), gcoef, poly_keys(r.exps), r.coef, r.mass, rel, what)


def pseries_keys(exps, trig, kind):
    exps, trig, kind = to_np(exps), to_np(trig), to_np(kind)
    return np.ascontiguousarray(np.concatenate(
        [kind.astype(np.int32)[None, :], trig, exps], axis=0).T)


def assert_pseries_close(g, r, rel=1e-12, what=""):
    """Poisson product: per key |gpu - oracle| <= rel * sum|contributions| (oracle kept zeros).

    Also checks the GPU output is in canonical order (kind, then trig multipliers
    from the highest index, then exponents from the highest index) without repeats.
    """
    ge, gt, gk, gc = (to_np(x) for x in g[:4])
    np_, nt = ge.shape[0], gt.shape[0]
    cols = lambda e, t, k: np.concatenate([e, t, k.astype(np.int32)[None, :]], axis=0).T
    gk_rows = cols(ge, gt, gk)   # least significant column first
    ok_rows = cols(r.exps, r.trig, r.kind)
    packed = _pack_rows(np.concatenate([ok_rows, gk_rows]))
    if packed is None:
        gkeys = pseries_keys(ge, gt, gk)
        okeys = pseries_keys(r.exps, r.trig, r.kind)
        _assert_keyed_close(gkeys, gc, okeys, r.coef, r.mass, rel, what)
        return
    po, pg = packed[: ok_rows.shape[0]], packed[ok_rows.shape[0]:]
    assert (np.diff(pg) > 0).all(), f"{what}: GPU output not strictly in canonical order"
    assert (np.diff(po) > 0).all(), f"{what}: oracle output not in canonical order"
    pos = np.searchsorted(po, pg)
    ok = (pos < po.shape[0])
    ok[ok] = po[pos[ok]] == pg[ok]
    assert ok.all(), f"{what}: {int((~ok).sum())} GPU keys the oracle never produced"
    ov = r.coef.copy()
    gv = np.zeros_like(ov)
    gv[pos] = gc
    err = np.abs(gv - ov)
    bad = err > rel * r.mass
    assert not bad.any(), (f"{what}: {int(bad.sum())} keys beyond {rel} x mass; worst ratio "
                           f"{(err / np.maximum(r.mass, 1e-300)).max():.3e}")


def _pseries_sort_cols(np_, nt):
    # np.lexsort: last key is primary -> list least significant first
    cols = [1 + nt + k for k in range(np_)] + [1 + k for k in range(nt)] + [0]
    return cols


def _pack_rows(rows: np.ndarray):
    """One int64 per row (mixed radix over the columns' ranges), or None if it overflows."""
    if rows.shape[0] == 0:
        return np.zeros(0, np.int64)
    lo = rows.min(axis=0).astype(np.int64)
    span = rows.max(axis=0).astype(np.int64) - lo + 1
    if float(np.prod(span.astype(np.float64))) >= 2.0 ** 62:
        return None
    out = np.zeros(rows.shape[0], np.int64)
    for c in range(rows.shape[1] - 1, -1, -1):
        out = out * span[c] + (rows[:, c].astype(np.int64) - lo[c])
    return out


def _assert_keyed_close(gkeys, gcoef, okeys, ocoef, omass, rel, what):
    # join on the key rows
    allk = np.concatenate([okeys, gkeys])
    packed = _pack_rows(allk)
    if packed is not None:
        _, inv = np.unique(packed, return_inverse=True)
    else:
        _, inv = np.unique(allk, axis=0, return_inverse=True)
    inv = inv.ravel()
    oid, gid = inv[: okeys.shape[0]], inv[okeys.shape[0]:]
    m = inv.max() + 1 if inv.size else 0
    ov = np.zeros(m); gv = np.zeros(m); mass = np.zeros(m)
    present_o = np.zeros(m, bool)
    ov[oid] = ocoef; mass[oid] = omass; present_o[oid] = True
    gv[gid] = gcoef
    extra = ~present_o[gid]
    assert not extra.any(), f"{what}: {int(extra.sum())} GPU keys the oracle never produced"
    assert np.unique(gid).shape[0] == gid.shape[0], f"{what}: repeated GPU keys"
    err = np.abs(gv - ov)
    bad = err > rel * mass
    assert not bad.any(), (f"{what}: {int(bad.sum())} keys beyond {rel} x mass; worst ratio "
                           f"{(err / np.maximum(mass, 1e-300)).max():.3e}")
    # keys the GPU dropped must be exact zeros there, i.e. within tolerance of 0
    return True
