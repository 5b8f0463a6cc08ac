"""Truncated multiplication (degree bound, Sec. 3) on the GPU against the oracle.

The library returns a truncated product sorted by its graded code: degree
first, then the other variables in the usual order.  The oracle returns the
ordinary order, so its terms are re-sorted by that key before the term-by-term
comparison (bit-exact for int64, 1e-12 x mass for float64).
"""
import math
import os
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_close, assert_poly_equal, assert_pseries_close, to_np
from pins import degrees
from workloads import (PSeries, Poly, dense_total_degree, random_poly, random_pseries,
                       workload_cfg2)

pytestmark = pytest.mark.gpu
NT = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1004_4548_gb300 as k
    k.load()
    return k


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def graded_rows(exps, mask):
    """Exponent rows in graded significance: the mask's highest-index variable is
    replaced by the degree, which becomes the last (most significant) row."""
    v = exps.shape[0]
    m = mask if mask else (1 << v) - 1
    r = max(k for k in range(v) if (m >> k) & 1)
    rows = [exps[k].astype(np.int64) for k in range(v) if k != r] + [degrees(exps, mask)]
    return np.stack(rows)


def graded_poly(r, mask):
    """Oracle polynomial result re-sorted into graded order."""
    idx = np.lexsort(graded_rows(r.exps, mask))
    return SimpleNamespace(exps=r.exps[:, idx], coef=r.coef[idx],
                           mass=None if r.mass is None else r.mass[idx], overflow=r.overflow)


def check_poly(kron, f, g, N, mask, path, what):
    opts = dict(path=path, trunc_degree=N, trunc_mask=mask)
    ex, cf, _, box = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), **opts)
    ex, cf = to_np(ex), to_np(cf)
    r = oracle.poly_mul(f, g, nthreads=NT, trunc=(N, mask))
    if ex.shape[1]:
        assert (degrees(ex, mask) <= N).all(), f"{what}: term above the bound"
        key = graded_rows(ex, mask)
        assert (np.lexsort(key) == np.arange(ex.shape[1])).all(), f"{what}: not in graded order"
        assert (ex.min(axis=1) >= box[0]).all() and (ex.max(axis=1) <= box[1]).all(), f"{what}: box"
    if f.coef.dtype == np.float64:
        assert_poly_close(ex, cf, r, 1e-12, what)
    else:
        assert_poly_equal(ex, cf, graded_poly(r, mask), what)
    return ex.shape[1]


PATHS = (1, 2)   # dense, hash


@pytest.mark.parametrize("path", PATHS)
def test_truncated_dense_square_closed_form(kron, path):
    """All monomials of degree <= 20 in 4 variables, squared, truncated at 20:
    exactly the C(24, 4) monomials of degree <= 20 survive."""
    f, g = workload_cfg2()
    n = check_poly(kron, f, g, 20, 0, path, f"cfg2 trunc 20 path={path}")
    assert n == math.comb(24, 4) == 10626


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("mask,N", [(0, 4), (0b0110, 3), (0b1000, -1), (0b0101, 0), (0, 100), (0, -40)])
def test_truncated_random_laurent(kron, path, mask, N):
    f = random_poly(4, 3000, [-4, 0, -6, -2], [5, 7, 3, 6], 2100)
    g = random_poly(4, 2500, [-4, 0, -6, -2], [5, 7, 3, 6], 2101)
    n = check_poly(kron, f, g, N, mask, path, f"laurent mask={mask:b} N={N} path={path}")
    if N == -40:
        assert n == 0
    if N == 100:   # above every degree: the full product, re-sorted
        assert n == oracle.poly_mul(f, g, nthreads=NT).coef.shape[0]


@pytest.mark.parametrize("path", PATHS)
def test_truncated_float64(kron, path):
    f = random_poly(3, 2000, -5, 5, 2200, "f64")
    g = random_poly(3, 1800, -5, 5, 2201, "f64")
    check_poly(kron, f, g, 1, 0b011, path, f"f64 trunc path={path}")


def test_truncated_drops_operand_terms(kron):
    """Terms whose own degree leaves no partner are dropped before the product;
    the rest still multiply exactly (many blocks, ragged tail)."""
    f = dense_total_degree(3, 14, -50, 50, 2300)
    g = dense_total_degree(3, 9, -50, 50, 2301)
    for N in (0, 3, 9, 15, 22):
        for path in PATHS:
            check_poly(kron, f, g, N, 0, path, f"dense factors N={N} path={path}")


def test_truncated_single_variable_mask_one_term(kron):
    f = Poly(np.array([[2], [-3]], np.int32), np.array([7], np.int64))
    g = Poly(np.array([[1, 5], [4, 0]], np.int32), np.array([3, -2], np.int64))
    for N, want in ((3, 1), (2, 0), (7, 2)):
        for path in PATHS:
            n = check_poly(kron, f, g, N, 0b01, path, f"tiny N={N}")
            assert n == want


def graded_pseries_view(ex, tr, kd, cf, mask):
    return (graded_rows(ex, mask), tr, kd, cf)


def graded_pseries(r, mask):
    """Oracle Poisson result with graded exponent rows, re-sorted into the
    library's order: kind, then trig multipliers, then the graded part."""
    ge = graded_rows(r.exps, mask)
    idx = np.lexsort(np.concatenate([ge, r.trig.astype(np.int64), r.kind.astype(np.int64)[None, :]]))
    return SimpleNamespace(exps=ge[:, idx], trig=r.trig[:, idx], kind=r.kind[idx], coef=r.coef[idx],
                           mass=r.mass[idx])


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("mask,N", [(0, 2), (0b10, 0), (0b11, -3)])
def test_truncated_poisson(kron, path, mask, N):
    f = random_pseries(2, 3, 3000, 4, 5, 2400)
    g = random_pseries(2, 3, 2600, 4, 5, 2401)
    F = PSeries(dev(f.exps), dev(f.trig), dev(f.kind), dev(f.coef))
    G = PSeries(dev(g.exps), dev(g.trig), dev(g.kind), dev(g.coef))
    out = kron.poisson_mul(F, G, path=path, trunc_degree=N, trunc_mask=mask)
    ex, tr, kd, cf = (to_np(x) for x in out[:4])
    r = oracle.poisson_mul(f, g, nthreads=NT, trunc=(N, mask), keep_zero=True)
    if ex.shape[1]:
        assert (degrees(ex, mask) <= N).all()
    ro = graded_pseries(r, mask)
    assert_pseries_close(graded_pseries_view(ex, tr, kd, cf, mask), ro, 1e-12,
                         f"poisson trunc mask={mask:b} N={N} path={path}")


def test_truncated_batch_matches_single_calls(kron):
    pairs, opts = [], []
    for s in range(12):
        f = random_poly(3, 300 + 97 * s, -3, 4, 2500 + s)
        g = random_poly(3, 200 + 61 * s, -3, 4, 2600 + s)
        pairs.append((f, g))
        opts.append(dict(trunc_degree=s - 4, trunc_mask=[0, 0b001, 0b110][s % 3]))
    fp = random_pseries(2, 2, 500, 3, 3, 2700)
    gp = random_pseries(2, 2, 400, 3, 3, 2701)
    pairs.append((fp, gp))
    opts.append(dict(trunc_degree=1, trunc_mask=0))
    out = kron.kron_mul_batch(pairs, opts=opts)
    for (f, g), o, res in zip(pairs, opts, out):
        assert res["status"] == 0
        N, mask = o["trunc_degree"], o["trunc_mask"]
        if isinstance(f, Poly):
            r = graded_poly(oracle.poly_mul(f, g, trunc=(N, mask)), mask)
            assert_poly_equal(to_np(res["exps"]), to_np(res["coef"]), r, f"batch N={N}")
        else:
            r = oracle.poisson_mul(f, g, trunc=(N, mask), keep_zero=True)
            ro = graded_pseries(r, mask)
            view = graded_pseries_view(to_np(res["exps"]), to_np(res["trig"]), to_np(res["kind"]),
                                       to_np(res["coef"]), mask)
            assert_pseries_close(view, ro, 1e-12, "batch poisson")


def test_truncated_prepared_batch_replays(kron):
    import torch
    pairs = []
    for s in range(6):
        f = random_poly(3, 800, -3, 5, 2800 + s)
        g = random_poly(3, 700, -3, 5, 2900 + s)
        pairs.append((Poly(dev(f.exps), dev(f.coef)), Poly(dev(g.exps), dev(g.coef))))
    opts = [dict(trunc_degree=2 + s, trunc_mask=0) for s in range(6)]
    b = kron.PreparedBatch(pairs, opts=opts)
    try:
        first = [(to_np(r["exps"]).copy(), to_np(r["coef"]).copy()) for r in b.first_results()]
        for f, _ in pairs:
            f.coef.mul_(3)
        b.launch()
        torch.cuda.synchronize()
        for (ex, cf), r in zip(first, b.results()):
            assert r["status"] == 0
            assert np.array_equal(to_np(r["exps"]), ex)
            assert np.array_equal(to_np(r["coef"]), 3 * cf)
    finally:
        b.close()


def test_truncation_invalid_mask(kron):
    f = random_poly(2, 50, 0, 4, 3000)
    with pytest.raises(kron.KronError) as e:
        kron.poly_mul(dev(f.exps), dev(f.coef), dev(f.exps), dev(f.coef), trunc_degree=3, trunc_mask=0b100)
    assert e.value.status == kron.KR_ERR_INVALID
