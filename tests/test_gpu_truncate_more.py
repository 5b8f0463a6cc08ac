"""Truncation by harmonic order and by coefficient magnitude (Sec. 3) on the
GPU against the oracle, alone, together, with the degree bound, in key
windows, in batches and in graph replays.

Neither criterion changes the coding, so the output is in the canonical order
(or the graded order when a degree bound is also given) and compares term by
term with the oracle: bit-exact keys, float64 coefficients within 1e-12 of the
summed magnitudes.
"""
import os

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_close, assert_pseries_close, to_np
from pins import powers_of_ten
from test_gpu_truncate import graded_pseries, graded_pseries_view
from workloads import PSeries, Poly, Rng, random_poly, random_pseries, workload_cfg4

pytestmark = pytest.mark.gpu
NT = max(1, min(16, os.cpu_count() or 1))
REL = 1e-12


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


def dps(p):
    return PSeries(dev(p.exps), dev(p.trig), dev(p.kind), dev(p.coef))


def harmonic_orders(trig, mask):
    nt = trig.shape[0]
    m = mask if mask else (1 << nt) - 1
    return sum(np.abs(trig[k].astype(np.int64)) for k in range(nt) if (m >> k) & 1)


@pytest.fixture(scope="module")
def series():
    f = random_pseries(2, 3, 3000, 4, 5, 4100)
    g = random_pseries(2, 3, 2600, 4, 5, 4101)
    return f, g


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("mask,N", [(0, 0), (0, 4), (0b010, 2), (0b101, 7), (0, 100), (0b001, -1)])
def test_harmonic_truncation(kron, series, path, mask, N):
    f, g = series
    out = kron.poisson_mul(dps(f), dps(g), path=path, harmonic_order=N, harmonic_mask=mask)
    ex, tr, kd, cf = (to_np(x) for x in out[:4])
    r = oracle.poisson_mul(f, g, nthreads=NT, harmonic=(N, mask), keep_zero=True)
    if N < 0:
        assert cf.shape[0] == 0 and r.coef.shape[0] == 0
        return
    assert (harmonic_orders(tr, mask) <= N).all()
    assert_pseries_close((ex, tr, kd, cf), r, REL, f"harmonic mask={mask:b} N={N} path={path}")


@pytest.fixture(scope="module")
def magnitudes():
    """Poisson series with coefficients spread over nine decades."""
    rng = Rng(4200)
    f = random_pseries(2, 3, 3000, 4, 5, 4201)
    g = random_pseries(2, 3, 2600, 4, 5, 4202)
    return powers_of_ten(f, rng.ints(0, 8, f.n), rng), powers_of_ten(g, rng.ints(0, 8, g.n), rng)


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("eps", [1e-3, 3.7e-7, 1e-12, 1e-30])
def test_coefficient_truncation_poisson(kron, magnitudes, path, eps):
    f, g = magnitudes
    out = kron.poisson_mul(dps(f), dps(g), path=path, coef_min=eps)
    r = oracle.poisson_mul(f, g, nthreads=NT, coef_min=eps, keep_zero=True)
    assert_pseries_close(tuple(to_np(x) for x in out[:4]), r, REL, f"coef eps={eps} path={path}")


@pytest.mark.parametrize("eps", [0.5, 2e-4, 1e-9])
def test_coefficient_truncation_polynomial(kron, eps):
    rng = Rng(4300)
    f0 = random_poly(4, 4000, -5, 5, 4301, "f64")
    g0 = random_poly(4, 3500, -5, 5, 4302, "f64")
    f, g = powers_of_ten(f0, rng.ints(0, 6, f0.n), rng), powers_of_ten(g0, rng.ints(0, 6, g0.n), rng)
    for path in (0, 1, 2):   # a bound always takes the hash path
        ex, cf, _, _ = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), path=path,
                                     coef_min=eps)
        r = oracle.poly_mul(f, g, nthreads=NT, coef_min=eps, keep_zero=True)
        assert_poly_close(to_np(ex), to_np(cf), r, REL, f"polynomial coef eps={eps} path={path}")


def test_coefficient_bound_is_inclusive(kron):
    f = Poly(np.array([[1], [0]], np.int32), np.array([2.0]))
    g = Poly(np.array([[0], [1]], np.int32), np.array([3.0]))
    ex, cf, _, _ = kron.poly_mul(f.exps, f.coef, g.exps, g.coef, coef_min=6.0, host_out=True)
    assert to_np(cf).tolist() == [6.0]
    ex, cf, _, _ = kron.poly_mul(f.exps, f.coef, g.exps, g.coef, coef_min=np.nextafter(6.0, 7.0), host_out=True)
    assert to_np(cf).shape[0] == 0
    one = lambda c: PSeries(np.zeros((1, 1), np.int32), np.ones((1, 1), np.int32), np.zeros(1, np.uint8),
                            np.array([c]))
    for path in (1, 2):
        out = kron.poisson_mul(one(2.0), one(3.0), path=path, coef_min=6.0, host_out=True)
        assert sorted(to_np(out[3]).tolist()) == [3.0, 3.0]   # cos 0 and cos 2y, 1/2 * 6 each
        out = kron.poisson_mul(one(2.0), one(3.0), path=path, coef_min=np.nextafter(6.0, 7.0), host_out=True)
        assert to_np(out[3]).shape[0] == 0


@pytest.mark.parametrize("path", [1, 2])
def test_all_three_bounds_together(kron, magnitudes, path):
    f, g = magnitudes
    opts = dict(trunc_degree=2, trunc_mask=0b01, harmonic_order=6, harmonic_mask=0b011, coef_min=1e-9)
    out = kron.poisson_mul(dps(f), dps(g), path=path, **opts)
    ex, tr, kd, cf = (to_np(x) for x in out[:4])
    r = oracle.poisson_mul(f, g, nthreads=NT, trunc=(2, 0b01), harmonic=(6, 0b011), coef_min=1e-9,
                           keep_zero=True)
    assert_pseries_close(graded_pseries_view(ex, tr, kd, cf, 0b01), graded_pseries(r, 0b01), REL,
                         f"three bounds path={path}")


@pytest.mark.parametrize("path", [1, 2])
def test_truncated_windows_make_the_product(kron, magnitudes, path):
    from paper_1004_4548_gb300 import shard
    f, g = magnitudes
    F, G = dps(f), dps(g)
    opts = dict(path=path, harmonic_order=5, coef_min=1e-8)
    cuts = shard.split_points(F, G, 4, **opts)
    parts = [shard.mul_window(F, G, a, b, **opts) for a, b in zip(cuts, cuts[1:])]
    got = [np.concatenate([to_np(p[k]) for p in parts], axis=-1) for k in range(4)]
    r = oracle.poisson_mul(f, g, nthreads=NT, harmonic=(5, 0), coef_min=1e-8, keep_zero=True)
    assert_pseries_close(tuple(got), r, REL, f"truncated windows path={path}")


def test_cfg4_truncated_every_term(kron):
    """cfg4's distributions at 2500 terms per operand (|C| = 10^-(|i|_1 + |j|_1 - u):
    the magnitudes fall with the size of the exponents and multipliers, as in
    the series of celestial mechanics), truncated at coefficient products of
    1e-38 (about 14% of the pairs) and harmonic order 20."""
    f, g = workload_cfg4(2500)
    r = oracle.poisson_mul(f, g, nthreads=NT, harmonic=(20, 0), coef_min=1e-38, keep_zero=True)
    full = oracle.poisson_mul(f, g, nthreads=NT, keep_zero=True)
    assert 0 < r.coef.shape[0] < full.coef.shape[0] // 2
    for path in (1, 2):
        out = kron.poisson_mul(dps(f), dps(g), path=path, harmonic_order=20, coef_min=1e-38)
        assert_pseries_close(tuple(to_np(x) for x in out[:4]), r, REL, f"cfg4 truncated path={path}")


def test_truncated_batch_and_replay(kron, magnitudes):
    """Mixed truncation options in one batch; a prepared batch replays with
    the coefficients negated (same magnitudes, same kept pairs: every result
    negated exactly)."""
    import torch
    f, g = magnitudes
    pairs, opts = [], []
    for s in range(6):
        fs = PSeries(f.exps[:, : 400 + 100 * s], f.trig[:, : 400 + 100 * s], f.kind[: 400 + 100 * s],
                     f.coef[: 400 + 100 * s])
        gs = PSeries(g.exps[:, : 300 + 50 * s], g.trig[:, : 300 + 50 * s], g.kind[: 300 + 50 * s],
                     g.coef[: 300 + 50 * s])
        pairs.append((fs, gs))
        opts.append([dict(coef_min=1e-7), dict(harmonic_order=4), dict(coef_min=1e-5, harmonic_order=6)][s % 3])
    fp = random_poly(3, 900, -3, 3, 4400, "f64")
    gp = random_poly(3, 800, -3, 3, 4401, "f64")
    pairs.append((fp, gp))
    opts.append(dict(coef_min=0.3))

    def want(pair, o, sign=1.0):
        a, b = pair
        if isinstance(a, Poly):
            return oracle.poly_mul(Poly(a.exps, sign * a.coef), b, coef_min=o.get("coef_min"), keep_zero=True)
        h = (o["harmonic_order"], 0) if "harmonic_order" in o else None
        return oracle.poisson_mul(PSeries(a.exps, a.trig, a.kind, sign * a.coef), b, harmonic=h,
                                  coef_min=o.get("coef_min"), keep_zero=True)

    def check(res, sign, what):
        for i, (pair, o, r) in enumerate(zip(pairs, opts, res)):
            assert r["status"] == 0, f"{what} {i}: status {r['status']}"
            w = want(pair, o, sign)
            if isinstance(pair[0], Poly):
                assert_poly_close(to_np(r["exps"]), to_np(r["coef"]), w, REL, f"{what} {i}")
            else:
                assert_pseries_close((r["exps"], r["trig"], r["kind"], r["coef"]), w, REL, f"{what} {i}")

    check(kron.kron_mul_batch(pairs, opts=opts), 1.0, "batch")
    D = []
    for a, b in pairs:
        if isinstance(a, Poly):
            D.append((Poly(dev(a.exps), dev(a.coef)), Poly(dev(b.exps), dev(b.coef))))
        else:
            D.append((dps(a), dps(b)))
    pb = kron.PreparedBatch(D, opts=opts)
    try:
        check(pb.first_results(), 1.0, "prepared")
        for a, _ in D:
            a.coef.neg_()
        pb.launch()
        torch.cuda.synchronize()
        check(pb.results(), -1.0, "replay, f negated")
    finally:
        pb.close()


def test_truncation_option_errors(kron):
    f = random_poly(2, 50, 0, 4, 4500)
    with pytest.raises(kron.KronError) as e:   # a coefficient bound on int64 coefficients
        kron.poly_mul(dev(f.exps), dev(f.coef), dev(f.exps), dev(f.coef), coef_min=1.0)
    assert e.value.status == kron.KR_ERR_INVALID
    ff = random_poly(2, 50, 0, 4, 4501, "f64")
    with pytest.raises(kron.KronError) as e:   # no trig variables to count
        kron.poly_mul(dev(ff.exps), dev(ff.coef), dev(ff.exps), dev(ff.coef), harmonic_order=3)
    assert e.value.status == kron.KR_ERR_INVALID
    p = random_pseries(1, 2, 30, 2, 3, 4502)
    big = PSeries(p.exps.copy(), p.trig.copy(), p.kind.copy(), p.coef.copy())
    big.trig[1, 0] = 40000   # a counted multiplier beyond the 16-bit lanes
    with pytest.raises(kron.KronError) as e:
        kron.poisson_mul(dps(big), dps(p), harmonic_order=3)
    assert e.value.status == kron.KR_ERR_INVALID
    out = kron.poisson_mul(dps(big), dps(p), harmonic_order=3, harmonic_mask=0b01)   # not counted: fine
    r = oracle.poisson_mul(big, p, harmonic=(3, 0b01), keep_zero=True)
    assert_pseries_close(tuple(to_np(x) for x in out[:4]), r, REL, "uncounted large multiplier")
