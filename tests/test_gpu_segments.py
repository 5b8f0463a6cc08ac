"""Dense products whose terms come in runs of consecutive codes against the
oracle, bit-exact: full tiles of f terms, the dense walk's steps without range
tests (int32-range coefficients), and the tiles and windows cut at run ends.

Cases: one long run per operand (a dense univariate product), boxes with
dropped monomials (ragged runs), coefficients at the int32 ends (the sums wrap
modulo 2^64), block sizes from the smallest to the largest, key windows,
truncation by degree, and a batch.  Each also runs on the hash path, which
shares no accumulation code with the dense one.
"""
import os

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_equal, to_np
from workloads import Poly, Rng, dense_box, dense_total_degree

pytestmark = pytest.mark.gpu
NT = max(1, min(16, os.cpu_count() or 1))
I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1


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


def run(kron, f, g, **opts):
    ex, cf, _, _ = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), **opts)
    return to_np(ex), to_np(cf)


def extremes(p, seed):
    """p with a third of its coefficients at the int32 ends."""
    rng = Rng(seed)
    u = rng.ints(0, 2, p.coef.shape[0])
    c = np.where(u == 0, I32_MIN, np.where(u == 1, I32_MAX, p.coef)).astype(np.int64)
    return Poly(p.exps, c)


def univariate(lo, hi, seed):
    return dense_box([lo], [hi], 1.0, -(1 << 20), 1 << 20, seed)


CASES = {
    "univariate long runs": lambda: (univariate(0, 4999, 7001), univariate(-300, 2999, 7002)),
    "univariate int32 ends": lambda: (extremes(univariate(-50, 2100, 7003), 7004),
                                      extremes(univariate(0, 1700, 7005), 7006)),
    "box 2 vars, 15% dropped": lambda: (dense_box([-7, 0], [40, 60], 0.85, -999, 999, 7007),
                                        dense_box([0, -5], [33, 20], 0.85, -999, 999, 7008)),
    # short runs: the term form
    "box 3 vars, 40% dropped": lambda: (dense_box([0, 0, 0], [20, 9, 7], 0.6, -(1 << 30), 1 << 30, 7009),
                                        dense_box([-3, 0, 0], [11, 12, 5], 0.6, -(1 << 30), 1 << 30, 7010)),
    # several output blocks (code range 51 x 41 x 21), runs of ~10 codes
    "box 3 vars, 10% dropped": lambda: (dense_box([0, 0, 0], [25, 20, 10], 0.9, -(1 << 30), 1 << 30, 7017),
                                        dense_box([0, -4, 0], [24, 15, 9], 0.9, -(1 << 30), 1 << 30, 7018)),
    "simplex degree 12 in 3 vars": lambda: (dense_total_degree(3, 12, -(1 << 20), 1 << 20, 7011),
                                            dense_total_degree(3, 12, -(1 << 20), 1 << 20, 7012)),
    "box 2 vars int32 ends": lambda: (extremes(dense_box([0, 0], [60, 30], 0.9, -5, 5, 7013), 7014),
                                      extremes(dense_box([0, 0], [45, 25], 0.9, -5, 5, 7015), 7016)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_runs_bit_exact(kron, name):
    f, g = CASES[name]()
    r = oracle.poly_mul(f, g, nthreads=NT)
    for path in (kron.KR_PATH_AUTO, kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        ex, cf = run(kron, f, g, path=path)
        assert_poly_equal(ex, cf, r, f"{name} path={path}")


@pytest.mark.parametrize("S", [256, 2048, 8192, 27648])
def test_block_sizes(kron, S):
    f, g = CASES["box 2 vars, 15% dropped"]()
    r = oracle.poly_mul(f, g, nthreads=NT)
    ex, cf = run(kron, f, g, path=kron.KR_PATH_DENSE, block_slots=S)
    assert_poly_equal(ex, cf, r, f"S={S}")


def test_key_windows_concatenate(kron):
    f, g = CASES["simplex degree 12 in 3 vars"]()
    r = oracle.poly_mul(f, g, nthreads=NT)
    # output codes: variable 0 least significant, widths of the product box
    w = [int(f.exps[k].max() - f.exps[k].min() + g.exps[k].max() - g.exps[k].min() + 1) for k in range(3)]
    W = w[0] * w[1] * w[2]
    cuts = [0, 1, 777, W // 3, W // 3 + 1, (2 * W) // 3 + 5, W]
    parts = [run(kron, f, g, path=kron.KR_PATH_DENSE, code_lo=a, code_hi=b) for a, b in zip(cuts, cuts[1:])]
    ex = np.concatenate([p[0] for p in parts], axis=1)
    cf = np.concatenate([p[1] for p in parts])
    assert_poly_equal(ex, cf, r, "windows")


def test_truncated_by_degree(kron):
    from test_gpu_truncate import graded_poly
    f, g = CASES["simplex degree 12 in 3 vars"]()
    for N in (5, 13, 24):
        ex, cf, _, _ = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef),
                                     path=kron.KR_PATH_DENSE, trunc_degree=N)
        r = oracle.poly_mul(f, g, nthreads=NT, trunc=(N, 0))
        assert_poly_equal(to_np(ex), to_np(cf), graded_poly(r, 0), f"trunc {N}")


def test_batch(kron):
    pairs = [CASES[n]() for n in ("univariate long runs", "box 3 vars, 10% dropped",
                                  "simplex degree 12 in 3 vars", "box 2 vars int32 ends")]
    out = kron.kron_mul_batch(pairs)
    for i, ((f, g), o) in enumerate(zip(pairs, out)):
        assert o["status"] == 0
        assert_poly_equal(o["exps"], o["coef"], oracle.poly_mul(f, g, nthreads=NT), f"batch product {i}")
