"""The seeded input generators, which both the oracle tests and the CUDA parity
tests draw from: the random stream against its published definition, and the
generated series against the validity rules the library's inputs obey.  CPU
only."""
import math

import numpy as np

from workloads import (Rng, batch_mix, dense_box, dense_total_degree, mp_sparse, poisson_random,
                       random_poly, total_degree_tuples, workload_cfg4)


def test_splitmix64_matches_its_published_outputs():
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; Vigna's reference code):
    the widely published first outputs for seeds 0 and 1234567.  The same
    values on every host make the synthetic inputs identical on x86 and Arm."""
    assert [int(x) for x in Rng(0).u64(4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(x) for x in Rng(1234567).u64(3)] == [6457827717110365317, 3203168211198807973,
                                                      9817491932198370423]


def test_stream_is_counter_based():
    """Draws in pieces continue the same stream as one draw of the total."""
    a = Rng(99)
    pieces = np.concatenate([a.u64(3), a.u64(0), a.u64(17), a.u64(1)])
    assert np.array_equal(pieces, Rng(99).u64(21))


def test_derived_draws_stay_in_range():
    r = Rng(7)
    x = r.ints(-5, 9, 20000)
    assert x.min() == -5 and x.max() == 9
    z = r.nonzero_ints(-3, 3, 20000)
    assert (z != 0).all() and z.min() == -3 and z.max() == 3
    u = r.uniform(20000)
    assert (u >= 0).all() and (u < 1).all()
    p = r.perm(1000)
    assert np.array_equal(np.sort(p), np.arange(1000))


def _distinct_columns(*arrays):
    rows = np.concatenate([np.atleast_2d(a).astype(np.int64) for a in arrays], axis=0).T
    return np.unique(rows, axis=0).shape[0] == rows.shape[0]


def test_polynomial_generators_give_distinct_monomials():
    for v, D in ((1, 9), (3, 5), (4, 10)):
        t = total_degree_tuples(v, D)
        assert t.shape == (math.comb(v + D, v), v) and (t >= 0).all() and (t.sum(axis=1) <= D).all()
        assert np.unique(t, axis=0).shape[0] == t.shape[0]
    p = dense_total_degree(4, 6, -9, 9, 11)
    assert _distinct_columns(p.exps) and (p.coef != 0).all() and p.coef.dtype == np.int64
    f, g = mp_sparse("f", 6, -9, 9, 12), mp_sparse("g", 6, -9, 9, 13)
    assert f.n == g.n == math.comb(5 + 6, 5) and _distinct_columns(f.exps) and _distinct_columns(g.exps)
    assert (f.exps[2] % 2 == 0).all() and (f.exps[3] % 3 == 0).all() and (f.exps[4] % 5 == 0).all()
    assert (g.exps[0] % 5 == 0).all() and (g.exps[1] % 3 == 0).all() and (g.exps[2] % 2 == 0).all()
    q = random_poly(3, 150, [-2, 0, -4], [3, 4, 1], 14)   # of the box's 180 monomials
    assert q.n == 150 and _distinct_columns(q.exps)
    assert random_poly(3, 500, [-2, 0, -4], [3, 4, 1], 14).n == 180   # capped at the box
    lo, hi = np.array([-2, 0, -4]), np.array([3, 4, 1])
    assert ((q.exps >= lo[:, None]) & (q.exps <= hi[:, None])).all()
    b = dense_box([-1, 0], [5, 3], 0.5, -7, 7, 15)
    assert _distinct_columns(b.exps) and (b.coef != 0).all() and 0 < b.n < 7 * 4


def _assert_valid_series(s):
    """Every term canonical (the highest-index nonzero multiplier positive), no
    sine of the zero multiplier vector, no two terms with one key."""
    t = s.trig.T
    nz = t != 0
    zero = ~nz.any(axis=1)
    last = t.shape[1] - 1 - np.argmax(nz[:, ::-1], axis=1)
    lead = t[np.arange(t.shape[0]), last]
    assert ((lead > 0) | zero).all()
    assert not (zero & (s.kind == 1)).any()
    assert _distinct_columns(s.exps, s.trig, s.kind)


def test_poisson_generator_gives_valid_series():
    """Valid series, with the magnitudes of the benchmark series:
    |C| = 10^-(|i|_1 + |j|_1) * 10^u, u in [0, 1)."""
    for s in (poisson_random(3000, 3, 4, 4, 8, 16), workload_cfg4(2000)[0]):
        _assert_valid_series(s)
        l1 = np.abs(s.exps).sum(axis=0) + np.abs(s.trig).sum(axis=0)
        e = np.log10(np.abs(s.coef)) + l1
        assert (e >= -1e-12).all() and (e < 1 + 1e-12).all()


def test_batch_mix_is_uneven_and_reproducible():
    a = batch_mix(64, seed_base=77, max_terms=400)
    b = batch_mix(64, seed_base=77, max_terms=400)
    assert len(a) == len(b) == 64
    sizes = []
    for k, ((fa, ga), (fb, gb)) in enumerate(zip(a, b)):
        assert np.array_equal(fa.coef, fb.coef) and np.array_equal(ga.exps, gb.exps)
        sizes.append(fa.n * ga.n)
        for p in (fa, ga):
            if k % 2:   # odd products: Poisson series
                _assert_valid_series(p)
            else:
                assert _distinct_columns(p.exps) and (p.coef != 0).all()
    assert max(sizes) > 10 * min(sizes)
