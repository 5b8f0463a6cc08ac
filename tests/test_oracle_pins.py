"""Pins for the oracle: its results checked against what the mathematics fixes,
never against itself.  CPU only.

Every pin is a function returning a list of failure messages, so the planted
mistake test at the end can check that each deliberate error in the oracle is
caught by at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from pins import (M61, as_dict, box_convolution, degrees, eval_level_truncated, eval_mod_m31,
                  eval_mod_p, eval_poly_real, eval_pseries, eval_truncated_mod_m31,
                  eval_truncated_pseries, fourier_coefficients, powers_of_ten, sample_grid)
from workloads import (PSeries, Poly, Rng, dense_total_degree, fateman, random_poly,
                       random_pseries, total_degree_tuples, workload_cfg1,
                       workload_cfg2, workload_cfg3)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NT = max(1, min(16, os.cpu_count() or 1))


# ---------------------------------------------------------------------------
# pins as functions (plant = which oracle build to check)
# ---------------------------------------------------------------------------

# thread counts every multi-threaded pin runs with: one thread takes no merge,
# three and four split f unevenly and merge the partial maps
THREADS = (1, 3, 4)


def pin_bruteforce(plant=0):
    """Small random Laurent polynomials: oracle == dense N-d convolution, on one
    thread and with the f terms split over three and four threads (the float64
    partial sums then go through the merge)."""
    errs = []
    cases = [(1, 12, -5, 6), (2, 40, -3, 4), (3, 60, [-2, 0, -4], [3, 4, 1]),
             (3, 80, 0, 5)]
    for s, (v, n, lo, hi) in enumerate(cases):
        for dt in ("i64", "f64"):
            f = random_poly(v, n, lo, hi, 100 + s, dt)
            g = random_poly(v, n + 7, lo, hi, 200 + s, dt)
            want = box_convolution(f, g)
            for nt in THREADS:
                r = oracle.poly_mul(f, g, nthreads=nt, plant=plant)
                got = as_dict(r.exps, r.coef)
                if dt == "i64":
                    if got != {k: int(x) for k, x in want.items()}:
                        errs.append(f"bruteforce mismatch v={v} {dt} threads={nt}")
                else:
                    keys = set(got) | set(want)
                    bad = [k for k in keys
                           if abs(got.get(k, 0.0) - want.get(k, 0.0)) > 1e-12 * 16 * n]
                    if bad:
                        errs.append(f"bruteforce mismatch v={v} {dt} threads={nt}: {len(bad)} keys")
    return errs


def pin_mass(plant=0):
    """The per-key mass (sum of |contribution|), the basis of the float64
    tolerance, equals its exact value.

    * Polynomials: the mass of f*g is the product of |f| and |g|, computed
      here by dense N-d convolution (a different algorithm), on one thread
      and on three and four (the masses of the partial maps add).
    * Poisson series: every pair of terms emits two terms of magnitude
      |C D| / 2 (Eq. 6 with the 1/2 of the identities), so each hand-worked
      single-term case has mass 3 per emitted term (C D = 6), 6 where both
      terms land on one key; and in 2 cos 3y - 2 cos y times 3 cos y the two
      contributions to cos 2y cancel (coefficient 0, mass 6).
    """
    errs = []
    for s, (v, n, lo, hi) in enumerate([(2, 60, -3, 4), (3, 90, [-2, 0, -4], [3, 4, 1])]):
        f = random_poly(v, n, lo, hi, 2100 + s, "f64")
        g = random_poly(v, n + 9, lo, hi, 2200 + s, "f64")
        want = box_convolution(Poly(f.exps, np.abs(f.coef)), Poly(g.exps, np.abs(g.coef)))
        for nt in THREADS:
            r = oracle.poly_mul(f, g, nthreads=nt, plant=plant, keep_zero=True)
            got = as_dict(r.exps, r.mass)
            if set(got) != set(want) or any(abs(got[k] - want[k]) > 1e-13 * want[k] for k in want):
                errs.append(f"polynomial mass differs from the |f| |g| convolution v={v} threads={nt}")
    for tf, kf, tg, kg, terms in WERNER_CASES:
        f = PSeries(np.array([[-1]], np.int32), np.array(tf, np.int32)[:, None],
                    np.array([kf], np.uint8), np.array([2.0]))
        g = PSeries(np.array([[3]], np.int32), np.array(tg, np.int32)[:, None],
                    np.array([kg], np.uint8), np.array([3.0]))
        r = oracle.poisson_mul(f, g, plant=plant)
        got = sorted((tuple(int(x) for x in r.trig[:, i]), int(r.kind[i]), float(r.mass[i]))
                     for i in range(r.coef.shape[0]))
        want = sorted((t, k, abs(c)) for t, k, c in terms)   # no contribution cancels here
        if got != want:
            errs.append(f"werner mass {tf},{kf} x {tg},{kg}: got {got}, want {want}")
    f = PSeries(np.zeros((1, 2), np.int32), np.array([[3, 1]], np.int32), np.zeros(2, np.uint8),
                np.array([2.0, -2.0]))
    g = PSeries(np.zeros((1, 1), np.int32), np.array([[1]], np.int32), np.zeros(1, np.uint8),
                np.array([3.0]))
    for nt in (1, 2):
        r = oracle.poisson_mul(f, g, nthreads=nt, plant=plant, keep_zero=True)
        got = {int(r.trig[0, i]): (float(r.coef[i]), float(r.mass[i])) for i in range(r.coef.shape[0])}
        if got != {0: (-3.0, 3.0), 2: (0.0, 6.0), 4: (3.0, 3.0)}:
            errs.append(f"cancelling Poisson mass threads={nt}: {got}")
    return errs


# Single-term Poisson products worked by hand from the product-to-sum
# identities (Eq. 6 with the factor 1/2), C = 2, D = 3:
# (f trig, f kind, g trig, g kind, expected [(trig, kind, coef)]) with 2 trig
# vars.  x exponents: f has x^-1, g has x^3; the product always carries x^2.
WERNER_CASES = [
        ((1, 1), 0, (0, 1), 0, [((1, 0), 0, 3.0), ((1, 2), 0, 3.0)]),           # cos cos
        ((1, 1), 0, (0, 1), 1, [((1, 2), 1, 3.0), ((1, 0), 1, -3.0)]),          # cos sin
        ((1, 1), 1, (0, 1), 0, [((1, 2), 1, 3.0), ((1, 0), 1, 3.0)]),           # sin cos
        ((1, 1), 1, (0, 1), 1, [((1, 0), 0, 3.0), ((1, 2), 0, -3.0)]),          # sin sin
        ((0, 1), 0, (1, 1), 0, [((1, 0), 0, 3.0), ((1, 2), 0, 3.0)]),           # a-b negated, cos
        ((0, 1), 1, (1, 1), 0, [((1, 2), 1, 3.0), ((1, 0), 1, -3.0)]),          # a-b negated, sin
        ((0, 1), 0, (1, 1), 1, [((1, 2), 1, 3.0), ((1, 0), 1, 3.0)]),           # cos sin, negated
        ((1, 0), 0, (0, 1), 0, [((-1, 1), 0, 3.0), ((1, 1), 0, 3.0)]),          # (1,-1) -> (-1,1)
        ((1, 0), 1, (0, 1), 0, [((1, 1), 1, 3.0), ((-1, 1), 1, -3.0)]),         # sin of (1,-1)
        ((1, 0), 1, (1, 0), 0, [((2, 0), 1, 3.0)]),                             # sin 0 dropped
        ((1, 0), 1, (1, 0), 1, [((0, 0), 0, 3.0), ((2, 0), 0, -3.0)]),          # cos 0 kept
        ((1, 0), 0, (1, 0), 0, [((0, 0), 0, 3.0), ((2, 0), 0, 3.0)]),
        ((1, 1), 0, (0, 0), 0, [((1, 1), 0, 6.0)]),                             # t_g = 0: C*D
        ((1, 0), 1, (0, 0), 0, [((1, 0), 1, 6.0)]),
]


def pin_werner(plant=0):
    """Single-term Poisson products against the product-to-sum identities (Eq. 6, with 1/2)."""
    errs = []
    C, D = 2.0, 3.0
    for tf, kf, tg, kg, want in WERNER_CASES:
        f = PSeries(np.array([[-1]], np.int32), np.array(tf, np.int32)[:, None],
                    np.array([kf], np.uint8), np.array([C]))
        g = PSeries(np.array([[3]], np.int32), np.array(tg, np.int32)[:, None],
                    np.array([kg], np.uint8), np.array([D]))
        r = oracle.poisson_mul(f, g, plant=plant)
        got = sorted((tuple(int(x) for x in r.trig[:, i]), int(r.kind[i]), float(r.coef[i]))
                     for i in range(r.coef.shape[0]))
        if sorted(want) != got or (r.coef.shape[0] and not (r.exps == 2).all()):
            errs.append(f"werner {tf},{kf} x {tg},{kg}: got {got}, want {sorted(want)}")
    return errs


def pin_random_angles(plant=0):
    """F(x, y) * G(x, y) == H(x, y) at random real x and angles y."""
    errs = []
    rng = Rng(77)
    for s, (np_, nt, n) in enumerate([(1, 1, 20), (2, 3, 60), (3, 4, 150)]):
        f = random_pseries(np_, nt, n, 3, 4, 300 + s)
        g = random_pseries(np_, nt, n + 11, 3, 4, 400 + s)
        pts = [(0.5 + rng.uniform(np_), 2 * math.pi * rng.uniform(nt)) for _ in range(4)]
        for nth in THREADS:
            h = oracle.poisson_mul(f, g, nthreads=nth, plant=plant)
            H = PSeries(h.exps, h.trig, h.kind, h.coef)
            for x, y in pts:
                fv, fm = eval_pseries(f, x, y)
                gv, gm = eval_pseries(g, x, y)
                hv, _ = eval_pseries(H, x, y)
                if abs(fv * gv - hv) > 1e-12 * fm * gm:
                    errs.append(f"random angles np={np_} nt={nt} threads={nth}: {fv * gv} vs {hv}")
                    break
    return errs


def pin_canonical(plant=0):
    """Every output multiplier vector is canonical and no sine of the zero vector survives."""
    errs = []
    f = random_pseries(2, 3, 80, 2, 3, 501)
    g = random_pseries(2, 3, 90, 2, 3, 502)
    h = oracle.poisson_mul(f, g, plant=plant)
    for i in range(h.coef.shape[0]):
        t = h.trig[:, i]
        nz = np.nonzero(t)[0]
        if nz.size == 0:
            if h.kind[i] == 1:
                errs.append("sine of the zero vector in the output")
        elif t[nz[-1]] <= 0:
            errs.append(f"non-canonical output vector {t.tolist()}")
            break
    return errs


def pin_mod_p(plant=0):
    """h(x) == f(x) g(x) mod 2^61 - 1 at random points (Laurent: inverses)."""
    errs = []
    for s, (v, n, lo, hi) in enumerate([(2, 50, -6, 6), (4, 120, [-3, 0, -1, -8], [5, 9, 2, 0])]):
        f = random_poly(v, n, lo, hi, 600 + s)
        g = random_poly(v, n, lo, hi, 700 + s)
        h = oracle.poly_mul(f, g, plant=plant)
        rng = Rng(800 + s)
        for _ in range(3):
            pt = [int(x) for x in rng.ints(2, M61 - 1, v)]
            lhs = eval_mod_p(h.exps, h.coef, pt)
            rhs = eval_mod_p(f.exps, f.coef, pt) * eval_mod_p(g.exps, g.coef, pt) % M61
            if lhs != rhs:
                errs.append(f"mod-p evaluation mismatch v={v}")
                break
    return errs


def _table1_rows():
    return [tuple(map(int, l.split())) for l in open(os.path.join(GOLDEN, "table1_codes.txt"))
            if l.strip() and not l.startswith("#")]


def _box(v, hi, shift, dt):
    """Every monomial of the box [shift, shift + hi]^v, coefficient 1."""
    e = np.array(np.meshgrid(*[np.arange(hi + 1)] * v, indexing="ij")).reshape(v, -1) + shift
    return Poly(e.astype(np.int32), np.ones(e.shape[1], np.int64 if dt == "i64" else np.float64))


def pin_order(plant=0):
    """Output order (Sec. 2, Table 1): ascending Kronecker code, variable 0
    varying fastest.  The product of the boxes [0, 1]^3 and [0, 2]^3 fills
    [0, 3]^3 with positive coefficients, so its 64 terms must come out in the
    order of Table 1's codes (c = (1, 4, 16)): Table 1's rows at their code's
    position, and every term at position x + 4 y + 16 z; the same with the
    box shifted to negative exponents, float64 coefficients and the f terms
    split over three threads.  Poisson series: cosines before sines, then
    the multiplier vectors and then the polynomial exponents, each compared
    from the highest-index variable down (the ascending order of the coding
    that puts the kind above the trig part above the polynomial part)."""
    errs = []
    rows = _table1_rows()
    for shift, nth, dt in ((0, 1, "i64"), (-2, 3, "i64"), (-1, 3, "f64")):
        f, g = _box(3, 1, shift, dt), _box(3, 2, 0, dt)
        r = oracle.poly_mul(f, g, nthreads=nth, plant=plant)
        if r.coef.shape[0] != 64:
            errs.append(f"box product shift={shift}: {r.coef.shape[0]} terms, want 64")
            continue
        x, y, z = (r.exps.astype(np.int64) - shift)
        if not np.array_equal(x + 4 * y + 16 * z, np.arange(64)):
            errs.append(f"box product shift={shift} threads={nth} {dt}: not in Table 1's code order")
        for zz, yy, xx, code in rows:
            if (int(x[code]), int(y[code]), int(z[code])) != (xx, yy, zz):
                errs.append(f"Table 1 row ({zz}, {yy}, {xx}) not at position {code} (shift={shift})")
                break
    for nth in (1, 3):
        f = random_pseries(2, 3, 70, 2, 3, 2501)
        g = random_pseries(2, 3, 75, 2, 3, 2502)
        h = oracle.poisson_mul(f, g, nthreads=nth, plant=plant)
        keys = [(int(h.kind[i]),) + tuple(int(t) for t in h.trig[::-1, i])
                + tuple(int(e) for e in h.exps[::-1, i]) for i in range(h.coef.shape[0])]
        if any(a >= b for a, b in zip(keys, keys[1:])):
            errs.append(f"Poisson output not strictly ascending (kind, trig, poly) threads={nth}")
    return errs


def pin_cancellation(plant=0):
    """Terms whose contributions cancel leave the output, worked by hand:
    (x - y)(x + y) = x^2 - y^2, (x + 1/x)(x - 1/x) = x^2 - x^-2 (Laurent),
    and 3 cos y (2 cos 3y - 2 cos y) = -3 + 3 cos 4y (Eq. 6 with the 1/2: the
    two contributions to cos 2y cancel); kept as zeros only on request."""
    errs = []
    cases = [((np.array([[1, 0], [0, 1]]), [1, -1]), (np.array([[1, 0], [0, 1]]), [1, 1]),
              {(2, 0): 1, (0, 2): -1}, {(1, 1): 0}),
             ((np.array([[1, -1]]), [1, 1]), (np.array([[1, -1]]), [1, -1]),
              {(2,): 1, (-2,): -1}, {(0,): 0})]
    for (ef, cf), (eg, cg), want, zeros in cases:
        for dt in ("i64", "f64"):
            typ = np.int64 if dt == "i64" else np.float64
            f = Poly(ef.astype(np.int32), np.array(cf, typ))
            g = Poly(eg.astype(np.int32), np.array(cg, typ))
            for keep in (False, True):
                r = oracle.poly_mul(f, g, plant=plant, keep_zero=keep)
                w = {**want, **zeros} if keep else want
                if as_dict(r.exps, r.coef) != w:
                    errs.append(f"cancellation {dt} keep_zero={keep}: {as_dict(r.exps, r.coef)}, want {w}")
    f = PSeries(np.zeros((1, 2), np.int32), np.array([[3, 1]], np.int32), np.zeros(2, np.uint8),
                np.array([2.0, -2.0]))
    g = PSeries(np.zeros((1, 1), np.int32), np.array([[1]], np.int32), np.zeros(1, np.uint8),
                np.array([3.0]))
    r = oracle.poisson_mul(f, g, plant=plant)
    got = {(int(r.trig[0, i]), int(r.kind[i])): float(r.coef[i]) for i in range(r.coef.shape[0])}
    if got != {(0, 0): -3.0, (4, 0): 3.0}:
        errs.append(f"cancelling Poisson product: {got}")
    return errs


def pin_compensated(plant=0):
    """float64 sums are compensated (Neumaier 1974), so a sum whose exact value
    is a double comes out exact however its parts cancel: in
    (1e16 + x - 1e16 x^2)(x^2 + x + 1) the x^2 coefficient gathers 1e16, 1 and
    -1e16 (exactly 1; an uncompensated running sum gives 0 or 2, since 1e16 + 1
    is not a double), on one thread and with the three f terms on three
    threads (the partial sums then meet in the merge); likewise for a Poisson
    series, where each contribution carries the 1/2 of Eq. 6."""
    errs = []
    f = Poly(np.array([[0, 1, 2]], np.int32), np.array([1e16, 1.0, -1e16]))
    g = Poly(np.array([[2, 1, 0]], np.int32), np.array([1.0, 1.0, 1.0]))
    for nth in (1, 3):
        r = oracle.poly_mul(f, g, nthreads=nth, plant=plant)
        got = as_dict(r.exps, r.coef)
        if got.get((2,)) != 1.0:
            errs.append(f"compensated sum threads={nth}: x^2 coefficient {got.get((2,))}, want 1.0")
    z = lambda n: np.zeros((1, n), np.int32)
    F = PSeries(np.array([[0, 1, 2]], np.int32), z(3), np.zeros(3, np.uint8), np.array([2e16, 2.0, -2e16]))
    G = PSeries(np.array([[2, 1, 0]], np.int32), z(3), np.zeros(3, np.uint8), np.array([1.0, 1.0, 1.0]))
    for nth in (1, 3):
        r = oracle.poisson_mul(F, G, nthreads=nth, plant=plant)
        got = {int(r.exps[0, i]): float(r.coef[i]) for i in range(r.coef.shape[0])}
        if got.get(2) != 2.0:   # cos 0 cos 0 = 1/2 + 1/2: each pair gives C D in two halves
            errs.append(f"compensated Poisson sum threads={nth}: x^2 coefficient {got.get(2)}, want 2.0")
    return errs


# ---------------------------------------------------------------------------
# the pins, run on the oracle
# ---------------------------------------------------------------------------

def test_generator_counts_match_paper():
    for line in open(os.path.join(GOLDEN, "paper_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, v, D, n = line.split()
        assert total_degree_tuples(int(v), int(D)).shape[0] == int(n)
        assert math.comb(int(v) + int(D), int(v)) == int(n)


def test_oracle_bruteforce():
    assert pin_bruteforce() == []


def test_oracle_werner_single_terms():
    assert pin_werner() == []


def test_oracle_random_angles():
    assert pin_random_angles() == []


def test_oracle_mass_exact():
    assert pin_mass() == []


def test_oracle_canonical_output():
    assert pin_canonical() == []


def test_oracle_mod_p_small():
    assert pin_mod_p() == []


def test_oracle_output_order_table1():
    assert pin_order() == []


def test_oracle_cancellation():
    assert pin_cancellation() == []


def test_oracle_compensated_sums():
    assert pin_compensated() == []


def test_oracle_cfg1_bruteforce():
    f, g = workload_cfg1()
    r = oracle.poly_mul(f, g)
    want = box_convolution(f, g)
    assert as_dict(r.exps, r.coef) == {k: int(x) for k, x in want.items()}
    assert r.coef.shape[0] == math.comb(4 + 20, 4) == 10626
    assert not r.overflow


@pytest.mark.parametrize("v,D", [(1, 7), (2, 5), (3, 4), (4, 3), (5, 2)])
def test_oracle_closed_form_count(v, D):
    """Product of two dense total-degree-D polynomials has C(v + 2D, v) terms."""
    f = dense_total_degree(v, D, 1, 9, 900 + v)
    g = dense_total_degree(v, D, 1, 9, 950 + v)
    r = oracle.poly_mul(f, g)
    assert r.coef.shape[0] == math.comb(v + 2 * D, v)
    assert (r.exps.sum(axis=0) <= 2 * D).all() and (r.exps >= 0).all()


def test_oracle_cfg2_count_and_eval():
    f, g = workload_cfg2()
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert r.coef.shape[0] == math.comb(4 + 40, 4) == 135751
    assert not r.overflow
    rng = Rng(2024)
    for _ in range(3):
        pt = [int(x) for x in rng.ints(2, (1 << 31) - 2, 4)]
        assert eval_mod_m31(r.exps, r.coef, pt) == \
            eval_mod_m31(f.exps, f.coef, pt) * eval_mod_m31(g.exps, g.coef, pt) % ((1 << 31) - 1)


def test_oracle_cfg3_support_and_eval():
    """MP-sparse structure: the key set is exactly the set of pairwise exponent sums."""
    f, g = workload_cfg3()
    r = oracle.poly_mul(f, g, nthreads=NT, keep_zero=True)
    assert not r.overflow
    hi = (f.exps.max(axis=1) + g.exps.max(axis=1) + 1).astype(np.int64)
    sums = []
    for ch in np.array_split(np.arange(f.n), 16):
        s = f.exps[:, ch][:, :, None].astype(np.int64) + g.exps[:, None, :]
        sums.append(np.unique(np.ravel_multi_index(tuple(s.reshape(5, -1)), tuple(hi))))
    support = np.unique(np.concatenate(sums))
    got = np.ravel_multi_index(tuple(r.exps.astype(np.int64)), tuple(hi))
    assert got.shape[0] == support.shape[0] == 5821335
    assert np.array_equal(np.sort(got), support)
    rng = Rng(3003)
    for _ in range(3):
        pt = [int(x) for x in rng.ints(2, (1 << 31) - 2, 5)]
        assert eval_mod_m31(r.exps, r.coef, pt) == \
            eval_mod_m31(f.exps, f.coef, pt) * eval_mod_m31(g.exps, g.coef, pt) % ((1 << 31) - 1)


def test_fateman_operands_and_small_product():
    """Fateman's operands (Sec. 5) are (1+x+y+z+t)^n and that plus one: their
    evaluations at a point are closed forms, and so is the product's."""
    M = (1 << 31) - 1
    f, g = fateman(30)
    assert f.n == g.n == math.comb(34, 4) == 46376
    assert int(f.coef.astype(np.uint64).sum(dtype=np.uint64)) == 5 ** 30 % (1 << 64)
    f, g = fateman(6)
    r = oracle.poly_mul(f, g)
    assert r.coef.shape[0] == math.comb(4 + 12, 4) and not r.overflow
    rng = Rng(3131)
    for _ in range(3):
        pt = [int(x) for x in rng.ints(2, M - 1, 4)]
        s = (1 + sum(pt)) % M
        fv = pow(s, 6, M)
        assert eval_mod_m31(f.exps, f.coef, pt) == fv
        assert eval_mod_m31(g.exps, g.coef, pt) == (fv + 1) % M
        assert eval_mod_m31(r.exps, r.coef, pt) == fv * (fv + 1) % M


def test_oracle_int64_wraps_and_flags_overflow():
    big = (1 << 62) + 12345
    f = Poly(np.array([[0, 1]], np.int32), np.array([big, 3], np.int64))
    g = Poly(np.array([[0, 1]], np.int32), np.array([7, big], np.int64))
    r = oracle.poly_mul(f, g)
    assert r.overflow
    exact = {0: big * 7, 1: big * big + 3 * 7, 2: 3 * big}
    for i in range(r.coef.shape[0]):
        e = int(r.exps[0, i])
        w = exact[e] % (1 << 64)
        w = w - (1 << 64) if w >= (1 << 63) else w
        assert int(r.coef[i]) == w


def test_oracle_threads_and_shards_agree():
    f = random_poly(3, 400, -5, 5, 11)
    g = random_poly(3, 300, -5, 5, 12)
    a = oracle.poly_mul(f, g, nthreads=1)
    b = oracle.poly_mul(f, g, nthreads=4)
    assert np.array_equal(a.exps, b.exps) and np.array_equal(a.coef, b.coef)
    parts = [oracle.poly_mul(f, g, shard=(3, s)) for s in range(3)]
    merged = {}
    for p in parts:
        d = as_dict(p.exps, p.coef)
        assert not (set(d) & set(merged))
        merged.update(d)
    assert merged == as_dict(a.exps, a.coef)
    keys = a.exps.T.copy()
    sh = oracle.shard_of_keys(keys, 3)
    for s in range(3):
        assert set(as_dict(a.exps[:, sh == s], a.coef[sh == s])) == set(as_dict(parts[s].exps, parts[s].coef))
    assert oracle.key_hash(keys[0]) % 3 == sh[0]


def test_oracle_pseries_shards_and_mass():
    f = random_pseries(2, 2, 120, 2, 3, 21)
    g = random_pseries(2, 2, 110, 2, 3, 22)
    full = oracle.poisson_mul(f, g, nthreads=3)
    assert (full.mass >= np.abs(full.coef) * (1 - 1e-15)).all()
    n = sum(oracle.poisson_mul(f, g, shard=(4, s)).coef.shape[0] for s in range(4))
    assert n == full.coef.shape[0]


def pin_truncation(plant=0):
    """Degree-truncated products (Sec. 3): the full product's convolution restricted
    to degree <= N, the graded evaluation, and the count of a dense truncated square."""
    errs = []
    cases = [(3, 70, [-2, 0, -3], [3, 4, 2], 0b111, 2), (3, 70, [-2, 0, -3], [3, 4, 2], 0b010, 5),
             (3, 70, [-2, 0, -3], [3, 4, 2], 0b101, -1), (2, 40, 0, 6, 0, 7), (4, 50, -2, 3, 0b1001, 0)]
    for s, (v, n, lo, hi, mask, N) in enumerate(cases):
        f = random_poly(v, n, lo, hi, 1300 + s)
        g = random_poly(v, n + 5, lo, hi, 1400 + s)
        r = oracle.poly_mul(f, g, plant=plant, trunc=(N, mask))
        m = mask if mask else (1 << v) - 1
        want = {k: int(c) for k, c in box_convolution(f, g).items()
                if sum(k[j] for j in range(v) if (m >> j) & 1) <= N}
        if as_dict(r.exps, r.coef) != want:
            errs.append(f"truncated convolution mismatch v={v} mask={mask:b} N={N}")
    for s, (mask, N) in enumerate([(0, 5), (0b0110, 3), (0b1000, -2)]):
        f = random_poly(4, 400, -3, 4, 1500 + s)
        g = random_poly(4, 350, -3, 4, 1600 + s)
        r = oracle.poly_mul(f, g, plant=plant, trunc=(N, mask))
        if (degrees(r.exps, mask) > N).any():
            errs.append("truncated product holds a term above the bound")
        rng = Rng(1700 + s)
        for _ in range(2):
            pt = [int(x) for x in rng.ints(2, (1 << 31) - 2, 4)]
            if eval_mod_m31(r.exps, r.coef, pt) != eval_truncated_mod_m31(f, g, pt, mask, N):
                errs.append(f"graded evaluation mismatch mask={mask:b} N={N}")
                break
    f = dense_total_degree(3, 6, 1, 9, 1801)
    g = dense_total_degree(3, 6, 1, 9, 1802)
    r = oracle.poly_mul(f, g, plant=plant, trunc=(8, 0))
    if r.coef.shape[0] != math.comb(3 + 8, 3):
        errs.append(f"dense truncated square: {r.coef.shape[0]} terms, want {math.comb(11, 3)}")
    rng = Rng(1900)
    for s, (mask, N) in enumerate([(0, 1), (0b10, 0)]):
        f = random_pseries(2, 2, 120, 3, 3, 1910 + s)
        g = random_pseries(2, 2, 130, 3, 3, 1920 + s)
        h = oracle.poisson_mul(f, g, plant=plant, trunc=(N, mask))
        H = PSeries(h.exps, h.trig, h.kind, h.coef)
        for _ in range(3):
            x = 0.5 + rng.uniform(2)
            y = 2 * math.pi * rng.uniform(2)
            want, mag = eval_truncated_pseries(f, g, x, y, mask, N)
            got, _ = eval_pseries(H, x, y)
            if abs(got - want) > 1e-12 * mag:
                errs.append(f"truncated Poisson evaluation mismatch mask={mask:b} N={N}")
                break
    return errs


def test_oracle_truncation():
    assert pin_truncation() == []


def pin_coef_truncation(plant=0):
    """Truncation by coefficient magnitude (Sec. 3): a pair contributes when
    |C_f C_g| >= eps.  With coefficients +-10^-level (1 + u/10) and
    eps = 0.5 * 10^-N the kept pairs are exactly those whose levels add up to
    at most N, so the truncated product evaluates to the sum of F_a G_b over
    a + b <= N (reached from f and g alone, at random points and angles).  At
    the boundary: 2 * 3 against eps = 6 is kept and against the next double
    above 6 is not; for Poisson series the bound applies to C_f C_g before the
    1/2 of the product-to-sum identities."""
    errs = []
    rng = Rng(2300)
    for s, (v, n, lo, hi) in enumerate([(2, 70, -3, 4), (3, 90, [-2, 0, -4], [3, 4, 1])]):
        f0 = random_poly(v, n, lo, hi, 2310 + s, "f64")
        g0 = random_poly(v, n + 13, lo, hi, 2320 + s, "f64")
        lf, lg = rng.ints(0, 4, f0.n), rng.ints(0, 4, g0.n)
        f, g = powers_of_ten(f0, lf, rng), powers_of_ten(g0, lg, rng)
        for N in (0, 3, 5, 8):
            for nth in (1, 3):
                h = oracle.poly_mul(f, g, nthreads=nth, plant=plant, coef_min=0.5 * 10.0 ** -N)
                for _ in range(2):
                    x = 0.5 + rng.uniform(v)
                    want, mag = eval_level_truncated(
                        f, g, lf, lg, N, lambda p, sel: eval_poly_real(p.exps[:, sel], p.coef[sel], x))
                    got, _ = eval_poly_real(h.exps, h.coef, x)
                    if abs(got - want) > 1e-12 * mag:
                        errs.append(f"coefficient-truncated polynomial v={v} N={N} threads={nth}")
                        break
    for s, (np_, nt, n) in enumerate([(1, 2, 60), (2, 3, 80)]):
        f0 = random_pseries(np_, nt, n, 2, 3, 2330 + s)
        g0 = random_pseries(np_, nt, n + 9, 2, 3, 2340 + s)
        lf, lg = rng.ints(0, 4, f0.n), rng.ints(0, 4, g0.n)
        f, g = powers_of_ten(f0, lf, rng), powers_of_ten(g0, lg, rng)
        for N in (1, 4, 7):
            h = oracle.poisson_mul(f, g, nthreads=2, plant=plant, coef_min=0.5 * 10.0 ** -N)
            H = PSeries(h.exps, h.trig, h.kind, h.coef)
            for _ in range(2):
                x = 0.5 + rng.uniform(np_)
                y = 2 * math.pi * rng.uniform(nt)
                sub = lambda p, sel: eval_pseries(PSeries(p.exps[:, sel], p.trig[:, sel], p.kind[sel],
                                                          p.coef[sel]), x, y)
                want, mag = eval_level_truncated(f, g, lf, lg, N, sub)
                got, _ = eval_pseries(H, x, y)
                if abs(got - want) > 1e-12 * mag:
                    errs.append(f"coefficient-truncated Poisson np={np_} nt={nt} N={N}")
                    break
    # the boundary, on a polynomial and a Poisson product
    f = Poly(np.array([[1], [0]], np.int32), np.array([2.0]))
    g = Poly(np.array([[0], [1]], np.int32), np.array([3.0]))
    for eps, want in ((6.0, {(1, 1): 6.0}), (np.nextafter(6.0, 7.0), {})):
        r = oracle.poly_mul(f, g, plant=plant, coef_min=eps)
        if as_dict(r.exps, r.coef) != want:
            errs.append(f"coefficient bound at eps={eps!r}: {as_dict(r.exps, r.coef)}")
    f = PSeries(np.zeros((1, 1), np.int32), np.array([[1]], np.int32), np.zeros(1, np.uint8), np.array([2.0]))
    g = PSeries(np.zeros((1, 1), np.int32), np.array([[1]], np.int32), np.zeros(1, np.uint8), np.array([3.0]))
    for eps, want in ((6.0, {0: 3.0, 2: 3.0}), (np.nextafter(6.0, 7.0), {})):
        r = oracle.poisson_mul(f, g, plant=plant, coef_min=eps)
        got = {int(r.trig[0, i]): float(r.coef[i]) for i in range(r.coef.shape[0])}
        if got != want:
            errs.append(f"Poisson coefficient bound at eps={eps!r}: {got}")
    return errs


def pin_harmonic_truncation(plant=0):
    """Truncation by the order of the Fourier harmonics (Sec. 3): a term is kept
    when the sum of |multiplier| over the chosen trig variables is at most N.
    Pinned by the 2-D FFT of F G sampled on a grid of angles (a different
    algorithm): the truncated product's Fourier coefficients must be those of
    F G for every harmonic of order <= N and zero above; plus hand-worked
    cases (cos y cos y = 1/2 + 1/2 cos 2y; a mask that counts one variable)."""
    errs = []
    rng = Rng(2400)
    M = 16   # product multipliers lie in [-6, 6]: no aliasing on 16 points
    for s in range(2):
        f = random_pseries(1, 2, 40, 2, 3, 2410 + s)
        g = random_pseries(1, 2, 45, 2, 3, 2420 + s)
        scale = float(np.abs(f.coef).sum() * np.abs(g.coef).sum())
        x = 0.5 + rng.uniform(1)
        # coefficients of F G: from the product of the sampled values
        full = fourier_coefficients(sample_grid(f, x, M) * sample_grid(g, x, M))
        k = np.fft.fftfreq(M, 1.0 / M).astype(int)
        K1, K2 = np.meshgrid(k, k, indexing="ij")
        for mask in (0, 0b10):
            order = (np.abs(K1) if mask in (0, 0b01) else 0) + (np.abs(K2) if mask in (0, 0b10) else 0)
            for N in (0, 2, 3, 5):
                h = oracle.poisson_mul(f, g, nthreads=2, plant=plant, harmonic=(N, mask), keep_zero=True)
                H = PSeries(h.exps, h.trig, h.kind, h.coef)
                got = fourier_coefficients(sample_grid(H, x, M))
                want = np.where(order <= N, full, 0.0)
                if np.abs(got - want).max() > 1e-12 * scale:
                    errs.append(f"harmonic truncation mask={mask:b} N={N}: Fourier coefficients differ")
    one = lambda t, c: PSeries(np.zeros((1, 1), np.int32), np.array(t, np.int32)[:, None],
                               np.zeros(1, np.uint8), np.array([c]))
    for N, want in ((0, {(0,): 0.5}), (1, {(0,): 0.5}), (2, {(0,): 0.5, (2,): 0.5})):
        r = oracle.poisson_mul(one([1], 1.0), one([1], 1.0), plant=plant, harmonic=(N, 0))
        got = {tuple(int(v) for v in r.trig[:, i]): float(r.coef[i]) for i in range(r.coef.shape[0])}
        if got != want:
            errs.append(f"cos y * cos y at harmonic order <= {N}: {got}")
    # (1, 1) and (-1, 1): difference (2, 0), sum (0, 2); only variable 0 counts
    r = oracle.poisson_mul(one([1, 1], 1.0), one([-1, 1], 1.0), plant=plant, harmonic=(1, 0b01))
    got = {tuple(int(v) for v in r.trig[:, i]): float(r.coef[i]) for i in range(r.coef.shape[0])}
    if got != {(0, 2): 0.5}:
        errs.append(f"masked harmonic order: {got}")
    return errs


def test_oracle_coefficient_truncation():
    assert pin_coef_truncation() == []


def test_oracle_harmonic_truncation():
    assert pin_harmonic_truncation() == []


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by some pin
# ---------------------------------------------------------------------------

PLANTS = {
    1: "product-to-sum halves dropped",
    2: "wrong sign in cos*sin",
    3: "difference taken as g - f",
    4: "canonical sign from the lowest-index multiplier",
    5: "last term of g skipped",
    6: "first exponent of f used twice",
    7: "degree bound applied as < N instead of <= N",
    8: "thread merge drops the other thread's running sum",
    9: "mass counts every contribution twice",
    10: "thread merge drops the other thread's mass",
    11: "coefficient bound applied as > eps instead of >= eps",
    12: "coefficient bound applied after the product-to-sum 1/2",
    13: "harmonic order bound applied as < N instead of <= N",
    14: "harmonic order counts every trig variable, ignoring the mask",
    15: "polynomial output ordered with variable 0 most significant",
    16: "zero int64 sums kept in the output",
    17: "Poisson output ordered by the polynomial part before the trig part",
    18: "a negated sine keeps its sign",
    19: "the difference term's polynomial exponents subtracted",
    20: "the compensation dropped from the float64 sums",
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_mistake_is_caught(plant):
    caught = (pin_werner(plant) + pin_canonical(plant) + pin_random_angles(plant)
              + pin_bruteforce(plant) + pin_mod_p(plant) + pin_truncation(plant)
              + pin_mass(plant) + pin_coef_truncation(plant) + pin_harmonic_truncation(plant)
              + pin_order(plant) + pin_cancellation(plant) + pin_compensated(plant))
    assert caught, f"planted mistake {plant} ({PLANTS[plant]}) escaped every pin"
