"""Parity of the CUDA path (through the C ABI) with the oracle.

int64 products: bit-exact.  float64 products: per output term
|gpu - oracle| <= 1e-12 * (sum of |contributions| to that term).
"""
import math
import os

import numpy as np
import pytest

import oracle
from gpu_compare import (assert_poly_close, assert_poly_equal, assert_pseries_close, to_np)
from workloads import (PSeries, Poly, Rng, fateman, poisson_random, random_poly, random_pseries,
                       workload_cfg1, workload_cfg2, workload_cfg3, workload_cfg4)

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


def run_poly(k, f, g, device_inputs=True, **opts):
    if device_inputs:
        ex, cf, _, _ = k.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), **opts)
    else:
        ex, cf, _, _ = k.poly_mul(f.exps, f.coef, g.exps, g.coef, host_out=True, **opts)
    return to_np(ex), to_np(cf)


def run_pseries(k, f, g, device_inputs=True, **opts):
    if device_inputs:
        F = PSeries(dev(f.exps), dev(f.trig), dev(f.kind), dev(f.coef))
        G = PSeries(dev(g.exps), dev(g.trig), dev(g.kind), dev(g.coef))
        out = k.poisson_mul(F, G, **opts)
    else:
        out = k.poisson_mul(f, g, host_out=True, **opts)
    return tuple(to_np(x) for x in out[:4])


# ---------------------------------------------------------------------------
# the benchmark workloads
# ---------------------------------------------------------------------------

def test_cfg1_dense_and_hash_bit_exact(kron):
    f, g = workload_cfg1()
    r = oracle.poly_mul(f, g)
    for path in (kron.KR_PATH_AUTO, kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        ex, cf = run_poly(kron, f, g, path=path)
        assert_poly_equal(ex, cf, r, f"cfg1 path={path}")


def test_cfg2_dense_bit_exact(kron):
    f, g = workload_cfg2()
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert r.coef.shape[0] == 135751 and not r.overflow
    ex, cf = run_poly(kron, f, g)
    assert_poly_equal(ex, cf, r, "cfg2 dense")
    for S in (2048, 27648):
        ex, cf = run_poly(kron, f, g, path=kron.KR_PATH_DENSE, block_slots=S)
        assert_poly_equal(ex, cf, r, f"cfg2 dense S={S}")


def test_cfg3_hash_bit_exact(kron):
    f, g = workload_cfg3()
    r = oracle.poly_mul(f, g, nthreads=NT)
    ex, cf = run_poly(kron, f, g)
    assert_poly_equal(ex, cf, r, "cfg3 hash")


def test_cfg4_reduced_full_compare(kron):
    """cfg4's distributions at 2500 terms per operand, every output term compared."""
    f, g = workload_cfg4(2500)
    r = oracle.poisson_mul(f, g, nthreads=NT, keep_zero=True)
    for path in (kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        out = run_pseries(kron, f, g, path=path)
        assert_pseries_close(out, r, REL, f"cfg4 n=2500 path={path}")


def test_cfg4_full_size_sampled_shard(kron):
    """Full cfg4 (20000 x 20000 terms) on the GPU; one 1/4096 slice of the output
    keys (FNV-1a shard) recomputed exactly by the oracle."""
    f, g = workload_cfg4()
    mod, sid = 4096, 17
    r = oracle.poisson_mul(f, g, nthreads=NT, shard=(mod, sid), keep_zero=True)
    assert r.coef.shape[0] > 1000
    keysets = []
    for path in (kron.KR_PATH_AUTO, kron.KR_PATH_HASH):   # AUTO takes the dense path here
        ge, gt, gk, gc = run_pseries(kron, f, g, path=path)
        keys = np.concatenate([gk.astype(np.int32)[None, :], gt, ge], axis=0).T
        sel = oracle.shard_of_keys(keys, mod) == sid
        assert_pseries_close((ge[:, sel], gt[:, sel], gk[sel], gc[sel]), r, REL, f"cfg4 shard path={path}")
        keysets.append((ge, gt, gk))
        del gc, keys, sel
    # both paths produce the same terms (zeros dropped alike)
    for a, b in zip(*keysets):
        assert np.array_equal(a, b)


def test_fateman_full_size_mod_2_64(kron):
    """Fateman's benchmark at full size (Sec. 5): (1+x+y+z+t)^30 times itself plus one,
    46376 x 46376 terms, the true multinomial coefficients.  The sums exceed int64;
    both sides reduce them modulo 2^64.  Every output term's exponents, the closed-form
    count C(4 + 60, 4), and a 1/997 slice of the coefficients are checked against the
    oracle (exact 128-bit sums, reduced)."""
    f, g = fateman()
    ex, cf = run_poly(kron, f, g)
    assert ex.shape[1] == math.comb(64, 4) == 635376
    assert (ex.sum(axis=0) <= 60).all() and (ex >= 0).all()
    mod, sid = 997, 5
    sel = oracle.shard_of_keys(np.ascontiguousarray(ex.T), mod) == sid
    r = oracle.poly_mul(f, g, nthreads=NT, shard=(mod, sid))
    assert r.overflow and r.coef.shape[0] > 300
    assert_poly_equal(ex[:, sel], cf[sel], r, "fateman slice")


# ---------------------------------------------------------------------------
# random cases: sizes spanning several tiles plus ragged tails
# ---------------------------------------------------------------------------

POLY_CASES = [
    # v, nf, ng, lo, hi
    (1, 1, 1, -3, 3),
    (1, 37, 1000, -500, 700),
    (2, 1, 777, -40, 40),
    (3, 513, 257, [-5, 0, -9], [6, 30, 2]),
    (4, 2000, 1500, -6, 6),
    (5, 3000, 4100, [0, -2, -3, 0, -1], [9, 7, 5, 11, 3]),
    (7, 1200, 900, -2, 3),
    (2, 20000, 300, [-5000, -3], [5000, 4]),      # radix-sorted operand
]


@pytest.mark.parametrize("case", range(len(POLY_CASES)))
@pytest.mark.parametrize("dtype", ["i64", "f64"])
def test_random_poly(kron, case, dtype):
    v, nf, ng, lo, hi = POLY_CASES[case]
    f = random_poly(v, nf, lo, hi, 1000 + case, dtype)
    g = random_poly(v, ng, lo, hi, 2000 + case, dtype)
    r = oracle.poly_mul(f, g, nthreads=NT, keep_zero=(dtype == "f64"))
    for path in (kron.KR_PATH_AUTO, kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        for device_inputs in (True, False):
            try:
                ex, cf = run_poly(kron, f, g, device_inputs, path=path)
            except kron.KronError as e:
                if e.status == kron.KR_ERR_INVALID and path == kron.KR_PATH_DENSE:
                    continue   # code range too large for a dense array
                raise
            what = f"case {case} {dtype} path={path} dev={device_inputs}"
            if dtype == "i64":
                assert_poly_equal(ex, cf, r, what)
            else:
                assert_poly_close(ex, cf, r, REL, what)


PS_CASES = [
    # npoly, ntrig, nf, ng, prange, trange
    (0, 1, 1, 1, 0, 3),
    (1, 1, 40, 33, 3, 5),
    (2, 3, 700, 1100, 3, 4),
    (3, 4, 3000, 2500, 4, 8),
    (1, 6, 1500, 1700, 2, 2),
]


@pytest.mark.parametrize("case", range(len(PS_CASES)))
def test_random_pseries(kron, case):
    np_, nt, nf, ng, pr, tr = PS_CASES[case]
    f = random_pseries(np_, nt, nf, pr, tr, 3000 + case)
    g = random_pseries(np_, nt, ng, pr, tr, 4000 + case)
    r = oracle.poisson_mul(f, g, nthreads=NT, keep_zero=True)
    for path in (kron.KR_PATH_AUTO, kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        for device_inputs in (True, False):
            out = run_pseries(kron, f, g, device_inputs, path=path)
            assert_pseries_close(out, r, REL, f"pseries case {case} path={path} dev={device_inputs}")


def test_werner_special_cases_on_gpu(kron):
    """t_g = 0, t_f = t_g, and non-canonical sums/differences through the hash path."""
    f = PSeries(np.array([[0, 1, -1, 2]], np.int32), np.array([[1, 1, 2, 0], [1, 0, 1, 1]], np.int32),
                np.array([0, 1, 0, 1], np.uint8), np.array([2.0, -3.0, 0.5, 7.0]))
    g = PSeries(np.array([[3, -1, 0]], np.int32), np.array([[0, 1, 1], [0, 0, 1]], np.int32),
                np.array([0, 1, 1], np.uint8), np.array([5.0, 11.0, -13.0]))
    r = oracle.poisson_mul(f, g, keep_zero=True)
    out = run_pseries(kron, f, g)
    assert_pseries_close(out, r, REL, "werner special")


# ---------------------------------------------------------------------------
# path independence, capacity contract, regrowth, errors, coding entry points
# ---------------------------------------------------------------------------

def test_dense_equals_hash_bit_exact(kron):
    for s in range(3):
        f = random_poly(4, 1500 + 97 * s, -7, 7, 50 + s)
        g = random_poly(4, 1300 + 31 * s, -7, 7, 60 + s)
        a = run_poly(kron, f, g, path=kron.KR_PATH_DENSE)
        b = run_poly(kron, f, g, path=kron.KR_PATH_HASH)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_capacity_two_phase(kron):
    import ctypes
    from paper_1004_4548_gb300 import binding as B
    f = random_poly(3, 300, -4, 4, 71)
    g = random_poly(3, 200, -4, 4, 72)
    r = oracle.poly_mul(f, g)
    ctx = kron.context()
    cap = 5
    F = B.kr_poly(3, f.n, f.exps.ctypes.data, f.coef.ctypes.data, 0)
    G = B.kr_poly(3, g.n, g.exps.ctypes.data, g.coef.ctypes.data, 0)
    ex = np.zeros((3, cap), np.int32); cf = np.zeros(cap, np.int64)
    H = B.kr_poly_out(3, cap, 0, ex.ctypes.data, cf.ctypes.data, None)
    st = ctx.L.poly_mul(ctx.h, ctypes.byref(F), ctypes.byref(G), ctypes.byref(H), None, None)
    assert st == kron.KR_ERR_CAPACITY and H.nterms == r.coef.shape[0]
    n = int(H.nterms)
    ex = np.zeros((3, n), np.int32); cf = np.zeros(n, np.int64)
    H = B.kr_poly_out(3, n, 0, ex.ctypes.data, cf.ctypes.data, None)
    assert ctx.L.kron_fetch_poly(ctx.h, ctypes.byref(H), None) == kron.KR_OK
    assert_poly_equal(ex, cf, r, "two-phase fetch")


def test_table_full_regrows(kron):
    f, g = workload_cfg3()
    f = Poly(f.exps[:, :1500].copy(), f.coef[:1500].copy())
    g = Poly(g.exps[:, :1500].copy(), g.coef[:1500].copy())
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert r.coef.shape[0] > 4096
    ex, cf = run_poly(kron, f, g, path=kron.KR_PATH_HASH, table_slots=4096, probe_limit=64)
    assert_poly_equal(ex, cf, r, "after regrowth")
    ex, cf = run_poly(kron, f, g, path=kron.KR_PATH_HASH, table_slots=1024, probe_limit=64, max_regrow=2)
    assert_poly_equal(ex, cf, r, "after two regrowths")
    with pytest.raises(kron.KronError) as e:
        run_poly(kron, f, g, path=kron.KR_PATH_HASH, table_slots=4096, probe_limit=64, max_regrow=-1)
    assert e.value.status == kron.KR_ERR_TABLE_FULL


def test_large_table_regrows_and_float64(kron):
    """Forced down to 2^20 slots, the MP-sparse product's 5.8 M keys overfill
    the table: it grows until they fit, and the result is still exact.  A
    float64 product with millions of output terms (a table far larger than
    L2) matches within the tolerance."""
    f, g = workload_cfg3()
    r = oracle.poly_mul(f, g, nthreads=NT)
    ex, cf = run_poly(kron, f, g, path=kron.KR_PATH_HASH, table_slots=1 << 20)
    assert_poly_equal(ex, cf, r, "MP-sparse after regrowth")
    f = random_poly(5, 3000, -20, 20, 5500, "f64")
    g = random_poly(5, 2800, -20, 20, 5501, "f64")
    r = oracle.poly_mul(f, g, nthreads=NT, keep_zero=True)
    assert r.coef.shape[0] > 4_000_000
    ex, cf = run_poly(kron, f, g, path=kron.KR_PATH_HASH)
    assert_poly_close(ex, cf, r, REL, "large float64 hash product")


def test_error_statuses(kron):
    f = random_poly(2, 50, -3, 3, 81)
    dup = Poly(np.concatenate([f.exps, f.exps[:, :1]], axis=1), np.concatenate([f.coef, f.coef[:1]]))
    with pytest.raises(kron.KronError) as e:
        run_poly(kron, dup, f)
    assert e.value.status == kron.KR_ERR_DUP
    big = Poly(np.array([[0, 1 << 22], [0, 1 << 22], [0, 1 << 22]], np.int32), np.array([1, 2], np.int64))
    with pytest.raises(kron.KronError) as e:
        run_poly(kron, big, big)
    assert e.value.status == kron.KR_ERR_OVERFLOW
    p = random_pseries(1, 2, 20, 2, 3, 82)
    bad = PSeries(p.exps.copy(), p.trig.copy(), p.kind.copy(), p.coef.copy())
    bad.trig[:, 0] = [0, -1]   # highest-index multiplier negative: not canonical
    with pytest.raises(kron.KronError) as e:
        run_pseries(kron, bad, p)
    assert e.value.status == kron.KR_ERR_INVALID


def test_empty_and_single_terms(kron):
    f = random_poly(3, 10, -2, 2, 91)
    e = Poly(np.zeros((3, 0), np.int32), np.zeros(0, np.int64))
    ex, cf, _, _ = kron.poly_mul(e.exps, e.coef, f.exps, f.coef, host_out=True)
    assert to_np(cf).shape[0] == 0
    one = Poly(np.array([[1], [-2], [0]], np.int32), np.array([3], np.int64))
    r = oracle.poly_mul(one, f)
    assert_poly_equal(*run_poly(kron, one, f), r, "single term")


def test_encode_decode_roundtrip(kron):
    rows = [list(map(int, l.split())) for l in open(os.path.join(os.path.dirname(__file__),
            "golden", "table1_codes.txt")) if l.strip() and not l.startswith("#")]
    exps = np.array([[x for z, y, x, c in rows], [y for z, y, x, c in rows], [z for z, y, x, c in rows]],
                    np.int32)
    codes = to_np(kron.kron_encode(dev(exps), [0, 0, 0], [3, 3, 3]))
    assert list(codes) == [c for *_, c in rows]
    back = to_np(kron.kron_decode(dev(codes), [0, 0, 0], [3, 3, 3]))
    assert np.array_equal(back, exps)
    # exhaustive round trip on a Laurent box, host buffers
    lo, hi = np.array([-3, 2, -1, 0], np.int32), np.array([1, 5, 4, 2], np.int32)
    grid = np.stack(np.meshgrid(*[np.arange(a, b + 1) for a, b in zip(lo, hi)], indexing="ij"), 0)
    allp = grid.reshape(4, -1).astype(np.int32)
    c = to_np(kron.kron_encode(allp, lo, hi))
    assert np.array_equal(np.sort(c), np.arange(allp.shape[1]))
    assert np.array_equal(to_np(kron.kron_decode(c, lo, hi)), allp)
    with pytest.raises(kron.KronError) as e:
        kron.kron_encode(allp, lo, hi - 1)
    assert e.value.status == kron.KR_ERR_RANGE


def test_peak_probes_report_rates(kron):
    """The roofline denominators: positive chip-wide rates, and the int64
    accumulate in two 32-bit atomics no slower than one 64-bit atomic add."""
    r64 = kron.kr_probe_smem_atomic_rate(0, False, 2)
    rsplit = kron.kr_probe_smem_accumulate_rate(0, 2)
    assert r64 > 1e10 and rsplit > 1e10
    assert rsplit > 0.8 * r64
    # the hash path's ceiling: random insert-or-adds and plain adds in a 2^22-slot table
    ins = kron.kr_probe_table_update_rate(22, 1 << 20, 1 << 23, 0, 0, 2)
    add = kron.kr_probe_table_update_rate(22, 1 << 20, 1 << 23, 1, 0, 2)
    assert ins > 1e9 and add > 1e9
    assert kron.kr_probe_table_update_rate(22, 1 << 22, 1 << 23, 0, 0, 1) < 0   # load above 0.7 refused
    # float64 adds into an 8-byte-slot array (the Poisson dense path's ceiling); 2^31 slots
    # only in this mode, and no fourth mode
    assert kron.kr_probe_table_update_rate(24, 1 << 22, 1 << 23, 2, 0, 2) > 1e9
    assert kron.kr_probe_table_update_rate(31, 1 << 20, 1 << 20, 0, 0, 1) < 0
    assert kron.kr_probe_table_update_rate(22, 1 << 20, 1 << 20, 3, 0, 1) < 0
    # multiply-add rates: the 32 x 32 -> 64-bit form no slower than the 64-bit one
    r0, r1, r2 = (kron.kr_probe_alu_rate(k, 0, 2) for k in (0, 1, 2))
    assert min(r0, r1, r2) > 1e11 and r1 > 0.8 * r0
    assert kron.kr_probe_alu_rate(3, 0, 1) < 0


def test_bounded_wait_gives_up_and_reports(kron):
    """A look-back wait on a chunk that never publishes ends by itself with
    KR_ERR_TIMEOUT, and the device stays usable for the next product."""
    assert kron.kr_selftest_bounded_wait(0) == kron.KR_ERR_TIMEOUT
    f, g = workload_cfg1()
    r = oracle.poly_mul(f, g)
    ex, cf = run_poly(kron, f, g)
    assert_poly_equal(ex, cf, r, "after the self-test")


# ---------------------------------------------------------------------------
# limits: the most variables, exponents near the int32 ends, code ranges near
# 2^63, int64 wrap on the hash path
# ---------------------------------------------------------------------------

def test_sixteen_variables(kron):
    """KR_MAXV polynomial variables (product width 3 per variable: W = 3^16)."""
    f = random_poly(16, 900, 0, 1, 5100)
    g = random_poly(16, 700, 0, 1, 5101)
    r = oracle.poly_mul(f, g, nthreads=NT)
    for path in (kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        ex, cf = run_poly(kron, f, g, path=path)
        assert_poly_equal(ex, cf, r, f"16 variables path={path}")


def test_poisson_sixteen_variables(kron):
    f = random_pseries(6, 10, 600, 1, 1, 5200)
    g = random_pseries(6, 10, 500, 1, 1, 5201)
    r = oracle.poisson_mul(f, g, nthreads=NT, keep_zero=True)
    for path in (kron.KR_PATH_AUTO, kron.KR_PATH_HASH):
        out = run_pseries(kron, f, g, path=path)
        assert_pseries_close(out, r, REL, f"16 poisson variables path={path}")


def test_exponents_near_int32_ends(kron):
    """Boxes far from the origin: the codes use offsets, the decode restores them."""
    big = (1 << 30) - 20
    f = random_poly(3, 400, [-big, big - 8, 0], [-big + 6, big, 9], 5300)
    g = random_poly(3, 300, [-big, big - 8, -4], [-big + 9, big, 3], 5301)
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert r.exps[0].min() < -(1 << 31) + 100 and r.exps[1].max() > (1 << 31) - 100
    for path in (kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        ex, cf = run_poly(kron, f, g, path=path)
        assert_poly_equal(ex, cf, r, f"int32 ends path={path}")
    # one step further and the product's exponents leave int32
    h = Poly(np.array([[(1 << 30) + 5]], np.int32), np.array([1], np.int64))
    with pytest.raises(kron.KronError) as e:
        run_poly(kron, h, h)
    assert e.value.status == kron.KR_ERR_OVERFLOW


def test_code_range_near_two_to_63(kron):
    """A product whose code range is just below 2^63 (hash path), and one just above."""
    # widths 2^21 - 1 in three variables: W = (2^21 - 1)^3 = 2^63 - 3 * 2^42 + 3 * 2^21 - 1
    hi = (1 << 20) - 1
    f = Poly(np.array([[0, hi, 5, 0], [0, 7, hi, 3], [0, 1, 2, hi]], np.int32), np.array([1, -2, 3, 4], np.int64))
    g = Poly(np.array([[0, hi, 9], [0, 0, hi], [hi, 4, 0]], np.int32), np.array([5, 6, -7], np.int64))
    r = oracle.poly_mul(f, g)
    ex, cf = run_poly(kron, f, g)
    assert_poly_equal(ex, cf, r, "code range near 2^63")
    g2 = Poly(g.exps.copy(), g.coef.copy())
    g2.exps[0, 0] = -4   # w_0 = 2^21 + 3: the range passes 2^63 - 1
    with pytest.raises(kron.KronError) as e:
        run_poly(kron, f, g2)
    assert e.value.status == kron.KR_ERR_OVERFLOW


def test_int64_wrap_on_hash_path(kron):
    """Sums beyond int64 wrap modulo 2^64 on the hash path as on the dense path."""
    rng = Rng(5400)
    f = random_poly(3, 300, -2, 2, 5401)
    g = random_poly(3, 250, -2, 2, 5402)
    f.coef[:] = rng.ints(1 << 61, (1 << 62) - 1, f.n)
    g.coef[:] = rng.ints(-(1 << 62), -(1 << 61), g.n)
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert r.overflow
    for path in (kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
        ex, cf = run_poly(kron, f, g, path=path)
        assert_poly_equal(ex, cf, r, f"wrap path={path}")
