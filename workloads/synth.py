"""Seeded generators for the benchmark workloads and for random test cases.

Term layout everywhere (the layout the library boundary takes):

* ``Poly``: ``exps`` int32 array of shape ``[nvars, n]`` (structure of arrays,
  one row per variable), ``coef`` int64 or float64 of shape ``[n]``.
* ``PSeries`` (Poisson series, one term = C * x^a * cos|sin(j . y)):
  ``exps`` int32 ``[npoly, n]``, ``trig`` int32 ``[ntrig, n]``, ``kind`` uint8
  ``[n]`` (0 = cos, 1 = sin), ``coef`` float64 ``[n]``.  Inputs are valid
  series: trig multiplier vectors are in canonical sign (the highest-index
  nonzero multiplier is positive), a sine never has the zero multiplier vector,
  and no two terms share (exps, trig, kind).

Terms are emitted in a seeded random order: sorting them is part of the
multiplication pipeline, not of the input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class Rng:
    """Counter-based SplitMix64: output k (k = 1, 2, ...) is mix(seed + k*gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.seed + k * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def ints(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (int64); modulo bias < 2^-40 for the ranges used."""
        span = np.uint64(hi - lo + 1)
        return (self.u64(n) % span).astype(np.int64) + lo

    def nonzero_ints(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] without 0 (lo <= 0 <= hi)."""
        u = self.ints(lo, hi - 1, n)
        return np.where(u >= 0, u + 1, u)

    def uniform(self, n: int) -> np.ndarray:
        """Uniform doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def perm(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")


@dataclass
class Poly:
    exps: np.ndarray      # int32 [nvars, n]
    coef: np.ndarray      # int64 or float64 [n]

    @property
    def nvars(self) -> int:
        return int(self.exps.shape[0])

    @property
    def n(self) -> int:
        return int(self.coef.shape[0])


@dataclass
class PSeries:
    exps: np.ndarray      # int32 [npoly, n]
    trig: np.ndarray      # int32 [ntrig, n]
    kind: np.ndarray      # uint8 [n], 0 = cos, 1 = sin
    coef: np.ndarray      # float64 [n]

    @property
    def npoly(self) -> int:
        return int(self.exps.shape[0])

    @property
    def ntrig(self) -> int:
        return int(self.trig.shape[0])

    @property
    def n(self) -> int:
        return int(self.coef.shape[0])


def total_degree_tuples(v: int, D: int) -> np.ndarray:
    """All nonnegative integer v-tuples with sum <= D, shape [count, v]."""
    rows = np.zeros((1, 0), dtype=np.int32)
    for _ in range(v):
        room = D - rows.sum(axis=1)
        reps = room + 1
        base = np.repeat(rows, reps, axis=0)
        starts = np.repeat(np.cumsum(reps) - reps, reps)
        col = (np.arange(base.shape[0]) - starts).astype(np.int32)
        rows = np.concatenate([base, col[:, None]], axis=1)
    return rows


def _soa(rows: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(rows.T.astype(np.int32))


def dense_total_degree(v: int, D: int, coef_lo: int, coef_hi: int, seed: int) -> Poly:
    """All monomials of total degree <= D in v variables, nonzero int64 coefficients."""
    rng = Rng(seed)
    rows = total_degree_tuples(v, D)
    rows = rows[rng.perm(rows.shape[0])]
    coef = rng.nonzero_ints(coef_lo, coef_hi, rows.shape[0])
    return Poly(_soa(rows), coef)


def mp_sparse(side: str, D: int, coef_lo: int, coef_hi: int, seed: int) -> Poly:
    """Monagan-Pearce sparse structure: one term per (a,b,c,d,e) with sum <= D.

    f: x^a y^b z^(2c) t^(3d) u^(5e);  g: x^(5a) y^(3b) z^(2c) t^d u^e.
    """
    w = {"f": (1, 1, 2, 3, 5), "g": (5, 3, 2, 1, 1)}[side]
    rng = Rng(seed)
    rows = total_degree_tuples(5, D) * np.asarray(w, dtype=np.int32)
    rows = rows[rng.perm(rows.shape[0])]
    coef = rng.nonzero_ints(coef_lo, coef_hi, rows.shape[0])
    return Poly(_soa(rows), coef)


def _canonical_mask(trig_rows: np.ndarray) -> np.ndarray:
    """True where the highest-index nonzero multiplier is positive (input validity)."""
    nz = trig_rows != 0
    any_nz = nz.any(axis=1)
    last = trig_rows.shape[1] - 1 - np.argmax(nz[:, ::-1], axis=1)
    lastval = trig_rows[np.arange(trig_rows.shape[0]), last]
    return any_nz & (lastval > 0)


def poisson_random(n: int, npoly: int, ntrig: int, prange: int, trange: int,
                   seed: int, mag: str = "norm") -> PSeries:
    """n distinct Poisson terms, exponents U[-prange, prange], multipliers U[-trange, trange].

    Invalid draws (non-canonical multiplier vector, sine of the zero vector) and
    repeated keys are rejected.  mag="norm": |C| = 10^-(|i|_1 + |j|_1) * 10^u,
    u ~ U[0, 1), random sign.
    """
    rng = Rng(seed)
    keep_p, keep_t, keep_k = [], [], []
    have = 0
    while have < n:
        m = max(2 * (n - have), 1024)
        p = rng.ints(-prange, prange, m * npoly).reshape(m, npoly).astype(np.int32)
        t = rng.ints(-trange, trange, m * ntrig).reshape(m, ntrig).astype(np.int32)
        k = (rng.u64(m) >> np.uint64(63)).astype(np.uint8)
        zero = ~(t != 0).any(axis=1)
        ok = _canonical_mask(t) | (zero & (k == 0))
        keep_p.append(p[ok]); keep_t.append(t[ok]); keep_k.append(k[ok])
        P = np.concatenate(keep_p); T = np.concatenate(keep_t); K = np.concatenate(keep_k)
        key = np.concatenate([P, T, K[:, None].astype(np.int32)], axis=1)
        _, first = np.unique(key, axis=0, return_index=True)
        first = np.sort(first)
        keep_p, keep_t, keep_k = [P[first]], [T[first]], [K[first]]
        have = first.shape[0]
    P, T, K = keep_p[0][:n], keep_t[0][:n], keep_k[0][:n]
    sign = np.where((rng.u64(n) >> np.uint64(63)) == 1, -1.0, 1.0)
    u = rng.uniform(n)
    if mag == "norm":
        l1 = np.abs(P).sum(axis=1) + np.abs(T).sum(axis=1)
        coef = sign * 10.0 ** (u - l1)
    else:
        coef = sign * (0.5 + u)
    return PSeries(_soa(P), _soa(T), np.ascontiguousarray(K), coef.astype(np.float64))


def dense_box(lo, hi, keep: float, coef_lo: int, coef_hi: int, seed: int) -> Poly:
    """The monomials of the box lo <= e <= hi (variable 0 fastest), each kept
    with probability keep; nonzero int64 coefficients uniform in [coef_lo, coef_hi].
    Long runs of consecutive exponents of variable 0, broken where a monomial
    was dropped."""
    rng = Rng(seed)
    lo = [int(x) for x in lo]
    hi = [int(x) for x in hi]
    axes = [np.arange(a, b + 1, dtype=np.int64) for a, b in zip(lo, hi)]
    grid = np.stack(np.meshgrid(*axes[::-1], indexing="ij")[::-1], axis=-1).reshape(-1, len(lo))
    if keep < 1.0:
        grid = grid[rng.uniform(grid.shape[0]) < keep]
    coef = rng.nonzero_ints(coef_lo, coef_hi, grid.shape[0])
    perm = rng.perm(grid.shape[0])
    return Poly(_soa(grid[perm].astype(np.int32)), coef[perm])


def random_poly(nvars: int, n: int, lo, hi, seed: int, dtype="i64",
                coef_range=(-1000, 1000)) -> Poly:
    """n distinct random monomials, exponent k uniform in [lo[k], hi[k]]."""
    rng = Rng(seed)
    lo = np.broadcast_to(np.asarray(lo, dtype=np.int64), (nvars,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.int64), (nvars,))
    box = int(np.prod((hi - lo + 1).astype(np.float64)))
    n = min(n, box)
    rows = np.zeros((0, nvars), dtype=np.int32)
    while rows.shape[0] < n:
        m = 2 * (n - rows.shape[0]) + 16
        cols = [rng.ints(int(lo[k]), int(hi[k]), m) for k in range(nvars)]
        cand = np.stack(cols, axis=1).astype(np.int32)
        allr = np.concatenate([rows, cand])
        _, first = np.unique(allr, axis=0, return_index=True)
        rows = allr[np.sort(first)]
    rows = rows[:n]
    if dtype == "i64":
        coef = rng.nonzero_ints(coef_range[0], coef_range[1], n)
    else:
        sign = np.where((rng.u64(n) >> np.uint64(63)) == 1, -1.0, 1.0)
        coef = sign * (0.25 + rng.uniform(n))
    return Poly(_soa(rows), coef)


def random_pseries(npoly: int, ntrig: int, n: int, prange: int, trange: int,
                   seed: int) -> PSeries:
    return poisson_random(n, npoly, ntrig, prange, trange, seed, mag="unit")


# ----------------------------------------------------------------------------
# The five benchmark workloads.
# ----------------------------------------------------------------------------

def workload_cfg1():
    """Dense path, tiny: 4 vars, all monomials of degree <= 10, coef U[-100,100]\\{0}."""
    return (dense_total_degree(4, 10, -100, 100, 1001),
            dense_total_degree(4, 10, -100, 100, 1002))


def workload_cfg2():
    """Dense path, moderately sparse: degree <= 20 (10626 terms), coef U[-2^20, 2^20]\\{0}."""
    return (dense_total_degree(4, 20, -(1 << 20), 1 << 20, 2001),
            dense_total_degree(4, 20, -(1 << 20), 1 << 20, 2002))


def workload_cfg3():
    """Hash path: Monagan-Pearce sparse structure, degree 12 (6188 terms), coef U[-1000,1000]\\{0}."""
    return (mp_sparse("f", 12, -1000, 1000, 3001),
            mp_sparse("g", 12, -1000, 1000, 3002))


def workload_cfg4(n: int = 20000):
    """Poisson series: 3 poly vars in [-4,4], 4 trig vars in [-8,8], n terms per operand."""
    return (poisson_random(n, 3, 4, 4, 8, 4001),
            poisson_random(n, 3, 4, 4, 8, 4002))


def fateman(power: int = 30, seed: int = 6001):
    """Fateman's benchmark operands: f = (1 + x + y + z + t)^power, g = f + 1.

    The coefficients are the multinomial coefficients of the expansion, reduced
    modulo 2^64 into int64 (the library's integer arithmetic wraps modulo 2^64).
    Terms in a seeded random order.
    """
    rows = total_degree_tuples(4, power)
    # multinomial coefficient power! / (a! b! c! d! e!) with e = power - a - b - c - d
    fact = [1]
    for k in range(1, power + 1):
        fact.append(fact[-1] * k)
    coef = []
    for a, b, c, d in rows.tolist():
        e = power - a - b - c - d
        m = fact[power] // (fact[a] * fact[b] * fact[c] * fact[d] * fact[e])
        m %= 1 << 64
        coef.append(m - (1 << 64) if m >= 1 << 63 else m)
    coef = np.array(coef, dtype=np.int64)
    gcoef = coef.copy()
    zero = np.nonzero((rows == 0).all(axis=1))[0][0]
    gcoef[zero] = np.int64((int(gcoef[zero]) + 1 + (1 << 63)) % (1 << 64) - (1 << 63))
    rng = Rng(seed)
    pf, pg = rng.perm(rows.shape[0]), rng.perm(rows.shape[0])
    return Poly(_soa(rows[pf]), coef[pf]), Poly(_soa(rows[pg]), gcoef[pg])


def _batch_operand(rng: Rng, v: int, poisson: bool):
    lo, hi = math.log(50.0), math.log(20000.0)
    n = int(round(math.exp(lo + (hi - lo) * float(rng.uniform(1)[0]))))
    weighted = bool(rng.u64(1)[0] >> np.uint64(63))
    D = 20
    for d in range(4, 21):
        if math.comb(v + d, v) >= n:
            D = d
            break
    n = min(n, math.comb(v + D, v))
    rows = total_degree_tuples(v, D)
    rows = rows[rng.perm(rows.shape[0])[:n]]
    if weighted:
        w = np.asarray([1, 2, 3, 5], dtype=np.int32)[rng.ints(0, 3, v)]
        rows = rows * w
        emax = D * w
    else:
        emax = np.full(v, D, dtype=np.int32)
    if not poisson:
        coef = rng.nonzero_ints(-1000, 1000, n)
        return Poly(_soa(rows), coef)
    npoly = v - v // 2
    P = rows[:, :npoly] - (emax[:npoly] // 2)
    T = rows[:, npoly:].copy()
    nt = T.shape[1]
    # random signs on every multiplier except the highest-index nonzero one,
    # which stays positive: the vectors are then valid (canonical) inputs
    nz = T != 0
    last = nt - 1 - np.argmax(nz[:, ::-1], axis=1)
    sgn = np.where(rng.ints(0, 1, n * nt).reshape(n, nt) == 1, -1, 1).astype(np.int32)
    sgn[np.arange(n), last] = 1
    T = T * sgn
    K = (rng.u64(n) >> np.uint64(63)).astype(np.uint8)
    K[~nz.any(axis=1)] = 0
    sign = np.where((rng.u64(n) >> np.uint64(63)) == 1, -1.0, 1.0)
    l1 = np.abs(P).sum(axis=1) + np.abs(T).sum(axis=1)
    coef = sign * 10.0 ** (rng.uniform(n) - l1 / max(D, 1))
    return PSeries(_soa(P), _soa(T), K, coef.astype(np.float64))


def batch_mix(nprod: int = 4096, seed_base: int = 5000, max_terms: int | None = None):
    """The uneven batch: product k uses seed seed_base + k.

    Even k: int64 polynomial product; odd k: float64 Poisson series product.
    Per product: v ~ U{2..6}; per operand: n ~ logU[50, 20000], dense or
    weighted (weights from {1,2,3,5}) total-degree structure with p = 1/2, D the
    smallest degree in [4, 20] with C(v+D, v) >= n, a seeded n-subset of the
    degree-D tuples.  Poisson operands use v - v//2 polynomial variables
    (shifted to signed exponents) and v//2 trig multipliers (random signs,
    canonical).  max_terms truncates operands (for small test batches).
    """
    out = []
    for k in range(nprod):
        rng = Rng(seed_base + k)
        v = int(rng.ints(2, 6, 1)[0])
        poisson = (k % 2) == 1
        f = _batch_operand(rng, v, poisson)
        g = _batch_operand(rng, v, poisson)
        if max_terms is not None:
            f, g = _truncate(f, max_terms), _truncate(g, max_terms)
        out.append((f, g))
    return out


def _truncate(p, m):
    if p.n <= m:
        return p
    if isinstance(p, Poly):
        return Poly(np.ascontiguousarray(p.exps[:, :m]), p.coef[:m].copy())
    return PSeries(np.ascontiguousarray(p.exps[:, :m]), np.ascontiguousarray(p.trig[:, :m]),
                   p.kind[:m].copy(), p.coef[:m].copy())


def arrival_times(n: int, rate: float, seed: int) -> np.ndarray:
    """Poisson-process arrival times (seconds) for n requests at `rate` per second."""
    u = Rng(seed).uniform(n)
    return np.cumsum(-np.log1p(-u) / rate)
