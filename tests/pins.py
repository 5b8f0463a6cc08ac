"""Independent checks ("pins") for the oracle: textbook routines that reach the
product by a different road than the oracle's ordered map.

* ``box_convolution``: direct N-dimensional convolution of dense coefficient
  boxes (the product of polynomials is the convolution of their coefficient
  arrays; Laurent exponents are shifted into the box first).
* ``eval_mod_p`` / ``eval_mod_m31``: evaluation at a point modulo a prime
  (Schwartz-Zippel: distinct polynomials agree at a random point with
  probability <= degree / p).
* ``eval_pseries``: evaluation of a Poisson series at real x and angles y.
* ``eval_truncated_mod_m31`` / ``eval_truncated_pseries``: the value of the
  part of f*g of degree <= N, reached from f and g alone: the degree of a
  product term is the sum of its factors' degrees, so that part is the sum of
  the products of f's and g's degree-homogeneous parts whose degrees add up
  to at most N.
"""
from __future__ import annotations

import numpy as np

M61 = (1 << 61) - 1
M31 = (1 << 31) - 1


def box_convolution(f, g):
    """{exponent tuple: coefficient} of f*g by dense N-d convolution (nonzeros only)."""
    v = f.exps.shape[0]
    fmin, gmin = f.exps.min(axis=1), g.exps.min(axis=1)
    fdim = f.exps.max(axis=1) - fmin + 1
    gdim = g.exps.max(axis=1) - gmin + 1
    dt = f.coef.dtype
    G = np.zeros(tuple(gdim), dtype=dt)
    G[tuple(g.exps - gmin[:, None])] = g.coef
    out = np.zeros(tuple(fdim + gdim - 1), dtype=dt)
    fpos = (f.exps - fmin[:, None]).T
    for p, c in zip(fpos, f.coef):
        sl = tuple(slice(int(p[k]), int(p[k]) + int(gdim[k])) for k in range(v))
        out[sl] += c * G
    nz = np.nonzero(out)
    base = fmin + gmin
    keys = np.stack(nz, axis=1) + base
    return {tuple(int(x) for x in k): out[i] for k, i in zip(keys, zip(*nz))}


def as_dict(exps: np.ndarray, coef: np.ndarray):
    return {tuple(int(x) for x in exps[:, i]): coef[i] for i in range(coef.shape[0])}


def eval_mod_p(exps: np.ndarray, coef: np.ndarray, point, p: int = M61) -> int:
    """sum_i coef_i * prod_k x_k^e_ik mod p, exact (Python integers)."""
    inv = [pow(int(x), p - 2, p) for x in point]
    total = 0
    for i in range(coef.shape[0]):
        t = int(coef[i]) % p
        for k, x in enumerate(point):
            e = int(exps[k, i])
            t = t * (pow(int(x), e, p) if e >= 0 else pow(inv[k], -e, p)) % p
        total = (total + t) % p
    return total


def eval_mod_m31(exps: np.ndarray, coef: np.ndarray, point) -> int:
    """Vectorised evaluation modulo 2^31 - 1 (every product fits in 62 bits)."""
    p = M31
    acc = (coef.astype(np.int64) % p).astype(np.uint64)
    for k, x in enumerate(point):
        e = exps[k].astype(np.int64)
        lo, hi = int(e.min()), int(e.max())
        xi = pow(int(x), p - 2, p)
        table = np.array([pow(int(x), t, p) if t >= 0 else pow(xi, -t, p)
                          for t in range(lo, hi + 1)], dtype=np.uint64)
        acc = (acc * table[e - lo]) % np.uint64(p)
    # sum in chunks to stay below 2^64
    s = 0
    for c in np.array_split(acc, max(1, acc.shape[0] // (1 << 20))):
        s = (s + int(c.sum())) % p
    return s


def eval_pseries(s, x: np.ndarray, y: np.ndarray):
    """(value, magnitude) of a Poisson series at x (real, > 0) and angles y."""
    mono = np.prod(x[:, None] ** s.exps.astype(np.float64), axis=0)
    phase = (s.trig.astype(np.float64) * y[:, None]).sum(axis=0)
    trig = np.where(s.kind == 0, np.cos(phase), np.sin(phase))
    terms = s.coef * mono * trig
    return float(terms.sum()), float(np.abs(s.coef * mono).sum())


def degrees(exps: np.ndarray, mask: int) -> np.ndarray:
    """Degree of every term in the variables of the bit mask (0 = all)."""
    v = exps.shape[0]
    m = mask if mask else (1 << v) - 1
    rows = [k for k in range(v) if (m >> k) & 1]
    return exps[rows].astype(np.int64).sum(axis=0)


def eval_truncated_mod_m31(f, g, point, mask: int, N: int) -> int:
    """Value modulo 2^31 - 1 of the degree <= N part of f*g at `point`."""
    df, dg = degrees(f.exps, mask), degrees(g.exps, mask)
    F = {int(d): eval_mod_m31(f.exps[:, df == d], f.coef[df == d], point) for d in np.unique(df)}
    G = {int(d): eval_mod_m31(g.exps[:, dg == d], g.coef[dg == d], point) for d in np.unique(dg)}
    return sum(a * b for d1, a in F.items() for d2, b in G.items() if d1 + d2 <= N) % M31


def eval_truncated_pseries(f, g, x: np.ndarray, y: np.ndarray, mask: int, N: int):
    """(value, magnitude) of the part of f*g whose polynomial degree is <= N."""
    df, dg = degrees(f.exps, mask), degrees(g.exps, mask)
    val, mag = 0.0, 0.0
    for d1 in np.unique(df):
        sf = type(f)(f.exps[:, df == d1], f.trig[:, df == d1], f.kind[df == d1], f.coef[df == d1])
        a, am = eval_pseries(sf, x, y)
        for d2 in np.unique(dg):
            if d1 + d2 > N:
                continue
            sg = type(g)(g.exps[:, dg == d2], g.trig[:, dg == d2], g.kind[dg == d2], g.coef[dg == d2])
            b, bm = eval_pseries(sg, x, y)
            val += a * b
            mag += am * bm
    return val, mag


def eval_poly_real(exps: np.ndarray, coef: np.ndarray, x: np.ndarray):
    """(value, magnitude) of a float64 polynomial at the real point x (x > 0)."""
    mono = np.prod(x[:, None] ** exps.astype(np.float64), axis=0)
    return float((coef * mono).sum()), float(np.abs(coef * mono).sum())


def powers_of_ten(p, levels: np.ndarray, rng):
    """A copy of p whose coefficients are +-10^-level * (1 + u / 10), u in [0, 1):
    the magnitude of a product of two such coefficients lies in
    [10^-(a+b), 1.21 * 10^-(a+b)), so |C_f C_g| >= 0.5 * 10^-N exactly when
    a + b <= N, whatever the rounding."""
    mag = 10.0 ** (-levels.astype(np.float64)) * (1.0 + 0.1 * rng.uniform(levels.shape[0]))
    c = np.where(p.coef < 0, -mag, mag)
    if hasattr(p, "trig"):
        return type(p)(p.exps, p.trig, p.kind, c)
    return type(p)(p.exps, c)


def eval_level_truncated(f, g, lf, lg, N, evaluate):
    """(value, magnitude) of sum over level pairs with a + b <= N of F_a * G_b:
    the product keeping the pairs with a + b <= N, reached from f and g alone."""
    val, mag = 0.0, 0.0
    for a in np.unique(lf):
        va, ma = evaluate(f, lf == a)
        for b in np.unique(lg):
            if a + b > N:
                continue
            vb, mb = evaluate(g, lg == b)
            val += va * vb
            mag += ma * mb
    return val, mag


def sample_grid(s, x: np.ndarray, M: int) -> np.ndarray:
    """Values of a Poisson series with two trig variables at the real point x
    on the M x M grid of angles y = 2 pi (m1, m2) / M."""
    grid = 2.0 * np.pi * np.arange(M) / M
    y1, y2 = np.meshgrid(grid, grid, indexing="ij")
    mono = np.prod(x[:, None] ** s.exps.astype(np.float64), axis=0)
    vals = np.zeros((M, M))
    for i in range(s.coef.shape[0]):
        ph = s.trig[0, i] * y1 + s.trig[1, i] * y2
        vals += s.coef[i] * mono[i] * (np.cos(ph) if s.kind[i] == 0 else np.sin(ph))
    return vals


def fourier_coefficients(vals: np.ndarray) -> np.ndarray:
    """Complex Fourier coefficients c_k of grid samples of a trig polynomial,
    S(y) = sum_k c_k exp(i k.y), by the 2-D FFT: c_k = FFT[k mod M] / M^2
    (exact for |k_m| < M / 2)."""
    return np.fft.fft2(vals) / vals.size
