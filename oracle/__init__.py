"""Oracle for sparse Laurent polynomial and Poisson series multiplication.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does, and it
imports nothing from the library.  The arithmetic lives in ``oracle.cpp`` (a
plain std::map multiplier over explicit exponent vectors; no Kronecker codes),
compiled here with g++ on first use.

Results come back in the library's canonical order (variable 0 least
significant; Poisson keys ordered by kind, trig multipliers, exponents).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.cpp")
_libs: dict[int, ctypes.CDLL] = {}
_lock = threading.Lock()


def build(plant: int = 0) -> str:
    """Compile oracle.cpp (plant > 0: a variant with planted mistake `plant`)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liborc.so" if plant == 0 else f"liborc_plant{plant}.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               f"-DORC_PLANT={plant}", "-o", tmp, _SRC])
        os.replace(tmp, out)
    return out


def _lib(plant: int = 0) -> ctypes.CDLL:
    with _lock:
        if plant not in _libs:
            L = ctypes.CDLL(build(plant))
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.orc_poly_mul.restype = vp
            L.orc_poly_mul.argtypes = [i32, i64, vp, vp, i64, vp, vp, i32, i32, i64, i64, i32]
            L.orc_poisson_mul.restype = vp
            L.orc_poisson_mul.argtypes = [i32, i32, i64, vp, vp, vp, vp, i64, vp, vp, vp, vp,
                                          i32, i64, i64, i32]
            u32 = ctypes.c_uint32
            L.orc_poly_mul_trunc.restype = vp
            L.orc_poly_mul_trunc.argtypes = L.orc_poly_mul.argtypes + [u32, i64]
            L.orc_poisson_mul_trunc.restype = vp
            L.orc_poisson_mul_trunc.argtypes = L.orc_poisson_mul.argtypes + [u32, i64]
            L.orc_poly_mul_tr.restype = vp
            L.orc_poly_mul_tr.argtypes = L.orc_poly_mul.argtypes + [ctypes.POINTER(OrcTrunc)]
            L.orc_poisson_mul_tr.restype = vp
            L.orc_poisson_mul_tr.argtypes = L.orc_poisson_mul.argtypes + [ctypes.POINTER(OrcTrunc)]
            L.orc_result_nterms.restype = i64
            L.orc_result_nterms.argtypes = [vp]
            L.orc_result_overflow.restype = i32
            L.orc_result_overflow.argtypes = [vp]
            L.orc_result_copy.restype = None
            L.orc_result_copy.argtypes = [vp, vp, vp, vp, vp, vp]
            L.orc_result_free.restype = None
            L.orc_result_free.argtypes = [vp]
            L.orc_key_hash.restype = ctypes.c_uint64
            L.orc_key_hash.argtypes = [vp, i32]
            _libs[plant] = L
        return _libs[plant]


class OrcTrunc(ctypes.Structure):
    """Every truncation criterion at once (oracle.cpp's OrcTrunc)."""
    _fields_ = [("deg_on", ctypes.c_int32), ("deg_mask", ctypes.c_uint32), ("deg_max", ctypes.c_int64),
                ("harm_on", ctypes.c_int32), ("harm_mask", ctypes.c_uint32), ("harm_max", ctypes.c_int64),
                ("coef_on", ctypes.c_int32), ("coef_min", ctypes.c_double)]


def _orc_trunc(trunc, harmonic, coef_min):
    t = OrcTrunc()
    if trunc is not None:
        t.deg_on, t.deg_max, t.deg_mask = 1, int(trunc[0]), int(trunc[1] or 0)
    if harmonic is not None:
        t.harm_on, t.harm_max, t.harm_mask = 1, int(harmonic[0]), int(harmonic[1] or 0)
    if coef_min is not None:
        t.coef_on, t.coef_min = 1, float(coef_min)
    return t


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class PolyResult:
    exps: np.ndarray          # int32 [nvars, n]
    coef: np.ndarray          # int64 or float64 [n]
    mass: np.ndarray | None   # float64 [n]: sum of |contribution| (float64 only)
    overflow: bool            # an int64 sum left the int64 range (value is mod 2^64)


@dataclass
class PSeriesResult:
    exps: np.ndarray          # int32 [npoly, n]
    trig: np.ndarray          # int32 [ntrig, n]
    kind: np.ndarray          # uint8 [n]
    coef: np.ndarray          # float64 [n]
    mass: np.ndarray          # float64 [n]


def _trunc_mask(trunc, nv):
    deg, mask = trunc
    return (int(mask) if mask else (1 << nv) - 1), int(deg)


def poly_mul(f, g, nthreads: int = 1, shard: tuple[int, int] = (1, 0),
             keep_zero: bool = False, plant: int = 0, trunc=None, coef_min=None) -> PolyResult:
    """h = f * g by the definition.  f, g: objects with .exps [v, n] int32, .coef.

    trunc = (N, mask): keep the pairs whose product term has degree <= N in the
    variables of the bit mask (0 = all variables).  coef_min = eps (float64
    coefficients only): keep the pairs with |C_f * C_g| >= eps."""
    L = _lib(plant)
    is_f64 = f.coef.dtype == np.float64
    ef = np.ascontiguousarray(f.exps, dtype=np.int32)
    eg = np.ascontiguousarray(g.exps, dtype=np.int32)
    dt = np.float64 if is_f64 else np.int64
    cf = np.ascontiguousarray(f.coef, dtype=dt)
    cg = np.ascontiguousarray(g.coef, dtype=dt)
    nv = ef.shape[0]
    args = (nv, cf.shape[0], _p(ef), _p(cf), cg.shape[0], _p(eg), _p(cg),
            int(is_f64), nthreads, shard[0], shard[1], int(keep_zero))
    if coef_min is not None:
        t = _orc_trunc(None if trunc is None else _trunc_mask(trunc, nv)[::-1], None, coef_min)
        r = L.orc_poly_mul_tr(*args, ctypes.byref(t))
    elif trunc is None:
        r = L.orc_poly_mul(*args)
    else:
        r = L.orc_poly_mul_trunc(*args, *_trunc_mask(trunc, nv))
    if not r:
        raise ValueError("oracle rejected the arguments")
    try:
        n = L.orc_result_nterms(r)
        exps = np.zeros((nv, n), np.int32)
        coef = np.zeros(n, dt)
        mass = np.zeros(n, np.float64) if is_f64 else None
        L.orc_result_copy(r, _p(exps), None, None, _p(coef), _p(mass) if is_f64 else None)
        return PolyResult(exps, coef, mass, bool(L.orc_result_overflow(r)))
    finally:
        L.orc_result_free(r)


def poisson_mul(f, g, nthreads: int = 1, shard: tuple[int, int] = (1, 0),
                keep_zero: bool = False, plant: int = 0, trunc=None, harmonic=None,
                coef_min=None) -> PSeriesResult:
    """h = f * g for Poisson series, by the product-to-sum identities.

    trunc = (N, mask) truncates by the degree of the polynomial part;
    harmonic = (N, mask) keeps the terms whose harmonic order (sum of
    |multiplier| over the trig variables of mask, 0 = all) is <= N;
    coef_min = eps keeps the pairs with |C_f * C_g| >= eps."""
    L = _lib(plant)
    np_, nt = f.exps.shape[0], f.trig.shape[0]
    a = [np.ascontiguousarray(x) for x in (f.exps.astype(np.int32), f.trig.astype(np.int32),
                                           f.kind.astype(np.uint8), f.coef.astype(np.float64))]
    b = [np.ascontiguousarray(x) for x in (g.exps.astype(np.int32), g.trig.astype(np.int32),
                                           g.kind.astype(np.uint8), g.coef.astype(np.float64))]
    args = (np_, nt, a[3].shape[0], *[_p(x) for x in a], b[3].shape[0],
            *[_p(x) for x in b], nthreads, shard[0], shard[1], int(keep_zero))
    if harmonic is not None or coef_min is not None:
        t = _orc_trunc(None if trunc is None else _trunc_mask(trunc, np_)[::-1], harmonic, coef_min)
        r = L.orc_poisson_mul_tr(*args, ctypes.byref(t))
    elif trunc is None:
        r = L.orc_poisson_mul(*args)
    else:
        r = L.orc_poisson_mul_trunc(*args, *_trunc_mask(trunc, np_))
    if not r:
        raise ValueError("oracle rejected the arguments")
    try:
        n = L.orc_result_nterms(r)
        exps = np.zeros((np_, n), np.int32)
        trig = np.zeros((nt, n), np.int32)
        kind = np.zeros(n, np.uint8)
        coef = np.zeros(n, np.float64)
        mass = np.zeros(n, np.float64)
        L.orc_result_copy(r, _p(exps), _p(trig), _p(kind), _p(coef), _p(mass))
        return PSeriesResult(exps, trig, kind, coef, mass)
    finally:
        L.orc_result_free(r)


def key_hash(comps) -> int:
    """FNV-1a hash of one key as the shard filter computes it."""
    c = np.ascontiguousarray(np.asarray(comps, dtype=np.int32))
    return int(_lib().orc_key_hash(_p(c), c.shape[0]))


def shard_of_keys(keys: np.ndarray, mod: int) -> np.ndarray:
    """Shard index of each row of `keys` (int32 [n, len]) under the oracle's filter.

    Poisson keys are laid out (kind, trig..., poly...); polynomial keys are the
    exponent vector.  Vectorised FNV-1a, so a test can restrict a large result
    to the shard the oracle computed.
    """
    h = np.full(keys.shape[0], 14695981039346656037, dtype=np.uint64)
    prime = np.uint64(1099511628211)
    with np.errstate(over="ignore"):
        for t in range(keys.shape[1]):
            h ^= keys[:, t].astype(np.int64).astype(np.uint32).astype(np.uint64)
            h *= prime
    return (h % np.uint64(mod)).astype(np.int64)
