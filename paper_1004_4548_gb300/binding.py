"""ctypes binding of libkron (include/kron.h).

Argument marshalling only: every step of a multiplication runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; outputs
are torch tensors on the context's device unless host outputs are asked for.
PyTorch supplies device memory and the current stream, nothing else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

KR_MAXV = 16
KR_OK, KR_ERR_INVALID, KR_ERR_RANGE, KR_ERR_OVERFLOW, KR_ERR_DUP, KR_ERR_OOM, \
    KR_ERR_CAPACITY, KR_ERR_TIMEOUT, KR_ERR_CUDA, KR_ERR_TABLE_FULL, KR_ERR_TOO_LARGE = range(11)
KR_I64, KR_F64 = 0, 1
KR_PATH_AUTO, KR_PATH_DENSE, KR_PATH_HASH = 0, 1, 2

_vp = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64


class kr_poly(ctypes.Structure):
    _fields_ = [("nvars", _i32), ("nterms", _i64), ("exps", _vp), ("coef", _vp), ("type", ctypes.c_int)]


class kr_poly_out(ctypes.Structure):
    _fields_ = [("nvars", _i32), ("capacity", _i64), ("nterms", _i64), ("exps", _vp), ("coef", _vp),
                ("codes", _vp), ("omin", _i32 * KR_MAXV), ("omax", _i32 * KR_MAXV)]


class kr_pseries(ctypes.Structure):
    _fields_ = [("npoly", _i32), ("ntrig", _i32), ("nterms", _i64), ("exps", _vp), ("trig", _vp),
                ("kind", _vp), ("coef", _vp)]


class kr_pseries_out(ctypes.Structure):
    _fields_ = [("npoly", _i32), ("ntrig", _i32), ("capacity", _i64), ("nterms", _i64), ("exps", _vp),
                ("trig", _vp), ("kind", _vp), ("coef", _vp), ("codes", _vp)]


class kr_opts(ctypes.Structure):
    _fields_ = [("path", _i32), ("block_slots", _i32), ("load_factor", ctypes.c_double),
                ("probe_limit", _i32), ("unsorted", _i32), ("max_regrow", _i32),
                ("table_slots", _i64), ("truncate", _i32), ("trunc_mask", ctypes.c_uint32),
                ("trunc_degree", _i64), ("code_lo", _i64), ("code_hi", _i64),
                ("trunc_harmonic", _i32), ("harmonic_mask", ctypes.c_uint32), ("harmonic_order", _i64),
                ("coef_min", ctypes.c_double)]


class kr_job(ctypes.Structure):
    _fields_ = [("kind", _i32), ("f", kr_poly), ("g", kr_poly), ("pf", kr_pseries), ("pg", kr_pseries),
                ("opts", kr_opts)]


class kr_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("path", _i32), ("nterms", _i64), ("exps", _vp), ("trig", _vp),
                ("kind", _vp), ("coef", _vp)]


# name -> (restype, argtypes); every symbol include/kron.h declares
SIGNATURES = {
    "kr_ctx_create": (ctypes.c_int, [_i32, ctypes.POINTER(_vp)]),
    "kr_ctx_destroy": (None, [_vp]),
    "kr_last_error": (ctypes.c_char_p, [_vp]),
    "kron_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kr_ctx_scratch_bytes": (_i64, [_vp]),
    "kr_ctx_set_profiling": (ctypes.c_int, [_vp, _i32]),
    "kr_ctx_trim": (ctypes.c_int, [_vp]),
    "kr_ctx_stage_count": (_i32, [_vp]),
    "kr_ctx_stage": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_double)]),
    "kr_ctx_launch_count": (_i64, [_vp]),
    "kr_probe_smem_atomic_rate": (ctypes.c_double, [_i32, _i32, _i32]),
    "kr_probe_smem_accumulate_rate": (ctypes.c_double, [_i32, _i32]),
    "kr_selftest_bounded_wait": (ctypes.c_int, [_i32]),
    "kr_probe_table_update_rate": (ctypes.c_double, [_i32, _i32, _i64, _i64, _i32, _i32]),
    "kr_probe_alu_rate": (ctypes.c_double, [_i32, _i32, _i32]),
    "kron_dense_product_static": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.c_int, _i64,
                                                 _vp, _vp]),
    "kron_plan": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "kron_encode": (ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "kron_decode": (ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "poly_mul": (ctypes.c_int, [_vp, ctypes.POINTER(kr_poly), ctypes.POINTER(kr_poly),
                                ctypes.POINTER(kr_poly_out), ctypes.POINTER(kr_opts), _vp]),
    "poisson_mul": (ctypes.c_int, [_vp, ctypes.POINTER(kr_pseries), ctypes.POINTER(kr_pseries),
                                   ctypes.POINTER(kr_pseries_out), ctypes.POINTER(kr_opts), _vp]),
    "kron_fetch_poly": (ctypes.c_int, [_vp, ctypes.POINTER(kr_poly_out), _vp]),
    "kron_mul_batch": (ctypes.c_int, [_vp, ctypes.POINTER(kr_job), _i32, ctypes.POINTER(kr_result), _i64, _vp]),
    "kron_split_hist": (ctypes.c_int, [_vp, ctypes.POINTER(kr_job), _i32, _i64, ctypes.c_uint64,
                                       ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp]),
    "kron_batch_prepare": (ctypes.c_int, [_i32, ctypes.POINTER(kr_job), _i32, ctypes.POINTER(_vp),
                                          ctypes.POINTER(kr_result), _vp]),
    "kron_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "kron_batch_results": (ctypes.c_int, [_vp, ctypes.POINTER(kr_result), _i32]),
    "kron_batch_destroy": (None, [_vp]),
    "kron_batch_graph_kernels": (_i64, [_vp]),
    "kron_fetch_pseries": (ctypes.c_int, [_vp, ctypes.POINTER(kr_pseries_out), _vp]),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libkron.so (building it first when stale and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            try:
                path = _build.build()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise ImportError(f"libkron.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


class KronError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def _check(L, ctx, st: int, what: str):
    if st != KR_OK:
        detail = L.kr_last_error(ctx).decode() if ctx else ""
        raise KronError(st, f"{what}: {L.kron_strerror(st).decode()}" + (f" ({detail})" if detail else ""))


# ----------------------------------------------------------------------------
# array marshalling
# ----------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _ptr_len(a, dtype):
    """(pointer, keep-alive object) for a torch tensor or numpy array of `dtype`."""
    if a is None:
        return None, None
    try:
        torch = _torch()
        if isinstance(a, torch.Tensor):
            tdt = {np.int32: torch.int32, np.int64: torch.int64, np.float64: torch.float64,
                   np.uint8: torch.uint8}[dtype]
            t = a.contiguous()
            if t.dtype != tdt:
                t = t.to(tdt)
            return t.data_ptr(), t
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr


def _out_ptr(out, shape, dtype):
    """Pointer of a caller-supplied output array.  It must already have the
    dtype, the shape and a contiguous layout: a converted copy would take the
    result in its place and the caller's array would never see it."""
    shape = tuple(int(x) for x in shape)
    ok = False
    try:
        torch = _torch()
        if isinstance(out, torch.Tensor):
            tdt = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
            if out.dtype == tdt and out.is_contiguous() and tuple(out.shape) == shape:
                return out.data_ptr()
    except ImportError:
        pass
    if isinstance(out, np.ndarray):
        ok = out.dtype == np.dtype(dtype) and out.flags.c_contiguous and out.shape == shape
        if ok:
            return out.ctypes.data
    raise ValueError(f"out must be a contiguous {np.dtype(dtype).name} array of shape {shape}")


def _stream_ptr(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream


def _opts(path=0, block_slots=0, load_factor=0.0, probe_limit=0, unsorted=0, max_regrow=0,
          table_slots=0, trunc_degree=None, trunc_mask=0, code_lo=0, code_hi=0,
          harmonic_order=None, harmonic_mask=0, coef_min=0.0):
    """kr_opts from keywords; trunc_degree (an int) asks for the truncated product
    of degree <= trunc_degree in the variables of trunc_mask (0 = all);
    [code_lo, code_hi) restricts the product to a window of output keys;
    harmonic_order (an int) keeps the Poisson terms whose harmonic order in the
    trig variables of harmonic_mask (0 = all) is at most that; coef_min > 0
    keeps the pairs of float64 terms with |C_f * C_g| >= coef_min."""
    t = trunc_degree is not None
    h = harmonic_order is not None
    return kr_opts(path, block_slots, load_factor, probe_limit, unsorted, max_regrow, table_slots,
                   1 if t else 0, int(trunc_mask) if t else 0, int(trunc_degree) if t else 0,
                   int(code_lo), int(code_hi), 1 if h else 0, int(harmonic_mask) if h else 0,
                   int(harmonic_order) if h else 0, float(coef_min))


class Context:
    """One libkron context (scratch arenas, kept result) on one CUDA device."""

    def __init__(self, device: int = 0):
        self.L = load()
        self.device = device
        h = _vp()
        st = self.L.kr_ctx_create(device, ctypes.byref(h))
        _check(self.L, None, st, "kr_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.kr_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def scratch_bytes(self) -> int:
        return int(self.L.kr_ctx_scratch_bytes(self.h))

    def trim(self):
        """Release the context's cached device and pinned scratch."""
        _check(self.L, self.h, self.L.kr_ctx_trim(self.h), "kr_ctx_trim")

    def set_profiling(self, on: bool = True):
        _check(self.L, self.h, self.L.kr_ctx_set_profiling(self.h, int(on)), "kr_ctx_set_profiling")

    def stages(self):
        """[(stage name, milliseconds)] of the last multiplication (profiling on)."""
        out = []
        for i in range(int(self.L.kr_ctx_stage_count(self.h))):
            nm, ms = ctypes.c_char_p(), ctypes.c_double()
            self.L.kr_ctx_stage(self.h, i, ctypes.byref(nm), ctypes.byref(ms))
            out.append((nm.value.decode(), float(ms.value)))
        return out

    def launch_count(self) -> int:
        return int(self.L.kr_ctx_launch_count(self.h))


_default: dict[int, Context] = {}


def context(device: int = 0) -> Context:
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def _alloc(shape, dtype, device, host):
    torch = _torch()
    tdt = {np.int32: torch.int32, np.int64: torch.int64, np.float64: torch.float64,
           np.uint8: torch.uint8}[dtype]
    if host:
        return torch.empty(shape, dtype=tdt, pin_memory=False)
    return torch.empty(shape, dtype=tdt, device=f"cuda:{device}")


# ----------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------

def kr_probe_smem_atomic_rate(device: int = 0, f64: bool = False, reps: int = 5) -> float:
    """Shared-memory 64-bit atomic adds per second, whole chip (measured)."""
    return float(load().kr_probe_smem_atomic_rate(device, int(f64), reps))


def kr_probe_table_update_rate(log2_slots: int, distinct: int, updates: int, mode: int = 0,
                               device: int = 0, reps: int = 5) -> float:
    """Random insert-or-adds (mode 0) or plain adds (mode 1) per second into a
    table of 2^log2_slots 16-byte slots (the hash path's ceiling), or float64
    adds (mode 2) into an array of 2^log2_slots 8-byte slots (the Poisson dense
    path's ceiling)."""
    return float(load().kr_probe_table_update_rate(device, log2_slots, distinct, updates, mode, reps))


def kr_probe_alu_rate(kind: int, device: int = 0, reps: int = 5) -> float:
    """Multiply-adds per second: 0 = int64, 1 = 32 x 32 -> 64 bit, 2 = float64 FMA."""
    return float(load().kr_probe_alu_rate(device, kind, reps))


def kr_selftest_bounded_wait(device: int = 0) -> int:
    """Status of the bounded-wait self-test: KR_ERR_TIMEOUT when a wait on a
    predecessor that never publishes gave up and was reported."""
    return int(load().kr_selftest_bounded_wait(device))


def kr_probe_smem_accumulate_rate(device: int = 0, reps: int = 5) -> float:
    """Measured conflict-free rate of the dense kernel's int64 shared-memory
    accumulate (two 32-bit atomics with a carry), accumulates per second."""
    return float(load().kr_probe_smem_accumulate_rate(device, reps))


def kron_plan(emin, emax):
    """(c, W) of the box [emin, emax] (host only)."""
    L = load()
    emin = np.ascontiguousarray(emin, dtype=np.int32)
    emax = np.ascontiguousarray(emax, dtype=np.int32)
    n = emin.shape[0]
    c = np.zeros(n, np.int64)
    W = ctypes.c_int64(0)
    st = L.kron_plan(emin.ctypes.data, emax.ctypes.data, n, c.ctypes.data, ctypes.addressof(W))
    _check(L, None, st, "kron_plan")
    return c, int(W.value)


def kron_encode(exps, emin, emax, ctx: Context | None = None, stream=None, out=None):
    """codes[i] = c . (exps[:, i] - emin) for the box [emin, emax]."""
    ctx = ctx or context()
    nv, n = int(exps.shape[0]), int(exps.shape[1])
    pe, ke = _ptr_len(exps, np.int32)
    emin = np.ascontiguousarray(emin, dtype=np.int32)
    emax = np.ascontiguousarray(emax, dtype=np.int32)
    if out is None:
        out = _alloc((n,), np.int64, ctx.device, host=False)
    po = _out_ptr(out, (n,), np.int64)
    st = ctx.L.kron_encode(ctx.h, pe, n, nv, emin.ctypes.data, emax.ctypes.data, po, _stream_ptr(stream))
    _check(ctx.L, ctx.h, st, "kron_encode")
    return out


def kron_decode(codes, emin, emax, ctx: Context | None = None, stream=None, out=None):
    """exps[k, i] = (codes[i] / c_k) mod w_k + emin[k]."""
    ctx = ctx or context()
    emin = np.ascontiguousarray(emin, dtype=np.int32)
    emax = np.ascontiguousarray(emax, dtype=np.int32)
    nv, n = emin.shape[0], int(codes.shape[0])
    pc, kc = _ptr_len(codes, np.int64)
    if out is None:
        out = _alloc((nv, n), np.int32, ctx.device, host=False)
    po = _out_ptr(out, (nv, n), np.int32)
    st = ctx.L.kron_decode(ctx.h, pc, n, nv, emin.ctypes.data, emax.ctypes.data, po, _stream_ptr(stream))
    _check(ctx.L, ctx.h, st, "kron_decode")
    return out


def poly_mul(f_exps, f_coef, g_exps, g_coef, ctx: Context | None = None, stream=None,
             capacity: int | None = None, host_out: bool = False, want_codes: bool = False, **opts):
    """Product of two sparse polynomials.

    f_exps, g_exps: int32 [nvars, n]; coefficients int64 or float64 [n].
    Returns (exps int32 [nvars, m], coef [m], codes int64 [m] or None, (omin, omax)).
    """
    ctx = ctx or context()
    nv = int(f_exps.shape[0])
    is_f64 = str(getattr(f_coef, "dtype", "")).endswith("float64")
    cdt = np.float64 if is_f64 else np.int64
    pfe, k1 = _ptr_len(f_exps, np.int32)
    pge, k2 = _ptr_len(g_exps, np.int32)
    pfc, k3 = _ptr_len(f_coef, cdt)
    pgc, k4 = _ptr_len(g_coef, cdt)
    f = kr_poly(nv, int(f_exps.shape[1]), pfe, pfc, KR_F64 if is_f64 else KR_I64)
    g = kr_poly(nv, int(g_exps.shape[1]), pge, pgc, KR_F64 if is_f64 else KR_I64)
    o = _opts(**opts)
    cap = capacity if capacity is not None else max(16, f.nterms + g.nterms)

    def outbuf(cap):
        ex = _alloc((nv, cap), np.int32, ctx.device, host_out)
        cf = _alloc((cap,), cdt, ctx.device, host_out)
        cd = _alloc((cap,), np.int64, ctx.device, host_out) if want_codes else None
        h = kr_poly_out(nv, cap, 0, ex.data_ptr(), cf.data_ptr(), cd.data_ptr() if cd is not None else None)
        return h, ex, cf, cd

    h, ex, cf, cd = outbuf(cap)
    sp = _stream_ptr(stream)
    st = ctx.L.poly_mul(ctx.h, ctypes.byref(f), ctypes.byref(g), ctypes.byref(h), ctypes.byref(o), sp)
    if st == KR_ERR_CAPACITY:
        h, ex, cf, cd = outbuf(int(h.nterms))
        st = ctx.L.kron_fetch_poly(ctx.h, ctypes.byref(h), sp)
    _check(ctx.L, ctx.h, st, "poly_mul")
    n = int(h.nterms)
    box = (np.array(h.omin[:nv], np.int32), np.array(h.omax[:nv], np.int32))
    return ex[:, :n], cf[:n], (cd[:n] if cd is not None else None), box


def poisson_mul(f, g, ctx: Context | None = None, stream=None, capacity: int | None = None,
                host_out: bool = False, want_codes: bool = False, **opts):
    """Product of two Poisson series.

    f, g: objects with exps int32 [npoly, n], trig int32 [ntrig, n], kind uint8 [n],
    coef float64 [n].  Returns (exps, trig, kind, coef, codes or None).
    """
    ctx = ctx or context()
    npoly, ntrig = int(f.exps.shape[0]), int(f.trig.shape[0])
    keep = []

    def desc(s):
        pe, a = _ptr_len(s.exps, np.int32)
        pt, b = _ptr_len(s.trig, np.int32)
        pk, c = _ptr_len(s.kind, np.uint8)
        pc, d = _ptr_len(s.coef, np.float64)
        keep.extend([a, b, c, d])
        return kr_pseries(npoly, ntrig, int(s.coef.shape[0]), pe, pt, pk, pc)

    F, G = desc(f), desc(g)
    o = _opts(**opts)
    cap = capacity if capacity is not None else max(16, 2 * (F.nterms + G.nterms))

    def outbuf(cap):
        ex = _alloc((npoly, cap), np.int32, ctx.device, host_out)
        tr = _alloc((ntrig, cap), np.int32, ctx.device, host_out)
        kd = _alloc((cap,), np.uint8, ctx.device, host_out)
        cf = _alloc((cap,), np.float64, ctx.device, host_out)
        cd = _alloc((cap,), np.int64, ctx.device, host_out) if want_codes else None
        h = kr_pseries_out(npoly, ntrig, cap, 0, ex.data_ptr() if npoly else None, tr.data_ptr(),
                           kd.data_ptr(), cf.data_ptr(), cd.data_ptr() if cd is not None else None)
        return h, ex, tr, kd, cf, cd

    h, ex, tr, kd, cf, cd = outbuf(cap)
    sp = _stream_ptr(stream)
    st = ctx.L.poisson_mul(ctx.h, ctypes.byref(F), ctypes.byref(G), ctypes.byref(h), ctypes.byref(o), sp)
    if st == KR_ERR_CAPACITY:
        h, ex, tr, kd, cf, cd = outbuf(int(h.nterms))
        st = ctx.L.kron_fetch_pseries(ctx.h, ctypes.byref(h), sp)
    _check(ctx.L, ctx.h, st, "poisson_mul")
    n = int(h.nterms)
    return ex[:, :n], tr[:, :n], kd[:n], cf[:n], (cd[:n] if cd is not None else None)


def kron_dense_product_static(fcode, fcoef, gcode, gcoef, W: int, out=None, stream=None):
    """Dense product array out[W] of two sorted, coded operands, using only the
    library's static scratch array (no allocation inside the library).

    All arrays are CUDA torch tensors; out (int64 or float64 [W]) is allocated
    here by torch when not given.
    """
    L = load()
    torch = _torch()
    if fcoef.dtype not in (torch.int64, torch.float64) or gcoef.dtype != fcoef.dtype:
        raise ValueError("fcoef and gcoef must both be int64 or both float64")
    if fcode.dtype != torch.int64 or gcode.dtype != torch.int64:
        raise ValueError("codes must be int64")
    if fcode.shape[0] != fcoef.shape[0] or gcode.shape[0] != gcoef.shape[0]:
        raise ValueError("each operand needs one coefficient per code")
    if out is None:
        out = torch.empty((W,), dtype=fcoef.dtype, device=fcoef.device)
    if out.dtype != fcoef.dtype or out.numel() < W:
        raise ValueError(f"out must hold at least W = {W} elements of the coefficient type")
    ts = (fcode, fcoef, gcode, gcoef, out)
    if any(not t.is_cuda or t.device != fcoef.device for t in ts):
        raise ValueError("every array must be a CUDA tensor on one device")
    if any(t.dim() != 1 or not t.is_contiguous() for t in ts):
        raise ValueError("every array must be one-dimensional and contiguous")
    is_f64 = fcoef.dtype == torch.float64
    st = L.kron_dense_product_static(fcode.data_ptr(), fcoef.data_ptr(), int(fcode.shape[0]),
                                     gcode.data_ptr(), gcoef.data_ptr(), int(gcode.shape[0]),
                                     KR_F64 if is_f64 else KR_I64, int(W), out.data_ptr(),
                                     _stream_ptr(stream))
    _check(L, None, st, "kron_dense_product_static")
    return out


class _DevArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


def _view(ptr, shape, typestr, device):
    torch = _torch()
    if not ptr or any(d == 0 for d in shape):
        dt = {"<i4": torch.int32, "<i8": torch.int64, "<f8": torch.float64, "|u1": torch.uint8}[typestr]
        return torch.empty(shape, dtype=dt, device=f"cuda:{device}")
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device=f"cuda:{device}")


def kron_split_hist(f, g, nbins: int = 65536, nsamples: int = 1 << 22, seed: int = 1,
                    ctx: Context | None = None, stream=None, **opts):
    """Work histogram of f * g over nbins equal slices of its key range.

    Returns (hist int64 [nbins], krange): hist[b] counts sampled output keys k
    with k * nbins // krange == b.
    """
    ctx = ctx or context()
    jobs, keep = _make_jobs([(f, g)], [opts])
    hist = np.zeros(nbins, np.int64)
    kr = _i64(0)
    st = ctx.L.kron_split_hist(ctx.h, jobs, int(nbins), int(nsamples), int(seed) & ((1 << 64) - 1),
                               hist.ctypes.data_as(ctypes.POINTER(_i64)), ctypes.byref(kr),
                               _stream_ptr(stream))
    _check(ctx.L, ctx.h, st, "kron_split_hist")
    return hist, int(kr.value)


def kron_mul_batch(pairs, ctx: Context | None = None, stream=None, wave_pairs: int = 0, opts=None):
    """Multiply many (f, g) pairs in one batched pipeline.

    pairs: list of (f, g), each a Poly-like (.exps, .coef) or PSeries-like
    (.exps, .trig, .kind, .coef) object with numpy or torch arrays.
    opts: None, one dict of kr_opts fields for all, or a list of dicts.
    Returns a list of dicts {status, path, exps, trig, kind, coef}: torch views
    of library-owned device memory, valid until the next batch on the context.
    """
    ctx = ctx or context()
    n = len(pairs)
    jobs, keep = _make_jobs(pairs, opts)
    res = (kr_result * max(1, n))()
    st = ctx.L.kron_mul_batch(ctx.h, jobs, n, res, int(wave_pairs), _stream_ptr(stream))
    _check(ctx.L, ctx.h, st, "kron_mul_batch")
    return _results(jobs, res, n, ctx.device)


def _make_jobs(pairs, opts):
    n = len(pairs)
    jobs = (kr_job * max(1, n))()
    keep = []
    for i, (f, g) in enumerate(pairs):
        o = opts[i] if isinstance(opts, (list, tuple)) else (opts or {})
        jobs[i].opts = _opts(**o)
        if hasattr(f, "trig"):
            def desc(p):
                pe, a = _ptr_len(p.exps, np.int32)
                pt, b = _ptr_len(p.trig, np.int32)
                pk, c = _ptr_len(p.kind, np.uint8)
                pc, d = _ptr_len(p.coef, np.float64)
                keep.extend([a, b, c, d])
                return kr_pseries(int(p.exps.shape[0]), int(p.trig.shape[0]), int(p.coef.shape[0]),
                                  pe, pt, pk, pc)
            jobs[i].kind = 1
            jobs[i].pf = desc(f)
            jobs[i].pg = desc(g)
        else:
            is_f64 = str(getattr(f.coef, "dtype", "")).endswith("float64")
            cdt = np.float64 if is_f64 else np.int64
            def desc(p):
                pe, a = _ptr_len(p.exps, np.int32)
                pc, b = _ptr_len(p.coef, cdt)
                keep.extend([a, b])
                return kr_poly(int(p.exps.shape[0]), int(p.coef.shape[0]), pe, pc, KR_F64 if is_f64 else KR_I64)
            jobs[i].kind = 0
            jobs[i].f = desc(f)
            jobs[i].g = desc(g)
    return jobs, keep


def _results(jobs, res, n, device):
    out = []
    for i in range(n):
        r = res[i]
        m = int(r.nterms)
        d = {"status": int(r.status), "path": int(r.path), "nterms": m}
        if jobs[i].kind == 1:
            npl, nt = jobs[i].pf.npoly, jobs[i].pf.ntrig
            d["exps"] = _view(r.exps, (npl, m), "<i4", device)
            d["trig"] = _view(r.trig, (nt, m), "<i4", device)
            d["kind"] = _view(r.kind, (m,), "|u1", device)
            d["coef"] = _view(r.coef, (m,), "<f8", device)
        else:
            nv = jobs[i].f.nvars
            d["exps"] = _view(r.exps, (nv, m), "<i4", device)
            d["coef"] = _view(r.coef, (m,), "<f8" if jobs[i].f.type == KR_F64 else "<i8", device)
        out.append(d)
    return out


class PreparedBatch:
    """A batch captured into a CUDA graph (kron_batch_prepare).

    The operands must be CUDA tensors whose exponents stay fixed; their
    coefficients may be changed in place between launches.
    """

    def __init__(self, pairs, device: int = 0, stream=None, opts=None):
        self.L = load()
        self.n = len(pairs)
        self.device = device
        self.jobs, self._keep = _make_jobs(pairs, opts)
        self._res = (kr_result * max(1, self.n))()
        h = _vp()
        st = self.L.kron_batch_prepare(device, self.jobs, self.n, ctypes.byref(h), self._res, _stream_ptr(stream))
        _check(self.L, None, st, "kron_batch_prepare")
        self.h = h

    def first_results(self):
        return _results(self.jobs, self._res, self.n, self.device)

    def launch(self, stream=None):
        _check(self.L, None, self.L.kron_batch_launch(self.h, _stream_ptr(stream)), "kron_batch_launch")

    def graph_kernels(self) -> int:
        """Kernel launches in one replay (the kernel nodes of the captured graph)."""
        return int(self.L.kron_batch_graph_kernels(self.h))

    def results(self):
        """Statuses and device views after the launch's stream has been synchronised."""
        res = (kr_result * max(1, self.n))()
        _check(self.L, None, self.L.kron_batch_results(self.h, res, self.n), "kron_batch_results")
        return _results(self.jobs, res, self.n, self.device)

    def close(self):
        if getattr(self, "h", None):
            self.L.kron_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
