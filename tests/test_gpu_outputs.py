"""Where the library reads a product's operands and writes its terms, against
the oracle (bit-exact): device arrays, pinned host arrays (read and written by
the GPU through their device mapping), pageable host arrays (staged through
device scratch), with and
without the code array, and with a capacity below the term count (the call
reports KR_ERR_CAPACITY and kron_fetch_poly then fills larger arrays).
Through the C ABI, as a caller of include/kron.h would."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_equal
from workloads import workload_cfg1, workload_cfg2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1004_4548_gb300 as k
    from paper_1004_4548_gb300 import binding as B
    L = k.load()
    return k, B, L, k.Context(0)


def buffers(kind, nv, cap, codes):
    import torch
    kw = {"cuda": dict(device="cuda:0"), "pinned": dict(pin_memory=True), "pageable": dict()}[kind]
    ex = torch.empty((nv, cap), dtype=torch.int32, **kw)
    cf = torch.empty((cap,), dtype=torch.int64, **kw)
    cd = torch.empty((cap,), dtype=torch.int64, **kw) if codes else None
    return ex, cf, cd


def inputs(kind, p):
    """The operand's arrays where the outputs go: device, pinned host (read by
    the kernels in place) or pageable host (staged)."""
    import torch
    e, c = torch.from_numpy(np.ascontiguousarray(p.exps)), torch.from_numpy(np.ascontiguousarray(p.coef))
    if kind == "cuda":
        return e.cuda(), c.cuda()
    if kind == "pinned":
        return e.pin_memory(), c.pin_memory()
    return e, c


def mul(env, f, g, kind, cap, codes):
    import torch
    k, B, L, ctx = env
    fe, fc = inputs(kind, f)
    ge, gc = inputs(kind, g)
    nv = f.exps.shape[0]
    F = B.kr_poly(nv, f.n, fe.data_ptr(), fc.data_ptr(), B.KR_I64)
    G = B.kr_poly(nv, g.n, ge.data_ptr(), gc.data_ptr(), B.KR_I64)
    ex, cf, cd = buffers(kind, nv, cap, codes)
    H = B.kr_poly_out(nv, cap, 0, ex.data_ptr(), cf.data_ptr(), cd.data_ptr() if codes else None)
    O = B.kr_opts()
    st = L.poly_mul(ctx.h, ctypes.byref(F), ctypes.byref(G), ctypes.byref(H), ctypes.byref(O), None)
    if st == k.KR_ERR_CAPACITY:
        n = int(H.nterms)
        assert n > cap
        ex, cf, cd = buffers(kind, nv, n, codes)
        H = B.kr_poly_out(nv, n, 0, ex.data_ptr(), cf.data_ptr(), cd.data_ptr() if codes else None)
        st = L.kron_fetch_poly(ctx.h, ctypes.byref(H), None)
    assert st == 0, L.kr_last_error(ctx.h).decode()
    torch.cuda.synchronize()
    n = int(H.nterms)
    ld = ex.shape[1]
    exps = ex.cpu().numpy()[:, :n] if ld >= n else None
    return exps, cf.cpu().numpy()[:n], (cd.cpu().numpy()[:n] if codes else None), n


@pytest.mark.parametrize("kind", ["cuda", "pinned", "pageable"])
@pytest.mark.parametrize("codes", [False, True])
@pytest.mark.parametrize("short", [False, True])
def test_outputs(env, kind, codes, short):
    f, g = workload_cfg2() if not short else workload_cfg1()
    r = oracle.poly_mul(f, g, nthreads=8)
    m = r.coef.shape[0]
    cap = m // 3 if short else m + 17   # below the count: a capacity retry; above: spare room
    exps, coef, cd, n = mul(env, f, g, kind, cap, codes)
    assert n == m
    assert_poly_equal(exps, coef, r, f"{kind} codes={codes} cap={cap}")
    if codes:
        # the codes ascend and decode to the exponents: variable 0 least significant
        # over the output box of widths w_k
        assert (np.diff(cd) > 0).all()
        lo = r.exps.min(axis=1).astype(np.int64)
        w = (r.exps.max(axis=1) - r.exps.min(axis=1) + 1).astype(np.int64)
        # the library's box is the sum of the operand boxes; take its widths
        fw = f.exps.max(axis=1).astype(np.int64) - f.exps.min(axis=1) + g.exps.max(axis=1) - g.exps.min(axis=1) + 1
        flo = f.exps.min(axis=1).astype(np.int64) + g.exps.min(axis=1)
        c = np.zeros(n, dtype=np.int64)
        mult = 1
        for k in range(exps.shape[0]):
            c += (exps[k].astype(np.int64) - flo[k]) * mult
            mult *= int(fw[k])
        assert np.array_equal(c, cd)
        assert (lo >= flo).all() and (w <= fw).all()


@pytest.mark.parametrize("kind", ["cuda", "pinned", "pageable"])
def test_poisson_operands_in_each_memory(env, kind):
    """A Poisson product whose operands (exponents, multipliers, kinds,
    coefficients) are device arrays, pinned host arrays read in place, or
    pageable host arrays staged by copies; outputs in device memory."""
    import torch
    from gpu_compare import assert_pseries_close
    from workloads import PSeries, random_pseries
    k = env[0]
    f = random_pseries(2, 3, 700, 3, 4, 8201)
    g = random_pseries(2, 3, 900, 3, 4, 8202)
    r = oracle.poisson_mul(f, g, nthreads=8, keep_zero=True)

    def put(p):
        arrs = [torch.from_numpy(np.ascontiguousarray(a)) for a in (p.exps, p.trig, p.kind, p.coef)]
        if kind == "cuda":
            arrs = [a.cuda() for a in arrs]
        elif kind == "pinned":
            arrs = [a.pin_memory() for a in arrs]
        return PSeries(*arrs)

    out = k.poisson_mul(put(f), put(g))
    torch.cuda.synchronize()
    got = tuple(a.cpu().numpy() for a in out[:4])
    assert_pseries_close(got, r, 1e-12, f"poisson operands {kind}")
