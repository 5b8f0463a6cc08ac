"""The entry point that allocates nothing (kron_dense_product_static), through
the C ABI, against the oracle.

Its callers are programs that cannot let a library allocate or free device
memory: their memory belongs to their own allocator or a fixed budget, or the
device synchronisation that an allocation or a free brings is unacceptable to
them.  The entry point keeps its scratch in a static device array shared by
all calls, so the check runs several different products in a row (the later
ones must not see leftovers of the earlier ones) and watches the device's
free memory across them.  This file is collected last so that a failure here
comes after every other test has run.
"""
import gc
import os

import numpy as np
import pytest

import oracle
from workloads import random_poly, workload_cfg1

pytestmark = pytest.mark.gpu
NT = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1004_4548_gb300 as k
    k.load()
    return k


def _box(f, g):
    """The product's coding box: output widths, the coding vector c_0 = 1,
    c_k = w_0 ... w_{k-1}, and each operand's own minimum as its offset."""
    fmin, gmin = f.exps.min(axis=1).astype(np.int64), g.exps.min(axis=1).astype(np.int64)
    w = f.exps.max(axis=1).astype(np.int64) + g.exps.max(axis=1) - fmin - gmin + 1
    c = np.concatenate([[1], np.cumprod(w)[:-1]]).astype(np.int64)
    return w, c, fmin, gmin


def _codes(exps, c, lo):
    return ((exps.astype(np.int64) - lo[:, None]) * c[:, None]).sum(axis=0)


def _case(f, g):
    """Sorted device codes and coefficients of both operands, and the oracle's
    product scattered into a dense array over the product's code range."""
    import torch
    w, c, fmin, gmin = _box(f, g)
    W = int(np.prod(w))
    ops = []
    for p, lo in ((f, fmin), (g, gmin)):
        cd = _codes(p.exps, c, lo)
        o = np.argsort(cd, kind="stable")
        ops += [torch.from_numpy(cd[o]).cuda(), torch.from_numpy(np.ascontiguousarray(p.coef[o])).cuda()]
    is_f64 = f.coef.dtype == np.float64
    r = oracle.poly_mul(f, g, nthreads=NT, keep_zero=is_f64)
    hc = _codes(r.exps, c, fmin + gmin)
    want = np.zeros(W, dtype=f.coef.dtype)
    want[hc] = r.coef
    mass = None
    if is_f64:
        mass = np.zeros(W)
        mass[hc] = r.mass
    return ops, W, want, mass


def _check(got, want, mass, what):
    if mass is None:
        assert np.array_equal(got, want), f"{what}: {int((got != want).sum())} codes differ"
    else:
        # per output code: |difference| <= 1e-12 * sum of |contributions|
        bad = np.abs(got - want) > 1e-12 * mass
        assert not bad.any(), f"{what}: {int(bad.sum())} codes beyond the tolerance"


def test_static_scratch_entry_matches_oracle_in_a_row(kron):
    import torch
    cases = [workload_cfg1(),
             (random_poly(3, 900, [-5, 0, -7], [6, 9, 3], 501, "f64"),
              random_poly(3, 700, [-5, 0, -7], [6, 9, 3], 502, "f64")),
             (random_poly(2, 3000, -300, 300, 503), random_poly(2, 2500, -300, 300, 504))]
    prepared = [_case(f, g) for f, g in cases]
    outs = [torch.empty(W, dtype=ops[1].dtype, device="cuda") for ops, W, _, _ in prepared]
    # first calls: the library looks up the array's address, and every kernel
    # the loop below runs (the library's and torch's fill and copy) is loaded
    # (CUDA loads a module's code into device memory on first use)
    for (ops, W, _, _), out in zip(prepared, outs):
        out.fill_(7)
        kron.kron_dense_product_static(*ops, W, out=out)
        out.cpu()
    torch.cuda.synchronize()
    gc.collect()
    free0 = torch.cuda.mem_get_info()[0]
    # torch's count of device allocation requests (cumulative; frees of other
    # tests' tensors do not move it)
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for rnd in range(2):
        for k, ((ops, W, want, mass), out) in enumerate(zip(prepared, outs)):
            out.fill_(7)   # garbage the call must overwrite in full
            kron.kron_dense_product_static(*ops, W, out=out)
            torch.cuda.synchronize()
            _check(out.cpu().numpy(), want, mass, f"round {rnd} case {k}")
    assert torch.cuda.mem_get_info()[0] == free0, "device memory was allocated during the calls"
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0


def test_static_scratch_entry_rejects_too_large(kron):
    import torch
    one = torch.zeros(1, dtype=torch.int64, device="cuda")
    L = kron.load()
    p = one.data_ptr()
    st = L.kron_dense_product_static(p, p, 1, p, p, 1, kron.binding.KR_I64, (1 << 24) + 1, p, None)
    assert st == kron.KR_ERR_TOO_LARGE
    with pytest.raises(ValueError):
        kron.kron_dense_product_static(one, one, one, one, 16, out=one)   # out shorter than W


def test_static_scratch_entry_broken_preconditions_stay_in_bounds(kron):
    """Codes below zero, out of order, or with a pair sum past W: the call
    returns, out is all zeros, and the memory around out is untouched."""
    import torch
    W = 64
    guard = 4096
    buf = torch.full((guard + W + guard,), 1234567, dtype=torch.int64, device="cuda")
    out = buf[guard:guard + W]
    f = torch.tensor([0, 2, 5], dtype=torch.int64, device="cuda")
    fk = torch.tensor([3, -4, 5], dtype=torch.int64, device="cuda")
    for g in ([-3, 1], [5, 1], [0, 60], [-(1 << 40), 1 << 40]):
        gd = torch.tensor(g, dtype=torch.int64, device="cuda")
        gk = torch.tensor([7, 11], dtype=torch.int64, device="cuda")
        kron.kron_dense_product_static(f, fk, gd, gk, W, out=out)
        torch.cuda.synchronize()
        assert (out == 0).all(), f"g codes {g}: out not cleared"
        assert (buf[:guard] == 1234567).all() and (buf[guard + W:] == 1234567).all(), \
            f"g codes {g}: memory outside out was written"
    # and a valid product right after is exact
    gd = torch.tensor([1, 3], dtype=torch.int64, device="cuda")
    gk = torch.tensor([7, 11], dtype=torch.int64, device="cuda")
    kron.kron_dense_product_static(f, fk, gd, gk, W, out=out)
    torch.cuda.synchronize()
    want = np.zeros(W, np.int64)
    for a, ca in zip([0, 2, 5], [3, -4, 5]):
        for b, cb in zip([1, 3], [7, 11]):
            want[a + b] += ca * cb
    assert np.array_equal(out.cpu().numpy(), want)
