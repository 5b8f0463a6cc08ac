"""The entry point that allocates nothing (kron_dense_product_static) against
the regular entry point (poly_mul), through the C ABI.

Its callers are programs that cannot let a library allocate or free device
memory (their memory belongs to their own allocator or a fixed budget, or an
allocation's device synchronisation is unacceptable to them).  The entry point
keeps its scratch in a static device array shared by all calls, so the check
runs two different products in a row: the second must not see leftovers of
the first.  This file is collected last so that a failure here comes after
every other test has run.
"""
import numpy as np
import pytest

from workloads import random_poly, workload_cfg1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1004_4548_gb300 as k
    k.load()
    return k


def _dense_from_poly_mul(kron, f, g):
    """Reference: poly_mul's sparse product scattered into a dense code array."""
    import torch
    ex, cf, codes, (omin, omax) = kron.poly_mul(f.exps, f.coef, g.exps, g.coef, want_codes=True)
    w = (omax.astype(np.int64) - omin + 1)
    W = int(np.prod(w))
    dense = np.zeros(W, dtype=f.coef.dtype)
    dense[codes.cpu().numpy()] = cf.cpu().numpy()
    return dense, w, W


def _coded_sorted(kron, p, w):
    """Codes of p in the product's box (offset by p's own minimum), sorted, on the device."""
    import torch
    lo = p.exps.min(axis=1).astype(np.int32)
    hi = (lo + w - 1).astype(np.int32)
    codes = kron.kron_encode(p.exps, lo, hi).cpu().numpy()
    order = np.argsort(codes, kind="stable")
    return (torch.from_numpy(codes[order]).cuda(),
            torch.from_numpy(np.ascontiguousarray(p.coef[order])).cuda())


def test_static_scratch_entry_matches_poly_mul_twice(kron):
    cases = [workload_cfg1(),
             (random_poly(3, 900, [-5, 0, -7], [6, 9, 3], 501, "f64"),
              random_poly(3, 700, [-5, 0, -7], [6, 9, 3], 502, "f64"))]
    for f, g in cases:
        want, w, W = _dense_from_poly_mul(kron, f, g)
        fc, fk = _coded_sorted(kron, f, w)
        gc, gk = _coded_sorted(kron, g, w)
        got = kron.kron_dense_product_static(fc, fk, gc, gk, W).cpu().numpy()
        if f.coef.dtype == np.int64:
            assert np.array_equal(got, want)
        else:
            # per output code: |difference| <= 1e-12 * sum of |contributions|
            fcn, gcn = fc.cpu().numpy(), gc.cpu().numpy()
            fa, ga = np.abs(fk.cpu().numpy()), np.abs(gk.cpu().numpy())
            mass = np.zeros(W)
            np.add.at(mass, (fcn[:, None] + gcn[None, :]).ravel(), (fa[:, None] * ga[None, :]).ravel())
            assert (np.abs(got - want) <= 1e-12 * mass).all()


def test_static_scratch_entry_rejects_too_large(kron):
    import torch
    one = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(kron.KronError) as e:
        kron.kron_dense_product_static(one, one, one, one, (1 << 24) + 1, out=one)
    assert e.value.status == kron.KR_ERR_TOO_LARGE
