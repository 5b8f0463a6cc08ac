"""Ordering of large hash-path outputs over wide code ranges (at least 2^20
terms over more than 2^30 codes: the partition into fine buckets and their
ranking in shared memory), bit-exact against the oracle: random terms spread
thinly over the range, and dense clusters whose fine buckets are too full for
shared memory (ranked in device memory instead)."""
import os

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_equal, to_np
from workloads import Poly, Rng, dense_box, random_poly

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


def run(kron, f, g, **opts):
    import torch
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ex, cf, _, _ = kron.poly_mul(d(f.exps), d(f.coef), d(g.exps), d(g.coef), path=kron.KR_PATH_HASH, **opts)
    return to_np(ex), to_np(cf)


def test_thin_terms_over_a_wide_range(kron):
    f = random_poly(5, 2048, -20, 20, 8101)
    g = random_poly(5, 2048, -20, 20, 8102)
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert r.coef.shape[0] >= 1 << 20
    ex, cf = run(kron, f, g)
    assert_poly_equal(ex, cf, r, "thin terms")


def test_dense_clusters_over_a_wide_range(kron):
    # f: a dense 128 x 128 box in variables 0 and 1; g: 64 terms far apart in
    # variable 2 (and near 0 in the others): 64 shifted copies of a dense block
    box = dense_box([0, 0, 0], [127, 127, 0], 1.0, -50, 50, 8103)
    rng = Rng(8104)
    shifts = np.unique(rng.ints(0, 1000000, 200))[:64].astype(np.int32)
    gex = np.zeros((3, shifts.shape[0]), dtype=np.int32)
    gex[0] = rng.ints(0, 3, shifts.shape[0]).astype(np.int32)
    gex[2] = shifts
    g = Poly(gex, rng.nonzero_ints(-50, 50, shifts.shape[0]))
    r = oracle.poly_mul(box, g, nthreads=NT)
    assert r.coef.shape[0] >= 1 << 20
    ex, cf = run(kron, box, g)
    assert_poly_equal(ex, cf, r, "dense clusters")
