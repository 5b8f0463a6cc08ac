"""Key windows on the GPU: a product computed window by window (the way the
ranks of a group compute it) concatenates to the whole product, and each
window holds exactly the product's terms with keys in it."""
import os

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_equal, assert_pseries_close, to_np
from workloads import PSeries, Poly, random_poly, random_pseries, workload_cfg2, workload_cfg3

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


def dev_poly(p):
    import torch
    return Poly(torch.from_numpy(p.exps).cuda(), torch.from_numpy(p.coef).cuda())


def dev_pseries(p):
    import torch
    return PSeries(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (p.exps, p.trig, p.kind, p.coef)))


def windows_concat(kron, F, G, cuts, **opts):
    from paper_1004_4548_gb300 import shard
    parts = [shard.mul_window(F, G, a, b, **opts) for a, b in zip(cuts, cuts[1:])]
    return [np.concatenate([to_np(p[k]) for p in parts], axis=-1) for k in range(len(parts[0]))], \
        [to_np(p[-1]).shape[0] for p in parts]


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("nparts", [2, 3, 7])
def test_poly_windows_make_the_product(kron, path, nparts):
    from paper_1004_4548_gb300 import shard
    f, g = workload_cfg2()
    F, G = dev_poly(f), dev_poly(g)
    cuts = shard.split_points(F, G, nparts, path=path)
    assert cuts[0] == 0 and cuts == sorted(cuts) and len(cuts) == nparts + 1
    (ex, cf), sizes = windows_concat(kron, F, G, cuts, path=path)
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert_poly_equal(ex, cf, r, f"{nparts} windows path={path}")
    # equal sampled work: every window holds a fair share of the output terms
    assert min(sizes) > 0


def test_poly_hash_windows_mp_sparse(kron):
    from paper_1004_4548_gb300 import shard
    f, g = workload_cfg3()
    F, G = dev_poly(f), dev_poly(g)
    cuts = shard.split_points(F, G, 4, path=2)
    (ex, cf), _ = windows_concat(kron, F, G, cuts, path=2)
    r = oracle.poly_mul(f, g, nthreads=NT)
    assert_poly_equal(ex, cf, r, "MP-sparse hash windows")


@pytest.mark.parametrize("path", [1, 2])
def test_truncated_product_windows(kron, path):
    from paper_1004_4548_gb300 import shard
    f = random_poly(4, 3000, [-4, 0, -6, -2], [5, 7, 3, 6], 3100)
    g = random_poly(4, 2500, [-4, 0, -6, -2], [5, 7, 3, 6], 3101)
    F, G = dev_poly(f), dev_poly(g)
    opts = dict(path=path, trunc_degree=3, trunc_mask=0b0110)
    cuts = shard.split_points(F, G, 5, **opts)
    (ex, cf), _ = windows_concat(kron, F, G, cuts, **opts)
    # the truncated product's order is by degree first: compare as sets of terms
    r = oracle.poly_mul(f, g, nthreads=NT, trunc=(3, 0b0110))
    got = {tuple(int(x) for x in ex[:, i]): int(cf[i]) for i in range(cf.shape[0])}
    want = {tuple(int(x) for x in r.exps[:, i]): int(r.coef[i]) for i in range(r.coef.shape[0])}
    assert len(got) == cf.shape[0] and got == want


@pytest.mark.parametrize("path", [1, 2])
def test_poisson_windows_make_the_product(kron, path):
    from paper_1004_4548_gb300 import shard
    f = random_pseries(2, 3, 3000, 4, 5, 3200)
    g = random_pseries(2, 3, 2600, 4, 5, 3201)
    F, G = dev_pseries(f), dev_pseries(g)
    cuts = shard.split_points(F, G, 4, path=path)
    (ex, tr, kd, cf), _ = windows_concat(kron, F, G, cuts, path=path)
    r = oracle.poisson_mul(f, g, nthreads=NT, keep_zero=True)
    assert_pseries_close((ex, tr, kd, cf), r, 1e-12, f"poisson windows path={path}")


def test_window_edges(kron):
    f = random_poly(3, 400, -3, 3, 3300)
    g = random_poly(3, 300, -3, 3, 3301)
    F, G = dev_poly(f), dev_poly(g)
    full_ex, full_cf, codes, _ = kron.poly_mul(F.exps, F.coef, G.exps, G.coef, want_codes=True)
    codes = to_np(codes)
    for path in (1, 2):
        # a window holding exactly one term, one beyond every key, and an empty one
        k = int(codes[len(codes) // 2])
        ex, cf, cd, _ = kron.poly_mul(F.exps, F.coef, G.exps, G.coef, path=path, code_lo=k, code_hi=k + 1,
                                      want_codes=True)
        assert to_np(cf).shape[0] == 1 and int(to_np(cd)[0]) == k
        assert np.array_equal(to_np(ex)[:, 0], to_np(full_ex)[:, len(codes) // 2])
        ex, cf, _, _ = kron.poly_mul(F.exps, F.coef, G.exps, G.coef, path=path,
                                     code_lo=int(codes[-1]) + 1, code_hi=1 << 62)
        assert to_np(cf).shape[0] == 0
        ex, cf, _, _ = kron.poly_mul(F.exps, F.coef, G.exps, G.coef, path=path, code_lo=50, code_hi=50)
        assert to_np(cf).shape[0] == 0
        # host output buffers get absolute codes
        ex, cf, cd, _ = kron.poly_mul(f.exps, f.coef, g.exps, g.coef, path=path, code_lo=k, code_hi=1 << 62,
                                      host_out=True, want_codes=True)
        assert np.array_equal(to_np(cd), codes[codes >= k])


def test_split_hist_counts(kron):
    f, g = workload_cfg2()
    F, G = dev_poly(f), dev_poly(g)
    hist, krange = kron.binding.kron_split_hist(F, G, nbins=1024, nsamples=1 << 20)
    assert hist.sum() == 1 << 20 and krange == 41 ** 4
    again, _ = kron.binding.kron_split_hist(F, G, nbins=1024, nsamples=1 << 20)
    assert np.array_equal(hist, again)
    fp = random_pseries(2, 2, 500, 3, 3, 3400)
    gp = random_pseries(2, 2, 400, 3, 3, 3401)
    hist, krange = kron.binding.kron_split_hist(dev_pseries(fp), dev_pseries(gp), nbins=512, nsamples=1 << 16)
    assert (1 << 17) * 0.9 < hist.sum() <= 1 << 17   # two keys per pair, less the vanishing sines
