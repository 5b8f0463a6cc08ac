"""Operand front end on the GPU: large operands of a call with few operands are
encoded, ranked and gathered by one cluster of CTAs per operand (the key bitmap
spread over the cluster's shared memory); calls with many operands rank each
one in one CTA.  Both against the oracle, plus repeated keys in different
slices of the bitmap, truncation, Poisson terms and a CUDA-graph replay."""
import os

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_equal, assert_pseries_close, to_np
from workloads import PSeries, Poly, random_poly, random_pseries

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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def large():
    f = random_poly(4, 6000, -6, 6, 7001)
    g = random_poly(4, 5000, -6, 6, 7002)
    return f, g, oracle.poly_mul(f, g, nthreads=NT)


def test_cluster_front_end_is_used_and_exact(kron, large):
    f, g, r = large
    ctx = kron.binding.Context()
    ctx.set_profiling(True)
    try:
        for path in (kron.KR_PATH_AUTO, kron.KR_PATH_DENSE, kron.KR_PATH_HASH):
            ex, cf, _, _ = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), ctx=ctx, path=path)
            assert_poly_equal(to_np(ex), to_np(cf), r, f"cluster front end path={path}")
            names = [n for n, _ in ctx.stages()]
            assert "front" in names and "encode" not in names, names
    finally:
        ctx.close()


@pytest.mark.parametrize("copies", [20, 40])
def test_many_operands_one_cta_each(kron, large, copies):
    # 40 operands stay on the cluster front end, 80 go to one CTA each
    f, g, r = large
    out = kron.kron_mul_batch([(f, g)] * copies)
    for i, o in enumerate(out):
        assert o["status"] == 0
        assert_poly_equal(to_np(o["exps"]), to_np(o["coef"]), r, f"{copies} copies, product {i}")


@pytest.mark.parametrize("where", ["first", "last", "far"])
def test_repeated_key_in_large_operand(kron, large, where):
    f, g, _ = large
    n = f.coef.shape[0]
    src = {"first": 0, "last": n - 1, "far": n // 2}[where]
    # the copy goes to the front (the other slice's threads see it first) or the back
    exps = np.concatenate([f.exps[:, src:src + 1], f.exps], axis=1) if where == "far" else \
        np.concatenate([f.exps, f.exps[:, src:src + 1]], axis=1)
    coef = np.concatenate([f.coef[:1], f.coef]) if where == "far" else np.concatenate([f.coef, f.coef[:1]])
    with pytest.raises(kron.KronError) as e:
        kron.poly_mul(dev(exps), dev(coef), dev(g.exps), dev(g.coef))
    assert e.value.status == kron.KR_ERR_DUP


@pytest.mark.parametrize("path", [1, 2])
def test_truncated_large_operands(kron, path):
    f = random_poly(4, 4000, [-4, 0, -6, -2], [5, 7, 3, 6], 7101)
    g = random_poly(4, 3500, [-4, 0, -6, -2], [5, 7, 3, 6], 7102)
    for N, mask in ((3, 0b0110), (0, 0b1111), (9, 0b0001)):
        r = oracle.poly_mul(f, g, nthreads=NT, trunc=(N, mask))
        ex, cf, _, _ = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), path=path,
                                     trunc_degree=N, trunc_mask=mask)
        # the library returns graded order: compare both in plain lexicographic order
        ex, cf = to_np(ex), to_np(cf)
        a, b = np.lexsort(ex[::-1]), np.lexsort(r.exps[::-1])
        what = f"truncated N={N} mask={mask:b} path={path}"
        assert ex.shape == r.exps.shape, what
        assert np.array_equal(ex[:, a], r.exps[:, b]) and np.array_equal(cf[a], r.coef[b]), what


@pytest.mark.parametrize("path", [0, 1, 2])
def test_large_poisson_operands(kron, path):
    f = random_pseries(2, 2, 4000, 4, 4, 7201)
    g = random_pseries(2, 2, 3000, 4, 4, 7202)
    F = PSeries(*(dev(x) for x in (f.exps, f.trig, f.kind, f.coef)))
    G = PSeries(*(dev(x) for x in (g.exps, g.trig, g.kind, g.coef)))
    out = kron.poisson_mul(F, G, path=path)
    ro = oracle.poisson_mul(f, g, nthreads=NT, keep_zero=True)
    assert_pseries_close(tuple(to_np(x) for x in out[:4]), ro, 1e-12, f"large Poisson path={path}")


def test_graph_replay_with_cluster_front_end(kron, large):
    import torch
    f, g, r = large
    F = Poly(dev(f.exps), dev(f.coef))
    G = Poly(dev(g.exps), dev(g.coef))
    pb = kron.PreparedBatch([(F, G), (G, F)])
    try:
        for it in range(2):
            pb.launch()
            torch.cuda.synchronize()
            out = pb.results()
            for k in range(2):
                assert out[k]["status"] == 0
                assert_poly_equal(to_np(out[k]["exps"]), to_np(out[k]["coef"]), r, f"replay {it} product {k}")
    finally:
        pb.close()


@pytest.mark.parametrize("path", [0, 1, 2])
def test_operands_taking_several_rounds(kron, path):
    # 40000 terms: more than one term per thread of the cluster and round, so the
    # keys wait in the sort-key array between the passes
    f = random_poly(3, 40000, 0, 60, 7301)
    g = random_poly(3, 60, -5, 5, 7302)
    r = oracle.poly_mul(f, g, nthreads=NT)
    ctx = kron.binding.Context()
    ctx.set_profiling(True)
    try:
        ex, cf, _, _ = kron.poly_mul(dev(f.exps), dev(f.coef), dev(g.exps), dev(g.coef), ctx=ctx, path=path)
        assert "front" in [n for n, _ in ctx.stages()]
    finally:
        ctx.close()
    assert_poly_equal(to_np(ex), to_np(cf), r, f"several rounds path={path}")
    # a repeated key found in the second round
    exps = np.concatenate([f.exps, f.exps[:, 39990:39991]], axis=1)
    coef = np.concatenate([f.coef, f.coef[:1]])
    with pytest.raises(kron.KronError) as e:
        kron.poly_mul(dev(exps), dev(coef), dev(g.exps), dev(g.coef), path=path)
    assert e.value.status == kron.KR_ERR_DUP


def test_fateman_operands_on_the_cluster_front_end(kron):
    # Fateman's operands (46376 terms, key range 6.9e6 bits) are ranked by the
    # cluster front end; the product of a slice of f with all of g is checked
    from workloads import fateman
    f, g = fateman()
    fs = Poly(np.ascontiguousarray(f.exps[:, ::97]), np.ascontiguousarray(f.coef[::97]))
    r = oracle.poly_mul(fs, g, nthreads=NT)
    ctx = kron.binding.Context()
    ctx.set_profiling(True)
    try:
        ex, cf, _, _ = kron.poly_mul(dev(fs.exps), dev(fs.coef), dev(g.exps), dev(g.coef), ctx=ctx)
        assert "front" in [n for n, _ in ctx.stages()]
    finally:
        ctx.close()
    assert_poly_equal(to_np(ex), to_np(cf), r, "Fateman slice")
