"""The batched entry point, the served loop and graph replays: every product
of a mixed batch is checked against the oracle (int64 bit-exact; float64
Poisson products within 1e-12 of the summed magnitudes), across wave splits,
arrival orders, replays, and with invalid or empty jobs in the mix."""
import os

import numpy as np
import pytest

import oracle
from gpu_compare import assert_poly_equal, assert_pseries_close
from workloads import PSeries, Poly, batch_mix, random_poly

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


@pytest.fixture(scope="module")
def mix():
    return batch_mix(96, seed_base=5000, max_terms=700)


_oracle_cache = {}


def _oracle(f, g, scale=1):
    """The oracle's product, cached per operand pair (the cache keeps the
    operands alive, so their ids stay theirs); scale multiplies f's coefficients."""
    key = (id(f), id(g), scale)
    if key not in _oracle_cache:
        if isinstance(f, PSeries):
            fs = PSeries(f.exps, f.trig, f.kind, f.coef * scale)
            r = oracle.poisson_mul(fs, g, nthreads=NT, keep_zero=True)
        else:
            r = oracle.poly_mul(Poly(f.exps, f.coef * scale), g, nthreads=NT)
        _oracle_cache[key] = (f, g, r)
    return _oracle_cache[key][2]


def _check_one(f, g, r, what, scale=1):
    ro = _oracle(f, g, scale)
    if isinstance(f, PSeries):
        assert_pseries_close((r["exps"], r["trig"], r["kind"], r["coef"]), ro, 1e-12, what)
    else:
        assert_poly_equal(r["exps"], r["coef"], ro, what)


def _check_batch(kron, mix, out, what):
    for i, ((f, g), r) in enumerate(zip(mix, out)):
        assert r["status"] == 0, f"{what}: product {i} status {r['status']}"
        _check_one(f, g, r, f"{what} product {i}")


def test_batch_equals_alone(kron, mix):
    out = kron.kron_mul_batch(mix)
    _check_batch(kron, mix, out, "one wave")


def test_batch_waves(kron, mix):
    out = kron.kron_mul_batch(mix, wave_pairs=2_000_000)
    _check_batch(kron, mix[:48], out[:48], "small waves")


def test_batch_arrival_order_does_not_matter(kron, mix):
    perm = np.random.default_rng(5).permutation(len(mix))
    b = kron.kron_mul_batch([mix[i] for i in perm])
    for j, i in enumerate(perm):
        f, g = mix[i]
        assert b[j]["status"] == 0
        _check_one(f, g, b[j], f"permuted batch, product {i}")


def test_batch_per_job_errors(kron):
    f = random_poly(3, 200, -4, 4, 71)
    g = random_poly(3, 150, -4, 4, 72)
    bad = Poly(np.concatenate([f.exps, f.exps[:, :1]], axis=1), np.concatenate([f.coef, f.coef[:1]]))
    empty = Poly(np.zeros((3, 0), np.int32), np.zeros(0, np.int64))
    out = kron.kron_mul_batch([(f, g), (bad, g), (empty, g), (g, f)])
    assert out[0]["status"] == 0 and out[3]["status"] == 0
    assert out[1]["status"] == kron.KR_ERR_DUP
    assert out[2]["status"] == 0 and out[2]["nterms"] == 0
    r = oracle.poly_mul(f, g)
    assert_poly_equal(out[0]["exps"], out[0]["coef"], r, "beside failing jobs")
    assert_poly_equal(out[3]["exps"], out[3]["coef"], r, "commuted")


def test_served_results_equal_alone(kron):
    """Requests served by the continuous-batching loop (two workers, batches
    overlapping on the GPU) return the same products as one call each."""
    import torch
    from paper_1004_4548_gb300.serve import Request, Server
    from workloads import arrival_times
    mix = batch_mix(40, seed_base=7000, max_terms=400)

    def dev(p):
        if isinstance(p, PSeries):
            return PSeries(*(torch.from_numpy(x).cuda() for x in (p.exps, p.trig, p.kind, p.coef)))
        return Poly(torch.from_numpy(p.exps).cuda(), torch.from_numpy(p.coef).cuda())

    t = arrival_times(len(mix), rate=400.0, seed=11)
    reqs = [Request(dev(f), dev(g), float(a)) for (f, g), a in zip(mix, t)]
    stats = Server(workers=2, max_batch=8, mem_budget=8e9).run(reqs, time_limit=60.0)
    assert stats.completed == len(mix) and stats.batches >= 2
    for i, ((f, g), r) in enumerate(zip(mix, reqs)):
        assert r.status == 0
        _check_one(f, g, r.result, f"served {i}")


def test_prepared_batch_graph_replay(kron):
    """A batch captured into a CUDA graph: the replay reproduces the prepared
    results, and replays again correctly after the coefficients change in place
    (doubling every f coefficient doubles every product coefficient exactly)."""
    import torch
    mix = batch_mix(24, seed_base=8000, max_terms=500)

    def dev(p):
        if isinstance(p, PSeries):
            return PSeries(*(torch.from_numpy(x.copy()).cuda() for x in (p.exps, p.trig, p.kind, p.coef)))
        return Poly(torch.from_numpy(p.exps.copy()).cuda(), torch.from_numpy(p.coef.copy()).cuda())

    D = [(dev(f), dev(g)) for f, g in mix]
    pb = kron.PreparedBatch(D)
    for i, (a, (f, g)) in enumerate(zip(pb.first_results(), mix)):
        assert a["status"] == 0
        _check_one(f, g, a, f"prepared run, product {i}")
    for it in range(2):
        pb.launch()
        torch.cuda.synchronize()
        for i, (a, (f, g)) in enumerate(zip(pb.results(), mix)):
            assert a["status"] == 0, f"replay {it} product {i}: status {a['status']}"
            _check_one(f, g, a, f"replay {it}, product {i}")
    for f, g in D:
        f.coef.mul_(2)
    pb.launch()
    torch.cuda.synchronize()
    for i, (a, (f, g)) in enumerate(zip(pb.results(), mix)):
        assert a["status"] == 0
        _check_one(f, g, a, f"replay with doubled f, product {i}", scale=2)
    pb.close()
