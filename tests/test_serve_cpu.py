"""Host logic of the continuous-batching server, with the library call faked (CPU)."""
import threading

import numpy as np
import torch

from paper_1004_4548_gb300 import binding as B
from paper_1004_4548_gb300 import serve
from workloads import Poly


class _FakeCtx:
    def __init__(self, *a, **k):
        self.trims = 0

    def trim(self):
        self.trims += 1

    def scratch_bytes(self):
        return 0

    def close(self):
        pass


class _FakeStream:
    def synchronize(self):
        pass


class _FakeWorker:
    def __init__(self, device):
        self.ctx = _FakeCtx()
        self.stream = _FakeStream()
        self.busy = False
        self.retrying = False
        self.thread = None


def _requests(n, big_every=0):
    reqs = []
    for i in range(n):
        m = 400 if big_every and i % big_every == 0 else 3
        f = Poly(np.zeros((1, m), np.int32), np.ones(m, np.int64))
        reqs.append(serve.Request(f, f, arrival=0.0005 * i))
    return reqs


def _fake_batch(fail_first_oom: set, fail_always: bool, calls: list, lock):
    def run(pairs, ctx=None, stream=None, wave_pairs=0):
        with lock:
            calls.append(len(pairs))
            big = any(f.coef.shape[0] > 100 for f, _ in pairs)
            key = id(ctx)
            if big and (fail_always or key not in fail_first_oom):
                fail_first_oom.add(key)
                raise B.KronError(B.KR_ERR_OOM, "kron_mul_batch: out of memory (fake)")
        return [{"status": 0, "nterms": 1, "coef": torch.ones(1)} for _ in pairs]
    return run


def test_oom_batch_is_retried_alone(monkeypatch):
    monkeypatch.setattr(serve, "_Worker", _FakeWorker)
    calls, lock = [], threading.Lock()
    monkeypatch.setattr(B, "kron_mul_batch", _fake_batch(set(), False, calls, lock))
    srv = serve.Server(workers=2, giant=1e12)
    st = srv.run(_requests(60, big_every=20), time_limit=30)
    assert st.completed == 60 and st.extra["failed"] == 0
    assert sum(w.ctx.trims for w in srv.workers) >= 1
    assert srv.hold == 0 and not any(w.retrying for w in srv.workers)


def test_batch_failing_twice_reports_its_requests(monkeypatch):
    monkeypatch.setattr(serve, "_Worker", _FakeWorker)
    calls, lock = [], threading.Lock()
    monkeypatch.setattr(B, "kron_mul_batch", _fake_batch(set(), True, calls, lock))
    srv = serve.Server(workers=2, giant=1e12)
    reqs = _requests(40, big_every=10)
    st = srv.run(reqs, time_limit=30)
    failed = [r for r in reqs if r.status == B.KR_ERR_OOM]
    assert failed and all(any(x is r for x in reqs) for r in failed)
    assert st.completed + st.extra["failed"] == 40
    assert all(r.done >= 0 for r in reqs)


def _recording_batch(log: list, lock, active: list, delay=0.0005):
    """A fake library call that records every batch (its requests' term-product
    counts and how many batches ran at the same time) and answers each product
    with its own pair count, so that results can be matched to requests."""
    import time

    def run(pairs, ctx=None, stream=None, wave_pairs=0):
        with lock:
            active[0] += 1
            log.append(([f.coef.shape[0] * g.coef.shape[0] for f, g in pairs], active[0]))
        time.sleep(delay)
        with lock:
            active[0] -= 1
        return [{"status": 0, "nterms": int(f.coef.shape[0] * g.coef.shape[0]),
                 "coef": torch.ones(1)} for f, g in pairs]
    return run


def _mixed_requests(n, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        m = int(rng.choice([2, 5, 20, 900]))
        f = Poly(np.zeros((1, m), np.int32), np.ones(m, np.int64))
        g = Poly(np.zeros((1, m), np.int32), np.ones(m, np.int64))
        reqs.append(serve.Request(f, g, arrival=0.0002 * i))
    return reqs


def test_giants_run_alone_and_results_match_requests(monkeypatch):
    monkeypatch.setattr(serve, "_Worker", _FakeWorker)
    log, lock, active = [], threading.Lock(), [0]
    monkeypatch.setattr(B, "kron_mul_batch", _recording_batch(log, lock, active))
    srv = serve.Server(workers=2, giant=500_000, giant_policy="alone")   # 900 x 900 = 810,000 pairs: a giant
    reqs = _mixed_requests(120)
    st = srv.run(reqs, time_limit=60)
    assert st.completed == 120 and st.extra["failed"] == 0
    for sizes, concurrent in log:
        if any(p > 500_000 for p in sizes):
            assert len(sizes) == 1 and concurrent == 1, (sizes, concurrent)
    assert sum(len(s) for s, _ in log) == 120
    for r in reqs:
        assert r.status == 0 and r.result["nterms"] == r.pairs


def test_batches_respect_the_work_and_memory_caps(monkeypatch):
    monkeypatch.setattr(serve, "_Worker", _FakeWorker)
    log, lock, active = [], threading.Lock(), [0]
    monkeypatch.setattr(B, "kron_mul_batch", _recording_batch(log, lock, active, delay=0.002))
    work_cap, budget = 1000.0, 5e6
    srv = serve.Server(workers=2, giant=1e12, work_cap=work_cap, mem_budget=budget, max_batch=8)
    reqs = [serve.Request(Poly(np.zeros((1, m), np.int32), np.ones(m, np.int64)),
                          Poly(np.zeros((1, m), np.int32), np.ones(m, np.int64)), arrival=0.0)
            for m in [5] * 40 + [20] * 10]
    st = srv.run(reqs, time_limit=60)
    assert st.completed == 50
    for sizes, _ in log:
        assert len(sizes) <= 8
        if len(sizes) > 1:
            assert sum(sizes) <= work_cap
    # a 5 MB budget admits at most four requests of the 1 MB-plus prediction at once
    assert max(len(s) for s, _ in log) <= 4
    # arrival order is kept among requests that fit: the first batch starts with the oldest
    assert log[0][0][0] == 25


def test_shared_policy_runs_one_giant_at_a_time_beside_small_batches(monkeypatch):
    """giant_policy "shared": a very large request starts on a free worker
    without waiting for the others, never beside another very large one, and
    smaller requests keep being served on the other worker meanwhile."""
    import time
    monkeypatch.setattr(serve, "_Worker", _FakeWorker)
    lock = threading.Lock()
    state = {"giants": 0, "max_giants": 0, "small_beside_giant": 0, "batches": []}

    def run(pairs, ctx=None, stream=None, wave_pairs=0):
        sizes = [f.coef.shape[0] * g.coef.shape[0] for f, g in pairs]
        giant = any(p > 500_000 for p in sizes)
        with lock:
            state["batches"].append(sizes)
            if giant:
                state["giants"] += 1
                state["max_giants"] = max(state["max_giants"], state["giants"])
            elif state["giants"]:
                state["small_beside_giant"] += 1
        time.sleep(0.004 if giant else 0.0005)
        with lock:
            if giant:
                state["giants"] -= 1
        return [{"status": 0, "nterms": int(p), "coef": torch.ones(1)} for p in sizes]

    monkeypatch.setattr(B, "kron_mul_batch", run)
    srv = serve.Server(workers=2, giant=500_000, giant_policy="shared")
    reqs = _mixed_requests(160, seed=3)
    st = srv.run(reqs, time_limit=60)
    assert st.completed == 160 and st.extra["failed"] == 0
    assert state["max_giants"] == 1
    assert state["small_beside_giant"] > 0
    for sizes in state["batches"]:
        if any(p > 500_000 for p in sizes):
            assert len(sizes) == 1
    for r in reqs:
        assert r.status == 0 and r.result["nterms"] == r.pairs
