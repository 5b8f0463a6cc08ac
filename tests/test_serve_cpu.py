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
