"""Continuous-batching request loop over kron_mul_batch.

Requests (pairs of series to multiply) arrive over time.  A dispatcher keeps a
FIFO of arrived requests and, whenever a worker is free, admits the oldest
ones into a batch as long as the batch's predicted scratch and output memory
stays within the memory still free (the budget minus what batches already on
the GPU hold).  Each worker owns a library context and a CUDA stream and runs
its batch with one kron_mul_batch call; while it runs (the call releases the
interpreter lock) the dispatcher forms and starts the next batch on another
worker, so the batches' work overlaps on the device.  Results stay on the
device: each request gets its own copy of its product (torch tensors).

The memory prediction per product is the term-product count times 16 bytes
times the observed ratio of output terms to term-products (updated after
every batch, separately for polynomials and Poisson series), plus the dense
array or hash table it needs.

A batch is also capped in work (term-products): the oldest waiting request
always starts the batch, and later requests join it only while the cap holds,
so a small request never waits behind a very large one in the same batch
and can overtake it on the other worker.  A request above `giant` term
products runs in a batch of its own.  With giant_policy "alone" it waits at
the head of the queue until no batch is running and no other batch starts
while it runs, so that it has the GPU to itself.  With "shared" it starts on
the first free worker (at most one such request at a time) and the other
workers go on serving the smaller requests meanwhile, which then never wait
behind it.  A batch of one request goes through the single-product call
(poly_mul / poisson_mul), which waits on the device once instead of three
times.  A worker releases its
context's cached scratch after a batch when it holds more than `trim_bytes`.
A worker whose batch runs out of device memory releases its context's cached
scratch, holds off new batches, waits until the other workers are idle and
runs the batch once more; a batch that fails again (or fails otherwise)
reports the failure on its requests instead of dropping them.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B


@dataclass
class Request:
    f: object
    g: object
    arrival: float            # seconds after the start of the run
    start: float = -1.0
    done: float = -1.0
    result: dict | None = None
    status: int = -1

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def pairs(self) -> int:
        return int(self.f.coef.shape[0]) * int(self.g.coef.shape[0])

    @property
    def poisson(self) -> bool:
        return hasattr(self.f, "trig")


@dataclass
class ServeStats:
    completed: int
    wall_s: float
    products_per_s: float
    p50_ms: float
    p99_ms: float
    mean_batch: float
    batches: int
    rejected: int = 0
    extra: dict = field(default_factory=dict)


class _Worker:
    def __init__(self, device: int):
        import torch
        self.ctx = B.Context(device)
        self.stream = torch.cuda.Stream(device=device)
        self.busy = False
        self.retrying = False
        self.thread = None


class Server:
    """Continuous batching over `workers` contexts on one GPU."""

    def __init__(self, device: int = 0, workers: int = 2, mem_budget: float = 64e9,
                 max_batch: int = 256, wave_pairs: int = 0, work_cap: float = 5e7,
                 giant: float = 2e7, trim_bytes: float = 96e9, giant_alone: bool = True,
                 giant_policy: str = "shared", queue_scale: int = 0, work_cap_max: float = 4e8):
        if giant_policy not in ("alone", "shared"):
            raise ValueError("giant_policy must be 'alone' or 'shared'")
        self.device = device
        self.work_cap = work_cap
        self.giant = giant
        self.giant_alone = giant_alone
        self.giant_policy = giant_policy
        self.giants_running = 0
        # queue_scale > 0: the work cap grows with the queue, work_cap * (1 + waiting /
        # queue_scale) up to work_cap_max, so that a long queue is drained in larger
        # batches (fewer launches and waits per product) while a short one keeps small
        # batches and their short latency
        self.queue_scale = queue_scale
        self.work_cap_max = work_cap_max
        self.trim_bytes = trim_bytes
        self.exclusive = False
        self.hold = 0             # workers retrying alone after running out of memory
        self.retry_lock = threading.Lock()
        self.errors: list[str] = []
        self.workers = [_Worker(device) for _ in range(workers)]
        self.mem_budget = mem_budget
        self.max_batch = max_batch
        self.wave_pairs = wave_pairs
        self.ratio = {False: 0.3, True: 1.0}   # output terms per term-product, learned
        self.lock = threading.Lock()
        self.in_flight_bytes = 0.0

    def warm_up(self, requests: list[Request], n: int = 2):
        """Runs the largest requests (by term-products: the n largest polynomial
        products and the n largest Poisson products) once on every worker, so
        that each context's scratch has grown before serving starts (a growth
        frees and allocates device memory, which waits for the whole device)."""
        for w in self.workers:
            with_torch_stream(w.stream, lambda: [self._mul(w, [r]) for r in largest(requests, n)])
            w.stream.synchronize()

    def close(self):
        """Release the workers' contexts (their scratch and results)."""
        for w in self.workers:
            if w.thread is not None:
                w.thread.join()
            w.ctx.close()

    def predict_bytes(self, r: Request) -> float:
        out_terms = r.pairs * self.ratio[r.poisson]
        # output (16 B) + ordering scratch (16 B) + table at load 0.5 (32 B) per term
        return 64.0 * out_terms + 1e6

    def _mul(self, w: _Worker, batch: list[Request], stream=None):
        stream = w.stream if stream is None else stream
        if len(batch) == 1 and hasattr(batch[0].f.coef, "is_cuda"):
            # one request: the single-product call (its outputs are the caller's tensors)
            r = batch[0]
            if r.poisson:
                e, t, k, c, _ = B.poisson_mul(r.f, r.g, ctx=w.ctx, stream=stream)
                return [{"status": 0, "nterms": int(c.shape[0]), "exps": e, "trig": t, "kind": k,
                         "coef": c, "owned": True}]
            e, c, _, _ = B.poly_mul(r.f.exps, r.f.coef, r.g.exps, r.g.coef, ctx=w.ctx, stream=stream)
            return [{"status": 0, "nterms": int(c.shape[0]), "exps": e, "coef": c, "owned": True}]
        return B.kron_mul_batch([(r.f, r.g) for r in batch], ctx=w.ctx, stream=stream,
                                wave_pairs=self.wave_pairs)

    def _retry_alone(self, w: _Worker, batch: list[Request]):
        """After running out of memory: free cached scratch, wait for the other
        workers to finish their batches (no new ones start), run once more."""
        import torch
        with self.lock:
            self.hold += 1
            w.retrying = True
        try:
            w.ctx.trim()
            with self.retry_lock:   # one retry at a time; others waiting here have trimmed too
                while any(x.busy and not x.retrying for x in self.workers if x is not w):
                    time.sleep(0.0005)
                torch.cuda.empty_cache()
                return self._mul(w, batch)
        finally:
            with self.lock:
                self.hold -= 1
                w.retrying = False

    def _shared_batch(self, pending: list[Request], room: float):
        """The next batch under giant_policy "shared": the oldest request that
        is very large, alone, when it is the oldest of all and no other very
        large one runs; otherwise the oldest smaller requests within the caps
        (very large ones keep their place)."""
        head = pending[0]
        if head.pairs > self.giant:
            if self.giants_running == 0:
                return [head], self.predict_bytes(head)
        cap = self.work_cap
        if self.queue_scale > 0:
            cap = min(self.work_cap_max, self.work_cap * (1 + len(pending) / self.queue_scale))
        batch, used, work = [], 0.0, 0.0
        for r in pending:
            if r.pairs > self.giant:
                continue
            b = self.predict_bytes(r)
            if not batch:
                if b > room and self.in_flight_bytes > 0:
                    break   # wait for memory to come back
            elif used + b > room or work + r.pairs > cap or len(batch) >= self.max_batch:
                continue    # later, smaller requests may still fit
            batch.append(r)
            used += b
            work += r.pairs
        return batch, used

    def _run_batch(self, w: _Worker, batch: list[Request], t0: float, bytes_: float):
        import torch
        out = None
        stream = w.stream
        try:
            with torch.cuda.stream(stream):
                now = time.perf_counter() - t0
                for r in batch:
                    r.start = now
                try:
                    out = self._mul(w, batch, stream)
                except B.KronError as e:
                    if e.status != B.KR_ERR_OOM:
                        raise
                    out = self._retry_alone(w, batch)
                # results are library-owned until the context's next batch: copy them out
                stream.synchronize()
                for r, o in zip(batch, out):
                    r.status = o["status"]
                    if o.get("owned"):
                        r.result = {k: v for k, v in o.items() if k != "owned"}
                    else:
                        r.result = {k: (v.clone() if hasattr(v, "clone") else v) for k, v in o.items()}
                stream.synchronize()
            done = time.perf_counter() - t0
            obs = {False: [0, 0], True: [0, 0]}
            for r, o in zip(batch, out):
                r.done = done
                obs[r.poisson][0] += o["nterms"]
                obs[r.poisson][1] += r.pairs
            with self.lock:
                for k, (n, p) in obs.items():
                    if p > 0:
                        self.ratio[k] = 0.7 * self.ratio[k] + 0.3 * max(n / p, 1e-4)
        except Exception as e:   # the batch failed as a whole: report it on every request
            done = time.perf_counter() - t0
            self.errors.append(f"{type(e).__name__}: {e}"[:200])
            for r in batch:
                if r.done < 0:
                    r.status = getattr(e, "status", -2)
                    r.done = done
                    r.result = None
        finally:
            try:
                if w.ctx.scratch_bytes() > self.trim_bytes:
                    w.ctx.trim()
            except Exception:
                pass
            with self.lock:
                self.in_flight_bytes -= bytes_
                if any(r.pairs > self.giant for r in batch):
                    self.exclusive = False
                    if self.giant_policy == "shared":
                        self.giants_running -= 1
                w.busy = False

    def run(self, requests: list[Request], time_limit: float = 120.0) -> ServeStats:
        """Serve requests (sorted by arrival) until all are done or time_limit passes."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending: list[Request] = []
        nxt = 0
        batches = 0
        sizes = []
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            if nxt >= len(reqs) and not pending and all(not w.busy for w in self.workers):
                break
            if now > time_limit:
                break
            free = [w for w in self.workers if not w.busy]
            if self.exclusive or self.hold:
                free = []
            if pending and free:
                with self.lock:
                    room = self.mem_budget - self.in_flight_bytes
                batch, used, work = [], 0.0, 0.0
                idle = all(not w.busy for w in self.workers)
                if self.giant_policy == "shared":
                    batch, used = self._shared_batch(pending, room)
                    if batch:
                        taken = set(id(r) for r in batch)
                        pending = [r for r in pending if id(r) not in taken]
                        w = free[0]
                        with self.lock:
                            w.busy = True
                            self.in_flight_bytes += used
                            if batch[0].pairs > self.giant:
                                self.giants_running += 1
                        w.thread = threading.Thread(target=self._run_batch, args=(w, batch, t0, used))
                        w.thread.start()
                        batches += 1
                        sizes.append(len(batch))
                        continue
                    time.sleep(0.0002)   # nothing may start now
                    continue
                elif pending[0].pairs > self.giant and not idle and self.giant_alone:
                    # the oldest request is very large: no new batch starts
                    # until the GPU is free, then it runs alone
                    time.sleep(0.0002)
                    continue
                if pending[0].pairs > self.giant:
                    # the oldest request is very large: it starts on the free
                    # worker and no new batch starts until it is done
                    batch.append(pending[0])
                    used += self.predict_bytes(pending[0])
                for r in ([] if pending[0].pairs > self.giant else pending):
                    b = self.predict_bytes(r)
                    if r.pairs > self.giant:
                        continue
                    if not batch:
                        if b > room and self.in_flight_bytes > 0:
                            break   # wait for memory to come back
                    elif (used + b > room or work + r.pairs > self.work_cap
                          or len(batch) >= self.max_batch):
                        continue    # later, smaller requests may still fit
                    batch.append(r)
                    used += b
                    work += r.pairs
                if batch:
                    if batch[0].pairs > self.giant:
                        self.exclusive = True
                    taken = set(id(r) for r in batch)
                    pending = [r for r in pending if id(r) not in taken]
                    w = free[0]
                    with self.lock:
                        w.busy = True
                        self.in_flight_bytes += used
                    w.thread = threading.Thread(target=self._run_batch, args=(w, batch, t0, used))
                    w.thread.start()
                    batches += 1
                    sizes.append(len(batch))
                    continue
            if not pending and nxt < len(reqs):
                time.sleep(max(0.0, min(reqs[nxt].arrival - now, 0.002)))
            else:
                time.sleep(0.0002)
        for w in self.workers:
            if w.thread is not None:
                w.thread.join()
        wall = time.perf_counter() - t0
        done = [r for r in reqs if r.done >= 0 and r.status == 0]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        failed = sum(1 for r in reqs if r.done >= 0 and r.status != 0)
        return ServeStats(completed=len(done), wall_s=wall,
                          extra={"failed": failed, "errors": sorted(set(self.errors))[:3]},
                          products_per_s=len(done) / wall if wall > 0 else 0.0,
                          p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                          mean_batch=float(np.mean(sizes)) if sizes else 0.0, batches=batches,
                          rejected=len(reqs) - len(done))


def largest(requests: list[Request], n: int) -> list[Request]:
    """The n largest polynomial and the n largest Poisson requests by term-products."""
    out = []
    for poisson in (False, True):
        rs = sorted((r for r in requests if r.poisson == poisson), key=lambda r: -r.pairs)
        out += rs[:n]
    return out


def with_torch_stream(stream, fn):
    import torch
    with torch.cuda.stream(stream):
        return fn()


def _single(ctx, r: Request):
    if r.poisson:
        return B.poisson_mul(r.f, r.g, ctx=ctx)
    return B.poly_mul(r.f.exps, r.f.coef, r.g.exps, r.g.coef, ctx=ctx)


def serve_one_by_one(requests: list[Request], device: int = 0, time_limit: float = 120.0,
                     warm: bool = False) -> ServeStats:
    """The baseline: one poly_mul / poisson_mul call per request, in arrival
    order (warm: the largest requests run once first, untimed, as the server's
    warm_up does)."""
    import torch
    ctx = B.Context(device)
    if warm:
        for r in largest(requests, 2):
            _single(ctx, r)
        torch.cuda.synchronize()
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if now > time_limit:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.start = time.perf_counter() - t0
        r.result = _single(ctx, r)
        r.status = 0
        r.done = time.perf_counter() - t0
    wall = time.perf_counter() - t0
    ctx.close()
    done = [r for r in reqs if r.done >= 0]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    return ServeStats(completed=len(done), wall_s=wall, products_per_s=len(done) / wall if wall > 0 else 0.0,
                      p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                      mean_batch=1.0, batches=len(done), rejected=len(reqs) - len(done))
