"""Benchmark: term-products per second of sparse polynomial multiplication on GB300.

One step = one call of the library's poly_mul on the dense-path workload
(two 4-variable polynomials with every monomial of total degree <= 20, 10626
terms each, int64 coefficients in [-2^20, 2^20]; 112,911,876 term-products,
135,751 output terms): range scan, host plan, Kronecker encode, sort, dense
block planning, shared-memory accumulation, compaction and decode of the
product into device buffers.  Inputs are resident in HBM when the timed
region starts; L2 is flushed (a 256 MB write) between timed steps.

The line also carries the hash path (Monagan-Pearce sparse structure) and the
Poisson path as secondary measurements under "paths".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own replica of the workload (independent
products, no collective on the data path): "scaling": "weak".  With several
ranks the line also carries "sharded": one large product (full-size
Fateman) split over the ranks by output key window and gathered with one
all_gather, strong scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "M term-products/s (dense path, moderately sparse workload)"
UNIT = "M term-products/s"
WORKLOAD = ("dense path: f, g = all 4-variable monomials of total degree <= 20 "
            "(10626 terms each), int64 coefficients uniform in [-2^20, 2^20], seeds 2001/2002")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-paths", action="store_true", help="skip the secondary hash/Poisson lines")
    ap.add_argument("--paths", default="", help="comma-separated subset of the secondary lines (default: all)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline (profiler runs)")
    ap.add_argument("--block-slots", type=int, default=0, help="dense output block size (0 = library default)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched / served measurements")
    ap.add_argument("--batch-products", type=int, default=4096, help="products in the uneven batch")
    ap.add_argument("--cpu-full", action="store_true",
                    help="time the oracle on the whole dense and hash workloads, one thread and every core, and exit")
    ap.add_argument("--case", default="", choices=["", "cfg3", "cfg4s", "cfg4", "cfg4h", "cfg2"],
                    help="profiling runs: time only this case (cfg4s = cfg4 at 5000 terms, cfg4h = cfg4 on "
                         "the hash path, cfg2 = the headline product)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch of k_dense_accum on this workload, from
# one ncu capture of the kernel on it; valid only for the kernel source it was
# taken on, identified by the leading hex digits of its SHA-256.
DENSE_TRAFFIC = {"source": "kr_dense.cu", "source_sha256": "9d91294c0d87e967", "bytes": 2740480}
# DRAM traffic of the polynomial hash insert kernel on the MP-sparse product,
# per launch (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture)
HASH_TRAFFIC = {"source": "kr_hash.cu", "source_sha256": "5724b523f77891fd", "bytes": 590288640 + 641475328}


def kernel_traffic(rec):
    """A recorded DRAM traffic figure, or None once the kernel's source differs
    from the one the counters were taken on."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_1004_4548_gb300", "csrc", rec["source"]), "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    return rec["bytes"] if rec["source_sha256"] and sha.startswith(rec["source_sha256"]) else None


def dense_traffic():
    return kernel_traffic(DENSE_TRAFFIC)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
# The oracle's sample of the workload: a fixed slice, so that every run (and
# both arms) times the same work.  The multi-threaded rate still depends on
# the slice (thread start-up and the final merge of the per-thread maps are
# amortised over it), which is why it is fixed rather than sized by a budget.
CPU_SAMPLE_MT = 4096   # f terms x all g terms, every core
CPU_SAMPLE_ST = 512    # f terms x all g terms, one thread


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(f, g, single: bool = True):
    """The oracle on the host's cores over the fixed sample (and on one thread)."""
    import oracle
    from workloads import Poly
    cores = os.cpu_count() or 1

    def rate(m, threads):
        fs = Poly(np.ascontiguousarray(f.exps[:, :m]), f.coef[:m].copy())
        t = time.perf_counter()
        oracle.poly_mul(fs, g, nthreads=threads)
        dt = time.perf_counter() - t
        return m * g.n / dt / 1e6, dt

    m = min(f.n, CPU_SAMPLE_MT)
    v, dt = rate(m, cores)
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"first {m} of {f.n} f terms x all {g.n} g terms of the workload "
                     f"({m * g.n} term-products, {dt:.2f} s, std::map oracle, {cores} threads)"}
    if single:
        m1 = min(f.n, CPU_SAMPLE_ST)
        v1, dt1 = rate(m1, 1)
        out["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                "sample": f"first {m1} f terms x all {g.n} g terms "
                                          f"({m1 * g.n} term-products, {dt1:.2f} s)"}
    return out


def cpu_full():
    """The oracle on the whole dense (degree 20) and hash (MP-sparse) workloads,
    one thread and every core: one JSON line per run."""
    import oracle
    from workloads import workload_cfg2, workload_cfg3
    cores = os.cpu_count() or 1
    model = cpu_model()
    for name, (f, g) in (("dense path, degree-20 workload", workload_cfg2()),
                         ("hash path, MP-sparse workload", workload_cfg3())):
        for threads in (cores, 1):
            t = time.perf_counter()
            r = oracle.poly_mul(f, g, nthreads=threads)
            dt = time.perf_counter() - t
            print(json.dumps({"cpu_full": name, "threads": threads, "cpu_model": model, "seconds": dt,
                              "term_products": f.n * g.n, "output_terms": int(r.coef.shape[0]),
                              "value": f.n * g.n / dt / 1e6, "unit": UNIT}), flush=True)


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from workloads import workload_cfg2
    f, g = workload_cfg2()
    vals = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(f, g, single=(i == args.warmup + args.steps - 1))
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    # each step times a bounded sample; ms_per_step is the time the whole workload
    # (all f x g term-products) takes at the measured rate
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f.n * g.n / (v * 1e6) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.cpu_full:
        cpu_full()
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import ctypes
    import paper_1004_4548_gb300 as kron
    from paper_1004_4548_gb300 import binding as B
    from workloads import workload_cfg2, workload_cfg3, workload_cfg4, PSeries, fateman

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.case:
        profile_case(args)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    ctx = kron.Context(local)
    L = ctx.L

    f, g = workload_cfg2()
    tp = f.n * g.n
    fe, fc = torch.from_numpy(f.exps).to(dev), torch.from_numpy(f.coef).to(dev)
    ge, gc = torch.from_numpy(g.exps).to(dev), torch.from_numpy(g.coef).to(dev)
    F = B.kr_poly(4, f.n, fe.data_ptr(), fc.data_ptr(), B.KR_I64)
    G = B.kr_poly(4, g.n, ge.data_ptr(), gc.data_ptr(), B.KR_I64)
    # output buffers sized by a first call
    ex0, cf0, _, _ = kron.poly_mul(fe, fc, ge, gc, ctx=ctx)
    nout = int(cf0.shape[0])
    oe = torch.empty((4, nout), dtype=torch.int32, device=dev)
    oc = torch.empty((nout,), dtype=torch.int64, device=dev)
    H = B.kr_poly_out(4, nout, 0, oe.data_ptr(), oc.data_ptr(), None)
    O = B.kr_opts()
    O.block_slots = args.block_slots
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        st = L.poly_mul(ctx.h, ctypes.byref(F), ctypes.byref(G), ctypes.byref(H), ctypes.byref(O), sp)
        if st != 0:
            raise RuntimeError(f"poly_mul failed: {st} {L.kr_last_error(ctx.h).decode()}")

    for _ in range(max(3, args.warmup)):
        step()
    assert int(H.nterms) == nout
    # ---- timed region
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    accum_ms = []
    l0 = ctx.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - l0
    # the dominant kernel's duration: the library's CUDA events around it, on
    # the launch stream, in a separate pass (the events are not in the timed loop)
    ctx.set_profiling(True)
    for i in range(args.steps):
        flush.zero_()
        step()
        accum_ms.extend(ms for name, ms in ctx.stages() if name == "dense_accum")
    stages = ctx.stages()
    ctx.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = world * tp / (ms * 1e-3) / 1e6

    # ---- roofline of the dominant kernel (dense accumulation): one int64
    # shared-memory accumulate per term-product, in the kernel's form (two
    # 32-bit atomics with a carry); the peak is that accumulate's measured
    # conflict-free chip-wide rate
    peak_smem = kron.kr_probe_smem_accumulate_rate(local, 5)
    peak_64 = kron.kr_probe_smem_atomic_rate(local, False, 5)
    acc_ms = statistics.mean(accum_ms) if accum_ms else float("nan")
    achieved = tp / (acc_ms * 1e-3) / 1e9   # G shared-memory accumulates (term-products) per second
    roof = {"bound": "alu", "kernel": "k_dense_accum",
            "achieved": achieved, "peak": peak_smem / 1e9, "unit": "G smem-accumulates/s",
            "frac": achieved / (peak_smem / 1e9) if peak_smem > 0 else None,
            "peak_source": "measured: kr_probe_smem_accumulate_rate (conflict-free int64 accumulates as "
                           "two 32-bit shared-memory atomics with carry, all SMs, best of 5)",
            "peak_64bit_atomic_adds": peak_64 / 1e9,
            # the other denominators of the accumulate: the multiply-add forms, in G ops/s
            "peak_int64_muladd": kron.kr_probe_alu_rate(0, local, 3) / 1e9,
            "peak_imad_wide_32x32": kron.kr_probe_alu_rate(1, local, 3) / 1e9,
            "peak_fp64_fma": kron.kr_probe_alu_rate(2, local, 3) / 1e9,
            "peak_f64_smem_atomic_adds": kron.kr_probe_smem_atomic_rate(local, True, 3) / 1e9,
            "kernel_ms": acc_ms, "algorithmic_units_per_launch": tp,
            "traffic": dense_traffic()}

    # ---- end to end through the C ABI with pinned host buffers
    hfe = torch.from_numpy(f.exps).pin_memory(); hfc = torch.from_numpy(f.coef).pin_memory()
    hge = torch.from_numpy(g.exps).pin_memory(); hgc = torch.from_numpy(g.coef).pin_memory()
    hoe = torch.empty((4, nout), dtype=torch.int32).pin_memory()
    hoc = torch.empty((nout,), dtype=torch.int64).pin_memory()
    Fh = B.kr_poly(4, f.n, hfe.data_ptr(), hfc.data_ptr(), B.KR_I64)
    Gh = B.kr_poly(4, g.n, hge.data_ptr(), hgc.data_ptr(), B.KR_I64)
    Hh = B.kr_poly_out(4, nout, 0, hoe.data_ptr(), hoc.data_ptr(), None)
    ctx.set_profiling(False)

    def step_host():
        st = L.poly_mul(ctx.h, ctypes.byref(Fh), ctypes.byref(Gh), ctypes.byref(Hh), ctypes.byref(O), sp)
        if st != 0:
            raise RuntimeError(f"poly_mul (host buffers) failed: {st}")

    for _ in range(3):
        step_host()
    e2e_ms = []
    for i in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step_host()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    assert np.array_equal(hoc.numpy(), oc.cpu().numpy()), "host-buffer result differs"
    e2e = {"value": world * tp / (statistics.mean(e2e_ms) * 1e-3) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(f.exps.nbytes + f.coef.nbytes + g.exps.nbytes + g.coef.nbytes),
           "d2h_bytes_per_step": int(hoe.numel() * 4 + hoc.numel() * 8),
           "ms_per_step": statistics.mean(e2e_ms)}

    # ---- secondary paths
    paths = {}
    if not args.no_paths:
        want = set(args.paths.split(",")) if args.paths else None
        sel = lambda name: want is None or name in want
        ctx.set_profiling(True)
        hbm = measured_peaks().get("hbm_gbs")
        if sel("hash_cfg3"):
            h3 = time_poly(kron, ctx, *workload_cfg3(), dev, stream, flush, "hash_insert",
                           max(3, args.steps // 2))
            # 24 B per term-product: an 8 B key probe read, an 8 B coefficient read and write
            roof3 = hbm_roofline("k_hash_insert_poly", h3["term_products"], h3["kernel_ms"], 24, hbm,
                                 kernel_traffic(HASH_TRAFFIC))
            # the ceiling of the same insert routine on random keys, at this product's
            # table size (2^24 slots) and key count, and of plain random adds
            ins = kron.kr_probe_table_update_rate(24, h3["output_terms"], h3["term_products"], 0, local, 3)
            add = kron.kr_probe_table_update_rate(24, h3["output_terms"], h3["term_products"], 1, local, 3)
            roof3["ceiling_insert_per_s"] = ins
            roof3["ceiling_random_add_per_s"] = add
            # the same random insert-or-adds into a table L2 holds (2^22 slots, 64 MB)
            roof3["ceiling_insert_l2_table_per_s"] = kron.kr_probe_table_update_rate(
                22, 1 << 21, h3["term_products"], 0, local, 3)
            roof3["frac_of_insert_ceiling"] = (h3["term_products"] / (h3["kernel_ms"] * 1e-3)) / ins \
                if ins > 0 else None
            h3["roofline"] = roof3
            paths["hash_cfg3"] = h3
        if sel("poisson_cfg4") or sel("poisson_cfg4_hash") or sel("poisson_cfg4_truncated"):
            f4, g4 = workload_cfg4()
            if sel("poisson_cfg4"):
                p4 = time_pseries(kron, ctx, f4, g4, dev, stream, flush, 3, hbm_gbs=hbm)
                # second denominator: random float64 adds into a key-indexed array of
                # 2^32 8-byte slots (34 GB; the product's array is 46.6 GB), two per pair
                upd = 2 * p4["term_products"]
                ceil = kron.kr_probe_table_update_rate(32, min(p4["output_terms"], (7 << 32) // 10), upd, 2,
                                                       local, 3)
                p4["roofline"]["ceiling_random_f64_add_per_s"] = ceil
                p4["roofline"]["frac_of_update_ceiling"] = (upd / (p4["kernel_ms"] * 1e-3)) / ceil \
                    if ceil > 0 else None
                paths["poisson_cfg4"] = p4
            if sel("poisson_cfg4_hash"):
                p4h = time_pseries(kron, ctx, f4, g4, dev, stream, flush, 3, path=kron.KR_PATH_HASH,
                                   hbm_gbs=hbm)
                # second denominator: random insert-or-adds (the insert routine, as the
                # polynomial kernel issues them) into 2^30 16-byte slots, two per pair
                upd = 2 * p4h["term_products"]
                ceil = kron.kr_probe_table_update_rate(30, min(p4h["output_terms"], (7 << 30) // 10), upd, 0,
                                                       local, 3)
                p4h["roofline"]["ceiling_insert_per_s"] = ceil
                p4h["roofline"]["frac_of_insert_ceiling"] = (upd / (p4h["kernel_ms"] * 1e-3)) / ceil \
                    if ceil > 0 else None
                paths["poisson_cfg4_hash"] = p4h
            if sel("poisson_cfg4_truncated"):
                # Sec. 3's truncation of a Poisson product: pairs with |C_f C_g| >= 1e-38 (about 14%
                # of them; the magnitudes fall with the exponents and multipliers) and terms of
                # harmonic order <= 20; the rate counts every pair of the product
                paths["poisson_cfg4_truncated"] = time_pseries(kron, ctx, f4, g4, dev, stream, flush, 3,
                                                               hbm_gbs=hbm, kernel_name="k_hash_insert_trunc",
                                                               harmonic_order=20, coef_min=1e-38)
                paths["poisson_cfg4_truncated"]["context"] = (
                    "the Poisson workload truncated by coefficient magnitude (|C_f C_g| >= 1e-38) and "
                    "harmonic order (<= 20); units are all 4e8 pairs of the untruncated product")
        fa, ga = fateman()
        if sel("fateman_full"):
            paths["fateman_full"] = time_poly(kron, ctx, fa, ga, dev, stream, flush, "dense_accum", 5)
            paths["fateman_full"]["context"] = ("Fateman's benchmark, (1+x+y+z+t)^30 times itself plus one, "
                                                "true coefficients modulo 2^64; the paper's Table 5: 4.29 s "
                                                "on one Core2Quad core with double coefficients")
        if sel("fateman_truncated"):
            # the same product truncated at total degree 30 (Sec. 3): only the pairs whose degrees
            # add up to at most 30 are multiplied; the rate counts those pairs
            paths["fateman_truncated"] = time_poly(kron, ctx, fa, ga, dev, stream, flush, "dense_accum", 5,
                                                   units=kept_pairs(fa, ga, 30), trunc_degree=30)
            paths["fateman_truncated"]["context"] = ("Fateman's product truncated at total degree 30: "
                                                     "term-products counted over the kept pairs")
        if sel("cfg2_windows4"):
            # the headline product as 4 output key windows of equal sampled work, one call each
            # (what 4 ranks of a split run compute), the sampling of the split included
            paths["cfg2_windows4"] = time_windows(kron, ctx, f, g, dev, stream, flush, 4, max(3, args.steps // 2))
        ctx.set_profiling(False)

    batched = None
    if not args.no_batch:
        ctx.trim()
        batched = time_batched(kron, ctx, dev, args.batch_products)

    # ---- one product split over the ranks (only with several ranks)
    sharded = None
    if world > 1 and not args.no_paths:
        sharded = time_sharded(kron, ctx, dev, stream, world, rank, max(3, args.steps // 2), 2)
    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "term_products": tp, "output_terms": nout,
                           "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roof,
                "e2e": e2e, "gpu_launches": launches,
                "clocks": clk,
                "stages_ms_last_step": {k: round(v, 4) for k, v in stages},
                "wall_s_timed": wall,
                "sm_cycles_per_term_product": (clk["sm_mhz"] * 1e6 * ms * 1e-3 / tp * num_sms)
                if clk.get("sm_mhz") else None,
                "paths": paths,
                "batched": batched}
        if sharded is not None:
            line["sharded"] = sharded
        line["cpu_baseline"] = None if args.no_cpu else cpu_baseline(f, g)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def profile_case(args):
    """One secondary case only, for profiler captures (small device footprint)."""
    import torch
    import paper_1004_4548_gb300 as kron
    from workloads import workload_cfg3, workload_cfg4
    dev = torch.device("cuda", 0)
    ctx = kron.Context(0)
    ctx.set_profiling(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    if args.case == "cfg3":
        r = time_poly(kron, ctx, *workload_cfg3(), dev, stream, flush, "hash_insert", args.steps)
    elif args.case == "cfg4":
        r = time_pseries(kron, ctx, *workload_cfg4(), dev, stream, flush, args.steps)
    elif args.case == "cfg4h":
        r = time_pseries(kron, ctx, *workload_cfg4(), dev, stream, flush, args.steps, path=kron.KR_PATH_HASH)
    elif args.case == "cfg2":
        from workloads import workload_cfg2
        r = time_poly(kron, ctx, *workload_cfg2(), dev, stream, flush, "dense_accum", args.steps)
    else:
        f, g = workload_cfg4(5000)
        r = time_pseries(kron, ctx, f, g, dev, stream, flush, args.steps)
    print(json.dumps({"case": args.case, **{k: v for k, v in r.items() if k != "stages_ms_last_step"}}))


def time_batched(kron, ctx, dev, nprod):
    """The uneven batch (BASELINE configs[4]): batched in chunks vs one call per
    product, and the continuous-batching server vs one-by-one service under
    Poisson arrivals."""
    import torch
    from paper_1004_4548_gb300.serve import Request, Server, serve_one_by_one
    from workloads import PSeries, Poly, arrival_times, batch_mix
    mix = batch_mix(nprod)

    def todev(p):
        if isinstance(p, PSeries):
            return PSeries(*(torch.from_numpy(x).to(dev) for x in (p.exps, p.trig, p.kind, p.coef)))
        return Poly(torch.from_numpy(p.exps).to(dev), torch.from_numpy(p.coef).to(dev))

    D = [(todev(f), todev(g)) for f, g in mix]
    tp = sum(f.n * g.n for f, g in mix)
    chunk = 128
    from paper_1004_4548_gb300 import autotune
    tuned = autotune.load_table()
    topts = [autotune.opts_for(f, g, tuned) for f, g in mix] if tuned else None
    # warm-up: one untimed pass over every chunk, so that the context's scratch
    # has grown to the largest chunk before either timed pass
    for a in range(0, nprod, chunk):
        kron.kron_mul_batch(D[a:a + chunk], ctx=ctx, opts=topts[a:a + chunk] if topts else None)
    torch.cuda.synchronize()
    # the library's built-in rules
    t = time.perf_counter()
    outputs = 0
    launches0 = ctx.launch_count()
    for a in range(0, nprod, chunk):
        out = kron.kron_mul_batch(D[a:a + chunk], ctx=ctx)
        outputs += sum(r["nterms"] for r in out)
        assert all(r["status"] == 0 for r in out)
    torch.cuda.synchronize()
    bt = time.perf_counter() - t
    b_launches = ctx.launch_count() - launches0
    # the same batches with the options of the tuned table
    t = time.perf_counter()
    for a in range(0, nprod, chunk):
        kron.kron_mul_batch(D[a:a + chunk], ctx=ctx, opts=topts[a:a + chunk] if topts else None)
    torch.cuda.synchronize()
    bt_tuned = time.perf_counter() - t
    # one call per product
    t = time.perf_counter()
    lat = []
    launches0 = ctx.launch_count()
    for f, g in D:
        t0 = time.perf_counter()
        if isinstance(f, PSeries):
            kron.poisson_mul(f, g, ctx=ctx)
        else:
            kron.poly_mul(f.exps, f.coef, g.exps, g.coef, ctx=ctx)
        lat.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    pt = time.perf_counter() - t
    p_launches = ctx.launch_count() - launches0
    res = {"workload": f"{nprod} products, operands log-uniform 50-20000 terms, 2-6 variables, "
                       "dense or weighted total-degree structure, half int64 polynomials and half "
                       "float64 Poisson series (seeds 5000+k)",
           "term_products": tp, "output_terms": outputs,
           "batched": {"products_per_s": nprod / bt, "M_term_products_per_s": tp / bt / 1e6,
                       "wall_s": bt, "chunk": chunk, "gpu_launches": b_launches,
                       "options": "library defaults",
                       "autotuned_products_per_s": nprod / bt_tuned if tuned else None,
                       "tuned_classes": len(tuned)},
           "one_call_per_product": {"products_per_s": nprod / pt, "M_term_products_per_s": tp / pt / 1e6,
                                    "wall_s": pt, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                                    "p99_ms": float(np.percentile(lat, 99) * 1e3),
                                    "gpu_launches": p_launches}}
    # CUDA graph replay of prepared batches against kron_mul_batch: the whole
    # uneven batch, in the same chunks, each chunk's graph replayed twice
    graph = {"chunks": 0, "replay_s": 0.0, "batch_call_s": 0.0, "products": 0, "graph_kernels": 0,
             "batch_call_launches": 0}
    for a in range(0, nprod, chunk):
        part = D[a:a + chunk]
        pb = kron.PreparedBatch(part, device=dev.index or 0)
        pb.launch()
        torch.cuda.synchronize()
        reps = 2
        t = time.perf_counter()
        for _ in range(reps):
            pb.launch()
        torch.cuda.synchronize()
        graph["replay_s"] += (time.perf_counter() - t) / reps
        assert all(r["status"] == 0 for r in pb.results())
        graph["graph_kernels"] += pb.graph_kernels()
        pb.close()
        l0 = ctx.launch_count()
        t = time.perf_counter()
        for _ in range(reps):
            kron.kron_mul_batch(part, ctx=ctx)
        torch.cuda.synchronize()
        graph["batch_call_s"] += (time.perf_counter() - t) / reps
        graph["batch_call_launches"] += (ctx.launch_count() - l0) // reps
        graph["chunks"] += 1
        graph["products"] += len(part)
        ctx.trim()
    graph["replay_products_per_s"] = graph["products"] / graph["replay_s"]
    graph["batch_call_products_per_s"] = graph["products"] / graph["batch_call_s"]
    res["cuda_graph"] = graph
    # CUDA graphs where launches dominate: 512 small products (<= 200 terms per operand)
    small = [(todev(f), todev(g)) for f, g in batch_mix(512, seed_base=9000, max_terms=200)]
    pb = kron.PreparedBatch(small, device=dev.index or 0)
    pb.launch()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(5):
        pb.launch()
    torch.cuda.synchronize()
    rs = (time.perf_counter() - t) / 5
    pb.close()
    t = time.perf_counter()
    for _ in range(5):
        kron.kron_mul_batch(small, ctx=ctx)
    torch.cuda.synchronize()
    cs = (time.perf_counter() - t) / 5
    res["cuda_graph_small_products"] = {"products": 512, "max_terms": 200, "replay_s": rs,
                                        "batch_call_s": cs, "replay_products_per_s": 512 / rs,
                                        "batch_call_products_per_s": 512 / cs}
    ctx.trim()
    # serving: Poisson arrivals at 0.5 and 0.8 of the batched throughput, each
    # rate with three arrival seeds (a p99 of 2048 requests rests on a few
    # of them); both arms warm (their contexts' scratch grown by the largest
    # requests first, untimed); medians over the seeds
    serve = {}
    cap = nprod / bt
    nreq = min(nprod, 2048)
    for frac in (0.5, 0.8):
        rate = frac * cap
        runs = []
        for seed in (99, 7, 31):
            t_arr = arrival_times(nreq, rate, seed=seed)
            reqs = [Request(f, g, float(a)) for (f, g), a in zip(D[:nreq], t_arr)]
            server = Server(device=dev.index or 0, workers=2, max_batch=chunk, mem_budget=60e9)   # library defaults
            server.warm_up(reqs)
            st = server.run(reqs, time_limit=60.0)
            server.close()
            reqs1 = [Request(f, g, float(a)) for (f, g), a in zip(D[:nreq], t_arr)]
            st1 = serve_one_by_one(reqs1, device=dev.index or 0, warm=True,
                                   time_limit=min(60.0, float(t_arr[-1]) * 1.5 + 5))
            runs.append((seed, st, st1))
            torch.cuda.empty_cache()
        med = lambda xs: float(statistics.median(xs))
        serve[f"rate_{frac}"] = {
            "arrival_rate_per_s": rate, "requests": nreq, "arrival_seeds": [s for s, _, _ in runs],
            "continuous_batching": {
                "completed": min(st.completed for _, st, _ in runs),
                "products_per_s": med([st.products_per_s for _, st, _ in runs]),
                "p50_ms": med([st.p50_ms for _, st, _ in runs]), "p99_ms": med([st.p99_ms for _, st, _ in runs]),
                "p99_ms_per_seed": [st.p99_ms for _, st, _ in runs],
                "mean_batch": med([st.mean_batch for _, st, _ in runs]),
                "failed": sum(st.extra.get("failed", 0) for _, st, _ in runs),
                "errors": sorted(set(e for _, st, _ in runs for e in st.extra.get("errors", [])))[:3],
                "policy": {"giant_policy": "shared", "giant": 2e7, "work_cap": 5e7, "workers": 2,
                           "warm_up": "largest requests once per context"}},
            "one_by_one": {
                "completed": min(st1.completed for _, _, st1 in runs),
                "products_per_s": med([st1.products_per_s for _, _, st1 in runs]),
                "p50_ms": med([st1.p50_ms for _, _, st1 in runs]), "p99_ms": med([st1.p99_ms for _, _, st1 in runs]),
                "p99_ms_per_seed": [st1.p99_ms for _, _, st1 in runs],
                "note": "one context, warm; requests still queued at the time limit are not counted"}}
    res["serving"] = serve
    return res


def time_sharded(kron, ctx, dev, stream, world, rank, steps, warmup):
    """One large product split over the ranks by output key window (Sec. 4's
    disjoint output ranges): full-size Fateman, rank r computing window r of
    equal sampled work, then the packed all_gather of the windows' terms, so
    that every rank holds the whole product.  Strong scaling; the time is the
    maximum over ranks."""
    import torch
    import torch.distributed as dist
    from paper_1004_4548_gb300 import shard
    from workloads import Poly, fateman
    f, g = fateman()
    F = Poly(torch.from_numpy(f.exps).to(dev), torch.from_numpy(f.coef).to(dev))
    G = Poly(torch.from_numpy(g.exps).to(dev), torch.from_numpy(g.coef).to(dev))
    cuts = shard.split_points(F, G, world, ctx=ctx)
    times, wtimes, nterms = [], [], 0
    for it in range(warmup + steps):
        dist.barrier()
        torch.cuda.synchronize()
        a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        part = shard.mul_window(F, G, cuts[rank], cuts[rank + 1], ctx=ctx)
        m.record(stream)
        whole = shard.gather_parts(part)
        b.record(stream)
        torch.cuda.synchronize()
        if it >= warmup:
            t = torch.tensor([a.elapsed_time(b), a.elapsed_time(m)], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            times.append(float(t[0]))
            wtimes.append(float(t[1]))
        nterms = int(whole[-1].shape[0])
    ms = statistics.mean(times)
    tp = f.n * g.n
    return {"workload": "Fateman's benchmark at full size, 46376 x 46376 terms, split by output key window",
            "ranks": world, "scaling": "strong", "ms_per_step": ms, "value": tp / (ms * 1e-3) / 1e6,
            "unit": UNIT, "window_ms_max": statistics.mean(wtimes), "output_terms": nterms,
            "cuts": [int(c) for c in cuts],
            "exchange": "one all_gather of the term counts and one of the packed windows (NCCL)"}


def kept_pairs(f, g, N):
    """Term pairs of f * g whose total degrees add up to at most N."""
    df = np.bincount(f.exps.sum(axis=0) - f.exps.sum(axis=0).min())
    dg = np.bincount(g.exps.sum(axis=0) - g.exps.sum(axis=0).min())
    lo = int(f.exps.sum(axis=0).min() + g.exps.sum(axis=0).min())
    conv = np.convolve(df.astype(np.float64), dg.astype(np.float64))
    return int(round(conv[:max(0, N - lo + 1)].sum()))


def time_windows(kron, ctx, f, g, dev, stream, flush, nparts, steps):
    import torch
    from paper_1004_4548_gb300 import shard
    from workloads import Poly
    F = Poly(torch.from_numpy(f.exps).to(dev), torch.from_numpy(f.coef).to(dev))
    G = Poly(torch.from_numpy(g.exps).to(dev), torch.from_numpy(g.coef).to(dev))

    def run():
        cuts = shard.split_points(F, G, nparts, ctx=ctx)
        return [shard.mul_window(F, G, a, b, ctx=ctx) for a, b in zip(cuts, cuts[1:])], cuts

    parts, cuts = run()
    times = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        parts, cuts = run()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    tp = f.n * g.n
    ms = statistics.mean(times)
    return {"value": tp / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "term_products": tp,
            "output_terms": int(sum(p[1].shape[0] for p in parts)), "windows": nparts,
            "window_terms": [int(p[1].shape[0]) for p in parts],
            "context": "one product as key windows of equal sampled work, computed one after another"}


def time_poly(kron, ctx, f, g, dev, stream, flush, kernel, steps, units=None, **opts):
    import torch
    fe, fc = torch.from_numpy(f.exps).to(dev), torch.from_numpy(f.coef).to(dev)
    ge, gc = torch.from_numpy(g.exps).to(dev), torch.from_numpy(g.coef).to(dev)
    for _ in range(2):
        ex, cf, _, _ = kron.poly_mul(fe, fc, ge, gc, ctx=ctx, **opts)
    times, kt = [], []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ex, cf, _, _ = kron.poly_mul(fe, fc, ge, gc, ctx=ctx, **opts)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        kt.extend(ms for n, ms in ctx.stages() if n == kernel)
    tp = f.n * g.n if units is None else units
    ms = statistics.mean(times)
    kms = statistics.mean(kt)
    return {"value": tp / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "term_products": tp,
            "output_terms": int(cf.shape[0]), "kernel": kernel, "kernel_ms": kms,
            "kernel_rate": tp / (kms * 1e-3) / 1e6, "stages_ms_last_step": dict(ctx.stages())}


# Algorithmic bytes per term-product of the Poisson accumulation: each pair
# updates two keys.  Hash table: per update an 8 B key probe read and an 8 B
# coefficient read and write (48 B a pair).  Dense array indexed by key: per
# update one 8 B coefficient read and write (32 B a pair).
POISSON_BYTES = {"hash": 48, "dense": 32}


def hbm_roofline(kernel, units, kms, bytes_per_unit, hbm_gbs, traffic=None):
    achieved = units * bytes_per_unit / (kms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
            "frac": achieved / hbm_gbs if hbm_gbs else None, "traffic": traffic,
            "algorithmic_bytes_per_term_product": bytes_per_unit, "units_per_launch": units,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, read + write)"}


def time_pseries(kron, ctx, f, g, dev, stream, flush, steps, path=0, hbm_gbs=None, kernel_name=None,
                 **opts):
    import torch
    from workloads import PSeries
    F = PSeries(*(torch.from_numpy(x).to(dev) for x in (f.exps, f.trig, f.kind, f.coef)))
    G = PSeries(*(torch.from_numpy(x).to(dev) for x in (g.exps, g.trig, g.kind, g.coef)))
    out = kron.poisson_mul(F, G, ctx=ctx, path=path, **opts)
    times, kt = [], []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = kron.poisson_mul(F, G, ctx=ctx, capacity=int(out[3].shape[0]), path=path, **opts)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
        kt.extend(ms for n, ms in ctx.stages() if n == "hash_insert")
    tp = f.n * g.n
    ms = statistics.mean(times)
    kms = statistics.mean(kt)
    form = "hash" if path == 2 else "dense"   # the automatic choice is the dense array here
    r = {"value": tp / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "term_products": tp,
         "output_terms": int(out[3].shape[0]), "kernel": "hash_insert", "kernel_ms": kms,
         "kernel_rate": tp / (kms * 1e-3) / 1e6, "accumulator": form,
         "stages_ms_last_step": dict(ctx.stages())}
    if hbm_gbs:
        r["roofline"] = hbm_roofline(kernel_name or "k_hash_insert_pseries", tp, kms, POISSON_BYTES[form],
                                     hbm_gbs)
    return r


if __name__ == "__main__":
    main()
