"""bench.py's reference arm (the oracle timed on the host's cores) prints the
contract's JSON line without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "dtype", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_hbm_roofline_arithmetic():
    """achieved = units x algorithmic bytes / kernel time; frac = achieved / peak
    (the hash insert of the Monagan-Pearce product: 38,291,344 term-products of
    24 B in 0.9776 ms is 940 GB/s)."""
    b = _bench_module()
    r = b.hbm_roofline("k_hash_insert_poly", 38_291_344, 0.9776, 24, 6787.0, traffic=1_231_763_968)
    assert abs(r["achieved"] - 940.05) < 0.01
    assert abs(r["frac"] - r["achieved"] / 6787.0) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 1_231_763_968
    assert b.hbm_roofline("k", 1, 1.0, 8, None)["frac"] is None


def test_clock_record_reports_median_max_and_reasons():
    """The clock record taken during the timed region: median SM clock, the
    maximum clock, and every throttle reason seen active in any sample."""
    b = _bench_module()

    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = b.Clocks(0)
    c.proc = FakeProc()
    c.lines = ["2070, 2070, 812.4, 0x0, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1398.0, 0x4, Not Active, Not Active, Not Active, Active",
               "1500, 2070, 1390.1, 0x8, Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "short line"]
    r = c.stop()
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert b.Clocks(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_recorded_traffic_applies_only_to_its_kernel_source():
    """A DRAM traffic figure taken by ncu on one kernel source is reported
    only while that source is unchanged (its SHA-256 prefix matches)."""
    b = _bench_module()
    rec = dict(b.DENSE_TRAFFIC)
    assert b.kernel_traffic(rec) in (rec["bytes"], None)
    assert b.kernel_traffic(dict(rec, source_sha256="0" * 16)) is None
    assert b.kernel_traffic(dict(rec, source="no_such_file.cu")) is None
