"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
symbol include/kron.h declares, and its host-side coding plan reproduces the
paper's worked examples.  No device compute is called here."""
import math
import os
import re

import numpy as np
import pytest

import paper_1004_4548_gb300 as kron
from paper_1004_4548_gb300 import binding
from workloads import total_degree_tuples

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def declared_functions():
    text = open(os.path.join(ROOT, "include", "kron.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s+\**(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


def test_library_builds_and_loads():
    L = kron.load()
    assert os.path.exists(kron.lib_path())
    assert L is not None


def test_every_declared_symbol_is_exported():
    L = kron.load()
    names = declared_functions()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(L, n), f"{n} declared in kron.h but not exported"
    assert set(binding.SIGNATURES) <= set(names)


def test_table1_codes():
    """Table 1: three variables in [0, 3]; c = (1, 4, 16), Eq. 2: 3 + 4 = 7."""
    c, W = kron.kron_plan([0, 0, 0], [3, 3, 3])
    assert list(c) == [1, 4, 16] and W == 64
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "table1_codes.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 10
    for z, y, x, code in rows:
        assert c[0] * x + c[1] * y + c[2] * z == code


@pytest.mark.parametrize("seed", range(5))
def test_table2_rows(seed):
    """Table 2: codes of the generalised substitution in terms of w0."""
    rng = np.random.default_rng(seed)
    lo = rng.integers(-20, 5, size=3).astype(np.int32)
    hi = lo + rng.integers(2, 9, size=3).astype(np.int32)
    c, W = kron.kron_plan(lo, hi)
    w0 = int(hi[0] - lo[0] + 1)
    assert W == int(np.prod((hi - lo + 1).astype(np.int64)))
    for l in open(os.path.join(GOLDEN, "table2_rows.txt")):
        if not l.strip() or l.startswith("#"):
            continue
        d1, d0, a, b = l.split()
        e = lo.astype(np.int64).copy()
        e[1] = lo[1] + int(d1)
        e[0] = hi[0] if d0 == "max" else lo[0] + int(d0)
        code = int(np.dot(c, e - lo))
        assert code == int(a) + int(b) * w0


def test_overflow_boundary():
    # 2^63 - 1 = 7^2 * 73 * 127 * 337 * 92737 * 649657: accepted
    w = [7, 7, 73, 127, 337, 92737, 649657]
    assert math.prod(w) == (1 << 63) - 1
    c, W = kron.kron_plan([0] * 7, [x - 1 for x in w])
    assert W == (1 << 63) - 1
    # 2^63: rejected
    with pytest.raises(kron.KronError) as e:
        kron.kron_plan([0, 0, 0], [(1 << 21) - 1] * 3)
    assert e.value.status == kron.KR_ERR_OVERFLOW
    with pytest.raises(kron.KronError) as e:
        kron.kron_plan([3], [2])
    assert e.value.status == kron.KR_ERR_INVALID


def test_fateman_density_matches_paper():
    """Sec. 3: the Fateman factors have about one nonzero monomial every 300 codes
    when coded with the widths of the product (the reading used throughout)."""
    rows = total_degree_tuples(4, 30)
    assert rows.shape[0] == 46376
    c, W = kron.kron_plan([0] * 4, [60] * 4)
    assert W == 61 ** 4
    assert 290 < W / rows.shape[0] < 310


def test_ctypes_structures_match_the_header(tmp_path):
    """Every structure the binding passes across the C ABI has the header's
    size and field offsets (a C program built against include/kron.h prints
    them; a field name missing from the header fails its build)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [binding.kr_poly, binding.kr_poly_out, binding.kr_pseries, binding.kr_pseries_out,
               binding.kr_opts, binding.kr_job, binding.kr_result]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "kron.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for fname, _ in st._fields_:
            lines.append(f'  printf("{n}.{fname} %zu\\n", offsetof({n}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for fname, _ in st._fields_:
            assert int(got[f"{n}.{fname}"]) == getattr(st, fname).offset, f"{n}.{fname}"


def test_caller_outputs_are_used_as_given_or_rejected():
    """A caller-supplied output of another dtype, shape or layout would be
    replaced by a converted copy that alone receives the result: the binding
    refuses it instead (no device call is made here)."""
    import torch
    good = np.zeros((3, 5), np.int32)
    assert binding._out_ptr(good, (3, 5), np.int32) == good.ctypes.data
    t = torch.zeros(7, dtype=torch.int64)
    assert binding._out_ptr(t, (7,), np.int64) == t.data_ptr()
    bad = [(np.zeros((3, 5), np.int64), (3, 5), np.int32),           # dtype
           (np.zeros((5, 3), np.int32).T, (3, 5), np.int32),         # layout
           (np.zeros((3, 6), np.int32), (3, 5), np.int32),           # shape
           (torch.zeros(7, dtype=torch.int32), (7,), np.int64),
           (torch.zeros(14, dtype=torch.int64)[::2], (7,), np.int64),
           ([0] * 7, (7,), np.int64)]
    for out, shape, dt in bad:
        with pytest.raises(ValueError):
            binding._out_ptr(out, shape, dt)


def test_coding_entries_reject_boxes_wider_than_int32():
    """A variable whose width exceeds 2^31 - 1 is a valid box for kron_plan
    (W = 2^32 here) but not for the 32-bit coding kernels: kron_encode and
    kron_decode refuse it on the host, before any device work (no context is
    needed to reach that check)."""
    L = kron.load()
    lo = np.array([-(1 << 31)], np.int32)
    hi = np.array([(1 << 31) - 1], np.int32)
    c, W = kron.kron_plan(lo, hi)
    assert W == 1 << 32
    codes = np.zeros(1, np.int64)
    exps = np.zeros((1, 1), np.int32)
    st = L.kron_decode(None, codes.ctypes.data, 1, 1, lo.ctypes.data, hi.ctypes.data, exps.ctypes.data, None)
    assert st == binding.KR_ERR_OVERFLOW
    st = L.kron_encode(None, exps.ctypes.data, 1, 1, lo.ctypes.data, hi.ctypes.data, codes.ctypes.data, None)
    assert st == binding.KR_ERR_OVERFLOW
    # width exactly 2^31 - 1 passes the check; the call then stops at the
    # missing context, still before any device work
    lo2 = np.array([-(1 << 30)], np.int32)
    hi2 = np.array([(1 << 30) - 2], np.int32)
    st = L.kron_decode(None, codes.ctypes.data, 1, 1, lo2.ctypes.data, hi2.ctypes.data, exps.ctypes.data, None)
    assert st == binding.KR_ERR_INVALID
