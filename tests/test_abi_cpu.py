"""The C-ABI library loads and exports every entry point include/eik.h
declares; host-only entry points work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eik.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1110_6220_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eik_[a-z_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared()
    for must in ("eik_plan_create", "eik_solve", "eik_plan_destroy", "eik_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_uses_the_same_names():
    from paper_1110_6220_gb300 import eik
    for name in declared():
        assert callable(getattr(eik, name)), name


def test_binding_constants_match_the_header():
    """Every EIK_ enumerator and #define in include/eik.h has the same value
    in the Python binding, and the ctypes structures have the C sizes."""
    from paper_1110_6220_gb300 import eik
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = item.partition("=")
            nxt = int(val.strip(), 0) if val.strip() else nxt
            consts[name.strip()] = nxt
            nxt += 1
    for name, expr in re.findall(r"#define[ \t]+(EIK_\w+)[ \t]+([^\n]+)", text):
        expr = re.sub(r"(\d+)u\b", r"\1", expr.strip())
        assert re.fullmatch(r"[\d\s()<]+", expr), (name, expr)  # integers and shifts only
        consts[name] = eval(expr)
    assert "EIK_METHOD_HCM_LSM" in consts and "EIK_NOALLOC_SCRATCH_BYTES" in consts
    for name, val in consts.items():
        assert getattr(eik, name) == val, name


def test_structure_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the C structures have the C compiler's size and
    field offsets (gcc compiles a probe against include/eik.h)."""
    import shutil
    import subprocess
    from paper_1110_6220_gb300 import eik
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    structs = [eik.eik_plan_desc, eik.eik_instance, eik.eik_stats, eik.eik_tune_result]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "eik.h"', "int main(void) {"]
    for s in structs:
        n = s.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in s._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for s in structs:
        n = s.__name__
        assert int(got[n]) == ctypes.sizeof(s), n
        for f, _ in s._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(s, f).offset, f"{n}.{f}"


def test_strerror_and_workspace_size_without_gpu():
    from paper_1110_6220_gb300 import eik
    assert eik.eik_strerror(0) == "ok"
    assert "invalid" in eik.eik_strerror(-1)
    assert eik.eik_strerror(12345) == "unknown eik status"
    ok = eik.make_desc(129, 129, 1 / 128, 8)
    assert eik.eik_plan_workspace_bytes(ok) > 129 * 129 * 16
    for bad in (eik.make_desc(1, 129, 0.1), eik.make_desc(129, 129, 0.0),
                eik.make_desc(129, 129, 0.1, cell_k=6), eik.make_desc(129, 129, 0.1, precision=7)):
        assert eik.eik_plan_workspace_bytes(bad) == 0


def test_plan_create_rejects_bad_descriptors_before_touching_cuda():
    from paper_1110_6220_gb300 import eik
    with pytest.raises(eik.EikError) as e:
        eik.eik_plan_create(eik.make_desc(129, 1, 0.1))
    assert e.value.code == eik.EIK_EINVAL


def test_tune_table_round_trip_and_use_without_gpu(tmp_path):
    """A loaded table decides k and the schedule for descriptors that leave
    them open (seen through the workspace size, which needs no GPU: the
    value-ordered schedule adds its bucket rings); save writes back what was
    loaded; malformed files merge nothing; reset restores the built-in
    choice."""
    from paper_1110_6220_gb300 import eik
    eik.eik_tune_reset()
    F64, R = eik.EIK_FP64, eik.EIK_FP32_REFINE
    FIFO, ORD = eik.EIK_SCHED_FIFO, eik.EIK_SCHED_ORDERED

    def ws(n, k, prec, sched=0):
        return eik.eik_plan_workspace_bytes(eik.make_desc(n, n, 1 / (n - 1), k, prec, schedule=sched))

    d0 = eik.make_desc(1025, 1025, 1 / 1024, 0, F64)
    w32_fifo, w32_ord = ws(1025, 32, F64, FIFO), ws(1025, 32, F64, ORD)
    assert w32_ord == w32_fifo + 32 * 2048 * 8 + 1024  # 33^2 cells -> rings of 2048
    # built in: one FP64 grid at k = 8 in value order from ~512^2 (k = 16
    # from ~8192^2); FP32 + refinement k = 8 first in, first out up to
    # ~2048^2, k = 16 in value order from ~4096^2
    assert eik.eik_plan_workspace_bytes(d0) == ws(1025, 8, F64, ORD)
    for n, k, sched in ((1025, 8, FIFO), (2049, 8, FIFO), (4097, 16, ORD), (8193, 16, ORD)):
        assert ws(n, 0, R) == ws(n, k, R, sched), n
    for n, k, sched in ((129, 8, FIFO), (513, 8, ORD), (4097, 8, ORD), (8193, 16, ORD)):
        assert ws(n, 0, F64) == ws(n, k, F64, sched), n
    f = tmp_path / "tune.txt"
    # class: FP64, single grid, side 2^10 (a version-4 line: first in, first out)
    f.write_text("eik-tune 4\n0 0 10 32 8 8 0 1 0 0 1.5\n")
    assert eik.eik_tune_load(str(f)) == 0
    assert eik.eik_plan_workspace_bytes(d0) == w32_fifo
    # another side class keeps the built-in choice
    assert ws(129, 0, F64) == ws(129, 8, F64, FIFO)
    g = tmp_path / "out.txt"
    assert eik.eik_tune_save(str(g)) == 0
    lines = g.read_text().splitlines()
    assert lines[0] == "eik-tune 5"
    assert [float(x) for x in lines[1].split()] == [0, 0, 10, 32, 8, 8, 0, 1, 0, 0, 1.5, 0, 31]
    # the saved table loads back as it was
    assert eik.eik_tune_load(str(g)) == 0
    assert eik.eik_plan_workspace_bytes(d0) == w32_fifo
    # version 5: the value-ordered schedule, window 2
    v5 = tmp_path / "v5.txt"
    v5.write_text("eik-tune 5\n0 0 10 32 8 8 0 1 0 0 1.5 1 2\n")
    assert eik.eik_tune_load(str(v5)) == 0
    assert eik.eik_plan_workspace_bytes(d0) == w32_ord
    # a schedule named in the descriptor wins over the table
    assert eik.eik_plan_workspace_bytes(eik.make_desc(1025, 1025, 1 / 1024, 0, F64, schedule=FIFO)) == w32_fifo
    bad = tmp_path / "bad.txt"
    bad.write_text("eik-tune 4\n1 0 10 12 8 8 0 0 0 0 1.0\n")  # k = 12 is not a cell size
    assert eik.eik_tune_load(str(bad)) == eik.EIK_EINVAL
    bad.write_text("eik-tune 5\n1 0 10 16 8 8 0 1 0 0 1.0 1 32\n")  # windows are 0..31 in the table
    assert eik.eik_tune_load(str(bad)) == eik.EIK_EINVAL
    bad.write_text("eik-tune 5\n1 0 10 16 8 8 0 1 0 0 1.0\n")  # version 5 lines carry 13 fields
    assert eik.eik_tune_load(str(bad)) == eik.EIK_EINVAL
    bad.write_text("something else\n")
    assert eik.eik_tune_load(str(bad)) == eik.EIK_EINVAL
    assert eik.eik_tune_load(str(tmp_path / "missing.txt")) == eik.EIK_EINVAL
    assert eik.eik_plan_workspace_bytes(d0) == w32_ord
    eik.eik_tune_reset()
    assert eik.eik_plan_workspace_bytes(d0) == ws(1025, 8, F64, ORD)


def test_method_descriptor_rules_without_gpu():
    """Methods and their allowed forms, seen through eik_plan_workspace_bytes
    (0 for a refused descriptor, no GPU needed): FHCM, FMSM and HCM with
    locking are FP64 only; FMSM needs cells of 8 or more, and cell_k = 0
    gives it 8 or more; HCM with locking takes every cell size and needs the
    same workspace as HCM; an unknown method is refused."""
    from paper_1110_6220_gb300 import eik
    F64, R = eik.EIK_FP64, eik.EIK_FP32_REFINE
    ws = lambda k, prec, m: eik.eik_plan_workspace_bytes(eik.make_desc(257, 257, 1 / 256, k, prec, method=m))
    for m in (eik.EIK_METHOD_HCM, eik.EIK_METHOD_FHCM, eik.EIK_METHOD_FMSM, eik.EIK_METHOD_HCM_LSM):
        assert ws(8, F64, m) > 0
    assert ws(8, R, eik.EIK_METHOD_HCM) > 0
    assert ws(8, R, eik.EIK_METHOD_FHCM) == 0
    assert ws(8, R, eik.EIK_METHOD_FMSM) == 0
    assert ws(8, R, eik.EIK_METHOD_HCM_LSM) == 0
    assert ws(4, F64, eik.EIK_METHOD_FMSM) == 0
    assert ws(4, F64, eik.EIK_METHOD_HCM) > 0
    assert ws(0, F64, eik.EIK_METHOD_FMSM) > 0
    for k in (4, 8, 16, 32, 64):
        assert ws(k, F64, eik.EIK_METHOD_HCM_LSM) == ws(k, F64, eik.EIK_METHOD_HCM)
    assert ws(8, F64, 4) == 0


def test_schedule_descriptor_rules_without_gpu():
    """The descriptor's schedule and window: every EIK_SCHED_* and windows
    0..32 are accepted, anything else refused; naming the value-ordered
    schedule adds its bucket rings to the workspace (32 per cell, a power of
    two >= the grid's cells), the other schedules do not."""
    from paper_1110_6220_gb300 import eik
    ws = lambda sched, win=0, k=8: eik.eik_plan_workspace_bytes(
        eik.make_desc(257, 257, 1 / 256, k, eik.EIK_FP64, schedule=sched, window=win))
    base = ws(eik.EIK_SCHED_FIFO)
    assert base > 0 and ws(eik.EIK_SCHED_ROUNDS) == base
    assert ws(eik.EIK_SCHED_ORDERED) == base + 32 * 2048 * 8 + 1024  # 33^2 cells -> rings of 2048
    for w in (0, 1, 17, 32):
        assert ws(eik.EIK_SCHED_ORDERED, w) > 0
    assert ws(eik.EIK_SCHED_ORDERED, 33) == 0
    assert ws(eik.EIK_SCHED_ORDERED, -1) == 0
    assert ws(4) == 0 and ws(-1) == 0
