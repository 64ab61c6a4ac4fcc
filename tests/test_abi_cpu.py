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
