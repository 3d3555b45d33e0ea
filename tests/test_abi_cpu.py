"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/lc.h declares.  No compute call is made here."""
import os
import re

from paper_1807_10727_gb300 import _build, lc

HEADER = os.path.join(_build.INCLUDE, "lc.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:lc_status|const char\*)\s+(lc_\w+)\s*\(", text, re.M)))


def test_header_declarations_are_bound():
    assert set(declared_symbols()) == set(lc.EXPORTED)


def test_library_builds_and_exports_every_symbol():
    path = _build.build_lc()
    lib = lc.load(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings():
    lc.load(_build.build_lc())
    assert lc.lc_status_str(0) == "ok"
    assert "invalid" in lc.lc_status_str(1)
    assert lc.lc_status_str(99) == "unknown status"


def test_compiled_for_sm103a_only():
    assert _build.ARCH_FLAGS == ["-gencode", "arch=compute_103a,code=sm_103a"]
