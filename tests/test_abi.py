"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/anyseq.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(anyseq_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_04561_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    assert "anyseq_align_batch" in names and "anyseq_align_long" in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"


def test_binding_names_match_header():
    import paper_2002_04561_gb300 as pkg
    assert set(pkg.EXPORTS) <= set(declared_functions())


def test_host_only_calls(lib):
    import paper_2002_04561_gb300 as pkg
    pkg.load()
    assert "sm_103a" in pkg.version()
    assert list(pkg.encode_dna("ACGTacgt")) == [0, 1, 2, 3, 0, 1, 2, 3]
    with pytest.raises(pkg.AnyseqError) as ei:
        pkg.encode_dna("ACGN")
    assert ei.value.status == 2
