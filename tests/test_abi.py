"""The C-ABI library builds, loads and exports every function include/gfd.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gfd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(gfd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gfd_graph_load", "gfd_graph_free", "gfd_validate", "gfd_validate_batch",
                     "gfd_result_matches", "gfd_result_violations", "gfd_result_tuples",
                     "gfd_result_free", "gfd_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2608_02321_gb300 as g
    lib = g.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in g._SIGS, f"binding lacks a signature for {name}"


def test_binding_has_no_extra_symbols():
    import paper_2608_02321_gb300 as g
    assert set(g._SIGS) == set(declared_functions())


def test_last_error_is_empty_initially():
    import paper_2608_02321_gb300 as g
    lib = g.load_library()
    assert lib.gfd_last_error() == b""
