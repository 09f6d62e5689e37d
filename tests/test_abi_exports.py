"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point that
include/probesim.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1709_06955_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared():
    with open(os.path.join(ROOT, "include", "probesim.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(probesim_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("probesim_graph_create", "probesim_insert_edges", "probesim_delete_edges", "probesim_single_source",
              "probesim_topk", "probesim_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1709_06955_gb300 import probesim
    assert sorted(probesim.EXPORTS) == declared()


def test_struct_layouts_match_header(lib):
    """Field offsets of the binding's structs follow the C layout of the header."""
    from paper_1709_06955_gb300 import probesim as P
    assert ctypes.sizeof(P.Config) == 40
    assert P.Query.eps.offset == 8 and ctypes.sizeof(P.Query) == 32
    assert ctypes.sizeof(P.Stats) == 224


def test_product_path_has_no_fallback(tmp_path):
    """Loading the binding without the built library raises instead of falling back."""
    from paper_1709_06955_gb300 import probesim
    saved = probesim._lib
    probesim._lib = None
    try:
        with pytest.raises(RuntimeError):
            probesim.load(str(tmp_path / "missing.so"))
    finally:
        probesim._lib = saved


def test_package_does_not_import_oracle():
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_1709_06955_gb300.probesim, "
            "paper_1709_06955_gb300.synth; assert 'oracle' not in sys.modules" % ROOT)
    subprocess.check_call([sys.executable, "-c", code])
