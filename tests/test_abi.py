"""The C-ABI library loads and exports every function include/gabp.h declares (CPU only)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "gabp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gabp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_core_calls():
    names = _declared()
    for core in ("gabp_create", "gabp_solve", "gabp_marginal_precisions", "gabp_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__

    __graft_entry__.build()
    import paper_0811_2518_gb300 as gb

    L = ctypes.CDLL(gb.library_path)
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) == set(gb.exported_symbols())


def test_status_strings_and_defaults():
    import paper_0811_2518_gb300 as gb

    assert gb.gabp_status_string(gb.GABP_OK) == "converged"
    assert "breakdown" in gb.gabp_status_string(gb.GABP_BREAKDOWN)
    o = gb.gabp_options_default()
    assert o.variant == gb.GABP_VARIANT_NODE and o.precision == gb.GABP_PREC_FP64 and o.check_every == 16


def test_library_has_no_oracle_dependency():
    """The product never links, imports or names the oracle."""
    pkg = os.path.join(ROOT, "paper_0811_2518_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "orc_gabp" not in txt and "gabp_oracle" not in txt, f
