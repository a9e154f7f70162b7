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


def test_options_mirror_matches_the_c_layout(tmp_path):
    """The ctypes mirror of gabp_options has the C struct's size and every field's offset, so a
    field added on one side only cannot shift the others (checked with the host C compiler)."""
    import shutil
    import subprocess

    import paper_0811_2518_gb300 as gb

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest

        pytest.skip("no host C compiler")
    fields = [f for f, _ in gb.Options._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "gabp.h"', "int main(void) {",
            '  printf("size %zu\\n", sizeof(gabp_options));']
    prog += [f'  printf("{f} %zu\\n", offsetof(gabp_options, {f}));' for f in fields]
    prog += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.split("\n") if line)
    assert int(out["size"]) == ctypes.sizeof(gb.Options)
    for f in fields:
        assert int(out[f]) == getattr(gb.Options, f).offset, f


def test_profile_mirror_matches_the_c_layout(tmp_path):
    import shutil
    import subprocess

    import paper_0811_2518_gb300 as gb

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest

        pytest.skip("no host C compiler")
    prog = ("#include <stdio.h>\n#include <stddef.h>\n#include \"gabp.h\"\nint main(void) {\n"
            '  printf("%zu %zu %zu %zu\\n", sizeof(gabp_profile), offsetof(gabp_profile, ms),\n'
            "         offsetof(gabp_profile, rounds), offsetof(gabp_profile, launches));\n  return 0;\n}\n")
    c = tmp_path / "prof.c"
    c.write_text(prog)
    exe = tmp_path / "prof"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    size, ms, rounds, launches = map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split())
    assert size == ctypes.sizeof(gb.Profile)
    assert (ms, rounds, launches) == (gb.Profile.ms.offset, gb.Profile.rounds.offset, gb.Profile.launches.offset)


def test_binding_argument_counts_match_the_header():
    """Every ctypes signature takes as many arguments as the header's declaration."""
    import paper_0811_2518_gb300 as gb

    src = open(os.path.join(ROOT, "include", "gabp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = dict(re.findall(r"\b(gabp_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S))
    for name, (args, _) in gb._SIGNATURES.items():
        params = decls[name].strip()
        n = 0 if params in ("", "void") else len(params.split(","))
        assert n == len(args), (name, n, len(args))


def test_limits_and_bad_arguments_rejected_without_gpu():
    """Size limits and bad arguments are refused before any CUDA call (so on a machine without a
    GPU too): nnz >= 2^31 - 1, n < 1, nnz < n, null arrays, a memory space other than 0 or 1,
    out-of-range options (freeze_precisions, accel, multi_mode), and the dense and least-squares
    entries' bad shapes; queries on a null handle."""
    import numpy as np

    import paper_0811_2518_gb300 as gb

    L = gb.lib
    P = ctypes.c_void_p
    h = P()
    rp = np.zeros(3, dtype=np.int32)
    ci = np.zeros(2, dtype=np.int32)
    va = np.ones(2)
    ptrs = (P(rp.ctypes.data), P(ci.ctypes.data), P(va.ctypes.data))
    INV = gb.GABP_ERR_INVALID
    for n, nnz in ((2, 2 ** 31 - 1), (2, 2 ** 31), (0, 2), (3, 2)):
        assert L.gabp_create(ctypes.byref(h), n, nnz, *ptrs, 0, None, None) == INV, (n, nnz)
    assert L.gabp_create(ctypes.byref(h), 2, 2, None, ptrs[1], ptrs[2], 0, None, None) == INV
    assert L.gabp_create(ctypes.byref(h), 2, 2, *ptrs, 2, None, None) == INV
    for field, bad in (("freeze_precisions", 2), ("accel", 3), ("multi_mode", 4), ("check_every", 0)):
        o = gb.gabp_options_default()
        setattr(o, field, bad)
        assert L.gabp_create(ctypes.byref(h), 2, 2, *ptrs, 0, None, ctypes.byref(o)) == INV, field
    A = np.eye(3)
    nnz = ctypes.c_int64(0)
    for n, lda, mem in ((0, 3, 0), (3, 2, 0), (3, 3, 2)):
        assert L.gabp_create_dense(ctypes.byref(h), n, P(A.ctypes.data), lda, mem, None, None,
                                   ctypes.byref(nnz)) == INV, (n, lda, mem)
    assert L.gabp_create_dense(ctypes.byref(h), 3, None, 3, 0, None, None, None) == INV
    assert L.gabp_create_lsq(ctypes.byref(h), 0, 2, 2, *ptrs, 1.0, 0, None, None) == INV
    assert L.gabp_create_lsq(ctypes.byref(h), 2, 2, 2, *ptrs, -1.0, 0, None, None) == INV
    r = ctypes.c_int32(0)
    assert L.gabp_last_freeze(None, ctypes.byref(r), None) == INV
    assert L.gabp_solve(None, None, None, ctypes.c_double(1e-10), 10, None, None) == INV
    assert L.gabp_destroy(None) == gb.GABP_OK
