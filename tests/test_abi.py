"""The C ABI library builds, loads without a GPU, and exports every entry point include/*.h declares."""
import glob
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^JACOBI_API\s+[\w\s\*]+?\b(jacobi_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("jacobi_setup", "jacobi_solve", "jacobi_destroy", "jacobi_setup_ex", "jacobi_solve_ex"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_5805_gb300 as jac
    lib = jac.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(jac.EXPORTS)


def test_status_strings_without_gpu():
    import paper_1403_5805_gb300 as jac
    lib = jac.load()
    assert lib.jacobi_status_string(jac.ERR_ZERO_DIAGONAL).decode().startswith("zero diagonal")
    assert lib.jacobi_status_string(12345).decode() == "unknown status"


def test_struct_layouts_match_header():
    import ctypes
    import paper_1403_5805_gb300 as jac
    # jacobi_stats: 2 x int64, 2 x double, 2 x int32; jacobi_desc: see include/jacobi.h
    assert ctypes.sizeof(jac.JacobiStats) == 40
    assert ctypes.sizeof(jac.JacobiDesc) == 120
    # jacobi_csr_desc: 2 x int64, 4 pointers, 2 x int32, 1 pointer, 4 x int32, 1 double
    assert ctypes.sizeof(jac.JacobiCsrDesc) == 88


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """With the library absent the binding raises instead of falling back to anything else."""
    from paper_1403_5805_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libjacobi.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()
