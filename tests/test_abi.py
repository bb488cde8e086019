"""The C-ABI library loads on a machine without a GPU and exports every
function that include/tb.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tb_[a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tb_build", "tb_build_batched", "tb_moments", "tb_free", "tb_tree_status",
                 "tb_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2312_06102_gb300 import compile_lib
    path = compile_lib.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults_without_gpu():
    import paper_2312_06102_gb300 as tb
    from paper_2312_06102_gb300 import compile_lib
    compile_lib.build()
    assert tb.status_string(0) == "ok"
    assert "capacity" in tb.status_string(4)
    p = tb.lib().tb_default_params()
    assert p.n_crit == 16 and p.mom_mode == 0 and p.cell_capacity == 0


def test_no_cpu_fallback_in_binding():
    """The product binding never imports the oracle."""
    for f in ("__init__.py", "_lib.py"):
        src = open(os.path.join(ROOT, "paper_2312_06102_gb300", f)).read()
        assert "oracle" not in src.replace("no CPU fallback", "")
