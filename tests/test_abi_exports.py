"""The C-ABI library loads without a GPU and exports every function that
include/riann.h declares; the Python binding covers each of them.  Symbol
lookups only: nothing is called."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "riann.h")
LIB = os.path.join(ROOT, "paper_1508_07953_gb300", "_lib", "libriann.so")
BINDING = os.path.join(ROOT, "paper_1508_07953_gb300", "riann.py")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)           # comments mention calls too
    src = re.sub(r"//[^\n]*", "", src)
    return sorted(set(re.findall(r"\b(riann_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1508_07953_gb300 import build_lib    # nvcc cross-compiles without a GPU
        build_lib.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("riann_build_reference_index", "riann_annf_frame", "riann_exact_nn", "riann_knn_frame",
                 "riann_build_unit_index", "riann_stack_frames", "riann_cluster_references", "riann_batch_run",
                 "riann_server_step", "riann_anchor_frame", "riann_reconstruct", "riann_random_field",
                 "riann_status"):
        assert must in names, must
    assert len(names) >= 50


def test_every_declared_function_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in riann.h but not exported: {missing}"


def test_binding_covers_every_function():
    src = open(BINDING).read()
    unbound = [n for n in declared_functions() if f"_lib.{n}" not in src]
    assert not unbound, f"not bound in riann.py: {unbound}"
