"""The product path has no CPU fallback: without the CUDA library the binding
refuses to import, and every compute entry point refuses host tensors before
anything runs.  Nothing here launches work."""
import importlib.util
import os
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BINDING = os.path.join(ROOT, "paper_1508_07953_gb300", "riann.py")
LIB = os.path.join(ROOT, "paper_1508_07953_gb300", "_lib", "libriann.so")


def test_binding_refuses_to_import_without_the_library(tmp_path):
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    shutil.copy(BINDING, pkg / "riann.py")                  # no _lib/ beside it
    spec = importlib.util.spec_from_file_location("riann_without_lib", pkg / "riann.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError, match="CUDA library not found"):
        spec.loader.exec_module(mod)


@pytest.fixture(scope="module")
def rt():
    if not os.path.exists(LIB):
        from paper_1508_07953_gb300 import build_lib    # nvcc cross-compiles without a GPU
        build_lib.build()
    from paper_1508_07953_gb300 import riann
    return riann


def _host(shape, dtype=None):
    import torch
    return torch.from_numpy(np.zeros(shape, np.uint8 if dtype is None else dtype))


def test_host_tensors_are_refused(rt):
    # refused in the binding, before the library is called: a host tensor is
    # a ValueError, and on a machine without a GPU the stream lookup fails
    # first for the calls that take a stream before their tensors
    patches, keys = _host((16, 8, 8, 1)), _host((2, 8, 8, 1))
    frame, field = _host((12, 12)), _host((5, 5), np.int32)
    idx = rt.RiannIndex(0, 16, 2, 1)                          # no handle: never reaches the library
    calls = [
        lambda: rt.riann_build_reference_index(patches, keys),
        lambda: rt.riann_build_unit_index(patches, keys),
        lambda: rt.riann_cluster_references(patches, 4),
        lambda: rt.riann_stack_frames(frame, frame, frame),
        lambda: rt.annf(idx, frame, field),
        lambda: rt.knn(idx, frame, field, 4),
        lambda: rt.riann_reconstruct(idx, field, frame),
        lambda: rt.riann_reconstruct_payload(idx, patches, field, frame),
    ]
    for call in calls:
        with pytest.raises((ValueError, RuntimeError)):
            call()
    with pytest.raises(ValueError, match="CUDA tensor"):
        rt.riann_build_reference_index(patches, keys)
