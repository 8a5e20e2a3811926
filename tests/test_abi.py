"""The C-ABI library loads and exports every symbol include/pb.h declares
(no compute: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "pb.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pb_[a-z_0-9]+)\s*\(", src, re.M)))


def test_header_declares_the_documented_entry_points():
    names = _declared()
    for want in ["pb_graph_from_edges", "pb_rank", "pb_count_global", "pb_count_vertex", "pb_count_edge",
                 "pb_wedge_count", "pb_graph_free", "pb_last_error"]:
        assert want in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1907_08607_gb300 import build as b
    import paper_1907_08607_gb300 as pb
    path = b.build()
    lib = pb.load_library(path)
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value
    assert set(pb.ABI_SYMBOLS) == set(_declared())
    assert lib.pb_status_string(1) == b"PB_ERR_INVALID"


def test_product_path_has_no_cpu_fallback():
    """The binding refuses to run without a CUDA device instead of computing
    on the host."""
    import torch
    import paper_1907_08607_gb300 as pb
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        pb.Graph.from_edges(2, 2, [0, 1], [0, 1])


def test_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1907_08607_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    txt = f.read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "pb_oracle" not in txt, fn


def test_error_paths_return_status_without_a_device():
    """Calls that need no device reject bad arguments with PB_ERR_INVALID;
    graph construction on a machine without a CUDA device returns an error
    status (and a message) instead of aborting."""
    import numpy as np
    import torch
    from paper_1907_08607_gb300 import build as b
    import paper_1907_08607_gb300 as pb
    lib = pb.load_library(b.build())
    for code, name in pb.STATUS.items():
        assert lib.pb_status_string(code).decode() == name
    assert lib.pb_set_retrieval(None, 0) == 1
    assert lib.pb_set_butterfly_aggregation(None, 0) == 1
    assert lib.pb_graph_free(None) in (0, 1)
    assert lib.pb_wedge_count(None, None) == 1
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    u = np.array([0, 1], np.uint32)
    out = ctypes.c_void_p()
    rc = lib.pb_graph_from_edges(2, 2, 2, ctypes.c_void_p(u.ctypes.data), ctypes.c_void_p(u.ctypes.data), 0, None,
                                 ctypes.byref(out))
    assert rc != 0 and out.value is None
    assert lib.pb_last_error()
