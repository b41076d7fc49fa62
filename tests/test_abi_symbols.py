"""The C-ABI library builds for sm_103a, loads, and exports every function include/tt.h declares.
No compute call is made (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", fn)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(tt_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("tt_apply_transport", "tt_round", "tt_axpy", "tt_dot", "tt_step"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2602_00290_gb300 import _build
    path = _build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2602_00290_gb300 import _build, lib
    _build.build()
    assert lib().tt_status_string(0) == b"ok"
    assert lib().tt_status_string(3) == b"rank capacity exceeded"


def test_binding_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2602_00290_gb300 as tt
    with pytest.raises(RuntimeError):
        tt.Context(0)
