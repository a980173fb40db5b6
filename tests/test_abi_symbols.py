"""The C-ABI library loads and exports every entry point include/pfire.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pf_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2502_18738_gb300 as pf
    pf.build()
    lib = ctypes.CDLL(pf.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 18
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(pf.EXPORTED_SYMBOLS) == declared


def test_version_string_without_gpu():
    import paper_2502_18738_gb300 as pf
    pf.build()
    assert "sm_103a" in pf.pf_version()


def test_binding_rejects_non_cuda_tensors():
    import pytest
    import torch
    import paper_2502_18738_gb300 as pf
    with pytest.raises(TypeError):
        pf._ptr(torch.zeros(4), torch.float32, 4, "x")
