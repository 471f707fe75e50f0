"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/oefe.h declares; argument errors come back as status codes."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "oefe.h")).read()
    return sorted(set(re.findall(r"\bint\s+(oefe_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import paper_2010_09701_gb300 as P
    from paper_2010_09701_gb300 import build_ext
    build_ext.build()
    lib = P.load()
    declared = header_symbols()
    assert len(declared) >= 20
    bound = sorted(n for n, _, _ in P.SIGNATURES)
    assert bound == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_symbols_are_exported_by_the_shared_object():
    import subprocess
    from paper_2010_09701_gb300 import build_ext
    lib = build_ext.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(oefe_\w+)", out))
    assert set(header_symbols()) <= exported


def test_create_without_gpu_reports_cuda_error():
    import ctypes
    import torch
    import paper_2010_09701_gb300 as P
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = P.load()
    h = ctypes.c_void_p()
    assert lib.oefe_create(ctypes.byref(h), 0, None) == P.binding.ERR_CUDA
    assert lib.oefe_destroy(None) == 0
    assert lib.oefe_mesh(None, 1.0, None, None, 1) == P.binding.ERR_ARG


def test_no_oracle_import_in_product_code():
    pkg = os.path.join(ROOT, "paper_2010_09701_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower().replace("oracle-free", ""), f
