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


def test_occupations_host_call_matches_oracle():
    # oefe_occupations is host-only: it runs here without a GPU
    import numpy as np
    import paper_2010_09701_gb300 as P
    from oracle import solver
    rng = np.random.default_rng(4)
    eigs = [np.sort(rng.uniform(-5, 2, 12)), np.sort(rng.uniform(-5, 2, 9))]
    w = [0.25, 0.75]
    for Ne in (3.0, 7.5, 12.0):
        mu, occ, eb = P.occupations(eigs, w, Ne, 500.0)
        mu_o = solver.fermi_level(eigs, w, Ne, 500.0)
        occ_o = solver.occupations(eigs, w, mu_o)
        assert abs(sum(o.sum() for o in occ) - Ne) < 1e-10
        for a, b in zip(occ, occ_o):
            assert np.allclose(a, b, atol=1e-9)
        assert abs(eb - solver.band_energy(eigs, w, mu_o)) < 1e-8
    with pytest.raises(P.OefeError):
        P.occupations(eigs, w, 100.0)
