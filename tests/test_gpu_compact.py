"""Storage and width limits of the FP64-class path: the compact layout of the
FP64 / FP32-pair cell matrices (whole matrices only for cells with several
quadrature leaves, enrichment strips for single-leaf cells) gives the same
products as the full layout; blocks wider than one pass (64 vectors for an
operator application, 128 per k-point for the batched filter) go through in
column chunks and match the oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_cases import paired, rel, to_gpu
from oracle import solver

pytestmark = pytest.mark.gpu

KS = [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)]


def colerr(out, ref):
    return np.max(np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0))


def _case(k):
    # a 4^3 mesh: 48 single-leaf cells and 16 refined around the two nuclei
    return paired(ks=[k], n=4, a=8.0)


@pytest.mark.parametrize("products", ["native", "pairs"])
@pytest.mark.parametrize("k", KS)
def test_compact_layout_same_products(k, products):
    from paper_2010_09701_gb300 import (F64_NATIVE, F64_PAIRS, STORE_COMPACT, STORE_F64, STORE_F64PAIR, OefeError,
                                        binding)
    prs, ctx, V, Vd = _case(k)
    pr = prs[0]
    pair_bits = STORE_F64PAIR if products == "pairs" else 0
    ctx.set_f64_products(F64_PAIRS if products == "pairs" else F64_NATIVE)
    X = to_gpu(W.random_vectors(pr.n, 11, complex_=pr.complex, seed=41))
    ctx.build_hamiltonian(Vd, STORE_F64 | pair_bits)
    Yf = torch.empty_like(X)
    ctx.apply_h(0, X, Yf)
    Af = torch.empty_like(X)
    ctx.apply_a(0, X, Af)
    ncells = len(pr.cells)
    full = {e: ctx.cell_matrix(0, e, complex_=pr.complex) for e in range(ncells)}
    ctx.build_hamiltonian(Vd, STORE_F64 | pair_bits | STORE_COMPACT)
    Yc = torch.empty_like(X)
    ctx.apply_h(0, X, Yc)
    Ac = torch.empty_like(X)
    ctx.apply_a(0, X, Ac)
    # the same stored values read from other addresses: the same numbers
    assert rel(Yc.cpu().numpy(), Yf.cpu().numpy()) < 1e-15
    assert rel(Ac.cpu().numpy(), Af.cpu().numpy()) < 1e-15
    # and the oracle's H X
    scale = abs(pr.assemble_H()) @ np.abs(X.cpu().numpy())
    assert np.max(np.abs(Yc.cpu().numpy() - pr.apply_H(X.cpu().numpy())) / scale) < (3.2e-12 if pair_bits else 1e-13)
    # whole matrices are kept for the refined cells only
    kept = 0
    for e in range(ncells):
        try:
            H = ctx.cell_matrix(0, e, complex_=pr.complex)
        except OefeError as err:
            assert err.code == binding.ERR_STATE
            continue
        kept += 1
        assert np.array_equal(H, full[e])
    assert kept == 16
    # back to the full layout
    ctx.build_hamiltonian(Vd, STORE_F64 | pair_bits)
    ctx.apply_h(0, X, Yc)
    assert rel(Yc.cpu().numpy(), Yf.cpu().numpy()) < 1e-15
    ctx.set_f64_products(F64_NATIVE)


def test_compact_needs_fp64_copy():
    from paper_2010_09701_gb300 import STORE_BF16X3, STORE_COMPACT, OefeError, binding
    prs, ctx, V, Vd = _case(KS[1])
    with pytest.raises(OefeError) as e:
        ctx.build_hamiltonian(Vd, STORE_BF16X3 | STORE_COMPACT)
    assert e.value.code == binding.ERR_ARG


@pytest.mark.parametrize("k", KS)
def test_wide_blocks_in_chunks(k):
    # 150 vectors: three passes of the operator application and of the per-k FP64 filter
    from paper_2010_09701_gb300 import STORE_COMPACT, STORE_F64
    prs, ctx, V, Vd = _case(k)
    pr = prs[0]
    ctx.build_hamiltonian(Vd, STORE_F64 | STORE_COMPACT)
    X = W.random_vectors(pr.n, 150, complex_=pr.complex, seed=43)
    Y = torch.empty_like(to_gpu(X))
    ctx.apply_h(0, to_gpu(X), Y)
    scale = abs(pr.assemble_H()) @ np.abs(X)
    assert np.max(np.abs(Y.cpu().numpy() - pr.apply_H(X)) / scale) < 1e-13
    a, b, a0 = 5.0, 2500.0, -10.0
    ref = solver.chebyshev_filter(pr.apply_A, X, 6, a, b, a0)
    Xd = to_gpu(X)
    ctx.chebyshev_filter(0, Xd, 6, a, b, a0)
    assert colerr(Xd.cpu().numpy(), ref) < 1e-10


def test_batched_filter_in_column_groups():
    # 300 vectors per k-point (three groups of at most 128), compact FP64 storage, BF16x6 split:
    # the plain low-precision filter and the defect form from arbitrary pairs, against the oracle
    from paper_2010_09701_gb300 import FILTER_BF16X3, STORE_BF16X6, STORE_COMPACT, STORE_F64
    prs, ctx, V, Vd = paired(ks=[(0.3, 0.0, 0.0), (-0.3, 0.1, 0.0)], n=4, a=8.0)
    ctx.build_hamiltonian(Vd, STORE_F64 | STORE_BF16X6 | STORE_COMPACT)
    nvs = [300, 260]
    a, b, a0, deg = 5.0, 2500.0, -10.0, 5
    Xs = [W.random_vectors(pr.n, nv, complex_=True, seed=50 + i) for i, (pr, nv) in enumerate(zip(prs, nvs))]
    refs = [solver.chebyshev_filter(pr.apply_A, Xk, deg, a, b, a0) for pr, Xk in zip(prs, Xs)]
    Xl = [to_gpu(Xk, torch.complex64) for Xk in Xs]
    ctx.filter_batched(Xl, deg, a, b, a0, FILTER_BF16X3)
    for out, ref in zip(Xl, refs):
        assert colerr(out.cpu().numpy().astype(np.complex128), ref) < 5e-5
    rng = np.random.default_rng(7)
    th = [rng.uniform(a0, a, nv) for nv in nvs]
    for rep in range(2):   # the second call replays the three cached graphs
        Xd = [to_gpu(Xk) for Xk in Xs]
        ctx.filter_batched_defect(Xd, deg, a, b, a0, th, FILTER_BF16X3)
        for out, ref in zip(Xd, refs):
            assert colerr(out.cpu().numpy(), ref) < 5e-5, rep
