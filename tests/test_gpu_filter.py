"""GPU parity of M^{-1}H application and of the Chebyshev filter (Sec. IV)
against the oracle, FP64 and FP32 paths, with ragged column counts."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_cases import c1_pair, paired, rel, to_gpu
from oracle import solver

pytestmark = pytest.mark.gpu

KS = [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)]


def gpu_dtype(pr, fp32=False):
    if pr.complex:
        return torch.complex64 if fp32 else torch.complex128
    return torch.float32 if fp32 else torch.float64


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("nv", [1, 7, 37])
def test_apply_h_and_a(k, nv):
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    X = W.random_vectors(pr.n, nv, complex_=pr.complex, seed=nv)
    Xd = to_gpu(X)
    Y = torch.empty_like(Xd)
    ctx.apply_h(0, Xd, Y)
    assert rel(Y.cpu().numpy(), pr.apply_H(X)) < 1e-13
    ctx.apply_a(0, Xd, Y)
    assert rel(Y.cpu().numpy(), pr.apply_A(X)) < 1e-13


def test_apply_with_leading_dimension():
    prs, ctx, V, _ = paired()
    pr = prs[0]
    X = W.random_vectors(pr.n, 5, seed=2)
    big = torch.zeros(pr.n, 9, dtype=torch.float64, device="cuda")
    big[:, :5] = to_gpu(X)
    out = torch.full((pr.n, 9), 7.0, dtype=torch.float64, device="cuda")
    ctx.apply_a(0, big[:, :5], out[:, :5])
    assert rel(out[:, :5].cpu().numpy(), pr.apply_A(X)) < 1e-13
    assert torch.all(out[:, 5:] == 7.0)


def bounds(pr):
    import scipy.linalg as sla
    ev = sla.eigh(pr.assemble_H().toarray(), pr.dense_M(), eigvals_only=True)
    return ev[6], ev[-1] * 1.01, ev[0] - 1.0


@pytest.mark.parametrize("k", KS)
def test_filter_fp64(k):
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, 12, complex_=pr.complex, seed=3)
    ref = solver.chebyshev_filter(pr.apply_A, X, 9, a, b, a0)
    Xd = to_gpu(X)
    ctx.chebyshev_filter(0, Xd, 9, a, b, a0)
    assert rel(Xd.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("k", KS)
def test_filter_fp32(k):
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, 33, complex_=pr.complex, seed=4)
    ref = solver.chebyshev_filter(pr.apply_A, X, 9, a, b, a0)
    Xd = to_gpu(X, gpu_dtype(pr, fp32=True))
    ctx.chebyshev_filter(0, Xd, 9, a, b, a0)
    # FP32 cell products: error ~ eps32 * (filter growth); compare column-normalized
    out = Xd.cpu().numpy().astype(ref.dtype)
    nrm = np.linalg.norm(ref, axis=0)
    assert np.max(np.linalg.norm(out - ref, axis=0) / nrm) < 2e-5


def test_filter_single_degree_and_degenerate_shapes():
    prs, ctx, V, _ = paired(a=5.0, n=1, p=4, Zs=(3,), pos=[[1.0, 1.5, 2.0]], quad=(5, 6, 2), r0=1.2, rc=2.0)
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, 3, seed=1)
    for m in (1, 2, 3):
        ref = solver.chebyshev_filter(pr.apply_A, X, m, a, b, a0)
        Xd = to_gpu(X)
        ctx.chebyshev_filter(0, Xd, m, a, b, a0)
        assert rel(Xd.cpu().numpy(), ref) < 1e-11


def test_filter_c1():
    # the first configuration: 8^3 graded cells, p = 4, two nuclei, 20 vectors, degree 20
    w = W.config_c1()
    prs, ctx, V, _ = c1_pair()
    pr = prs[0]
    X = W.random_vectors(pr.n, 20, seed=w.seed)
    Xd = to_gpu(X)
    # bounds: a from the free spectrum region, b from a Lanczos estimate on the oracle
    b = solver.lanczos_upper_bound(pr.apply_H, pr.apply_M, pr.apply_Minv, W.random_vectors(pr.n, 1, seed=9)[:, 0], 25)
    a, a0 = 0.0, -0.5 * 14 ** 2 - 1.0
    ref = solver.chebyshev_filter(pr.apply_A, X, w.degree, a, b, a0)
    ctx.chebyshev_filter(0, Xd, w.degree, a, b, a0)
    assert rel(Xd.cpu().numpy(), ref) < 1e-10
    # Lanczos bound: after the top Ritz value converges, orthogonality is lost and
    # the residual term differs run to run; both bounds must sit above the top
    # Ritz value of the oracle's run and agree to a few per cent.
    v0 = to_gpu(W.random_vectors(pr.n, 1, seed=9))
    bg = ctx.upper_bound(0, v0, 25)
    assert abs(bg - b) < 2e-2 * abs(b)


def test_upper_bound_small():
    import scipy.linalg as sla
    prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)])
    pr = prs[0]
    ev = sla.eigh(pr.assemble_H().toarray(), pr.dense_M(), eigvals_only=True)
    v0 = to_gpu(W.random_vectors(pr.n, 1, complex_=True, seed=3))
    bg = ctx.upper_bound(0, v0, 30)
    assert ev[-1] - 1e-8 <= bg < 1.2 * ev[-1]


def test_argument_errors():
    from paper_2010_09701_gb300 import OefeError, binding
    prs, ctx, V, _ = paired()
    pr = prs[0]
    Xd = to_gpu(W.random_vectors(pr.n, 4, complex_=True, seed=1))
    with pytest.raises(OefeError) as e:
        ctx.apply_h(0, Xd, torch.empty_like(Xd))     # k = 0 needs a real dtype
    assert e.value.code == binding.ERR_ARG
    Xr = to_gpu(W.random_vectors(pr.n, 4, seed=1))
    with pytest.raises(OefeError) as e:
        ctx.chebyshev_filter(0, Xr, 3, 1.0, 0.5, 0.0)   # b < a
    assert e.value.code == binding.ERR_ARG
    with pytest.raises(OefeError) as e:
        ctx.apply_h(3, Xr, torch.empty_like(Xr))
    assert e.value.code == binding.ERR_ARG
    from paper_2010_09701_gb300 import Context
    c2 = Context(0)
    with pytest.raises(OefeError) as e:
        c2.quadrature(3, 3, 1)
    assert e.value.code == binding.ERR_STATE


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("deg", [2, 3, 9])
def test_filter_mixed_last_fp64(k, deg):
    from paper_2010_09701_gb300 import FILTER_LAST_FP64
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, 21, complex_=pr.complex, seed=deg)
    ref = solver.chebyshev_filter(pr.apply_A, X, deg, a, b, a0)
    Xd = to_gpu(X)
    ctx.chebyshev_filter(0, Xd, deg, a, b, a0, flags=FILTER_LAST_FP64)
    out = Xd.cpu().numpy()
    nrm = np.linalg.norm(ref, axis=0)
    err = np.max(np.linalg.norm(out - ref, axis=0) / nrm)
    assert err < 2e-5
    assert err > 1e-13          # the FP32 degrees did run


@pytest.mark.parametrize("k", KS)
def test_apply_h_c1_sum_factorized_cells(k):
    # the graded 8^3 mesh: 496 single-leaf cells take the sum-factorized FP64 product, the 16
    # octree-refined cells around the nuclei the dense one
    w = W.config_c1()
    xb = W.mesh_breakpoints(w)
    prs, ctx, V, _ = paired(a=w.a, p=w.p, Zs=tuple(w.Z), pos=w.pos, xb=xb, quad=w.quad_params(), r0=w.r0,
                            rc=w.rc, sigma=w.sigma, ks=[k])
    pr = prs[0]
    X = W.random_vectors(pr.n, 13, complex_=pr.complex, seed=21)
    Y = torch.empty_like(to_gpu(X))
    ctx.apply_h(0, to_gpu(X), Y)
    HX = pr.apply_H(X)
    assert rel(Y.cpu().numpy(), HX) < 1e-13
    # rounding of any summation order: |dY| <= c eps (|H| |X|) row by row
    scale = abs(pr.assemble_H()) @ np.abs(X)
    assert np.max(np.abs(Y.cpu().numpy() - HX) / scale) < 1e-13
    ctx.apply_a(0, to_gpu(X), Y)
    Ya = Y.cpu().numpy()
    # M^{-1}: the lumped CFE rows scale row by row; the enrichment rows go through (M^oo)^{-1},
    # whose condition number amplifies the rounding of H X, so they are checked by the residual
    nh = pr.nh
    assert np.max(np.abs(Ya[:nh] - HX[:nh] / pr.m[:, None]) * pr.m[:, None] / scale[:nh]) < 1e-13
    res = pr.Moo @ Ya[nh:] - HX[nh:]
    assert np.linalg.norm(res) < 1e-13 * np.linalg.norm(pr.Moo, 2) * np.linalg.norm(Ya[nh:])


@pytest.mark.parametrize("k", KS)
def test_apply_h_c1_fp32_pair_products(k):
    # FP32-pair arithmetic on the 496 single-leaf cells (the refined cells stay FP64). Each pair
    # operation rounds at about u = 2^-48 instead of 2^-53, so the row-wise rounding bound of the
    # FP64 test (1e-13 of |H| |X|, about 900 u64) becomes 900 u = 3.2e-12.
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS, STORE_F64, STORE_F64PAIR, OefeError
    w = W.config_c1()
    xb = W.mesh_breakpoints(w)
    prs, ctx, V, _ = paired(a=w.a, p=w.p, Zs=tuple(w.Z), pos=w.pos, xb=xb, quad=w.quad_params(), r0=w.r0,
                            rc=w.rc, sigma=w.sigma, ks=[k], store=STORE_F64 | STORE_F64PAIR)
    pr = prs[0]
    X = W.random_vectors(pr.n, 13, complex_=pr.complex, seed=22)
    Xd = to_gpu(X)
    Yp = torch.empty_like(Xd)
    Yn = torch.empty_like(Xd)
    ctx.set_f64_products(F64_PAIRS)
    ctx.apply_h(0, Xd, Yp)
    ctx.set_f64_products(F64_NATIVE)
    ctx.apply_h(0, Xd, Yn)
    HX = pr.apply_H(X)
    scale = abs(pr.assemble_H()) @ np.abs(X)
    err = np.max(np.abs(Yp.cpu().numpy() - HX) / scale)
    assert err < 3.2e-12
    # the pair path ran: it differs from FP64 by more than FP64 rounding alone
    assert np.max(np.abs(Yp.cpu().numpy() - Yn.cpu().numpy()) / scale) > 1e-15
    # every launch shape of the pair product gives the same products
    ctx.set_f64_products(F64_PAIRS)
    Ys = torch.empty_like(Xd)
    for shape in (0, 1, 2):
        ctx.set_product_shape(shape)
        ctx.apply_h(0, Xd, Ys)
        ys = Ys.cpu().numpy()
        assert np.max(np.abs(ys - HX) / scale) < 3.2e-12
        assert np.max(np.abs(ys - Yp.cpu().numpy()) / scale) < 1e-14
    ctx.set_product_shape(-1)
    with pytest.raises(OefeError):
        ctx.set_product_shape(3)
    ctx.set_f64_products(F64_NATIVE)
    with pytest.raises(OefeError):
        ctx.set_f64_products(7)
    # an operator without the pair copy refuses pair products
    ctx.build_hamiltonian(to_gpu(V), STORE_F64)
    ctx.set_f64_products(F64_PAIRS)
    with pytest.raises(OefeError):
        ctx.apply_h(0, Xd, Yp)
    ctx.set_f64_products(F64_NATIVE)
