"""GPU parity of Cholesky-QR, Rayleigh-Ritz (Eq. ProjKS), the density
(Eq. rho) and the adjoint of H.X against the oracle."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import workloads as W
from gpu_cases import c1_pair, paired, rel, to_gpu
from oracle import solver

pytestmark = pytest.mark.gpu

KS = [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)]


def _products(ctx, products):
    # FP32-pair arithmetic rounds at u = 2^-48, 2^5 times the FP64 unit: the FP64 tolerances scale
    # by 32
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS
    ctx.set_f64_products(F64_PAIRS if products == "pairs" else F64_NATIVE)
    return 32.0 if products == "pairs" else 1.0


def _store(products):
    from paper_2010_09701_gb300 import STORE_BF16X3, STORE_F32, STORE_F64, STORE_F64PAIR
    return STORE_F64 | STORE_F32 | STORE_BF16X3 | (STORE_F64PAIR if products == "pairs" else 0)


@pytest.mark.parametrize("products", ["native", "pairs"])
@pytest.mark.parametrize("k", KS)
def test_orthonormalize(k, products):
    prs, ctx, V, _ = paired(ks=[k], store=_store(products))
    f = _products(ctx, products)
    pr = prs[0]
    Y = W.random_vectors(pr.n, 10, complex_=pr.complex, seed=5)
    Yd = to_gpu(Y)
    ctx.orthonormalize(0, Yd)
    Q = Yd.cpu().numpy()
    assert np.allclose(Q.conj().T @ pr.apply_M(Q), np.eye(10), atol=1e-12 * f)
    Qo = solver.cholqr(Y, pr.apply_M)
    # same span: Q = Qo U with U unitary -> Qo^+ M Q unitary
    U = Qo.conj().T @ pr.apply_M(Q)
    assert np.allclose(U.conj().T @ U, np.eye(10), atol=1e-11 * f)
    # CholQR is deterministic: the factors agree too
    assert rel(Q, Qo) < 1e-10 * f


@pytest.mark.parametrize("case", ["c1_real_64", "complex_24", "complex_64", "real_150", "real_300", "complex_100"])
def test_orthonormalize_tensor_core_gram(case):  # Gram and rotations on the tensor cores
    # pair mode takes the Gram matrices on the tensor cores (exact bf16 digits, about 2^-46 of the
    # row and column maxima per term): Q^+ M Q = I and Q against the native FP64 path within the
    # pair tolerances (32x the FP64 ones); 64 real vectors fill the 128-row MMA tile, and so do 64
    # complex ones (128 real rows: the benchmark's shape)
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS
    if case == "c1_real_64":
        prs, ctx, V, _ = c1_pair()
        nv = 64
    elif case == "complex_64":
        prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)], n=4, a=8.0)
        nv = 64
    elif case in ("real_150", "real_300"):   # wider than one digit tile: the digits cut inside the MMA
        # kernels; a real Gram matrix runs only its tiles that meet the upper triangle (4 of 6, 9 of 15)
        prs, ctx, V, _ = paired(n=4, a=8.0)
        nv = int(case.split("_")[1])
    elif case == "complex_100":
        prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)], n=4, a=8.0)
        nv = 100
    else:
        prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)])
        nv = 24
    pr = prs[0]
    Y = W.random_vectors(pr.n, nv, complex_=pr.complex, seed=31)
    ctx.set_f64_products(F64_PAIRS)
    Yp = to_gpu(Y)
    ctx.orthonormalize(0, Yp)
    ctx.set_f64_products(F64_NATIVE)
    Yn = to_gpu(Y)
    ctx.orthonormalize(0, Yn)
    Q = Yp.cpu().numpy()
    assert np.allclose(Q.conj().T @ pr.apply_M(Q), np.eye(nv), atol=32e-12)
    assert rel(Q, Yn.cpu().numpy()) < 32e-10


def test_orthonormalize_rank_deficient_reports_cholesky():
    from paper_2010_09701_gb300 import OefeError, binding
    prs, ctx, V, _ = paired()
    pr = prs[0]
    Y = W.random_vectors(pr.n, 4, seed=5)
    Y[:, 3] = Y[:, 1]
    with pytest.raises(OefeError) as e:
        ctx.orthonormalize(0, to_gpu(Y))
    assert e.value.code == binding.ERR_CHOLESKY


@pytest.mark.parametrize("products", ["native", "pairs"])
@pytest.mark.parametrize("k", KS)
def test_rayleigh_ritz(k, products):
    prs, ctx, V, _ = paired(ks=[k], store=_store(products))
    f = _products(ctx, products)
    pr = prs[0]
    Q = solver.cholqr(W.random_vectors(pr.n, 9, complex_=pr.complex, seed=6), pr.apply_M)
    eps_o, X_o = solver.rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
    Qd = to_gpu(Q)
    eps, res = ctx.rayleigh_ritz(0, Qd, resid=True)
    assert np.max(np.abs(eps - eps_o)) < 1e-10 * f * max(1, np.max(np.abs(eps_o)))
    res_o = solver.residual_norms(pr, X_o, eps_o)
    assert np.allclose(res, res_o, rtol=1e-8 * f, atol=1e-12 * f)
    # rotated vectors: unique up to a phase per (non-degenerate) column
    X = Qd.cpu().numpy()
    ph = np.sum(np.conj(X_o) * pr.apply_M(X), axis=0)
    assert np.allclose(np.abs(ph), 1.0, atol=1e-9 * f)


@pytest.mark.parametrize("k", KS)
def test_rayleigh_ritz_tensor_core_64(k):
    # the benchmark's shape in pair mode: 64 vectors (64 complex = 128 real rows, a full MMA tile),
    # Gram matrices and rotations on the tensor cores, H X by FP32-pair products on the single-leaf
    # cells of a 4^3 mesh, the projected problem by pair then FP64 Jacobi sweeps
    from paper_2010_09701_gb300 import F64_PAIRS, STORE_F64, STORE_F64PAIR
    prs, ctx, V, _ = paired(ks=[k], n=4, a=8.0, store=STORE_F64 | STORE_F64PAIR)
    ctx.set_f64_products(F64_PAIRS)
    f = 32.0
    pr = prs[0]
    nv = 64
    Q = solver.cholqr(W.random_vectors(pr.n, nv, complex_=pr.complex, seed=6), pr.apply_M)
    eps_o, X_o = solver.rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
    Qd = to_gpu(Q)
    eps, res = ctx.rayleigh_ritz(0, Qd, resid=True)
    assert np.max(np.abs(eps - eps_o)) < 1e-10 * f * max(1, np.max(np.abs(eps_o)))
    res_o = solver.residual_norms(pr, X_o, eps_o)
    assert np.allclose(res, res_o, rtol=1e-8 * f, atol=1e-12 * f * max(1, np.max(np.abs(eps_o))))
    # the rotated vectors span the same Ritz directions: |<x_o, M x>| = 1 per well-separated column
    X = Qd.cpu().numpy()
    gaps = np.minimum(np.abs(np.diff(eps_o, prepend=-np.inf)), np.abs(np.diff(eps_o, append=np.inf)))
    sep = gaps > 1e-6 * max(1, np.max(np.abs(eps_o)))
    ph = np.sum(np.conj(X_o) * pr.apply_M(X), axis=0)
    assert np.allclose(np.abs(ph[sep]), 1.0, atol=1e-9 * f)


@pytest.mark.parametrize("products", ["native", "pairs"])
@pytest.mark.parametrize("k", KS)
def test_adjoint_entry_points(k, products):
    # oefe_band_trace, oefe_band_trace_vjp and oefe_apply_h_vjp through the C ABI against the
    # oracle: the trace, 2 alpha H X, alpha w_q sum |u|^2, H G and w_q Re sum conj(u_G) u_X
    # (pairs: the fields and the products in FP32 pairs, 32 times the FP64 tolerances)
    prs, ctx, V, Vd = paired(ks=[k], n=4, a=8.0, store=_store(products))
    f = _products(ctx, products)
    pr = prs[0]
    X = W.random_vectors(pr.n, 5, complex_=pr.complex, seed=13)
    G = W.random_vectors(pr.n, 5, complex_=pr.complex, seed=14)
    Xd, Gd = to_gpu(X), to_gpu(G)
    HX = torch.empty_like(Xd)
    e = ctx.band_trace(0, Xd, HX)
    HXo = pr.apply_H(X)
    assert abs(e - np.real(np.sum(np.conj(X) * HXo))) < 1e-12 * f * abs(e)
    assert rel(HX.cpu().numpy(), HXo) < 1e-12 * f
    assert abs(ctx.band_trace(0, Xd) - e) <= 1e-13 * f * abs(e)   # into the context's workspace
    alpha = -0.7
    gV = torch.empty(pr.quad.nq, dtype=torch.float64, device="cuda")
    gX = torch.empty_like(Xd)
    ctx.band_trace_vjp(0, Xd, alpha, gV, gX)
    assert rel(gV.cpu().numpy(), alpha * solver.band_trace_grad_V(pr, X)) < 1e-12 * f
    assert rel(gX.cpu().numpy(), 2 * alpha * HXo) < 1e-12 * f
    gV2 = torch.empty_like(gV)
    gX2 = torch.empty_like(Xd)
    ctx.apply_h_vjp(0, Xd, Gd, gV2, gX2)
    uG = [pr.values_at_points(e_, G) for e_ in range(pr.mesh.ncells)]
    uX = [pr.values_at_points(e_, X) for e_ in range(pr.mesh.ncells)]
    cross = np.concatenate([np.real(np.sum(np.conj(a) * b, axis=1)) for a, b in zip(uG, uX)]) * pr.quad.weights
    assert rel(gV2.cpu().numpy(), cross) < 1e-12 * f
    assert rel(gX2.cpu().numpy(), pr.apply_H(G)) < 1e-12 * f
    # either output alone
    gV3 = torch.empty_like(gV)
    ctx.apply_h_vjp(0, Xd, Gd, gV3, None)
    assert torch.equal(gV3, gV2)
    # G = X gives the band-trace gradient
    ctx.apply_h_vjp(0, Xd, Xd, gV3, None)
    assert rel(gV3.cpu().numpy(), solver.band_trace_grad_V(pr, X)) < 1e-12 * f
    from paper_2010_09701_gb300 import F64_NATIVE
    ctx.set_f64_products(F64_NATIVE)


@pytest.mark.parametrize("products", ["native", "pairs"])
@pytest.mark.parametrize("nv", [97, 150])
@pytest.mark.parametrize("k", KS)
def test_rayleigh_ritz_wide(k, nv, products):
    # projected problems too large for one CTA's shared memory: the Jacobi rounds spread over the GPU
    # (odd nv: one index sits out each round); in pair mode the Gram matrices and the rotation of
    # more than 64 vectors on the tensor cores with the digits cut in the kernels
    prs, ctx, V, _ = paired(ks=[k], n=4, a=8.0, store=_store(products))
    f = _products(ctx, products)
    pr = prs[0]
    Q = solver.cholqr(W.random_vectors(pr.n, nv, complex_=pr.complex, seed=16), pr.apply_M)
    eps_o, X_o = solver.rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
    Qd = to_gpu(Q)
    eps, res = ctx.rayleigh_ritz(0, Qd, resid=True)
    assert np.max(np.abs(eps - eps_o)) < 1e-10 * f * max(1, np.max(np.abs(eps_o)))
    res_o = solver.residual_norms(pr, X_o, eps_o)
    assert np.allclose(res, res_o, rtol=1e-8 * f, atol=1e-12 * f * max(1, np.max(np.abs(eps_o))))
    X = Qd.cpu().numpy()
    # M-orthonormal Ritz vectors spanning the oracle's: |<x_o, M x>| = 1 where the values are apart
    assert np.allclose(X.conj().T @ pr.apply_M(X), np.eye(nv), atol=1e-11 * f)
    gaps = np.minimum(np.abs(np.diff(eps_o, prepend=-np.inf)), np.abs(np.diff(eps_o, append=np.inf)))
    sep = gaps > 1e-6 * max(1, np.max(np.abs(eps_o)))
    ph = np.sum(np.conj(X_o) * pr.apply_M(X), axis=0)
    assert np.allclose(np.abs(ph[sep]), 1.0, atol=1e-9 * f)
    from paper_2010_09701_gb300 import F64_NATIVE
    ctx.set_f64_products(F64_NATIVE)


@pytest.mark.parametrize("k", KS)
def test_density_and_band_trace_grad(k):
    prs, ctx, V, Vd = paired(ks=[k])
    pr = prs[0]
    X = W.random_vectors(pr.n, 6, complex_=pr.complex, seed=8)
    occ = np.array([2.0, 2.0, 1.5, 1.0, 0.2, 0.0])
    rho_o = solver.density([pr], [X], [occ])
    rho = torch.zeros(pr.quad.nq, dtype=torch.float64, device="cuda")
    ctx.density([to_gpu(X)], [occ], rho)
    assert rel(rho.cpu().numpy(), rho_o) < 1e-12
    g_o = solver.band_trace_grad_V(pr, X)
    g = torch.zeros_like(rho)
    ctx.band_trace_grad(0, to_gpu(X), g)
    assert rel(g.cpu().numpy(), g_o) < 1e-12


@pytest.mark.parametrize("k", KS)
def test_density_and_band_trace_grad_fp32_pairs(k):
    # the fields in FP32-pair arithmetic: each operation rounds at about u = 2^-48, so the FP64
    # bound of 1e-12 (about 9000 u64) becomes 3.2e-12 (900 u)
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS
    prs, ctx, V, Vd = paired(ks=[k])
    pr = prs[0]
    X = W.random_vectors(pr.n, 6, complex_=pr.complex, seed=18)
    occ = np.array([2.0, 2.0, 1.5, 1.0, 0.2, 0.0])
    rho_o = solver.density([pr], [X], [occ])
    ctx.set_f64_products(F64_PAIRS)
    rho = torch.zeros(pr.quad.nq, dtype=torch.float64, device="cuda")
    ctx.density([to_gpu(X)], [occ], rho)
    assert rel(rho.cpu().numpy(), rho_o) < 3.2e-12
    g_o = solver.band_trace_grad_V(pr, X)
    g = torch.zeros_like(rho)
    ctx.band_trace_grad(0, to_gpu(X), g)
    assert rel(g.cpu().numpy(), g_o) < 3.2e-12
    ctx.set_f64_products(F64_NATIVE)
    g2 = torch.zeros_like(rho)
    ctx.band_trace_grad(0, to_gpu(X), g2)
    assert rel(g2.cpu().numpy(), g_o) < 1e-12


def test_density_two_kpoints():
    ks = [(0.3, 0.0, 0.0), (-0.3, 0.1, 0.0)]
    prs, ctx, V, Vd = paired(ks=ks)
    Xs = [W.random_vectors(pr.n, 5, complex_=True, seed=i) for i, pr in enumerate(prs)]
    occs = [np.array([1.0, 1.0, 0.5, 0.25, 0.0]) * 0.5, np.array([1.0, 0.9, 0.5, 0.1, 0.0]) * 0.5]
    rho_o = solver.density(prs, Xs, occs)
    rho = torch.zeros(prs[0].quad.nq, dtype=torch.float64, device="cuda")
    ctx.density([to_gpu(x) for x in Xs], occs, rho)
    assert rel(rho.cpu().numpy(), rho_o) < 1e-12


@pytest.mark.parametrize("products", ["native", "pairs"])
def test_density_grad_one_field_pass(products):
    # density over two k-points and the band-trace gradient of the second from the same field pass:
    # the oracle's density and gradient, and the separate calls' results (same arithmetic per point)
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS
    ks = [(0.3, 0.0, 0.0), (-0.3, 0.1, 0.0)]
    prs, ctx, V, Vd = paired(ks=ks)
    ctx.set_f64_products(F64_PAIRS if products == "pairs" else F64_NATIVE)
    tol = 3.2e-12 if products == "pairs" else 1e-12
    Xs = [W.random_vectors(pr.n, 5 + i, complex_=True, seed=40 + i) for i, pr in enumerate(prs)]
    occs = [np.array([1.0, 1.0, 0.5, 0.25, 0.0]) * 0.5, np.array([1.0, 0.9, 0.5, 0.1, 0.0, 0.0]) * 0.5]
    Xd = [to_gpu(x) for x in Xs]
    nq = prs[0].quad.nq
    rho = torch.zeros(nq, dtype=torch.float64, device="cuda")
    g = torch.full((nq,), 7.0, dtype=torch.float64, device="cuda")   # overwritten
    ctx.density_grad(Xd, occs, rho, 1, g)
    assert rel(rho.cpu().numpy(), solver.density(prs, Xs, occs)) < tol
    assert rel(g.cpu().numpy(), solver.band_trace_grad_V(prs[1], Xs[1])) < tol
    rho1 = torch.zeros_like(rho)
    g1 = torch.zeros_like(rho)
    ctx.density(Xd, occs, rho1)
    ctx.band_trace_grad(1, Xd[1], g1)
    assert rel(rho.cpu().numpy(), rho1.cpu().numpy()) < 1e-14 and rel(g.cpu().numpy(), g1.cpu().numpy()) < 1e-14
    with pytest.raises(Exception):
        ctx.density_grad(Xd, occs, rho, 2, g)
    ctx.set_f64_products(F64_NATIVE)


@pytest.mark.parametrize("k", KS)
def test_autograd_band_trace(k):
    from paper_2010_09701_gb300.autograd import apply_h, band_trace
    prs, ctx, V, Vd = paired(ks=[k])
    pr = prs[0]
    X = W.random_vectors(pr.n, 3, complex_=pr.complex, seed=11)
    Vt = Vd.clone().requires_grad_(True)
    Xt = to_gpu(X).requires_grad_(True)
    E = band_trace(Vt, Xt, ctx, 0)
    E.backward()
    assert abs(E.item() - np.real(np.sum(np.conj(X) * pr.apply_H(X)))) < 1e-12 * abs(E.item())
    assert rel(Vt.grad.cpu().numpy(), solver.band_trace_grad_V(pr, X)) < 1e-12
    assert rel(Xt.grad.cpu().numpy(), 2 * pr.apply_H(X)) < 1e-12
    # central differences on the GPU path itself, h = 1e-4 (E is affine in V)
    rng = np.random.default_rng(0)
    for q in rng.choice(pr.quad.nq, 4, replace=False):
        Vp, Vm = Vd.clone(), Vd.clone()
        Vp[q] += 1e-4
        Vm[q] -= 1e-4
        fd = (band_trace(Vp, Xt.detach(), ctx, 0).item() - band_trace(Vm, Xt.detach(), ctx, 0).item()) / 2e-4
        assert abs(fd - Vt.grad[q].item()) < 1e-6 * max(1.0, abs(fd))
    # vector-Jacobian product of Y = H(V) X
    G = W.random_vectors(pr.n, 3, complex_=pr.complex, seed=12)
    Vt2 = Vd.clone().requires_grad_(True)
    Xt2 = to_gpu(X).requires_grad_(True)
    Y = apply_h(Vt2, Xt2, ctx, 0)
    Y.backward(to_gpu(G))
    uG = [pr.values_at_points(e, G) for e in range(pr.mesh.ncells)]
    uX = [pr.values_at_points(e, X) for e in range(pr.mesh.ncells)]
    cross = np.concatenate([np.real(np.sum(np.conj(a) * b, axis=1)) for a, b in zip(uG, uX)]) * pr.quad.weights
    assert rel(Vt2.grad.cpu().numpy(), cross) < 1e-11
    assert rel(Xt2.grad.cpu().numpy(), pr.apply_H(G)) < 1e-12


def test_c1_pass_eigenvalues_and_density():
    # one full pass on the first configuration, GPU FP64 against the oracle:
    # eigenvalues within 1e-8 Ha and density L2 error within 1e-8
    w = W.config_c1()
    prs, ctx, V, Vd = c1_pair()
    pr = prs[0]
    X = W.random_vectors(pr.n, 20, seed=w.seed)
    b = solver.lanczos_upper_bound(pr.apply_H, pr.apply_M, pr.apply_Minv, W.random_vectors(pr.n, 1, seed=9)[:, 0], 25)
    a, a0 = 0.0, -0.5 * 14 ** 2 - 1.0
    Y = solver.chebyshev_filter(pr.apply_A, X, w.degree, a, b, a0)
    Q = solver.cholqr(Y, pr.apply_M)
    eps_o, Xo = solver.rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
    mu = solver.fermi_level([eps_o], [1.0], w.nelectrons)
    occ = solver.occupations([eps_o], [1.0], mu)[0]
    rho_o = solver.density([pr], [Xo], [occ])

    Xd = to_gpu(X)
    ctx.chebyshev_filter(0, Xd, w.degree, a, b, a0)
    ctx.orthonormalize(0, Xd)
    eps = ctx.rayleigh_ritz(0, Xd)
    assert np.max(np.abs(eps - eps_o)) < 1e-8
    occ_g = solver.occupations([eps], [1.0], solver.fermi_level([eps], [1.0], w.nelectrons))[0]
    rho = torch.zeros(pr.quad.nq, dtype=torch.float64, device="cuda")
    ctx.density([Xd], [occ_g], rho)
    r = rho.cpu().numpy()
    wq = pr.quad.weights
    assert np.sqrt(np.sum(wq * (r - rho_o) ** 2)) / np.sqrt(np.sum(wq * rho_o ** 2)) < 1e-8
