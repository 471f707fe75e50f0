"""Pins of the oracle against what the paper and the mathematics fix.

Each test would fail on a plausible mistake in the oracle (a dropped term, a
wrong sign or index, a transposed operand); the comment on each says which.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from cases import oracle_problem, small_case, switched_coulomb, uniform_xb
from oracle import solver
from oracle.enrichment import Enrichment, cutoff, hermite_eval
from oracle.fe1d import gauss, gll, lagrange

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- 1D rules
def test_gll_p4_textbook():
    # tests/golden/gll_p4.txt: closed-form GLL nodes/weights for p = 4
    ref = np.loadtxt(os.path.join(GOLDEN, "gll_p4.txt"))
    x, w = gll(4)
    assert np.allclose(x, ref[:, 0], atol=1e-15, rtol=0)
    assert np.allclose(w, ref[:, 1], atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_gll_exactness(p):
    x, w = gll(p)
    assert abs(w.sum() - 2.0) < 1e-14
    for deg in range(2 * p):          # exact to degree 2p - 1
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(w, x ** deg) - exact) < 1e-13
    # not exact at degree 2p (catches a wrong weight formula that is still symmetric)
    assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("n", [2, 5, 9])
def test_gauss_exactness(n):
    t, w = gauss(n)
    for deg in range(2 * n):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(w, t ** deg) - exact) < 1e-13


@pytest.mark.parametrize("p", [2, 4, 6])
def test_lagrange_partition_and_derivative(p):
    xi, _ = gll(p)
    x = np.random.default_rng(3).uniform(-1, 1, 50)
    V, D = lagrange(xi, x)
    assert np.allclose(V.sum(1), 1.0, atol=1e-13)           # partition of unity
    assert np.allclose(D.sum(1), 0.0, atol=1e-11)
    # interpolation of a degree-p polynomial is exact, so is its derivative
    f = lambda s: 0.3 * s ** p - s ** 2 + 0.5 * s + 2
    df = lambda s: 0.3 * p * s ** (p - 1) - 2 * s + 0.5
    assert np.allclose(V @ f(xi), f(x), atol=1e-12)
    assert np.allclose(D @ f(xi), df(x), atol=1e-10)
    # Kronecker property at the nodes
    Vn, _ = lagrange(xi, xi)
    assert np.allclose(Vn, np.eye(p + 1), atol=1e-14)


# ---------------------------------------------------------------- mesh, quadrature
def test_mesh_mass_and_quadrature_volume():
    w = W.config_c1()
    pr = oracle_problem(w.a, W.mesh_breakpoints(w), w.p, w.pos, w.Z, quad=(5, 5, 1))
    assert pr.mesh.nh == (8 * 4) ** 3
    assert abs(pr.m.sum() - w.a ** 3) < 1e-12 * w.a ** 3
    assert abs(pr.quad.weights.sum() - w.a ** 3) < 1e-11 * w.a ** 3
    # exact integration of a polynomial over the box: int x^2 y dV = a^6 / 6
    x = pr.quad.points
    assert abs(np.dot(pr.quad.weights, x[:, 0] ** 2 * x[:, 1]) - w.a ** 6 / 6) < 1e-10 * w.a ** 6
    # graded breakpoints include both nuclear coordinates on each axis
    for d in range(3):
        assert np.any(np.abs(pr.mesh.xb[d] - w.a / 4) < 1e-12)
        assert np.all(np.diff(pr.mesh.xb[d]) > 0)


def test_octree_leaves_count():
    # a nucleus at a vertex touches 8 cells; each gets 7 (depth-1) + 8 leaves at depth 2 -> 15 leaves
    a = 4.0
    pr = oracle_problem(a, uniform_xb(a, 2), 2, [[0, 0, 0]], [1], quad=(3, 3, 2), r0=1.0, rc=1.5)
    counts = np.diff(pr.quad.offset) // 27
    assert sorted(set(counts.tolist())) == [15]
    assert abs(pr.quad.weights.sum() - a ** 3) < 1e-12


# ---------------------------------------------------------------- enrichment inputs and functions
@pytest.mark.parametrize("nl", [(1, 0), (2, 0), (2, 1)])
def test_hydrogenic_radial_normalized(nl):
    # the synthetic atomic orbitals are normalized bound states: int R^2 r^2 dr = 1
    from scipy.integrate import quad
    for Z in (1, 6, 14):
        f = lambda r: W.hydrogenic_radial(nl[0], nl[1], Z, r)[0] ** 2 * r * r
        assert abs(quad(f, 0, 60 / Z, limit=200)[0] - 1) < 1e-10


def test_hermite_table_accuracy():
    Z = 14
    R, dR = W.radial_tables([Z], rc=4.0, ngrid=2000)
    r = np.random.default_rng(1).uniform(0, 3.999, 2000)
    for j, (n, l, _) in enumerate(W.ORBITALS_1S_2P[:3]):
        v, d = hermite_eval(R[0, j], dR[0, j], 4.0, r)
        ex, dex = W.hydrogenic_radial(n, l, Z, r)
        scale = np.max(np.abs(R[0, j]))
        # cubic Hermite error bound h^4 max|f''''| / 384, with |f''''| <= Z^4 max|f| here
        dr = 4.0 / 1999
        assert np.max(np.abs(v - ex)) < dr ** 4 / 384 * Z ** 4 * scale
        assert np.max(np.abs(v - ex)) > 0.0
        assert np.max(np.abs(d - dex)) < dr ** 3 / 24 * Z ** 4 * scale


def test_cutoff_properties():
    r = np.linspace(0, 5, 5001)
    h, dh = cutoff(r, 3.0, 4.0)
    assert np.all(h[r <= 3.0] == 1.0) and np.all(h[r >= 4.0] == 0.0)
    assert np.all(np.diff(h) <= 1e-15)                     # monotone
    mid = (r > 3.01) & (r < 3.99)
    fd = (cutoff(r + 1e-6, 3.0, 4.0)[0] - cutoff(r - 1e-6, 3.0, 4.0)[0]) / 2e-6
    assert np.allclose(dh[mid], fd[mid], atol=1e-7)


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.45)])
def test_enrichment_gradient_fd(k):
    # product rule, phase sign and the -ik term of the Bloch gradient
    a = 7.0
    R, dR = W.radial_tables([6, 14], rc=4.0)
    enr = Enrichment(a, [[0.5, 0.5, 0.5], [3.5, 3.5, 3.6]], W.orbital_lm_codes(), R, dR, 3.0, 4.0)
    x = np.random.default_rng(2).uniform(0, a, (40, 3))
    hstep = 1e-6
    for nu in range(enr.nO):
        v, g = enr.values(nu, x, np.array(k))
        for d in range(3):
            e = np.zeros(3)
            e[d] = hstep
            fd = (enr.values(nu, x + e, np.array(k))[0] - enr.values(nu, x - e, np.array(k))[0]) / (2 * hstep)
            assert np.allclose(g[:, d], fd, atol=2e-5 * max(1.0, np.max(np.abs(g))))


def test_enrichment_periodic_and_bloch():
    # N^A(x + a n) = N^A(x): the phase uses x - R_I^x, not x (Eq. UOEFEAtomic)
    a = 7.0
    R, dR = W.radial_tables([6], rc=3.0)
    enr = Enrichment(a, [[1.0, 2.0, 3.0]], W.orbital_lm_codes(), R, dR, 2.0, 3.0)
    x = np.random.default_rng(4).uniform(0, a, (30, 3))
    k = np.array([0.2, 0.1, -0.3])
    for nu in range(enr.nO):
        v1, _ = enr.values(nu, x, k)
        v2, _ = enr.values(nu, x + a * np.array([1, -1, 2]), k)
        assert np.allclose(v1, v2, atol=1e-13)


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_orthogonalized_overlap_block_diagonal(k):
    # T^+ M^EFE T with T = [[I, -C^T],[0, I]] is block-diagonal and its OO block is M^oo
    # (Eqs. orthC, MOEFE, Moo): fails if c is transposed, conjugated wrongly or mis-scaled.
    pr, _ = small_case(k=k)
    Me = pr.efe_overlap_dense()
    T = np.eye(pr.n, dtype=pr.dtype)
    T[:pr.nh, pr.nh:] = -pr.c.T
    MO = T.conj().T @ Me @ T
    scale = np.max(np.abs(Me))
    assert np.max(np.abs(MO[:pr.nh, pr.nh:])) < 1e-13 * scale
    assert np.allclose(MO[pr.nh:, pr.nh:], pr.Moo, atol=1e-13 * scale)
    assert np.allclose(np.diag(MO[:pr.nh, :pr.nh]), pr.m, rtol=1e-14)
    sla.cholesky(pr.Moo, lower=True)                       # Hermitian positive definite


def test_orthogonalization_locality():
    # c_{nu,l} = 0 on nodes whose CFE support does not meet the enrichment ball (Sec. III A)
    pr, _ = small_case()
    X = pr.mesh.node_coords()
    for nu in range(pr.nO):
        R = pr.enr.pos[pr.enr.atom_of(nu)]
        d = X - R
        d -= pr.mesh.a * np.round(d / pr.mesh.a)
        far = np.sqrt((d ** 2).sum(1)) > pr.enr.rc + 2 * np.sqrt(3) * pr.mesh.a / pr.mesh.nc[0]
        assert np.all(pr.c[nu, far] == 0)
        assert np.any(pr.c[nu] != 0)


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_hamiltonian_hermitian(k):
    pr, _ = small_case(k=k)
    H = pr.assemble_H().toarray()
    assert np.max(np.abs(H - H.conj().T)) <= 1e-13 * np.max(np.abs(H))


def test_constant_potential_constant_function():
    # k = 0, V = const: M^{-1} H^O [1; 0] = V [1; 0] (kinetic of a constant vanishes,
    # Gauss row sums equal GLL lumped weights, partition of unity kills the
    # enrichment rows through T^+). Exercises c, T, Moo and the quadrature together.
    pr, _ = small_case()
    pr.build(np.full(pr.quad.nq, -0.7))
    one = np.zeros((pr.n, 1))
    one[:pr.nh] = 1.0
    Y = pr.apply_A(one)
    assert np.allclose(Y[:pr.nh], -0.7, atol=1e-12)
    assert np.max(np.abs(Y[pr.nh:])) < 1e-11
    pr.build(np.zeros(pr.quad.nq))
    assert np.max(np.abs(pr.apply_H(one))) < 1e-12


def test_free_electron_spectrum():
    # V = 0, no enrichment: the lowest eigenvalues approach |k + G|^2 / 2 and the
    # error falls roughly like h^(2p) under refinement (Sec. V B rate of convergence).
    a = 8.5
    k = np.array([0.25, 0.25, 0.0]) * 2 * np.pi / a
    G = 2 * np.pi / a * np.array([[i, j, l] for i in range(-2, 3) for j in range(-2, 3) for l in range(-2, 3)])
    exact = np.sort(0.5 * np.sum((k + G) ** 2, 1))[:6]
    errs = []
    for n in (2, 3):
        pr = oracle_problem(a, uniform_xb(a, n), 3, np.zeros((0, 3)), [], k=k, enrich=False)
        pr.build(np.zeros(pr.quad.nq))
        H = pr.assemble_H().toarray()
        ev = sla.eigh(H, np.diag(pr.m), eigvals_only=True)[:6]
        errs.append(np.max(np.abs(ev - exact)))
    assert errs[1] < 2e-3
    assert errs[0] / errs[1] > (3 / 2) ** 4                # at least 4th order (p = 3 -> 2p = 6)


def test_hydrogenic_levels():
    # single bare nucleus, enrichment = its own 1s/2s/2p: eigenvalues -Z^2/(2 n^2).
    # The remaining error is the quadrature of the -Z/r singularity times the cusp
    # (falls with octree depth) and the CFE basis for the cut-off tails.
    a, Z = 10.26, 6
    pos = np.array([[0.0, 0.0, 0.0]])
    pr = oracle_problem(a, uniform_xb(a, 4), 4, pos, [Z], quad=(5, 8, 8), r0=3.5, rc=4.5)
    V = switched_coulomb(pr.quad.points, a, pos[0], Z)
    pr.build(V)
    H = pr.assemble_H().toarray()
    ev = sla.eigh(H, pr.dense_M(), eigvals_only=True)[:5]
    exact = np.array([-Z ** 2 / 2] + [-Z ** 2 / 8] * 4)
    assert abs(ev[0] - exact[0]) < 1.5e-4          # 1s: -18 Ha
    assert abs(ev[1] - exact[1]) < 2e-5            # 2s: -4.5 Ha
    assert np.max(np.abs(ev[2:] - exact[2:])) < 5e-6
    assert np.ptp(ev[2:]) < 1e-9                   # 2p triplet stays degenerate


# ---------------------------------------------------------------- filter, QR, RR
def test_chebyshev_closed_form():
    # scaled recurrence = T_m((lam - c)/e) / T_m((a0 - c)/e)
    from numpy.polynomial import chebyshev as C
    a_, b_, a0 = -1.0, 30.0, -20.0
    e, c = (b_ - a_) / 2, (b_ + a_) / 2
    for m in (1, 2, 5, 20):
        cm = np.zeros(m + 1)
        cm[m] = 1
        for lam in (-19.0, -5.0, 0.0, 7.5, 29.0):
            ref = C.chebval((lam - c) / e, cm) / C.chebval((a0 - c) / e, cm)
            assert abs(solver.chebyshev_scalar(lam, m, a_, b_, a0) - ref) < 1e-12 * max(1, abs(ref))


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_filter_on_eigenvector(k):
    # on an exact eigenvector of M^{-1}H the filter multiplies by the scalar gain
    pr, _ = small_case(k=k, n=1, p=3)
    H = pr.assemble_H().toarray()
    ev, U = sla.eigh(H, pr.dense_M())
    a_, b_, a0 = ev[4], ev[-1] + 1, ev[0] - 1
    for j in (0, 2, 10):
        Y = solver.chebyshev_filter(pr.apply_A, U[:, [j]], 8, a_, b_, a0)
        g = solver.chebyshev_scalar(ev[j], 8, a_, b_, a0)
        assert np.allclose(Y[:, 0], g * U[:, j], atol=1e-9 * max(1, abs(g)) * np.max(np.abs(U[:, j])))


def test_cholqr_and_rr_converge():
    pr, _ = small_case(k=(0.1, 0.2, -0.3), n=2, p=2)
    H = pr.assemble_H().toarray()
    Md = pr.dense_M()
    ev = sla.eigh(H, Md, eigvals_only=True)
    nv = 8
    X = W.random_vectors(pr.n, nv, complex_=True, seed=0)
    b_ = ev[-1] * 1.01
    for it in range(60):
        a_ = ev[0] - 1 if it == 0 else eps[-1]
        a0 = ev[0] - 1 if it == 0 else eps[0]
        Y = solver.chebyshev_filter(pr.apply_A, X, 10, a_, b_, a0)
        Q = solver.cholqr(Y, pr.apply_M)
        G = Q.conj().T @ pr.apply_M(Q)
        assert np.allclose(G, np.eye(nv), atol=1e-12)
        eps, X = solver.rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
    assert np.max(np.abs(eps[:nv - 2] - ev[:nv - 2])) < 1e-10
    res = solver.residual_norms(pr, X, eps)
    assert np.all(res[:nv - 2] < 1e-8)


def test_cholqr_span():
    # span invariance: the M-orthogonal projector equals the one from Householder QR of M^{1/2} Y
    pr, _ = small_case(n=1, p=3)
    Y = W.random_vectors(pr.n, 6, seed=5)
    Q = solver.cholqr(Y, pr.apply_M)
    Md = pr.dense_M()
    Ms = sla.sqrtm(Md).real
    Qh, _ = np.linalg.qr(Ms @ Y)
    P1 = Ms @ Q @ Q.T @ Ms
    P2 = Qh @ Qh.T
    assert np.allclose(P1, P2, atol=1e-10)


# ---------------------------------------------------------------- occupations, density, adjoint
def test_fermi_level_and_band_energy():
    eps = [np.array([-3.0, -1.0, 0.5, 2.0]), np.array([-2.5, -0.9, 0.6, 1.9])]
    w = [0.5, 0.5]
    mu = solver.fermi_level(eps, w, 4.0, T=500.0)
    occ = solver.occupations(eps, w, mu)
    assert abs(sum(o.sum() for o in occ) - 4.0) < 1e-10
    assert -0.9 < mu < 0.5
    Eb = solver.band_energy(eps, w, mu)
    assert abs(Eb - (2 * 0.5 * (-3 - 1) + 2 * 0.5 * (-2.5 - 0.9))) < 1e-8   # T=500 K: sharp


def test_density_of_basis_vectors():
    # u = N^C (x^c - Gamma x^o) + N^A x^o: the constant vector gives u = 1, a unit
    # enrichment coefficient gives N^O_nu = N^A_nu - sum_l c_{nu,l} N^C_l (Eq. UOEFESplit)
    pr, _ = small_case(k=(0.2, 0.0, 0.1))
    one = np.zeros((pr.n, 1))
    one[:pr.nh] = 1.0
    rho = solver.density([pr], [one], [np.ones(1)])
    assert np.allclose(rho, 1.0, atol=1e-12)
    nu = 3
    X = np.zeros((pr.n, 1), complex)
    X[pr.nh + nu] = 1.0
    e = int(np.argmax([len(a) for a in pr.actA]))
    x, _ = pr.quad.cell(e)
    NA, _ = pr.enr.values(nu, x, pr.k)
    NB = pr.phiC[e] @ pr.c[nu, pr.mesh.cell_nodes(e)]
    U = pr.values_at_points(e, X)[:, 0]
    assert np.allclose(U, NA - NB, atol=1e-13)


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_adjoint_fd(k):
    # d tr(X^+ H X)/dV_q against central differences (H is affine in V: FD is exact up to rounding)
    pr, V = small_case(k=k)
    X = W.random_vectors(pr.n, 3, complex_=pr.complex, seed=7)
    g = solver.band_trace_grad_V(pr, X)
    rng = np.random.default_rng(0)
    for q in rng.choice(pr.quad.nq, 6, replace=False):
        h = 1e-4
        Vp, Vm = V.copy(), V.copy()
        Vp[q] += h
        Vm[q] -= h
        pr.build(Vp)
        tp = np.real(np.sum(np.conj(X) * pr.apply_H(X)))
        pr.build(Vm)
        tm = np.real(np.sum(np.conj(X) * pr.apply_H(X)))
        assert abs((tp - tm) / (2 * h) - g[q]) < 1e-7 * max(1.0, abs(g[q]))
    pr.build(V)


def test_density_integral_and_trace_identity():
    # sum_q w_q rho_q = sum_v occ_v ||u_v||^2_L2 (the adjoint's trace identity), and for
    # M-normalized low eigenvectors ||u||_L2 = 1 up to the GLL mass lumping (Eq. orthCGLL).
    pr, _ = small_case(n=2, p=3)
    ev, U = sla.eigh(pr.assemble_H().toarray(), pr.dense_M())
    Q = U[:, :4]
    occ = np.array([2.0, 2.0, 1.0, 0.5])
    rho = solver.density([pr], [Q], [occ])
    tot = np.dot(pr.quad.weights, rho)
    assert abs(tot - occ.sum()) < 0.02 * occ.sum()
    g = solver.band_trace_grad_V(pr, Q * np.sqrt(occ)[None, :])
    assert abs(g.sum() - tot) < 1e-12 * tot


def test_lanczos_upper_bound():
    pr, _ = small_case(n=1, p=3)
    ev = sla.eigh(pr.assemble_H().toarray(), pr.dense_M(), eigvals_only=True)
    v0 = W.random_vectors(pr.n, 1, seed=3)[:, 0]
    b = solver.lanczos_upper_bound(pr.apply_H, pr.apply_M, pr.apply_Minv, v0, 30)
    assert b >= ev[-1] - 1e-8
    assert b < ev[-1] * 1.2


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_residual_norms_closed_form(k):
    # residual of a mixture of two exact eigenvectors (Sec. IV, Eq. ProjKS; the residual norm
    # ||H u - eps M u||_{M^-1} / ||u||_M). With M-orthonormal eigenpairs (eps_i, u_i), (eps_j, u_j) of H u = eps M u and
    # u = s (u_i + d u_j):
    #   H u - t M u = s M [(eps_i - t) u_i + d (eps_j - t) u_j],
    #   ||.||_{M^-1}^2 = s^2 [(eps_i - t)^2 + d^2 (eps_j - t)^2],  ||u||_M^2 = s^2 (1 + d^2),
    # and at the Rayleigh quotient t = (eps_i + d^2 eps_j) / (1 + d^2) the ratio is
    # |d| |eps_i - eps_j| / (1 + d^2). The lumped-plus-enrichment mass is far from a multiple of I,
    # so the 2-norm, or M in place of M^-1, gives other numbers; the scale s = 3.7 catches a dropped
    # denominator.
    pr, _ = small_case(k=k, n=1, p=3)
    H = pr.assemble_H().toarray()
    Md = pr.dense_M()
    md = np.real(np.diag(Md))[: pr.nh]
    assert md.max() / md.min() > 3.0          # the pin needs a non-uniform mass
    ev, U = sla.eigh(H, Md)
    pairs = [(0, 3, 0.5), (2, 7, -0.2), (5, 1, 1.3), (9, 4, 0.05)]
    s = 3.7
    X = np.stack([s * (U[:, i] + d * U[:, j]) for i, j, d in pairs], axis=1)
    rq = np.array([(ev[i] + d * d * ev[j]) / (1 + d * d) for i, j, d in pairs])
    expect = np.array([abs(d) * abs(ev[i] - ev[j]) / (1 + d * d) for i, j, d in pairs])
    got = solver.residual_norms(pr, X, rq)
    assert np.allclose(got, expect, rtol=1e-9, atol=1e-12)
    # any other shift t: the general form above
    t = rq + np.array([0.3, -1.1, 0.7, 2.0])
    expect_t = np.array([math.sqrt(((ev[i] - tt) ** 2 + d * d * (ev[j] - tt) ** 2) / (1 + d * d))
                         for (i, j, d), tt in zip(pairs, t)])
    assert np.allclose(solver.residual_norms(pr, X, t), expect_t, rtol=1e-9, atol=1e-12)
    # an exact eigenvector at its eigenvalue has no residual
    assert np.max(solver.residual_norms(pr, s * U[:, :6], ev[:6])) < 1e-9 * np.max(np.abs(ev[:6]))


def test_subspace_iteration_with_locking_matches_dense_eigensolve():
    # the filtered subspace iteration (Sec. IV) converges to the lowest eigenpairs of the dense
    # generalized problem; locking the leading converged Ritz vectors (residual below 1e-9) keeps
    # that accuracy while filtering far fewer columns
    pr, _ = small_case(p=3)
    ev = sla.eigh(pr.assemble_H().toarray(), pr.dense_M(), eigvals_only=True)
    X0 = W.random_vectors(pr.n, 12, seed=3)
    b = ev[-1] * 1.01
    eps, _, res, work = solver.subspace_iteration(pr, X0, 12, 40, b)
    assert np.max(np.abs(eps[:8] - ev[:8])) < 1e-10 and np.max(res[-1][:8]) < 1e-12
    eps_l, _, res_l, work_l = solver.subspace_iteration(pr, X0, 12, 40, b, lock_tol=1e-9)
    assert np.max(np.abs(eps_l[:8] - ev[:8])) < 1e-10 and np.max(res_l[-1][:8]) < 1e-8
    assert sum(work_l) < 0.5 * sum(work)
