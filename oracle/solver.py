"""Chebyshev-filtered subspace iteration and what follows it (Sec. IV; Sec. II
Eqs. rho, fd, ne and the band energy).
"""
import numpy as np
import scipy.linalg as sla

KB_HA_PER_K = 3.166811563e-6   # Boltzmann constant in Hartree / K


def chebyshev_filter(apply_A, X, m, a, b, a0):
    """Degree-m Chebyshev filter p_m(A) X (Sec. IV, the filtered vectors Y~).

    The unwanted interval [a, b] is mapped to [-1, 1] (e = (b-a)/2 and
    c = (b+a)/2); the polynomial is scaled so that its value at a0 (a point
    below the wanted spectrum) stays O(1), with the three-term recurrence of
    the scaled Chebyshev polynomials (Zhou, Saad, Tiago, Chelikowsky 2006,
    cited by the paper):

      sigma_1 = e / (a0 - c),  Y_1 = (sigma_1 / e) (A - c) X,
      sigma_{j+1} = 1 / (2 / sigma_1 - sigma_j),
      Y_{j+1} = (2 sigma_{j+1} / e) (A - c) Y_j - sigma_j sigma_{j+1} Y_{j-1}.
    """
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma = e / (a0 - c)
    sigma1 = sigma
    gamma = 2.0 / sigma1
    Xp = X
    Y = (sigma1 / e) * (apply_A(X) - c * X)
    for _ in range(2, m + 1):
        sigma2 = 1.0 / (gamma - sigma)
        Yn = (2.0 * sigma2 / e) * (apply_A(Y) - c * Y) - (sigma * sigma2) * Xp
        Xp, Y = Y, Yn
        sigma = sigma2
    return Y


def chebyshev_scalar(lam, m, a, b, a0):
    """The same recurrence on a scalar eigenvalue: the filter's gain on an eigenvector."""
    return chebyshev_filter(lambda x: lam * x, np.ones(1), m, a, b, a0)[0]


def cholqr(Y, apply_M, passes=2):
    """Orthonormalize in the M inner product: S = Y^+ M Y = L L^+, Q = Y L^{-+};
    repeated ``passes`` times (Sec. IV, orthonormalization before projection)."""
    Q = Y
    for _ in range(passes):
        S = Q.conj().T @ apply_M(Q)
        S = 0.5 * (S + S.conj().T)
        Lc = np.linalg.cholesky(S)
        Q = sla.solve_triangular(Lc.conj(), Q.T, lower=True).T
    return Q


def rayleigh_ritz(Q, apply_H, apply_M):
    """Galerkin projection onto span(Q) and the reduced generalized eigenproblem
    (Eq. ProjKS): H^Q = Q^+ H Q, M^Q = Q^+ M Q, H^Q u = eps M^Q u; returns the
    ascending Ritz values and the rotated vectors Q u."""
    Hq = Q.conj().T @ apply_H(Q)
    Mq = Q.conj().T @ apply_M(Q)
    Hq = 0.5 * (Hq + Hq.conj().T)
    Mq = 0.5 * (Mq + Mq.conj().T)
    eps, U = sla.eigh(Hq, Mq)
    return eps, Q @ U


def fermi_dirac(eps, mu, T):
    """Fractional occupancy (Eq. fd)."""
    x = (np.asarray(eps) - mu) / (KB_HA_PER_K * T)
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def fermi_level(eps_k, w_k, Ne, T=500.0, tol=1e-12):
    """mu with 2 sum_k w_k sum_a f(eps, mu) = N_e (Eq. ne), by bisection."""
    allE = np.concatenate([np.asarray(e) for e in eps_k])
    lo, hi = allE.min() - 1.0, allE.max() + 1.0

    def count(mu):
        return sum(2.0 * w * np.sum(fermi_dirac(e, mu, T)) for e, w in zip(eps_k, w_k))

    mid = 0.5 * (lo + hi)
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        n = count(mid)
        if abs(n - Ne) < tol:
            break
        if n < Ne:
            lo = mid
        else:
            hi = mid
    return mid


def occupations(eps_k, w_k, mu, T=500.0):
    """Per-vector density weights 2 w_k f(eps, mu) (Eq. rho)."""
    return [2.0 * w * fermi_dirac(e, mu, T) for e, w in zip(eps_k, w_k)]


def band_energy(eps_k, w_k, mu, T=500.0):
    """E_band = 2 sum_k w_k sum_a f(eps, mu) eps (Sec. II, band energy)."""
    return sum(2.0 * w * np.sum(fermi_dirac(e, mu, T) * e) for e, w in zip(eps_k, w_k))


def density(problems, Xs, occs):
    """rho(x_q) = sum_k sum_a occ_{k,a} |u_{a,k}(x_q)|^2 at every quadrature point (Eq. rho)."""
    pr0 = problems[0]
    rho = np.zeros(pr0.quad.nq)
    for pr, X, occ in zip(problems, Xs, occs):
        for e in pr.cells:
            s = slice(pr.quad.offset[e], pr.quad.offset[e + 1])
            U = pr.values_at_points(e, X)
            rho[s] += np.sum(np.abs(U) ** 2 * occ[None, :], axis=1)
    return rho


def band_trace_grad_V(pr, X):
    """d tr(X^+ H^O X) / d V_q = w_q sum_v |u_v(x_q)|^2 (H^O is linear in V through
    the (|k|^2/2 + V) N_m^* N_n term of Eq. HOEFEelelements)."""
    g = np.zeros(pr.quad.nq)
    for e in pr.cells:
        s = slice(pr.quad.offset[e], pr.quad.offset[e + 1])
        U = pr.values_at_points(e, X)
        g[s] = pr.quad.weights[s] * np.sum(np.abs(U) ** 2, axis=1)
    return g


def residual_norms(pr, X, eps):
    """r_a = ||H u_a - eps_a M u_a||_{M^-1} / ||u_a||_M."""
    R = pr.apply_H(X) - pr.apply_M(X) * eps[None, :]
    num = np.sqrt(np.real(np.sum(np.conj(R) * pr.apply_Minv(R), axis=0)))
    den = np.sqrt(np.real(np.sum(np.conj(X) * pr.apply_M(X), axis=0)))
    return num / den


def lanczos_upper_bound(apply_H, apply_M, apply_Minv, v0, steps):
    """Upper bound of the spectrum of M^{-1} H: largest Ritz value of a k-step
    Lanczos run in the M inner product plus the norm of the last residual."""
    v0 = np.asarray(v0).reshape(-1, 1)
    q = v0 / np.sqrt(np.real(np.vdot(v0, apply_M(v0))))
    q_prev = np.zeros_like(q)
    beta = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = apply_Minv(apply_H(q))
        alpha = np.real(np.vdot(q, apply_M(w)))
        w = w - alpha * q - beta * q_prev
        beta = np.sqrt(np.real(np.vdot(w, apply_M(w))))
        alphas.append(alpha)
        betas.append(beta)
        q_prev, q = q, w / beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    return np.max(np.linalg.eigvalsh(T)) + betas[-1]


def subspace_iteration(pr, X, m, passes, b, lock_tol=None):
    """Chebyshev-filtered subspace iteration (Sec. IV) from the block X: per pass the degree-m filter
    with a = the largest Ritz value of the previous pass (the largest eigenvalue of the first
    Rayleigh-Ritz before the first pass), a0 one below the smallest, b the given upper bound; then
    Cholesky-QR and Rayleigh-Ritz over the whole block.

    With ``lock_tol``, the Ritz vectors whose residual (``residual_norms``) is below it stay out of
    the next filter (locking: the leading converged columns keep their vectors; the filter runs on
    the rest) but take part in the orthonormalization and the projection. Reading: the locked set
    is the longest leading run of converged Ritz vectors in ascending order, so the filtered
    columns are one contiguous block.

    Returns (eps, X, residuals per pass, filtered column-degrees per pass)."""
    Q = cholqr(X, pr.apply_M)
    eps, X = rayleigh_ritz(Q, pr.apply_H, pr.apply_M)
    res_hist, work = [], []
    nlock = 0
    for _ in range(passes):
        a, a0 = float(eps[-1]), float(eps[0]) - 1.0
        Y = X.copy()
        Y[:, nlock:] = chebyshev_filter(pr.apply_A, X[:, nlock:], m, a, b, a0)
        work.append(m * (X.shape[1] - nlock))
        eps, X = rayleigh_ritz(cholqr(Y, pr.apply_M), pr.apply_H, pr.apply_M)
        r = residual_norms(pr, X, eps)
        res_hist.append(r)
        if lock_tol is not None:
            ok = r < lock_tol
            nlock = int(np.argmin(ok)) if not np.all(ok) else len(ok)
            nlock = min(nlock, X.shape[1] - 1)   # keep one column filtered: a keeps moving
    return eps, X, res_hist, work
