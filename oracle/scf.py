"""The self-consistent field iteration around the hot path (Sec. II: the Kohn-Sham equations with
V_eff = V_xc + phi_tot, the density of Eq. rho, the total energy E_tot; Sec. IV: the fixed-point
iteration rho_in -> V_eff -> eigenstates -> rho_out, mixed until the density stops changing).
TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings:
* phi_tot = phi_aux + sum_I (V_N,I - V_N,I^smear) (Eq. eqnpoissontotsmear), phi_aux from the
  periodic Poisson solve of ``electrostatics`` with the smeared nuclei and the input density.
* The eigenstates of each pass are the lowest ``nstates`` of the generalized problem
  H^O u = eps M^O u, taken exactly (sparse shift-invert Lanczos) rather than by the filter: the
  oracle of the driver checks the physics of the loop, the filter has its own oracle.
* E_tot is evaluated with the input density of the pass (the density the potentials come from),
  E_tot = E_band + E_xc[rho] + E_elec[rho] - int rho V_xc - int rho phi_tot; at self-consistency it
  is the Kohn-Sham total energy.
* The first input density is the neutralizing smeared charge sum_I Z_I g(|x - R_I|).
* With ``degree`` set, the eigenstates of every pass but the first come from the paper's
  Chebyshev-filtered subspace iteration instead (Sec. IV): one filter pass of that degree on the
  previous pass's states, with a = the largest previous Ritz value, a0 one below the smallest and b
  a Lanczos upper bound of the new operator, then Cholesky-QR and Rayleigh-Ritz. The first pass
  takes exact eigenstates (an initial subspace).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import electrostatics as es
from . import solver, xc
from .operators import Problem


class SCF:
    def __init__(self, mesh, quad, enr, pos, Z, nstates, ks=((0.0, 0.0, 0.0),), w_k=None, T=500.0,
                 degree=None):
        self.mesh, self.quad = mesh, quad
        self.pos = np.asarray(pos, float).reshape(-1, 3)
        self.Z = np.asarray(Z, float)
        self.a = mesh.a
        self.nstates, self.T = int(nstates), float(T)
        self.problems = [Problem(mesh, quad, enr, k) for k in ks]
        self.w_k = np.full(len(ks), 1.0 / len(ks)) if w_k is None else np.asarray(w_k, float)
        self.nelec = float(np.sum(self.Z))
        self.rc = es.cutoff_radii(self.pos, self.a)
        x = quad.points
        self.b = es.smeared_nuclear_charge(x, self.pos, self.Z, self.rc, self.a)
        self.corr = es.nuclear_correction(x, self.pos, self.Z, self.rc, self.a)
        self.A, self.tabs = es.poisson_matrices(mesh, quad)
        self.lu = es.poisson_factor(self.A)
        self.prev = {}
        self.degree = degree

    def initial_density(self):
        return -self.b

    def potentials(self, rho):
        """phi_aux, phi_tot, eps_xc, V_xc at the points, from the density rho."""
        nodal = es.solve_poisson(self.mesh, self.quad, self.b + rho, self.A, self.tabs, self.lu)
        phi_aux = es.field_at_points(self.mesh, self.quad, nodal, self.tabs)
        exc, vxc = xc.lda(rho)
        return phi_aux, phi_aux + self.corr, exc, vxc

    def filtered(self, pr, V):
        """One pass of the Chebyshev-filtered subspace iteration from the previous pass's states."""
        pr.build(V)
        eps0, X0 = self.prev[id(pr)][:2]
        b = solver.lanczos_upper_bound(pr.apply_H, pr.apply_M, pr.apply_Minv, X0[:, -1], 20)
        Y = solver.chebyshev_filter(pr.apply_A, X0, self.degree, float(eps0[-1]), b, float(eps0[0]) - 1.0)
        vals, vecs = solver.rayleigh_ritz(solver.cholqr(Y, pr.apply_M), pr.apply_H, pr.apply_M)
        self.prev[id(pr)] = (vals, vecs) + tuple(self.prev[id(pr)][2:])
        return vals, vecs

    def eigenstates(self, pr, V):
        if self.degree is not None and id(pr) in self.prev:
            return self.filtered(pr, V)
        pr.build(V)
        H = pr.assemble_H().tocsc()
        M = sp.block_diag((sp.diags(pr.m), sp.csr_matrix(pr.Moo))).tocsc()
        prev = self.prev.get(id(pr))
        if prev is not None:
            # the previous pass's levels as the start and the factor of its shifted operator as the
            # preconditioner: block LOBPCG converges in a few sweeps while the potential settles
            vals0, vecs0, lu = prev
            P = spla.LinearOperator(H.shape, matvec=lu.solve, dtype=float)
            vals, vecs, hist = spla.lobpcg(H, vecs0, B=M, M=P, largest=False, tol=1e-10, maxiter=200,
                                           retResidualNormsHistory=True)
            res = hist[-1] if len(hist) else np.inf
            if np.all(np.asarray(res) < 1e-8):
                order = np.argsort(vals)
                vals, vecs = vals[order], vecs[:, order]
                self.prev[id(pr)] = (vals, vecs, lu)
                return vals, vecs
        # shift-and-invert Lanczos below the 1s level of the bare largest nucleus, -Z^2/2, under which
        # no Kohn-Sham level lies (the electrons' Hartree potential is positive and the LDA
        # exchange-correlation potential is far smaller)
        sigma = -float(np.max(self.Z)) ** 2 - 1.0
        lu = spla.splu((H - sigma * M).tocsc())
        OP = spla.LinearOperator(H.shape, matvec=lu.solve, dtype=float)
        vals, vecs = spla.eigsh(H, k=self.nstates, M=M, sigma=sigma, which="LM", OPinv=OP,
                                ncv=max(2 * self.nstates + 1, 20), tol=1e-12)
        order = np.argsort(vals)
        vals, vecs = vals[order], vecs[:, order]
        self.prev[id(pr)] = (vals, vecs, lu)
        return vals, vecs

    def step(self, rho_in):
        """One pass: (rho_out, E_tot, eigenvalues per k, mu)."""
        phi_aux, phi_tot, exc, vxc = self.potentials(rho_in)
        V = vxc + phi_tot
        eps, Xs = [], []
        for pr in self.problems:
            e, X = self.eigenstates(pr, V)
            eps.append(e)
            Xs.append(X)
        mu = solver.fermi_level(eps, self.w_k, self.nelec, self.T)
        occ = solver.occupations(eps, self.w_k, mu, self.T)
        rho_out = solver.density(self.problems, Xs, occ)
        w = self.quad.weights
        e_band = solver.band_energy(eps, self.w_k, mu, self.T)
        e_xc = float(np.sum(w * rho_in * exc))
        e_elec = es.electrostatic_energy(self.quad, self.pos, self.Z, self.rc, self.a, rho_in, self.b, phi_aux)
        e_tot = e_band + e_xc + e_elec - float(np.sum(w * rho_in * vxc)) - float(np.sum(w * rho_in * phi_tot))
        return rho_out, e_tot, eps, mu

    def run(self, mixer, maxit=40, tol=1e-6, rho0=None):
        """Mixed passes until || rho_out - rho_in ||_L2 < tol; returns (rho, E_tot history, residual
        history, eigenvalues of the last pass)."""
        rho = self.initial_density() if rho0 is None else rho0
        w = self.quad.weights
        etot, res = [], []
        eps = None
        for _ in range(maxit):
            rho_out, e, eps, _ = self.step(rho)
            etot.append(e)
            res.append(float(np.sqrt(np.sum(w * (rho_out - rho) ** 2))))
            if res[-1] < tol:
                break
            rho = mixer(rho, rho_out)
        return rho, etot, res, eps
