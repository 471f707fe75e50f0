"""Discrete OEFE operators (Sec. III A, Eqs. orthC, orthCGLL, KSEigGenDiscrete,
HOEFEelelements, MOEFE, Moo, KSEignStandDiscrete, MOEFEInv).

Notation. Cell e has n_loc = (p+1)^3 CFE functions N^C_a and the enrichment
functions act(e) (see ``enrichment.active_sets``). On the cell's point set
(``quadrature``) the EFE cell matrix is

  H_e[m, n] = sum_q w_q [ 1/2 grad phi_m^* . grad phi_n
                          - (i/2) (phi_m^* k.grad phi_n - (k.grad phi_m)^* phi_n)
                          + (|k|^2/2 + V_q) phi_m^* phi_n ]          (Eq. HOEFEelelements)

for phi = [N^C_a ; N^A_nu]. Reading: the paper's k-term -i k.(phi_m^* grad phi_n)
is written in its Hermitian form; the two agree after integration by parts on
the periodic cell and the Hermitian form keeps every cell matrix Hermitian under
inexact quadrature.

Orthogonalization (Eq. orthCGLL): c_{nu,l} = [int N^A_nu N^C_l] / m_l, numerator
on the cell point sets, denominator the GLL-lumped mass. With
T = [[I, -C^T], [0, I]] mapping OEFE coefficients to the non-orthogonal
{N^C, N^A} basis (Eq. UOEFESplit, UOEFEOrtho), the OEFE matrices are
H^O = T^+ H^EFE T and M^O = T^+ M^EFE T with the lumped CC block, which gives
the block-diagonal M^O = diag(m) (+) M^oo with
M^oo = M^AA - C diag(m) C^+ (Eqs. MOEFE, Moo). Reading: M^oo is the Galerkin
projection through T; quadrature of int N^O N^O directly would leave a
non-zero C-O block under lumping.

Because T restricted to a cell only involves that cell's nodes and act(e), the
cell matrices H^O_e = T_e^+ H_e T_e assemble to H^O exactly.
"""
import numpy as np
import scipy.sparse as sp

from .enrichment import active_sets
from .fe1d import lagrange


def cfe_basis(mesh, quad, e):
    """CFE values (nq, n_loc) and gradients (3, nq, n_loc) at the cell's points."""
    lo, hi = mesh.cell_box(e)
    h = hi - lo
    ref = quad.reference_coords(e)
    V, D = [], []
    for d in range(3):
        v, dv = lagrange(mesh.xi, ref[:, d])
        V.append(v)
        D.append(dv * (2.0 / h[d]))
    P = mesh.P

    def kron(a, b, c):  # index i + P (j + P k) with a over i (x), b over j, c over k
        return (c[:, :, None, None] * b[:, None, :, None] * a[:, None, None, :]).reshape(len(a), P ** 3)

    phi = kron(V[0], V[1], V[2])
    grad = np.stack([kron(D[0], V[1], V[2]), kron(V[0], D[1], V[2]), kron(V[0], V[1], D[2])])
    return phi, grad


class Problem:
    """Everything the method fixes for one geometry and one k-point.

    ``cells`` restricts the operator to a block of cells (a bounded sample of
    a large workload): the cell matrices of those cells are built with the
    exact orthogonalizing coefficients (tabulating the neighbouring cells as
    well), vectors hold only the rows those cells touch (CFE rows first, in
    global order), and M^oo is the enrichment overlap of the tabulated cells.
    """

    def __init__(self, mesh, quad, enr, k=(0.0, 0.0, 0.0), cells=None):
        self.mesh, self.quad, self.enr = mesh, quad, enr
        self.k = np.asarray(k, float)
        self.complex = bool(np.any(self.k))
        self.dtype = complex if self.complex else float
        self.m = mesh.lumped_mass()
        self.actA, self.act = active_sets(mesh, enr)
        self.nh, self.nO = mesh.nh, enr.nO
        self.nh_full = mesh.nh
        if cells is None:
            self.cells = list(range(mesh.ncells))
            self.tab_cells = self.cells
        else:
            self.cells = sorted(set(int(e) for e in cells))
            self.tab_cells = sorted({f for e in self.cells for f in mesh.neighbours(e)})
        self.rows = None
        self._basis()
        self._orthogonalize()
        if cells is not None:
            g = np.unique(np.concatenate([self._gindex(e) for e in self.cells]))
            self.rows = g
            nh_loc = int(np.sum(g < self.nh_full))
            sub = g[nh_loc:] - self.nh_full
            self.m = self.m[g[:nh_loc]]
            self.Moo = self.Moo[np.ix_(sub, sub)]
            self.nh, self.nO = nh_loc, len(sub)
        self.n = self.nh + self.nO

    # -- cell-level tabulation -------------------------------------------------
    def _basis(self):
        self.phiC, self.gradC, self.phiA, self.gradA = {}, {}, {}, {}
        for e in self.tab_cells:
            phi, grad = cfe_basis(self.mesh, self.quad, e)
            x, _ = self.quad.cell(e)
            na = len(self.act[e])
            pa = np.zeros((len(x), na), self.dtype)
            ga = np.zeros((3, len(x), na), self.dtype)
            for j, nu in enumerate(self.act[e]):
                v, g = self.enr.values(nu, x, self.k)
                pa[:, j] = v
                ga[:, :, j] = g.T
            self.phiC[e] = phi
            self.gradC[e] = grad
            self.phiA[e] = pa
            self.gradA[e] = ga

    def _orthogonalize(self):
        """c (Eq. orthCGLL) and M^oo (Eq. Moo). On a block of cells only the columns of c of the
        tabulated cells' nodes can be nonzero; c then holds those columns (``c_cols`` maps a global
        node to its column), the full mesh keeps every column."""
        if self.tab_cells is self.cells:
            cols_nodes = None
            m = self.m
            ncol = self.nh
        else:
            cols_nodes = np.unique(np.concatenate([self.mesh.cell_nodes(e) for e in self.tab_cells]))
            self.c_cols = np.full(self.nh, -1, dtype=np.int64)
            self.c_cols[cols_nodes] = np.arange(len(cols_nodes))
            m = self.m[cols_nodes]
            ncol = len(cols_nodes)
        c = np.zeros((self.nO, ncol), self.dtype)
        MAA = np.zeros((self.nO, self.nO), self.dtype)
        for e in self.tab_cells:
            _, w = self.quad.cell(e)
            nodes, act = self._ccols(self.mesh.cell_nodes(e)), self.act[e]
            d = self.phiC[e].T @ (w[:, None] * self.phiA[e])          # int N^C_l N^A_nu
            np.add.at(c, (act[None, :], nodes[:, None]), d)
            MAA[np.ix_(act, act)] += self.phiA[e].conj().T @ (w[:, None] * self.phiA[e])
        c /= m[None, :]
        self.c = c
        self.MAA = MAA
        self.Moo = MAA - (c.conj() * m[None, :]) @ c.T
        self.Moo = 0.5 * (self.Moo + self.Moo.conj().T)

    def _ccols(self, nodes):
        """Columns of c of global nodes."""
        return nodes if getattr(self, "c_cols", None) is None else self.c_cols[nodes]

    def gamma(self, e):
        """Gamma_e = C^T restricted to (nodes(e), act(e)), shape (n_loc, n_a)."""
        return self.c[np.ix_(self.act[e], self._ccols(self.mesh.cell_nodes(e)))].T

    def _gindex(self, e):
        return np.concatenate([self.mesh.cell_nodes(e), self.nh_full + self.act[e]])

    def index(self, e):
        """Rows of the OEFE vector touched by cell e: its nodes, then nh + act(e)."""
        g = self._gindex(e)
        return g if self.rows is None else np.searchsorted(self.rows, g)

    # -- cell Hamiltonians -----------------------------------------------------
    def efe_cell(self, e, V_e):
        """EFE cell matrix H_e (Eq. HOEFEelelements, Hermitian k-term reading)."""
        _, w = self.quad.cell(e)
        phi = np.concatenate([self.phiC[e], self.phiA[e]], axis=1)
        grad = np.concatenate([self.gradC[e], self.gradA[e]], axis=2)
        H = 0.5 * sum(grad[d].conj().T @ (w[:, None] * grad[d]) for d in range(3))
        H = H + phi.conj().T @ ((w * (V_e + 0.5 * self.k @ self.k))[:, None] * phi)
        if self.complex:
            kg = np.tensordot(self.k, grad, axes=(0, 0))
            A = phi.conj().T @ (w[:, None] * kg)
            H = H - 0.5j * (A - A.conj().T)
        return H

    def oefe_cell(self, e, V_e):
        """H^O_e = T_e^+ H_e T_e, rows/cols ordered as ``index(e)``."""
        H = self.efe_cell(e, V_e)
        nl = self.mesh.nloc
        na = len(self.act[e])
        T = np.eye(nl + na, dtype=self.dtype)
        T[:nl, nl:] = -self.gamma(e)
        return T.conj().T @ H @ T

    def build(self, V):
        """Cell matrices H^O_e for all cells from V at every quadrature point."""
        self.HO = {}
        for e in self.cells:
            s = slice(self.quad.offset[e], self.quad.offset[e + 1])
            self.HO[e] = self.oefe_cell(e, V[s])
        return self.HO

    # -- global operators ------------------------------------------------------
    def apply_H(self, X):
        """Y = H^O X by cell-wise gather / multiply / scatter-add."""
        Y = np.zeros(X.shape, np.result_type(X.dtype, self.dtype))
        for e in self.cells:
            idx = self.index(e)
            np.add.at(Y, idx, self.HO[e] @ X[idx])
        return Y

    def apply_M(self, X):
        Y = np.empty(X.shape, np.result_type(X.dtype, self.dtype))
        Y[:self.nh] = self.m[:, None] * X[:self.nh]
        Y[self.nh:] = self.Moo @ X[self.nh:]
        return Y

    def apply_Minv(self, Y):
        """(M^O)^{-1} Y: diagonal CFE block, dense solve for the enrichment block (Eq. MOEFEInv)."""
        import scipy.linalg as sla
        Z = np.empty(Y.shape, np.result_type(Y.dtype, self.dtype))
        Z[:self.nh] = Y[:self.nh] / self.m[:, None]
        Z[self.nh:] = sla.cho_solve(sla.cho_factor(self.Moo, lower=True), Y[self.nh:])
        return Z

    def apply_A(self, X):
        """A = (M^O)^{-1} H^O (Eq. KSEignStandDiscrete)."""
        return self.apply_Minv(self.apply_H(X))

    def assemble_H(self):
        """Sparse global H^O (small meshes only)."""
        rows, cols, vals = [], [], []
        for e in self.cells:
            idx = self.index(e)
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(self.HO[e].ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n, self.n))

    def dense_M(self):
        M = np.zeros((self.n, self.n), self.dtype)
        M[np.arange(self.nh), np.arange(self.nh)] = self.m
        M[self.nh:, self.nh:] = self.Moo
        return M

    def efe_overlap_dense(self):
        """Non-orthogonalized EFE overlap (lumped CC block) for conditioning studies (Sec. V A)."""
        M = np.zeros((self.n, self.n), self.dtype)
        M[np.arange(self.nh), np.arange(self.nh)] = self.m
        B = (self.c * self.m[None, :]).T                                # int N^C_l N^A_nu
        M[:self.nh, self.nh:] = B
        M[self.nh:, :self.nh] = B.conj().T
        M[self.nh:, self.nh:] = self.MAA
        return M

    # -- fields at quadrature points -------------------------------------------
    def values_at_points(self, e, X):
        """u(x_q) on cell e for the columns of X (Eq. UOEFE):
        u = N^C (X^c - Gamma_e X^o) + N^A X^o."""
        idx = self.index(e)
        nl = self.mesh.nloc
        Xo = X[idx[nl:]]
        Xt = X[idx[:nl]] - self.gamma(e) @ Xo
        return self.phiC[e] @ Xt + self.phiA[e] @ Xo
