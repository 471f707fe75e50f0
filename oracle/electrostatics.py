"""Total electrostatic potential with smeared nuclear charges (Sec. II, Eqs. eqnpoisson,
eqnsmeared, eqngr, eqnpoissonaux, eqnpoissontotsmear, eqnnuc, eqnnucsmear, eqnvg) and the
electrostatic energy E_elec (Sec. II, energy equations), for the oracle of the SCF driver that
surrounds the hot path. TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings:
* r_c,I, "the largest values that avoid overlap between neighbouring smeared charges": half the
  distance from nucleus I to its nearest other nucleus or periodic image of itself (minimal image;
  an image is a cell edge a away), so that r_c,I + r_c,J never exceeds the distance between I and J.
* The Poisson problem of Eq. eqnpoissonaux is solved on the periodic cell with the continuous FE
  basis alone (A_mn = (1/4 pi) int grad N_m . grad N_n, c_m = int N_m f); its right-hand side is
  neutral (the smeared charges integrate to -sum Z and rho to the electron count) and the solution
  is taken with zero mean over the cell (the constant is not fixed by a periodic Poisson problem;
  it cancels in E_elec for a neutral cell). The paper enriches phi_aux with one function per atom;
  the oracle refines the mesh instead.
* Minimal images throughout: no r_c exceeds half the cell edge.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import cfe_basis


def smeared_charge(r, rc):
    """g(r, r_c) (Eq. eqngr): a unit charge on the ball r <= r_c, zero outside."""
    r = np.asarray(r, float)
    inside = -21.0 * (r - rc) ** 3 * (6.0 * r * r + 3.0 * r * rc + rc * rc) / (5.0 * np.pi * rc ** 8)
    return np.where(r <= rc, inside, 0.0)


def smeared_potential(r, rc):
    """v_g(r, r_c) (Eq. eqnvg): the potential of g, 1/r outside the ball."""
    r = np.asarray(r, float)
    inside = (9 * r ** 7 - 30 * r ** 6 * rc + 28 * r ** 5 * rc ** 2 - 14 * r ** 2 * rc ** 5 + 12 * rc ** 7) / (5 * rc ** 8)
    with np.errstate(divide="ignore"):
        outside = 1.0 / np.where(r > 0, r, 1.0)
    return np.where(r <= rc, inside, outside)


def self_energy_integral(rc):
    """I_g(r_c) = 10976 / (17875 r_c), the value the paper gives with its energy expression."""
    return 10976.0 / (17875.0 * rc)


def minimal_image(d, a):
    return d - a * np.round(d / a)


def cutoff_radii(pos, a):
    """r_c,I: half the distance to the nearest other nucleus or own periodic image (minimal image)."""
    pos = np.asarray(pos, float).reshape(-1, 3)
    rc = np.full(len(pos), 0.5 * a)
    for i in range(len(pos)):
        for j in range(len(pos)):
            if i != j:
                rc[i] = min(rc[i], 0.5 * np.linalg.norm(minimal_image(pos[i] - pos[j], a)))
    return rc


def _dist(x, R, a):
    return np.linalg.norm(minimal_image(np.asarray(x, float) - R, a), axis=-1)


def smeared_nuclear_charge(x, pos, Z, rc, a):
    """b_smear(x) = -sum_I Z_I g(|x - R_I|, r_c,I) (Eq. eqnsmeared)."""
    out = np.zeros(len(x))
    for R, z, r in zip(np.asarray(pos, float).reshape(-1, 3), Z, rc):
        out -= z * smeared_charge(_dist(x, R, a), r)
    return out


def nuclear_correction(x, pos, Z, rc, a):
    """sum_I (V_N,I - V_N,I^smear)(|x - R_I|) = sum_I -Z_I (1/r - v_g(r, r_c,I)) (Eqs. eqnnuc,
    eqnnucsmear), zero outside every ball. Undefined at a nucleus itself."""
    out = np.zeros(len(x))
    for R, z, r0 in zip(np.asarray(pos, float).reshape(-1, 3), Z, rc):
        r = _dist(x, R, a)
        with np.errstate(divide="ignore", invalid="ignore"):
            out -= z * np.where(r <= r0, 1.0 / r - smeared_potential(r, r0), 0.0)
    return out


def poisson_matrices(mesh, quad):
    """The CFE stiffness (1/4 pi) int grad N_m . grad N_n and, per cell, the values of the basis at
    the cell's points (for the load vector)."""
    rows, cols, vals = [], [], []
    tabs = {}
    for e in range(mesh.ncells):
        phi, grad = cfe_basis(mesh, quad, e)
        _, w = quad.cell(e)
        Ae = sum(grad[d].T @ (w[:, None] * grad[d]) for d in range(3)) / (4.0 * np.pi)
        n = mesh.cell_nodes(e)
        rows.append(np.repeat(n, len(n)))
        cols.append(np.tile(n, len(n)))
        vals.append(Ae.ravel())
        tabs[e] = phi
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(mesh.nh, mesh.nh))
    return A, tabs


def poisson_factor(A):
    """Sparse LU of the stiffness with node 0 held at zero (the constants are the null space of the
    periodic problem: holding one node removes it; the mean is restored after the solve)."""
    return spla.splu(A[1:, 1:].tocsc())


def solve_poisson(mesh, quad, f, A=None, tabs=None, lu=None):
    """Nodal values of phi with -(1/4 pi) lap phi = f on the periodic cell, zero mean (the reading
    above). f: values at every quadrature point; its integral must vanish. lu: ``poisson_factor``
    of A (then a direct solve), else conjugate gradients."""
    if A is None:
        A, tabs = poisson_matrices(mesh, quad)
    c = np.zeros(mesh.nh)
    for e in range(mesh.ncells):
        _, w = quad.cell(e)
        s = slice(quad.offset[e], quad.offset[e + 1])
        np.add.at(c, mesh.cell_nodes(e), tabs[e].T @ (w * f[s]))
    m = mesh.lumped_mass()
    # the constants span the null space: project them out of the load, solve, then remove the mean
    c -= m * (np.sum(c) / np.sum(m))
    if lu is not None:
        phi = np.concatenate([[0.0], lu.solve(c[1:])])
    else:
        phi, info = spla.cg(A, c, rtol=1e-13, atol=0.0, maxiter=20 * mesh.nh)
        if info != 0:
            raise RuntimeError("Poisson CG did not converge")
    return phi - np.sum(m * phi) / np.sum(m)


def field_at_points(mesh, quad, nodal, tabs=None):
    """A CFE nodal field interpolated at every quadrature point (tabs: the basis values per cell, as
    ``poisson_matrices`` returns them, else tabulated here)."""
    out = np.zeros(quad.nq)
    for e in range(mesh.ncells):
        phi = tabs[e] if tabs is not None else cfe_basis(mesh, quad, e)[0]
        out[quad.offset[e]:quad.offset[e + 1]] = phi @ nodal[mesh.cell_nodes(e)]
    return out


def electrostatic_energy(quad, pos, Z, rc, a, rho, b_smear, phi_aux):
    """E_elec: (1/2) int (b_smear + rho) phi_aux + sum_I int_{Omega_I} rho (V_N,I - V_N,I^smear)
    + sum_I (1/2) Z_I^2 (I_g(r_c,I) - v_g(0, r_c,I)); every field at the quadrature points."""
    w = quad.weights
    e = 0.5 * np.sum(w * (b_smear + rho) * phi_aux)
    e += np.sum(w * rho * nuclear_correction(quad.points, pos, Z, rc, a))
    for z, r in zip(Z, rc):
        e += 0.5 * z * z * (self_energy_integral(r) - float(smeared_potential(0.0, r)))
    return e
