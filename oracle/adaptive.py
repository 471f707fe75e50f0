"""Convergence-driven adaptive quadrature (Sec. III B): each cell's box is split recursively into
octants until a set of trial integrals involving the enrichment functions has converged.
TEST INFRASTRUCTURE ONLY (see the package docstring); the fixed recipe of ``quadrature`` is what the
rest of the oracle and the CUDA library use.

Readings (the paper defers the details to earlier work):
* Trial integrals of a box: for every enrichment function whose support meets it, int |N^A|^2 and
  int |grad N^A|^2 (the integrands of the overlap and kinetic blocks, the sharpest ones).
* A box has converged when its n-point tensor Gauss rule and the sum of the same rule over its eight
  octants agree to ``tol`` (absolute, per trial integral, scaled by the cell's volume fraction of
  the unit cell so that the total error over the mesh stays below ``tol``); the octants' estimate
  is then kept. Boxes meeting no support keep the plain rule; the recursion stops at ``max_depth``.
"""
import numpy as np

from .quadrature import box_point_dist2, tensor_gauss_box


def _octants(lo, hi):
    mid = 0.5 * (lo + hi)
    out = []
    for cz in range(2):
        for cy in range(2):
            for cx in range(2):
                c = (cx, cy, cz)
                out.append((np.array([lo[d] if c[d] == 0 else mid[d] for d in range(3)]),
                            np.array([mid[d] if c[d] == 0 else hi[d] for d in range(3)])))
    return out


def trial_integrands(enr, funcs):
    """Point values (npts, 2 len(funcs)) of |N^A_nu|^2 and |grad N^A_nu|^2 at the Gamma point."""
    zero = np.zeros(3)

    def f(x):
        cols = []
        for nu in funcs:
            v, g = enr.values(nu, x, zero)
            cols.append(np.abs(v) ** 2)
            cols.append(np.sum(np.abs(g) ** 2, axis=1))
        return np.stack(cols, axis=1)

    return f


def adaptive_leaves(lo, hi, f, n, tol, max_depth, level=0):
    """Leaves (lo, hi) of the box's adaptive octree for the trial integrands f (see above)."""
    p, w = tensor_gauss_box(lo, hi, n)
    coarse = w @ f(p)
    kids = _octants(lo, hi)
    fine = 0.0
    for clo, chi in kids:
        cp, cw = tensor_gauss_box(clo, chi, n)
        fine = fine + cw @ f(cp)
    if level >= max_depth or np.max(np.abs(fine - coarse)) <= tol:
        return kids
    out = []
    for clo, chi in kids:
        out += adaptive_leaves(clo, chi, f, n, tol, max_depth, level + 1)
    return out


class AdaptiveQuadrature:
    """Point sets of every cell (``offset[e]:offset[e+1]``), the layout of ``Quadrature``: cells
    whose box meets no enrichment support take ``nq_cell`` points per axis, the others the adaptive
    leaves of their trial integrals with ``nq_enr`` points per axis."""

    def __init__(self, mesh, enr, nq_cell, nq_enr, tol, max_depth):
        self.mesh = mesh
        vol = mesh.a ** 3
        pts, wts, off, self.leaves = [], [], [0], []
        for e in range(mesh.ncells):
            lo, hi = mesh.cell_box(e)
            funcs = [I * enr.nfun + j for I in range(enr.natoms)
                     if box_point_dist2(lo, hi, enr.pos[I], mesh.a) < enr.rc ** 2 for j in range(enr.nfun)]
            if not funcs:
                leaves, n = [(lo, hi)], nq_cell
            else:
                share = tol * np.prod(hi - lo) / vol
                leaves, n = adaptive_leaves(lo, hi, trial_integrands(enr, funcs), nq_enr, share, max_depth), nq_enr
            self.leaves.append(leaves)
            for l0, l1 in leaves:
                p, w = tensor_gauss_box(l0, l1, n)
                pts.append(p)
                wts.append(w)
            off.append(off[-1] + len(leaves) * n ** 3)
        self.points = np.concatenate(pts)
        self.weights = np.concatenate(wts)
        self.offset = np.array(off)
        self.nq = len(self.weights)

    def cell(self, e):
        s = slice(self.offset[e], self.offset[e + 1])
        return self.points[s], self.weights[s]

    def reference_coords(self, e):
        lo, hi = self.mesh.cell_box(e)
        x, _ = self.cell(e)
        return 2.0 * (x - lo) / (hi - lo) - 1.0
