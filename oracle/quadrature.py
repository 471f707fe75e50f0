"""Per-cell quadrature point sets (Sec. III B, adaptive quadrature).

The paper refines the quadrature near nuclei by recursive subdivision until
trial integrals converge and defers the details to earlier work. Reading
taken here: a deterministic recipe with the same intent.

* A cell whose box meets no enrichment support (no ball |x - R_I| < r_c)
  gets a tensor Gauss rule with ``nq_cell`` points per axis.
* A cell that meets a support gets ``nq_enr`` points per axis.
* A cell whose closed box holds a nucleus (any periodic image) is split into
  8 children, and every child that still holds a nucleus is split again, up
  to ``depth`` levels; every leaf gets the ``nq_enr`` Gauss rule.

Point order: cells ascending; within a cell, leaves in depth-first order with
children (cx, cy, cz) enumerated cx fastest; within a leaf, qx fastest.
One point set per cell serves every term of the Hamiltonian, the
orthogonalizing integrals, the enrichment overlap and the density.
"""
import numpy as np

from .fe1d import gauss

TOUCH_TOL = 1e-12


def _images(x, a):
    return (x - a, x, x + a)


def box_holds_point(lo, hi, R, a):
    """True if some periodic image of R lies in the closed box [lo, hi]."""
    tol = TOUCH_TOL * a
    for d in range(3):
        if not any(lo[d] - tol <= y <= hi[d] + tol for y in _images(R[d], a)):
            return False
    return True


def box_point_dist2(lo, hi, R, a):
    """Squared distance from the box to the nearest periodic image of R."""
    s = 0.0
    for d in range(3):
        best = np.inf
        for y in _images(R[d], a):
            t = max(lo[d] - y, 0.0, y - hi[d])
            best = min(best, t)
        s += best * best
    return s


def cell_class(lo, hi, pos, a, rc):
    """0 plain, 1 meets an enrichment support, 2 holds a nucleus."""
    if any(box_holds_point(lo, hi, R, a) for R in pos):
        return 2
    if any(box_point_dist2(lo, hi, R, a) < rc * rc for R in pos):
        return 1
    return 0


def _leaves(lo, hi, pos, a, level, depth):
    if level < depth and any(box_holds_point(lo, hi, R, a) for R in pos):
        mid = 0.5 * (lo + hi)
        out = []
        for cz in range(2):
            for cy in range(2):
                for cx in range(2):
                    c = (cx, cy, cz)
                    clo = np.array([lo[d] if c[d] == 0 else mid[d] for d in range(3)])
                    chi = np.array([mid[d] if c[d] == 0 else hi[d] for d in range(3)])
                    out += _leaves(clo, chi, pos, a, level + 1, depth)
        return out
    return [(lo, hi)]


def tensor_gauss_box(lo, hi, n):
    """Points (n^3, 3) and weights of the n-point Gauss rule on a box, qx fastest."""
    t, w = gauss(n)
    xs = [lo[d] + (t + 1) / 2 * (hi[d] - lo[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    W = (w[None, None, :] * w[None, :, None] * w[:, None, None]).ravel() * np.prod(hi - lo) / 8.0
    return pts, W


class Quadrature:
    """Point sets of every cell; ``offset[e]:offset[e+1]`` slices cell e.

    ``cells`` (optional) limits the point sets to those cells, the others get none: a bounded
    sample of a large mesh (every listed cell has exactly the points it has in the full set)."""

    def __init__(self, mesh, pos, rc, nq_cell, nq_enr, depth, cells=None):
        self.mesh = mesh
        keep = None if cells is None else set(int(e) for e in cells)
        pts, wts, off, cls = [], [], [0], []
        for e in range(mesh.ncells):
            if keep is not None and e not in keep:
                cls.append(-1)
                off.append(off[-1])
                continue
            lo, hi = mesh.cell_box(e)
            c = cell_class(lo, hi, pos, mesh.a, rc)
            cls.append(c)
            if c == 0:
                leaves = [(lo, hi)]
                n = nq_cell
            else:
                leaves = _leaves(lo, hi, pos, mesh.a, 0, depth) if c == 2 else [(lo, hi)]
                n = nq_enr
            for (l0, l1) in leaves:
                p, w = tensor_gauss_box(l0, l1, n)
                pts.append(p)
                wts.append(w)
            off.append(off[-1] + sum(n ** 3 for _ in leaves))
        self.points = np.concatenate(pts)
        self.weights = np.concatenate(wts)
        self.offset = np.array(off)
        self.cls = np.array(cls)
        self.nq = len(self.weights)

    def cell(self, e):
        s = slice(self.offset[e], self.offset[e + 1])
        return self.points[s], self.weights[s]

    def reference_coords(self, e):
        """Points of cell e mapped to the reference cube [-1, 1]^3."""
        lo, hi = self.mesh.cell_box(e)
        x, _ = self.cell(e)
        return 2.0 * (x - lo) / (hi - lo) - 1.0
