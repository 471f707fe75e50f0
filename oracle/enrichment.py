"""Atomic enrichment functions (Sec. III A, Eqs. UOEFEAtomic, KSAtomicTrunc,
CutoffProperties).

N^A_nu(x) = exp(-i k.(x - R_I^x)) psi_nlm(|x - R_I^x|, angles) h(|x - R_I^x|)
with R_I^x the periodic image of nucleus I nearest to x (Eq. UOEFEAtomic).

Readings (the paper defers these details elsewhere):
* radial part R(r): tabulated on a uniform grid [0, rc] together with R'(r),
  interpolated by cubic Hermite polynomials; zero for r >= rc;
* angular part: real harmonics, S_s = 1/sqrt(4 pi), S_{p_d} = sqrt(3/(4 pi)) x_d / r;
* cutoff: h = phi(s) / (phi(s) + phi(1 - s)), s = (rc - r) / (rc - r0),
  phi(t) = exp(-1/t) for t > 0, else 0. It is 1 for r <= r0 and 0 for r >= rc,
  i.e. rc = r0 (1 + 1/t) in the paper's notation.
"""
import math

import numpy as np

INV_SQRT_4PI = 1.0 / math.sqrt(4.0 * math.pi)
SQRT_3_4PI = math.sqrt(3.0 / (4.0 * math.pi))


def hermite_eval(R, dR, rc, r):
    """Cubic Hermite interpolant of tabulated (R, R') on a uniform grid [0, rc]."""
    n = len(R)
    dr = rc / (n - 1)
    r = np.asarray(r, float)
    inside = r < rc
    s = np.where(inside, r, 0.0) / dr
    i = np.minimum(np.floor(s).astype(int), n - 2)
    t = s - i
    h00 = 2 * t ** 3 - 3 * t ** 2 + 1
    h10 = t ** 3 - 2 * t ** 2 + t
    h01 = -2 * t ** 3 + 3 * t ** 2
    h11 = t ** 3 - t ** 2
    val = h00 * R[i] + h10 * dr * dR[i] + h01 * R[i + 1] + h11 * dr * dR[i + 1]
    d00 = 6 * t ** 2 - 6 * t
    d10 = 3 * t ** 2 - 4 * t + 1
    d01 = -6 * t ** 2 + 6 * t
    d11 = 3 * t ** 2 - 2 * t
    der = (d00 * R[i] + d10 * dr * dR[i] + d01 * R[i + 1] + d11 * dr * dR[i + 1]) / dr
    return np.where(inside, val, 0.0), np.where(inside, der, 0.0)


def _phi(t):
    tt = np.where(t > 0, t, 1.0)
    return np.where(t > 0, np.exp(-1.0 / tt), 0.0)


def _dphi(t):
    tt = np.where(t > 0, t, 1.0)
    return np.where(t > 0, np.exp(-1.0 / tt) / (tt * tt), 0.0)


def cutoff(r, r0, rc):
    """Smooth cutoff h(r) and dh/dr (Eq. CutoffProperties)."""
    s = (rc - np.asarray(r, float)) / (rc - r0)
    f, g = _phi(s), _phi(1.0 - s)
    den = f + g
    h = f / den
    dhds = (_dphi(s) * g + f * _dphi(1.0 - s)) / den ** 2
    return h, -dhds / (rc - r0)


def nearest_image_disp(x, R, a):
    """x - R_I^x: displacement from the nearest periodic image (Eq. UOEFEAtomic)."""
    d = np.asarray(x, float) - R
    return d - a * np.round(d / a)


class Enrichment:
    """Enrichment data: atoms, one radial table per (atom, function), angular codes."""

    def __init__(self, a, pos, lm, R, dR, r0, rc):
        self.a = float(a)
        self.pos = np.asarray(pos, float)
        self.lm = np.asarray(lm, int)          # per function of an atom: 0 s, 1..3 p_x,p_y,p_z
        self.R = np.asarray(R, float)          # (natoms, nfun, ngrid)
        self.dR = np.asarray(dR, float)
        self.r0, self.rc = float(r0), float(rc)
        self.natoms = len(self.pos)
        self.nfun = len(self.lm)
        self.nO = self.natoms * self.nfun

    def atom_of(self, nu):
        return nu // self.nfun

    def psi(self, nu, x):
        """Real truncated orbital psi~ and its gradient at points x (npts, 3)."""
        I, j = divmod(nu, self.nfun)
        d = nearest_image_disp(x, self.pos[I], self.a)
        r = np.sqrt(np.sum(d * d, axis=1))
        rs = np.where(r > 0, r, 1.0)
        Rv, Rd = hermite_eval(self.R[I, j], self.dR[I, j], self.rc, r)
        h, hd = cutoff(r, self.r0, self.rc)
        u = d / rs[:, None]                      # unit vector (0 at r = 0)
        u[r == 0] = 0.0
        code = self.lm[j]
        if code == 0:
            val = INV_SQRT_4PI * Rv * h
            grad = (INV_SQRT_4PI * (Rd * h + Rv * hd))[:, None] * u
        else:
            m = code - 1
            g = Rv * h / rs
            gp = (Rd * h + Rv * hd) / rs - Rv * h / (rs * rs)
            val = SQRT_3_4PI * d[:, m] * g
            grad = SQRT_3_4PI * (d[:, m] * gp)[:, None] * u
            grad[:, m] += SQRT_3_4PI * g
        return val, grad, d

    def values(self, nu, x, k):
        """N^A_nu and its gradient at x for Bloch vector k (complex unless k = 0)."""
        val, grad, d = self.psi(nu, x)
        if not np.any(k):
            return val, grad
        ph = np.exp(-1j * (d @ np.asarray(k, float)))
        return ph * val, ph[:, None] * (grad - 1j * np.asarray(k, float)[None, :] * val[:, None])


def active_sets(mesh, enr):
    """act_A(e): functions whose support meets cell e; act(e): functions whose
    orthogonalized form N^O = N^A - sum_l c_l N^C can be non-zero on e, i.e. the
    union of act_A over the cells sharing a node with e (Eq. UOEFEOrtho and the
    locality remark after Eq. orthCGLL)."""
    from .quadrature import box_point_dist2
    actA = []
    for e in range(mesh.ncells):
        lo, hi = mesh.cell_box(e)
        atoms = [I for I in range(enr.natoms)
                 if box_point_dist2(lo, hi, enr.pos[I], mesh.a) < enr.rc ** 2]
        actA.append(np.array([I * enr.nfun + j for I in atoms for j in range(enr.nfun)], int))
    act = []
    for e in range(mesh.ncells):
        s = set()
        for f in mesh.neighbours(e):
            s.update(actA[f].tolist())
        act.append(np.array(sorted(s), int))
    return actA, act
