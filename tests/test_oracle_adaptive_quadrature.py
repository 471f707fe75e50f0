"""Pins of the oracle's convergence-driven adaptive quadrature (Sec. III B): exact on polynomials
without refinement, the enrichment functions' trial integrals to the requested tolerance against
radial integrals of the same functions, far fewer points than refining everywhere, the refinement
inside the supports."""
import numpy as np

from cases import uniform_xb
import workloads as W
from oracle.adaptive import AdaptiveQuadrature, adaptive_leaves, trial_integrands
from oracle.enrichment import Enrichment
from oracle.mesh import Mesh
from oracle.quadrature import Quadrature, box_point_dist2, tensor_gauss_box


def small_enrichment(a=6.0):
    pos = np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, a / 2]])
    Z = np.array([3, 4])
    R, dR = W.radial_tables(Z, W.ORBITALS_1S_2P, rc=2.5, ngrid=2000)
    return pos, Enrichment(a, pos, W.orbital_lm_codes(W.ORBITALS_1S_2P), R, dR, 1.5, 2.5)


def test_polynomials_need_no_refinement():
    # a degree-7 polynomial per axis is integrated exactly by 4 Gauss points: the first split agrees
    lo, hi = np.array([0.0, -1.0, 0.5]), np.array([1.5, 0.5, 2.0])

    def f(x):
        return (x[:, :1] ** 7 - 2 * x[:, 1:2] ** 5 * x[:, 2:3] ** 3 + 1.0)

    leaves = adaptive_leaves(lo, hi, f, 4, 1e-12, 6)
    assert len(leaves) == 8
    exact = (1.5 ** 8 / 8 * 1.5 * 1.5 - 2 * ((0.5 ** 6 - 1.0) / 6) * ((2.0 ** 4 - 0.5 ** 4) / 4) * 1.5
             + 1.5 ** 3)
    total = sum(float(tensor_gauss_box(l0, l1, 4)[1] @ f(tensor_gauss_box(l0, l1, 4)[0])[:, 0]) for l0, l1 in leaves)
    assert abs(total - exact) < 1e-12 * abs(exact)


def radial_reference(enr, pos, nu):
    """int |N^A_nu|^2 and int |grad N^A_nu|^2 over all space by radial Gauss-Legendre quadrature of the
    oracle's own function values along an axis (the support of radius r_c fits in the cell, so the
    cell sum is the full-space integral): s functions 4 pi int r^2 f^2, 4 pi int r^2 f'^2; p functions
    (4 pi / 3) int r^2 f^2 and (4 pi / 3) int (r^2 f'^2 + 2 f^2), f along the function's own axis."""
    lm = enr.lm[nu % enr.nfun]
    ax = np.zeros(3)
    ax[max(lm - 1, 0)] = 1.0
    t, w = np.polynomial.legendre.leggauss(400)
    n2 = g2 = 0.0
    for r0, r1 in ((0.0, 0.5), (0.5, enr.r0), (enr.r0, enr.rc)):   # the cusp and the cutoff shell apart
        r = r0 + (r1 - r0) * (t + 1) / 2
        v, g = enr.values(nu, pos[nu // enr.nfun][None, :] + r[:, None] * ax[None, :], np.zeros(3))
        f, df = np.real(v), np.real(g @ ax)
        c = 4 * np.pi if lm == 0 else 4 * np.pi / 3
        n2 += c * (r1 - r0) / 2 * np.sum(w * r * r * f * f)
        g2 += c * (r1 - r0) / 2 * np.sum(w * (r * r * df * df + (0.0 if lm == 0 else 2 * f * f)))
    return n2, g2


def test_trial_integrals_match_radial_integrals_with_few_points():
    a = 6.0
    pos, enr = small_enrichment(a)
    mesh = Mesh(a, uniform_xb(a, 2), 3)
    tol = 1e-3
    aq = AdaptiveQuadrature(mesh, enr, 5, 8, tol, 8)
    ia = aq.weights @ trial_integrands(enr, list(range(enr.nO)))(aq.points)
    ref = np.concatenate([radial_reference(enr, pos, nu) for nu in range(enr.nO)])
    assert np.max(np.abs(ia - ref)) < tol
    # the refinement sits inside the supports (at the nuclei and in the cutoff shell r0 < r < r_c,
    # where the smooth truncation bends the functions): the smallest leaf is within r_c of a nucleus
    vols = [(np.prod(l1 - l0), l0, l1) for leaves in aq.leaves for (l0, l1) in leaves]
    vmin, l0, l1 = min(vols, key=lambda t: t[0])
    assert min(box_point_dist2(l0, l1, R, a) for R in pos) < enr.rc ** 2
    # far fewer points than splitting every enriched cell down to the smallest leaf
    lo, hi = mesh.cell_box(0)
    depth = int(round(np.log(np.prod(hi - lo) / vmin) / np.log(8)))
    enriched = sum(1 for leaves in aq.leaves if len(leaves) > 1)
    assert depth >= 3 and aq.nq < enriched * 8 ** depth * 8 ** 3 / 3
