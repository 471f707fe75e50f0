"""Local-density exchange and correlation (Sec. II: LDA with the Ceperley-Alder data in the
Perdew-Zunger parametrization), spin-unpolarized, Hartree atomic units. TEST INFRASTRUCTURE ONLY.

With r_s = (3 / (4 pi rho))^(1/3):
  exchange     eps_x = -(3/4) (3 rho / pi)^(1/3)
  correlation  eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)              (r_s >= 1)
               eps_c = A ln r_s + B + C r_s ln r_s + D r_s                     (r_s < 1)
with the published unpolarized constants gamma = -0.1423, beta1 = 1.0529, beta2 = 0.3334,
A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116. V_xc = d(rho eps_xc)/d rho = eps_xc -
(r_s / 3) d eps_xc / d r_s; E_xc = int rho eps_xc. Reading: points with rho <= 1e-30 (outside the
atoms' tails, or a round-off negative density) contribute nothing.
"""
import numpy as np

GAMMA, BETA1, BETA2 = -0.1423, 1.0529, 0.3334
A_PZ, B_PZ, C_PZ, D_PZ = 0.0311, -0.048, 0.0020, -0.0116
RHO_MIN = 1e-30


def _rs(rho):
    return (3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0)


def eps_c_and_derivative(rs):
    """eps_c(r_s) and d eps_c / d r_s, both branches of the fit."""
    rs = np.asarray(rs, float)
    hi = rs >= 1.0
    s = np.sqrt(rs)
    den = 1.0 + BETA1 * s + BETA2 * rs
    e_lo_density = GAMMA / den
    de_lo_density = -GAMMA * (0.5 * BETA1 / s + BETA2) / den ** 2
    lnr = np.log(rs)
    e_hi_density = A_PZ * lnr + B_PZ + C_PZ * rs * lnr + D_PZ * rs
    de_hi_density = A_PZ / rs + C_PZ * (lnr + 1.0) + D_PZ
    return np.where(hi, e_lo_density, e_hi_density), np.where(hi, de_lo_density, de_hi_density)


def lda(rho):
    """(eps_xc, V_xc) at the given densities."""
    rho = np.asarray(rho, float)
    ok = rho > RHO_MIN
    r = np.where(ok, rho, 1.0)
    ex = -0.75 * (3.0 * r / np.pi) ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex                          # d(rho eps_x)/d rho, eps_x ~ rho^(1/3)
    rs = _rs(r)
    ec, dec = eps_c_and_derivative(rs)
    vc = ec - rs / 3.0 * dec
    return np.where(ok, ex + ec, 0.0), np.where(ok, vx + vc, 0.0)


def xc_energy(rho, w):
    """E_xc = sum_q w_q rho_q eps_xc(rho_q)."""
    e, _ = lda(rho)
    return float(np.sum(w * np.asarray(rho) * e))
