"""Density mixing of the self-consistent field iteration (Sec. IV: linear mixing, and the
n-stage Anderson mixing the paper's runs use). TEST INFRASTRUCTURE ONLY.

Each step has an input density rho_in and the output rho_out of the Kohn-Sham map, with residual
F = rho_out - rho_in.
  linear:    rho_next = rho_in + alpha F
  Anderson:  over the last m input densities and residuals, the coefficients c (sum c_i = 1) that
             minimize || sum_i c_i F_i ||_w (w: quadrature weights, the L2 norm over the cell);
             rho_next = sum_i c_i (rho_in,i + alpha F_i).
Reading: the constrained least-squares problem is solved in the usual difference form (one
unconstrained least-squares solve on the differences of consecutive residuals), which is the
same minimization.
"""
import numpy as np


def linear(rho_in, rho_out, alpha):
    return rho_in + alpha * (rho_out - rho_in)


class Anderson:
    def __init__(self, alpha, history=20, weights=None):
        self.alpha, self.m, self.w = float(alpha), int(history), weights
        self.xs, self.fs = [], []

    def step(self, rho_in, rho_out):
        x = np.asarray(rho_in, float)
        f = np.asarray(rho_out, float) - x
        self.xs.append(x.copy())
        self.fs.append(f.copy())
        if len(self.xs) > self.m:
            self.xs.pop(0)
            self.fs.pop(0)
        w = np.ones_like(f) if self.w is None else self.w
        sw = np.sqrt(w)
        k = len(self.fs)
        if k == 1:
            return x + self.alpha * f
        # c = e_last - D g with D the differences of consecutive residuals: minimize |F_last - D g|
        D = np.stack([(self.fs[i + 1] - self.fs[i]) * sw for i in range(k - 1)], axis=1)
        g, *_ = np.linalg.lstsq(D, self.fs[-1] * sw, rcond=None)
        xbar = self.xs[-1].copy()
        fbar = self.fs[-1].copy()
        for i in range(k - 1):
            xbar -= g[i] * (self.xs[i + 1] - self.xs[i])
            fbar -= g[i] * (self.fs[i + 1] - self.fs[i])
        return xbar + self.alpha * fbar
