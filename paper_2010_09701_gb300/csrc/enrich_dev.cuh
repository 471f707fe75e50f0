// Device evaluation of one atomic enrichment function and its gradient
// (Eqs. UOEFEAtomic, KSAtomicTrunc, CutoffProperties); shared by the
// operator construction and the density kernels.
#pragma once
#include "oefe_internal.h"

namespace {

struct EnrParams {
  const double* pos;
  const int* lm;
  const double* R;
  const double* dR;
  int nfun, ngrid;
  double a, r0, rc;
};

__device__ inline double phi_step(double t) { return t > 0 ? exp(-1.0 / t) : 0.0; }
__device__ inline double dphi_step(double t) { return t > 0 ? exp(-1.0 / t) / (t * t) : 0.0; }

// Truncated orbital times Bloch phase and its gradient (Eqs. UOEFEAtomic, KSAtomicTrunc).
__device__ void enrichment_value(const EnrParams& E, int nu, const double x[3], const double k[3],
                                 cd* val, cd grad[3]) {
  const int I = nu / E.nfun, j = nu % E.nfun;
  double d[3];
  for (int t = 0; t < 3; ++t) {
    double v = x[t] - E.pos[3 * I + t];
    d[t] = v - E.a * rint(v / E.a);  // nearest periodic image (ties to even)
  }
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double rs = r > 0 ? r : 1.0;
  double u[3];
  for (int t = 0; t < 3; ++t) u[t] = r > 0 ? d[t] / rs : 0.0;
  // cubic Hermite interpolation of the radial table
  double Rv = 0, Rd = 0;
  if (r < E.rc) {
    const double* Rt = E.R + (size_t)(I * E.nfun + j) * E.ngrid;
    const double* dRt = E.dR + (size_t)(I * E.nfun + j) * E.ngrid;
    const double dr = E.rc / (E.ngrid - 1);
    const double s = r / dr;
    int i = (int)floor(s);
    if (i > E.ngrid - 2) i = E.ngrid - 2;
    const double t = s - i;
    const double t2 = t * t, t3 = t2 * t;
    const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
    Rv = h00 * Rt[i] + h10 * dr * dRt[i] + h01 * Rt[i + 1] + h11 * dr * dRt[i + 1];
    const double d00 = 6 * t2 - 6 * t, d10 = 3 * t2 - 4 * t + 1, d01 = -6 * t2 + 6 * t, d11 = 3 * t2 - 2 * t;
    Rd = (d00 * Rt[i] + d10 * dr * dRt[i] + d01 * Rt[i + 1] + d11 * dr * dRt[i + 1]) / dr;
  }
  // smooth cutoff h(r) (Eq. CutoffProperties)
  const double sc = (E.rc - r) / (E.rc - E.r0);
  const double f = phi_step(sc), g = phi_step(1.0 - sc);
  const double den = f + g;
  const double h = f / den;
  const double hd = -((dphi_step(sc) * g + f * dphi_step(1.0 - sc)) / (den * den)) / (E.rc - E.r0);
  double v, gr[3];
  const int code = E.lm[j];
  if (code == 0) {
    const double c0 = 0.28209479177387814;  // 1 / sqrt(4 pi)
    v = c0 * Rv * h;
    const double gs = c0 * (Rd * h + Rv * hd);
    for (int t = 0; t < 3; ++t) gr[t] = gs * u[t];
  } else {
    const int m = code - 1;
    const double c1 = 0.4886025119029199;   // sqrt(3 / (4 pi))
    const double gg = Rv * h / rs;
    const double gp = (Rd * h + Rv * hd) / rs - Rv * h / (rs * rs);
    v = c1 * d[m] * gg;
    for (int t = 0; t < 3; ++t) gr[t] = c1 * (d[m] * gp) * u[t];
    gr[m] += c1 * gg;
  }
  if (k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0) {
    *val = mkc(v, 0.0);
    for (int t = 0; t < 3; ++t) grad[t] = mkc(gr[t], 0.0);
    return;
  }
  const double th = k[0] * d[0] + k[1] * d[1] + k[2] * d[2];
  double sn, cs;
  sincos(th, &sn, &cs);
  const cd ph = mkc(cs, -sn);  // exp(-i k.(x - R))
  *val = ph * mkc(v, 0.0);
  for (int t = 0; t < 3; ++t) grad[t] = ph * mkc(gr[t], -k[t] * v);
}

// Lagrange polynomials on the nodes xn (P of them) and their derivatives at x.
__device__ void lagrange_eval(const double* xn, int P, double x, double* L, double* D) {
  for (int a = 0; a < P; ++a) {
    double v = 1.0;
    for (int b = 0; b < P; ++b)
      if (b != a) v *= (x - xn[b]) / (xn[a] - xn[b]);
    L[a] = v;
    double s = 0.0;
    for (int c = 0; c < P; ++c) {
      if (c == a) continue;
      double term = 1.0 / (xn[a] - xn[c]);
      for (int b = 0; b < P; ++b)
        if (b != a && b != c) term *= (x - xn[b]) / (xn[a] - xn[b]);
      s += term;
    }
    D[a] = s;
  }
}

}  // namespace
