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

// What the functions of one atom share at a point x: the nearest-image offset, r, the unit vector,
// the cutoff h(r) and h'(r) (Eq. CutoffProperties) and the Bloch phase exp(-i k.(x - R)).
struct AtomGeom {
  double d[3], u[3], r, rs, h, hd;
  cd ph;
  bool kz;
};

__device__ inline void atom_geom(const EnrParams& E, int I, const double x[3], const double k[3], bool grad,
                                 AtomGeom& G) {
  for (int t = 0; t < 3; ++t) {
    double v = x[t] - E.pos[3 * I + t];
    G.d[t] = v - E.a * rint(v / E.a);  // nearest periodic image (ties to even)
  }
  G.r = sqrt(G.d[0] * G.d[0] + G.d[1] * G.d[1] + G.d[2] * G.d[2]);
  G.rs = G.r > 0 ? G.r : 1.0;
  for (int t = 0; t < 3; ++t) G.u[t] = G.r > 0 ? G.d[t] / G.rs : 0.0;
  const double sc = (E.rc - G.r) / (E.rc - E.r0);
  const double f = phi_step(sc), g = phi_step(1.0 - sc);
  const double den = f + g;
  G.h = f / den;
  G.hd = grad ? -((dphi_step(sc) * g + f * dphi_step(1.0 - sc)) / (den * den)) / (E.rc - E.r0) : 0.0;
  G.kz = k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0;
  if (!G.kz) {
    const double th = k[0] * G.d[0] + k[1] * G.d[1] + k[2] * G.d[2];
    double sn, cs;
    sincos(th, &sn, &cs);
    G.ph = mkc(cs, -sn);
  } else {
    G.ph = mkc(1.0, 0.0);
  }
}

// Function j of atom I at the point described by G: radial table (cubic Hermite), real harmonic,
// cutoff and phase (Eqs. UOEFEAtomic, KSAtomicTrunc); grad may be null.
__device__ inline void atom_function(const EnrParams& E, int I, int j, const AtomGeom& G, const double k[3],
                                     cd* val, cd* grad) {
  const double r = G.r, rs = G.rs;
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
    if (grad) {
      const double d00 = 6 * t2 - 6 * t, d10 = 3 * t2 - 4 * t + 1, d01 = -6 * t2 + 6 * t, d11 = 3 * t2 - 2 * t;
      Rd = (d00 * Rt[i] + d10 * dr * dRt[i] + d01 * Rt[i + 1] + d11 * dr * dRt[i + 1]) / dr;
    }
  }
  const double h = G.h, hd = G.hd;
  double v, gr[3] = {0.0, 0.0, 0.0};
  const int code = E.lm[j];
  if (code == 0) {
    const double c0 = 0.28209479177387814;  // 1 / sqrt(4 pi)
    v = c0 * Rv * h;
    if (grad) {
      const double gs = c0 * (Rd * h + Rv * hd);
      for (int t = 0; t < 3; ++t) gr[t] = gs * G.u[t];
    }
  } else {
    const int m = code - 1;
    const double c1 = 0.4886025119029199;   // sqrt(3 / (4 pi))
    const double gg = Rv * h / rs;
    v = c1 * G.d[m] * gg;
    if (grad) {
      const double gp = (Rd * h + Rv * hd) / rs - Rv * h / (rs * rs);
      for (int t = 0; t < 3; ++t) gr[t] = c1 * (G.d[m] * gp) * G.u[t];
      gr[m] += c1 * gg;
    }
  }
  if (G.kz) {
    *val = mkc(v, 0.0);
    if (grad)
      for (int t = 0; t < 3; ++t) grad[t] = mkc(gr[t], 0.0);
    return;
  }
  *val = G.ph * mkc(v, 0.0);
  if (grad)
    for (int t = 0; t < 3; ++t) grad[t] = G.ph * mkc(gr[t], -k[t] * v);
}

// Truncated orbital times Bloch phase and its gradient (Eqs. UOEFEAtomic, KSAtomicTrunc).
__device__ inline void enrichment_value(const EnrParams& E, int nu, const double x[3], const double k[3], cd* val,
                                        cd grad[3]) {
  const int I = nu / E.nfun, j = nu % E.nfun;
  AtomGeom G;
  atom_geom(E, I, x, k, true, G);
  atom_function(E, I, j, G, k, val, grad);
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
