// Sum-factorized application of the CFE-CFE block of a single-leaf cell's Hamiltonian
// (Eq. HOEFEelelements): the potential term through the leaf's Gauss points and the kinetic and
// k terms as Kronecker products of the leaf's 1D matrices. Shared by the FP64 cell products
// (sumfac.cu) and the operator transform (build.cu).
#pragma once
#include "oefe_internal.h"

namespace {

constexpr int SF_MAXN1 = 12;
constexpr int SF_MAXP = 8;
constexpr int SF_L = 8;                                  // offsets (doubles) of the per-cell tables
constexpr int SF_M = SF_L + 3 * SF_MAXN1 * SF_MAXP;      // L[3][n1][P], then M, K, A [3][P][P]
constexpr int SF_K = SF_M + 3 * SF_MAXP * SF_MAXP;
constexpr int SF_A = SF_K + 3 * SF_MAXP * SF_MAXP;
constexpr int SF_STRIDE = 896;                          // doubles per cell (n1, L, M, K, A)
constexpr int SF_EXTRA = 6 * SF_MAXP * SF_MAXP;         // per CTA: K/2 and -(k/2) A, [2][3][P][P]

// Per CTA: the cell's tables (tab, SF_STRIDE), Gr = K_d / 2 and Gi = -(k_d / 2) A_d, and the point
// weights Ws = w_q (V_q + |k|^2 / 2). Ends with a barrier.
__device__ inline void sf_prepare(const double* src, double* tab, double* Gr, double* Gi, double* Ws,
                                  const double* qw, const double* veff, int64_t q0, const double k[3]) {
  for (int t = threadIdx.x; t < SF_STRIDE; t += blockDim.x) tab[t] = src[t];
  for (int t = threadIdx.x; t < 3 * SF_MAXP * SF_MAXP; t += blockDim.x) {
    const int d = t / (SF_MAXP * SF_MAXP);
    Gr[t] = 0.5 * src[SF_K + t];
    Gi[t] = -0.5 * k[d] * src[SF_A + t];
  }
  const int n1 = (int)src[0];
  const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  for (int q = threadIdx.x; q < n1 * n1 * n1; q += blockDim.x) Ws[q] = qw[q0 + q] * (veff[q0 + q] + 0.5 * kk);
  __syncthreads();
}

// Ys (P^3 rows x J = NV * R components, R = 2 for complex: re, im interleaved) += H_CC Xs.
// Ab, Bb: work arrays of nbuf * J doubles. All threads of the CTA take part; ends with a barrier.
template <bool CPLX, int NV>
__device__ void sf_cc(const double* tab, const double* Gr, const double* Gi, const double* Ws, int P,
                      const double* Xs, double* Ys, double* Ab, double* Bb) {
  constexpr int R = CPLX ? 2 : 1;
  constexpr int J = NV * R;
  const int P2 = P * P, P3 = P2 * P;
  const int n1 = (int)tab[0], n2 = n1 * n1, n3 = n2 * n1;
  const double* L0 = tab + SF_L;                      // L0[qx * SF_MAXP + a]
  const double* L1 = L0 + SF_MAXN1 * SF_MAXP;
  const double* L2 = L1 + SF_MAXN1 * SF_MAXP;
  const double* M0 = tab + SF_M;                      // M0[a * SF_MAXP + a2]
  const double* M1 = M0 + SF_MAXP * SF_MAXP;
  const double* M2 = M1 + SF_MAXP * SF_MAXP;
  // ---- potential term: to the points, weight, back
  for (int t = threadIdx.x; t < P2 * n1 * J; t += blockDim.x) {   // T1[(c,b,qx)] = sum_a L0[qx][a] X[(a,b,c)]
    const int j = t % J, r = t / J, qx = r % n1, cb = r / n1;
    double s = 0.0;
    for (int a = 0; a < P; ++a) s = fma(L0[qx * SF_MAXP + a], Xs[(size_t)(a + P * cb) * J + j], s);
    Ab[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P * n2 * J; t += blockDim.x) {   // T2[(c,qy,qx)] = sum_b L1[qy][b] T1[(c,b,qx)]
    const int j = t % J, r = t / J, qx = r % n1, qy = (r / n1) % n1, c = r / n2;
    double s = 0.0;
    for (int b = 0; b < P; ++b) s = fma(L1[qy * SF_MAXP + b], Ab[(size_t)((c * P + b) * n1 + qx) * J + j], s);
    Bb[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n3 * J; t += blockDim.x) {       // U[q] = W_q sum_c L2[qz][c] T2[(c,qy,qx)]
    const int j = t % J, q = t / J, qxy = q % n2, qz = q / n2;
    double s = 0.0;
    for (int c = 0; c < P; ++c) s = fma(L2[qz * SF_MAXP + c], Bb[(size_t)(c * n2 + qxy) * J + j], s);
    Ab[t] = s * Ws[q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P * n2 * J; t += blockDim.x) {   // back in z
    const int j = t % J, r = t / J, qxy = r % n2, c = r / n2;
    double s = 0.0;
    for (int qz = 0; qz < n1; ++qz) s = fma(L2[qz * SF_MAXP + c], Ab[(size_t)(qz * n2 + qxy) * J + j], s);
    Bb[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P2 * n1 * J; t += blockDim.x) {  // back in y
    const int j = t % J, r = t / J, qx = r % n1, b = (r / n1) % P, c = r / (n1 * P);
    double s = 0.0;
    for (int qy = 0; qy < n1; ++qy) s = fma(L1[qy * SF_MAXP + b], Bb[(size_t)((c * n1 + qy) * n1 + qx) * J + j], s);
    Ab[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P3 * J; t += blockDim.x) {       // back in x, into Y
    const int j = t % J, m = t / J, a = m % P, cb = m / P;
    double s = 0.0;
    for (int qx = 0; qx < n1; ++qx) s = fma(L0[qx * SF_MAXP + a], Ab[(size_t)(cb * n1 + qx) * J + j], s);
    Ys[t] += s;
  }
  __syncthreads();

  // ---- kinetic and k terms: sum_d G_d in position d, M elsewhere; G_d = K_d/2 - (i/2) k_d A_d
  //   Z_M = M2 x, Z_G = G2 x (along z); W1 = M1 Z_M, W2 = G1 Z_M + M1 Z_G (along y);
  //   y += G0 W1 + M0 W2 (along x)
  double* ZM = Ab;
  double* ZG = Ab + (size_t)P3 * J;
  double* W1 = Bb;
  double* W2 = Bb + (size_t)P3 * J;
  for (int t = threadIdx.x; t < P3 * NV; t += blockDim.x) {
    const int v = t % NV, m = t / NV, ab = m % P2, c = m / P2;
    double mr = 0, mi = 0, gr = 0, gi = 0;
    for (int c2 = 0; c2 < P; ++c2) {
      const double* x = Xs + (size_t)(ab + P2 * c2) * J + v * R;
      const double mm = M2[c * SF_MAXP + c2], kv = Gr[2 * SF_MAXP * SF_MAXP + c * SF_MAXP + c2];
      mr = fma(mm, x[0], mr);
      gr = fma(kv, x[0], gr);
      if (CPLX) {
        const double av = Gi[2 * SF_MAXP * SF_MAXP + c * SF_MAXP + c2];
        mi = fma(mm, x[1], mi);
        gi = fma(kv, x[1], gi);
        gr = fma(-av, x[1], gr);
        gi = fma(av, x[0], gi);
      }
    }
    ZM[(size_t)m * J + v * R] = mr;
    ZG[(size_t)m * J + v * R] = gr;
    if (CPLX) {
      ZM[(size_t)m * J + v * R + 1] = mi;
      ZG[(size_t)m * J + v * R + 1] = gi;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P3 * NV; t += blockDim.x) {
    const int v = t % NV, m = t / NV, a = m % P, b = (m / P) % P, c = m / P2;
    double w1r = 0, w1i = 0, w2r = 0, w2i = 0;
    for (int b2 = 0; b2 < P; ++b2) {
      const size_t o = (size_t)(a + P * b2 + P2 * c) * J + v * R;
      const double mm = M1[b * SF_MAXP + b2], kv = Gr[SF_MAXP * SF_MAXP + b * SF_MAXP + b2];
      w1r = fma(mm, ZM[o], w1r);
      w2r = fma(kv, ZM[o], w2r);
      w2r = fma(mm, ZG[o], w2r);
      if (CPLX) {
        const double av = Gi[SF_MAXP * SF_MAXP + b * SF_MAXP + b2];
        w1i = fma(mm, ZM[o + 1], w1i);
        w2i = fma(kv, ZM[o + 1], w2i);
        w2r = fma(-av, ZM[o + 1], w2r);
        w2i = fma(av, ZM[o], w2i);
        w2i = fma(mm, ZG[o + 1], w2i);
      }
    }
    W1[(size_t)m * J + v * R] = w1r;
    W2[(size_t)m * J + v * R] = w2r;
    if (CPLX) {
      W1[(size_t)m * J + v * R + 1] = w1i;
      W2[(size_t)m * J + v * R + 1] = w2i;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P3 * NV; t += blockDim.x) {
    const int v = t % NV, m = t / NV, a = m % P, bc = m / P;
    double yr = 0, yi = 0;
    for (int a2 = 0; a2 < P; ++a2) {
      const size_t o = (size_t)(a2 + P * bc) * J + v * R;
      const double mm = M0[a * SF_MAXP + a2], kv = Gr[a * SF_MAXP + a2];
      yr = fma(kv, W1[o], yr);
      yr = fma(mm, W2[o], yr);
      if (CPLX) {
        const double av = Gi[a * SF_MAXP + a2];
        yi = fma(kv, W1[o + 1], yi);
        yr = fma(-av, W1[o + 1], yr);
        yi = fma(av, W1[o], yi);
        yi = fma(mm, W2[o + 1], yi);
      }
    }
    Ys[(size_t)m * J + v * R] += yr;
    if (CPLX) Ys[(size_t)m * J + v * R + 1] += yi;
  }
  __syncthreads();

}

}  // namespace
