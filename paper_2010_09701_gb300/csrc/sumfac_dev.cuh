// Sum-factorized application of the CFE-CFE block of a single-leaf cell's Hamiltonian
// (Eq. HOEFEelelements): the potential term through the leaf's Gauss points and the kinetic and
// k terms as Kronecker products of the leaf's 1D matrices. Shared by the FP64 cell products
// (sumfac.cu) and the operator transform (build.cu). Written once for FP64 (V = double) and for
// FP32 pairs (V = f2, pair_dev.cuh).
#pragma once
#include "oefe_internal.h"
#include "pair_dev.cuh"

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
// weights Ws = w_q (V_q + |k|^2 / 2), formed in FP64 and converted to V. Ends with a barrier.
template <typename V>
__device__ inline void sf_prepare(const double* src, V* tab, V* Gr, V* Gi, V* Ws, const double* qw,
                                  const double* veff, int64_t q0, const double k[3]) {
  for (int t = threadIdx.x; t < SF_STRIDE; t += blockDim.x) tab[t] = v_from<V>(src[t]);
  for (int t = threadIdx.x; t < 3 * SF_MAXP * SF_MAXP; t += blockDim.x) {
    const int d = t / (SF_MAXP * SF_MAXP);
    Gr[t] = v_from<V>(0.5 * src[SF_K + t]);
    Gi[t] = v_from<V>(-0.5 * k[d] * src[SF_A + t]);
  }
  const int n1 = (int)src[0];
  const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  for (int q = threadIdx.x; q < n1 * n1 * n1; q += blockDim.x) Ws[q] = v_from<V>(qw[q0 + q] * (veff[q0 + q] + 0.5 * kk));
  __syncthreads();
}

// Ys (P^3 rows x J = NV * R components, R = 2 for complex: re, im interleaved) += H_CC Xs.
// Ab, Bb: work arrays of nbuf * J doubles. All threads of the CTA take part; ends with a barrier.
template <typename V, bool CPLX, int NV>
__device__ void sf_cc(const V* tab, const V* Gr, const V* Gi, const V* Ws, int P, const V* Xs, V* Ys, V* Ab,
                      V* Bb) {
  using A = typename AccOf<V>::type;
  constexpr int R = CPLX ? 2 : 1;
  constexpr int J = NV * R;
  const int P2 = P * P, P3 = P2 * P;
  const int n1 = (int)v_to(tab[0]), n2 = n1 * n1, n3 = n2 * n1;
  const V* L0 = tab + SF_L;                           // L0[qx * SF_MAXP + a]
  const V* L1 = L0 + SF_MAXN1 * SF_MAXP;
  const V* L2 = L1 + SF_MAXN1 * SF_MAXP;
  const V* M0 = tab + SF_M;                           // M0[a * SF_MAXP + a2]
  const V* M1 = M0 + SF_MAXP * SF_MAXP;
  const V* M2 = M1 + SF_MAXP * SF_MAXP;
  // ---- potential term: to the points, weight, back
  for (int t = threadIdx.x; t < P2 * n1 * J; t += blockDim.x) {   // T1[(c,b,qx)] = sum_a L0[qx][a] X[(a,b,c)]
    const int j = t % J, r = t / J, qx = r % n1, cb = r / n1;
    Ab[t] = v_dot<V>(P, [&](int a) { return L0[qx * SF_MAXP + a]; },
                     [&](int a) { return Xs[(size_t)(a + P * cb) * J + j]; });
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P * n2 * J; t += blockDim.x) {   // T2[(c,qy,qx)] = sum_b L1[qy][b] T1[(c,b,qx)]
    const int j = t % J, r = t / J, qx = r % n1, qy = (r / n1) % n1, c = r / n2;
    Bb[t] = v_dot<V>(P, [&](int b) { return L1[qy * SF_MAXP + b]; },
                     [&](int b) { return Ab[(size_t)((c * P + b) * n1 + qx) * J + j]; });
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n3 * J; t += blockDim.x) {       // U[q] = W_q sum_c L2[qz][c] T2[(c,qy,qx)]
    const int j = t % J, q = t / J, qxy = q % n2, qz = q / n2;
    const V s = v_dot<V>(P, [&](int c) { return L2[qz * SF_MAXP + c]; },
                         [&](int c) { return Bb[(size_t)(c * n2 + qxy) * J + j]; });
    Ab[t] = v_mul(s, Ws[q]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P * n2 * J; t += blockDim.x) {   // back in z
    const int j = t % J, r = t / J, qxy = r % n2, c = r / n2;
    Bb[t] = v_dot<V>(n1, [&](int qz) { return L2[qz * SF_MAXP + c]; },
                     [&](int qz) { return Ab[(size_t)(qz * n2 + qxy) * J + j]; });
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P2 * n1 * J; t += blockDim.x) {  // back in y
    const int j = t % J, r = t / J, qx = r % n1, b = (r / n1) % P, c = r / (n1 * P);
    Ab[t] = v_dot<V>(n1, [&](int qy) { return L1[qy * SF_MAXP + b]; },
                     [&](int qy) { return Bb[(size_t)((c * n1 + qy) * n1 + qx) * J + j]; });
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P3 * J; t += blockDim.x) {       // back in x, into Y
    const int j = t % J, m = t / J, a = m % P, cb = m / P;
    const V s = v_dot<V>(n1, [&](int qx) { return L0[qx * SF_MAXP + a]; },
                         [&](int qx) { return Ab[(size_t)(cb * n1 + qx) * J + j]; });
    Ys[t] = v_add(Ys[t], s);
  }
  __syncthreads();

  // ---- kinetic and k terms: sum_d G_d in position d, M elsewhere; G_d = K_d/2 - (i/2) k_d A_d
  //   Z_M = M2 x, Z_G = G2 x (along z); W1 = M1 Z_M, W2 = G1 Z_M + M1 Z_G (along y);
  //   y += G0 W1 + M0 W2 (along x)
  V* ZM = Ab;
  V* ZG = Ab + (size_t)P3 * J;
  V* W1 = Bb;
  V* W2 = Bb + (size_t)P3 * J;
  for (int t = threadIdx.x; t < P3 * NV; t += blockDim.x) {
    const int v = t % NV, m = t / NV, ab = m % P2, c = m / P2;
    A mr = v_zero<V>(), mi = v_zero<V>(), gr = v_zero<V>(), gi = v_zero<V>();
    for (int c2 = 0; c2 < P; ++c2) {
      const V* x = Xs + (size_t)(ab + P2 * c2) * J + v * R;
      const V mm = M2[c * SF_MAXP + c2], kv = Gr[2 * SF_MAXP * SF_MAXP + c * SF_MAXP + c2];
      v_mac(mr, mm, x[0]);
      v_mac(gr, kv, x[0]);
      if (CPLX) {
        const V av = Gi[2 * SF_MAXP * SF_MAXP + c * SF_MAXP + c2];
        v_mac(mi, mm, x[1]);
        v_mac(gi, kv, x[1]);
        v_mac(gr, v_neg(av), x[1]);
        v_mac(gi, av, x[0]);
      }
    }
    ZM[(size_t)m * J + v * R] = v_fin(mr);
    ZG[(size_t)m * J + v * R] = v_fin(gr);
    if (CPLX) {
      ZM[(size_t)m * J + v * R + 1] = v_fin(mi);
      ZG[(size_t)m * J + v * R + 1] = v_fin(gi);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P3 * NV; t += blockDim.x) {
    const int v = t % NV, m = t / NV, a = m % P, b = (m / P) % P, c = m / P2;
    A w1r = v_zero<V>(), w1i = v_zero<V>(), w2r = v_zero<V>(), w2i = v_zero<V>();
    for (int b2 = 0; b2 < P; ++b2) {
      const size_t o = (size_t)(a + P * b2 + P2 * c) * J + v * R;
      const V mm = M1[b * SF_MAXP + b2], kv = Gr[SF_MAXP * SF_MAXP + b * SF_MAXP + b2];
      v_mac(w1r, mm, ZM[o]);
      v_mac(w2r, kv, ZM[o]);
      v_mac(w2r, mm, ZG[o]);
      if (CPLX) {
        const V av = Gi[SF_MAXP * SF_MAXP + b * SF_MAXP + b2];
        v_mac(w1i, mm, ZM[o + 1]);
        v_mac(w2i, kv, ZM[o + 1]);
        v_mac(w2r, v_neg(av), ZM[o + 1]);
        v_mac(w2i, av, ZM[o]);
        v_mac(w2i, mm, ZG[o + 1]);
      }
    }
    W1[(size_t)m * J + v * R] = v_fin(w1r);
    W2[(size_t)m * J + v * R] = v_fin(w2r);
    if (CPLX) {
      W1[(size_t)m * J + v * R + 1] = v_fin(w1i);
      W2[(size_t)m * J + v * R + 1] = v_fin(w2i);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P3 * NV; t += blockDim.x) {
    const int v = t % NV, m = t / NV, a = m % P, bc = m / P;
    A yr = v_zero<V>(), yi = v_zero<V>();
    for (int a2 = 0; a2 < P; ++a2) {
      const size_t o = (size_t)(a2 + P * bc) * J + v * R;
      const V mm = M0[a * SF_MAXP + a2], kv = Gr[a * SF_MAXP + a2];
      v_mac(yr, kv, W1[o]);
      v_mac(yr, mm, W2[o]);
      if (CPLX) {
        const V av = Gi[a * SF_MAXP + a2];
        v_mac(yi, kv, W1[o + 1]);
        v_mac(yr, v_neg(av), W1[o + 1]);
        v_mac(yi, av, W1[o]);
        v_mac(yi, mm, W2[o + 1]);
      }
    }
    Ys[(size_t)m * J + v * R] = v_add(Ys[(size_t)m * J + v * R], v_fin(yr));
    if (CPLX) Ys[(size_t)m * J + v * R + 1] = v_add(Ys[(size_t)m * J + v * R + 1], v_fin(yi));
  }
  __syncthreads();

}

}  // namespace
