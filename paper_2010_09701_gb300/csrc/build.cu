// GPU construction of the OEFE operators (Sec. III A):
//  * enrichment tabulation at the quadrature points (Eqs. UOEFEAtomic, KSAtomicTrunc),
//  * orthogonalizing coefficients c_{nu,l} (Eq. orthCGLL) and M^oo (Eq. Moo),
//  * EFE cell matrices (Eq. HOEFEelelements) by sum factorization over each
//    tensor-product leaf of the cell's point set,
//  * H^O_e = T_e^+ H_e T_e (Eq. UOEFESplit), stored in FP64 and/or FP32.
// All arithmetic is FP64 (complex for k != 0).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "oefe_internal.h"
#include "pair_dev.cuh"
#include "enrich_dev.cuh"
#include "sumfac_dev.cuh"

namespace {

constexpr int MAXP = 8;     // P = p + 1 <= 8
constexpr int MAXN1 = 12;   // Gauss points per axis per leaf
constexpr int BT = 256;     // threads per CTA of the cell kernels
constexpr int TT = 352;     // threads per CTA of the transform: one local node each (n_loc <= 343 at p = 6)
constexpr int TJB = 8;      // enrichment columns per pass of the transform
constexpr size_t SMEM_SETUP = 212 * 1024;  // setup mode: one CTA per SM
constexpr size_t SMEM_BUILD = 96 * 1024;   // build mode: two CTAs per SM

// A complex value in arithmetic V (FP64 or an FP32 pair): the cell-matrix accumulator of the
// per-step build, 16 bytes either way.
template <typename V>
struct VC {
  V re, im;
};


// Tabulate N^A and grad N^A for (point, active function) pairs of a batch of cells.
// tab entry layout: 4 complex values (value, d/dx, d/dy, d/dz) per (q, j), j fastest.
// Active sets hold whole atoms (nfun consecutive functions), so one thread takes one (point, atom)
// and evaluates what the atom's functions share (offset, cutoff, phase) once.
__global__ void k_tabulate(EnrParams E, const double* qxyz, const int64_t* q_off, const int* act_off,
                           const int* act_idx, int e0, int ncell_b, const int64_t* tab_off,
                           double kx, double ky, double kz, cd* tab) {
  const int64_t total = E.nfun > 0 ? tab_off[ncell_b] / E.nfun : 0;
  const double k[3] = {kx, ky, kz};
  for (int64_t tb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tb < total;
       tb += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = tb * E.nfun;
    int lo = 0, hi = ncell_b - 1;
    while (lo < hi) {  // last b with tab_off[b] <= t
      int mid = (lo + hi + 1) / 2;
      if (tab_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int e = e0 + lo;
    const int ne = act_off[e + 1] - act_off[e];
    const int64_t r = t - tab_off[lo];
    const int64_t q = q_off[e] + r / ne;
    const int j0 = (int)(r % ne);
    const int I = act_idx[act_off[e] + j0] / E.nfun;
    const double x[3] = {qxyz[3 * q], qxyz[3 * q + 1], qxyz[3 * q + 2]};
    AtomGeom G;
    atom_geom(E, I, x, k, true, G);
    for (int f = 0; f < E.nfun; ++f) {
      cd v, g[3];
      atom_function(E, I, f, G, k, &v, g);
      cd* o = tab + 4 * (t + f);
      o[0] = v;
      o[1] = g[0];
      o[2] = g[1];
      o[3] = g[2];
    }
  }
}

// A CTA's share of the build (mode 0): leaves [l0, l1) of batch cell b. slot < 0 writes the
// cell matrix itself (and adds the cached V-independent blocks); slot >= 0 writes partial `slot`,
// added to the cell matrix afterwards in a fixed order (deterministic sums).
struct BuildItem {
  int b, l0, l1, slot;
};

struct BuildArgs {
  const Leaf* leaves;
  const int* leaf_off;
  const double* qxyz;
  const double* qw;
  const double* veff;       // null in the setup mode
  const double* cellbox;
  const double* gll;
  const double* gauss_w;    // [n][i] table, 13 x 12
  const int* act_off;
  const int64_t* tab_off;
  const int64_t* q_off;
  const cd* tab;
  int e0, P, nloc, npad, ne_max;
  double k[3];
  // 0: EFE blocks with weights w (V + |k|^2/2) plus the cached V-independent CA0, AA0 -> HE (the
  //    setup pass that forms the transformed V-independent blocks, with V = 0);
  // 1: setup (d, M^AA, V-independent EFE enrichment blocks CA0, AA0)
  int mode;
  cd* HE;                   // mode 0: (batch, npad, npad)
  cd* dblk;                 // mode 1: (ncells, nloc, ne_max)
  cd* MAAblk;               // mode 1: (ncells, ne_max, ne_max)
  cd* E0;                   // per cell: V-independent CA (nloc x ne_max) then AA (ne_max x ne_max)
  const BuildItem* items;   // mode 0: one CTA per item (a cell's leaf range); null: one CTA per cell
  cd* HP;                   // mode 0: partial cell matrices of the items with slot >= 0
  size_t smem;              // dynamic shared memory of the launch
};

// One CTA per cell (or per leaf range of a cell), accumulating over the cell's tensor-product leaves.
//
// Setup (mode 1, once per k): d = int N^C N^A and M^AA = int conj(N^A) N^A for
// the orthogonalization, and the V-independent parts of the enrichment
// blocks of Eq. HOEFEelelements (kinetic and k terms) into the cache E0.
// Mode 0 (setup, V = 0): the CC block (kinetic, k term and the potential
// term on the leaf points, by sum factorization; Hermitian half computed),
// the potential parts of the CA and AA blocks, plus the cached E0; the
// transform then turns these into the V-independent OEFE blocks.
__global__ void __launch_bounds__(BT) k_build_cell(BuildArgs A) {
  extern __shared__ double smem[];
  const BuildItem it = A.items ? A.items[blockIdx.x] : BuildItem{(int)blockIdx.x, -1, -1, -1};
  const int b = it.b;
  const int e = A.e0 + b;
  const int P = A.P, nloc = A.nloc, npad = A.npad;
  const int ne = A.act_off[e + 1] - A.act_off[e];
  const double* box = A.cellbox + 6 * e;
  const double kk = A.k[0] * A.k[0] + A.k[1] * A.k[1] + A.k[2] * A.k[2];
  const bool kz = kk == 0.0;
  const size_t e0s = (size_t)nloc * A.ne_max + (size_t)A.ne_max * A.ne_max;
  cd* CA0 = A.E0 + (size_t)e * e0s;                 // nloc x ne_max
  cd* AA0 = CA0 + (size_t)nloc * A.ne_max;          // ne_max x ne_max

  __shared__ double Lt[3][MAXN1][MAXP], Dt[3][MAXN1][MAXP], w1[3][MAXN1];
  __shared__ double Mm[3][MAXP][MAXP], Km[3][MAXP][MAXP], Am[3][MAXP][MAXP];
  __shared__ double xn[MAXP];
  if (threadIdx.x < P) xn[threadIdx.x] = A.gll[threadIdx.x];

  cd* HE = A.HE ? (it.slot < 0 ? A.HE + (size_t)b * npad * npad : A.HP + (size_t)it.slot * npad * npad) : nullptr;
  const bool vmode = A.mode == 0;   // a cell matrix is formed
  cd* dB = A.dblk ? A.dblk + (size_t)e * nloc * A.ne_max : nullptr;
  cd* MB = A.MAAblk ? A.MAAblk + (size_t)e * A.ne_max * A.ne_max : nullptr;
  if (vmode) {
    for (int i = threadIdx.x; i < npad * npad; i += BT) HE[i] = mkc(0, 0);
  } else {
    for (int i = threadIdx.x; i < nloc * A.ne_max; i += BT) { dB[i] = mkc(0, 0); CA0[i] = mkc(0, 0); }
    for (int i = threadIdx.x; i < A.ne_max * A.ne_max; i += BT) { MB[i] = mkc(0, 0); AA0[i] = mkc(0, 0); }
  }
  __syncthreads();

  const cd* tabc = A.tab ? A.tab + 4 * A.tab_off[b] : nullptr;  // this cell's tabulation, (q, j) j fastest
  const int l_begin = it.l0 >= 0 ? it.l0 : A.leaf_off[e], l_end = it.l0 >= 0 ? it.l1 : A.leaf_off[e + 1];
  for (int li = l_begin; li < l_end; ++li) {
    const Leaf L = A.leaves[li];
    const int n1 = L.n1, n2 = n1 * n1, n3 = n2 * n1;
    const int64_t q0 = L.q0;
    const int64_t ql0 = q0 - A.q_off[e];  // leaf offset within the cell
    // 1D tables: reference coordinate of the leaf's points on each axis
    if (threadIdx.x < 3 * n1) {
      const int d = threadIdx.x / n1, i = threadIdx.x % n1;
      const int64_t qi = q0 + (d == 0 ? i : d == 1 ? i * n1 : i * n2);
      const double x = A.qxyz[3 * qi + d];
      const double xi = 2.0 * (x - box[d]) / box[3 + d] - 1.0;
      double Lv[MAXP], Dv[MAXP];
      lagrange_eval(xn, P, xi, Lv, Dv);
      for (int a = 0; a < P; ++a) {
        Lt[d][i][a] = Lv[a];
        Dt[d][i][a] = Dv[a] * (2.0 / box[3 + d]);
      }
      w1[d][i] = A.gauss_w[n1 * 12 + i] * (L.hi[d] - L.lo[d]) / 2.0;
    }
    __syncthreads();

    if (vmode) {
      // 1D mass, stiffness and antisymmetric gradient matrices of the leaf
      for (int t = threadIdx.x; t < 3 * P * P; t += BT) {
        const int d = t / (P * P), a = (t / P) % P, a2 = t % P;
        double m = 0, kq = 0, g1 = 0, g2 = 0;
        for (int i = 0; i < n1; ++i) {
          m += w1[d][i] * Lt[d][i][a] * Lt[d][i][a2];
          kq += w1[d][i] * Dt[d][i][a] * Dt[d][i][a2];
          g1 += w1[d][i] * Lt[d][i][a] * Dt[d][i][a2];
          g2 += w1[d][i] * Dt[d][i][a] * Lt[d][i][a2];
        }
        Mm[d][a][a2] = m;
        Km[d][a][a2] = kq;
        Am[d][a][a2] = g1 - g2;
      }
      // potential weight field W_q (V_q + |k|^2 / 2)
      double* Wv = smem;                       // n3
      double* S1 = Wv + n3;                    // n2 * P * P  [(qx,qy)][c][c']
      double* S2 = S1 + n2 * P * P;            // cx * P^4    [qx][b][b'][c][c']
      for (int q = threadIdx.x; q < n3; q += BT) Wv[q] = A.qw[q0 + q] * (A.veff[q0 + q] + 0.5 * kk);
      __syncthreads();
      for (int t = threadIdx.x; t < n2 * P * P; t += BT) {
        const int qxy = t / (P * P), c = (t / P) % P, c2 = t % P;
        double s = 0;
        for (int qz = 0; qz < n1; ++qz) s += Wv[qxy + n2 * qz] * Lt[2][qz][c] * Lt[2][qz][c2];
        S1[t] = s;
      }
      __syncthreads();
      const int P2 = P * P, P4 = P2 * P2;
      const int budget = (int)((A.smem / sizeof(double) - n3 - (size_t)n2 * P2) / P4);
      const int cx = min(n1, max(1, budget));
      for (int qx0 = 0; qx0 < n1; qx0 += cx) {
        const int nx = min(cx, n1 - qx0);
        for (int t = threadIdx.x; t < nx * P4; t += BT) {
          const int ix = t / P4, r = t % P4;
          const int bb = r / (P * P2), b2 = (r / P2) % P, cc = r % P2;  // (b, b', (c,c'))
          double s = 0;
          for (int qy = 0; qy < n1; ++qy)
            s += Lt[1][qy][bb] * Lt[1][qy][b2] * S1[((qx0 + ix) + n1 * qy) * P2 + cc];
          S2[t] = s;
        }
        __syncthreads();
        const bool first = qx0 == 0;
        // Hermitian half: entries m <= n, mirrored
        for (int t = threadIdx.x; t < nloc * nloc; t += BT) {
          const int m = t / nloc, n = t % nloc;
          if (m > n) continue;
          const int a = m % P, bb = (m / P) % P, c = m / P2;
          const int a2 = n % P, b2 = (n / P) % P, c2 = n / P2;
          const int ridx = (bb * P + b2) * P2 + c * P + c2;
          double v = 0;
          for (int ix = 0; ix < nx; ++ix) v += Lt[0][qx0 + ix][a] * Lt[0][qx0 + ix][a2] * S2[ix * P4 + ridx];
          double im = 0;
          if (first) {
            v += 0.5 * (Km[0][a][a2] * Mm[1][bb][b2] * Mm[2][c][c2] + Mm[0][a][a2] * Km[1][bb][b2] * Mm[2][c][c2] +
                        Mm[0][a][a2] * Mm[1][bb][b2] * Km[2][c][c2]);
            if (!kz)
              im = -0.5 * (A.k[0] * Am[0][a][a2] * Mm[1][bb][b2] * Mm[2][c][c2] +
                           A.k[1] * Mm[0][a][a2] * Am[1][bb][b2] * Mm[2][c][c2] +
                           A.k[2] * Mm[0][a][a2] * Mm[1][bb][b2] * Am[2][c][c2]);
          }
          cd* h = HE + (size_t)m * npad + n;
          h->x += v;
          h->y += im;
          if (m != n) {
            cd* h2 = HE + (size_t)n * npad + m;
            h2->x += v;
            h2->y -= im;
          }
        }
        __syncthreads();
      }
    }

    // enrichment columns: staged contraction of the CFE factors against the
    // enrichment fields of the leaf.
    //   mode 0: F0 = w (V + |k|^2/2) N                                 -> CA (potential part)
    //   mode 1: F0 = -(i/2) w k.grad N, F_d = w (grad_d N / 2 + (i/2) k_d N) -> CA0;  Fd = w N -> d
    {
      cd* F = reinterpret_cast<cd*>(smem);     // 5 fields * n3
      cd* G = F + (A.mode == 1 ? 5 : 1) * n3;                // 4 (setup) or 1 fields of n2 * P
      cd* Hs = G + (A.mode == 1 ? 4 : 1) * n2 * P;           // 3 (setup) or 1 fields of n1 * P * P
      const bool full = A.mode == 1;
      for (int j = 0; j < ne; ++j) {
        for (int q = threadIdx.x; q < n3; q += BT) {
          const double w = A.qw[q0 + q];
          const cd* tq = tabc + 4 * ((ql0 + q) * ne + j);
          if (!full) {
            F[q] = (w * (A.veff[q0 + q] + 0.5 * kk)) * tq[0];
          } else {
            const cd N = tq[0];
            const cd kg = A.k[0] * tq[1] + A.k[1] * tq[2] + A.k[2] * tq[3];
            F[q] = w * (mkc(0, -0.5) * kg);
            for (int d = 0; d < 3; ++d) F[(1 + d) * n3 + q] = w * (0.5 * tq[1 + d] + mkc(0, 0.5 * A.k[d]) * N);
            F[4 * n3 + q] = w * N;
          }
        }
        __syncthreads();
        // stage z: (qx,qy,c)
        for (int t = threadIdx.x; t < n2 * P; t += BT) {
          const int qxy = t / P, c = t % P;
          cd g0 = mkc(0, 0), gx = mkc(0, 0), gy = mkc(0, 0), gz = mkc(0, 0), gd = mkc(0, 0);
          for (int qz = 0; qz < n1; ++qz) {
            const int q = qxy + n2 * qz;
            const double l = Lt[2][qz][c];
            g0 = rfma(l, F[q], g0);
            if (full) {
              gx = rfma(l, F[n3 + q], gx);
              gy = rfma(l, F[2 * n3 + q], gy);
              gz = rfma(Dt[2][qz][c], F[3 * n3 + q], gz);
              gd = rfma(l, F[4 * n3 + q], gd);
            }
          }
          G[t] = g0 + gz;
          if (full) {
            G[n2 * P + t] = gx;
            G[2 * n2 * P + t] = gy;
            G[3 * n2 * P + t] = gd;
          }
        }
        __syncthreads();
        // stage y: (qx,b,c)
        for (int t = threadIdx.x; t < n1 * P * P; t += BT) {
          const int qx = t / (P * P), bb = (t / P) % P, c = t % P;
          cd h0 = mkc(0, 0), hx = mkc(0, 0), hy = mkc(0, 0), hd = mkc(0, 0);
          for (int qy = 0; qy < n1; ++qy) {
            const int g = (qx + n1 * qy) * P + c;
            h0 = rfma(Lt[1][qy][bb], G[g], h0);
            if (full) {
              hx = rfma(Lt[1][qy][bb], G[n2 * P + g], hx);
              hy = rfma(Dt[1][qy][bb], G[2 * n2 * P + g], hy);
              hd = rfma(Lt[1][qy][bb], G[3 * n2 * P + g], hd);
            }
          }
          Hs[t] = h0 + hy;
          if (full) {
            Hs[n1 * P * P + t] = hx;
            Hs[2 * n1 * P * P + t] = hd;
          }
        }
        __syncthreads();
        // stage x: (a,b,c) -> local node a + P (b + P c)
        for (int m = threadIdx.x; m < nloc; m += BT) {
          const int a = m % P, bc = m / P;
          const int bb = bc % P, c = bc / P;
          cd s = mkc(0, 0), sd = mkc(0, 0);
          for (int qx = 0; qx < n1; ++qx) {
            const int hidx = (qx * P + bb) * P + c;
            s = rfma(Lt[0][qx][a], Hs[hidx], s);
            if (full) {
              s = rfma(Dt[0][qx][a], Hs[n1 * P * P + hidx], s);
              sd = rfma(Lt[0][qx][a], Hs[2 * n1 * P * P + hidx], sd);
            }
          }
          if (!full) HE[(size_t)m * npad + nloc + j] += s;
          else {
            CA0[(size_t)m * A.ne_max + j] += s;
            dB[(size_t)m * A.ne_max + j] += sd;
          }
        }
        __syncthreads();
      }
    }

    // enrichment-enrichment block: pairs (i <= j) over the leaf points, staged
    // through shared memory in chunks of points
    {
      const bool full = A.mode == 1;
      const int comps = full ? 4 : 1;
      const int QC = max(1, min(32, (int)((A.smem - 32 * 8) / ((size_t)max(ne, 1) * comps * sizeof(cd)))));
      cd* Ns = reinterpret_cast<cd*>(smem);   // QC x ne x comps
      double* Ws = reinterpret_cast<double*>(Ns + (size_t)QC * ne * comps);  // QC
      const int npairs = ne * (ne + 1) / 2;
      for (int pb = 0; pb < npairs; pb += 4 * BT) {
        int pi[4], pj[4];
        cd acc0[4], acc1[4];
        for (int u = 0; u < 4; ++u) {
          acc0[u] = mkc(0, 0);
          acc1[u] = mkc(0, 0);
          const int pp = pb + threadIdx.x + u * BT;
          pi[u] = -1;
          pj[u] = -1;
          if (pp < npairs) {  // pair index -> (i, j), i <= j
            int i = 0, rem = pp;
            while (rem >= ne - i) { rem -= ne - i; ++i; }
            pi[u] = i;
            pj[u] = i + rem;
          }
        }
        for (int qc = 0; qc < n3; qc += QC) {
          const int nq = min(QC, n3 - qc);
          __syncthreads();
          for (int t = threadIdx.x; t < nq * ne * comps; t += BT) {
            const int q = t / (ne * comps), r = t % (ne * comps);
            const int j = r / comps, cpt = r % comps;
            Ns[t] = tabc[4 * ((ql0 + qc + q) * ne + j) + cpt];
          }
          for (int q = threadIdx.x; q < nq; q += BT) {
            const double w = A.qw[q0 + qc + q];
            Ws[q] = full ? w : w * (A.veff[q0 + qc + q] + 0.5 * kk);
          }
          __syncthreads();
          for (int u = 0; u < 4; ++u) {
            if (pi[u] < 0) continue;
            const int i = pi[u], j = pj[u];
            cd s0 = mkc(0, 0), s1 = mkc(0, 0);
            for (int q = 0; q < nq; ++q) {
              const cd* ti = Ns + ((size_t)q * ne + i) * comps;
              const cd* tj = Ns + ((size_t)q * ne + j) * comps;
              const double w = Ws[q];
              if (!full) {
                s0 = cfmac(w * ti[0], tj[0], s0);
              } else {
                cd v = 0.5 * (cmulc(ti[1], tj[1]) + cmulc(ti[2], tj[2]) + cmulc(ti[3], tj[3]));
                if (!kz) {
                  const cd kgj = A.k[0] * tj[1] + A.k[1] * tj[2] + A.k[2] * tj[3];
                  const cd kgi = A.k[0] * ti[1] + A.k[1] * ti[2] + A.k[2] * ti[3];
                  v += mkc(0, -0.5) * (cmulc(ti[0], kgj) - cmulc(kgi, tj[0]));
                }
                s0 += w * v;
                s1 += w * cmulc(ti[0], tj[0]);
              }
            }
            acc0[u] += s0;
            acc1[u] += s1;
          }
        }
        for (int u = 0; u < 4; ++u) {
          if (pi[u] < 0) continue;
          const int i = pi[u], j = pj[u];
          if (!full) {
            HE[(size_t)(nloc + i) * npad + nloc + j] += acc0[u];
            if (i != j) HE[(size_t)(nloc + j) * npad + nloc + i] += cconj(acc0[u]);
          } else {
            AA0[i * A.ne_max + j] += acc0[u];
            MB[i * A.ne_max + j] += acc1[u];
            if (i != j) {
              AA0[j * A.ne_max + i] += cconj(acc0[u]);
              MB[j * A.ne_max + i] += cconj(acc1[u]);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (vmode && it.slot < 0) {
    // cached V-independent EFE enrichment blocks CA0, AA0
    for (int t = threadIdx.x; t < nloc * ne; t += BT) {
      const int m = t / ne, j = t % ne;
      HE[(size_t)m * npad + nloc + j] += CA0[(size_t)m * A.ne_max + j];
    }
    for (int t = threadIdx.x; t < ne * ne; t += BT) {
      const int i = t / ne, j = t % ne;
      HE[(size_t)(nloc + i) * npad + nloc + j] += AA0[i * A.ne_max + j];
    }
  }
}


// ------------------------------------------------------------------ per-step build (OEFE basis)

struct OefeArgs {
  const Leaf* leaves;
  const int* leaf_off;
  const double* qxyz;
  const double* qw;
  const double* veff;
  const double* cellbox;
  const double* gll;
  const double* gauss_w;    // [n][i] table, 13 x 12
  const int* act_off;
  const void* NO;           // N^O per leaf, column-major: double / cd (V = double), float2 / float4 (f2)
  bool no_cplx;
  int e0, P, nloc, npad, ne_max;
  double k[3];
  void* HE;                 // VC<V> (batch, npad, npad)
  void* HP;                 // VC<V> partials of the split cells
  const cd* E0;             // per cell: V-independent OEFE blocks CO0 (nloc x ne_max), OO0 (ne_max^2)
  const BuildItem* items;
  size_t smem;
};

template <typename V>
__device__ inline VC<V> load_no(const OefeArgs& A, size_t o) {
  if constexpr (std::is_same<V, double>::value) {
    if (A.no_cplx) {
      const cd w = reinterpret_cast<const cd*>(A.NO)[o];
      return VC<V>{w.x, w.y};
    }
    return VC<V>{reinterpret_cast<const double*>(A.NO)[o], 0.0};
  } else {
    if (A.no_cplx) {
      const float4 w = reinterpret_cast<const float4*>(A.NO)[o];
      return VC<V>{f2{w.x, w.y}, f2{w.z, w.w}};
    }
    const float2 w = reinterpret_cast<const float2*>(A.NO)[o];
    return VC<V>{f2{w.x, w.y}, f2{0.0f, 0.0f}};
  }
}

// symmetric pair index of (i, j): max(i,j) (max(i,j) + 1) / 2 + min(i,j), and its inverse's larger
// member
__device__ __forceinline__ int sym_idx(int i, int j) {
  const int h = max(i, j), l = min(i, j);
  return h * (h + 1) / 2 + l;
}
__device__ __forceinline__ int sym_hi(int s) {
  int h = 0;
  while ((h + 1) * (h + 2) / 2 <= s) ++h;
  return h;
}

template <typename V>
__device__ inline void vc_add(VC<V>* h, V re, V im) {
  VC<V> x = *h;
  x.re = v_add(x.re, re);
  x.im = v_add(x.im, im);
  *h = x;
}

// The cell matrix of the V term in the OEFE basis plus the cached V-independent blocks (Eq.
// HOEFEelelements with Eq. UOEFESplit): per tensor-product leaf of the item,
//   CC += sum_q w_q (V_q + |k|^2/2) N_a N_b + the kinetic and k terms (sum factorization over the
//         leaf's Gauss points; Hermitian half, mirrored),
//   CO += sum_q w_q V_q N_a N^O_j                 (one column j at a time, staged z, y, x),
//   OO += sum_q w_q V_q conj(N^O_i) N^O_j          (pairs i <= j, mirrored),
// all in arithmetic V; then CO0, OO0 are added once per cell. One CTA per item (a cell's leaf
// range); slot >= 0 writes a partial summed afterwards in a fixed order.
template <typename V>
__global__ void __launch_bounds__(BT) k_build_oefe(OefeArgs A) {
  using Acc = typename AccOf<V>::type;
  extern __shared__ double smem_raw[];
  V* smem = reinterpret_cast<V*>(smem_raw);
  const BuildItem it = A.items[blockIdx.x];
  const int b = it.b, e = A.e0 + b;
  const int P = A.P, nloc = A.nloc, npad = A.npad;
  const int ne = A.act_off[e + 1] - A.act_off[e];
  const double* box = A.cellbox + 6 * e;
  const double kk = A.k[0] * A.k[0] + A.k[1] * A.k[1] + A.k[2] * A.k[2];
  const bool kz = kk == 0.0;

  __shared__ double xn[MAXP];
  __shared__ double Ld[3][MAXN1][MAXP], Dd[3][MAXN1][MAXP], w1[3][MAXN1];
  __shared__ V Lt[3][MAXN1][MAXP];                 // 1D Lagrange values at the leaf's points
  __shared__ V LL[3][MAXN1][MAXP * MAXP];          // products L[i][a] L[i][a2]
  __shared__ V Mm[3][MAXP][MAXP], Gr[3][MAXP][MAXP], Gi[3][MAXP][MAXP];   // M, K/2, -(k/2) A
  if (threadIdx.x < P) xn[threadIdx.x] = A.gll[threadIdx.x];

  // The item's first leaf writes every entry the store reads (CC, CO, OO; OC is CO^+), later leaves
  // add to them; the padding is never read.
  VC<V>* HE = reinterpret_cast<VC<V>*>(it.slot < 0 ? A.HE : A.HP) +
              (size_t)(it.slot < 0 ? b : it.slot) * npad * npad;

  for (int li = it.l0; li < it.l1; ++li) {
    const Leaf L = A.leaves[li];
    const int n1 = L.n1, n2 = n1 * n1, n3 = n2 * n1;
    const int64_t q0 = L.q0;
    const bool fst = li == it.l0;
    auto put = [&](VC<V>* h, V re, V im) {
      if (fst) *h = VC<V>{re, im};
      else vc_add(h, re, im);
    };
    if (threadIdx.x < 3 * n1) {
      const int d = threadIdx.x / n1, i = threadIdx.x % n1;
      const int64_t qi = q0 + (d == 0 ? i : d == 1 ? i * n1 : i * n2);
      const double xi = 2.0 * (A.qxyz[3 * qi + d] - box[d]) / box[3 + d] - 1.0;
      double Lv[MAXP], Dv[MAXP];
      lagrange_eval(xn, P, xi, Lv, Dv);
      for (int a = 0; a < P; ++a) {
        Ld[d][i][a] = Lv[a];
        Dd[d][i][a] = Dv[a] * (2.0 / box[3 + d]);
        Lt[d][i][a] = v_from<V>(Lv[a]);
      }
      for (int a = 0; a < P; ++a)
        for (int a2 = 0; a2 < P; ++a2) LL[d][i][a * P + a2] = v_from<V>(Lv[a] * Lv[a2]);
      w1[d][i] = A.gauss_w[n1 * 12 + i] * (L.hi[d] - L.lo[d]) / 2.0;
    }
    __syncthreads();
    // 1D mass, stiffness and antisymmetric gradient matrices of the leaf (FP64, then V)
    for (int t = threadIdx.x; t < 3 * P * P; t += BT) {
      const int d = t / (P * P), a = (t / P) % P, a2 = t % P;
      double m = 0, kq = 0, g1 = 0, g2 = 0;
      for (int i = 0; i < n1; ++i) {
        m = fma(w1[d][i] * Ld[d][i][a], Ld[d][i][a2], m);
        kq = fma(w1[d][i] * Dd[d][i][a], Dd[d][i][a2], kq);
        g1 = fma(w1[d][i] * Ld[d][i][a], Dd[d][i][a2], g1);
        g2 = fma(w1[d][i] * Dd[d][i][a], Ld[d][i][a2], g2);
      }
      Mm[d][a][a2] = v_from<V>(m);
      Gr[d][a][a2] = v_from<V>(0.5 * kq);
      Gi[d][a][a2] = v_from<V>(-0.5 * A.k[d] * (g1 - g2));
    }
    // ---- CC: potential weights W_q = w_q (V_q + |k|^2 / 2). The V term is symmetric in each of
    //      (a,a'), (b,b'), (c,c') separately, so the partial sums keep the symmetric pairs only
    //      (PS = P (P + 1) / 2 of them): T1[(qx,qy)][c<=c'], T2[qx][b<=b'][c<=c']
    const int P2 = P * P, PS = P * (P + 1) / 2;
    V* Wv = smem;                            // n3
    V* T1 = Wv + n3;                         // n2 * PS
    V* T2 = T1 + n2 * PS;                    // cx * PS * PS
    for (int q = threadIdx.x; q < n3; q += BT) Wv[q] = v_from<V>(A.qw[q0 + q] * (A.veff[q0 + q] + 0.5 * kk));
    __syncthreads();
    for (int t = threadIdx.x; t < n2 * PS; t += BT) {
      const int qxy = t / PS, cs = t % PS;
      const int c = sym_hi(cs), c2 = cs - c * (c + 1) / 2;   // c2 <= c
      T1[t] = v_dot<V>(n1, [&](int qz) { return Wv[qxy + n2 * qz]; }, [&](int qz) { return LL[2][qz][c * P + c2]; });
    }
    __syncthreads();
    const int budget = (int)((A.smem / sizeof(V) - n3 - (size_t)n2 * PS) / (PS * PS));
    const int cx = min(n1, max(1, budget));
    for (int qx0 = 0; qx0 < n1; qx0 += cx) {
      const int nx = min(cx, n1 - qx0);
      for (int t = threadIdx.x; t < nx * PS * PS; t += BT) {
        const int ix = t / (PS * PS), r = t % (PS * PS);
        const int bs = r / PS, cs = r % PS;
        const int bb = sym_hi(bs), b2 = bs - bb * (bb + 1) / 2;
        T2[t] = v_dot<V>(n1, [&](int qy) { return LL[1][qy][bb * P + b2]; },
                         [&](int qy) { return T1[((qx0 + ix) + n1 * qy) * PS + cs]; });
      }
      __syncthreads();
      const bool first = qx0 == 0;
      for (int t = threadIdx.x; t < nloc * nloc; t += BT) {
        const int m = t / nloc, n = t % nloc;
        if (m > n) continue;
        const int a = m % P, bb = (m / P) % P, c = m / P2;
        const int a2 = n % P, b2 = (n / P) % P, c2 = n / P2;
        const int ridx = sym_idx(bb, b2) * PS + sym_idx(c, c2);
        Acc vr = v_zero<V>();
        for (int ix = 0; ix < nx; ++ix) v_mac(vr, LL[0][qx0 + ix][a * P + a2], T2[ix * PS * PS + ridx]);
        V re = v_fin(vr), im = v_from<V>(0.0);
        if (first) {
          // kinetic: sum_d G_d in position d, M elsewhere (real part K/2, imaginary -(k/2) A)
          const V m0 = Mm[0][a][a2], m1 = Mm[1][bb][b2], m2 = Mm[2][c][c2];
          const V m12 = v_mul(m1, m2), m02 = v_mul(m0, m2), m01 = v_mul(m0, m1);
          Acc kr = v_zero<V>();
          v_mac(kr, Gr[0][a][a2], m12);
          v_mac(kr, Gr[1][bb][b2], m02);
          v_mac(kr, Gr[2][c][c2], m01);
          re = v_add(re, v_fin(kr));
          if (!kz) {
            Acc ki = v_zero<V>();
            v_mac(ki, Gi[0][a][a2], m12);
            v_mac(ki, Gi[1][bb][b2], m02);
            v_mac(ki, Gi[2][c][c2], m01);
            im = v_fin(ki);
          }
        }
        if (fst && first) {
          HE[(size_t)m * npad + n] = VC<V>{re, im};
          if (m != n) HE[(size_t)n * npad + m] = VC<V>{re, v_neg(im)};
        } else {
          vc_add(HE + (size_t)m * npad + n, re, im);
          if (m != n) vc_add(HE + (size_t)n * npad + m, re, v_neg(im));
        }
      }
      __syncthreads();
    }

    // ---- CO: column j of the V term, F_q = w_q V_q N^O_j(x_q), staged z, y, x. The weights w_q V_q
    //      of the leaf sit at the end of the shared memory (the CC stage is done with it) for CO and OO
    const size_t blk = (size_t)q0 * A.ne_max;
    V* WVs = smem + A.smem / sizeof(V) - n3;
    for (int q = threadIdx.x; q < n3; q += BT) WVs[q] = v_from<V>(A.qw[q0 + q] * A.veff[q0 + q]);
    __syncthreads();
    {
      VC<V>* F = reinterpret_cast<VC<V>*>(smem);    // n3
      VC<V>* G = F + n3;                            // n2 * P
      VC<V>* H = G + n2 * P;                        // n1 * P * P
      for (int j = 0; j < ne; ++j) {
        for (int q = threadIdx.x; q < n3; q += BT) {
          const V w = WVs[q];
          const VC<V> nv = load_no<V>(A, blk + (size_t)j * n3 + q);
          F[q] = VC<V>{v_mul(w, nv.re), v_mul(w, nv.im)};
        }
        __syncthreads();
        for (int t = threadIdx.x; t < n2 * P; t += BT) {     // z: (qx,qy,c)
          const int qxy = t / P, c = t % P;
          Acc gr = v_zero<V>(), gi = v_zero<V>();
          for (int qz = 0; qz < n1; ++qz) {
            const VC<V> f = F[qxy + n2 * qz];
            v_mac(gr, Lt[2][qz][c], f.re);
            v_mac(gi, Lt[2][qz][c], f.im);
          }
          G[t] = VC<V>{v_fin(gr), v_fin(gi)};
        }
        __syncthreads();
        for (int t = threadIdx.x; t < n1 * P * P; t += BT) {  // y: (qx,b,c)
          const int qx = t / (P * P), bb = (t / P) % P, c = t % P;
          Acc hr = v_zero<V>(), hi = v_zero<V>();
          for (int qy = 0; qy < n1; ++qy) {
            const VC<V> g = G[(qx + n1 * qy) * P + c];
            v_mac(hr, Lt[1][qy][bb], g.re);
            v_mac(hi, Lt[1][qy][bb], g.im);
          }
          H[t] = VC<V>{v_fin(hr), v_fin(hi)};
        }
        __syncthreads();
        for (int m = threadIdx.x; m < nloc; m += BT) {       // x: node a + P (b + P c)
          const int a = m % P, bc = m / P;
          const int bb = bc % P, c = bc / P;
          Acc sr = v_zero<V>(), si = v_zero<V>();
          for (int qx = 0; qx < n1; ++qx) {
            const VC<V> h = H[(qx * P + bb) * P + c];
            v_mac(sr, Lt[0][qx][a], h.re);
            v_mac(si, Lt[0][qx][a], h.im);
          }
          put(HE + (size_t)m * npad + nloc + j, v_fin(sr), v_fin(si));
        }
        __syncthreads();
      }
    }

    // ---- OO: pairs (i <= j) over the leaf points in chunks, with w V N^O_i staged beside N^O_i
    {
      const int QC = max(1, min(32, (int)((A.smem - (size_t)n3 * sizeof(V) - 64) / ((size_t)max(ne, 1) * 2 * sizeof(VC<V>)))));
      VC<V>* Ns = reinterpret_cast<VC<V>*>(smem);   // QC x ne
      VC<V>* Nw = Ns + (size_t)QC * ne;             // QC x ne: w V N
      const int npairs = ne * (ne + 1) / 2;
      for (int pb = 0; pb < npairs; pb += 2 * BT) {
        int pi[2], pj[2];
        Acc ar[2], ai[2];
        for (int u = 0; u < 2; ++u) {
          ar[u] = ai[u] = v_zero<V>();
          const int pp = pb + threadIdx.x + u * BT;
          pi[u] = -1;
          pj[u] = -1;
          if (pp < npairs) {  // pair index -> (i, j), i <= j
            int i = 0, rem = pp;
            while (rem >= ne - i) { rem -= ne - i; ++i; }
            pi[u] = i;
            pj[u] = i + rem;
          }
        }
        for (int qc = 0; qc < n3; qc += QC) {
          const int nq = min(QC, n3 - qc);
          __syncthreads();
          for (int t = threadIdx.x; t < nq * ne; t += BT) {
            const int q = t / ne, j = t % ne;
            const VC<V> nv = load_no<V>(A, blk + (size_t)j * n3 + qc + q);
            const V w = WVs[qc + q];
            Ns[t] = nv;
            Nw[t] = VC<V>{v_mul(w, nv.re), v_mul(w, nv.im)};
          }
          __syncthreads();
          for (int u = 0; u < 2; ++u) {
            if (pi[u] < 0) continue;
            const int i = pi[u], j = pj[u];
            for (int q = 0; q < nq; ++q) {   // conj(w N_i) N_j
              const VC<V> x = Nw[q * ne + i], y = Ns[q * ne + j];
              v_mac(ar[u], x.re, y.re);
              v_mac(ar[u], x.im, y.im);
              v_mac(ai[u], x.re, y.im);
              v_mac(ai[u], v_neg(x.im), y.re);
            }
          }
        }
        for (int u = 0; u < 2; ++u) {
          if (pi[u] < 0) continue;
          const int i = pi[u], j = pj[u];
          const V re = v_fin(ar[u]), im = v_fin(ai[u]);
          put(HE + (size_t)(nloc + i) * npad + nloc + j, re, im);
          if (i != j) put(HE + (size_t)(nloc + j) * npad + nloc + i, re, v_neg(im));
        }
      }
      __syncthreads();
    }
  }
  if (it.slot < 0) {
    // the cached V-independent OEFE blocks CO0, OO0
    const size_t e0s = (size_t)nloc * A.ne_max + (size_t)A.ne_max * A.ne_max;
    const cd* CO0 = A.E0 + (size_t)e * e0s;
    const cd* OO0 = CO0 + (size_t)nloc * A.ne_max;
    for (int t = threadIdx.x; t < nloc * ne; t += BT) {
      const int m = t / ne, j = t % ne;
      const cd v = CO0[(size_t)m * A.ne_max + j];
      vc_add(HE + (size_t)m * npad + nloc + j, v_from<V>(v.x), v_from<V>(v.y));
    }
    for (int t = threadIdx.x; t < ne * ne; t += BT) {
      const int i = t / ne, j = t % ne;
      const cd v = OO0[i * A.ne_max + j];
      vc_add(HE + (size_t)(nloc + i) * npad + nloc + j, v_from<V>(v.x), v_from<V>(v.y));
    }
  }
}

// Gamma_e[a][j] = c_{act(e)_j, node(e,a)} = (sum over cells sharing the node of d) / m_node
template <typename S>
__global__ void k_gamma(const int* cell_nodes, const int64_t* node_off, const int64_t* node_slot,
                        const int* act_off, const int* act_idx, const double* m, const cd* dblk,
                        int ncells, int nloc, int npad, int ne_max, S* gamma) {
  const int64_t total = (int64_t)ncells * nloc * ne_max;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % ne_max);
    const int64_t ea = t / ne_max;
    const int a = (int)(ea % nloc), e = (int)(ea / nloc);
    const int ne = act_off[e + 1] - act_off[e];
    cd s = mkc(0, 0);
    if (j < ne) {
      const int nu = act_idx[act_off[e] + j];
      const int g = cell_nodes[(size_t)e * nloc + a];
      for (int64_t sl = node_off[g]; sl < node_off[g + 1]; ++sl) {
        const int64_t slot = node_slot[sl];
        const int e2 = (int)(slot / npad), a2 = (int)(slot % npad);
        int lo = act_off[e2], hi = act_off[e2 + 1] - 1;  // binary search nu in act(e2)
        while (lo <= hi) {
          const int mid = (lo + hi) / 2;
          const int v = act_idx[mid];
          if (v == nu) {
            s += dblk[((size_t)e2 * nloc + a2) * ne_max + (mid - act_off[e2])];
            break;
          }
          if (v < nu) lo = mid + 1; else hi = mid - 1;
        }
      }
      s = (1.0 / m[g]) * s;
    }
    if constexpr (sizeof(S) == sizeof(cd)) gamma[t] = *reinterpret_cast<S*>(&s);
    else gamma[t] = s.x;
  }
}

template <typename S>
__device__ inline cd ld_s(const S* p, size_t i) {
  if constexpr (sizeof(S) == sizeof(cd)) { const cd* q = reinterpret_cast<const cd*>(p); return q[i]; }
  else return mkc(reinterpret_cast<const double*>(p)[i], 0.0);
}

// subtract sum over owned nodes m_l conj(c_i) c_j from the cell's M^AA block (Eq. Moo)
template <typename S>
__global__ void k_moo_cell(const int* act_off, const double* m, const int* cell_nodes, const S* gamma,
                           int P, int nloc, int ne_max, cd* MAAblk) {
  const int e = blockIdx.x;
  const int ne = act_off[e + 1] - act_off[e];
  const int p = P - 1;
  for (int t = threadIdx.x; t < ne * ne; t += blockDim.x) {
    const int i = t / ne, j = t % ne;
    cd s = mkc(0, 0);
    for (int a = 0; a < nloc; ++a) {
      const int ax = a % P, ay = (a / P) % P, az = a / (P * P);
      if (ax == p || ay == p || az == p) continue;  // each node owned by one cell
      const double mm = m[cell_nodes[(size_t)e * nloc + a]];
      const size_t base = ((size_t)e * nloc + a) * ne_max;
      s += mm * cmulc(ld_s(gamma, base + i), ld_s(gamma, base + j));
    }
    MAAblk[((size_t)e * ne_max + i) * ne_max + j] -= s;
  }
}

// M^oo[nu][mu] = sum over cells holding both of the per-cell blocks
template <typename S>
__global__ void k_moo_reduce(const int64_t* enr_off, const int64_t* enr_slot, const int* act_off,
                             const int* act_idx, int nO, int npad, int nloc, int ne_max,
                             const cd* MAAblk, S* Moo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nO * nO) return;
  const int nu = t / nO, mu = t % nO;
  cd s = mkc(0, 0);
  for (int64_t sl = enr_off[nu]; sl < enr_off[nu + 1]; ++sl) {
    const int64_t slot = enr_slot[sl];
    const int e = (int)(slot / npad), i = (int)(slot % npad) - nloc;
    int lo = act_off[e], hi = act_off[e + 1] - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) / 2;
      const int v = act_idx[mid];
      if (v == mu) {
        s += MAAblk[((size_t)e * ne_max + i) * ne_max + (mid - act_off[e])];
        break;
      }
      if (v < mu) lo = mid + 1; else hi = mid - 1;
    }
  }
  if constexpr (sizeof(S) == sizeof(cd)) reinterpret_cast<cd*>(Moo)[t] = s;
  else reinterpret_cast<double*>(Moo)[t] = s.x;
}

template <typename S>
__global__ void k_hermitize(S* A, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  if (i > j) return;
  if constexpr (sizeof(S) == sizeof(cd)) {
    cd* B = reinterpret_cast<cd*>(A);
    cd u = B[i * n + j], l = B[j * n + i];
    cd v = 0.5 * (u + cconj(l));
    B[i * n + j] = v;
    B[j * n + i] = cconj(v);
  } else {
    double* B = reinterpret_cast<double*>(A);
    double v = 0.5 * (B[i * n + j] + B[j * n + i]);
    B[i * n + j] = v;
    B[j * n + i] = v;
  }
}

// Where a finished OEFE cell matrix goes: the FP64 / FP32 / FP32-pair / bf16-split copies, or (the
// setup pass of the V-independent part) only its CO and OO blocks into the per-cell cache E0
// (CO: nloc x ne_max, then OO: ne_max x ne_max).
struct StoreOut {
  void* H64;
  void* H32;
  __nv_bfloat16* Hbf;
  float* Hp;
  int parts, nloc, npad, ne_max;
  cd* E0;
  // compact layout of H64 / Hp (KData::compact): cell -> dense-list position or sum-factorization
  // row, and where the strips start
  const int* dense_index;
  const int* sf_index;
  long long sf_base, strip;
  int compact;
};

// v in FP64 and as FP32 pairs (pr, pi): the pair copy and the bf16 splits are taken from the pairs
template <typename S>
__device__ inline void store_entry2(const StoreOut& O, int e, int ne, int r, int c, cd v, f2 pr, f2 pi) {
  const int nloc = O.nloc, npad = O.npad;
  if (O.E0) {
    if (c < nloc || c >= nloc + ne || r >= nloc + ne) return;
    cd* co = O.E0 + (size_t)e * ((size_t)nloc * O.ne_max + (size_t)O.ne_max * O.ne_max);
    if (r < nloc) co[(size_t)r * O.ne_max + (c - nloc)] = v;
    else co[(size_t)nloc * O.ne_max + (size_t)(r - nloc) * O.ne_max + (c - nloc)] = v;
    return;
  }
  const size_t o = (size_t)e * npad * npad + (size_t)r * npad + c;
  // H64 / Hp offset: the full layout, or the compact one (the CFE-CFE block of single-leaf cells and
  // rows beyond the enrichment strip are not kept)
  long long oc = (long long)o;
  if (O.compact) {
    const int d = O.dense_index[e];
    if (d >= 0) {
      oc = ((long long)d * npad + r) * npad + c;
    } else {
      const long long b = O.sf_base + (long long)O.sf_index[e] * O.strip;
      if (r < nloc) oc = (c >= nloc && c < nloc + O.ne_max) ? b + (long long)r * O.ne_max + (c - nloc) : -1;
      else oc = r < nloc + O.ne_max ? b + (long long)nloc * O.ne_max + (long long)(r - nloc) * npad + c : -1;
    }
  }
  if constexpr (sizeof(S) == sizeof(cd)) {
    if (O.H64 && oc >= 0) reinterpret_cast<cd*>(O.H64)[oc] = v;
    if (O.H32) reinterpret_cast<cf*>(O.H32)[o] = cf{(float)v.x, (float)v.y};
    if (O.Hp && oc >= 0) reinterpret_cast<float4*>(O.Hp)[oc] = make_float4(pr.h, pr.l, pi.h, pi.l);
  } else {
    if (O.H64 && oc >= 0) reinterpret_cast<double*>(O.H64)[oc] = v.x;
    if (O.H32) reinterpret_cast<float*>(O.H32)[o] = (float)v.x;
    if (O.Hp && oc >= 0) reinterpret_cast<float2*>(O.Hp)[oc] = make_float2(pr.h, pr.l);
  }
  if (O.Hbf) {
    // tile-contiguous: per cell [K tile of 64 columns][M tile of 128 rows][plane][128][64], so that
    // the planes of one part of one (K tile, M tile) are one contiguous block for the TMA loads;
    // planes: (re hi, re lo[, im hi, im lo]) split from the FP32 value, or (re hi, re mid, re lo
    // [, im hi, im mid, im lo]) from the FP32 pair x = h + l: each residual h - bf16(h) is exact in
    // FP32 and the low part joins the second residual (rounding 2^-24 of it, far below the split)
    const int parts = O.parts;
    const int nq = sizeof(S) == sizeof(cd) ? 2 : 1;
    const int PL = nq * parts;
    const size_t pl = 128 * 64;
    const int mtn = npad >> 7;
    const size_t base = (size_t)e * PL * npad * npad +
                        ((((size_t)(c >> 6) * mtn + (r >> 7)) * PL) * 128 + (r & 127)) * 64 + (c & 63);
    for (int q = 0; q < nq; ++q) {
      __nv_bfloat16* ob = O.Hbf + base + (size_t)q * parts * pl;
      const double x = q == 0 ? v.x : v.y;
      if (parts == 2) {
        const float xf = (float)x;
        const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
        ob[0] = hi;
        ob[pl] = __float2bfloat16_rn(xf - __bfloat162float(hi));
      } else {
        const float h = q == 0 ? pr.h : pi.h, l = q == 0 ? pr.l : pi.l;
        const __nv_bfloat16 b1 = __float2bfloat16_rn(h);
        const float r1 = __fadd_rn(__fsub_rn(h, __bfloat162float(b1)), l);
        const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 b3 = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(b2)));
        ob[0] = b1;
        ob[pl] = b2;
        ob[2 * pl] = b3;
      }
    }
  }
}

template <typename S>
__device__ inline void store_entry(const StoreOut& O, int e, int ne, int r, int c, cd v) {
  const bool need = O.Hp || (O.Hbf && O.parts == 3);
  store_entry2<S>(O, e, ne, r, c, v, need ? f2_from(v.x) : f2{0.0f, 0.0f}, need ? f2_from(v.y) : f2{0.0f, 0.0f});
}

// The finished cell matrices of a batch (k_build_oefe: CC, CO and OO in HE, OC = CO^+) into the
// stored copies; one CTA per cell. HE in arithmetic V: FP64 (cd) or FP32 pairs.
template <typename S, typename V>
__global__ void k_finish(const void* HEb, const int* act_off, int e0, StoreOut O) {
  const int b = blockIdx.x, e = e0 + b;
  const int ne = act_off[e + 1] - act_off[e];
  const int nloc = O.nloc, npad = O.npad, naug = nloc + ne;
  const VC<V>* HE = reinterpret_cast<const VC<V>*>(HEb) + (size_t)b * npad * npad;
  for (int t = threadIdx.x; t < npad * npad; t += blockDim.x) {
    const int r = t / npad, c = t % npad;
    VC<V> v{v_from<V>(0.0), v_from<V>(0.0)};
    if (r < naug && c < naug) {
      if (r >= nloc && c < nloc) {
        v = HE[(size_t)c * npad + r];
        v.im = v_neg(v.im);
      } else {
        v = HE[t];
      }
    }
    if constexpr (std::is_same<V, double>::value) store_entry<S>(O, e, ne, r, c, mkc(v.re, v.im));
    else store_entry2<S>(O, e, ne, r, c, mkc(f2_to(v.re), f2_to(v.im)), v.re, v.im);
  }
}

struct TransformSf {   // sum-factorized H_CC Gamma on single-leaf cells (null sf: dense everywhere)
  const double* sf;
  const int* sf_index;  // cell -> row of sf, or -1
  const double* qw;
  const double* veff;
  const int64_t* q_off;
  double k[3];
  int P, nbuf;
};

// H^O_e = T_e^+ H_e T_e: CO = CA - H_CC Gamma, OO = AA - Gamma^+ CO - CA^+ Gamma.
// One CTA per cell; writes the FP64 and/or FP32 stored matrices.
template <typename S>
__global__ void __launch_bounds__(TT, 1) k_transform(const cd* HEb, const S* gamma, const int* act_off,
                                                  int e0, int nloc, int npad, int ne_max, StoreOut O,
                                                  TransformSf T) {
  extern __shared__ double smem[];
  const int b = blockIdx.x, e = e0 + b;
  const int ne = act_off[e + 1] - act_off[e];
  const cd* HE = HEb + (size_t)b * npad * npad;
  const S* Gm = gamma + (size_t)e * nloc * ne_max;
  cd* CO = reinterpret_cast<cd*>(smem);          // nloc * TJB
  constexpr int JB = TJB;
  auto put = [&](int r, int c, cd v) { store_entry<S>(O, e, ne, r, c, v); };
  // CC block and zero padding
  for (int t = threadIdx.x; t < npad * npad; t += TT) {
    const int r = t / npad, c = t % npad;
    if (r < nloc && c < nloc) put(r, c, HE[(size_t)r * npad + c]);
    else if (r >= nloc + ne || c >= nloc + ne) put(r, c, mkc(0, 0));
  }
  const int sfi = T.sf ? T.sf_index[e] : -1;
  if (sfi >= 0) {
    // single-leaf cell: H_CC Gamma by sum factorization, four columns at a time
    constexpr bool CPLX = sizeof(S) == sizeof(cd);
    constexpr int NB4 = 4, R = CPLX ? 2 : 1, J = NB4 * R;
    const int P3 = T.P * T.P * T.P;
    double* tab = smem;
    double* Gr = tab + SF_STRIDE;
    double* Gi = Gr + 3 * SF_MAXP * SF_MAXP;
    double* Ws = Gi + 3 * SF_MAXP * SF_MAXP;
    double* Xs = Ws + T.nbuf;                  // P3 * J
    double* Ys = Xs + (size_t)P3 * J;          // P3 * J
    double* Ab = Ys + (size_t)P3 * J;          // nbuf * J
    double* Bb = Ab + (size_t)T.nbuf * J;      // nbuf * J
    cd* C4 = reinterpret_cast<cd*>(Bb + (size_t)T.nbuf * J);   // nloc * NB4
    sf_prepare(T.sf + (size_t)sfi * SF_STRIDE, tab, Gr, Gi, Ws, T.qw, T.veff, T.q_off[e], T.k);
    for (int j0 = 0; j0 < ne; j0 += NB4) {
      const int nj = min(NB4, ne - j0);
      for (int t = threadIdx.x; t < P3 * NB4; t += TT) {
        const int m = t / NB4, u = t % NB4;
        const cd g = u < nj ? ld_s(Gm, (size_t)m * ne_max + j0 + u) : mkc(0, 0);
        Xs[(size_t)m * J + u * R] = g.x;
        if (CPLX) Xs[(size_t)m * J + u * R + 1] = g.y;
      }
      for (int t = threadIdx.x; t < P3 * J; t += TT) Ys[t] = 0.0;
      __syncthreads();
      sf_cc<double, CPLX, NB4>(tab, Gr, Gi, Ws, T.P, Xs, Ys, Ab, Bb);
      for (int t = threadIdx.x; t < nloc * NB4; t += TT) {
        const int m = t / NB4, u = t % NB4;
        if (u < nj) {
          const cd hg = mkc(Ys[(size_t)m * J + u * R], CPLX ? Ys[(size_t)m * J + u * R + 1] : 0.0);
          const cd co = HE[(size_t)m * npad + nloc + j0 + u] - hg;
          C4[t] = co;
          put(m, nloc + j0 + u, co);
          put(nloc + j0 + u, m, cconj(co));
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < ne * nj; t += TT) {   // OO is Hermitian: i <= j, mirrored
        const int i = t / nj, u = t % nj, j = j0 + u;
        if (i > j) continue;
        cd s = HE[(size_t)(nloc + i) * npad + nloc + j];
        for (int m = 0; m < nloc; ++m) {
          s = cfmac(-ld_s(Gm, (size_t)m * ne_max + i), C4[m * NB4 + u], s);
          s = cfmac(-HE[(size_t)m * npad + nloc + i], ld_s(Gm, (size_t)m * ne_max + j), s);
        }
        put(nloc + i, nloc + j, s);
        if (i != j) put(nloc + j, nloc + i, cconj(s));
      }
      __syncthreads();
    }
    return;
  }
  cd* Gs = CO + (size_t)nloc * JB;               // Gamma[:, j0:j0+JB], nloc * JB
  for (int j0 = 0; j0 < ne; j0 += JB) {
    const int nj = min(JB, ne - j0);
    for (int t = threadIdx.x; t < nloc * JB; t += TT) {
      const int a = t / JB, u = t % JB;
      Gs[t] = u < nj ? ld_s(Gm, (size_t)a * ne_max + j0 + u) : mkc(0, 0);
    }
    __syncthreads();
    // CO[:, j0:j0+nj] = CA - H_CC Gamma, using H_CC Hermitian: (H_CC Gamma)[m] = sum_a conj(H[a][m]) Gamma[a];
    // one local node per thread, JB columns in registers
    for (int m = threadIdx.x; m < nloc; m += TT) {
      cd acc[JB];
#pragma unroll
      for (int u = 0; u < JB; ++u) acc[u] = mkc(0, 0);
      for (int a = 0; a < nloc; ++a) {
        const cd h = cconj(HE[(size_t)a * npad + m]);
        const cd* g = Gs + a * JB;
#pragma unroll
        for (int u = 0; u < JB; ++u) acc[u] = cfma(h, g[u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < JB; ++u) {
        if (u < nj) {
          const cd co = HE[(size_t)m * npad + nloc + j0 + u] - acc[u];
          CO[m * JB + u] = co;
          put(m, nloc + j0 + u, co);
          put(nloc + j0 + u, m, cconj(co));
        }
      }
    }
    __syncthreads();
    // OO[i][j] = AA[i][j] - sum_m conj(Gamma[m][i]) CO[m][j] - sum_m conj(CA[m][i]) Gamma[m][j];
    // OO is Hermitian: i <= j, mirrored
    for (int t = threadIdx.x; t < ne * nj; t += TT) {
      const int i = t / nj, u = t % nj, j = j0 + u;
      if (i > j) continue;
      cd s = HE[(size_t)(nloc + i) * npad + nloc + j];
      for (int m = 0; m < nloc; ++m) {
        s = cfmac(-ld_s(Gm, (size_t)m * ne_max + i), CO[m * JB + u], s);
        s = cfmac(-HE[(size_t)m * npad + nloc + i], Gs[m * JB + u], s);
      }
      put(nloc + i, nloc + j, s);
      if (i != j) put(nloc + j, nloc + i, cconj(s));
    }
    __syncthreads();
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
static int gauss_table(oefe_ctx* c, double** d_tab) {
  std::vector<double> tab(13 * 12, 0.0);
  for (int n = 1; n <= 12; ++n) {
    std::vector<double> x, w;
    gauss_rule(n, x, w);
    for (int i = 0; i < n; ++i) tab[n * 12 + i] = w[i];
  }
  OEFE_TRY(dev_alloc(c, (void**)d_tab, tab.size() * sizeof(double)));
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(*d_tab, tab.data(), tab.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
  return OEFE_OK;
}

static size_t smem_build_bytes(const oefe_ctx* c, int mode) {
  // worst case over the phases, all leaves use n1 <= max(nq_cell, nq_enr)
  const int n1 = std::max(c->nq_cell, c->nq_enr), P = c->P;
  const size_t n3 = (size_t)n1 * n1 * n1, n2 = (size_t)n1 * n1;
  const size_t cap = mode == 1 ? SMEM_SETUP : SMEM_BUILD;
  // the CC stage keeps at least one x-slab of P^4 partial sums
  const size_t cc_min = (n3 + n2 * P * P + (size_t)P * P * P * P) * 8;
  const size_t phase_cc = mode == 1 ? 0 : std::max(cc_min, std::min(cap, (n3 + n2 * P * P + (size_t)n1 * P * P * P * P) * 8));
  const size_t phase_ca = mode == 1 ? (5 * n3 + 4 * n2 * P + 3 * (size_t)n1 * P * P) * 16
                                    : (n3 + n2 * P + (size_t)n1 * P * P) * 16;
  const size_t phase_aa = 32 * (size_t)std::max(c->ne_max, 1) * 4 * 16 + 32 * 8;
  return std::max(std::max(phase_cc, phase_ca), phase_aa);
}

// Dynamic shared memory of k_build_oefe: the largest phase, capped so that two CTAs share an SM
// (the CC stage then takes its partial sums in chunks of qx)
static size_t smem_oefe_bytes(const oefe_ctx* c) {
  const int n1 = std::max(c->nq_cell, c->nq_enr), P = c->P, PS = P * (P + 1) / 2;
  const size_t n3 = (size_t)n1 * n1 * n1, n2 = (size_t)n1 * n1;
  const size_t cc_min = (n3 + n2 * PS + (size_t)PS * PS) * 8;
  const size_t cc = (n3 + n2 * PS + (size_t)n1 * PS * PS) * 8;
  const size_t co = (n3 + n2 * P + (size_t)n1 * P * P) * 16;
  const size_t oo = 32 * (size_t)std::max(c->ne_max, 1) * 2 * 16 + 64;
  const size_t cap = 82 * 1024;
  return std::max({cc_min, std::min(cap, cc), co, oo});
}

// Process cells in batches bounded by a scratch budget; calls fn(e0, e1, tab_off_host).
template <typename Fn>
static int for_cell_batches(oefe_ctx* c, size_t per_cell_fixed, size_t budget, bool with_tab, Fn fn) {
  int e0 = 0;
  while (e0 < c->ncells) {
    std::vector<int64_t> off(1, 0);
    size_t bytes = 0;
    int e1 = e0;
    while (e1 < c->ncells) {
      const int64_t ne = c->act_off[e1 + 1] - c->act_off[e1];
      const int64_t ent = (c->q_off[e1 + 1] - c->q_off[e1]) * ne;
      const size_t add = (with_tab ? (size_t)ent * 4 * sizeof(cd) : 0) + per_cell_fixed;
      if (e1 > e0 && bytes + add > budget) break;
      bytes += add;
      off.push_back(off.back() + ent);
      ++e1;
    }
    OEFE_TRY(fn(e0, e1, off));
    e0 = e1;
  }
  return OEFE_OK;
}

static EnrParams enr_params(const oefe_ctx* c) {
  EnrParams E;
  E.pos = c->d_pos;
  E.lm = c->d_lm;
  E.R = c->d_R;
  E.dR = c->d_dR;
  E.nfun = c->nfun;
  E.ngrid = c->ngrid;
  E.a = c->a;
  E.r0 = c->r0;
  E.rc = c->rc;
  return E;
}

// Sum the partial cell matrices of the split cells into their cell matrices, in slot order.
template <typename V>
__global__ void k_add_partials(void* HEv, const void* HPv, const int* red, int nred, int npad) {
  VC<V>* HE = reinterpret_cast<VC<V>*>(HEv);
  const VC<V>* HP = reinterpret_cast<const VC<V>*>(HPv);
  const int64_t n2 = (int64_t)npad * npad;
  for (int r = blockIdx.y; r < nred; r += gridDim.y) {
    const int b = red[3 * r], s0 = red[3 * r + 1], s1 = red[3 * r + 2];
    VC<V>* h = HE + (size_t)b * n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
      VC<V> s = h[t];
      for (int q = s0; q < s1; ++q) {
        const VC<V> x = HP[(size_t)q * n2 + t];
        s.re = v_add(s.re, x.re);
        s.im = v_add(s.im, x.im);
      }
      h[t] = s;
    }
  }
}

// Scratch budget of one batch of cells (tabulation + cell matrices + partials): a quarter of the
// free device memory, between 2 and 32 GB.
static size_t batch_budget() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return (size_t)6 << 30;
  return std::min<size_t>((size_t)32 << 30, std::max<size_t>((size_t)2 << 30, fr / 4));
}

// Run the cell kernel over all cells in batches (modes of k_build_cell): mode 1 and mode 0 tabulate
// the enrichment first, mode 2 reads N^O; mode 0 ends with the transform into the cache E0, mode 2
// with the store of the cell matrices. Where a cell matrix is formed the work is shared out as
// items of at most G leaves (cells refined toward a nucleus have tens of leaves, the others one),
// largest first, so that no cell's leaves serialize the launch.
static int run_cell_kernel(oefe_ctx* c, KData& K, int mode, const double* veff, double* d_gw, cd* dblk,
                           cd* MAAblk, int store) {
  const size_t n2b = (size_t)c->npad * c->npad * sizeof(cd);
  const bool vmode = mode != 1;
  const size_t hebytes = vmode ? n2b : 0;
  const bool pairs = mode == 2 && c->f64_products == OEFE_F64_PAIRS;
  const size_t smem = mode == 2 ? smem_oefe_bytes(c) : smem_build_bytes(c, mode);
  int per_sm = 0;
  if (mode == 2) {
    auto occ = [&](auto kern) -> int {
      OEFE_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      OEFE_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem));
      return OEFE_OK;
    };
    OEFE_TRY(pairs ? occ(k_build_oefe<f2>) : occ(k_build_oefe<double>));
  } else {
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_build_cell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    OEFE_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_cell, BT, smem));
  }
  const int resident = std::max(1, per_sm) * c->num_sms;
  return for_cell_batches(c, hebytes, batch_budget(), mode != 2, [&](int e0, int e1, const std::vector<int64_t>& off) -> int {
    const int nb = e1 - e0;
    // work items (build mode)
    std::vector<BuildItem> items;
    std::vector<int> red;  // (b, slot0, slot1) per split cell
    int nslot = 0;
    if (vmode) {
      long long leaves = 0;
      for (int e = e0; e < e1; ++e) leaves += c->leaf_off[e + 1] - c->leaf_off[e];
      const int G = (int)std::max<long long>(2, (leaves + 2 * resident - 1) / (2 * resident));
      for (int e = e0; e < e1; ++e) {
        const int l0 = c->leaf_off[e], l1 = c->leaf_off[e + 1];
        const int b = e - e0;
        items.push_back({b, l0, std::min(l1, l0 + G), -1});
        if (l1 - l0 > G) {
          const int s0 = nslot;
          for (int l = l0 + G; l < l1; l += G) items.push_back({b, l, std::min(l1, l + G), nslot++});
          red.insert(red.end(), {b, s0, nslot});
        }
      }
      std::stable_sort(items.begin(), items.end(),
                       [](const BuildItem& x, const BuildItem& y) { return x.l1 - x.l0 > y.l1 - y.l0; });
    }
    auto a256 = [](size_t x) { return ((x + 255) / 256) * 256; };
    const size_t tab_bytes = mode == 2 ? 0 : a256((size_t)off.back() * 4 * sizeof(cd));
    const size_t off_bytes = a256(off.size() * sizeof(int64_t));
    const size_t he_total = a256(hebytes * nb);
    const size_t hp_total = a256((size_t)nslot * n2b);
    const size_t it_bytes = a256(items.size() * sizeof(BuildItem));
    const size_t red_bytes = a256(red.size() * sizeof(int));
    OEFE_TRY(ensure_ws(c, tab_bytes + he_total + hp_total + off_bytes + it_bytes + red_bytes));
    char* base = (char*)c->ws;
    cd* tab = (cd*)base;
    cd* HE = (cd*)(base + tab_bytes);
    cd* HP = (cd*)(base + tab_bytes + he_total);
    int64_t* d_off = (int64_t*)(base + tab_bytes + he_total + hp_total);
    BuildItem* d_items = (BuildItem*)((char*)d_off + off_bytes);
    int* d_red = (int*)((char*)d_items + it_bytes);
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    if (!items.empty())
      OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(BuildItem), cudaMemcpyHostToDevice,
                                       c->stream));
    if (!red.empty())
      OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_red, red.data(), red.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (mode != 2 && off.back() > 0) {
      const int threads = 256;
      const int64_t blocks = std::min<int64_t>((off.back() / std::max(c->nfun, 1) + threads - 1) / threads, 1 << 20);
      OEFE_COUNTED k_tabulate<<<(unsigned)blocks, threads, 0, c->stream>>>(enr_params(c), c->d_qxyz, c->d_q_off, c->d_act_off,
                                                             c->d_act_idx, e0, nb, d_off, K.k[0], K.k[1], K.k[2], tab);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    }
    BuildArgs A;
    A.leaves = c->d_leaves;
    A.leaf_off = c->d_leaf_off;
    A.qxyz = c->d_qxyz;
    A.qw = c->d_qw;
    A.veff = veff;
    A.cellbox = c->d_cellbox;
    A.gll = c->d_gll;
    A.gauss_w = d_gw;
    A.act_off = c->d_act_off;
    A.tab_off = d_off;
    A.q_off = c->d_q_off;
    A.tab = tab;
    A.e0 = e0;
    A.P = c->P;
    A.nloc = c->nloc;
    A.npad = c->npad;
    A.ne_max = c->ne_max;
    for (int d = 0; d < 3; ++d) A.k[d] = K.k[d];
    A.mode = mode;
    A.HE = vmode ? HE : nullptr;
    A.dblk = dblk;
    A.MAAblk = MAAblk;
    A.E0 = (cd*)K.E0;
    A.items = vmode ? d_items : nullptr;
    A.HP = HP;
    A.smem = smem;
    const int grid = vmode ? (int)items.size() : nb;
    if (mode == 2) {
      OefeArgs B;
      B.leaves = c->d_leaves;
      B.leaf_off = c->d_leaf_off;
      B.qxyz = c->d_qxyz;
      B.qw = c->d_qw;
      B.veff = veff;
      B.cellbox = c->d_cellbox;
      B.gll = c->d_gll;
      B.gauss_w = d_gw;
      B.act_off = c->d_act_off;
      B.NO = pairs ? (const void*)K.NOp : (const void*)K.NO;
      B.no_cplx = K.cplx;
      B.e0 = e0;
      B.P = c->P;
      B.nloc = c->nloc;
      B.npad = c->npad;
      B.ne_max = c->ne_max;
      for (int d = 0; d < 3; ++d) B.k[d] = K.k[d];
      B.HE = HE;
      B.HP = HP;
      B.E0 = (const cd*)K.E0;
      B.items = d_items;
      B.smem = smem;
      if (pairs) OEFE_COUNTED k_build_oefe<f2><<<grid, BT, smem, c->stream>>>(B);
      else OEFE_COUNTED k_build_oefe<double><<<grid, BT, smem, c->stream>>>(B);
    } else {
      OEFE_COUNTED k_build_cell<<<grid, BT, smem, c->stream>>>(A);
    }
    OEFE_CUDA_TRY(c, cudaGetLastError());
    if (vmode && !red.empty()) {
      const int nred = (int)red.size() / 3;
      dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, ((int64_t)c->npad * c->npad + 255) / 256)),
             (unsigned)std::min(nred, 65535));
      if (pairs) OEFE_COUNTED k_add_partials<f2><<<g, 256, 0, c->stream>>>(HE, HP, d_red, nred, c->npad);
      else OEFE_COUNTED k_add_partials<double><<<g, 256, 0, c->stream>>>(HE, HP, d_red, nred, c->npad);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    }
    StoreOut O;
    O.H64 = (store & OEFE_STORE_F64) ? K.H64 : nullptr;
    O.H32 = (store & OEFE_STORE_F32) ? K.H32 : nullptr;
    O.Hbf = (store & (OEFE_STORE_BF16X3 | OEFE_STORE_BF16X6)) ? (__nv_bfloat16*)K.Hbf : nullptr;
    O.Hp = (store & OEFE_STORE_F64PAIR) ? K.Hp : nullptr;
    O.parts = K.bf_parts;
    O.nloc = c->nloc;
    O.npad = c->npad;
    O.ne_max = c->ne_max;
    O.E0 = nullptr;
    O.dense_index = c->d_dense_index;
    O.sf_index = c->d_sf_index;
    O.sf_base = (long long)c->n_dense * c->npad * c->npad;
    O.strip = (long long)compact_strip(c);
    O.compact = K.compact ? 1 : 0;
    if (mode == 2) {
      if (K.cplx && pairs) OEFE_COUNTED k_finish<cd, f2><<<nb, 256, 0, c->stream>>>(HE, c->d_act_off, e0, O);
      else if (K.cplx) OEFE_COUNTED k_finish<cd, double><<<nb, 256, 0, c->stream>>>(HE, c->d_act_off, e0, O);
      else if (pairs) OEFE_COUNTED k_finish<double, f2><<<nb, 256, 0, c->stream>>>(HE, c->d_act_off, e0, O);
      else OEFE_COUNTED k_finish<double, double><<<nb, 256, 0, c->stream>>>(HE, c->d_act_off, e0, O);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    }
    if (mode == 0) {
      // the V-independent OEFE blocks CO0, OO0 of each cell into the cache
      O = StoreOut{nullptr, nullptr, nullptr, nullptr, 0, c->nloc, c->npad, c->ne_max, (cd*)K.E0, nullptr, nullptr, 0, 0, 0};
      TransformSf T;
      T.sf = c->use_sumfac && c->n_sf > 0 ? c->d_sf : nullptr;
      T.sf_index = c->d_sf_index;
      T.qw = c->d_qw;
      T.veff = veff;
      T.q_off = c->d_q_off;
      for (int d = 0; d < 3; ++d) T.k[d] = K.k[d];
      T.P = c->P;
      T.nbuf = c->sf_nbuf;
      const size_t dense_smem = (size_t)c->nloc * TJB * 2 * sizeof(cd);
      const size_t sf_smem = T.sf ? ((size_t)SF_STRIDE + SF_EXTRA + c->sf_nbuf +
                                     (2 * (size_t)c->nloc + 2 * (size_t)c->sf_nbuf) * 4 * (K.cplx ? 2 : 1)) * sizeof(double) +
                                        (size_t)c->nloc * 4 * sizeof(cd)
                                  : 0;
      if (sf_smem > 227 * 1024) T.sf = nullptr;   // too large for one CTA: dense products on these cells
      const size_t tsmem = std::max(dense_smem, T.sf ? sf_smem : 0);
      OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_transform<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
      OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_transform<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)tsmem));
      if (K.cplx)
        OEFE_COUNTED k_transform<cd><<<nb, TT, tsmem, c->stream>>>(HE, (const cd*)K.gamma, c->d_act_off, e0, c->nloc, c->npad,
                                                     c->ne_max, O, T);
      else
        OEFE_COUNTED k_transform<double><<<nb, TT, tsmem, c->stream>>>(HE, K.gamma, c->d_act_off, e0, c->nloc, c->npad,
                                                         c->ne_max, O, T);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    }
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return OEFE_OK;
  });
}

int setup_kpoints(oefe_ctx* c, int nk, const double* k, const double* w) {
  if (!c->has_quad) { c->err = "kpoints: call oefe_quadrature first"; return OEFE_ERR_STATE; }
  if (nk < 1 || nk > 4096 || !k || !w) { c->err = "kpoints: need 1 <= nk <= 4096, k, w"; return OEFE_ERR_ARG; }
  for (auto& K : c->kd) {
    dev_free(K.gamma); dev_free(K.Moo); dev_free(K.Mooinv); dev_free(K.H64); dev_free(K.H32); dev_free(K.Hbf); dev_free(K.Hp);
    dev_free(K.E0); dev_free(K.NO); dev_free(K.NOp);
  }
  c->kd.assign(nk, KData());
  double* d_gw = nullptr;
  OEFE_TRY(gauss_table(c, &d_gw));
  cd *dblk = nullptr, *MAAblk = nullptr;
  const size_t dbytes = (size_t)c->ncells * c->nloc * std::max(c->ne_max, 1) * sizeof(cd);
  const size_t mbytes = (size_t)c->ncells * std::max(c->ne_max * c->ne_max, 1) * sizeof(cd);
  int st = dev_alloc(c, (void**)&dblk, dbytes);
  if (st == OEFE_OK) st = dev_alloc(c, (void**)&MAAblk, mbytes);
  double* vzero = nullptr;   // V = 0 for the pass that forms the V-independent OEFE blocks
  if (st == OEFE_OK && c->nO > 0) st = dev_alloc(c, (void**)&vzero, (size_t)std::max<int64_t>(c->nq, 1) * sizeof(double));
  if (st == OEFE_OK && vzero) {
    const cudaError_t ce = cudaMemsetAsync(vzero, 0, (size_t)std::max<int64_t>(c->nq, 1) * sizeof(double), c->stream);
    if (ce != cudaSuccess) { c->err = cudaGetErrorString(ce); st = OEFE_ERR_CUDA; }
  }
  for (int ik = 0; ik < nk && st == OEFE_OK; ++ik) {
    KData& K = c->kd[ik];
    for (int d = 0; d < 3; ++d) K.k[d] = k[3 * ik + d];
    K.w = w[ik];
    K.cplx = !(K.k[0] == 0.0 && K.k[1] == 0.0 && K.k[2] == 0.0);
    const size_t sb = K.cplx ? sizeof(cd) : sizeof(double);
    st = dev_alloc(c, (void**)&K.gamma, (size_t)c->ncells * c->nloc * std::max(c->ne_max, 1) * sb);
    if (st == OEFE_OK)
      st = dev_alloc(c, (void**)&K.E0, (size_t)c->ncells *
                                           ((size_t)c->nloc * std::max(c->ne_max, 1) + (size_t)c->ne_max * c->ne_max) *
                                           sizeof(cd));
    if (st == OEFE_OK) st = dev_alloc(c, (void**)&K.Moo, (size_t)std::max(c->nO * c->nO, 1) * sb);
    if (st == OEFE_OK) st = dev_alloc(c, (void**)&K.Mooinv, (size_t)std::max(c->nO * c->nO, 1) * sb);
    if (st != OEFE_OK || c->nO == 0) continue;
    st = run_cell_kernel(c, K, 1, nullptr, d_gw, dblk, MAAblk, 0);
    if (st != OEFE_OK) break;
    const int64_t tot = (int64_t)c->ncells * c->nloc * c->ne_max;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 1 << 20);
    if (K.cplx)
      OEFE_COUNTED k_gamma<cd><<<blocks, 256, 0, c->stream>>>(c->d_cell_nodes, c->d_node_off, c->d_node_slot, c->d_act_off,
                                                c->d_act_idx, c->d_m, dblk, c->ncells, c->nloc, c->npad, c->ne_max,
                                                (cd*)K.gamma);
    else
      OEFE_COUNTED k_gamma<double><<<blocks, 256, 0, c->stream>>>(c->d_cell_nodes, c->d_node_off, c->d_node_slot, c->d_act_off,
                                                    c->d_act_idx, c->d_m, dblk, c->ncells, c->nloc, c->npad,
                                                    c->ne_max, K.gamma);
    if (K.cplx)
      OEFE_COUNTED k_moo_cell<cd><<<c->ncells, 256, 0, c->stream>>>(c->d_act_off, c->d_m, c->d_cell_nodes, (const cd*)K.gamma,
                                                      c->P, c->nloc, c->ne_max, MAAblk);
    else
      OEFE_COUNTED k_moo_cell<double><<<c->ncells, 256, 0, c->stream>>>(c->d_act_off, c->d_m, c->d_cell_nodes, K.gamma, c->P,
                                                          c->nloc, c->ne_max, MAAblk);
    const int nb2 = (c->nO * c->nO + 255) / 256;
    if (K.cplx) {
      OEFE_COUNTED k_moo_reduce<cd><<<nb2, 256, 0, c->stream>>>(c->d_enr_off, c->d_enr_slot, c->d_act_off, c->d_act_idx, c->nO,
                                                  c->npad, c->nloc, c->ne_max, MAAblk, (cd*)K.Moo);
      OEFE_COUNTED k_hermitize<cd><<<nb2, 256, 0, c->stream>>>((cd*)K.Moo, c->nO);
    } else {
      OEFE_COUNTED k_moo_reduce<double><<<nb2, 256, 0, c->stream>>>(c->d_enr_off, c->d_enr_slot, c->d_act_off, c->d_act_idx,
                                                      c->nO, c->npad, c->nloc, c->ne_max, MAAblk, K.Moo);
      OEFE_COUNTED k_hermitize<double><<<nb2, 256, 0, c->stream>>>(K.Moo, c->nO);
    }
    OEFE_CUDA_TRY(c, cudaGetLastError());
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(K.Mooinv, K.Moo, (size_t)c->nO * c->nO * sb, cudaMemcpyDeviceToDevice,
                                     c->stream));
    int info = 0;
    st = chol_inverse_inplace(c, K.Mooinv, c->nO, K.cplx, true, &info);
    if (st == OEFE_OK && info != 0) {
      c->err = "kpoints: M^oo is not positive definite (leading minor " + std::to_string(info) + ")";
      st = OEFE_ERR_NOTPD_MOO;
    }
    // the orthogonalized enrichment at the points, and the V-independent OEFE blocks (kinetic,
    // k and |k|^2/2 terms) T^+ H_0 T of every cell into E0
    if (st == OEFE_OK) st = ensure_orth_enrichment(c, K);
    if (st == OEFE_OK) st = run_cell_kernel(c, K, 0, vzero, d_gw, nullptr, nullptr, 0);
  }
  cudaStreamSynchronize(c->stream);
  dev_free(dblk);
  dev_free(MAAblk);
  dev_free(vzero);
  dev_free(d_gw);
  if (st != OEFE_OK) return st;
  c->has_k = true;
  c->built = false;
  return OEFE_OK;
}

int build_hamiltonian(oefe_ctx* c, const double* veff, int store) {
  if (!c->has_k) { c->err = "build_hamiltonian: call oefe_kpoints first"; return OEFE_ERR_STATE; }
  if (!veff || !(store & (OEFE_STORE_F64 | OEFE_STORE_F32 | OEFE_STORE_BF16X3 | OEFE_STORE_BF16X6))) {
    c->err = "build_hamiltonian: need veff and a storage flag";
    return OEFE_ERR_ARG;
  }
  if ((store & OEFE_STORE_F64PAIR) && !(store & OEFE_STORE_F64)) {
    c->err = "build_hamiltonian: OEFE_STORE_F64PAIR goes with OEFE_STORE_F64 (the refined cells stay FP64)";
    return OEFE_ERR_ARG;
  }
  const bool compact = (store & OEFE_STORE_COMPACT) != 0;
  if (compact && !(store & OEFE_STORE_F64)) {
    c->err = "build_hamiltonian: OEFE_STORE_COMPACT is a layout of the OEFE_STORE_F64 (and F64PAIR) copies";
    return OEFE_ERR_ARG;
  }
  if (compact && !(c->use_sumfac && c->d_dense_index && c->d_sf_index)) {
    c->err = "build_hamiltonian: OEFE_STORE_COMPACT needs the sum-factorized products (p <= 7, hexahedral cells)";
    return OEFE_ERR_ARG;
  }
  double* d_gw = nullptr;
  OEFE_TRY(gauss_table(c, &d_gw));
  // V at the points, kept for the sum-factorized FP64 products of this operator
  if (!c->d_veff) OEFE_TRY(dev_alloc(c, (void**)&c->d_veff, (size_t)std::max<int64_t>(c->nq, 1) * sizeof(double)));
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(c->d_veff, veff, (size_t)c->nq * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  int st = OEFE_OK;
  for (auto& K : c->kd) {
    const size_t sb = K.cplx ? sizeof(cd) : sizeof(double);
    const size_t n = (size_t)c->ncells * c->npad * c->npad;
    const size_t n64 = h64_entries(c, compact);
    // keep existing buffers when the requested storage is unchanged
    auto keep = [&](void** p, bool want, size_t bytes) -> int {
      if (!want) { dev_free(*p); *p = nullptr; return OEFE_OK; }
      if (*p) return OEFE_OK;
      return dev_alloc(c, p, bytes);
    };
    if (compact != K.compact) {   // another layout: new FP64 / pair buffers
      dev_free(K.H64);
      dev_free(K.Hp);
      K.H64 = nullptr;
      K.Hp = nullptr;
    }
    K.compact = compact;
    st = keep((void**)&K.H64, store & OEFE_STORE_F64, n64 * sb);
    if (st == OEFE_OK) st = keep((void**)&K.H32, store & OEFE_STORE_F32, n * sb / 2);
    if (st == OEFE_OK) st = keep((void**)&K.Hp, store & OEFE_STORE_F64PAIR, n64 * sb);
    const int parts = (store & OEFE_STORE_BF16X6) ? 3 : (store & OEFE_STORE_BF16X3) ? 2 : 0;
    if (parts != K.bf_parts) {   // a different split: a new buffer
      dev_free(K.Hbf);
      K.Hbf = nullptr;
    }
    K.bf_parts = parts;
    if (st == OEFE_OK) st = keep(&K.Hbf, parts > 0, n * sb / 4 * parts);
    if (st == OEFE_OK && c->nO > 0) st = ensure_orth_enrichment(c, K);
    if (st == OEFE_OK) st = run_cell_kernel(c, K, 2, veff, d_gw, nullptr, nullptr, store);
    if (st != OEFE_OK) break;
    K.built = true;
  }
  cudaStreamSynchronize(c->stream);
  dev_free(d_gw);
  if (st == OEFE_OK && (store & (OEFE_STORE_BF16X3 | OEFE_STORE_BF16X6))) {
    // tensor maps of the split cell matrices, one per k-point
    const size_t mb = tensor_map_bytes();
    std::vector<unsigned char> maps(mb * c->kd.size());
    for (size_t ik = 0; ik < c->kd.size() && st == OEFE_OK; ++ik) st = make_cell_tmap(c, c->kd[ik], maps.data() + ik * mb);
    if (st == OEFE_OK && c->n_tmaps != (int)c->kd.size()) {
      dev_free(c->d_tmaps);
      c->d_tmaps = nullptr;
      c->n_tmaps = 0;
      st = dev_alloc(c, &c->d_tmaps, maps.size());
      if (st == OEFE_OK) c->n_tmaps = (int)c->kd.size();
    }
    if (st == OEFE_OK) {
      cudaMemcpy(c->d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice);
    }
  }
  if (st == OEFE_OK) c->built = true;
  return st;
}
