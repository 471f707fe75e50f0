// FP64 cell products by sum factorization (Eq. HOEFEelelements, CFE-CFE block).
//
// On a cell with one tensor-product leaf of n1^3 Gauss points, the CFE-CFE block of H_e is
//   H_CC = N^T diag(w (V + |k|^2/2)) N  +  sum_d G_d (x) M (x) M  (G_d in position d),
//   G_d = K_d / 2 - (i/2) k_d A_d,
// with N the tensor product of the 1D Lagrange tables at the Gauss points and M_d, K_d, A_d the
// 1D mass, stiffness and antisymmetric gradient matrices of the leaf (the same factors the build
// sums into the stored matrix). H_CC x is therefore applied without the dense (p+1)^3 x (p+1)^3
// block: three one-dimensional contractions to the points, the pointwise weight, three back,
// and seven one-dimensional contractions for the Kronecker terms. The blocks coupling the
// enrichment rows (T_e^+ H_e T_e, Eq. UOEFESplit) are read dense from the stored FP64 matrix.
// Cells refined into several leaves (those holding a nucleus) use the dense product.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "oefe_internal.h"
#include "sumfac_dev.cuh"

namespace {

constexpr int SF_THREADS = 256;

// host Lagrange values and derivatives on the GLL nodes (the construction's own formula)
void lagrange_host(const std::vector<double>& xn, double x, double* L, double* D) {
  const int P = (int)xn.size();
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

struct SfArgs {
  const double* sf;          // per listed cell: SF_STRIDE doubles
  const int* cells;          // listed cells
  const void* H;             // FP64 cell matrices (npad x npad per cell, or the compact layout)
  const float* Hp;           // the same as FP32 pairs (h, l per real part), for V = f2
  int compact, ne_max;       // compact layout: the listed cell's strip starts at sf_base + slot * strip
  long long sf_base, strip;
  const void* X;
  int ldx, nv;
  const int* cell_nodes;
  const int* act_off;
  const int* act_idx;
  int nloc, npad, P, nbuf;   // nbuf: doubles per vector component of each work buffer
  int64_t nh;
  const double* qw;
  const double* veff;
  const int64_t* q_off;
  double k[3];
  void* Z;
};

// Offset (in scalars) of entry (r, 0) of row r of a listed cell's matrix, and the first column that
// row holds: the full layout keeps every column; a compact strip keeps the enrichment columns of
// the node rows (column c at offset + c - nloc) and every column of the enrichment rows.
__device__ __forceinline__ long long sf_row(const SfArgs& A, int e, int slot, int r, int* c_first) {
  if (!A.compact) {
    *c_first = 0;
    return ((long long)e * A.npad + r) * A.npad;
  }
  const long long b = A.sf_base + (long long)slot * A.strip;
  if (r < A.nloc) {
    *c_first = A.nloc;
    return b + (long long)r * A.ne_max;
  }
  *c_first = 0;
  return b + (long long)A.nloc * A.ne_max + (long long)(r - A.nloc) * A.npad;
}

// one CTA per (block of NV vectors, listed cell): the vector blocks of a cell are adjacent in the
// launch order, so the cell's enrichment blocks come from DRAM once and from L2 after that.
// Components j = (vector, re/im) innermost. V = double: FP64; V = f2: FP32 pairs.
template <bool CPLX, int NV, typename V, int NT>
__global__ void __launch_bounds__(NT) k_cell_apply_sf(const SfArgs A) {
  using Acc = typename AccOf<V>::type;
  constexpr int R = CPLX ? 2 : 1;
  constexpr int J = NV * R;
  extern __shared__ double sm_raw[];
  V* sm = reinterpret_cast<V*>(sm_raw);
  const int e = A.cells[blockIdx.y];
  const int v0 = blockIdx.x * NV;
  const int P = A.P, nloc = A.nloc, npad = A.npad;
  const int ne = A.act_off[e + 1] - A.act_off[e];
  const int naug = nloc + ne;
  V* tab = sm;                                        // SF_STRIDE
  V* Gr = tab + SF_STRIDE;                            // K_d / 2            [3][SF_MAXP][SF_MAXP]
  V* Gi = Gr + 3 * SF_MAXP * SF_MAXP;                 // -(k_d / 2) A_d     [3][SF_MAXP][SF_MAXP]
  V* Ws = Gi + 3 * SF_MAXP * SF_MAXP;                 // w_q (V_q + |k|^2 / 2), nbuf
  V* Xs = Ws + A.nbuf;                                // npad * J
  V* Ys = Xs + (size_t)npad * J;                      // nloc * J
  V* Ab = Ys + (size_t)nloc * J;                      // nbuf * J
  V* Bb = Ab + (size_t)A.nbuf * J;                    // nbuf * J
  sf_prepare<V>(A.sf + (size_t)blockIdx.y * SF_STRIDE, tab, Gr, Gi, Ws, A.qw, A.veff, A.q_off[e], A.k);
  for (int t = threadIdx.x; t < npad * NV; t += NT) {
    const int r = t / NV, v = t % NV;
    double xr = 0.0, xi = 0.0;
    if (r < naug && v0 + v < A.nv) {
      const int64_t row = r < nloc ? (int64_t)A.cell_nodes[(size_t)e * nloc + r] : A.nh + A.act_idx[A.act_off[e] + r - nloc];
      if (CPLX) {
        const cd x = reinterpret_cast<const cd*>(A.X)[row * A.ldx + v0 + v];
        xr = x.x;
        xi = x.y;
      } else {
        xr = reinterpret_cast<const double*>(A.X)[row * A.ldx + v0 + v];
      }
    }
    Xs[(size_t)r * J + v * R] = v_from<V>(xr);
    if (CPLX) Xs[(size_t)r * J + v * R + 1] = v_from<V>(xi);
  }
  for (int t = threadIdx.x; t < nloc * J; t += NT) Ys[t] = v_from<V>(0.0);
  __syncthreads();
  sf_cc<V, CPLX, NV>(tab, Gr, Gi, Ws, P, Xs, Ys, Ab, Bb);

  // ---- enrichment blocks from the stored matrix: rows of the nodes get H_CO x_O, the enrichment
  //      rows get H_OC x_C + H_OO x_O; then every row of the product is written
  using S = typename std::conditional<CPLX, cd, double>::type;
  S* Z = reinterpret_cast<S*>(A.Z);
  if constexpr (std::is_same<V, double>::value) {
    // one (row, vector) per thread
    for (int t = threadIdx.x; t < naug * NV; t += NT) {
      const int v = t % NV, r = t / NV;
      if (v0 + v >= A.nv) continue;
      const int c0 = r < nloc ? nloc : 0;            // node rows: enrichment columns only
      int cf = 0;
      const long long ro = sf_row(A, e, blockIdx.y, r, &cf);
      const S* hr = reinterpret_cast<const S*>(A.H) + ro - cf;   // hr[c] for c >= cf
      double yr = 0, yi = 0;
      if (r < nloc) {
        yr = Ys[(size_t)r * J + v * R];
        if (CPLX) yi = Ys[(size_t)r * J + v * R + 1];
      }
      for (int cidx = c0; cidx < naug; ++cidx) {
        const double* x = Xs + (size_t)cidx * J + v * R;
        if constexpr (CPLX) {
          const cd h = hr[cidx];
          yr = fma(h.x, x[0], fma(-h.y, x[1], yr));
          yi = fma(h.x, x[1], fma(h.y, x[0], yi));
        } else {
          yr = fma(hr[cidx], x[0], yr);
        }
      }
      if constexpr (CPLX) Z[((size_t)e * npad + r) * A.nv + v0 + v] = mkc(yr, yi);
      else Z[((size_t)e * npad + r) * A.nv + v0 + v] = yr;
    }
  } else {
    // one item per thread, all NV vectors: each pair of the matrix is loaded once for NV * R
    // independent accumulations. Items: a node row over the ne enrichment columns, or a chunk of
    // at most EC columns of an enrichment row (the partial sums meet in shared memory), so that
    // the items have about the same length.
    int nch = min((naug + 47) / 48, A.nbuf / max(ne, 1));  // chunks of about 48 columns; the
    nch = max(nch, 1);                                      // partial sums must fit in Ab
    const int EC = (naug + nch - 1) / nch;
    V* part = Ab;                                          // (ne * nch) x J partial sums
    for (int it = threadIdx.x; it < nloc + ne * nch; it += NT) {
      int r, ca, cb, pidx = 0;
      if (it < nloc) {
        r = it;
        ca = nloc;
        cb = naug;
      } else {
        // consecutive items take the same chunk of consecutive enrichment rows, so that a warp reads
        // one row of the vectors per column (a broadcast) instead of one per chunk (chunks a multiple
        // of 128 bytes apart fall in the same banks)
        const int q = it - nloc, ch = q / ne, i = q % ne;
        r = nloc + i;
        ca = ch * EC;
        cb = min(naug, ca + EC);
        pidx = i * nch + ch;
      }
      Acc y[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const V s = it < nloc ? Ys[(size_t)r * J + j] : v_from<V>(0.0);
        y[j] = Acc{s.h, s.l};
      }
      if constexpr (CPLX) {
        int cf = 0;
        const long long ro = sf_row(A, e, blockIdx.y, r, &cf);
        const float4* hr = reinterpret_cast<const float4*>(A.Hp) + ro - cf;   // hr[c] for c >= cf
        float4 hn = ca < cb ? hr[ca] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int cidx = ca; cidx < cb; ++cidx) {
          const float4 h = hn;
          if (cidx + 1 < cb) hn = hr[cidx + 1];     // next pair in flight during the products
          const V hre{h.x, h.y}, him{h.z, h.w}, nhim = v_neg(him);
          const V* x = Xs + (size_t)cidx * J;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const V xr = x[2 * v], xi = x[2 * v + 1];
            v_mac(y[2 * v], hre, xr);
            v_mac(y[2 * v + 1], hre, xi);
            v_mac(y[2 * v], nhim, xi);
            v_mac(y[2 * v + 1], him, xr);
          }
        }
      } else {
        int cf = 0;
        const long long ro = sf_row(A, e, blockIdx.y, r, &cf);
        const float2* hr = reinterpret_cast<const float2*>(A.Hp) + ro - cf;   // hr[c] for c >= cf
        float2 hn = ca < cb ? hr[ca] : make_float2(0.f, 0.f);
        for (int cidx = ca; cidx < cb; ++cidx) {
          const float2 h = hn;
          if (cidx + 1 < cb) hn = hr[cidx + 1];
          const V hv{h.x, h.y};
          const V* x = Xs + (size_t)cidx * J;
#pragma unroll
          for (int v = 0; v < NV; ++v) v_mac(y[v], hv, x[v]);
        }
      }
      if (it < nloc) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (v0 + v >= A.nv) continue;
          if constexpr (CPLX) Z[((size_t)e * npad + r) * A.nv + v0 + v] = mkc(v_to(v_fin(y[2 * v])), v_to(v_fin(y[2 * v + 1])));
          else Z[((size_t)e * npad + r) * A.nv + v0 + v] = v_to(v_fin(y[v]));
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) part[(size_t)pidx * J + j] = v_fin(y[j]);
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ne * NV; t += NT) {   // enrichment rows: sum of the chunks
      const int i = t / NV, v = t % NV;
      if (v0 + v >= A.nv) continue;
      V sr = v_from<V>(0.0), si = v_from<V>(0.0);
      for (int ch = 0; ch < nch; ++ch) {
        const V* pp = part + (size_t)(i * nch + ch) * J + v * R;
        sr = v_add(sr, pp[0]);
        if (CPLX) si = v_add(si, pp[1]);
      }
      if constexpr (CPLX) Z[((size_t)e * npad + nloc + i) * A.nv + v0 + v] = mkc(v_to(sr), v_to(si));
      else Z[((size_t)e * npad + nloc + i) * A.nv + v0 + v] = v_to(sr);
    }
  }
}

template <bool CPLX>
size_t sf_smem(const oefe_ctx* c, int nv_blk) {
  const int R = CPLX ? 2 : 1;
  return ((size_t)SF_STRIDE + SF_EXTRA + c->sf_nbuf +
          ((size_t)c->npad + c->nloc + 2 * (size_t)c->sf_nbuf) * nv_blk * R) * sizeof(double);
}

}  // namespace

// Per-cell tables of the single-leaf cells (host, once per quadrature): L_d at the Gauss points,
// M_d, K_d, A_d, by the formulas of the operator build (Eq. HOEFEelelements).
int setup_sumfac(oefe_ctx* c) {
  dev_free(c->d_sf);
  dev_free(c->d_sf_cells);
  dev_free(c->d_dense_cells);
  dev_free(c->d_sf_index);
  dev_free(c->d_dense_index);
  c->d_sf = nullptr;
  c->d_sf_cells = c->d_dense_cells = c->d_sf_index = c->d_dense_index = nullptr;
  c->n_sf = c->n_dense = 0;
  const int P = c->P;
  if (P > SF_MAXP || c->nloc != P * P * P) return OEFE_OK;
  std::vector<int> sfc, den;
  std::vector<double> tabs;
  int n1max = 1;
  std::vector<double> gx[13], gw[13];
  for (int e = 0; e < c->ncells; ++e) {
    const int l0 = c->leaf_off[e], l1 = c->leaf_off[e + 1];
    const Leaf& L = c->leaves[l0];
    if (l1 - l0 != 1 || L.n1 > SF_MAXN1) { den.push_back(e); continue; }
    const int n1 = L.n1;
    if (gw[n1].empty()) gauss_rule(n1, gx[n1], gw[n1]);
    n1max = std::max(n1max, n1);
    double lo[3], hi[3];
    cell_box(c, e, lo, hi);
    std::vector<double> t(SF_STRIDE, 0.0);
    t[0] = n1;
    double Lt[3][SF_MAXN1][SF_MAXP], Dt[3][SF_MAXN1][SF_MAXP], w1[3][SF_MAXN1];
    for (int d = 0; d < 3; ++d) {
      const double h = hi[d] - lo[d];
      for (int i = 0; i < n1; ++i) {
        const int64_t qi = L.q0 + (d == 0 ? i : d == 1 ? (int64_t)i * n1 : (int64_t)i * n1 * n1);
        const double xi = 2.0 * (c->qxyz[3 * qi + d] - lo[d]) / h - 1.0;
        double Lv[SF_MAXP], Dv[SF_MAXP];
        lagrange_host(c->gll_x, xi, Lv, Dv);
        for (int a = 0; a < P; ++a) {
          Lt[d][i][a] = Lv[a];
          Dt[d][i][a] = Dv[a] * (2.0 / h);
          t[SF_L + (d * SF_MAXN1 + i) * SF_MAXP + a] = Lv[a];
        }
        w1[d][i] = gw[n1][i] * (L.hi[d] - L.lo[d]) / 2.0;
      }
      for (int a = 0; a < P; ++a)
        for (int a2 = 0; a2 < P; ++a2) {
          double m = 0, kq = 0, g1 = 0, g2 = 0;
          for (int i = 0; i < n1; ++i) {
            m += w1[d][i] * Lt[d][i][a] * Lt[d][i][a2];
            kq += w1[d][i] * Dt[d][i][a] * Dt[d][i][a2];
            g1 += w1[d][i] * Lt[d][i][a] * Dt[d][i][a2];
            g2 += w1[d][i] * Dt[d][i][a] * Lt[d][i][a2];
          }
          const int o = (d * SF_MAXP + a) * SF_MAXP + a2;
          t[SF_M + o] = m;
          t[SF_K + o] = kq;
          t[SF_A + o] = g1 - g2;
        }
    }
    sfc.push_back(e);
    tabs.insert(tabs.end(), t.begin(), t.end());
  }
  // work buffers: every intermediate of the contractions (n1 may be below P) and two P^3 blocks
  c->sf_nbuf = std::max({n1max * n1max * n1max, P * P * n1max, P * n1max * n1max, 2 * c->nloc});
  if (!sfc.empty()) {
    OEFE_TRY(dev_alloc(c, (void**)&c->d_sf, tabs.size() * sizeof(double)));
    OEFE_CUDA_TRY(c, cudaMemcpy(c->d_sf, tabs.data(), tabs.size() * sizeof(double), cudaMemcpyHostToDevice));
    OEFE_TRY(dev_alloc(c, (void**)&c->d_sf_cells, sfc.size() * sizeof(int)));
    OEFE_CUDA_TRY(c, cudaMemcpy(c->d_sf_cells, sfc.data(), sfc.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  std::vector<int> index(c->ncells, -1);
  for (size_t i = 0; i < sfc.size(); ++i) index[sfc[i]] = (int)i;
  OEFE_TRY(dev_alloc(c, (void**)&c->d_sf_index, index.size() * sizeof(int)));
  OEFE_CUDA_TRY(c, cudaMemcpy(c->d_sf_index, index.data(), index.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!den.empty()) {
    OEFE_TRY(dev_alloc(c, (void**)&c->d_dense_cells, den.size() * sizeof(int)));
    OEFE_CUDA_TRY(c, cudaMemcpy(c->d_dense_cells, den.data(), den.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  std::vector<int> dindex(c->ncells, -1);
  for (size_t i = 0; i < den.size(); ++i) dindex[den[i]] = (int)i;
  OEFE_TRY(dev_alloc(c, (void**)&c->d_dense_index, dindex.size() * sizeof(int)));
  OEFE_CUDA_TRY(c, cudaMemcpy(c->d_dense_index, dindex.data(), dindex.size() * sizeof(int), cudaMemcpyHostToDevice));
  c->n_sf = (int)sfc.size();
  c->n_dense = (int)den.size();
  return OEFE_OK;
}

bool sumfac_ready(const oefe_ctx* c) { return c->use_sumfac && c->n_sf > 0 && c->d_veff; }

// Products of the listed single-leaf cells (FP64, real or complex) into Z (ncells x npad x nv).
int launch_cell_apply_sf(oefe_ctx* c, const KData& K, const void* X, int ldx, int nv, bool cplx, void* Z,
                         cudaStream_t st) {
  SfArgs A;
  A.sf = c->d_sf;
  A.cells = c->d_sf_cells;
  A.H = K.H64;
  A.Hp = K.Hp;
  A.compact = K.compact ? 1 : 0;
  A.ne_max = c->ne_max;
  A.sf_base = (long long)c->n_dense * c->npad * c->npad;
  A.strip = (long long)compact_strip(c);
  A.X = X;
  A.ldx = ldx;
  A.nv = nv;
  A.cell_nodes = c->d_cell_nodes;
  A.act_off = c->d_act_off;
  A.act_idx = c->d_act_idx;
  A.nloc = c->nloc;
  A.npad = c->npad;
  A.P = c->P;
  A.nbuf = c->sf_nbuf;
  A.nh = c->nh;
  A.qw = c->d_qw;
  A.veff = c->d_veff;
  A.q_off = c->d_q_off;
  for (int d = 0; d < 3; ++d) A.k[d] = K.k[d];
  A.Z = Z;
  auto go = [&](auto kern, size_t smem, int nvb, int nthreads) -> int {
    if (smem > 227 * 1024) { c->err = "sum factorization: work arrays exceed shared memory"; return OEFE_ERR_ARG; }
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((nv + nvb - 1) / nvb, c->n_sf);
    OEFE_COUNTED kern<<<grid, nthreads, smem, st>>>(A);
    OEFE_CUDA_TRY(c, cudaGetLastError());
    return OEFE_OK;
  };
  if (c->f64_products == OEFE_F64_PAIRS) {
    if (!K.Hp) { c->err = "FP32-pair products: build the operator with OEFE_STORE_F64PAIR"; return OEFE_ERR_STATE; }
    // launch shapes: one CTA of 512 threads per SM over 4 (complex) vectors, or two CTAs of 384 or
    // of 512 threads per SM over 2 vectors each (half the shared memory, the cell's enrichment
    // blocks read twice as often); the fastest on this operator is kept after timing each once
    auto run = [&](int v) -> int {
      if (cplx) {
        if (v == 0) return go(k_cell_apply_sf<true, 4, f2, 512>, sf_smem<true>(c, 4), 4, 512);
        if (v == 1) return go(k_cell_apply_sf<true, 2, f2, 384>, sf_smem<true>(c, 2), 2, 384);
        return go(k_cell_apply_sf<true, 2, f2, 512>, sf_smem<true>(c, 2), 2, 512);
      }
      if (v == 0) return go(k_cell_apply_sf<false, 8, f2, 512>, sf_smem<false>(c, 8), 8, 512);
      if (v == 1) return go(k_cell_apply_sf<false, 4, f2, 384>, sf_smem<false>(c, 4), 4, 384);
      return go(k_cell_apply_sf<false, 4, f2, 512>, sf_smem<false>(c, 4), 4, 512);
    };
    if (c->sf_variant < 0) {   // first use: time each on this operator (after one warm launch)
      constexpr int NVAR = 3;
      cudaEvent_t ev[NVAR + 1];
      for (auto& e : ev) OEFE_CUDA_TRY(c, cudaEventCreate(&e));
      int s = run(0);
      if (s == OEFE_OK) cudaEventRecord(ev[0], st);
      for (int v = 0; v < NVAR && s == OEFE_OK; ++v) {
        s = run(v);
        cudaEventRecord(ev[v + 1], st);
      }
      if (s == OEFE_OK) {
        OEFE_CUDA_TRY(c, cudaEventSynchronize(ev[NVAR]));
        float best = 1e30f;
        for (int v = 0; v < NVAR; ++v) {
          float ms = 0;
          cudaEventElapsedTime(&ms, ev[v], ev[v + 1]);
          if (ms < best) { best = ms; c->sf_variant = v; }
        }
        // Z holds the last variant's product; the products of all variants are the same numbers
      }
      for (auto& e : ev) cudaEventDestroy(e);
      return s;
    }
    return run(c->sf_variant);
  }
  if (cplx) return go(k_cell_apply_sf<true, 4, double, SF_THREADS>, sf_smem<true>(c, 4), 4, SF_THREADS);
  return go(k_cell_apply_sf<false, 8, double, SF_THREADS>, sf_smem<false>(c, 8), 8, SF_THREADS);
}

// FP64 operations (an FMA counts two) of one FP64 application of the cell products to nv vectors:
// single-leaf cells by the stages of k_cell_apply_sf, the others dense (3 real multiplications
// per complex product, one per real one).
double fp64_product_flops(const oefe_ctx* c, bool cplx, int nv) {
  const double P = c->P, P2 = P * P, P3 = P2 * P;
  const bool sf = sumfac_ready(c);
  double fma = 0.0;
  std::vector<char> is_sf(c->ncells, 0);
  if (sf)
    for (int e = 0; e < c->ncells; ++e) is_sf[e] = c->leaf_off[e + 1] - c->leaf_off[e] == 1;
  for (int e = 0; e < c->ncells; ++e) {
    const double ne = c->act_off[e + 1] - c->act_off[e], naug = c->nloc + ne;
    if (!is_sf[e]) { fma += naug * naug * (cplx ? 3.0 : 1.0); continue; }
    const double n1 = c->leaves[c->leaf_off[e]].n1;
    const double vpart = 2.0 * (P2 * n1 * P + P * n1 * n1 * P + n1 * n1 * n1 * P);  // to the points and back
    const double kin = cplx ? (6.0 + 8.0 + 6.0) * P * P3 : (2.0 + 3.0 + 2.0) * P * P3;
    const double enr = (c->nloc * ne + ne * naug) * (cplx ? 4.0 : 1.0);
    fma += vpart * (cplx ? 2.0 : 1.0) + kin + enr;
  }
  return 2.0 * fma * nv;
}
