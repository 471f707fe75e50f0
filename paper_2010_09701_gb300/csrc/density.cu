// Fields at the quadrature points (Eq. UOEFE, Eq. rho):
//   u(x_q) = sum_a N^C_a(x_q) (X^c - Gamma_e X^o)_a + sum_j N^A_j(x_q) X^o_j
//          = sum_a N^C_a(x_q) X^c_a + sum_j N^O_j(x_q) X^o_j,
//   N^O_j(x_q) = N^A_j(x_q) - sum_a N^C_a(x_q) Gamma_aj   (the orthogonalized enrichment),
// then
//   density:          rho_q += sum_v occ_v |u_v(x_q)|^2
//   band-trace grad:  g_q    = w_q sum_v |u_v(x_q)|^2  (adjoint of H.X w.r.t. V_q),
//   VJP of Y = H X:   g_q    = w_q Re sum_v conj(u_G,v(x_q)) u_X,v(x_q) (cotangent G of Y).
// N^O depends on k only: it is tabulated once per k-point (k_orth_enrichment) and kept; the
// fields then take the CFE part by sum factorization per tensor-product leaf and the enrichment
// part as a dense product with the table (k_fields), in FP64 or FP32-pair arithmetic.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "oefe_internal.h"
#include "enrich_dev.cuh"
#include "pair_dev.cuh"

namespace {

constexpr int MAXP = 8;
constexpr int MAXN1 = 12;
constexpr int DT = 256;
constexpr int NBO = 4;   // columns of Gamma per pass of the tabulation
constexpr int FT = 512;  // threads per CTA of the fields

struct OrthArgs {
  EnrParams E;
  const Leaf* leaves;
  const double* qxyz;
  const double* cellbox;
  const double* gll;
  const int* act_off;
  const int* act_idx;
  int nleaves, P, nloc, ne_max;
  double k[3];
  bool cplx;
  const void* gamma;  // (ncells, nloc, ne_max)
  cd* na;             // per-CTA scratch: max leaf points * ne_max
  int64_t na_stride;
  void* NO;           // out: scalars
  float* NOp;         // out: FP32 pairs (or null)
};

__device__ inline cd ldG(const OrthArgs& A, size_t i) {
  if (A.cplx) return reinterpret_cast<const cd*>(A.gamma)[i];
  return mkc(reinterpret_cast<const double*>(A.gamma)[i], 0.0);
}

// N^O at the points of every leaf: the enrichment values (one (point, atom) per thread: the active
// set holds whole atoms, whose functions share the offset, cutoff and phase) minus the CFE
// interpolant of Gamma's columns, NBO columns per pass by sum factorization. FP64.
__global__ void __launch_bounds__(DT) k_orth_enrichment(OrthArgs A) {
  extern __shared__ double smem[];
  __shared__ double Lt[3][MAXN1][MAXP];
  __shared__ double xn[MAXP];
  if (threadIdx.x < A.P) xn[threadIdx.x] = A.gll[threadIdx.x];
  const int P = A.P, nloc = A.nloc, NB = NBO;
  cd* na = A.na + (size_t)blockIdx.x * A.na_stride;
  for (int li = blockIdx.x; li < A.nleaves; li += gridDim.x) {
    const Leaf L = A.leaves[li];
    const int e = L.cell;
    const int ne = A.act_off[e + 1] - A.act_off[e];
    const double* box = A.cellbox + 6 * e;
    const int n1 = L.n1, n2 = n1 * n1, n3 = n2 * n1;
    __syncthreads();
    if (threadIdx.x < 3 * n1) {
      const int d = threadIdx.x / n1, i = threadIdx.x % n1;
      const int64_t qi = L.q0 + (d == 0 ? i : d == 1 ? i * n1 : i * n2);
      const double xi = 2.0 * (A.qxyz[3 * qi + d] - box[d]) / box[3 + d] - 1.0;
      double Lv[MAXP], Dv[MAXP];
      lagrange_eval(xn, P, xi, Lv, Dv);
      for (int a = 0; a < P; ++a) Lt[d][i][a] = Lv[a];
    }
    const int nat = A.E.nfun > 0 ? ne / A.E.nfun : 0;
    for (int t = threadIdx.x; t < n3 * nat; t += DT) {
      const int q = t / nat, j0 = (t % nat) * A.E.nfun;
      const int64_t qg = L.q0 + q;
      const double x[3] = {A.qxyz[3 * qg], A.qxyz[3 * qg + 1], A.qxyz[3 * qg + 2]};
      const int I = A.act_idx[A.act_off[e] + j0] / A.E.nfun;
      AtomGeom G;
      atom_geom(A.E, I, x, A.k, false, G);
      for (int f = 0; f < A.E.nfun; ++f) atom_function(A.E, I, f, G, A.k, &na[q * ne + j0 + f], nullptr);
    }
    cd* Xt = reinterpret_cast<cd*>(smem);   // nloc * NB: -Gamma[:, v0:v0+NB]
    cd* T1 = Xt + nloc * NB;                // n1 * P * P * NB   [qx][b][c][v]
    cd* T2 = T1 + n1 * P * P * NB;          // n2 * P * NB       [qx][qy][c][v]
    const size_t blk = (size_t)L.q0 * A.ne_max;
    for (int v0 = 0; v0 < A.ne_max; v0 += NB) {
      __syncthreads();
      for (int t = threadIdx.x; t < nloc * NB; t += DT) {
        const int a = t / NB, u = t % NB;
        Xt[t] = v0 + u < ne ? -ldG(A, ((size_t)e * nloc + a) * A.ne_max + v0 + u) : mkc(0, 0);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < n1 * P * P * NB; t += DT) {
        const int u = t % NB, r = t / NB;
        const int c = r % P, bb = (r / P) % P, qx = r / (P * P);
        cd s = mkc(0, 0);
        for (int a = 0; a < P; ++a) s = rfma(Lt[0][qx][a], Xt[(a + P * (bb + P * c)) * NB + u], s);
        T1[t] = s;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < n2 * P * NB; t += DT) {
        const int u = t % NB, r = t / NB;
        const int c = r % P, qy = (r / P) % n1, qx = r / (P * n1);
        cd s = mkc(0, 0);
        for (int bb = 0; bb < P; ++bb) s = rfma(Lt[1][qy][bb], T1[((qx * P + bb) * P + c) * NB + u], s);
        T2[t] = s;
      }
      __syncthreads();
      // z stage plus the enrichment value; column-major store (point fastest)
      for (int t = threadIdx.x; t < n3 * NB; t += DT) {
        const int q = t % n3, u = t / n3;
        const int qx = q % n1, qy = (q / n1) % n1, qz = q / n2;
        if (v0 + u >= A.ne_max) continue;
        cd s = v0 + u < ne ? na[q * ne + v0 + u] : mkc(0, 0);
        for (int c = 0; c < P; ++c) s = rfma(Lt[2][qz][c], T2[((qx * n1 + qy) * P + c) * NB + u], s);
        const size_t o = blk + (size_t)(v0 + u) * n3 + q;
        if (A.cplx) {
          reinterpret_cast<cd*>(A.NO)[o] = s;
          if (A.NOp) {
            const float rh = __double2float_rn(s.x), ih = __double2float_rn(s.y);
            reinterpret_cast<float4*>(A.NOp)[o] =
                make_float4(rh, __double2float_rn(s.x - (double)rh), ih, __double2float_rn(s.y - (double)ih));
          }
        } else {
          reinterpret_cast<double*>(A.NO)[o] = s.x;
          if (A.NOp) {
            const float h = __double2float_rn(s.x);
            reinterpret_cast<float2*>(A.NOp)[o] = make_float2(h, __double2float_rn(s.x - (double)h));
          }
        }
      }
    }
  }
}

size_t orth_smem(const oefe_ctx* c) {
  const int n1 = std::max(c->nq_cell, c->nq_enr), P = c->P;
  return ((size_t)c->nloc * NBO + (size_t)n1 * P * P * NBO + (size_t)n1 * n1 * P * NBO) * sizeof(cd);
}

struct FieldArgs {
  const Leaf* leaves;
  const double* qxyz;
  const double* cellbox;
  const double* gll;
  const int* cell_nodes;
  const int* act_off;
  const int* act_idx;
  int nleaves, P, nloc, ne_max, n1max;
  int64_t nh;
  const void* X;      // F64 or C128 rows, ld
  int ld, nv;
  const void* NO;     // N^O: scalars (V = double) or FP32 pairs (V = f2)
  const double* occ;  // nv weights (density) or null (gradient: weight 1, times w_q)
  const double* qw;
  double* out;        // nq
  bool accumulate;    // density: out += ; gradient: out =
  double scale;       // gradient: out = scale w_q (...)
  // with the density (occ set, accumulate): out2 (nq, overwritten, or null) = w_q sum_v |u_v|^2 of
  // the same fields, the band-trace gradient of these columns
  double* out2;
  // cross mode (X2 != null): a pass of RNB takes RNB/2 columns of X and the same columns of X2; the
  // point's sum is Re sum_v conj(u_X2,v) u_X,v instead of sum_v |u_X,v|^2
  const void* X2;
  int ld2;
};

// u_v(x_q) for RNB vectors per pass (4: one CTA per SM; 2: half the shared memory, two CTAs per SM): CFE part by sum factorization (x, y, z stages over the leaf's
// Gauss points), enrichment part sum_j N^O_j(x_q) X^o_j with one point per thread over all RNB
// vectors; |u|^2 weighted by occ accumulated per point. V = double: FP64; V = f2: FP32 pairs.
template <typename V, bool CPLX, int RNB>
__global__ void __launch_bounds__(FT) k_fields(FieldArgs A) {
  constexpr int R = CPLX ? 2 : 1;
  constexpr int J = RNB * R;
  using Acc = typename AccOf<V>::type;
  extern __shared__ double smem_raw[];
  __shared__ V Lt[3][MAXN1][MAXP];
  __shared__ double xn[MAXP];
  if (threadIdx.x < A.P) xn[threadIdx.x] = A.gll[threadIdx.x];
  const int P = A.P, nloc = A.nloc, n1m = A.n1max;
  V* Xt = reinterpret_cast<V*>(smem_raw);          // nloc * J
  V* Xo = Xt + (size_t)nloc * J;                   // ne_max * J
  V* T1 = Xo + (size_t)A.ne_max * J;               // n1 * P * P * J   [qx][b][c][j]
  V* T2 = T1 + (size_t)n1m * P * P * J;            // n2 * P * J       [qx][qy][c][j]
  V* U = T2 + (size_t)n1m * n1m * P * J;           // n3 * J
  V* rho = U + (size_t)n1m * n1m * n1m * J;        // 2 x n3: one per half of the vectors (4 x n3
                                                   // with out2: the unweighted sums after them)
  const bool dual = A.out2 != nullptr;
  for (int li = blockIdx.x; li < A.nleaves; li += gridDim.x) {
    const Leaf L = A.leaves[li];
    const int e = L.cell;
    const int ne = A.act_off[e + 1] - A.act_off[e];
    const double* box = A.cellbox + 6 * e;
    const int n1 = L.n1, n2 = n1 * n1, n3 = n2 * n1;
    __syncthreads();
    if (threadIdx.x < 3 * n1) {
      const int d = threadIdx.x / n1, i = threadIdx.x % n1;
      const int64_t qi = L.q0 + (d == 0 ? i : d == 1 ? i * n1 : i * n2);
      const double xi = 2.0 * (A.qxyz[3 * qi + d] - box[d]) / box[3 + d] - 1.0;
      double Lv[MAXP], Dv[MAXP];
      lagrange_eval(xn, P, xi, Lv, Dv);
      for (int a = 0; a < P; ++a) Lt[d][i][a] = v_from<V>(Lv[a]);
    }
    for (int q = threadIdx.x; q < (dual ? 4 : 2) * n3; q += FT) rho[q] = v_from<V>(0.0);
    const size_t blk = (size_t)L.q0 * A.ne_max;
    const bool cross = A.X2 != nullptr;
    constexpr int HV = RNB / 2, HJ = HV * R;
    // slot u of a pass: column v0 + u of X, or (cross mode) column v0 / 2 + u % HV of X (u < HV) or
    // of X2 (u >= HV)
    auto column = [&](int v0, int u, const void** M, int* ld) -> int {
      if (!cross) {
        *M = A.X;
        *ld = A.ld;
        return v0 + u;
      }
      *M = u < HV ? A.X : A.X2;
      *ld = u < HV ? A.ld : A.ld2;
      return v0 / 2 + u % HV;
    };
    const int vend = cross ? 2 * A.nv : A.nv;
    for (int v0 = 0; v0 < vend; v0 += RNB) {
      __syncthreads();
      for (int t = threadIdx.x; t < ne * RNB; t += FT) {
        const int j = t / RNB, u = t % RNB;
        double xr = 0.0, xi = 0.0;
        const void* M;
        int ldm;
        const int v = column(v0, u, &M, &ldm);
        if (v < A.nv) {
          const int64_t row = A.nh + A.act_idx[A.act_off[e] + j];
          if (CPLX) {
            const cd x = reinterpret_cast<const cd*>(M)[row * ldm + v];
            xr = x.x;
            xi = x.y;
          } else {
            xr = reinterpret_cast<const double*>(M)[row * ldm + v];
          }
        }
        Xo[(size_t)j * J + u * R] = v_from<V>(xr);
        if (CPLX) Xo[(size_t)j * J + u * R + 1] = v_from<V>(xi);
      }
      for (int t = threadIdx.x; t < nloc * RNB; t += FT) {
        const int a = t / RNB, u = t % RNB;
        double xr = 0.0, xi = 0.0;
        const void* M;
        int ldm;
        const int v = column(v0, u, &M, &ldm);
        if (v < A.nv) {
          const int64_t row = A.cell_nodes[(size_t)e * nloc + a];
          if (CPLX) {
            const cd x = reinterpret_cast<const cd*>(M)[row * ldm + v];
            xr = x.x;
            xi = x.y;
          } else {
            xr = reinterpret_cast<const double*>(M)[row * ldm + v];
          }
        }
        Xt[(size_t)a * J + u * R] = v_from<V>(xr);
        if (CPLX) Xt[(size_t)a * J + u * R + 1] = v_from<V>(xi);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < n1 * P * P * J; t += FT) {   // x stage
        const int j = t % J, r = t / J;
        const int c = r % P, bb = (r / P) % P, qx = r / (P * P);
        T1[t] = v_dot<V>(P, [&](int a) { return Lt[0][qx][a]; },
                         [&](int a) { return Xt[(size_t)(a + P * (bb + P * c)) * J + j]; });
      }
      __syncthreads();
      for (int t = threadIdx.x; t < n2 * P * J; t += FT) {       // y stage
        const int j = t % J, r = t / J;
        const int c = r % P, qy = (r / P) % n1, qx = r / (P * n1);
        T2[t] = v_dot<V>(P, [&](int bb) { return Lt[1][qy][bb]; },
                         [&](int bb) { return T1[(size_t)((qx * P + bb) * P + c) * J + j]; });
      }
      __syncthreads();
      for (int t = threadIdx.x; t < n3 * J; t += FT) {           // z stage
        const int j = t % J, q = t / J;
        const int qx = q % n1, qy = (q / n1) % n1, qz = q / n2;
        U[t] = v_dot<V>(P, [&](int c) { return Lt[2][qz][c]; },
                        [&](int c) { return T2[(size_t)((qx * n1 + qy) * P + c) * J + j]; });
      }
      __syncthreads();
      // enrichment part and |u|^2: items (point, half of the RNB vectors)
      for (int tq = threadIdx.x; tq < 2 * n3; tq += FT) {
        const int q = tq >> 1, h = tq & 1;
        Acc y[HJ];
#pragma unroll
        for (int j = 0; j < HJ; ++j) {
          const V u0 = U[(size_t)q * J + h * HJ + j];
          if constexpr (std::is_same<V, double>::value) y[j] = u0;
          else y[j] = Acc{u0.h, u0.l};
        }
        for (int jj = 0; jj < ne; ++jj) {
          const size_t o = blk + (size_t)jj * n3 + q;
          const V* x = Xo + (size_t)jj * J + h * HJ;
          if constexpr (CPLX) {
            V nr, ni;
            if constexpr (std::is_same<V, double>::value) {
              const cd w = reinterpret_cast<const cd*>(A.NO)[o];
              nr = w.x;
              ni = w.y;
            } else {
              const float4 w = reinterpret_cast<const float4*>(A.NO)[o];
              nr = V{w.x, w.y};
              ni = V{w.z, w.w};
            }
            const V nni = v_neg(ni);
#pragma unroll
            for (int u = 0; u < HV; ++u) {
              v_mac(y[2 * u], nr, x[2 * u]);
              v_mac(y[2 * u + 1], nr, x[2 * u + 1]);
              v_mac(y[2 * u], nni, x[2 * u + 1]);
              v_mac(y[2 * u + 1], ni, x[2 * u]);
            }
          } else {
            V nr;
            if constexpr (std::is_same<V, double>::value) {
              nr = reinterpret_cast<const double*>(A.NO)[o];
            } else {
              const float2 w = reinterpret_cast<const float2*>(A.NO)[o];
              nr = V{w.x, w.y};
            }
#pragma unroll
            for (int u = 0; u < HV; ++u) v_mac(y[u], nr, x[u]);
          }
        }
        V s = rho[h * n3 + q];
        V s2 = dual ? rho[(2 + h) * n3 + q] : v_from<V>(0.0);
        if (cross) {
          // the partner item (same point, other half: adjacent threads of one warp, both active)
          // holds the X2 fields of the same columns; the X half takes Re conj(u_X2) u_X
          const unsigned mask = __activemask();
#pragma unroll
          for (int j = 0; j < HJ; ++j) {
            const V mine = v_fin(y[j]);
            V other;
            if constexpr (std::is_same<V, double>::value) {
              other = __shfl_xor_sync(mask, mine, 1);
            } else {
              other.h = __shfl_xor_sync(mask, mine.h, 1);
              other.l = __shfl_xor_sync(mask, mine.l, 1);
            }
            if (h == 0) {
              const int u = j / R;
              if (v0 / 2 + u < A.nv) {
                Acc m = v_zero<V>();
                v_mac(m, mine, other);   // Re: x_r g_r + x_i g_i over the two components
                s = v_add(s, v_fin(m));
              }
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < HV; ++u) {
            const int v = v0 + h * HV + u;
            if (v >= A.nv) continue;
            Acc m = v_zero<V>();
            const V yr = v_fin(y[u * R]);
            v_mac(m, yr, yr);
            if constexpr (CPLX) {
              const V yi = v_fin(y[u * R + 1]);
              v_mac(m, yi, yi);
            }
            const V w = v_from<V>(A.occ ? A.occ[v] : 1.0);
            s = v_add(s, v_mul(w, v_fin(m)));
            if (dual) s2 = v_add(s2, v_fin(m));
          }
        }
        rho[h * n3 + q] = s;
        if (dual) rho[(2 + h) * n3 + q] = s2;
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n3; q += FT) {
      const int64_t qg = L.q0 + q;
      const double r = v_to(v_add(rho[q], rho[n3 + q]));
      if (A.accumulate) A.out[qg] += r;
      else A.out[qg] = A.scale * A.qw[qg] * r;
      if (dual) A.out2[qg] = A.qw[qg] * v_to(v_add(rho[2 * n3 + q], rho[3 * n3 + q]));
    }
  }
}

template <typename V>
size_t field_smem(const oefe_ctx* c, bool cplx, int rnb, bool dual = false) {
  const int n1 = std::max(c->nq_cell, c->nq_enr), P = c->P;
  const size_t J = (size_t)rnb * (cplx ? 2 : 1);
  const size_t n3 = (size_t)n1 * n1 * n1;
  return ((size_t)c->nloc * J + (size_t)std::max(c->ne_max, 1) * J + (size_t)n1 * P * P * J +
          (size_t)n1 * n1 * P * J + n3 * J + (dual ? 4 : 2) * n3) * sizeof(V);
}

}  // namespace

// N^O of k-point K (and its FP32-pair copy when the context runs pair products), once per k
int ensure_orth_enrichment(oefe_ctx* c, KData& K) {
  const bool pairs = c->f64_products == OEFE_F64_PAIRS;
  if (K.NO && (K.NOp || !pairs)) return OEFE_OK;
  const int nem = std::max(c->ne_max, 1);
  const size_t n = (size_t)c->nq * nem;
  const size_t sb = K.cplx ? sizeof(cd) : sizeof(double);
  if (!K.NO) OEFE_TRY(dev_alloc(c, &K.NO, n * sb));
  if (pairs && !K.NOp) OEFE_TRY(dev_alloc(c, (void**)&K.NOp, n * sb));
  const size_t smem = orth_smem(c);
  if (smem > 220 * 1024) { c->err = "fields: quadrature too large for the interpolation tiles"; return OEFE_ERR_ARG; }
  const int grid = std::max(1, std::min((int)c->leaves.size(), 2 * c->num_sms));
  const int n1 = std::max(c->nq_cell, c->nq_enr);
  const int64_t stride = (int64_t)n1 * n1 * n1 * nem;
  OEFE_TRY(ensure_ws2(c, (size_t)grid * stride * sizeof(cd) + 256));
  OrthArgs A;
  A.E.pos = c->d_pos; A.E.lm = c->d_lm; A.E.R = c->d_R; A.E.dR = c->d_dR;
  A.E.nfun = c->nfun; A.E.ngrid = c->ngrid; A.E.a = c->a; A.E.r0 = c->r0; A.E.rc = c->rc;
  A.leaves = c->d_leaves;
  A.qxyz = c->d_qxyz;
  A.cellbox = c->d_cellbox;
  A.gll = c->d_gll;
  A.act_off = c->d_act_off;
  A.act_idx = c->d_act_idx;
  A.nleaves = (int)c->leaves.size();
  A.P = c->P;
  A.nloc = c->nloc;
  A.ne_max = nem;
  for (int d = 0; d < 3; ++d) A.k[d] = K.k[d];
  A.cplx = K.cplx;
  A.gamma = K.gamma;
  A.na = (cd*)c->ws2;
  A.na_stride = stride;
  A.NO = K.NO;
  A.NOp = pairs ? K.NOp : nullptr;
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_orth_enrichment, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  OEFE_COUNTED k_orth_enrichment<<<grid, DT, smem, c->stream>>>(A);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

namespace {

int run_fields(oefe_ctx* c, KData& K, const void* X, int nv, int ld, int dtype, const double* occ, double* out,
               bool accumulate, double scale = 1.0, const void* X2 = nullptr, int ld2 = 0, double* out2 = nullptr) {
  OEFE_TRY(ensure_orth_enrichment(c, K));
  const bool pairs = c->f64_products == OEFE_F64_PAIRS;
  const bool cplx = dtype == OEFE_C128;
  FieldArgs A;
  A.leaves = c->d_leaves;
  A.qxyz = c->d_qxyz;
  A.cellbox = c->d_cellbox;
  A.gll = c->d_gll;
  A.cell_nodes = c->d_cell_nodes;
  A.act_off = c->d_act_off;
  A.act_idx = c->d_act_idx;
  A.nleaves = (int)c->leaves.size();
  A.P = c->P;
  A.nloc = c->nloc;
  A.ne_max = std::max(c->ne_max, 1);
  A.n1max = std::max(c->nq_cell, c->nq_enr);
  A.nh = c->nh;
  A.X = X;
  A.ld = ld;
  A.nv = nv;
  A.NO = pairs ? (const void*)K.NOp : (const void*)K.NO;
  A.occ = occ;
  A.qw = c->d_qw;
  A.out = out;
  A.accumulate = accumulate;
  A.scale = scale;
  A.X2 = X2;
  A.ld2 = ld2;
  A.out2 = out2;
  const bool dual = out2 != nullptr;
  const int grid = std::max(1, std::min((int)c->leaves.size(), c->num_sms));
  auto go = [&](auto kern, size_t smem) -> int {
    if (smem > 227 * 1024) { c->err = "fields: quadrature too large for the interpolation tiles"; return OEFE_ERR_ARG; }
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    OEFE_COUNTED kern<<<grid, FT, smem, c->stream>>>(A);
    OEFE_CUDA_TRY(c, cudaGetLastError());
    return OEFE_OK;
  };
  if (pairs) {
    // two pass widths, the faster kept after timing both at first use (same arithmetic per vector)
    auto run = [&](int v) -> int {
      if (v == 0 && field_smem<f2>(c, cplx, 4, dual) > 227 * 1024) v = 1;   // the wide pass does not fit
      if (cplx) return v == 0 ? go(k_fields<f2, true, 4>, field_smem<f2>(c, true, 4, dual))
                              : go(k_fields<f2, true, 2>, field_smem<f2>(c, true, 2, dual));
      return v == 0 ? go(k_fields<f2, false, 4>, field_smem<f2>(c, false, 4, dual))
                    : go(k_fields<f2, false, 2>, field_smem<f2>(c, false, 2, dual));
    };
    if (c->fields_variant < 0 && accumulate) {   // the density accumulates: time on a scratch copy of out
      double* scratch = nullptr;
      OEFE_TRY(dev_alloc(c, (void**)&scratch, (size_t)std::max<int64_t>(c->nq, 1) * sizeof(double)));
      double* keep = A.out;
      double* keep2 = A.out2;
      A.out = scratch;
      A.out2 = nullptr;
      cudaEvent_t ev[3];
      for (auto& e : ev) OEFE_CUDA_TRY(c, cudaEventCreate(&e));
      int s = run(0);
      if (s == OEFE_OK) { cudaEventRecord(ev[0], c->stream); s = run(1); }
      if (s == OEFE_OK) { cudaEventRecord(ev[1], c->stream); s = run(0); cudaEventRecord(ev[2], c->stream); }
      float t1 = 0, t0 = 0;
      if (s == OEFE_OK) {
        cudaEventSynchronize(ev[2]);
        cudaEventElapsedTime(&t1, ev[0], ev[1]);
        cudaEventElapsedTime(&t0, ev[1], ev[2]);
        c->fields_variant = t1 < t0 ? 1 : 0;
      }
      for (auto& e : ev) cudaEventDestroy(e);
      cudaStreamSynchronize(c->stream);
      dev_free(scratch);
      A.out = keep;
      A.out2 = keep2;
      if (s != OEFE_OK) return s;
    }
    return run(c->fields_variant > 0 ? 1 : 0);
  }
  if (cplx) {
    if (field_smem<double>(c, true, 4, dual) > 227 * 1024) return go(k_fields<double, true, 2>, field_smem<double>(c, true, 2, dual));
    return go(k_fields<double, true, 4>, field_smem<double>(c, true, 4, dual));
  }
  return go(k_fields<double, false, 4>, field_smem<double>(c, false, 4, dual));
}

int check_fields(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype) {
  if (!c->has_k) { c->err = "call oefe_kpoints first"; return OEFE_ERR_STATE; }
  if (ik < 0 || ik >= (int)c->kd.size()) { c->err = "k index out of range"; return OEFE_ERR_ARG; }
  if (!X || nv < 1 || ld < nv) { c->err = "need X and 1 <= nv <= ld"; return OEFE_ERR_ARG; }
  if (!(dtype == OEFE_F64 || dtype == OEFE_C128)) { c->err = "fields need F64 or C128 vectors"; return OEFE_ERR_ARG; }
  if (c->kd[ik].cplx != (dtype == OEFE_C128)) { c->err = "dtype does not match the k-point"; return OEFE_ERR_ARG; }
  return OEFE_OK;
}

}  // namespace

int density_grad(oefe_ctx* c, int nk, const void* const* X, const int* nv, const int* ld, int dtype, const double* occ,
                 double* rho, int ik_grad, double* gV) {
  if (nk != (int)c->kd.size() || !X || !nv || !ld || !occ || !rho) {
    c->err = "density: need one X, nv, ld per k-point, occ and rho";
    return OEFE_ERR_ARG;
  }
  if (gV && (ik_grad < 0 || ik_grad >= nk)) { c->err = "density: gradient k index out of range"; return OEFE_ERR_ARG; }
  int tot = 0;
  for (int ik = 0; ik < nk; ++ik) {
    const int dt = c->kd[ik].cplx ? OEFE_C128 : OEFE_F64;
    if (dtype != OEFE_F64 && dtype != OEFE_C128) { c->err = "density: dtype F64 or C128"; return OEFE_ERR_ARG; }
    OEFE_TRY(check_fields(c, ik, X[ik], nv[ik], ld[ik], dt));
    tot += nv[ik];
  }
  double* d_occ = nullptr;
  OEFE_TRY(dev_alloc(c, (void**)&d_occ, (size_t)tot * sizeof(double)));
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_occ, occ, (size_t)tot * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  OEFE_CUDA_TRY(c, cudaMemsetAsync(rho, 0, (size_t)c->nq * sizeof(double), c->stream));
  int off = 0, st = OEFE_OK;
  for (int ik = 0; ik < nk && st == OEFE_OK; ++ik) {
    const int dt = c->kd[ik].cplx ? OEFE_C128 : OEFE_F64;
    st = run_fields(c, c->kd[ik], X[ik], nv[ik], ld[ik], dt, d_occ + off, rho, true, 1.0, nullptr, 0,
                    ik == ik_grad ? gV : nullptr);
    off += nv[ik];
  }
  cudaStreamSynchronize(c->stream);
  dev_free(d_occ);
  return st;
}

int density(oefe_ctx* c, int nk, const void* const* X, const int* nv, const int* ld, int dtype, const double* occ,
            double* rho) {
  return density_grad(c, nk, X, nv, ld, dtype, occ, rho, -1, nullptr);
}

int band_trace_grad(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double* gV) {
  OEFE_TRY(check_fields(c, ik, X, nv, ld, dtype));
  if (!gV) { c->err = "need gV"; return OEFE_ERR_ARG; }
  OEFE_TRY(run_fields(c, c->kd[ik], X, nv, ld, dtype, nullptr, gV, false));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

// d/dV_q of Re sum conj(G) (H X) = w_q Re sum_v conj(u_G,v(x_q)) u_X,v(x_q), one fields pass over the
// columns of both blocks; scaled by `scale` (the band-trace gradient: G = X, any scale)
int fields_cross(oefe_ctx* c, int ik, const void* X, const void* G, int nv, int ld, int dtype, double scale,
                 double* gV) {
  OEFE_TRY(check_fields(c, ik, X, nv, ld, dtype));
  if (!gV) { c->err = "need gV"; return OEFE_ERR_ARG; }
  if (G) OEFE_TRY(run_fields(c, c->kd[ik], X, nv, ld, dtype, nullptr, gV, false, scale, G, ld));
  else OEFE_TRY(run_fields(c, c->kd[ik], X, nv, ld, dtype, nullptr, gV, false, scale));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}
