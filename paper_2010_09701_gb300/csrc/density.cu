// Fields at the quadrature points (Eq. UOEFE, Eq. rho):
//   u(x_q) = sum_a N^C_a(x_q) (X^c - Gamma_e X^o)_a + sum_j N^A_j(x_q) X^o_j
// interpolated per tensor-product leaf by sum factorization, then
//   density:          rho_q += sum_v occ_v |u_v(x_q)|^2
//   band-trace grad:  g_q    = w_q sum_v |u_v(x_q)|^2  (adjoint of H.X w.r.t. V_q).
#include <algorithm>
#include <cmath>

#include "oefe_internal.h"
#include "enrich_dev.cuh"

namespace {

constexpr int MAXP = 8;
constexpr int MAXN1 = 12;
constexpr int DT = 256;

struct FieldArgs {
  EnrParams E;
  const Leaf* leaves;
  const int* leaf_off;
  const double* qxyz;
  const double* qw;
  const double* cellbox;
  const double* gll;
  const int* cell_nodes;
  const int* act_off;
  const int* act_idx;
  int ncells, nleaves, P, nloc, ne_max, nbd;
  int64_t nh;
  double k[3];
  const void* X;      // F64 or C128 rows, ld
  int ld, nv;
  bool cplx;
  const void* gamma;  // (ncells, nloc, ne_max)
  const double* occ;  // nv weights (density) or null (gradient: weight 1, times w_q)
  cd* na;             // per-CTA scratch: max leaf points * ne_max
  int64_t na_stride;
  double* out;        // nq
  bool accumulate;    // density: out += ; gradient: out =
};

__device__ inline cd ldX(const FieldArgs& A, int64_t row, int v) {
  if (A.cplx) return reinterpret_cast<const cd*>(A.X)[row * A.ld + v];
  return mkc(reinterpret_cast<const double*>(A.X)[row * A.ld + v], 0.0);
}
__device__ inline cd ldG(const FieldArgs& A, size_t i) {
  if (A.cplx) return reinterpret_cast<const cd*>(A.gamma)[i];
  return mkc(reinterpret_cast<const double*>(A.gamma)[i], 0.0);
}

__global__ void __launch_bounds__(DT) k_fields(FieldArgs A) {
  extern __shared__ double smem[];
  __shared__ double Lt[3][MAXN1][MAXP];
  __shared__ double xn[MAXP];
  if (threadIdx.x < A.P) xn[threadIdx.x] = A.gll[threadIdx.x];
  const int P = A.P, nloc = A.nloc, NB = A.nbd;
  cd* na = A.na + (size_t)blockIdx.x * A.na_stride;
  // leaves are independent (each owns its points): balance the work over leaves
  for (int li = blockIdx.x; li < A.nleaves; li += gridDim.x) {
    const Leaf L = A.leaves[li];
    const int e = L.cell;
    const int ne = A.act_off[e + 1] - A.act_off[e];
    const double* box = A.cellbox + 6 * e;
    {
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
      // enrichment values of the leaf points, one (point, atom) per thread: the active set holds
      // whole atoms, whose functions share the offset, cutoff and phase
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
      cd* Xt = reinterpret_cast<cd*>(smem);   // nloc * NB
      cd* Xo = Xt + nloc * NB;                // ne_max * NB
      cd* T1 = Xo + A.ne_max * NB;            // n1 * P * P * NB   [qx][b][c][v]
      cd* T2 = T1 + n1 * P * P * NB;          // n2 * P * NB       [qx][qy][c][v]
      cd* U = T2 + n2 * P * NB;               // n3 * NB
      double* rho = reinterpret_cast<double*>(U + n3 * NB);  // n3
      for (int q = threadIdx.x; q < n3; q += DT) rho[q] = 0.0;
      for (int v0 = 0; v0 < A.nv; v0 += NB) {
        const int nb = min(NB, A.nv - v0);
        __syncthreads();
        for (int t = threadIdx.x; t < ne * NB; t += DT) {
          const int j = t / NB, u = t % NB;
          Xo[t] = u < nb ? ldX(A, A.nh + A.act_idx[A.act_off[e] + j], v0 + u) : mkc(0, 0);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nloc * NB; t += DT) {
          const int a = t / NB, u = t % NB;
          cd s = mkc(0, 0);
          if (u < nb) {
            s = ldX(A, A.cell_nodes[(size_t)e * nloc + a], v0 + u);
            for (int j = 0; j < ne; ++j) s = cfma(-ldG(A, ((size_t)e * nloc + a) * A.ne_max + j), Xo[j * NB + u], s);
          }
          Xt[t] = s;
        }
        __syncthreads();
        // x stage: T1[qx][b][c][v] = sum_a Lx[qx][a] Xt[a + P(b + P c)][v]
        for (int t = threadIdx.x; t < n1 * P * P * NB; t += DT) {
          const int u = t % NB, r = t / NB;
          const int c = r % P, bb = (r / P) % P, qx = r / (P * P);
          cd s = mkc(0, 0);
          for (int a = 0; a < P; ++a) s = rfma(Lt[0][qx][a], Xt[(a + P * (bb + P * c)) * NB + u], s);
          T1[t] = s;
        }
        __syncthreads();
        // y stage: T2[qx][qy][c][v] = sum_b Ly[qy][b] T1[qx][b][c][v]
        for (int t = threadIdx.x; t < n2 * P * NB; t += DT) {
          const int u = t % NB, r = t / NB;
          const int c = r % P, qy = (r / P) % n1, qx = r / (P * n1);
          cd s = mkc(0, 0);
          for (int bb = 0; bb < P; ++bb) s = rfma(Lt[1][qy][bb], T1[((qx * P + bb) * P + c) * NB + u], s);
          T2[t] = s;
        }
        __syncthreads();
        // z stage and the enrichment part: U[q][v], q = qx + n1 (qy + n1 qz)
        for (int t = threadIdx.x; t < n3 * NB; t += DT) {
          const int u = t % NB, q = t / NB;
          const int qx = q % n1, qy = (q / n1) % n1, qz = q / n2;
          cd s = mkc(0, 0);
          for (int c = 0; c < P; ++c) s = rfma(Lt[2][qz][c], T2[((qx * n1 + qy) * P + c) * NB + u], s);
          for (int j = 0; j < ne; ++j) s = cfma(na[q * ne + j], Xo[j * NB + u], s);
          U[t] = s;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += DT) {
          double s = 0;
          for (int u = 0; u < nb; ++u) s += (A.occ ? A.occ[v0 + u] : 1.0) * cabs2(U[q * NB + u]);
          rho[q] += s;
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < n3; q += DT) {
        const int64_t qg = L.q0 + q;
        if (A.accumulate) A.out[qg] += rho[q];
        else A.out[qg] = A.qw[qg] * rho[q];
      }
    }
  }
}

size_t field_smem(const oefe_ctx* c, int nb) {
  const int n1 = std::max(c->nq_cell, c->nq_enr), P = c->P;
  const size_t n3 = (size_t)n1 * n1 * n1;
  return ((size_t)c->nloc * nb + (size_t)std::max(c->ne_max, 1) * nb + (size_t)n1 * P * P * nb +
          (size_t)n1 * n1 * P * nb + n3 * nb) * sizeof(cd) + n3 * sizeof(double);
}

int run_fields(oefe_ctx* c, const KData& K, int kidx, const void* X, int nv, int ld, int dtype, const double* occ,
               double* out, bool accumulate) {
  int nb = 8;
  while (nb > 1 && field_smem(c, nb) > 200 * 1024) nb /= 2;
  const size_t smem = field_smem(c, nb);
  if (smem > 220 * 1024) { c->err = "fields: quadrature too large for the interpolation tiles"; return OEFE_ERR_ARG; }
  const int grid = std::max(1, std::min((int)c->leaves.size(), 2 * c->num_sms));
  const int n1 = std::max(c->nq_cell, c->nq_enr);
  const int64_t stride = (int64_t)n1 * n1 * n1 * std::max(c->ne_max, 1);
  OEFE_TRY(ensure_ws2(c, (size_t)grid * stride * sizeof(cd) + 256));
  FieldArgs A;
  A.E.pos = c->d_pos; A.E.lm = c->d_lm; A.E.R = c->d_R; A.E.dR = c->d_dR;
  A.E.nfun = c->nfun; A.E.ngrid = c->ngrid; A.E.a = c->a; A.E.r0 = c->r0; A.E.rc = c->rc;
  A.leaves = c->d_leaves;
  A.leaf_off = c->d_leaf_off;
  A.qxyz = c->d_qxyz;
  A.qw = c->d_qw;
  A.cellbox = c->d_cellbox;
  A.gll = c->d_gll;
  A.cell_nodes = c->d_cell_nodes;
  A.act_off = c->d_act_off;
  A.act_idx = c->d_act_idx;
  A.ncells = c->ncells;
  A.nleaves = (int)c->leaves.size();
  A.P = c->P;
  A.nloc = c->nloc;
  A.ne_max = std::max(c->ne_max, 1);
  A.nbd = nb;
  A.nh = c->nh;
  for (int d = 0; d < 3; ++d) A.k[d] = K.k[d];
  A.X = X;
  A.ld = ld;
  A.nv = nv;
  A.cplx = dtype == OEFE_C128;
  A.gamma = K.gamma;
  A.occ = occ;
  A.na = (cd*)c->ws2;
  A.na_stride = stride;
  A.out = out;
  A.accumulate = accumulate;
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_fields, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  OEFE_COUNTED k_fields<<<grid, DT, smem, c->stream>>>(A);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  (void)kidx;
  return OEFE_OK;
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

int density(oefe_ctx* c, int nk, const void* const* X, const int* nv, const int* ld, int dtype, const double* occ,
            double* rho) {
  if (nk != (int)c->kd.size() || !X || !nv || !ld || !occ || !rho) {
    c->err = "density: need one X, nv, ld per k-point, occ and rho";
    return OEFE_ERR_ARG;
  }
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
    st = run_fields(c, c->kd[ik], ik, X[ik], nv[ik], ld[ik], dt, d_occ + off, rho, true);
    off += nv[ik];
  }
  cudaStreamSynchronize(c->stream);
  dev_free(d_occ);
  return st;
}

int band_trace_grad(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double* gV) {
  OEFE_TRY(check_fields(c, ik, X, nv, ld, dtype));
  if (!gV) { c->err = "need gV"; return OEFE_ERR_ARG; }
  OEFE_TRY(run_fields(c, c->kd[ik], ik, X, nv, ld, dtype, nullptr, gV, false));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}
