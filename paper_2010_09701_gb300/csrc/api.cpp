// extern "C" entry points of liboefe (declared in include/oefe.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include <atomic>

#include "oefe_internal.h"

#define CTX_CHECK(ctx)          \
  do {                          \
    if (!(ctx)) return OEFE_ERR_ARG; \
    cudaSetDevice((ctx)->device);    \
  } while (0)

static void free_all(oefe_ctx* c) {
  for (auto& K : c->kd) {
    dev_free(K.gamma); dev_free(K.Moo); dev_free(K.Mooinv); dev_free(K.H64); dev_free(K.H32); dev_free(K.Hbf); dev_free(K.Hp);
    dev_free(K.E0); dev_free(K.NO); dev_free(K.NOp);
  }
  c->kd.clear();
  void* ptrs[] = {c->d_gll, c->d_m, c->d_cell_nodes, c->d_cellbox, c->d_pos, c->d_lm, c->d_R, c->d_dR,
                  c->d_act_off, c->d_act_idx, c->d_node_off, c->d_node_slot, c->d_enr_off, c->d_enr_slot,
                  c->d_qxyz, c->d_qw, c->d_leaves, c->d_leaf_off, c->d_q_off, c->d_dblk, c->ws, c->ws2,
                  c->d_status};
  for (void* p : ptrs) dev_free(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  for (cudaEvent_t e : c->bev_kernel) cudaEventDestroy(e);
  c->bev_kernel.clear();
  release_batch_graphs(c);
  if (c->bev_in) cudaEventDestroy(c->bev_in);
  if (c->bev_out) cudaEventDestroy(c->bev_out);
  if (c->bstream) cudaStreamDestroy(c->bstream);
  dev_free(c->d_tmaps);
  dev_free(c->d_sf);
  dev_free(c->d_sf_cells);
  dev_free(c->d_dense_cells);
  dev_free(c->d_sf_index);
  dev_free(c->d_dense_index);
  dev_free(c->d_rotp);
  c->d_rotp = nullptr;
  c->rotp_bytes = 0;
  dev_free(c->d_ozpart);
  c->d_ozpart = nullptr;
  c->ozpart_bytes = 0;
  dev_free(c->d_veff);
}

cudaEvent_t timing_event(oefe_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

static std::atomic<long long> g_launches{0};

long long oefe_launch_add(long long n) { return g_launches.fetch_add(n, std::memory_order_relaxed) + n; }

extern "C" {

int oefe_create(oefe_ctx_t* out, int device, void* cuda_stream) {
  if (!out) return OEFE_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return OEFE_ERR_CUDA;
  }
  oefe_ctx* c = new (std::nothrow) oefe_ctx();
  if (!c) return OEFE_ERR_OOM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return OEFE_ERR_CUDA;
  }
  if (dev_alloc(c, (void**)&c->d_status, 64) != OEFE_OK) {
    delete c;
    return OEFE_ERR_OOM;
  }
  cudaMemsetAsync(c->d_status, 0, 64, c->stream);
  *out = c;
  return OEFE_OK;
}

int oefe_destroy(oefe_ctx_t ctx) {
  if (!ctx) return OEFE_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return OEFE_OK;
}

int oefe_set_stream(oefe_ctx_t ctx, void* cuda_stream) {
  CTX_CHECK(ctx);
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = (cudaStream_t)cuda_stream;
  return OEFE_OK;
}

int oefe_last_error(oefe_ctx_t ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return OEFE_ERR_ARG;
  std::strncpy(buf, ctx->err.c_str(), len - 1);
  buf[len - 1] = 0;
  return OEFE_OK;
}

int oefe_mesh(oefe_ctx_t ctx, double a, const int ncell[3], const double* xb, int p) {
  CTX_CHECK(ctx);
  if (!ncell) return OEFE_ERR_ARG;
  return setup_mesh(ctx, a, ncell, xb, p);
}

int oefe_mesh_graded(oefe_ctx_t ctx, double a, int ncell, int p, int natoms, const double* pos, double ratio,
                     double* xb_out) {
  CTX_CHECK(ctx);
  if (ncell < 1 || natoms < 0 || (natoms > 0 && !pos) || !(ratio > 0) || !(a > 0)) {
    ctx->err = "mesh_graded: bad arguments";
    return OEFE_ERR_ARG;
  }
  std::vector<double> xb;
  for (int d = 0; d < 3; ++d) {
    std::vector<double> coords, out;
    for (int I = 0; I < natoms; ++I) coords.push_back(pos[3 * I + d]);
    graded_breakpoints(a, ncell, coords, ratio, out);
    xb.insert(xb.end(), out.begin(), out.end());
  }
  if (xb_out) std::memcpy(xb_out, xb.data(), xb.size() * sizeof(double));
  const int nc[3] = {ncell, ncell, ncell};
  return setup_mesh(ctx, a, nc, xb.data(), p);
}

int oefe_enrichment(oefe_ctx_t ctx, int natoms, const double* pos, int nfun, const int* lm, int ngrid,
                    const double* R, const double* dR, double r0, double rc) {
  CTX_CHECK(ctx);
  return setup_enrichment(ctx, natoms, pos, nfun, lm, ngrid, R, dR, r0, rc);
}

int oefe_quadrature(oefe_ctx_t ctx, int nq_cell, int nq_enr, int depth) {
  CTX_CHECK(ctx);
  return setup_quadrature(ctx, nq_cell, nq_enr, depth);
}

int oefe_quadrature_count(oefe_ctx_t ctx, int64_t* nq_total) {
  CTX_CHECK(ctx);
  if (!ctx->has_quad) { ctx->err = "quadrature not set"; return OEFE_ERR_STATE; }
  if (!nq_total) return OEFE_ERR_ARG;
  *nq_total = ctx->nq;
  return OEFE_OK;
}

int oefe_quadrature_points(oefe_ctx_t ctx, double* xyz, double* w) {
  CTX_CHECK(ctx);
  if (!ctx->has_quad) { ctx->err = "quadrature not set"; return OEFE_ERR_STATE; }
  if (xyz) std::memcpy(xyz, ctx->qxyz.data(), ctx->qxyz.size() * sizeof(double));
  if (w) std::memcpy(w, ctx->qw.data(), ctx->qw.size() * sizeof(double));
  return OEFE_OK;
}

int oefe_kpoints(oefe_ctx_t ctx, int nk, const double* k, const double* w) {
  CTX_CHECK(ctx);
  return setup_kpoints(ctx, nk, k, w);
}

int oefe_ndof(oefe_ctx_t ctx, int64_t* n_h, int* n_O) {
  CTX_CHECK(ctx);
  if (!ctx->has_enr) { ctx->err = "call oefe_enrichment first"; return OEFE_ERR_STATE; }
  if (n_h) *n_h = ctx->nh;
  if (n_O) *n_O = ctx->nO;
  return OEFE_OK;
}

int oefe_build_hamiltonian(oefe_ctx_t ctx, const double* veff_q, int store) {
  CTX_CHECK(ctx);
  return build_hamiltonian(ctx, veff_q, store);
}

int oefe_cell_info(oefe_ctx_t ctx, int cell, int* n_aug, int* idx) {
  CTX_CHECK(ctx);
  if (!ctx->has_enr) { ctx->err = "call oefe_enrichment first"; return OEFE_ERR_STATE; }
  if (cell < 0 || cell >= ctx->ncells || !n_aug) return OEFE_ERR_ARG;
  const int ne = ctx->act_off[cell + 1] - ctx->act_off[cell];
  *n_aug = ctx->nloc + ne;
  if (idx) {
    for (int a = 0; a < ctx->nloc; ++a) idx[a] = ctx->cell_nodes[(size_t)cell * ctx->nloc + a];
    for (int j = 0; j < ne; ++j) idx[ctx->nloc + j] = (int)ctx->nh + ctx->act_idx[ctx->act_off[cell] + j];
  }
  return OEFE_OK;
}

int oefe_cell_matrix(oefe_ctx_t ctx, int ik, int cell, void* H) {
  CTX_CHECK(ctx);
  if (!ctx->built) { ctx->err = "call oefe_build_hamiltonian first"; return OEFE_ERR_STATE; }
  if (ik < 0 || ik >= (int)ctx->kd.size() || cell < 0 || cell >= ctx->ncells || !H) return OEFE_ERR_ARG;
  const KData& K = ctx->kd[ik];
  if (!K.H64) { ctx->err = "FP64 cell matrices were not stored"; return OEFE_ERR_STATE; }
  const int ne = ctx->act_off[cell + 1] - ctx->act_off[cell];
  const int na = ctx->nloc + ne;
  const size_t sb = K.cplx ? 16 : 8;
  size_t slot = (size_t)cell;
  if (K.compact) {   // only the cells with several quadrature leaves are kept whole
    int d = -1;
    OEFE_CUDA_TRY(ctx, cudaMemcpy(&d, ctx->d_dense_index + cell, sizeof(int), cudaMemcpyDeviceToHost));
    if (d < 0) {
      ctx->err = "cell_matrix: the compact storage keeps only the enrichment strip of a single-leaf cell";
      return OEFE_ERR_STATE;
    }
    slot = (size_t)d;
  }
  const char* src = (const char*)K.H64 + slot * ctx->npad * ctx->npad * sb;
  OEFE_CUDA_TRY(ctx, cudaMemcpy2DAsync(H, na * sb, src, ctx->npad * sb, na * sb, na, cudaMemcpyDeviceToHost,
                                       ctx->stream));
  OEFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return OEFE_OK;
}

int oefe_overlap(oefe_ctx_t ctx, int ik, double* m, void* Moo) {
  CTX_CHECK(ctx);
  if (!ctx->has_k) { ctx->err = "call oefe_kpoints first"; return OEFE_ERR_STATE; }
  if (ik < 0 || ik >= (int)ctx->kd.size()) return OEFE_ERR_ARG;
  const KData& K = ctx->kd[ik];
  if (m) OEFE_CUDA_TRY(ctx, cudaMemcpyAsync(m, ctx->d_m, ctx->nh * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (Moo && ctx->nO > 0)
    OEFE_CUDA_TRY(ctx, cudaMemcpyAsync(Moo, K.Moo, (size_t)ctx->nO * ctx->nO * (K.cplx ? 16 : 8),
                                       cudaMemcpyDeviceToHost, ctx->stream));
  OEFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return OEFE_OK;
}

int oefe_apply_h(oefe_ctx_t ctx, int ik, const void* X, void* Y, int nv, int ld, int dtype) {
  CTX_CHECK(ctx);
  return apply_op(ctx, ik, X, Y, nv, ld, dtype, false);
}

int oefe_apply_a(oefe_ctx_t ctx, int ik, const void* X, void* Y, int nv, int ld, int dtype) {
  CTX_CHECK(ctx);
  return apply_op(ctx, ik, X, Y, nv, ld, dtype, true);
}

int oefe_apply_a_noalloc(oefe_ctx_t ctx, int ik, const void* X, void* Y, int nv, int ld, int dtype) {
  CTX_CHECK(ctx);
  return apply_a_noalloc(ctx, ik, X, Y, nv, ld, dtype);
}

int oefe_chebyshev_filter(oefe_ctx_t ctx, int ik, void* X, int nv, int ld, int dtype, int degree, double a, double b,
                          double a0, int flags) {
  CTX_CHECK(ctx);
  return cheb_filter(ctx, ik, X, nv, ld, dtype, degree, a, b, a0, flags);
}

int oefe_filter_batched(oefe_ctx_t ctx, int nk, void* const* X, const int* nv, const int* ld, int dtype, int degree,
                        const double* a, const double* b, const double* a0, int flags) {
  CTX_CHECK(ctx);
  return cheb_filter_batched(ctx, nk, X, nv, ld, dtype, degree, a, b, a0, flags);
}

int oefe_filter_batched_defect(oefe_ctx_t ctx, int nk, void* const* X, const int* nv, const int* ld, int dtype,
                               int degree, const double* a, const double* b, const double* a0, const double* theta,
                               int flags) {
  CTX_CHECK(ctx);
  return cheb_filter_batched_defect(ctx, nk, X, nv, ld, dtype, degree, a, b, a0, theta, flags);
}

int oefe_filter_autotune(oefe_ctx_t ctx, int nk, void* const* X, const int* nv, const int* ld, int dtype, double* ms) {
  CTX_CHECK(ctx);
  return filter_autotune(ctx, nk, X, nv, ld, dtype, ms);
}

int oefe_orthonormalize(oefe_ctx_t ctx, int ik, void* X, int nv, int ld, int dtype, double* cond_est) {
  CTX_CHECK(ctx);
  return orthonormalize(ctx, ik, X, nv, ld, dtype, cond_est);
}

int oefe_rayleigh_ritz(oefe_ctx_t ctx, int ik, void* X, int nv, int ld, int dtype, double* eig, double* resid) {
  CTX_CHECK(ctx);
  return rayleigh_ritz(ctx, ik, X, nv, ld, dtype, eig, resid);
}

int oefe_density(oefe_ctx_t ctx, int nk, const void* const* X, const int* nv, const int* ld, int dtype,
                 const double* occ, double* rho) {
  CTX_CHECK(ctx);
  return density(ctx, nk, X, nv, ld, dtype, occ, rho);
}

int oefe_density_grad(oefe_ctx_t ctx, int nk, const void* const* X, const int* nv, const int* ld, int dtype,
                      const double* occ, double* rho, int ik, double* gV) {
  CTX_CHECK(ctx);
  if (!gV) { ctx->err = "density_grad: need gV"; return OEFE_ERR_ARG; }
  return density_grad(ctx, nk, X, nv, ld, dtype, occ, rho, ik, gV);
}

int oefe_band_trace_grad(oefe_ctx_t ctx, int ik, const void* X, int nv, int ld, int dtype, double* gV) {
  CTX_CHECK(ctx);
  return band_trace_grad(ctx, ik, X, nv, ld, dtype, gV);
}

int oefe_band_trace(oefe_ctx_t ctx, int ik, const void* X, int nv, int ld, int dtype, double* e, void* HX) {
  CTX_CHECK(ctx);
  return band_trace(ctx, ik, X, nv, ld, dtype, e, HX);
}

int oefe_band_trace_vjp(oefe_ctx_t ctx, int ik, const void* X, int nv, int ld, int dtype, double alpha, double* gV,
                        void* gX) {
  CTX_CHECK(ctx);
  return band_trace_vjp(ctx, ik, X, nv, ld, dtype, alpha, gV, gX);
}

int oefe_apply_h_vjp(oefe_ctx_t ctx, int ik, const void* X, const void* Gy, double* gV, void* gX, int nv, int ld,
                     int dtype) {
  CTX_CHECK(ctx);
  return apply_h_vjp(ctx, ik, X, Gy, gV, gX, nv, ld, dtype);
}

int oefe_upper_bound(oefe_ctx_t ctx, int ik, const void* v0, int steps, int flags, double* b) {
  CTX_CHECK(ctx);
  return upper_bound(ctx, ik, v0, steps, flags, b);
}

int oefe_kernel_timing(oefe_ctx_t ctx, int dtype_mask) {
  CTX_CHECK(ctx);
  cudaStreamSynchronize(ctx->stream);
  ctx->timing = dtype_mask & 15;
  if (ctx->timing) {
    ctx->ev_used = 0;
    ctx->timing_extra_ms = 0;
    ctx->timing_extra_n = 0;
  }
  return OEFE_OK;
}

int oefe_occupations(int nk, const int* nv, const double* eig, const double* w, double n_electrons,
                     double temperature, double* occ, double* mu, double* e_band) {
  if (nk < 1 || !nv || !eig || !w || !occ || !(temperature > 0) || !(n_electrons >= 0)) return OEFE_ERR_ARG;
  int tot = 0;
  for (int k = 0; k < nk; ++k) {
    if (nv[k] < 0) return OEFE_ERR_ARG;
    tot += nv[k];
  }
  if (tot == 0) return OEFE_ERR_ARG;
  double wsum_states = 0;
  for (int k = 0, o = 0; k < nk; o += nv[k], ++k) wsum_states += 2.0 * w[k] * nv[k];
  if (n_electrons > wsum_states) return OEFE_ERR_ARG;
  const double kT = 3.166811563e-6 * temperature;
  double lo = eig[0], hi = eig[0];
  for (int i = 0; i < tot; ++i) { lo = std::min(lo, eig[i]); hi = std::max(hi, eig[i]); }
  lo -= 1.0;
  hi += 1.0;
  auto fermi = [&](double e, double m) { return 0.5 * (1.0 - std::tanh(0.5 * (e - m) / kT)); };
  auto count = [&](double m) {
    double s = 0;
    for (int k = 0, o = 0; k < nk; o += nv[k], ++k)
      for (int a = 0; a < nv[k]; ++a) s += 2.0 * w[k] * fermi(eig[o + a], m);
    return s;
  };
  double m = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    m = 0.5 * (lo + hi);
    const double n = count(m);
    if (std::fabs(n - n_electrons) < 1e-12) break;
    if (n < n_electrons) lo = m; else hi = m;
  }
  double eb = 0;
  for (int k = 0, o = 0; k < nk; o += nv[k], ++k)
    for (int a = 0; a < nv[k]; ++a) {
      const double f = fermi(eig[o + a], m);
      occ[o + a] = 2.0 * w[k] * f;
      eb += 2.0 * w[k] * f * eig[o + a];
    }
  if (mu) *mu = m;
  if (e_band) *e_band = eb;
  return OEFE_OK;
}

int oefe_release_workspace(oefe_ctx_t ctx) {
  CTX_CHECK(ctx);
  OEFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->bstream) OEFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->bstream));
  release_batch_graphs(ctx);   // they point into the workspace
  dev_free(ctx->ws);
  dev_free(ctx->ws2);
  ctx->ws = ctx->ws2 = nullptr;
  ctx->ws_bytes = ctx->ws2_bytes = 0;
  dev_free(ctx->d_ozpart);   // digit planes of the tensor-core Gram matrices and rotations
  ctx->d_ozpart = nullptr;
  ctx->ozpart_bytes = 0;
  dev_free(ctx->d_rotp);
  ctx->d_rotp = nullptr;
  ctx->rotp_bytes = 0;
  return OEFE_OK;
}

int oefe_product_flops(oefe_ctx_t ctx, int ik, int nv, double* flops) {
  CTX_CHECK(ctx);
  if (!ctx->has_quad || ik < 0 || ik >= (int)ctx->kd.size() || nv < 1 || !flops) return OEFE_ERR_ARG;
  *flops = fp64_product_flops(ctx, ctx->kd[ik].cplx, nv);
  return OEFE_OK;
}

int oefe_set_f64_products(oefe_ctx_t ctx, int mode) {
  CTX_CHECK(ctx);
  if (mode != OEFE_F64_NATIVE && mode != OEFE_F64_PAIRS) {
    ctx->err = "set_f64_products: mode must be OEFE_F64_NATIVE or OEFE_F64_PAIRS";
    return OEFE_ERR_ARG;
  }
  ctx->f64_products = mode;
  return OEFE_OK;
}

int oefe_set_product_shape(oefe_ctx_t ctx, int shape) {
  CTX_CHECK(ctx);
  if (shape < -1 || shape > 2) {
    ctx->err = "set_product_shape: shape must be -1 (timed at first use), 0, 1 or 2";
    return OEFE_ERR_ARG;
  }
  ctx->sf_variant = shape;
  return OEFE_OK;
}

int oefe_set_filter_shape(oefe_ctx_t ctx, int shape) {
  CTX_CHECK(ctx);
  return filter_set_shape(ctx, shape);
}

int oefe_launch_count(int64_t* n) {
  if (!n) return OEFE_ERR_ARG;
  *n = (int64_t)g_launches.load(std::memory_order_relaxed);
  return OEFE_OK;
}

int oefe_kernel_time(oefe_ctx_t ctx, double* ms, int64_t* launches) {
  CTX_CHECK(ctx);
  if (!ms || !launches) return OEFE_ERR_ARG;
  OEFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  double total = 0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float t = 0;
    OEFE_CUDA_TRY(ctx, cudaEventElapsedTime(&t, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
    total += t;
  }
  *ms = total + ctx->timing_extra_ms;
  *launches = (int64_t)(ctx->ev_used / 2) + ctx->timing_extra_n;
  return OEFE_OK;
}

}  // extern "C"
