// Application of H^O and of A = (M^O)^{-1} H^O, and the Chebyshev filter
// (Sec. IV). One filter degree is three kernels:
//   1. cell apply: gather X rows of a cell (its nodes, then its active
//      enrichment functions), Z_e = H^O_e X_e, write the cell product;
//   2. node update: for every global node sum the products of the cells that
//      share it, divide by the lumped mass (Eq. MOEFEInv, diagonal block) and
//      apply the three-term recurrence in the same pass;
//   3. enrichment update: reduce the enrichment rows over cells, apply the
//      dense FP64 (M^oo)^{-1} (Eq. MOEFEInv) and the recurrence.
#include <algorithm>
#include <cmath>

#include "oefe_internal.h"

namespace {

template <typename T> struct cplx { T x, y; };

template <typename T, bool C> struct Sc;
template <typename T> struct Sc<T, false> {
  using type = T;
  __device__ static T zero() { return T(0); }
  __device__ static T fma(T a, T b, T acc) { return a * b + acc; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T scale(T a, double s) { return (T)(a * (T)s); }
};
template <typename T> struct Sc<T, true> {
  using type = cplx<T>;
  __device__ static cplx<T> zero() { return {T(0), T(0)}; }
  __device__ static cplx<T> fma(cplx<T> a, cplx<T> b, cplx<T> acc) {
    return {acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x};
  }
  __device__ static cplx<T> add(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
  __device__ static cplx<T> scale(cplx<T> a, double s) { return {(T)(a.x * (T)s), (T)(a.y * (T)s)}; }
};

constexpr int NB = 32;     // columns per CTA of the cell apply (one per lane)
constexpr int CWARPS = 8;  // warps per CTA

// Z[e][r][v] = sum_k H_e[r][k] X[idx_e(k)][v] for one cell and one column block.
template <typename T, bool C>
__global__ void __launch_bounds__(CWARPS * 32) k_cell_apply(const typename Sc<T, C>::type* __restrict__ H,
                                                            const typename Sc<T, C>::type* __restrict__ X,
                                                            int ldx, int nv, const int* __restrict__ cell_nodes,
                                                            const int* __restrict__ act_off,
                                                            const int* __restrict__ act_idx, int nloc, int npad,
                                                            int64_t nh, typename Sc<T, C>::type* __restrict__ Z) {
  using S = typename Sc<T, C>::type;
  extern __shared__ unsigned char smem_raw[];
  S* Xs = reinterpret_cast<S*>(smem_raw);  // npad x NB
  const int e = blockIdx.x;
  const int v0 = blockIdx.y * NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ne = act_off[e + 1] - act_off[e];
  const int naug = nloc + ne;
  // gather X rows of the cell
  for (int r = warp; r < npad; r += CWARPS) {
    S val = Sc<T, C>::zero();
    if (r < naug && v0 + lane < nv) {
      const int64_t row = r < nloc ? (int64_t)cell_nodes[(size_t)e * nloc + r] : nh + act_idx[act_off[e] + r - nloc];
      val = X[row * ldx + v0 + lane];
    }
    Xs[r * NB + lane] = val;
  }
  __syncthreads();
  const S* He = H + (size_t)e * npad * npad;
  for (int r = warp; r < naug; r += CWARPS) {
    const S* hr = He + (size_t)r * npad;
    S acc = Sc<T, C>::zero();
    for (int k0 = 0; k0 < naug; k0 += 32) {
      const S hk = (k0 + lane < npad) ? hr[k0 + lane] : Sc<T, C>::zero();
      const int kmax = min(32, naug - k0);
      for (int kk = 0; kk < kmax; ++kk) {
        S h;
        if constexpr (C) {
          h.x = __shfl_sync(0xffffffffu, hk.x, kk);
          h.y = __shfl_sync(0xffffffffu, hk.y, kk);
        } else {
          h = __shfl_sync(0xffffffffu, hk, kk);
        }
        acc = Sc<T, C>::fma(h, Xs[(k0 + kk) * NB + lane], acc);
      }
    }
    if (v0 + lane < nv) Z[((size_t)e * npad + r) * nv + v0 + lane] = acc;
  }
}

// Node rows: y = sum of cell products; then
//   mode 0: Y = y; mode 1: Y = y / m; mode 2: Y = alpha (y/m - c X) + beta Xm1.
template <typename T, bool C>
__global__ void k_node_update(const typename Sc<T, C>::type* __restrict__ Z, const int64_t* __restrict__ node_off,
                              const int64_t* __restrict__ node_slot, const double* __restrict__ m, int64_t nh, int nv,
                              int mode, double alpha, double cshift, double beta,
                              const typename Sc<T, C>::type* __restrict__ Xk, int ldk,
                              const typename Sc<T, C>::type* __restrict__ Xm1, int ldm1,
                              typename Sc<T, C>::type* __restrict__ Y, int ldy) {
  using S = typename Sc<T, C>::type;
  const int64_t total = nh * nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = t / nv;
    const int v = (int)(t % nv);
    S y = Sc<T, C>::zero();
    for (int64_t s = node_off[g]; s < node_off[g + 1]; ++s) y = Sc<T, C>::add(y, Z[node_slot[s] * nv + v]);
    if (mode >= 1) y = Sc<T, C>::scale(y, 1.0 / m[g]);
    if (mode == 2) {
      const S xk = Xk[g * ldk + v];
      S out;
      if constexpr (C) {
        out.x = (T)(alpha * ((double)y.x - cshift * (double)xk.x));
        out.y = (T)(alpha * ((double)y.y - cshift * (double)xk.y));
        if (beta != 0.0) {
          const S xm = Xm1[g * ldm1 + v];
          out.x = (T)((double)out.x + beta * (double)xm.x);
          out.y = (T)((double)out.y + beta * (double)xm.y);
        }
      } else {
        out = (T)(alpha * ((double)y - cshift * (double)xk));
        if (beta != 0.0) out = (T)((double)out + beta * (double)Xm1[g * ldm1 + v]);
      }
      y = out;
    }
    Y[g * ldy + v] = y;
  }
}

// Enrichment rows: raw sums over cells (FP64 accumulation).
template <typename T, bool C>
__global__ void k_enr_reduce(const typename Sc<T, C>::type* __restrict__ Z, const int64_t* __restrict__ enr_off,
                             const int64_t* __restrict__ enr_slot, int nO, int nv, cd* __restrict__ Yo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nO * nv) return;
  const int nu = t / nv, v = t % nv;
  double sx = 0, sy = 0;
  for (int64_t s = enr_off[nu]; s < enr_off[nu + 1]; ++s) {
    const auto z = Z[enr_slot[s] * nv + v];
    if constexpr (C) { sx += (double)z.x; sy += (double)z.y; }
    else sx += (double)z;
  }
  Yo[t] = mkc(sx, sy);
}

// Enrichment rows: Y = Yo (mode 0), (M^oo)^{-1} Yo (mode 1), or the recurrence (mode 2).
template <typename T, bool C>
__global__ void k_enr_update(const cd* __restrict__ Yo, const void* __restrict__ Minv, int nO, int nv, int64_t nh,
                             int mode, double alpha, double cshift, double beta,
                             const typename Sc<T, C>::type* __restrict__ Xk, int ldk,
                             const typename Sc<T, C>::type* __restrict__ Xm1, int ldm1,
                             typename Sc<T, C>::type* __restrict__ Y, int ldy) {
  using S = typename Sc<T, C>::type;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nO * nv) return;
  const int nu = t / nv, v = t % nv;
  cd y = Yo[t];
  if (mode >= 1) {
    cd s = mkc(0, 0);
    for (int mu = 0; mu < nO; ++mu) {
      const cd yo = Yo[mu * nv + v];
      if constexpr (C) s += reinterpret_cast<const cd*>(Minv)[nu * nO + mu] * yo;
      else s += reinterpret_cast<const double*>(Minv)[nu * nO + mu] * yo;
    }
    y = s;
  }
  const int64_t row = nh + nu;
  if (mode == 2) {
    const S xk = Xk[row * ldk + v];
    double xr, xi = 0;
    if constexpr (C) { xr = (double)xk.x; xi = (double)xk.y; } else xr = (double)xk;
    cd out = mkc(alpha * (y.x - cshift * xr), alpha * (y.y - cshift * xi));
    if (beta != 0.0) {
      const S xm = Xm1[row * ldm1 + v];
      if constexpr (C) out += mkc(beta * (double)xm.x, beta * (double)xm.y);
      else out.x += beta * (double)xm;
    }
    y = out;
  }
  if constexpr (C) Y[row * ldy + v] = S{(T)y.x, (T)y.y};
  else Y[row * ldy + v] = (T)y.x;
}

// Y (ldy) <- X (ldx) with a precision change; n rows of nv scalars (reals counted by `width`).
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ X, int ldx, B* __restrict__ Y, int ldy, int64_t n, int width) {
  const int64_t total = n * width;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / width;
    const int c = (int)(t % width);
    Y[r * ldy + c] = (B)X[r * ldx + c];
  }
}

template <typename A, typename B>
int convert(oefe_ctx* c, const void* X, int ldx, void* Y, int ldy, int64_t n, int width) {
  const int64_t tot = n * width;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
  k_convert<A, B><<<blocks, 256, 0, c->stream>>>((const A*)X, ldx, (B*)Y, ldy, n, width);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

struct Step {
  int mode;  // 0 H X, 1 M^-1 H X, 2 recurrence
  double alpha, cshift, beta;
};

template <typename T, bool C>
int launch_step(oefe_ctx* c, const KData& K, int dtype, const void* Hm, const void* Xin, int ldin, int nv, const Step& st,
                const void* Xk, int ldk, const void* Xm1, int ldm1, void* Y, int ldy, void* Zbuf, cd* Yo, bool mma) {
  using S = typename Sc<T, C>::type;
  if ((c->timing >> dtype) & 1) cudaEventRecord(timing_event(c), c->stream);
  if (mma) {
    OEFE_TRY(launch_cell_mma(c, K, Xin, ldin, nv, C, Zbuf));
  } else {
    dim3 grid(c->ncells, (nv + NB - 1) / NB);
    const size_t smem = (size_t)c->npad * NB * sizeof(S);
    if (smem > 227 * 1024) { c->err = "cell matrices too large for the shared-memory gather"; return OEFE_ERR_ARG; }
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_apply<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_cell_apply<T, C><<<grid, CWARPS * 32, smem, c->stream>>>((const S*)Hm, (const S*)Xin, ldin, nv, c->d_cell_nodes,
                                                               c->d_act_off, c->d_act_idx, c->nloc, c->npad, c->nh,
                                                               (S*)Zbuf);
  }
  if ((c->timing >> dtype) & 1) cudaEventRecord(timing_event(c), c->stream);
  const int64_t tot = c->nh * nv;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
  k_node_update<T, C><<<blocks, 256, 0, c->stream>>>((const S*)Zbuf, c->d_node_off, c->d_node_slot, c->d_m, c->nh,
                                                     nv, st.mode, st.alpha, st.cshift, st.beta, (const S*)Xk, ldk,
                                                     (const S*)Xm1, ldm1, (S*)Y, ldy);
  if (c->nO > 0) {
    const int eb = (c->nO * nv + 127) / 128;
    k_enr_reduce<T, C><<<eb, 128, 0, c->stream>>>((const S*)Zbuf, c->d_enr_off, c->d_enr_slot, c->nO, nv, Yo);
    k_enr_update<T, C><<<eb, 128, 0, c->stream>>>(Yo, K.Mooinv, c->nO, nv, c->nh, st.mode, st.alpha, st.cshift,
                                                  st.beta, (const S*)Xk, ldk, (const S*)Xm1, ldm1, (S*)Y, ldy);
  }
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

int dispatch_step(oefe_ctx* c, const KData& K, int dtype, const void* Xin, int ldin, int nv, const Step& st,
                  const void* Xk, int ldk, const void* Xm1, int ldm1, void* Y, int ldy, void* Zbuf, cd* Yo,
                  bool mma = false) {
  switch (dtype) {
    case OEFE_F64: return launch_step<double, false>(c, K, dtype, K.H64, Xin, ldin, nv, st, Xk, ldk, Xm1, ldm1, Y, ldy, Zbuf, Yo, false);
    case OEFE_C128: return launch_step<double, true>(c, K, dtype, K.H64, Xin, ldin, nv, st, Xk, ldk, Xm1, ldm1, Y, ldy, Zbuf, Yo, false);
    case OEFE_F32: return launch_step<float, false>(c, K, dtype, K.H32, Xin, ldin, nv, st, Xk, ldk, Xm1, ldm1, Y, ldy, Zbuf, Yo, mma);
    case OEFE_C64: return launch_step<float, true>(c, K, dtype, K.H32, Xin, ldin, nv, st, Xk, ldk, Xm1, ldm1, Y, ldy, Zbuf, Yo, mma);
  }
  c->err = "unknown dtype";
  return OEFE_ERR_ARG;
}

int check_apply_args(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, bool mma = false) {
  if (!c->built) { c->err = "call oefe_build_hamiltonian first"; return OEFE_ERR_STATE; }
  if (ik < 0 || ik >= (int)c->kd.size()) { c->err = "k index out of range"; return OEFE_ERR_ARG; }
  if (!X || nv < 1 || ld < nv || nv > 8192) { c->err = "need X, 1 <= nv <= ld, nv <= 8192"; return OEFE_ERR_ARG; }
  if (dtype < 0 || dtype > 3) { c->err = "unknown dtype"; return OEFE_ERR_ARG; }
  const KData& K = c->kd[ik];
  if (K.cplx != dtype_complex(dtype)) {
    c->err = K.cplx ? "k != 0 needs a complex dtype" : "k = 0 needs a real dtype";
    return OEFE_ERR_ARG;
  }
  if (dtype_fp64(dtype) && !K.H64) { c->err = "FP64 cell matrices were not stored"; return OEFE_ERR_STATE; }
  if (!dtype_fp64(dtype) && !mma && !K.H32) { c->err = "FP32 cell matrices were not stored"; return OEFE_ERR_STATE; }
  if (mma && !K.Hbf) { c->err = "BF16x3 cell matrices were not stored"; return OEFE_ERR_STATE; }
  return OEFE_OK;
}

}  // namespace

int apply_op2(oefe_ctx* c, int ik, const void* X, int ldx, void* Y, int ldy, int nv, int dtype, bool minv) {
  OEFE_TRY(check_apply_args(c, ik, X, nv, std::min(ldx, ldy), dtype));
  if (!Y) { c->err = "need Y"; return OEFE_ERR_ARG; }
  const size_t es = dtype_bytes(dtype);
  const size_t zbytes = (((size_t)c->ncells * c->npad * nv * es + 255) / 256) * 256;
  const size_t yobytes = (size_t)std::max(c->nO, 1) * nv * sizeof(cd);
  OEFE_TRY(ensure_ws(c, zbytes + yobytes + 256));
  char* base = (char*)c->ws;
  Step st{minv ? 1 : 0, 1.0, 0.0, 0.0};
  OEFE_TRY(dispatch_step(c, c->kd[ik], dtype, X, ldx, nv, st, nullptr, 0, nullptr, 0, Y, ldy, base, (cd*)(base + zbytes)));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

int apply_op(oefe_ctx* c, int ik, const void* X, void* Y, int nv, int ld, int dtype, bool minv) {
  return apply_op2(c, ik, X, ld, Y, ld, nv, dtype, minv);
}

namespace {

// Degrees [j0, j1] of the scaled recurrence on buffers of one dtype. bufs[ip]
// holds Y_{j0-2} (ignored when j0 == 1), bufs[ic] Y_{j0-1}; on return *ip and
// *ic point at Y_{j1-1} and Y_{j1}.
int run_degrees(oefe_ctx* c, const KData& K, int dtype, void* bufs[3], int lds[3], int* ip, int* ic, int nv,
                int j0, int j1, double e, double cc, double* sigma, double sigma1, void* Zb, cd* Yo, bool mma) {
  const double gamma = 2.0 / sigma1;
  for (int j = j0; j <= j1; ++j) {
    Step st;
    if (j == 1) {
      st = Step{2, sigma1 / e, cc, 0.0};
    } else {
      const double sigma2 = 1.0 / (gamma - *sigma);
      st = Step{2, 2.0 * sigma2 / e, cc, -(*sigma) * sigma2};
      *sigma = sigma2;
    }
    const int in = 3 - *ip - *ic;
    OEFE_TRY(dispatch_step(c, K, dtype, bufs[*ic], lds[*ic], nv, st, bufs[*ic], lds[*ic], j == 1 ? nullptr : bufs[*ip],
                           lds[*ip], bufs[in], lds[in], Zb, Yo, mma));
    *ip = *ic;
    *ic = in;
  }
  return OEFE_OK;
}

size_t align256(size_t b) { return ((b + 255) / 256) * 256; }

}  // namespace

int cheb_filter(oefe_ctx* c, int ik, void* X, int nv, int ld, int dtype, int degree, double a, double b,
                double a0, int flags) {
  const bool mma = (flags & OEFE_FILTER_BF16X3) != 0;
  const bool mixed = (flags & OEFE_FILTER_LAST_FP64) != 0;
  OEFE_TRY(check_apply_args(c, ik, X, nv, ld, dtype, mma && !mixed));
  if (degree < 1 || !(b > a) || !(a0 < a)) { c->err = "filter: need degree >= 1, a0 < a < b"; return OEFE_ERR_ARG; }
  if (mma && !c->kd[ik].Hbf) { c->err = "filter: BF16X3 needs the BF16x3 cell matrices"; return OEFE_ERR_STATE; }
  if (mixed && !dtype_fp64(dtype)) {
    c->err = "filter: LAST_FP64 needs F64/C128 storage";
    return OEFE_ERR_ARG;
  }
  const KData& K = c->kd[ik];
  if (mixed && !mma && !K.H32) { c->err = "filter: LAST_FP64 needs the FP32 cell matrices"; return OEFE_ERR_STATE; }
  const int64_t n = c->nh + c->nO;
  const int dt32 = dtype == OEFE_C128 ? OEFE_C64 : OEFE_F32;
  const int width = dtype_complex(dtype) ? 2 * nv : nv;  // reals per row
  const size_t es = dtype_bytes(dtype);
  const size_t es_low = mixed ? dtype_bytes(dt32) : es;
  const size_t zbytes = align256((size_t)c->ncells * c->npad * nv * std::max(es, es_low));
  const size_t yobytes = align256((size_t)std::max(c->nO, 1) * nv * sizeof(cd));
  const size_t vbytes = align256((size_t)n * nv * es);
  const size_t vbytes_low = align256((size_t)n * nv * es_low);
  OEFE_TRY(ensure_ws(c, zbytes + yobytes + 2 * vbytes + (mixed ? 3 * vbytes_low : 0)));
  char* base = (char*)c->ws;
  void* Zb = base;
  cd* Yo = (cd*)(base + zbytes);
  void* B1 = base + zbytes + yobytes;
  void* B2 = base + zbytes + yobytes + vbytes;
  const double e = (b - a) / 2.0, cc = (b + a) / 2.0;
  const double sigma1 = e / (a0 - cc);
  double sigma = sigma1;
  void* bufs[3] = {X, B1, B2};
  int lds[3] = {ld, nv, nv};
  int ip = 1, ic = 0;
  if (!mixed || degree == 1) {
    OEFE_TRY(run_degrees(c, K, dtype, bufs, lds, &ip, &ic, nv, 1, degree, e, cc, &sigma, sigma1, Zb, Yo,
                         mma && !dtype_fp64(dtype)));
  } else {
    // degrees 1 .. m-1 in FP32 on private buffers, the last degree in FP64
    char* lowb = base + zbytes + yobytes + 2 * vbytes;
    void* L[3] = {lowb, lowb + vbytes_low, lowb + 2 * vbytes_low};
    int ldl[3] = {nv, nv, nv};
    if (dtype == OEFE_C128 || dtype == OEFE_F64) OEFE_TRY((convert<double, float>(c, X, ld * (dtype == OEFE_C128 ? 2 : 1), L[0], width, n, width)));
    int lp = 1, lc = 0;
    OEFE_TRY(run_degrees(c, K, dt32, L, ldl, &lp, &lc, nv, 1, degree - 1, e, cc, &sigma, sigma1, Zb, Yo, mma));
    // Y_{m-1} -> B1 (FP64); Y_{m-2} -> B2 (FP64), or X itself when m == 2
    OEFE_TRY((convert<float, double>(c, L[lc], width, B1, width, n, width)));
    int fp = 0;
    if (degree > 2) {
      OEFE_TRY((convert<float, double>(c, L[lp], width, B2, width, n, width)));
      fp = 2;
    }
    // last degree: inputs B1 (current) and bufs[fp] (previous), output X (or B2 when fp == 0)
    ip = fp;
    ic = 1;
    OEFE_TRY(run_degrees(c, K, dtype, bufs, lds, &ip, &ic, nv, degree, degree, e, cc, &sigma, sigma1, Zb, Yo, false));
  }
  if (ic != 0) {
    OEFE_CUDA_TRY(c, cudaMemcpy2DAsync(X, (size_t)ld * es, bufs[ic], (size_t)lds[ic] * es, (size_t)nv * es, (size_t)n,
                                       cudaMemcpyDeviceToDevice, c->stream));
  }
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (mma) {
    int flag = 0;
    OEFE_CUDA_TRY(c, cudaMemcpy(&flag, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      cudaMemset(c->d_status, 0, sizeof(int));
      c->err = "filter: a tensor-core pipeline wait timed out";
      return OEFE_ERR_TIMEOUT;
    }
  }
  return OEFE_OK;
}
