// The band trace E = tr(X^+ H^O X) and the adjoints of the cell-level application Y = H^O(V) X
// (H^O affine in the quadrature-point potential V through the (|k|^2/2 + V) N_m^* N_n term of
// Eq. HOEFEelelements, Hermitian):
//   dE/dV_q = w_q sum_v |u_v(x_q)|^2,              dE/dX (torch's convention) = 2 H^O X;
//   for a cotangent G of Y: d/dV_q = w_q Re sum_v conj(u_G,v(x_q)) u_X,v(x_q),   d/dX = H^O G,
// with u the field of a column at the quadrature points (Eq. UOEFE). The fields are recomputed
// from the vectors (no gathers are stored); every reduction runs on the GPU in a fixed order.
#include <algorithm>

#include "oefe_internal.h"

int fields_cross(oefe_ctx* c, int ik, const void* X, const void* G, int nv, int ld, int dtype, double scale,
                 double* gV);

namespace {

constexpr int RB = 256;      // threads per block of the reductions
constexpr int RPARTS = 1024; // partial sums of the first stage

// part[b] = Re sum over the rows of block-stride b of sum_v conj(X_rv) Y_rv (real views: x_r y_r + x_i y_i)
__global__ void k_trace_partial(const double* __restrict__ X, int ldx, const double* __restrict__ Y, int ldy,
                                int64_t n, int width, double* __restrict__ part) {
  __shared__ double red[RB];
  double s = 0.0;
  const int64_t total = n * width;
  for (int64_t t = blockIdx.x * (int64_t)RB + threadIdx.x; t < total; t += (int64_t)gridDim.x * RB) {
    const int64_t r = t / width;
    const int f = (int)(t % width);
    s = fma(X[r * ldx + f], Y[r * ldy + f], s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_trace_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[RB];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += RB) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Y <- alpha Y (real view, rows of `width` reals)
__global__ void k_scale_rows(double* __restrict__ Y, int ldy, int64_t n, int width, double alpha) {
  const int64_t total = n * width;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / width;
    const int f = (int)(t % width);
    Y[r * ldy + f] *= alpha;
  }
}

int check_fp64_block(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype) {
  if (!c->built) { c->err = "call oefe_build_hamiltonian first"; return OEFE_ERR_STATE; }
  if (ik < 0 || ik >= (int)c->kd.size()) { c->err = "k index out of range"; return OEFE_ERR_ARG; }
  if (!X || nv < 1 || ld < nv) { c->err = "need X and 1 <= nv <= ld"; return OEFE_ERR_ARG; }
  if (!(dtype == OEFE_F64 || dtype == OEFE_C128)) { c->err = "this call needs F64 or C128 vectors"; return OEFE_ERR_ARG; }
  if (c->kd[ik].cplx != (dtype == OEFE_C128)) { c->err = "dtype does not match the k-point"; return OEFE_ERR_ARG; }
  return OEFE_OK;
}

}  // namespace

int band_trace(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double* e, void* HX) {
  OEFE_TRY(check_fp64_block(c, ik, X, nv, ld, dtype));
  if (!e) { c->err = "band_trace: need e"; return OEFE_ERR_ARG; }
  const int64_t n = c->nh + c->nO;
  const int R = dtype == OEFE_C128 ? 2 : 1;
  const size_t es = dtype_bytes(dtype);
  const size_t hbytes = ((size_t)n * nv * es + 255) / 256 * 256;
  // H X into the caller's buffer (leading dimension ld), or into the second workspace (nv)
  OEFE_TRY(ensure_ws2(c, (HX ? 0 : hbytes) + (RPARTS + 8) * sizeof(double)));
  void* Y = HX ? HX : c->ws2;
  const int ldy = HX ? ld : nv;
  double* part = (double*)((char*)c->ws2 + (HX ? 0 : hbytes));
  OEFE_TRY(apply_op2(c, ik, X, ld, Y, ldy, nv, dtype, false));
  const int W = nv * R;
  const int nb = (int)std::min<int64_t>(RPARTS, std::max<int64_t>(1, (n * W + RB - 1) / RB));
  OEFE_COUNTED k_trace_partial<<<nb, RB, 0, c->stream>>>((const double*)X, ld * R, (const double*)Y, ldy * R, n, W, part);
  OEFE_COUNTED k_trace_final<<<1, RB, 0, c->stream>>>(part, nb, part + RPARTS);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(e, part + RPARTS, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

int band_trace_vjp(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, double alpha, double* gV,
                   void* gX) {
  OEFE_TRY(check_fp64_block(c, ik, X, nv, ld, dtype));
  if (!gV && !gX) { c->err = "band_trace_vjp: need gV or gX"; return OEFE_ERR_ARG; }
  if (gV) OEFE_TRY(fields_cross(c, ik, X, nullptr, nv, ld, dtype, alpha, gV));
  if (gX) {
    OEFE_TRY(apply_op2(c, ik, X, ld, gX, ld, nv, dtype, false));
    const int64_t n = c->nh + c->nO;
    const int R = dtype == OEFE_C128 ? 2 : 1;
    const int64_t tot = n * nv * R;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
    OEFE_COUNTED k_scale_rows<<<blocks, 256, 0, c->stream>>>((double*)gX, ld * R, n, nv * R, 2.0 * alpha);
    OEFE_CUDA_TRY(c, cudaGetLastError());
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return OEFE_OK;
}

int apply_h_vjp(oefe_ctx* c, int ik, const void* X, const void* Gy, double* gV, void* gX, int nv, int ld, int dtype) {
  OEFE_TRY(check_fp64_block(c, ik, X, nv, ld, dtype));
  if (!Gy) { c->err = "apply_h_vjp: need Gy"; return OEFE_ERR_ARG; }
  if (!gV && !gX) { c->err = "apply_h_vjp: need gV or gX"; return OEFE_ERR_ARG; }
  if (gV) OEFE_TRY(fields_cross(c, ik, X, Gy, nv, ld, dtype, 1.0, gV));
  if (gX) OEFE_TRY(apply_op2(c, ik, Gy, ld, gX, ld, nv, dtype, false));
  return OEFE_OK;
}
