// Subspace linear algebra in FP64 (Sec. IV): M-inner-product Gram matrices,
// Cholesky factorization and triangular inverse, Cholesky-QR, Rayleigh-Ritz
// (Eq. ProjKS) and a Lanczos upper bound of the spectrum.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "oefe_internal.h"
#include "pair_dev.cuh"

namespace {

template <typename S> struct Ops;
template <> struct Ops<double> {
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double conj(double a) { return a; }
  __host__ __device__ static double mul(double a, double b) { return a * b; }
  __host__ __device__ static double mulc(double a, double b) { return a * b; }  // conj(a) b
  __host__ __device__ static double re(double a) { return a; }
  __host__ __device__ static double scale(double a, double s) { return a * s; }
};
template <> struct Ops<cd> {
  __host__ __device__ static cd zero() { return mkc(0, 0); }
  __host__ __device__ static cd conj(cd a) { return cconj(a); }
  __host__ __device__ static cd mul(cd a, cd b) { return a * b; }
  __host__ __device__ static cd mulc(cd a, cd b) { return cmulc(a, b); }
  __host__ __device__ static double re(cd a) { return a.x; }
  __host__ __device__ static cd scale(cd a, double s) { return a * s; }
};

// acc += conj(a) b and acc += a b as explicit FMA chains (4 FP64 FMAs per complex product; the
// expression forms would compile to a multiply, an FMA and an add per real part)
__device__ __forceinline__ double fma_c(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ cd fma_c(cd a, cd b, cd acc) {
  return mkc(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double fma_n(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ cd fma_n(cd a, cd b, cd acc) {
  return mkc(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

// In-place lower Cholesky A = L L^+ of an n x n Hermitian matrix (single CTA).
// info = 0 on success, j+1 if the j-th pivot is not positive.
template <typename S>
__global__ void __launch_bounds__(1024) k_chol(S* A, int n, int* info) {
  __shared__ double piv;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = Ops<S>::re(A[(size_t)j * n + j]);
      if (!(d > 0.0) || !isfinite(d)) fail = j + 1;
      else {
        piv = sqrt(d);
        if constexpr (sizeof(S) == 8) A[(size_t)j * n + j] = piv;
        else A[(size_t)j * n + j] = mkc(piv, 0.0);
      }
    }
    __syncthreads();
    if (fail) break;
    const double inv = 1.0 / piv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + j] = Ops<S>::scale(A[(size_t)i * n + j], inv);
    __syncthreads();
    const int m = n - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int ii = t / m, ll = t % m;
      if (ll > ii) continue;
      const int i = j + 1 + ii, l = j + 1 + ll;
      A[(size_t)i * n + l] = A[(size_t)i * n + l] - Ops<S>::mul(A[(size_t)i * n + j], Ops<S>::conj(A[(size_t)l * n + j]));
    }
    __syncthreads();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, l = t % n;
    if (l > i) A[t] = Ops<S>::zero();
  }
  if (threadIdx.x == 0) *info = fail;
}

// Y = L^{-1} for lower-triangular L (one thread per column).
template <typename S>
__global__ void k_trinv(const S* L, S* Y, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) {
    if (i < c) { Y[(size_t)i * n + c] = Ops<S>::zero(); continue; }
    S s = Ops<S>::zero();
    if (i == c) {
      if constexpr (sizeof(S) == 8) s = 1.0; else s = mkc(1.0, 0.0);
    }
    for (int k = c; k < i; ++k) s = s - Ops<S>::mul(L[(size_t)i * n + k], Y[(size_t)k * n + c]);
    Y[(size_t)i * n + c] = Ops<S>::scale(s, 1.0 / Ops<S>::re(L[(size_t)i * n + i]));
  }
}

// B = Y^+ Y (inverse of L L^+ when Y = L^{-1})
template <typename S>
__global__ void k_yhy(const S* Y, S* B, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  S s = Ops<S>::zero();
  for (int k = max(i, j); k < n; ++k) s = s + Ops<S>::mulc(Y[(size_t)k * n + i], Y[(size_t)k * n + j]);
  B[t] = s;
}

// Partial Gram matrices S_part[chunk] = X[rows]^+ W[rows], tiles of 32 x 32. With herm, only the
// tiles on and above the diagonal (the result is Hermitian: X^+ M X, X^+ H X); blockIdx.y then
// enumerates those tile pairs.
constexpr int GT = 32;
constexpr int GR = 32;
template <typename S>
__global__ void __launch_bounds__(256) k_gram(const S* X, int ldx, const S* W, int ldw, int64_t n, int nv,
                                              int64_t rows_per_chunk, S* part, bool herm, int tiles) {
  __shared__ S xs[GR][GT];
  __shared__ S ws[GR][GT];
  int ti = blockIdx.y, tj = blockIdx.z;
  if (herm) {  // y -> (ti, tj), ti <= tj, row-major over the upper triangle of tiles
    int y = blockIdx.y;
    ti = 0;
    while (y >= tiles - ti) { y -= tiles - ti; ++ti; }
    tj = ti + y;
  }
  const int64_t r0 = blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;  // 2 x 2 entries each: (2ty..), (2tx..)
  S acc[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] = Ops<S>::zero();
  for (int64_t rb = r0; rb < r1; rb += GR) {
    for (int t = threadIdx.x; t < GR * GT; t += 256) {
      const int rr = t / GT, cc = t % GT;
      const int64_t r = rb + rr;
      const int ci = ti * GT + cc, cj = tj * GT + cc;
      xs[rr][cc] = (r < r1 && ci < nv) ? X[r * ldx + ci] : Ops<S>::zero();
      ws[rr][cc] = (r < r1 && cj < nv) ? W[r * ldw + cj] : Ops<S>::zero();
    }
    __syncthreads();
    for (int rr = 0; rr < GR; ++rr) {
      const S x0 = xs[rr][2 * ty], x1 = xs[rr][2 * ty + 1];
      const S w0 = ws[rr][2 * tx], w1 = ws[rr][2 * tx + 1];
      acc[0][0] = fma_c(x0, w0, acc[0][0]);
      acc[0][1] = fma_c(x0, w1, acc[0][1]);
      acc[1][0] = fma_c(x1, w0, acc[1][0]);
      acc[1][1] = fma_c(x1, w1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = ti * GT + 2 * ty + a, j = tj * GT + 2 * tx + b;
      if (i < nv && j < nv) part[((size_t)blockIdx.x * nv + i) * nv + j] = acc[a][b];
    }
}

template <typename S>
__global__ void k_sum_parts(const S* part, int nchunk, int nv, S* out, bool herm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nv) return;
  const int i = t / nv, j = t % nv;
  // below the diagonal tiles of a Hermitian result: the conjugate of the mirrored entry
  const bool mirror = herm && j / GT < i / GT;
  const int src = mirror ? j * nv + i : t;
  S s = Ops<S>::zero();
  for (int c = 0; c < nchunk; ++c) s = s + part[(size_t)c * nv * nv + src];
  out[t] = mirror ? Ops<S>::conj(s) : s;
}

// W = M X: lumped diagonal rows, dense M^oo rows.
template <typename S>
__global__ void k_apply_M(const S* X, int ldx, const double* m, const S* Moo, int64_t nh, int nO, int nv, S* W,
                          int ldw) {
  const int64_t total = (nh + nO) * nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / nv;
    const int v = (int)(t % nv);
    if (r < nh) {
      W[r * ldw + v] = Ops<S>::scale(X[r * ldx + v], m[r]);
    } else {
      const int nu = (int)(r - nh);
      S s = Ops<S>::zero();
      for (int mu = 0; mu < nO; ++mu) s = s + Ops<S>::mul(Moo[(size_t)nu * nO + mu], X[(nh + mu) * ldx + v]);
      W[r * ldw + v] = s;
    }
  }
}

// X[rows] <- X[rows] C (C nv x nv), or X C^+ when herm; with herm, C is lower triangular (the
// inverse Cholesky factor), so only k <= j contributes.
template <typename S>
__global__ void k_rotate(S* X, int ldx, int64_t n, int nv, const S* C, bool herm, int rows) {
  extern __shared__ unsigned char sm[];
  S* xs = reinterpret_cast<S*>(sm);
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int nr = (int)min((int64_t)rows, n - r0);
  if (nr <= 0) return;
  for (int t = threadIdx.x; t < nr * nv; t += blockDim.x) xs[t] = X[(r0 + t / nv) * ldx + t % nv];
  __syncthreads();
  for (int t = threadIdx.x; t < nr * nv; t += blockDim.x) {
    const int r = t / nv, j = t % nv;
    S s = Ops<S>::zero();
    if (herm) {
      for (int k = 0; k <= j; ++k) s = fma_n(xs[r * nv + k], Ops<S>::conj(C[(size_t)j * nv + k]), s);
    } else {
      for (int k = 0; k < nv; ++k) s = fma_n(xs[r * nv + k], C[(size_t)k * nv + j], s);
    }
    X[(r0 + r) * ldx + j] = s;
  }
}

// ---- the same two kernels in FP32-pair arithmetic (pair_dev.cuh); storage stays FP64
struct c2 {
  f2 r, i;
};
__device__ __forceinline__ c2 to_c2(double a) { return c2{f2_from(a), f2{0.0f, 0.0f}}; }
__device__ __forceinline__ c2 to_c2(cd a) { return c2{f2_from(a.x), f2_from(a.y)}; }
template <typename S>
__device__ __forceinline__ S from_acc(f2acc r, f2acc i);
template <>
__device__ __forceinline__ double from_acc<double>(f2acc r, f2acc) { return f2_to(f2_fin(r)); }
template <>
__device__ __forceinline__ cd from_acc<cd>(f2acc r, f2acc i) { return mkc(f2_to(f2_fin(r)), f2_to(f2_fin(i))); }

// Partial Gram matrices as k_gram, in pairs: acc += conj(x) w
template <typename S>
__global__ void __launch_bounds__(256) k_gram_pair(const S* X, int ldx, const S* W, int ldw, int64_t n, int nv,
                                                   int64_t rows_per_chunk, S* part, bool herm, int tiles) {
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  __shared__ c2 xs[GR][GT];
  __shared__ c2 ws[GR][GT];
  int ti = blockIdx.y, tj = blockIdx.z;
  if (herm) {
    int y = blockIdx.y;
    ti = 0;
    while (y >= tiles - ti) { y -= tiles - ti; ++ti; }
    tj = ti + y;
  }
  const int64_t r0 = blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  f2acc ar[2][2], ai[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) ar[a][b] = ai[a][b] = f2acc{0.0f, 0.0f};
  for (int64_t rb = r0; rb < r1; rb += GR) {
    for (int t = threadIdx.x; t < GR * GT; t += 256) {
      const int rr = t / GT, cc = t % GT;
      const int64_t r = rb + rr;
      const int ci = ti * GT + cc, cj = tj * GT + cc;
      xs[rr][cc] = (r < r1 && ci < nv) ? to_c2(X[r * ldx + ci]) : to_c2(Ops<S>::zero());
      ws[rr][cc] = (r < r1 && cj < nv) ? to_c2(W[r * ldw + cj]) : to_c2(Ops<S>::zero());
    }
    __syncthreads();
    for (int rr = 0; rr < GR; ++rr) {
      const c2 x[2] = {xs[rr][2 * ty], xs[rr][2 * ty + 1]};
      const c2 w[2] = {ws[rr][2 * tx], ws[rr][2 * tx + 1]};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          f2_mac(ar[a][b], x[a].r, w[b].r);
          if (CPLX) {
            f2_mac(ar[a][b], x[a].i, w[b].i);
            f2_mac(ai[a][b], x[a].r, w[b].i);
            f2_mac(ai[a][b], f2_neg(x[a].i), w[b].r);
          }
        }
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = ti * GT + 2 * ty + a, j = tj * GT + 2 * tx + b;
      if (i < nv && j < nv) part[((size_t)blockIdx.x * nv + i) * nv + j] = from_acc<S>(ar[a][b], ai[a][b]);
    }
}

// The small matrix of a rotation as pairs, transposed so that consecutive j are contiguous:
// Ct[k][j] = C[k][j], or conj(C[j][k]) for k <= j (herm, C lower triangular).
template <typename S>
__global__ void k_rot_pairs(const S* C, int nv, bool herm, c2* Ct) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nv) return;
  const int k = t / nv, j = t % nv;
  Ct[t] = herm ? (k <= j ? to_c2(Ops<S>::conj(C[(size_t)j * nv + k])) : to_c2(Ops<S>::zero()))
               : to_c2(C[(size_t)k * nv + j]);
}

// X[rows] <- X[rows] C (or X C^+ with herm) in pairs: Ct (k_rot_pairs) copied into shared memory
// once per CTA, rows staged, each thread one column j of two rows.
constexpr int RPT = 512;
template <typename S>
__global__ void __launch_bounds__(RPT) k_rotate_pair(S* X, int ldx, int64_t n, int nv, const c2* Cp, bool herm,
                                                     int rows) {
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  extern __shared__ unsigned char sm[];
  c2* Ct = reinterpret_cast<c2*>(sm);            // nv * nv
  c2* xs = Ct + (size_t)nv * nv;                 // rows * nv
  for (int t = threadIdx.x; t < nv * nv; t += RPT) Ct[t] = Cp[t];
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int nr = (int)min((int64_t)rows, n - r0);
  if (nr <= 0) return;
  for (int t = threadIdx.x; t < nr * nv; t += RPT) xs[t] = to_c2(X[(r0 + t / nv) * ldx + t % nv]);
  __syncthreads();
  const int npair = (nr + 1) / 2;
  for (int t = threadIdx.x; t < npair * nv; t += RPT) {
    const int rp = t / nv, j = t % nv;
    const int ra = 2 * rp, rb = min(2 * rp + 1, nr - 1);
    f2acc sr[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}}, si[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    const int kend = herm ? j + 1 : nv;
    for (int k = 0; k < kend; ++k) {
      const c2 cc = Ct[(size_t)k * nv + j];
      const c2 x[2] = {xs[(size_t)ra * nv + k], xs[(size_t)rb * nv + k]};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        f2_mac(sr[u], x[u].r, cc.r);
        if (CPLX) {
          f2_mac(sr[u], f2_neg(x[u].i), cc.i);
          f2_mac(si[u], x[u].r, cc.i);
          f2_mac(si[u], x[u].i, cc.r);
        }
      }
    }
    X[(r0 + ra) * ldx + j] = from_acc<S>(sr[0], si[0]);
    if (rb != ra) X[(r0 + rb) * ldx + j] = from_acc<S>(sr[1], si[1]);
  }
}

// Column norms for residuals: out[v] = sum_rows conj(R) M^{-1} R, with the
// lumped block divided by m and the enrichment block through (M^oo)^{-1}.
template <typename S>
__global__ void k_resid_norms(const S* R, int ldr, const double* m, const S* Mooinv, int64_t nh, int nO, int nv,
                              double* out) {
  const int v = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < nh; r += blockDim.x) {
    const S x = R[r * ldr + v];
    s += Ops<S>::re(Ops<S>::mulc(x, x)) / m[r];
  }
  for (int t = threadIdx.x; t < nO * nO; t += blockDim.x) {
    const int i = t / nO, j = t % nO;
    s += Ops<S>::re(Ops<S>::mulc(R[(nh + i) * ldr + v], Ops<S>::mul(Mooinv[t], R[(nh + j) * ldr + v])));
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[v] = red[0];
}

// out[v] = Re (U^+ Mq U)[v][v]: the M-norms^2 of the rotated vectors X U from the Gram matrix of X
template <typename S>
__global__ void k_quad_diag(const S* Mq, const S* U, int nv, double* out) {
  const int v = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    S row = Ops<S>::zero();
    for (int j = 0; j < nv; ++j) row = fma_n(Mq[(size_t)i * nv + j], U[(size_t)j * nv + v], row);
    s += Ops<S>::re(Ops<S>::mulc(U[(size_t)i * nv + v], row));
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[v] = red[0];
}

// Column equilibration of the first Cholesky-QR pass by exact powers of two: d_v = 2^-e with
// sqrt(S_vv) = f 2^e, f in [0.5, 1) (d_v = 1 when S_vv is not positive, so the factorization still
// reports it). The filtered block's columns differ by orders of magnitude (the filter's gain at the
// Ritz values), and a rotation whose operand digits share one exponent per row would otherwise
// resolve the small columns only relative to the largest column of the row.
template <typename S>
__global__ void k_gram_scales(const S* Sm, int nv, double* d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double s = Ops<S>::re(Sm[(size_t)v * nv + v]);
  double out = 1.0;
  if (s > 0.0 && isfinite(s)) {
    int e = 0;
    frexp(sqrt(s), &e);
    out = ldexp(1.0, -e);
  }
  d[v] = out;
}

// S_vw <- d_v d_w S_vw
template <typename S>
__global__ void k_scale_gram(S* Sm, int nv, const double* d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nv) return;
  Sm[t] = Ops<S>::scale(Sm[t], d[t / nv] * d[t % nv]);
}

// X_rv <- d_v X_rv
template <typename S>
__global__ void k_scale_cols(S* X, int ldx, int64_t n, int nv, const double* d) {
  const int64_t total = n * nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / nv;
    const int v = (int)(t % nv);
    X[r * ldx + v] = Ops<S>::scale(X[r * ldx + v], d[v]);
  }
}

// R = HX - MX diag(eps)
template <typename S>
__global__ void k_resid_vec(const S* HX, const S* MX, int ld, const double* eps, int64_t n, int nv, S* R) {
  const int64_t total = n * nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(t % nv);
    const int64_t r = t / nv;
    R[r * ld + v] = HX[r * ld + v] - Ops<S>::scale(MX[r * ld + v], eps[v]);
  }
}

// x <- sx x + a y + b z (real views of the vectors); when out != null, out <- x
// is not used; a plain elementwise update for the Lanczos recurrence.
__global__ void k_lanczos_axpy(double* x, const double* y, const double* z, double* unused, int64_t n, double sx,
                               double a, double b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = sx * x[i];
    if (y) v += a * y[i];
    if (z) v += b * z[i];
    x[i] = v;
  }
  (void)unused;
}

__global__ void k_to_float(const double* x, float* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void k_to_double(const float* x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// Re(x^+ y) over interleaved reals: partial sums per block, then one block sums them.
__global__ void k_dot_partial(const double* x, const double* y, int64_t n, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_dot_final(const double* part, int nb, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// ------------------------------------------------------------------ host helpers
// out = X^+ W (nv x nv); herm: the result is known to be Hermitian, only its upper tiles are summed
template <typename S>
int gram(oefe_ctx* c, const S* X, int ldx, const S* W, int ldw, int64_t n, int nv, S* out, S* part_buf,
         int nchunk, bool herm = true) {
  if (c->f64_products == OEFE_F64_PAIRS) {   // FP64-class on the tensor cores (exact bf16 digits)
    bool done = false;
    OEFE_TRY(gram_ozaki<S>(c, X, ldx, W, ldw, n, nv, out, &done));
    if (done) return OEFE_OK;
    return gram_ozaki_wide<S>(c, X, ldx, W, ldw, n, nv, out, herm);   // wider blocks: digits cut in the kernel
  }
  const int tiles = (nv + GT - 1) / GT;
  const int64_t rpc = (n + nchunk - 1) / nchunk;
  dim3 grid(nchunk, herm ? tiles * (tiles + 1) / 2 : tiles, herm ? 1 : tiles);
  if (c->f64_products == OEFE_F64_PAIRS)
    OEFE_COUNTED k_gram_pair<S><<<grid, 256, 0, c->stream>>>(X, ldx, W, ldw, n, nv, rpc, part_buf, herm, tiles);
  else
    OEFE_COUNTED k_gram<S><<<grid, 256, 0, c->stream>>>(X, ldx, W, ldw, n, nv, rpc, part_buf, herm, tiles);
  OEFE_COUNTED k_sum_parts<S><<<(nv * nv + 255) / 256, 256, 0, c->stream>>>(part_buf, nchunk, nv, out, herm);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

template <typename S>
int rotate(oefe_ctx* c, S* X, int ldx, int64_t n, int nv, const S* C, bool herm) {
  if (c->f64_products == OEFE_F64_PAIRS) {   // FP64-class on the tensor cores (exact bf16 digits)
    bool done = false;
    OEFE_TRY(rotate_ozaki<S>(c, X, ldx, n, nv, C, herm, &done));
    if (done) return OEFE_OK;
    return rotate_ozaki_wide<S>(c, X, ldx, n, nv, C, herm);   // wider blocks: digits cut in the kernel
  }
  if (c->f64_products == OEFE_F64_PAIRS) {
    // pairs: C (transposed, as pairs) and the staged rows in shared memory; rows per CTA such that
    // two CTAs share an SM (one stages while the other computes), else as many as fit
    const size_t cb = (size_t)nv * nv * sizeof(c2);
    const size_t rb = (size_t)nv * sizeof(c2);
    int prow = cb < 110 * 1024 ? (int)((110 * 1024 - cb) / rb) : 0;
    if (prow < 16) prow = cb < 200 * 1024 ? (int)((200 * 1024 - cb) / rb) : 0;
    prow = std::min(prow, 256);
    if (prow >= 16) {
      if (c->rotp_bytes < cb) {
        cudaStreamSynchronize(c->stream);
        dev_free(c->d_rotp);
        c->d_rotp = nullptr;
        c->rotp_bytes = 0;
        OEFE_TRY(dev_alloc(c, &c->d_rotp, cb));
        c->rotp_bytes = cb;
      }
      c2* Cp = (c2*)c->d_rotp;
      OEFE_COUNTED k_rot_pairs<S><<<(nv * nv + 255) / 256, 256, 0, c->stream>>>(C, nv, herm, Cp);
      const int64_t blocks = (n + prow - 1) / prow;
      const size_t smem = cb + (size_t)prow * rb;
      OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_rotate_pair<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      OEFE_COUNTED k_rotate_pair<S><<<(unsigned)blocks, RPT, smem, c->stream>>>(X, ldx, n, nv, Cp, herm, prow);
      OEFE_CUDA_TRY(c, cudaGetLastError());
      return OEFE_OK;
    }
  }
  const int rows = std::max(1, (int)((96 * 1024) / ((size_t)nv * sizeof(S))));
  const int64_t blocks = (n + rows - 1) / rows;
  const size_t smem = (size_t)rows * nv * sizeof(S);
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_rotate<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  OEFE_COUNTED k_rotate<S><<<(unsigned)blocks, 256, smem, c->stream>>>(X, ldx, n, nv, C, herm, rows);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

template <typename S>
int apply_M(oefe_ctx* c, const KData& K, const S* X, int ldx, int nv, S* W, int ldw) {
  const int64_t tot = (c->nh + c->nO) * nv;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
  OEFE_COUNTED k_apply_M<S><<<blocks, 256, 0, c->stream>>>(X, ldx, c->d_m, (const S*)K.Moo, c->nh, c->nO, nv, W, ldw);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

// row chunks of the Gram kernel: about four CTAs per SM over the upper tile pairs
int nchunks_for(oefe_ctx* c, int nv) {
  const int tiles = (nv + GT - 1) / GT;
  const int pairs = tiles * (tiles + 1) / 2;
  return std::max(1, std::min(1024, (4 * c->num_sms + pairs - 1) / pairs));
}

template <typename S>
int chol_inverse_t(oefe_ctx* c, S* A, int n, bool inverse, bool want_Linv, S* Y, int* info_host) {
  OEFE_TRY(ensure_ws2(c, 256));
  int* d_info = c->d_status;
  OEFE_COUNTED k_chol<S><<<1, 1024, 0, c->stream>>>(A, n, d_info);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(info_host, d_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (*info_host != 0) return OEFE_OK;
  if (inverse || want_Linv) {
    OEFE_COUNTED k_trinv<S><<<(n + 127) / 128, 128, 0, c->stream>>>(A, Y, n);
    if (inverse) OEFE_COUNTED k_yhy<S><<<(n * n + 255) / 256, 256, 0, c->stream>>>(Y, A, n);
    OEFE_CUDA_TRY(c, cudaGetLastError());
  }
  return OEFE_OK;
}

int check_fp64(oefe_ctx* c, int ik, const void* X, int nv, int ld, int dtype, bool need_h64 = true) {
  if (!c->built) { c->err = "call oefe_build_hamiltonian first"; return OEFE_ERR_STATE; }
  if (ik < 0 || ik >= (int)c->kd.size()) { c->err = "k index out of range"; return OEFE_ERR_ARG; }
  if (!X || nv < 1 || ld < nv || nv > 4096) { c->err = "need X, 1 <= nv <= ld, nv <= 4096"; return OEFE_ERR_ARG; }
  if (!(dtype == OEFE_F64 || dtype == OEFE_C128)) { c->err = "this call needs F64 or C128 vectors"; return OEFE_ERR_ARG; }
  if (c->kd[ik].cplx != (dtype == OEFE_C128)) { c->err = "dtype does not match the k-point"; return OEFE_ERR_ARG; }
  if (need_h64 && !c->kd[ik].H64) { c->err = "FP64 cell matrices were not stored"; return OEFE_ERR_STATE; }
  return OEFE_OK;
}

template <typename S>
int orthonormalize_t(oefe_ctx* c, int ik, S* X, int nv, int ld, double* cond) {
  const KData& K = c->kd[ik];
  const int64_t n = c->nh + c->nO;
  const int nchunk = nchunks_for(c, nv);
  const size_t wbytes = (((size_t)n * nv * sizeof(S) + 255) / 256) * 256;
  const size_t sbytes = (((size_t)nv * nv * sizeof(S) + 255) / 256) * 256;
  const size_t pbytes = (size_t)nchunk * nv * nv * sizeof(S);
  const size_t pbytes_a = ((pbytes + 255) / 256) * 256;
  OEFE_TRY(ensure_ws(c, wbytes + 2 * sbytes + pbytes_a + (size_t)nv * sizeof(double)));
  char* base = (char*)c->ws;
  S* W = (S*)base;
  S* Sm = (S*)(base + wbytes);
  S* Y = (S*)(base + wbytes + sbytes);
  S* part = (S*)(base + wbytes + 2 * sbytes);
  double* dsc = (double*)(base + wbytes + 2 * sbytes + pbytes_a);
  for (int pass = 0; pass < 2; ++pass) {
    OEFE_TRY(apply_M<S>(c, K, X, ld, nv, W, nv));
    OEFE_TRY(gram<S>(c, X, ld, W, nv, n, nv, Sm, part, nchunk));
    if (pass == 0) {
      // equilibrate: X <- X D, S <- D S D (exact); Q = (X D) (D S D)^{-1/2 Cholesky} spans the same
      // space and is the same matrix up to rounding
      OEFE_COUNTED k_gram_scales<S><<<(nv + 127) / 128, 128, 0, c->stream>>>(Sm, nv, dsc);
      OEFE_COUNTED k_scale_gram<S><<<(nv * nv + 255) / 256, 256, 0, c->stream>>>(Sm, nv, dsc);
      const int64_t tot = n * nv;
      const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
      OEFE_COUNTED k_scale_cols<S><<<blocks, 256, 0, c->stream>>>(X, ld, n, nv, dsc);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    }
    int info = 0;
    OEFE_TRY(chol_inverse_t<S>(c, Sm, nv, false, true, Y, &info));
    if (info != 0) {
      c->err = "orthonormalize: Gram matrix not positive definite at column " + std::to_string(info);
      return OEFE_ERR_CHOLESKY;
    }
    if (pass == 0 && cond) {
      std::vector<S> Lh((size_t)nv * nv);
      OEFE_CUDA_TRY(c, cudaMemcpyAsync(Lh.data(), Sm, Lh.size() * sizeof(S), cudaMemcpyDeviceToHost, c->stream));
      OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      double mx = 0, mn = 1e300;
      for (int i = 0; i < nv; ++i) {
        const double d = Ops<S>::re(Lh[(size_t)i * nv + i]);
        mx = std::max(mx, d);
        mn = std::min(mn, d);
      }
      *cond = (mx / mn) * (mx / mn);
    }
    OEFE_TRY(rotate<S>(c, X, ld, n, nv, Y, true));  // X <- X L^{-+}
  }
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

template <typename S>
int rayleigh_ritz_t(oefe_ctx* c, int ik, S* X, int nv, int ld, int dtype, double* eig, double* resid) {
  const KData& K = c->kd[ik];
  const int64_t n = c->nh + c->nO;
  const int nchunk = nchunks_for(c, nv);
  const size_t vbytes = (((size_t)n * nv * sizeof(S) + 255) / 256) * 256;
  const size_t sbytes = (((size_t)nv * nv * sizeof(S) + 255) / 256) * 256;
  const size_t pbytes = (((size_t)nchunk * nv * nv * sizeof(S) + 255) / 256) * 256;
  // ws is used by apply_op; keep HX, MX and small matrices in ws2
  OEFE_TRY(ensure_ws2(c, 2 * vbytes + 3 * sbytes + pbytes + (size_t)nv * 32 + 256));
  char* base = (char*)c->ws2;
  S* HX = (S*)base;
  S* MX = (S*)(base + vbytes);
  S* Hq = (S*)(base + 2 * vbytes);
  S* Mq = (S*)(base + 2 * vbytes + sbytes);
  S* U = (S*)(base + 2 * vbytes + 2 * sbytes);
  S* part = (S*)(base + 2 * vbytes + 3 * sbytes);
  double* d_eps = (double*)(base + 2 * vbytes + 3 * sbytes + pbytes);
  OEFE_TRY(apply_op2(c, ik, X, ld, HX, nv, nv, dtype, false));
  OEFE_TRY(apply_M<S>(c, K, X, ld, nv, MX, nv));
  OEFE_TRY(gram<S>(c, X, ld, HX, nv, n, nv, Hq, part, nchunk));
  OEFE_TRY(gram<S>(c, X, ld, MX, nv, n, nv, Mq, part, nchunk));
  std::vector<double> w(nv);
  OEFE_TRY(gpu_geneig<S>(c, Hq, Mq, nv, w.data(), U));
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_eps, w.data(), nv * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  OEFE_TRY(rotate<S>(c, X, ld, n, nv, U, false));
  if (resid) {
    OEFE_TRY(rotate<S>(c, HX, nv, n, nv, U, false));
    OEFE_TRY(rotate<S>(c, MX, nv, n, nv, U, false));
    const int64_t tot = n * nv;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
    OEFE_COUNTED k_resid_vec<S><<<blocks, 256, 0, c->stream>>>(HX, MX, nv, d_eps, n, nv, HX);  // HX <- residual
    double* d_num = d_eps + nv;
    OEFE_COUNTED k_resid_norms<S><<<nv, 256, 0, c->stream>>>(HX, nv, c->d_m, (const S*)K.Mooinv, c->nh, c->nO, nv, d_num);
    // ||u_v||_M^2 = (U^+ (X^+ M X) U)[v][v] from the Gram matrix taken before the rotation
    double* d_den = d_num + nv;
    OEFE_COUNTED k_quad_diag<S><<<nv, 256, 0, c->stream>>>(Mq, U, nv, d_den);
    std::vector<double> num(nv), den(nv);
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(num.data(), d_num, nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(den.data(), d_den, nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int v = 0; v < nv; ++v) resid[v] = std::sqrt(std::max(num[v], 0.0) / den[v]);
  }
  for (int v = 0; v < nv; ++v) eig[v] = w[v];
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

}  // namespace

int chol_inverse_inplace(oefe_ctx* c, double* A, int n, bool cplx, bool inverse, int* info_host) {
  if (n == 0) { *info_host = 0; return OEFE_OK; }
  const size_t sb = cplx ? sizeof(cd) : sizeof(double);
  OEFE_TRY(ensure_ws2(c, (size_t)n * n * sb + 256));
  if (cplx) return chol_inverse_t<cd>(c, (cd*)A, n, inverse, false, (cd*)c->ws2, info_host);
  return chol_inverse_t<double>(c, A, n, inverse, false, (double*)c->ws2, info_host);
}

int orthonormalize(oefe_ctx* c, int ik, void* X, int nv, int ld, int dtype, double* cond) {
  OEFE_TRY(check_fp64(c, ik, X, nv, ld, dtype));
  if (dtype == OEFE_C128) return orthonormalize_t<cd>(c, ik, (cd*)X, nv, ld, cond);
  return orthonormalize_t<double>(c, ik, (double*)X, nv, ld, cond);
}

int rayleigh_ritz(oefe_ctx* c, int ik, void* X, int nv, int ld, int dtype, double* eig, double* resid) {
  OEFE_TRY(check_fp64(c, ik, X, nv, ld, dtype));
  if (!eig) { c->err = "rayleigh_ritz: need eig"; return OEFE_ERR_ARG; }
  if (dtype == OEFE_C128) return rayleigh_ritz_t<cd>(c, ik, (cd*)X, nv, ld, dtype, eig, resid);
  return rayleigh_ritz_t<double>(c, ik, (double*)X, nv, ld, dtype, eig, resid);
}

int upper_bound(oefe_ctx* c, int ik, const void* v0, int steps, int flags, double* b) {
  const int dtype = (ik >= 0 && ik < (int)c->kd.size() && c->kd[ik].cplx) ? OEFE_C128 : OEFE_F64;
  const bool low = (flags & OEFE_FILTER_BF16X3) != 0;
  OEFE_TRY(check_fp64(c, ik, v0, 1, 1, dtype, !low));
  if (steps < 2 || steps > 1000 || !b) { c->err = "upper_bound: 2 <= steps <= 1000"; return OEFE_ERR_ARG; }
  const KData& K = c->kd[ik];
  if (low && !K.Hbf) { c->err = "upper_bound: BF16x3 cell matrices were not stored"; return OEFE_ERR_STATE; }
  const int64_t n = c->nh + c->nO;
  const size_t sb = dtype == OEFE_C128 ? sizeof(cd) : sizeof(double);
  const size_t vb = (((size_t)n * sb + 255) / 256) * 256;
  const int nparts = 1024;
  OEFE_TRY(ensure_ws2(c, 6 * vb + (nparts + 64) * sizeof(double)));
  char* base = (char*)c->ws2;
  void* q = base;
  void* qp = base + vb;
  void* w = base + 2 * vb;
  void* mw = base + 3 * vb;
  float* q32 = (float*)(base + 4 * vb);          // low-precision copies (half of vb each)
  float* w32 = (float*)(base + 5 * vb);
  double* d_part = (double*)(base + 6 * vb);
  double* d_dot = d_part + nparts;
  const int nr = dtype == OEFE_C128 ? 2 : 1;  // reals per entry
  const int64_t nreal = n * nr;
  std::vector<double> al, be;
  auto mdot = [&](const void* x, const void* y, double* out) -> int {  // re(x^+ M y)
    if (dtype == OEFE_C128) OEFE_TRY(apply_M<cd>(c, K, (const cd*)y, 1, 1, (cd*)mw, 1));
    else OEFE_TRY(apply_M<double>(c, K, (const double*)y, 1, 1, (double*)mw, 1));
    OEFE_COUNTED k_dot_partial<<<nparts, 256, 0, c->stream>>>((const double*)x, (const double*)mw, nreal, d_part);
    OEFE_COUNTED k_dot_final<<<1, 256, 0, c->stream>>>(d_part, nparts, d_dot);
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(out, d_dot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return OEFE_OK;
  };
  auto applyA = [&]() -> int {  // w = M^{-1} H q
    if (!low) return apply_op2(c, ik, q, 1, w, 1, 1, dtype, true);
    const int lb2 = (int)std::min<int64_t>((nreal + 255) / 256, (int64_t)c->num_sms * 16);
    OEFE_COUNTED k_to_float<<<lb2, 256, 0, c->stream>>>((const double*)q, q32, nreal);
    OEFE_TRY(apply_low(c, ik, q32, w32, dtype == OEFE_C128 ? OEFE_C64 : OEFE_F32));
    OEFE_COUNTED k_to_double<<<lb2, 256, 0, c->stream>>>(w32, (double*)w, nreal);
    OEFE_CUDA_TRY(c, cudaGetLastError());
    return OEFE_OK;
  };
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(q, v0, n * sb, cudaMemcpyDeviceToDevice, c->stream));
  OEFE_CUDA_TRY(c, cudaMemsetAsync(qp, 0, n * sb, c->stream));
  double nrm;
  OEFE_TRY(mdot(q, q, &nrm));
  const int lb = (int)std::min<int64_t>((nreal + 255) / 256, (int64_t)c->num_sms * 16);
  OEFE_COUNTED k_lanczos_axpy<<<lb, 256, 0, c->stream>>>((double*)q, nullptr, nullptr, nullptr, nreal, 1.0 / std::sqrt(nrm), 0, 0);
  double beta = 0.0;
  for (int it = 0; it < steps; ++it) {
    OEFE_TRY(applyA());
    double alpha;
    OEFE_TRY(mdot(q, w, &alpha));
    // w <- w - alpha q - beta qp
    OEFE_COUNTED k_lanczos_axpy<<<lb, 256, 0, c->stream>>>((double*)w, (const double*)q, (const double*)qp, nullptr, nreal, 1.0,
                                                -alpha, -beta);
    double bb;
    OEFE_TRY(mdot(w, w, &bb));
    beta = std::sqrt(std::max(bb, 0.0));
    al.push_back(alpha);
    be.push_back(beta);
    // qp <- q, q <- w / beta
    OEFE_COUNTED k_lanczos_axpy<<<lb, 256, 0, c->stream>>>((double*)qp, (const double*)q, nullptr, (double*)q, nreal, 0.0, 1.0, 0);
    OEFE_COUNTED k_lanczos_axpy<<<lb, 256, 0, c->stream>>>((double*)q, (const double*)w, nullptr, nullptr, nreal, 0.0, 1.0 / beta, 0);
    OEFE_CUDA_TRY(c, cudaGetLastError());
  }
  // largest eigenvalue of the Lanczos tridiagonal matrix
  std::vector<double> wv;
  OEFE_TRY(gpu_tridiag_eig(c, al, be, wv));
  *b = wv.back() + be.back();
  return OEFE_OK;
}
