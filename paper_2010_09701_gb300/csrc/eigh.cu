// Dense FP64 generalized Hermitian eigensolver for the projected problem of
// Rayleigh-Ritz (Eq. ProjKS), H^Q u = eps M^Q u, entirely on the GPU:
//   M^Q = L L^+ (Cholesky), C = L^{-1} H^Q L^{-+}, C = W diag(eps) W^+ by a
//   parallel cyclic Jacobi method (circle ordering: n/2 disjoint rotations per
//   round, n-1 rounds per sweep), U = L^{-+} W, eigenvalues ascending.
#include <algorithm>
#include <cmath>

#include "oefe_internal.h"
#include "pair_dev.cuh"

namespace {

constexpr int JT = 1024;
constexpr int MAXPAIRS = 512;   // n <= 1024

__device__ inline double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// C = op(A) op(B), n x n complex; op = conjugate transpose when the flag is set
__global__ void k_small_gemm(const cd* A, bool ca, const cd* B, bool cb, cd* C, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  cd s = mkc(0, 0);
  for (int k = 0; k < n; ++k) {
    const cd a = ca ? cconj(A[(size_t)k * n + i]) : A[(size_t)i * n + k];
    const cd b = cb ? cconj(B[(size_t)j * n + k]) : B[(size_t)k * n + j];
    s += a * b;
  }
  C[t] = s;
}

__global__ void k_hermitian_part(cd* A, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  if (i > j) return;
  const cd v = 0.5 * (A[(size_t)i * n + j] + cconj(A[(size_t)j * n + i]));
  A[(size_t)i * n + j] = v;
  A[(size_t)j * n + i] = cconj(v);
}

// Jacobi sweeps on A (n x n Hermitian, overwritten by its diagonal form), V <- eigenvectors.
// SM: A and V are staged in shared memory for the sweeps (when 2 n^2 complex values fit).
// init_v: start from V = I; otherwise from the V given (the sweeps continue an earlier phase).
template <bool SM>
__global__ void __launch_bounds__(JT) k_jacobi(cd* Ag, cd* Vg, int n, int max_sweeps, double tol, int* sweeps_out,
                                               bool init_v) {
  extern __shared__ cd jsm[];
  cd* A = SM ? jsm : Ag;
  cd* V = SM ? jsm + (size_t)n * n : Vg;
  if (SM) {
    for (int t = threadIdx.x; t < n * n; t += JT) {
      A[t] = Ag[t];
      if (!init_v) V[t] = Vg[t];
    }
    __syncthreads();
  }
  __shared__ double red[JT];
  __shared__ double cs_[MAXPAIRS], sn_[MAXPAIRS];
  __shared__ cd u_[MAXPAIRS];
  __shared__ int p_[MAXPAIRS], q_[MAXPAIRS];
  const int tid = threadIdx.x;
  const int m = n + (n & 1);  // even number of players; player n is a bye when n is odd
  const int np = m / 2;
  if (init_v)
    for (int t = tid; t < n * n; t += JT) V[t] = (t / n == t % n) ? mkc(1, 0) : mkc(0, 0);
  double fro = 0;
  for (int t = tid; t < n * n; t += JT) fro += cabs2(A[t]);
  fro = block_sum(fro, red);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0;
    for (int t = tid; t < n * n; t += JT)
      if (t / n != t % n) off += cabs2(A[t]);
    off = block_sum(off, red);
    if (off <= tol * tol * fro || off == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < np; k += JT) {
        // circle method: position 0 holds player m-1, position i holds (i - 1 + r) mod (m - 1)
        const int a = k == 0 ? m - 1 : (k - 1 + r) % (m - 1);
        const int b = (m - 1 - k - 1 + r) % (m - 1);
        int p = min(a, b), q = max(a, b);
        if (q >= n) { p_[k] = -1; continue; }
        const cd bpq = A[(size_t)p * n + q];
        const double beta = sqrt(cabs2(bpq));
        if (beta < 1e-300) { p_[k] = -1; continue; }
        const cd u = (1.0 / beta) * bpq;
        const double tau = (A[(size_t)q * n + q].x - A[(size_t)p * n + p].x) / (2.0 * beta);
        const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + tt * tt);
        p_[k] = p;
        q_[k] = q;
        cs_[k] = c;
        sn_[k] = tt * c;
        u_[k] = u;
      }
      __syncthreads();
      // rows: A <- G^+ A for every pair (disjoint rows)
      for (int t = tid; t < np * n; t += JT) {
        const int k = t / n, j = t % n;
        const int p = p_[k];
        if (p < 0) continue;
        const int q = q_[k];
        const double c = cs_[k], s = sn_[k];
        const cd ub = cconj(u_[k]);
        // G = [[c, s], [-conj(u) s, conj(u) c]]
        const cd g10 = -s * ub, g11 = c * ub;
        const cd apj = A[(size_t)p * n + j], aqj = A[(size_t)q * n + j];
        A[(size_t)p * n + j] = c * apj + cmulc(g10, aqj);
        A[(size_t)q * n + j] = s * apj + cmulc(g11, aqj);
      }
      __syncthreads();
      // columns: A <- A G, V <- V G
      for (int t = tid; t < np * n; t += JT) {
        const int k = t / n, i = t % n;
        const int p = p_[k];
        if (p < 0) continue;
        const int q = q_[k];
        const double c = cs_[k], s = sn_[k];
        const cd ub = cconj(u_[k]);
        const cd g10 = -s * ub, g11 = c * ub;
        const cd aip = A[(size_t)i * n + p], aiq = A[(size_t)i * n + q];
        A[(size_t)i * n + p] = c * aip + aiq * g10;
        A[(size_t)i * n + q] = s * aip + aiq * g11;
        const cd vip = V[(size_t)i * n + p], viq = V[(size_t)i * n + q];
        V[(size_t)i * n + p] = c * vip + viq * g10;
        V[(size_t)i * n + q] = s * vip + viq * g11;
      }
      __syncthreads();
      for (int k = tid; k < np; k += JT) {
        const int p = p_[k];
        if (p < 0) continue;
        A[(size_t)p * n + q_[k]] = mkc(0, 0);
        A[(size_t)q_[k] * n + p] = mkc(0, 0);
      }
      __syncthreads();
    }
  }
  if (tid == 0) *sweeps_out = sweep;
  if (SM) {
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += JT) {
      Ag[t] = A[t];
      Vg[t] = V[t];
    }
  }
}


// ---- the same cyclic Jacobi method for matrices too large for one CTA's shared memory, spread over
// the whole GPU: per round of the circle ordering one kernel takes the rotation of every pair from the
// current diagonal 2x2 blocks, a second applies them, each thread one 2x2 block of A (rows of one
// pair, columns of another: the row and the column rotation of that block commute with every other
// block's), a third rotates the columns of V. Same rotations and the same arithmetic per entry as
// k_jacobi (rows first, then columns, the rotated pair's off-diagonal entries set to zero).
struct JRot {
  int a, b;     // the pair's indices (b >= n: the bye of an odd n)
  int rot;      // 1 when the pair rotates
  double c, s;
  cd u;
};

__global__ void k_jg_params(const cd* __restrict__ A, int n, int r, JRot* __restrict__ R) {
  const int m = n + (n & 1), np = m / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int a = k == 0 ? m - 1 : (k - 1 + r) % (m - 1);
  const int b = (m - 1 - k - 1 + r) % (m - 1);
  JRot o;
  o.a = min(a, b);
  o.b = max(a, b);
  o.rot = 0;
  o.c = 1.0;
  o.s = 0.0;
  o.u = mkc(1, 0);
  if (o.b < n) {
    const int p = o.a, q = o.b;
    const cd bpq = A[(size_t)p * n + q];
    const double beta = sqrt(cabs2(bpq));
    if (beta >= 1e-300) {
      o.u = (1.0 / beta) * bpq;
      const double tau = (A[(size_t)q * n + q].x - A[(size_t)p * n + p].x) / (2.0 * beta);
      const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      o.c = 1.0 / sqrt(1.0 + tt * tt);
      o.s = tt * o.c;
      o.rot = 1;
    }
  }
  R[k] = o;
}

__global__ void k_jg_apply(cd* __restrict__ A, int n, const JRot* __restrict__ R) {
  const int m = n + (n & 1), np = m / 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)np * np) return;
  const int kr = (int)(t / np), kc = (int)(t % np);
  const JRot gr = R[kr], gc = R[kc];
  const int ri[2] = {gr.a, gr.b}, ci[2] = {gc.a, gc.b};
  cd x[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      x[i][j] = (ri[i] < n && ci[j] < n) ? A[(size_t)ri[i] * n + ci[j]] : mkc(0, 0);
  if (gr.rot) {   // rows: (x_p, x_q) <- (c x_p + conj(g10) x_q, s x_p + conj(g11) x_q)
    const cd ub = cconj(gr.u);
    const cd g10 = -gr.s * ub, g11 = gr.c * ub;
    for (int j = 0; j < 2; ++j) {
      const cd xp = x[0][j], xq = x[1][j];
      x[0][j] = gr.c * xp + cmulc(g10, xq);
      x[1][j] = gr.s * xp + cmulc(g11, xq);
    }
  }
  if (gc.rot) {   // columns: (y_p, y_q) <- (c y_p + y_q g10, s y_p + y_q g11)
    const cd ub = cconj(gc.u);
    const cd g10 = -gc.s * ub, g11 = gc.c * ub;
    for (int i = 0; i < 2; ++i) {
      const cd yp = x[i][0], yq = x[i][1];
      x[i][0] = gc.c * yp + yq * g10;
      x[i][1] = gc.s * yp + yq * g11;
    }
  }
  if (kr == kc && gr.rot) {
    x[0][1] = mkc(0, 0);
    x[1][0] = mkc(0, 0);
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (ri[i] < n && ci[j] < n) A[(size_t)ri[i] * n + ci[j]] = x[i][j];
}

__global__ void k_jg_vrot(cd* __restrict__ V, int n, const JRot* __restrict__ R) {
  const int m = n + (n & 1), np = m / 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)np * n) return;
  const int k = (int)(t / n), i = (int)(t % n);
  const JRot g = R[k];
  if (!g.rot) return;
  const cd ub = cconj(g.u);
  const cd g10 = -g.s * ub, g11 = g.c * ub;
  const cd vp = V[(size_t)i * n + g.a], vq = V[(size_t)i * n + g.b];
  V[(size_t)i * n + g.a] = g.c * vp + vq * g10;
  V[(size_t)i * n + g.b] = g.s * vp + vq * g11;
}

// out[0] = sum of |A_ij|^2 off the diagonal, out[1] = over all entries (one CTA)
__global__ void k_jg_norms(const cd* __restrict__ A, int n, double* out) {
  __shared__ double red[1024];
  double off = 0, all = 0;
  for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
    const double v = cabs2(A[t]);
    all += v;
    if (t / n != t % n) off += v;
  }
  off = block_sum(off, red);
  all = block_sum(all, red);
  if (threadIdx.x == 0) {
    out[0] = off;
    out[1] = all;
  }
}

__global__ void k_eye(cd* V, int n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < (long long)n * n) V[t] = (t / n == t % n) ? mkc(1, 0) : mkc(0, 0);
}

// ---- the sweeps in FP32-pair arithmetic (pair_dev.cuh), on the FP32 pipe: the same rotations
// (parameters taken in FP64 from the current entries), the row and column updates in pairs, until
// the off-diagonal part is below tol; k_jacobi then continues in FP64 from A and V until its own
// stopping test holds. When the pair sweeps already meet it (the usual case: Jacobi converges
// quadratically), the result carries the pair arithmetic's backward error, about 2^-48 ||A||.
struct c2j {
  f2 r, i;
};
__device__ __forceinline__ c2j c2j_from(cd a) { return c2j{f2_from(a.x), f2_from(a.y)}; }
__device__ __forceinline__ cd c2j_to(c2j a) { return mkc(f2_to(a.r), f2_to(a.i)); }
// x a + conj(g) b
__device__ __forceinline__ c2j rot_c(f2 x, c2j a, c2j g, c2j b) {
  f2acc r{0.0f, 0.0f}, i{0.0f, 0.0f};
  f2_mac(r, x, a.r);
  f2_mac(r, g.r, b.r);
  f2_mac(r, g.i, b.i);
  f2_mac(i, x, a.i);
  f2_mac(i, g.r, b.i);
  f2_mac(i, f2_neg(g.i), b.r);
  return c2j{f2_fin(r), f2_fin(i)};
}
// x a + b g
__device__ __forceinline__ c2j rot_n(f2 x, c2j a, c2j b, c2j g) {
  f2acc r{0.0f, 0.0f}, i{0.0f, 0.0f};
  f2_mac(r, x, a.r);
  f2_mac(r, b.r, g.r);
  f2_mac(r, f2_neg(b.i), g.i);
  f2_mac(i, x, a.i);
  f2_mac(i, b.r, g.i);
  f2_mac(i, b.i, g.r);
  return c2j{f2_fin(r), f2_fin(i)};
}

__global__ void __launch_bounds__(JT) k_jacobi_pair(cd* Ag, cd* Vg, int n, int max_sweeps, double tol) {
  extern __shared__ cd jsm[];
  c2j* A = reinterpret_cast<c2j*>(jsm);
  c2j* V = A + (size_t)n * n;
  __shared__ double red[JT];
  __shared__ f2 cs_[MAXPAIRS], sn_[MAXPAIRS];
  __shared__ c2j g10_[MAXPAIRS], g11_[MAXPAIRS];
  __shared__ int p_[MAXPAIRS], q_[MAXPAIRS];
  const int tid = threadIdx.x;
  const int m = n + (n & 1);
  const int np = m / 2;
  double fro = 0;
  for (int t = tid; t < n * n; t += JT) {
    const cd a = Ag[t];
    A[t] = c2j_from(a);
    V[t] = c2j_from((t / n == t % n) ? mkc(1, 0) : mkc(0, 0));
    fro += cabs2(a);
  }
  fro = block_sum(fro, red);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0;
    for (int t = tid; t < n * n; t += JT)
      if (t / n != t % n) off += cabs2(c2j_to(A[t]));
    off = block_sum(off, red);
    if (off <= tol * tol * fro || off == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < np; k += JT) {
        const int a = k == 0 ? m - 1 : (k - 1 + r) % (m - 1);
        const int b = (m - 1 - k - 1 + r) % (m - 1);
        int p = min(a, b), q = max(a, b);
        if (q >= n) { p_[k] = -1; continue; }
        const cd bpq = c2j_to(A[(size_t)p * n + q]);
        const double beta = sqrt(cabs2(bpq));
        if (beta < 1e-300) { p_[k] = -1; continue; }
        const cd u = (1.0 / beta) * bpq;
        const double tau = (f2_to(A[(size_t)q * n + q].r) - f2_to(A[(size_t)p * n + p].r)) / (2.0 * beta);
        const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
        const cd ub = cconj(u);
        p_[k] = p;
        q_[k] = q;
        cs_[k] = f2_from(c);
        sn_[k] = f2_from(s);
        g10_[k] = c2j_from(-s * ub);
        g11_[k] = c2j_from(c * ub);
      }
      __syncthreads();
      for (int t = tid; t < np * n; t += JT) {   // rows: A <- G^+ A
        const int k = t / n, j = t % n;
        const int p = p_[k];
        if (p < 0) continue;
        const int q = q_[k];
        const c2j apj = A[(size_t)p * n + j], aqj = A[(size_t)q * n + j];
        A[(size_t)p * n + j] = rot_c(cs_[k], apj, g10_[k], aqj);
        A[(size_t)q * n + j] = rot_c(sn_[k], apj, g11_[k], aqj);
      }
      __syncthreads();
      for (int t = tid; t < np * n; t += JT) {   // columns: A <- A G, V <- V G
        const int k = t / n, i = t % n;
        const int p = p_[k];
        if (p < 0) continue;
        const int q = q_[k];
        const c2j aip = A[(size_t)i * n + p], aiq = A[(size_t)i * n + q];
        A[(size_t)i * n + p] = rot_n(cs_[k], aip, aiq, g10_[k]);
        A[(size_t)i * n + q] = rot_n(sn_[k], aip, aiq, g11_[k]);
        const c2j vip = V[(size_t)i * n + p], viq = V[(size_t)i * n + q];
        V[(size_t)i * n + p] = rot_n(cs_[k], vip, viq, g10_[k]);
        V[(size_t)i * n + q] = rot_n(sn_[k], vip, viq, g11_[k]);
      }
      __syncthreads();
      for (int k = tid; k < np; k += JT) {
        const int p = p_[k];
        if (p < 0) continue;
        A[(size_t)p * n + q_[k]] = c2j{f2{0.0f, 0.0f}, f2{0.0f, 0.0f}};
        A[(size_t)q_[k] * n + p] = c2j{f2{0.0f, 0.0f}, f2{0.0f, 0.0f}};
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += JT) {
    Ag[t] = c2j_to(A[t]);
    Vg[t] = c2j_to(V[t]);
  }
}

// ascending order: rank of each diagonal entry (ties by index), then permute
__global__ void k_sort_eig(const cd* A, const cd* W, int n, double* eps, cd* Wsorted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double wi = A[(size_t)i * n + i].x;
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const double wj = A[(size_t)j * n + j].x;
    if (wj < wi || (wj == wi && j < i)) ++rank;
  }
  eps[rank] = wi;
  for (int r = 0; r < n; ++r) Wsorted[(size_t)r * n + rank] = W[(size_t)r * n + i];
}

template <typename S>
__global__ void k_to_cd(const S* A, cd* B, int n2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n2) return;
  if constexpr (sizeof(S) == sizeof(cd)) B[t] = reinterpret_cast<const cd*>(A)[t];
  else B[t] = mkc(reinterpret_cast<const double*>(A)[t], 0.0);
}

template <typename S>
__global__ void k_from_cd(const cd* B, S* A, int n2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n2) return;
  if constexpr (sizeof(S) == sizeof(cd)) reinterpret_cast<cd*>(A)[t] = B[t];
  else reinterpret_cast<double*>(A)[t] = B[t].x;
}

// lower Cholesky (single CTA), info = failing pivot + 1
__global__ void __launch_bounds__(1024) k_chol_cd(cd* A, int n, int* info) {
  __shared__ double piv;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(size_t)j * n + j].x;
      if (!(d > 0.0) || !isfinite(d)) fail = j + 1;
      else {
        piv = sqrt(d);
        A[(size_t)j * n + j] = mkc(piv, 0.0);
      }
    }
    __syncthreads();
    if (fail) break;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + j] = (1.0 / piv) * A[(size_t)i * n + j];
    __syncthreads();
    const int mm = n - j - 1;
    for (int t = threadIdx.x; t < mm * mm; t += blockDim.x) {
      const int ii = t / mm, ll = t % mm;
      if (ll > ii) continue;
      const int i = j + 1 + ii, l = j + 1 + ll;
      A[(size_t)i * n + l] -= A[(size_t)i * n + j] * cconj(A[(size_t)l * n + j]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x)
    if (t % n > t / n) A[t] = mkc(0, 0);
  if (threadIdx.x == 0) *info = fail;
}

__global__ void k_trinv_cd(const cd* L, cd* Y, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) {
    if (i < c) { Y[(size_t)i * n + c] = mkc(0, 0); continue; }
    cd s = i == c ? mkc(1, 0) : mkc(0, 0);
    for (int k = c; k < i; ++k) s -= L[(size_t)i * n + k] * Y[(size_t)k * n + c];
    Y[(size_t)i * n + c] = (1.0 / L[(size_t)i * n + i].x) * s;
  }
}

}  // namespace

// H, M: device n x n (double or cd). eps: host n. U: device n x n (same type).
// Returns OEFE_ERR_CHOLESKY if M is not positive definite.
template <typename S>
int gpu_geneig(oefe_ctx* c, const S* H, const S* M, int n, double* eps_host, S* U) {
  if (n > 2 * MAXPAIRS) { c->err = "eigensolver: n too large"; return OEFE_ERR_ARG; }
  const size_t nn = (size_t)n * n;
  // workspace: 6 complex n x n matrices + n doubles + ints, in a private allocation
  cd* base = nullptr;
  OEFE_TRY(dev_alloc(c, (void**)&base, 6 * nn * sizeof(cd) + (size_t)n * sizeof(double) + 64));
  cd *Hc = base, *Mc = base + nn, *Y = base + 2 * nn, *T = base + 3 * nn, *W = base + 4 * nn, *Ws = base + 5 * nn;
  double* d_eps = (double*)(base + 6 * nn);
  int* d_int = (int*)(d_eps + n);
  const int b = 256, g = (int)((nn + b - 1) / b);
  int st = OEFE_OK;
  OEFE_COUNTED k_to_cd<S><<<g, b, 0, c->stream>>>(H, Hc, (int)nn);
  OEFE_COUNTED k_to_cd<S><<<g, b, 0, c->stream>>>(M, Mc, (int)nn);
  OEFE_COUNTED k_hermitian_part<<<g, b, 0, c->stream>>>(Hc, n);
  OEFE_COUNTED k_hermitian_part<<<g, b, 0, c->stream>>>(Mc, n);
  OEFE_COUNTED k_chol_cd<<<1, 1024, 0, c->stream>>>(Mc, n, d_int);
  int info = 0;
  cudaMemcpyAsync(&info, d_int, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  if (info != 0) {
    c->err = "rayleigh_ritz: projected overlap not positive definite";
    st = OEFE_ERR_CHOLESKY;
  } else {
    OEFE_COUNTED k_trinv_cd<<<(n + 127) / 128, 128, 0, c->stream>>>(Mc, Y, n);   // Y = L^{-1}
    OEFE_COUNTED k_small_gemm<<<g, b, 0, c->stream>>>(Y, false, Hc, false, T, n);  // T = L^{-1} H
    OEFE_COUNTED k_small_gemm<<<g, b, 0, c->stream>>>(T, false, Y, true, Hc, n);   // C = T L^{-+}
    OEFE_COUNTED k_hermitian_part<<<g, b, 0, c->stream>>>(Hc, n);
    const size_t jsm = 2 * nn * sizeof(cd);
    if (jsm <= 200 * 1024) {
      cudaFuncSetAttribute(k_jacobi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
      bool init_v = true;
      if (c->f64_products == OEFE_F64_PAIRS) {
        // the sweeps down to about the pair precision on the FP32 pipe, the rest in FP64
        cudaFuncSetAttribute(k_jacobi_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
        OEFE_COUNTED k_jacobi_pair<<<1, JT, jsm, c->stream>>>(Hc, W, n, 40, 1e-12);
        init_v = false;
      }
      OEFE_COUNTED k_jacobi<true><<<1, JT, jsm, c->stream>>>(Hc, W, n, 40, 1e-15, d_int, init_v);
    } else {
      // the whole GPU per round: parameters, block updates, V; the stopping test of k_jacobi per sweep
      JRot* rot = reinterpret_cast<JRot*>(Ws);   // Ws is free until the sort below (n^2 cd >= n/2 JRot)
      double* nrm = d_eps;                      // two doubles, overwritten by the sort
      const int m = n + (n & 1), np = m / 2;
      const int gb = (int)(((long long)np * np + 255) / 256), gv = (int)(((long long)np * n + 255) / 256);
      OEFE_COUNTED k_eye<<<g, b, 0, c->stream>>>(W, n);
      double fro = -1.0;
      for (int sweep = 0; sweep <= 40 && st == OEFE_OK; ++sweep) {
        OEFE_COUNTED k_jg_norms<<<1, 1024, 0, c->stream>>>(Hc, n, nrm);
        double h[2] = {0, 0};
        if (cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
          c->err = "eigensolver: norm read-back failed";
          st = OEFE_ERR_CUDA;
          break;
        }
        if (fro < 0) fro = h[1];   // the Frobenius norm of the matrix the sweeps start from
        if (sweep == 40 || h[0] <= 1e-30 * fro || h[0] == 0.0) break;
        for (int r = 0; r < m - 1; ++r) {
          OEFE_COUNTED k_jg_params<<<(np + 127) / 128, 128, 0, c->stream>>>(Hc, n, r, rot);
          OEFE_COUNTED k_jg_apply<<<gb, 256, 0, c->stream>>>(Hc, n, rot);
          OEFE_COUNTED k_jg_vrot<<<gv, 256, 0, c->stream>>>(W, n, rot);
        }
      }
    }
    OEFE_COUNTED k_sort_eig<<<(n + 127) / 128, 128, 0, c->stream>>>(Hc, W, n, d_eps, Ws);
    OEFE_COUNTED k_small_gemm<<<g, b, 0, c->stream>>>(Y, true, Ws, false, T, n);   // U = L^{-+} W
    OEFE_COUNTED k_from_cd<S><<<g, b, 0, c->stream>>>(T, U, (int)nn);
    cudaMemcpyAsync(eps_host, d_eps, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (cudaGetLastError() != cudaSuccess) { c->err = "eigensolver launch failed"; st = OEFE_ERR_CUDA; }
    cudaStreamSynchronize(c->stream);
  }
  dev_free(base);
  return st;
}

template int gpu_geneig<double>(oefe_ctx*, const double*, const double*, int, double*, double*);
template int gpu_geneig<cd>(oefe_ctx*, const cd*, const cd*, int, double*, cd*);

// eigenvalues of a real symmetric tridiagonal (Lanczos) matrix, ascending
int gpu_tridiag_eig(oefe_ctx* c, const std::vector<double>& al, const std::vector<double>& be, std::vector<double>& w) {
  const int m = (int)al.size();
  std::vector<double> T((size_t)m * m, 0.0), I((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    T[(size_t)i * m + i] = al[i];
    I[(size_t)i * m + i] = 1.0;
    if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = be[i];
  }
  double *dT = nullptr;
  OEFE_TRY(dev_alloc(c, (void**)&dT, 3 * (size_t)m * m * sizeof(double)));
  cudaMemcpyAsync(dT, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(dT + (size_t)m * m, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  w.assign(m, 0.0);
  const int st = gpu_geneig<double>(c, dT, dT + (size_t)m * m, m, w.data(), dT + 2 * (size_t)m * m);
  cudaStreamSynchronize(c->stream);
  dev_free(dT);
  return st;
}
