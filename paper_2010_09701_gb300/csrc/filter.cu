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
                                                            int64_t nh, typename Sc<T, C>::type* __restrict__ Z,
                                                            const int* __restrict__ cells, int compact) {
  using S = typename Sc<T, C>::type;
  extern __shared__ unsigned char smem_raw[];
  S* Xs = reinterpret_cast<S*>(smem_raw);  // npad x NB
  const int e = cells ? cells[blockIdx.x] : blockIdx.x;
  // compact layout: the listed (dense) cells' matrices in list order
  const size_t hslot = compact ? (size_t)blockIdx.x : (size_t)e;
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
  const S* He = H + hslot * npad * npad;
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

// Complex FP64 cell products with three real multiplications per complex product (Gauss): with
// P1 = Re H Re X, P2 = Im H Im X, P3 = (Re H + Im H)(Re X + Im X), Re Z = P1 - P2 and
// Im Z = P3 - P1 - P2. The sum Re H + Im H is formed once per matrix entry by the lane that loads
// it, Re X + Im X once per gathered element, so a product costs 3 FMAs instead of 4 on the FP64
// pipe. Each warp takes two rows at once (one per half-warp), each lane one of 16 vectors.
constexpr int NB3 = 16;
__global__ void __launch_bounds__(CWARPS * 32) k_cell_apply_z3(const cd* __restrict__ H, const cd* __restrict__ X,
                                                              int ldx, int nv, const int* __restrict__ cell_nodes,
                                                              const int* __restrict__ act_off,
                                                              const int* __restrict__ act_idx, int nloc, int npad,
                                                              int64_t nh, cd* __restrict__ Z,
                                                              const int* __restrict__ cells, int compact) {
  extern __shared__ unsigned char smem_raw[];
  double* Xr = reinterpret_cast<double*>(smem_raw);  // npad x NB3 each
  double* Xi = Xr + (size_t)npad * NB3;
  double* Xs = Xi + (size_t)npad * NB3;
  const int e = cells ? cells[blockIdx.x] : blockIdx.x;
  const size_t hslot = compact ? (size_t)blockIdx.x : (size_t)e;   // compact layout: list order
  const int v0 = blockIdx.y * NB3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, hl = lane & 15;
  const int ne = act_off[e + 1] - act_off[e];
  const int naug = nloc + ne;
  for (int t = threadIdx.x; t < npad * NB3; t += CWARPS * 32) {
    const int r = t / NB3, v = t % NB3;
    cd x = mkc(0, 0);
    if (r < naug && v0 + v < nv) {
      const int64_t row = r < nloc ? (int64_t)cell_nodes[(size_t)e * nloc + r] : nh + act_idx[act_off[e] + r - nloc];
      x = X[row * ldx + v0 + v];
    }
    Xr[t] = x.x;
    Xi[t] = x.y;
    Xs[t] = x.x + x.y;
  }
  __syncthreads();
  const cd* He = H + hslot * npad * npad;
  for (int r0 = 2 * warp; r0 < naug; r0 += 2 * CWARPS) {
    const int r = r0 + half;
    const bool rv = r < naug;
    const cd* hr = He + (size_t)(rv ? r : r0) * npad;
    double p1 = 0.0, p2 = 0.0, p3 = 0.0;
    for (int k0 = 0; k0 < naug; k0 += 16) {
      const cd hk = (rv && k0 + hl < npad) ? hr[k0 + hl] : mkc(0, 0);
      const double hs = hk.x + hk.y;
      const int kmax = min(16, naug - k0);
      for (int kk = 0; kk < kmax; ++kk) {
        const double a = __shfl_sync(0xffffffffu, hk.x, kk, 16);
        const double b = __shfl_sync(0xffffffffu, hk.y, kk, 16);
        const double s = __shfl_sync(0xffffffffu, hs, kk, 16);
        const int k = (k0 + kk) * NB3 + hl;
        p1 = fma(a, Xr[k], p1);
        p2 = fma(b, Xi[k], p2);
        p3 = fma(s, Xs[k], p3);
      }
    }
    if (rv && v0 + hl < nv) Z[((size_t)e * npad + r) * nv + v0 + hl] = mkc(p1 - p2, p3 - p1 - p2);
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
      // the recurrence in the precision of the vectors (as the batched node update)
      const T al = (T)alpha, cs = (T)cshift, be = (T)beta;
      if constexpr (C) {
        out.x = al * (y.x - cs * xk.x);
        out.y = al * (y.y - cs * xk.y);
        if (beta != 0.0) {
          const S xm = Xm1[g * ldm1 + v];
          out.x += be * xm.x;
          out.y += be * xm.y;
        }
      } else {
        out = al * (y - cs * xk);
        if (beta != 0.0) out += be * Xm1[g * ldm1 + v];
      }
      y = out;
    }
    Y[g * ldy + v] = y;
  }
}

// Enrichment rows: raw sums over the cells' product rows of one enrichment function (FP64
// accumulation), by one CTA: the row offsets of the function's slots are staged in shared memory
// (chunks of ER_SC), each warp takes 32 vectors and one group of the slots (every G-th slot, eight
// loads in flight), and the groups' partial sums are added in a fixed order.
constexpr int ER_T = 1024;
constexpr int ER_SC = 2048;

template <typename S, bool C>
__device__ __forceinline__ void enr_reduce_cta(const S* __restrict__ Z, int nv, int64_t s0, int64_t s1,
                                               const int64_t* __restrict__ enr_slot, cd* __restrict__ yo) {
  __shared__ double2 red[ER_T];
  __shared__ int64_t off[ER_SC];
  constexpr int NW = ER_T / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nvc = (nv + 31) / 32;
  for (int vc0 = 0; vc0 < nvc; vc0 += NW) {
    const int nc = min(NW, nvc - vc0);   // vector chunks of this pass
    const int G = NW / nc;               // slot groups
    const int g = w / nc, v = (vc0 + w % nc) * 32 + lane;
    const bool active = g < G && v < nv;
    double sx = 0, sy = 0;
    auto add = [&](const S z) {
      if constexpr (C) { sx += (double)z.x; sy += (double)z.y; }
      else sx += (double)z;
    };
    for (int64_t c0 = s0; c0 < s1; c0 += ER_SC) {   // the same trip count in every thread
      const int m = (int)min((int64_t)ER_SC, s1 - c0);
      __syncthreads();
      for (int j = threadIdx.x; j < m; j += ER_T) off[j] = enr_slot[c0 + j] * nv;
      __syncthreads();
      if (active) {
        int j = g;
        for (; j + 7 * G < m; j += 8 * G) {
          S z[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) z[u] = Z[off[j + u * G] + v];
#pragma unroll
          for (int u = 0; u < 8; ++u) add(z[u]);
        }
        for (; j < m; j += G) add(Z[off[j] + v]);
      }
    }
    red[threadIdx.x] = make_double2(sx, sy);
    __syncthreads();
    if (w < nc) {
      double ax = 0, ay = 0;
      for (int gg = 0; gg < G; ++gg) {
        const double2 r = red[(gg * nc + w) * 32 + lane];
        ax += r.x;
        ay += r.y;
      }
      if (v < nv) yo[v] = mkc(ax, ay);
    }
    __syncthreads();
  }
}

// one CTA per enrichment function
template <typename T, bool C>
__global__ void __launch_bounds__(ER_T) k_enr_reduce(const typename Sc<T, C>::type* __restrict__ Z,
                                                     const int64_t* __restrict__ enr_off,
                                                     const int64_t* __restrict__ enr_slot, int nv, cd* __restrict__ Yo) {
  const int nu = blockIdx.x;
  enr_reduce_cta<typename Sc<T, C>::type, C>(Z, nv, enr_off[nu], enr_off[nu + 1], enr_slot, Yo + (size_t)nu * nv);
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

// Batched variants: blockIdx.y selects the k-point; per-k pointers and
// recurrence coefficients come from a parameter table.
struct NodeK {
  const void* Z;       // per-cell products; null: no product this degree (the iterate is zero)
  const void* Xk;      // current iterate; null: zero
  const void* Xm1;
  void* Y;
  cd* Yo;
  const void* Minv;
  int ldk, ldm1, ldy, nv, mode;
  double alpha, cshift, beta;
  // defect recurrence: Y += alpha coef[v] R[:, v] (R null: no addend)
  const void* R;
  const float* coef;
  int ldr;
};

// Node rows of every k-point in one launch (blockIdx.y = k): one warp per node row with all of its
// vectors. The product rows of up to 8 slots are loaded before any is summed, so their latencies
// overlap (the slot indices are warp-uniform broadcast loads); rows whose width and leading
// dimensions allow it move as float4. Complex rows are handled as interleaved reals (every
// operation here is componentwise). The recurrence runs in the filter's precision.
template <typename T, bool C>
__global__ void __launch_bounds__(256) k_node_update_multi(const NodeK* __restrict__ P,
                                                           const int64_t* __restrict__ node_off,
                                                           const int64_t* __restrict__ node_slot,
                                                           const double* __restrict__ m, int64_t nh) {
  const NodeK p = P[blockIdx.y];
  constexpr int R = C ? 2 : 1;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int W = p.nv * R;
  const int ldk = p.ldk * R, ldm1 = p.ldm1 * R, ldy = p.ldy * R, ldr = p.ldr * R;
  const T* Z = (const T*)p.Z;
  const T* Xk = (const T*)p.Xk;
  const T* Xm1 = (const T*)p.Xm1;
  const T* Rr = (const T*)p.R;
  const float* coef = p.coef;
  T* Y = (T*)p.Y;
  const T alpha = (T)p.alpha, cs = (T)p.cshift, beta = (T)p.beta;
  const bool has_z = Z != nullptr, has_k = Xk != nullptr, has_r = Rr != nullptr;
  const bool has_m1 = p.beta != 0.0 && Xm1 != nullptr;
  const bool vec = sizeof(T) == 4 && W % 4 == 0 && ldy % 4 == 0 && ((uintptr_t)Y & 15) == 0 &&
                   (!has_z || ((uintptr_t)Z & 15) == 0) &&
                   (!has_k || (ldk % 4 == 0 && ((uintptr_t)Xk & 15) == 0)) &&
                   (!has_m1 || (ldm1 % 4 == 0 && ((uintptr_t)Xm1 & 15) == 0)) &&
                   (!has_r || (ldr % 4 == 0 && ((uintptr_t)Rr & 15) == 0));
  if (vec && W <= 128) {
    // one float4 per lane covers a row: two nodes per pass of the warp, so that the dependent loads
    // of the two (slot range, slot indices, product rows) overlap; per node the same operations in
    // the same order as the general loop below
    const int f = 4 * lane;
    const bool act = f < W;
    for (int64_t g0 = warp0; g0 < nh; g0 += 2 * nwarps) {
      const int64_t gg[2] = {g0, g0 + nwarps};
      const bool ok[2] = {true, g0 + nwarps < nh};
      int64_t s0[2];
      int ns[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        s0[u] = ok[u] ? node_off[gg[u]] : 0;
        ns[u] = (ok[u] && has_z) ? (int)(node_off[gg[u] + 1] - s0[u]) : 0;
      }
      float4 acc[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
      const int nsm = max(ns[0], ns[1]);
      for (int s8 = 0; s8 < nsm; s8 += 4) {   // four slots per node at a time (most rows have one or two)
        int64_t sl[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i) sl[u][i] = s8 + i < ns[u] ? node_slot[s0[u] + s8 + i] : -1;
        float4 z[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i)
            z[u][i] = (sl[u][i] >= 0 && act) ? *reinterpret_cast<const float4*>((const float*)Z + sl[u][i] * W + f)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[u].x += z[u][i].x;
            acc[u].y += z[u][i].y;
            acc[u].z += z[u][i].z;
            acc[u].w += z[u][i].w;
          }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!ok[u] || !act) continue;
        const int64_t g = gg[u];
        const T minv = (T)(1.0 / m[g]);
        const float4 xk = has_k ? *reinterpret_cast<const float4*>((const float*)Xk + g * ldk + f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 o;
        o.x = (float)alpha * (acc[u].x * (float)minv - (float)cs * xk.x);
        o.y = (float)alpha * (acc[u].y * (float)minv - (float)cs * xk.y);
        o.z = (float)alpha * (acc[u].z * (float)minv - (float)cs * xk.z);
        o.w = (float)alpha * (acc[u].w * (float)minv - (float)cs * xk.w);
        if (has_m1) {
          const float4 xm = *reinterpret_cast<const float4*>((const float*)Xm1 + g * ldm1 + f);
          o.x += (float)beta * xm.x;
          o.y += (float)beta * xm.y;
          o.z += (float)beta * xm.z;
          o.w += (float)beta * xm.w;
        }
        if (has_r) {
          const float4 r = *reinterpret_cast<const float4*>((const float*)Rr + g * ldr + f);
          o.x += (float)alpha * coef[(f + 0) / R] * r.x;
          o.y += (float)alpha * coef[(f + 1) / R] * r.y;
          o.z += (float)alpha * coef[(f + 2) / R] * r.z;
          o.w += (float)alpha * coef[(f + 3) / R] * r.w;
        }
        *reinterpret_cast<float4*>((float*)Y + g * ldy + f) = o;
      }
    }
    return;
  }
  for (int64_t g = warp0; g < nh; g += nwarps) {
    const int64_t s0 = node_off[g];
    const int ns = has_z ? (int)(node_off[g + 1] - s0) : 0;
    const T minv = (T)(1.0 / m[g]);
    if (vec) {
      for (int f = 4 * lane; f < W; f += 128) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int s8 = 0; s8 < ns; s8 += 8) {
          // slot indices: the same address in every lane (one broadcast load each), then the rows
          int64_t sl[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) sl[u] = s8 + u < ns ? node_slot[s0 + s8 + u] : 0;
          float4 z[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            z[u] = s8 + u < ns ? *reinterpret_cast<const float4*>((const float*)Z + sl[u] * W + f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            acc.x += z[u].x;
            acc.y += z[u].y;
            acc.z += z[u].z;
            acc.w += z[u].w;
          }
        }
        const float4 xk = has_k ? *reinterpret_cast<const float4*>((const float*)Xk + g * ldk + f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 o;
        o.x = (float)alpha * (acc.x * (float)minv - (float)cs * xk.x);
        o.y = (float)alpha * (acc.y * (float)minv - (float)cs * xk.y);
        o.z = (float)alpha * (acc.z * (float)minv - (float)cs * xk.z);
        o.w = (float)alpha * (acc.w * (float)minv - (float)cs * xk.w);
        if (has_m1) {
          const float4 xm = *reinterpret_cast<const float4*>((const float*)Xm1 + g * ldm1 + f);
          o.x += (float)beta * xm.x;
          o.y += (float)beta * xm.y;
          o.z += (float)beta * xm.z;
          o.w += (float)beta * xm.w;
        }
        if (has_r) {   // component f + i belongs to vector (f + i) / R
          const float4 r = *reinterpret_cast<const float4*>((const float*)Rr + g * ldr + f);
          o.x += (float)alpha * coef[(f + 0) / R] * r.x;
          o.y += (float)alpha * coef[(f + 1) / R] * r.y;
          o.z += (float)alpha * coef[(f + 2) / R] * r.z;
          o.w += (float)alpha * coef[(f + 3) / R] * r.w;
        }
        *reinterpret_cast<float4*>((float*)Y + g * ldy + f) = o;
      }
    } else {
      for (int f = lane; f < W; f += 32) {
        T acc = T(0);
        for (int s = 0; s < ns; ++s) acc += Z[node_slot[s0 + s] * W + f];
        T o = alpha * (acc * minv - cs * (has_k ? Xk[g * ldk + f] : T(0)));
        if (has_m1) o += beta * Xm1[g * ldm1 + f];
        if (has_r) o += alpha * (T)coef[f / R] * Rr[g * ldr + f];
        Y[g * ldy + f] = o;
      }
    }
  }
}

// one CTA per (enrichment function, k-point)
template <typename T, bool C>
__global__ void __launch_bounds__(ER_T) k_enr_reduce_multi(const NodeK* __restrict__ P, const int64_t* __restrict__ enr_off,
                                                           const int64_t* __restrict__ enr_slot) {
  using S = typename Sc<T, C>::type;
  const NodeK& p = P[blockIdx.y];
  const int nu = blockIdx.x;
  enr_reduce_cta<S, C>((const S*)p.Z, p.nv, enr_off[nu], enr_off[nu + 1], enr_slot, p.Yo + (size_t)nu * p.nv);
}

template <typename T, bool C>
__global__ void k_enr_update_multi(const NodeK* __restrict__ P, int nO, int64_t nh) {
  using S = typename Sc<T, C>::type;
  const NodeK p = P[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nO * p.nv) return;
  const int nu = t / p.nv, v = t % p.nv;
  cd s = mkc(0, 0);
  if (p.Z) {   // no products at the first degree of the defect recurrence
    for (int mu = 0; mu < nO; ++mu) {
      const cd yo = p.Yo[mu * p.nv + v];
      if constexpr (C) s += reinterpret_cast<const cd*>(p.Minv)[nu * nO + mu] * yo;
      else s += reinterpret_cast<const double*>(p.Minv)[nu * nO + mu] * yo;
    }
  }
  const int64_t row = nh + nu;
  double xr = 0, xi = 0;
  if (p.Xk) {
    const S xk = ((const S*)p.Xk)[row * p.ldk + v];
    if constexpr (C) { xr = (double)xk.x; xi = (double)xk.y; } else xr = (double)xk;
  }
  cd out = mkc(p.alpha * (s.x - p.cshift * xr), p.alpha * (s.y - p.cshift * xi));
  if (p.beta != 0.0 && p.Xm1) {
    const S xm = ((const S*)p.Xm1)[row * p.ldm1 + v];
    if constexpr (C) out += mkc(p.beta * (double)xm.x, p.beta * (double)xm.y);
    else out.x += p.beta * (double)xm;
  }
  if (p.R) {
    const S r = ((const S*)p.R)[row * p.ldr + v];
    const double ac = p.alpha * (double)p.coef[v];
    if constexpr (C) out += mkc(ac * (double)r.x, ac * (double)r.y);
    else out.x += ac * (double)r;
  }
  if constexpr (C) ((S*)p.Y)[row * p.ldy + v] = S{(T)out.x, (T)out.y};
  else ((S*)p.Y)[row * p.ldy + v] = (T)out.x;
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
  OEFE_COUNTED k_convert<A, B><<<blocks, 256, 0, c->stream>>>((const A*)X, ldx, (B*)Y, ldy, n, width);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

// Defect form of the filter (p_m(A) Q = Q p_m(Theta) + D_m, see cheb_filter_batched):
// R = A Q - Q diag(theta) in low precision, from the FP64-class product AQ and the FP64 Q; real
// views, W reals per row, component f of a row belongs to vector f / Rs.
__global__ void k_defect_residual(const double* __restrict__ AQ, int ldaq, const double* __restrict__ Q, int ldq,
                                  const double* __restrict__ theta, int64_t n, int W, int Rs, float* __restrict__ Rl,
                                  int ldr) {
  const int64_t total = n * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / W;
    const int f = (int)(t % W);
    Rl[r * ldr + f] = (float)fma(-theta[f / Rs], Q[r * ldq + f], AQ[r * ldaq + f]);
  }
}

// X <- X p_m(theta) + D: the exactly scaled FP64 part plus the low-precision defect
__global__ void k_defect_finish(double* __restrict__ X, int ldx, const float* __restrict__ D, int ldd,
                                const double* __restrict__ pm, int64_t n, int W, int Rs) {
  const int64_t total = n * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / W;
    const int f = (int)(t % W);
    X[r * ldx + f] = fma(X[r * ldx + f], pm[f / Rs], (double)D[r * ldd + f]);
  }
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
  // FP64: single-leaf cells by sum factorization, the others dense
  const bool sf = sizeof(T) == 8 && sumfac_ready(c);
  const int* dense_cells = sf ? c->d_dense_cells : nullptr;
  const int ndense = sf ? c->n_dense : c->ncells;
  const int compact = (sizeof(T) == 8 && K.compact) ? 1 : 0;
  if (compact && !sf) { c->err = "compact FP64 storage needs the sum-factorized products"; return OEFE_ERR_STATE; }
  if (sf) OEFE_TRY(launch_cell_apply_sf(c, K, Xin, ldin, nv, C, Zbuf, c->stream));
  if (mma) {
    OEFE_TRY(launch_cell_mma(c, K, Xin, ldin, nv, C, Zbuf));
  } else if (ndense == 0) {
    // every cell was a single-leaf cell
  } else if (sizeof(T) == 8 && C) {
    dim3 grid(ndense, (nv + NB3 - 1) / NB3);
    const size_t smem = (size_t)c->npad * NB3 * 3 * sizeof(double);
    if (smem > 227 * 1024) { c->err = "cell matrices too large for the shared-memory gather"; return OEFE_ERR_ARG; }
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_apply_z3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    OEFE_COUNTED k_cell_apply_z3<<<grid, CWARPS * 32, smem, c->stream>>>((const cd*)Hm, (const cd*)Xin, ldin, nv,
                                                                        c->d_cell_nodes, c->d_act_off, c->d_act_idx,
                                                                        c->nloc, c->npad, c->nh, (cd*)Zbuf, dense_cells,
                                                                        compact);
  } else {
    dim3 grid(ndense, (nv + NB - 1) / NB);
    const size_t smem = (size_t)c->npad * NB * sizeof(S);
    if (smem > 227 * 1024) { c->err = "cell matrices too large for the shared-memory gather"; return OEFE_ERR_ARG; }
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_apply<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    OEFE_COUNTED k_cell_apply<T, C><<<grid, CWARPS * 32, smem, c->stream>>>((const S*)Hm, (const S*)Xin, ldin, nv, c->d_cell_nodes,
                                                               c->d_act_off, c->d_act_idx, c->nloc, c->npad, c->nh,
                                                               (S*)Zbuf, dense_cells, compact);
  }
  if ((c->timing >> dtype) & 1) cudaEventRecord(timing_event(c), c->stream);
  const int64_t tot = c->nh * nv;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
  OEFE_COUNTED k_node_update<T, C><<<blocks, 256, 0, c->stream>>>((const S*)Zbuf, c->d_node_off, c->d_node_slot, c->d_m, c->nh,
                                                     nv, st.mode, st.alpha, st.cshift, st.beta, (const S*)Xk, ldk,
                                                     (const S*)Xm1, ldm1, (S*)Y, ldy);
  if (c->nO > 0) {
    const int eb = (c->nO * nv + 127) / 128;
    OEFE_COUNTED k_enr_reduce<T, C><<<c->nO, ER_T, 0, c->stream>>>((const S*)Zbuf, c->d_enr_off, c->d_enr_slot, nv, Yo);
    OEFE_COUNTED k_enr_update<T, C><<<eb, 128, 0, c->stream>>>(Yo, K.Mooinv, c->nO, nv, c->nh, st.mode, st.alpha, st.cshift,
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

// vectors per pass of the operator application: the per-cell products of one pass are held at once
// (ncells x npad x chunk scalars), so wide blocks go through in column chunks
constexpr int APPLY_CHUNK = 64;

int apply_op2(oefe_ctx* c, int ik, const void* X, int ldx, void* Y, int ldy, int nv, int dtype, bool minv) {
  OEFE_TRY(check_apply_args(c, ik, X, nv, std::min(ldx, ldy), dtype));
  if (!Y) { c->err = "need Y"; return OEFE_ERR_ARG; }
  const size_t es = dtype_bytes(dtype);
  const int nvc_max = std::min(nv, APPLY_CHUNK);
  const size_t zbytes = (((size_t)c->ncells * c->npad * nvc_max * es + 255) / 256) * 256;
  const size_t yobytes = (size_t)std::max(c->nO, 1) * nvc_max * sizeof(cd);
  OEFE_TRY(ensure_ws(c, zbytes + yobytes + 256));
  char* base = (char*)c->ws;
  Step st{minv ? 1 : 0, 1.0, 0.0, 0.0};
  for (int c0 = 0; c0 < nv; c0 += APPLY_CHUNK) {
    const int nvc = std::min(APPLY_CHUNK, nv - c0);
    OEFE_TRY(dispatch_step(c, c->kd[ik], dtype, (const char*)X + (size_t)c0 * es, ldx, nvc, st, nullptr, 0, nullptr, 0,
                           (char*)Y + (size_t)c0 * es, ldy, base, (cd*)(base + zbytes)));
  }
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

int apply_op(oefe_ctx* c, int ik, const void* X, void* Y, int nv, int ld, int dtype, bool minv) {
  return apply_op2(c, ik, X, ld, Y, ld, nv, dtype, minv);
}

// Y = M^{-1} H X (or H X) with caller-provided scratch for the per-cell
// products and the enrichment sums; allocates nothing.
int apply_op_scratch(oefe_ctx* c, int ik, const void* X, int ldx, void* Y, int ldy, int nv, int dtype, bool minv,
                     void* scratch, size_t scratch_bytes) {
  OEFE_TRY(check_apply_args(c, ik, X, nv, std::min(ldx, ldy), dtype));
  if (!Y || !scratch) { c->err = "need Y and scratch"; return OEFE_ERR_ARG; }
  const size_t es = dtype_bytes(dtype);
  const size_t zbytes = (((size_t)c->ncells * c->npad * nv * es + 255) / 256) * 256;
  const size_t yobytes = (size_t)std::max(c->nO, 1) * nv * sizeof(cd);
  if (zbytes + yobytes > scratch_bytes) {
    c->err = "problem too large for the fixed scratch: needs " + std::to_string(zbytes + yobytes) + " bytes, limit " +
             std::to_string(scratch_bytes);
    return OEFE_ERR_ARG;
  }
  char* base = (char*)scratch;
  Step st{minv ? 1 : 0, 1.0, 0.0, 0.0};
  OEFE_TRY(dispatch_step(c, c->kd[ik], dtype, X, ldx, nv, st, nullptr, 0, nullptr, 0, Y, ldy, base, (cd*)(base + zbytes)));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return OEFE_OK;
}

// Y = M^{-1} H X for one low-precision column through the tensor-core products
int apply_low(oefe_ctx* c, int ik, const void* X, void* Y, int dtype) {
  const size_t es = dtype_bytes(dtype);
  const size_t zbytes = (((size_t)c->ncells * c->npad * es + 255) / 256) * 256;
  const size_t yobytes = (size_t)std::max(c->nO, 1) * sizeof(cd);
  OEFE_TRY(ensure_ws(c, zbytes + yobytes + 256));
  char* base = (char*)c->ws;
  Step st{1, 1.0, 0.0, 0.0};
  return dispatch_step(c, c->kd[ik], dtype, X, 1, 1, st, nullptr, 0, nullptr, 0, Y, 1, base, (cd*)(base + zbytes), true);
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
  if (nv > APPLY_CHUNK) {   // the columns are independent: wide blocks in chunks (bounded scratch)
    const size_t esx = dtype_bytes(dtype);
    for (int c0 = 0; c0 < nv; c0 += APPLY_CHUNK)
      OEFE_TRY(cheb_filter(c, ik, (char*)X + (size_t)c0 * esx, std::min(APPLY_CHUNK, nv - c0), ld, dtype, degree, a, b,
                           a0, flags));
    return OEFE_OK;
  }
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

// ---------------------------------------------------------------------------
// Batched multi-k filter: every k-point advances degree by degree together; one
// persistent tensor-core launch per degree covers all (k, cell, vector block)
// tiles, followed by the batched node / enrichment updates. The low-precision
// degrees are captured once in a CUDA graph on a private stream and replayed;
// the last degree (LAST_FP64) runs per k through the FP64 path.
namespace {

struct BatchPlan {
  int nk, jlow, nb, grid;
  int parts;   // bf16 parts of the split cell matrices
  bool tma;    // warp-specialized TMA kernel (required for three parts)
  bool defect; // defect recurrence: the first degree has no cell product (its iterate is zero)
  long long ntiles;
  std::vector<MmaK> mk;      // jlow * nk
  std::vector<NodeK> nd;     // jlow * nk
  std::vector<int> lc, lp;   // per k: final buffer indices after the low degrees
};

int batched_launch_degrees(oefe_ctx* c, const BatchPlan& P, bool cplx, const MmaK* d_mk, const NodeK* d_nd,
                           bool timed) {
  // node update: one warp per node, 8 warps per CTA, enough CTAs to fill every SM several times over
  const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->num_sms * 16, (c->nh + 7) / 8));
  int vmax = 0;
  for (int k = 0; k < P.nk; ++k) vmax = std::max(vmax, P.nd[k].nv);
  const int eb = (c->nO * vmax + 127) / 128;
  for (int j = 0; j < P.jlow; ++j) {
    const bool product = !(P.defect && j == 0);
    if (timed) cudaEventRecordWithFlags(c->bev_kernel[2 * j], c->bstream, cudaEventRecordExternal);
    if (!product) {
      // D_1 = alpha_1 R: nothing to multiply
    } else if (P.tma) {
      OEFE_TRY(launch_cell_mma_tma(c, c->d_tmaps, d_mk + (size_t)j * P.nk, nullptr, P.nk, P.ntiles, cplx, P.parts,
                                   (int)std::min<long long>(P.ntiles, c->num_sms), c->bstream, P.nb));
    } else if (P.grid > 0) {
      OEFE_TRY(launch_cell_mma_multi(c, d_mk + (size_t)j * P.nk, P.nk, P.ntiles, cplx, P.nb, P.grid, c->bstream));
    } else {  // one CTA per tile, one launch per k-point
      for (int k = 0; k < P.nk; ++k) {
        const MmaK& m = P.mk[(size_t)j * P.nk + k];
        OEFE_TRY(launch_cell_mma_ptrs(c, m.H, m.X, m.ldx, m.nv, m.Z, cplx, P.nb, c->bstream));
      }
    }
    if (timed) cudaEventRecordWithFlags(c->bev_kernel[2 * j + 1], c->bstream, cudaEventRecordExternal);
    dim3 g1(nblocks, P.nk), g2(std::max(eb, 1), P.nk), gr(std::max(c->nO, 1), P.nk);
    if (cplx) {
      OEFE_COUNTED k_node_update_multi<float, true><<<g1, 256, 0, c->bstream>>>(d_nd + (size_t)j * P.nk, c->d_node_off, c->d_node_slot,
                                                                   c->d_m, c->nh);
      if (c->nO > 0) {
        if (product)
          OEFE_COUNTED k_enr_reduce_multi<float, true><<<gr, ER_T, 0, c->bstream>>>(d_nd + (size_t)j * P.nk, c->d_enr_off,
                                                                       c->d_enr_slot);
        OEFE_COUNTED k_enr_update_multi<float, true><<<g2, 128, 0, c->bstream>>>(d_nd + (size_t)j * P.nk, c->nO, c->nh);
      }
    } else {
      OEFE_COUNTED k_node_update_multi<float, false><<<g1, 256, 0, c->bstream>>>(d_nd + (size_t)j * P.nk, c->d_node_off,
                                                                    c->d_node_slot, c->d_m, c->nh);
      if (c->nO > 0) {
        if (product)
          OEFE_COUNTED k_enr_reduce_multi<float, false><<<gr, ER_T, 0, c->bstream>>>(d_nd + (size_t)j * P.nk, c->d_enr_off,
                                                                        c->d_enr_slot);
        OEFE_COUNTED k_enr_update_multi<float, false><<<g2, 128, 0, c->bstream>>>(d_nd + (size_t)j * P.nk, c->nO, c->nh);
      }
    }
    OEFE_CUDA_TRY(c, cudaGetLastError());
  }
  return OEFE_OK;
}

}  // namespace

namespace {

// theta == nullptr: the plain filter. theta != nullptr: the defect form. With Q = X (FP64, on entry)
// and Theta = diag(theta), p_m(A) Q = Q p_m(Theta) + D_m, where D_0 = 0, D_1 = alpha_1 R and
//   D_j = alpha_j [(A - c) D_{j-1} + R p_{j-1}(Theta)] + beta_j D_{j-2},   R = A Q - Q Theta,
// (alpha_j, beta_j the coefficients of the scaled recurrence, p_j the scaled polynomials). R comes
// from one FP64-class product; every degree of D runs on the tensor cores; the result is formed in
// FP64. The low-precision rounding then scales with |D| (about the size of the residuals of Q)
// instead of with |p_m(A) Q|, so converged directions stay converged to FP64-class accuracy.
int filter_batched_impl(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype, int degree,
                        const double* a, const double* b, const double* a0, const double* theta, int flags) {
  if (!c->built) { c->err = "call oefe_build_hamiltonian first"; return OEFE_ERR_STATE; }
  const bool defect = theta != nullptr;
  if (nk < 1 || nk != (int)c->kd.size() || !X || !nv || !ld || !a || !b || !a0) {
    c->err = "filter_batched: one X, nv, ld, a, b, a0 per k-point of the context";
    return OEFE_ERR_ARG;
  }
  if (!(flags & OEFE_FILTER_BF16X3)) { c->err = "filter_batched runs on the tensor cores: pass OEFE_FILTER_BF16X3"; return OEFE_ERR_ARG; }
  // the defect form takes FP64 vectors and runs every degree on the tensor cores
  const bool mixed = !defect && (flags & OEFE_FILTER_LAST_FP64) != 0;
  const bool cplx = c->kd[0].cplx;
  for (int k = 0; k < nk; ++k) {
    OEFE_TRY(check_apply_args(c, k, X[k], nv[k], ld[k], dtype, !mixed && !defect));
    if (c->kd[k].cplx != cplx) { c->err = "filter_batched: all k-points must be real or all complex"; return OEFE_ERR_ARG; }
    if (!c->kd[k].Hbf) { c->err = "filter_batched: BF16x3 cell matrices were not stored"; return OEFE_ERR_STATE; }
    if (degree < 1 || !(b[k] > a[k]) || !(a0[k] < a[k])) { c->err = "filter_batched: need degree >= 1, a0 < a < b"; return OEFE_ERR_ARG; }
  }
  if (defect) {
    if (!dtype_fp64(dtype)) { c->err = "filter_batched_defect: needs F64/C128 vectors"; return OEFE_ERR_ARG; }
    size_t tot = 0;
    for (int k = 0; k < nk; ++k) tot += nv[k];
    for (size_t i = 0; i < tot; ++i)
      if (!std::isfinite(theta[i])) { c->err = "filter_batched_defect: theta must be finite"; return OEFE_ERR_ARG; }
  }
  if (mixed && !dtype_fp64(dtype)) { c->err = "filter_batched: LAST_FP64 needs F64/C128 storage"; return OEFE_ERR_ARG; }
  if (!mixed && !defect && dtype_fp64(dtype)) { c->err = "filter_batched: low-precision vectors (F32/C64) without LAST_FP64"; return OEFE_ERR_ARG; }
  const int dt_low = cplx ? OEFE_C64 : OEFE_F32;
  const size_t es_low = dtype_bytes(dt_low), es = dtype_bytes(dtype);
  const int64_t n = c->nh + c->nO;
  const int jlow = mixed ? degree - 1 : degree;
  if (jlow == 0) {   // (never in the defect form: jlow = degree >= 1)  // a single FP64 degree: no low-precision work to batch
    for (int k = 0; k < nk; ++k)
      OEFE_TRY(cheb_filter(c, k, X[k], nv[k], ld[k], dtype, degree, a[k], b[k], a0[k], 0));
    return OEFE_OK;
  }
  if (c->tune_nb == 0) { c->tune_nb = 64; c->tune_grid = c->num_sms; }
  const int parts = c->kd[0].bf_parts;
  for (int k = 1; k < nk; ++k)
    if (c->kd[k].bf_parts != parts) { c->err = "filter_batched: k-points with different splits"; return OEFE_ERR_STATE; }
  const bool tma = (c->use_tma || parts == 3) && c->d_tmaps;
  if (!tma && parts != 2) { c->err = "filter_batched: the split cell matrices have no tensor maps"; return OEFE_ERR_STATE; }
  if (tma) c->tune_nb = (!cplx && c->tma_nvt == 128) ? 128 : 64;
  // workspace: per k  Z | Yo | L0 L1 L2 | B1 B2 (mixed) or R, A Q, coefficients (defect)
  std::vector<size_t> off(nk + 1, 0);
  auto a256 = [](size_t x) { return ((x + 255) / 256) * 256; };
  std::vector<size_t> zb(nk), yb(nk), lb(nk), fb(nk), cb(nk);
  for (int k = 0; k < nk; ++k) {
    // products of the low-precision degrees (all nv[k] vectors), or of one FP64-class pass (chunks)
    zb[k] = a256((size_t)c->ncells * c->npad *
                 std::max((size_t)nv[k] * es_low, (size_t)std::min(nv[k], APPLY_CHUNK) * es));
    yb[k] = a256((size_t)std::max(c->nO, 1) * nv[k] * sizeof(cd));
    lb[k] = a256((size_t)n * nv[k] * es_low);
    fb[k] = (mixed || defect) ? a256((size_t)n * nv[k] * es) : 0;
    // defect: p_0 .. p_{m-1} per vector (float), then p_m and theta (double)
    cb[k] = defect ? a256((size_t)degree * nv[k] * sizeof(float)) + 2 * a256((size_t)nv[k] * sizeof(double)) : 0;
    off[k + 1] = off[k] + zb[k] + yb[k] + 3 * lb[k] + 2 * fb[k] + cb[k];
  }
  OEFE_TRY(ensure_ws(c, off[nk] + 256));
  char* base = (char*)c->ws;
  std::vector<void*> Zk(nk), L0(nk), L1(nk), L2(nk), F1(nk), F2(nk);
  std::vector<cd*> Yo(nk);
  std::vector<float*> coef(nk);
  std::vector<double*> pmv(nk), thv(nk);
  for (int k = 0; k < nk; ++k) {
    char* p = base + off[k];
    Zk[k] = p;
    Yo[k] = (cd*)(p + zb[k]);
    L0[k] = p + zb[k] + yb[k];
    L1[k] = p + zb[k] + yb[k] + lb[k];
    L2[k] = p + zb[k] + yb[k] + 2 * lb[k];
    F1[k] = p + zb[k] + yb[k] + 3 * lb[k];   // defect: A Q (FP64)
    F2[k] = p + zb[k] + yb[k] + 3 * lb[k] + fb[k];   // defect: R (low precision)
    char* q = p + zb[k] + yb[k] + 3 * lb[k] + 2 * fb[k];
    coef[k] = (float*)q;
    pmv[k] = (double*)(q + a256((size_t)degree * nv[k] * sizeof(float)));
    thv[k] = (double*)(q + a256((size_t)degree * nv[k] * sizeof(float)) + a256((size_t)nv[k] * sizeof(double)));
  }
  // plan: simulate the buffer rotation of the low-precision degrees
  BatchPlan P;
  P.nk = nk;
  P.jlow = jlow;
  P.nb = c->tune_nb;
  P.grid = c->tune_grid;
  P.parts = parts;
  P.tma = tma;
  P.defect = defect;
  P.ntiles = 0;
  std::vector<long long> tile0(nk);
  for (int k = 0; k < nk; ++k) {
    tile0[k] = P.ntiles;
    P.ntiles += (long long)c->ncells * ((nv[k] + P.nb - 1) / P.nb);
  }
  P.lc.assign(nk, 0);
  P.lp.assign(nk, 1);
  std::vector<double> sig(nk);
  for (int k = 0; k < nk; ++k) {
    const double e = (b[k] - a[k]) / 2.0;
    sig[k] = e / (a0[k] - (b[k] + a[k]) / 2.0);
  }
  const std::vector<double> sig1 = sig;
  for (int j = 1; j <= jlow; ++j) {
    for (int k = 0; k < nk; ++k) {
      // defect: D_0 = 0 is never read, so all three buffers are private
      void* bufs[3] = {(mixed || defect) ? L0[k] : X[k], L1[k], L2[k]};
      const int lds[3] = {(mixed || defect) ? nv[k] : ld[k], nv[k], nv[k]};
      const double e = (b[k] - a[k]) / 2.0, cc = (b[k] + a[k]) / 2.0;
      double alpha, beta;
      if (j == 1) {
        alpha = sig1[k] / e;
        beta = 0.0;
      } else {
        const double s2 = 1.0 / (2.0 / sig1[k] - sig[k]);
        alpha = 2.0 * s2 / e;
        beta = -sig[k] * s2;
        sig[k] = s2;
      }
      const int ic = P.lc[k], ip = P.lp[k], in = 3 - ic - ip;
      MmaK mk;
      mk.H = c->kd[k].Hbf;
      mk.X = (const float*)bufs[ic];
      mk.Z = (float*)Zk[k];
      mk.ldx = lds[ic];
      mk.nv = nv[k];
      mk.vblocks = (nv[k] + P.nb - 1) / P.nb;
      mk.tile0 = tile0[k];
      P.mk.push_back(mk);
      NodeK nd;
      nd.Z = Zk[k];
      nd.Xk = bufs[ic];
      nd.Xm1 = j == 1 ? nullptr : bufs[ip];
      nd.Y = bufs[in];
      nd.Yo = Yo[k];
      nd.Minv = c->kd[k].Mooinv;
      nd.ldk = lds[ic];
      nd.ldm1 = lds[ip];
      nd.ldy = lds[in];
      nd.nv = nv[k];
      nd.mode = 2;
      nd.alpha = alpha;
      nd.cshift = cc;
      nd.beta = beta;
      nd.R = nullptr;
      nd.coef = nullptr;
      nd.ldr = 0;
      if (defect) {
        if (j == 1) { nd.Z = nullptr; nd.Xk = nullptr; }   // D_0 = 0: no product, no shift term
        if (j <= 2) nd.Xm1 = nullptr;                      // D_{j-2} = D_0 = 0 (or none)
        nd.R = F2[k];                                      // R in low precision, rows of nv
        nd.ldr = nv[k];
        nd.coef = coef[k] + (size_t)(j - 1) * nv[k];       // p_{j-1}(theta) per vector
      }
      P.nd.push_back(nd);
      P.lp[k] = ic;
      P.lc[k] = in;
    }
  }
  // graph key: everything baked into the captured launches
  std::vector<double> key = {(double)nk, (double)degree, (double)flags, (double)dtype, (double)(uintptr_t)base,
                             (double)P.nb, (double)P.grid, (double)(c->timing & (1 << dt_low) ? 1 : 0),
                             (double)tma, (double)parts, (double)c->tune_merge, (double)defect};
  for (int k = 0; k < nk; ++k) {
    key.push_back((double)(uintptr_t)X[k]);
    key.push_back(nv[k]);
    key.push_back(ld[k]);
    key.push_back(a[k]);
    key.push_back(b[k]);
    key.push_back(a0[k]);
  }
  if (!c->bstream) {
    OEFE_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking));
    OEFE_CUDA_TRY(c, cudaEventCreateWithFlags(&c->bev_in, cudaEventDisableTiming));
    OEFE_CUDA_TRY(c, cudaEventCreateWithFlags(&c->bev_out, cudaEventDisableTiming));
  }
  const bool timed = (c->timing >> dt_low) & 1;
  // entries left without a graph by an earlier failed capture are dropped first
  for (size_t i = 0; i < c->bgraphs.size();) {
    if (c->bgraphs[i].exec) { ++i; continue; }
    dev_free(c->bgraphs[i].params);
    c->bgraphs.erase(c->bgraphs.begin() + i);
  }
  BatchGraph* G = nullptr;
  for (auto& g : c->bgraphs)
    if (g.key == key) G = &g;
  if (!G) {
    cudaStreamSynchronize(c->bstream);
    if (c->bgraphs.size() >= 4) {   // the oldest goes
      if (c->bgraphs.front().exec) cudaGraphExecDestroy(c->bgraphs.front().exec);
      dev_free(c->bgraphs.front().params);
      c->bgraphs.erase(c->bgraphs.begin());
    }
    c->bgraphs.emplace_back();
    G = &c->bgraphs.back();
    G->key = key;
    const size_t pbytes = P.mk.size() * sizeof(MmaK) + P.nd.size() * sizeof(NodeK) + 64;
    int sa = dev_alloc(c, &G->params, pbytes);
    if (sa != OEFE_OK) {
      c->bgraphs.pop_back();
      return sa;
    }
    MmaK* d_mk = (MmaK*)G->params;
    NodeK* d_nd = (NodeK*)((char*)G->params + ((P.mk.size() * sizeof(MmaK) + 15) / 16) * 16);
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_mk, P.mk.data(), P.mk.size() * sizeof(MmaK), cudaMemcpyHostToDevice, c->bstream));
    OEFE_CUDA_TRY(c, cudaMemcpyAsync(d_nd, P.nd.data(), P.nd.size() * sizeof(NodeK), cudaMemcpyHostToDevice, c->bstream));
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->bstream));
    if (timed) {
      while (c->bev_kernel.size() < (size_t)2 * jlow) {
        cudaEvent_t ev;
        OEFE_CUDA_TRY(c, cudaEventCreate(&ev));
        c->bev_kernel.push_back(ev);
      }
    }
    // set the kernels' shared-memory limits outside of the capture
    if (tma) OEFE_TRY(launch_cell_mma_tma(c, c->d_tmaps, d_mk, nullptr, nk, 0, cplx, parts, 1, c->bstream, P.nb));
    else if (P.grid > 0) OEFE_TRY(launch_cell_mma_multi(c, d_mk, nk, 0, cplx, P.nb, 1, c->bstream));
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->bstream));
    cudaGraph_t graph = nullptr;
    OEFE_CUDA_TRY(c, cudaStreamBeginCapture(c->bstream, cudaStreamCaptureModeThreadLocal));
    const long long launches0 = oefe_launch_add(0);
    int st = OEFE_OK;
    if (mixed) {
      for (int k = 0; k < nk && st == OEFE_OK; ++k) {
        const int width = cplx ? 2 * nv[k] : nv[k];
        const int64_t tot = n * width;
        const int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)c->num_sms * 32);
        OEFE_COUNTED k_convert<double, float><<<blocks, 256, 0, c->bstream>>>((const double*)X[k], ld[k] * (cplx ? 2 : 1),
                                                                 (float*)L0[k], width, n, width);
      }
    }
    if (st == OEFE_OK) st = batched_launch_degrees(c, P, cplx, d_mk, d_nd, timed);
    cudaError_t ce = cudaStreamEndCapture(c->bstream, &graph);
    // captured launches run at each replay, not here
    G->kernels = oefe_launch_add(0) - launches0;
    oefe_launch_add(-G->kernels);
    if (st == OEFE_OK && ce != cudaSuccess) {
      c->err = std::string("graph capture: ") + cudaGetErrorString(ce);
      st = OEFE_ERR_CUDA;
    }
    if (st == OEFE_OK) {
      ce = cudaGraphInstantiate(&G->exec, graph, 0);
      if (ce != cudaSuccess) {
        c->err = std::string("graph instantiate: ") + cudaGetErrorString(ce);
        st = OEFE_ERR_CUDA;
      }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != OEFE_OK) {
      dev_free(G->params);
      c->bgraphs.pop_back();
      return st;
    }
  }
  if (defect) {
    // per k: the scaled polynomials at theta (host, FP64), R = A Q - Q Theta from one FP64-class
    // product, on the caller's stream before the replay
    size_t t0 = 0;
    for (int k = 0; k < nk; ++k) {
      const double e = (b[k] - a[k]) / 2.0, cc = (b[k] + a[k]) / 2.0;
      const double s1 = e / (a0[k] - cc);
      std::vector<float> cf((size_t)degree * nv[k]);
      std::vector<double> pm(nv[k]), th(theta + t0, theta + t0 + nv[k]);
      for (int v = 0; v < nv[k]; ++v) {
        double pprev = 1.0, pcur = (s1 / e) * (th[v] - cc), sg = s1;   // p_0, p_1
        cf[v] = 1.0f;
        for (int j = 2; j <= degree; ++j) {
          cf[(size_t)(j - 1) * nv[k] + v] = (float)pcur;                 // p_{j-1}
          const double s2 = 1.0 / (2.0 / s1 - sg);
          const double pn = (2.0 * s2 / e) * (th[v] - cc) * pcur - sg * s2 * pprev;
          pprev = pcur;
          pcur = pn;
          sg = s2;
        }
        pm[v] = pcur;                                                    // p_m
      }
      t0 += nv[k];
      OEFE_CUDA_TRY(c, cudaMemcpyAsync(coef[k], cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
      OEFE_CUDA_TRY(c, cudaMemcpyAsync(pmv[k], pm.data(), pm.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      OEFE_CUDA_TRY(c, cudaMemcpyAsync(thv[k], th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      // A Q into F1 (FP64-class: FP32 pairs in pair mode), then R (low precision) over it, row by row
      const Step st{1, 1.0, 0.0, 0.0};
      for (int c0 = 0; c0 < nv[k]; c0 += APPLY_CHUNK)
        OEFE_TRY(dispatch_step(c, c->kd[k], dtype, (const char*)X[k] + (size_t)c0 * es, ld[k],
                               std::min(APPLY_CHUNK, nv[k] - c0), st, nullptr, 0, nullptr, 0, (char*)F1[k] + (size_t)c0 * es,
                               nv[k], Zk[k], Yo[k], false));
      const int Rs = cplx ? 2 : 1, W = nv[k] * Rs;
      const int blocks = (int)std::min<int64_t>((n * W + 255) / 256, (int64_t)c->num_sms * 32);
      OEFE_COUNTED k_defect_residual<<<blocks, 256, 0, c->stream>>>((const double*)F1[k], W, (const double*)X[k],
                                                                  ld[k] * Rs, thv[k], n, W, Rs, (float*)F2[k], W);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    }
  }
  // run: the private stream waits for the caller's stream and vice versa
  OEFE_CUDA_TRY(c, cudaEventRecord(c->bev_in, c->stream));
  OEFE_CUDA_TRY(c, cudaStreamWaitEvent(c->bstream, c->bev_in, 0));
  OEFE_CUDA_TRY(c, cudaGraphLaunch(G->exec, c->bstream));
  oefe_launch_add(G->kernels);
  OEFE_CUDA_TRY(c, cudaEventRecord(c->bev_out, c->bstream));
  OEFE_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->bev_out, 0));
  if (timed) {
    OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->bstream));
    for (int j = 0; j < jlow; ++j) {
      if (defect && j == 0) continue;   // no product at the first degree of the defect form
      float t = 0;
      OEFE_CUDA_TRY(c, cudaEventElapsedTime(&t, c->bev_kernel[2 * j], c->bev_kernel[2 * j + 1]));
      c->timing_extra_ms += t;
      c->timing_extra_n += 1;
    }
  }
  // finish per k: X p_m(theta) + D_m (defect), the last degree in FP64, or copy the low-precision result
  for (int k = 0; k < nk; ++k) {
    const KData& K = c->kd[k];
    if (defect) {
      const int Rs = cplx ? 2 : 1, W = nv[k] * Rs;
      void* L[3] = {L0[k], L1[k], L2[k]};
      const int blocks = (int)std::min<int64_t>((n * W + 255) / 256, (int64_t)c->num_sms * 32);
      OEFE_COUNTED k_defect_finish<<<blocks, 256, 0, c->stream>>>((double*)X[k], ld[k] * Rs, (const float*)L[P.lc[k]], W,
                                                                pmv[k], n, W, Rs);
      OEFE_CUDA_TRY(c, cudaGetLastError());
    } else if (mixed) {
      const int width = cplx ? 2 * nv[k] : nv[k];
      void* L[3] = {L0[k], L1[k], L2[k]};
      OEFE_TRY((convert<float, double>(c, L[P.lc[k]], width, F1[k], width, n, width)));
      void* bufs[3] = {X[k], F1[k], F2[k]};
      int lds[3] = {ld[k], nv[k], nv[k]};
      int fp = 0;
      if (degree > 2) {
        OEFE_TRY((convert<float, double>(c, L[P.lp[k]], width, F2[k], width, n, width)));
        fp = 2;
      }
      const double e = (b[k] - a[k]) / 2.0, cc = (b[k] + a[k]) / 2.0;
      double sg = e / (a0[k] - cc);
      const double s1 = sg;
      for (int j = 2; j < degree; ++j) sg = 1.0 / (2.0 / s1 - sg);
      // the FP64 degree in column chunks: the product buffer holds APPLY_CHUNK FP64 columns
      for (int c0 = 0; c0 < nv[k]; c0 += APPLY_CHUNK) {
        const int w = std::min(APPLY_CHUNK, nv[k] - c0);
        void* bq[3] = {(char*)bufs[0] + (size_t)c0 * es, (char*)bufs[1] + (size_t)c0 * es,
                       (char*)bufs[2] + (size_t)c0 * es};
        double sgq = sg;
        int ip = fp, ic = 1;
        OEFE_TRY(run_degrees(c, K, dtype, bq, lds, &ip, &ic, w, degree, degree, e, cc, &sgq, s1, Zk[k], Yo[k], false));
        if (ic != 0)
          OEFE_CUDA_TRY(c, cudaMemcpy2DAsync(bq[0], (size_t)ld[k] * es, bq[ic], (size_t)lds[ic] * es, (size_t)w * es,
                                             (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
      }
    } else if (P.lc[k] != 0) {
      void* L[3] = {X[k], L1[k], L2[k]};
      OEFE_CUDA_TRY(c, cudaMemcpy2DAsync(X[k], (size_t)ld[k] * es, L[P.lc[k]], (size_t)nv[k] * es, (size_t)nv[k] * es,
                                         (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int flag = 0;
  OEFE_CUDA_TRY(c, cudaMemcpy(&flag, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    cudaMemset(c->d_status, 0, sizeof(int));
    c->err = "filter_batched: a tensor-core pipeline wait timed out";
    return OEFE_ERR_TIMEOUT;
  }
  return OEFE_OK;
}

}  // namespace

namespace {

// vectors per k-point of one batched pass: wider blocks run as several passes over column groups
// (the columns of the filter are independent), which bounds the per-cell products and recurrence
// buffers; each group keeps its own captured graph
constexpr int FILTER_CHUNK = 128;

int filter_batched_groups(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype, int degree,
                          const double* a, const double* b, const double* a0, const double* theta, int flags) {
  int vmax = 0;
  bool ok = nk >= 1 && X && nv && ld;
  for (int k = 0; ok && k < nk; ++k) {
    ok = nv[k] >= 1;
    vmax = std::max(vmax, ok ? nv[k] : 0);
  }
  const int Q = (vmax + FILTER_CHUNK - 1) / FILTER_CHUNK;
  for (int k = 0; ok && k < nk; ++k) ok = nv[k] >= Q;
  if (!ok || Q <= 1 || dtype < 0 || dtype > 3)   // one pass (the call checks its arguments itself)
    return filter_batched_impl(c, nk, X, nv, ld, dtype, degree, a, b, a0, theta, flags);
  const size_t es = dtype_bytes(dtype);
  std::vector<size_t> toff(nk + 1, 0);
  for (int k = 0; k < nk; ++k) toff[k + 1] = toff[k] + nv[k];
  for (int q = 0; q < Q; ++q) {   // group q: columns [q nv / Q, (q + 1) nv / Q) of every k-point
    std::vector<void*> Xq(nk);
    std::vector<int> nvq(nk);
    std::vector<double> thq;
    for (int k = 0; k < nk; ++k) {
      const int c0 = (int)((long long)q * nv[k] / Q), c1 = (int)((long long)(q + 1) * nv[k] / Q);
      Xq[k] = (char*)X[k] + (size_t)c0 * es;
      nvq[k] = c1 - c0;
      if (theta) thq.insert(thq.end(), theta + toff[k] + c0, theta + toff[k] + c1);
    }
    OEFE_TRY(filter_batched_impl(c, nk, Xq.data(), nvq.data(), ld, dtype, degree, a, b, a0,
                                 theta ? thq.data() : nullptr, flags));
  }
  return OEFE_OK;
}

}  // namespace

int cheb_filter_batched(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype, int degree,
                        const double* a, const double* b, const double* a0, int flags) {
  return filter_batched_groups(c, nk, X, nv, ld, dtype, degree, a, b, a0, nullptr, flags);
}

int cheb_filter_batched_defect(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype,
                               int degree, const double* a, const double* b, const double* a0, const double* theta,
                               int flags) {
  if (!theta) { c->err = "filter_batched_defect: need theta"; return OEFE_ERR_ARG; }
  return filter_batched_groups(c, nk, X, nv, ld, dtype, degree, a, b, a0, theta, flags);
}

// the launch shapes the autotuner chooses among: vectors per tile, persistent grid (0: one CTA per
// tile), TMA kernel, merged real-part MMAs
struct FilterShape { int nb, grid, tma, merge; };
static FilterShape filter_shape(const oefe_ctx* c, int i) {
  const FilterShape s[6] = {{64, c->num_sms, 0, 0}, {32, c->num_sms, 0, 0}, {64, 0, 0, 0}, {64, c->num_sms, 1, 0},
                            {64, c->num_sms, 1, 1}, {128, c->num_sms, 1, 0}};
  return s[i];
}

static void keep_shape(oefe_ctx* c, const FilterShape& s) {
  c->tune_nb = s.nb;
  c->tune_grid = s.grid;
  c->use_tma = s.tma;
  c->tune_merge = s.merge;
  c->tma_nvt = s.tma ? s.nb : 64;
}

int filter_set_shape(oefe_ctx* c, int shape) {
  if (shape < -1 || shape > 5) { c->err = "set_filter_shape: shape must be -1 or 0..5"; return OEFE_ERR_ARG; }
  if (shape < 0) {
    c->tune_nb = 0;
    c->tune_grid = 0;
    c->use_tma = 1;
    c->tune_merge = -1;
    c->tma_nvt = 64;
  } else {
    keep_shape(c, filter_shape(c, shape));
  }
  return OEFE_OK;
}

int filter_autotune(oefe_ctx* c, int nk, void* const* X, const int* nv, const int* ld, int dtype, double* ms) {
  if (!c->built) { c->err = "call oefe_build_hamiltonian first"; return OEFE_ERR_STATE; }
  if (nk < 1 || nk != (int)c->kd.size() || !X || !nv || !ld) { c->err = "autotune: one X, nv, ld per k-point"; return OEFE_ERR_ARG; }
  const bool cplx = c->kd[0].cplx;
  for (int k = 0; k < nk; ++k) {
    OEFE_TRY(check_apply_args(c, k, X[k], nv[k], ld[k], dtype, true));
    if (!c->kd[k].Hbf) { c->err = "autotune: BF16x3 cell matrices were not stored"; return OEFE_ERR_STATE; }
  }
  // low-precision copies of the vectors and product buffers
  const int dt_low = cplx ? OEFE_C64 : OEFE_F32;
  const size_t es_low = dtype_bytes(dt_low);
  const int64_t n = c->nh + c->nO;
  std::vector<size_t> off(nk + 1, 0);
  for (int k = 0; k < nk; ++k)
    off[k + 1] = off[k] + (((size_t)n * nv[k] + (size_t)c->ncells * c->npad * nv[k]) * es_low + 255) / 256 * 256;
  OEFE_TRY(ensure_ws(c, off[nk] + 256));
  std::vector<void*> XL(nk), Z(nk);
  for (int k = 0; k < nk; ++k) {
    XL[k] = (char*)c->ws + off[k];
    Z[k] = (char*)c->ws + off[k] + (size_t)n * nv[k] * es_low;
    const int width = cplx ? 2 * nv[k] : nv[k];
    if (dtype_fp64(dtype)) OEFE_TRY((convert<double, float>(c, X[k], ld[k] * (cplx ? 2 : 1), XL[k], width, n, width)));
    else OEFE_CUDA_TRY(c, cudaMemcpy2DAsync(XL[k], (size_t)nv[k] * es_low, X[k], (size_t)ld[k] * es_low,
                                            (size_t)nv[k] * es_low, (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
  }
  FilterShape cands[6];
  for (int i = 0; i < 6; ++i) cands[i] = filter_shape(c, i);
  // the three-part split has only the TMA kernel; the two-part split also the one-CTA-per-tile
  // kernels; merged MMAs are for complex data, 128-vector TMA tiles for real data
  const int parts = c->kd[0].bf_parts;
  std::vector<int> order;
  if (parts != 3)
    for (int ci = 0; ci < 3; ++ci) order.push_back(ci);
  if (c->d_tmaps) {
    order.push_back(3);
    order.push_back(cplx ? 4 : 5);
  }
  if (order.empty()) { c->err = "autotune: no tensor maps for the split cell matrices"; return OEFE_ERR_STATE; }
  if (ms)
    for (int ci = 0; ci < 6; ++ci) ms[ci] = 0.0;
  double best = 1e300;
  int bi = order[0];
  MmaK* d_mk = nullptr;
  OEFE_TRY(dev_alloc(c, (void**)&d_mk, nk * sizeof(MmaK)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int st = OEFE_OK;
  for (size_t oi = 0; oi < order.size() && st == OEFE_OK; ++oi) {
    const int ci = order[oi];
    std::vector<MmaK> mk(nk);
    long long nt = 0;
    for (int k = 0; k < nk; ++k) {
      mk[k].H = c->kd[k].Hbf;
      mk[k].X = (const float*)XL[k];
      mk[k].Z = (float*)Z[k];
      mk[k].ldx = nv[k];
      mk[k].nv = nv[k];
      mk[k].vblocks = (nv[k] + cands[ci].nb - 1) / cands[ci].nb;
      mk[k].tile0 = nt;
      nt += (long long)c->ncells * mk[k].vblocks;
    }
    cudaMemcpyAsync(d_mk, mk.data(), nk * sizeof(MmaK), cudaMemcpyHostToDevice, c->stream);
    double tbest = 1e300;
    for (int rep = 0; rep < 3 && st == OEFE_OK; ++rep) {
      cudaEventRecord(e0, c->stream);
      if (cands[ci].tma) {
        c->tune_merge = cands[ci].merge;
        st = launch_cell_mma_tma(c, c->d_tmaps, d_mk, nullptr, nk, nt, cplx, parts,
                                 (int)std::min<long long>(nt, c->num_sms), c->stream, cands[ci].nb);
      } else if (cands[ci].grid > 0) {
        st = launch_cell_mma_multi(c, d_mk, nk, nt, cplx, cands[ci].nb, cands[ci].grid, c->stream);
      } else {
        for (int k = 0; k < nk && st == OEFE_OK; ++k)
          st = launch_cell_mma_ptrs(c, XL.size() ? c->kd[k].Hbf : nullptr, XL[k], nv[k], nv[k], Z[k], cplx,
                                    cands[ci].nb, c->stream);
      }
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) tbest = std::min(tbest, (double)t);
    }
    if (ms) ms[ci] = tbest;
    c->tune_ms[ci] = tbest;
    if (tbest < best) { best = tbest; bi = ci; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(c->stream);
  dev_free(d_mk);
  if (st != OEFE_OK) return st;
  int flag = 0;
  OEFE_CUDA_TRY(c, cudaMemcpy(&flag, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    cudaMemset(c->d_status, 0, sizeof(int));
    c->err = "autotune: a tensor-core pipeline wait timed out";
    return OEFE_ERR_TIMEOUT;
  }
  keep_shape(c, cands[bi]);
  return OEFE_OK;
}

void release_batch_graphs(oefe_ctx* c) {
  for (auto& g : c->bgraphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    dev_free(g.params);
  }
  c->bgraphs.clear();
}
