// FP64-class Gram matrices S = X^+ W of the subspace linear algebra (Sec. IV: Cholesky-QR and the
// projected matrices of Rayleigh-Ritz) on the tensor cores, by exact slicing of the operands
// (the Ozaki scheme).
//
// Real form: with A = [Re X | Im X]^T (2 nv rows) and B = [Re W | Im W] (2 nv columns),
// D = A B over the n rows gives Re S = D[i][j] + D[nv+i][nv+j] and Im S = D[i][nv+j] - D[nv+i][j].
// Per pass of 64 rows, each row of A (each column of B) is written as 7 digits of 7 bits with a
// common exponent E_i (F_j):  x = 2^(E-49) (c0 2^42 + c1 2^35 + ... + c6), c0 in [-128, 127], the
// others in [0, 127], exact to 2^(E-49) (truncation of x 2^(49-E) to an integer, taken from the
// bits of x by integer operations). A digit is exact
// in bf16; a product of two digits is at most 2^14 in magnitude (c0 c0 = (-128)^2 = 2^14 is the largest);
// the sum that one accumulator of level d = s + t
// (at most 7 digit pairs) takes over 64 rows stays below 2^24, so the FP32 accumulation of the
// tensor cores is exact. The levels d = 0..6 (28 digit products) are kept, the rest (below
// 2^-49 of the row and column maxima) dropped; levels 6..4 are combined in FP32 (2^-28 below
// level 0, so their rounding is about 2^-51 of it), levels 3..0 in FP32-pair arithmetic, and the
// passes are summed in pairs. Error: about 2^-46 of |x|max |w|max per term.
//
// Two kernels. k_oz_digits (one CTA per pass of 64 rows) writes the digit planes of an operand to
// global memory, already in the 128-byte-swizzled K-major layout the MMA reads, with the
// exponent of each operand row; it touches FP64 values only through their bits (integer
// operations). k_gram_oz (one CTA of 256 threads per (block of passes, half): half 0 takes the
// real parts of W's columns, half 1 the imaginary parts) streams the planes of each pass into
// shared memory with bulk copies; thread 0 issues the 112 MMAs (M 128, N 64, K 16) into 7
// tensor-memory accumulators (448 columns); while every thread reads its part of an accumulator
// row (two warps per lane quadrant, 32 columns each) and adds the combined pass to its running
// sums in pairs, the next pass's planes are already on their way. Every wait is bounded; on a timeout the CTA raises the error flag, waits for its copies and
// MMAs in flight and frees its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "oefe_internal.h"
#include "pair_dev.cuh"
#include "tcgen05_dev.cuh"
#include "ozaki_dev.cuh"

namespace {

constexpr int OZ_T = 256;           // threads per CTA of the MMA kernel: two warps per lane quadrant
constexpr int OZ_C = 32;            // accumulator columns of one thread's running sums
constexpr int OZ_K = 64;            // rows per pass (one 128-byte swizzle row of bf16)
constexpr int OZ_N = 64;            // columns of B per CTA
constexpr int PL = 128 * 128;       // one digit plane: 128 operand rows x 64 bf16
constexpr int PASS_BYTES = OZ_S * PL;
constexpr int BH = OZ_N * 128;      // the half of a plane one CTA takes from B
constexpr size_t OZ_SMEM = 1024 + (size_t)PASS_BYTES + (size_t)OZ_S * BH;
constexpr int OZ_TCOLS = 512;       // tensor-memory columns (7 x 64 used)
constexpr int DG_T = 256;           // threads per CTA of the digits kernel
// Exactness of one accumulator in FP32: at most OZ_S digit pairs per level, each product at most
// 2^14 in magnitude, summed over the rows one accumulator takes (OZ_K for a Gram pass, 2 OZ_K for a
// rotation, whose two K halves share the accumulators), must stay within 2^24.
static_assert((long long)OZ_S * OZ_K * (1LL << 14) <= (1LL << 24), "Gram pass: level sums must be exact in FP32");
static_assert((long long)OZ_S * 2 * OZ_K * (1LL << 14) <= (1LL << 24), "rotation: level sums must be exact in FP32");

__device__ __forceinline__ double ld_part(const void* M, int ld, long long r, int c, int part, bool cplx) {
  if (cplx) {
    const cd v = reinterpret_cast<const cd*>(M)[r * ld + c];
    return part ? v.y : v.x;
  }
  return reinterpret_cast<const double*>(M)[r * ld + c];
}

struct DigArgs {
  const void* M;
  int ld;
  long long n;
  int nv;
  bool cplx;
  bool right;                // operand rows: left (X): [Re cols | Im cols]; right (W): half h = row / 64
  unsigned char* planes;     // per pass PASS_BYTES
  int* exps;                 // per pass 128
};

// operand row r -> (column, part) of M, or -1 when the row is zero
__device__ __forceinline__ int op_col(const DigArgs& D, int r, int* part) {
  if (D.right) {
    *part = r / OZ_N;
    const int c = r % OZ_N;
    return (c < D.nv && (D.cplx || *part == 0)) ? c : -1;
  }
  if (D.cplx) {
    *part = r / max(D.nv, 1);
    return r < 2 * D.nv ? r % D.nv : -1;
  }
  *part = 0;
  return r < D.nv ? r : -1;
}

__global__ void __launch_bounds__(DG_T) k_oz_digits(const DigArgs D) {
  extern __shared__ unsigned long long dbits[];    // [128 operand rows][65]: bits of the pass, padded
  __shared__ int sE[128];
  const long long p = blockIdx.x, r0 = p * OZ_K;
  const int nk = (int)min((long long)OZ_K, D.n - r0);
  // loads: a warp takes 32 consecutive operand rows (consecutive columns of M) of one row of M;
  // eight loads in flight per thread
  for (int t0 = threadIdx.x; t0 < OZ_K * 128; t0 += 8 * DG_T) {
    unsigned long long v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * DG_T;
      const int k = t / 128, r = t % 128;
      int part;
      const int c = op_col(D, r, &part);
      v[u] = (t < OZ_K * 128 && c >= 0 && k < nk)
                 ? (unsigned long long)__double_as_longlong(ld_part(D.M, D.ld, r0 + k, c, part, D.cplx))
                 : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * DG_T;
      if (t < OZ_K * 128) dbits[(t % 128) * 65 + t / 128] = v[u];
    }
  }
  __syncthreads();
  if (threadIdx.x < 128) {
    int mex = 0;
    for (int k = 0; k < OZ_K; ++k) mex = max(mex, (int)((dbits[threadIdx.x * 65 + k] >> 52) & 0x7FF));
    const int E = mex ? mex - 1022 : 0;
    sE[threadIdx.x] = E;
    D.exps[p * 128 + threadIdx.x] = E;
  }
  __syncthreads();
  unsigned char* base = D.planes + (size_t)p * PASS_BYTES;
  for (int t = threadIdx.x; t < 128 * (OZ_K / 2); t += DG_T) {   // a warp: one row, 32 pairs of k
    const int r = t / (OZ_K / 2), kp = t % (OZ_K / 2);
    float c0[OZ_S], c1[OZ_S];
    digits7(dbits[r * 65 + 2 * kp], sE[r], c0);
    digits7(dbits[r * 65 + 2 * kp + 1], sE[r], c1);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s)
      *reinterpret_cast<__nv_bfloat162*>(base + (size_t)s * PL + swz(r, 2 * kp)) = __floats2bfloat162_rn(c0[s], c1[s]);
  }
}

struct OzArgs {
  const unsigned char* pa;   // digit planes of X (left operand), per pass PASS_BYTES
  const int* ea;             // exponents of X's operand rows, per pass 128
  const unsigned char* pb;   // digit planes of W (right operand)
  const int* eb;
  long long passes;
  long long passes_per_cta;
  bool cplx;
  int nv;
  double* part;              // (halves, blocks, 128, 64)
  int* err;
};

__global__ void __launch_bounds__(OZ_T, 1) k_gram_oz(const OzArgs A) {
  extern __shared__ __align__(1024) unsigned char oz_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + PASS_BYTES;
  __shared__ int Fexp[OZ_N];
  __shared__ uint64_t ld_bar, mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int half = blockIdx.y;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(OZ_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&ld_bar, 1);
    mbar_init(&mma_bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_slot;

  const long long pb = (long long)blockIdx.x * A.passes_per_cta, pe = min(A.passes, pb + A.passes_per_cta);
  const int nrowA = A.cplx ? 2 * A.nv : A.nv;
  const int row = tid & 127, ch = tid >> 7;   // accumulator row (tensor-memory lane) and column half
  auto load_pass = [&](long long p) {   // thread 0: the planes of pass p into shared memory
    mbar_expect_tx(&ld_bar, (uint32_t)(PASS_BYTES + OZ_S * BH));
    bulk_copy(smem_u32(sA), A.pa + (size_t)p * PASS_BYTES, PASS_BYTES, &ld_bar);
    for (int s = 0; s < OZ_S; ++s)
      bulk_copy(smem_u32(sB + s * BH), A.pb + (size_t)p * PASS_BYTES + (size_t)s * PL + (size_t)half * BH, BH, &ld_bar);
  };
  if (tid == 0 && pb < pe) load_pass(pb);
  f2 R[OZ_C];
#pragma unroll
  for (int j = 0; j < OZ_C; ++j) R[j] = f2{0.0f, 0.0f};
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  constexpr uint32_t ID = idesc_bf16(128, OZ_N, false);
  int it = 0;
  bool loads_out = pb < pe, mma_out = false;
  for (long long p = pb; p < pe; ++p, ++it) {
    bool ok = mbar_wait(&ld_bar, (uint32_t)(it & 1), &s_fail);
    if (__syncthreads_or(!ok)) { s_fail = 1; break; }
    loads_out = false;
    // the exponents of this pass, loaded while the MMAs run
    const int E = A.ea[p * 128 + row];
    if (tid < OZ_N) Fexp[tid] = A.eb[p * 128 + half * OZ_N + tid];
    // ---- the digit products of levels d = s + t <= 6 into accumulator d
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int d = 0; d < OZ_S; ++d)
#pragma unroll 1
        for (int s = 0; s <= d; ++s) {
          const int t = d - s;
#pragma unroll
          for (int ks = 0; ks < OZ_K / 16; ++ks)
            mma_bf16(taddr + d * OZ_N, sdesc(smem_u32(sA + s * PL) + ks * 32), sdesc(smem_u32(sB + t * BH) + ks * 32),
                     ID, (s == 0 && ks == 0) ? 0u : 1u);
        }
      mma_commit(&mma_bar);
    }
    mma_out = true;
    ok = mbar_wait(&mma_bar, (uint32_t)(it & 1), &s_fail);
    if (__syncthreads_or(!ok)) { s_fail = 1; break; }
    mma_out = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the planes are free: the next pass's copies run during this pass's epilogue
    if (tid == 0 && p + 1 < pe) load_pass(p + 1);
    loads_out = p + 1 < pe;
    // ---- combine the levels of (row, this half of the columns) and add them to the running sums;
    //      the scalings are exact multiplications by powers of two
#pragma unroll
    for (int g = 0; g < OZ_C / 16; ++g) {
      const int c0 = ch * OZ_C + 16 * g;
      // levels 6, 5, 4 by FP32 Horner steps in units of level 4 (their rounding, 2^-24 of a
      // quantity 2^-28 below level 0, is far below the pair precision); levels 3..0 in pairs
      float lo[16];
      {
        float v[16];
        tmem_ld16(taddr + lane_base + 6 * OZ_N + c0, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) lo[c] = v[c];
#pragma unroll
        for (int d = 5; d >= 4; --d) {
          tmem_ld16(taddr + lane_base + d * OZ_N + c0, v);
#pragma unroll
          for (int c = 0; c < 16; ++c) lo[c] = __fmaf_rn(lo[c], 0.0078125f, v[c]);
        }
      }
      f2 S[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) S[c] = f2{__fmul_rn(lo[c], 3.7252902984619141e-09f), 0.0f};   // 2^-28
#pragma unroll 1
      for (int d = 3; d >= 0; --d) {
        float v[16];
        tmem_ld16(taddr + lane_base + d * OZ_N + c0, v);
        const float w = __int_as_float((127 - 7 * d) << 23);   // 2^(-7 d)
#pragma unroll
        for (int c = 0; c < 16; ++c) S[c] = f2_add(S[c], f2{__fmul_rn(v[c], w), 0.0f});
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int sc = E + Fexp[c0 + c] - 14;
        f2 x;
        if (sc > -127 && sc < 128) {
          const float w = __int_as_float((sc + 127) << 23);
          x = f2{__fmul_rn(S[c].h, w), __fmul_rn(S[c].l, w)};
        } else {
          x = f2{ldexpf(S[c].h, sc), ldexpf(S[c].l, sc)};
        }
        R[16 * g + c] = f2_add(R[16 * g + c], x);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // copies and MMAs in flight have landed before the shared and tensor memory are released
  if (tid == 0 && s_fail) {
    if (mma_out) mbar_wait_drain(&mma_bar, (uint32_t)(it & 1));
    if (loads_out) mbar_wait_drain(&ld_bar, (uint32_t)(it & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (row < nrowA && !s_fail) {
    double* out = A.part + (((size_t)half * gridDim.x + blockIdx.x) * 128 + row) * OZ_N + ch * OZ_C;
#pragma unroll
    for (int j = 0; j < OZ_C; ++j) out[j] = f2_to(R[j]);
  }
  if (s_fail && tid == 0) atomicExch(A.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(OZ_TCOLS) : "memory");
}

// ------------------------------------------------------------------ rotations X <- X G
// Real form: A = the rows of X with K = [Re X | Im X] (K half 0: real parts of the 64 columns, half 1:
// imaginary parts), B = the real form of G, N half 0 the real parts of the products, half 1 the
// imaginary parts: B[(0, j)][(0, n)] = Re G_jn, B[(0, j)][(1, n)] = Im G_jn, B[(1, j)][(0, n)] =
// -Im G_jn, B[(1, j)][(1, n)] = Re G_jn. The exponent of an A row covers both K halves, so the two
// halves accumulate into the same (exact) accumulators: 7 pairs x 128 x 2^14 <= 2^24.

struct RotDigArgs {
  const void* X;
  int ldx;
  long long n;
  int nv;
  bool cplx;
  unsigned char* planes;   // per tile of 128 rows: 2 K halves x PASS_BYTES
  int* exps;               // per tile 128
};

// digits of 128 rows of X (one CTA per tile)
__global__ void __launch_bounds__(DG_T) k_oz_rot_digits(const RotDigArgs D) {
  extern __shared__ unsigned long long rbits[];   // [128 rows][129]: both K halves, padded
  __shared__ int sE[128];
  const long long tile = blockIdx.x, r0 = tile * 128;
  const int nr = (int)min(128ll, D.n - r0);
  const int kh_n = D.cplx ? 2 : 1;
  for (int t0 = threadIdx.x; t0 < 128 * 128; t0 += 8 * DG_T) {
    unsigned long long v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * DG_T;
      const int r = t / 128, k = t % 128, part = k / 64, c = k % 64;   // consecutive threads: one row
      v[u] = (t < 128 * 128 && r < nr && c < D.nv && part < kh_n)
                 ? (unsigned long long)__double_as_longlong(ld_part(D.X, D.ldx, r0 + r, c, part, D.cplx))
                 : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * DG_T;
      if (t < 128 * 128) rbits[(t / 128) * 129 + t % 128] = v[u];
    }
  }
  __syncthreads();
  if (threadIdx.x < 128) {
    int mex = 0;
    for (int k = 0; k < 128; ++k) mex = max(mex, (int)((rbits[threadIdx.x * 129 + k] >> 52) & 0x7FF));
    const int E = mex ? mex - 1022 : 0;
    sE[threadIdx.x] = E;
    D.exps[tile * 128 + threadIdx.x] = E;
  }
  __syncthreads();
  unsigned char* base = D.planes + (size_t)tile * 2 * PASS_BYTES;
  for (int t = threadIdx.x; t < 2 * 128 * (OZ_K / 2); t += DG_T) {   // a warp: one row, 32 pairs of k
    const int kh = t / (128 * (OZ_K / 2)), rem = t % (128 * (OZ_K / 2));
    const int r = rem / (OZ_K / 2), kp = rem % (OZ_K / 2);
    float c0[OZ_S], c1[OZ_S];
    digits7(rbits[r * 129 + kh * 64 + 2 * kp], sE[r], c0);
    digits7(rbits[r * 129 + kh * 64 + 2 * kp + 1], sE[r], c1);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s)
      *reinterpret_cast<__nv_bfloat162*>(base + (size_t)kh * PASS_BYTES + (size_t)s * PL + swz(r, 2 * kp)) =
          __floats2bfloat162_rn(c0[s], c1[s]);
  }
}

// digits of the real form of G (one thread per B column = N index n of half nh): planes
// [nh][kh][digit][64 rows][64 k], exponents [nh][64]; G[k][j] = herm ? (k <= j ? conj(C[j][k]) : 0) : C[k][j]
template <typename S>
__global__ void k_oz_rot_bdigits(const S* C, int nv, bool herm, unsigned char* planes, int* exps) {
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // 0..127: (nh, n)
  if (t >= 128) return;
  const int nh = t / 64, n = t % 64;
  auto G = [&](int k, int j) -> cd {   // entry of the rotation applied as X G
    if (k >= nv || j >= nv) return mkc(0, 0);
    cd v;
    if (herm) {
      if (k > j) return mkc(0, 0);
      if constexpr (CPLX) v = cconj(C[(size_t)j * nv + k]);
      else v = mkc(C[(size_t)j * nv + k], 0.0);
    } else {
      if constexpr (CPLX) v = C[(size_t)k * nv + j];
      else v = mkc(C[(size_t)k * nv + j], 0.0);
    }
    return v;
  };
  auto Bv = [&](int k) -> double {   // B[k][(nh, n)], k = (kh, j)
    const int kh = k / 64, j = k % 64;
    const cd g = G(j, n);
    if (kh == 0) return nh == 0 ? g.x : g.y;
    return nh == 0 ? -g.y : g.x;
  };
  int mex = 0;
  for (int k = 0; k < 128; ++k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(Bv(k));
    mex = max(mex, (int)((b >> 52) & 0x7FF));
  }
  const int E = mex ? mex - 1022 : 0;
  exps[nh * 64 + n] = E;
  for (int kh = 0; kh < 2; ++kh)
    for (int kp = 0; kp < OZ_K / 2; ++kp) {
      float c0[OZ_S], c1[OZ_S];
      digits7((unsigned long long)__double_as_longlong(Bv(kh * 64 + 2 * kp)), E, c0);
      digits7((unsigned long long)__double_as_longlong(Bv(kh * 64 + 2 * kp + 1)), E, c1);
      unsigned char* base = planes + (size_t)(nh * 2 + kh) * OZ_S * BH;
#pragma unroll
      for (int s = 0; s < OZ_S; ++s)
        *reinterpret_cast<__nv_bfloat162*>(base + (size_t)s * BH + swz(n, 2 * kp)) = __floats2bfloat162_rn(c0[s], c1[s]);
    }
}

struct RotArgs {
  const unsigned char* pa;   // tile digit planes (2 K halves per tile)
  const int* ea;             // tile row exponents
  const unsigned char* pb;   // G digit planes [nh][kh]
  const int* eb;             // [nh][64]
  long long tiles;
  long long n;
  int nv;
  bool cplx;
  void* X;                   // output rows (double or cd), ld
  int ldx;
  int* err;
};

__global__ void __launch_bounds__(OZ_T, 1) k_rot_oz(const RotArgs A) {
  extern __shared__ __align__(1024) unsigned char oz_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + PASS_BYTES;
  __shared__ int Fexp[OZ_N];
  __shared__ uint64_t ld_bar, mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(OZ_TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&ld_bar, 1);
    mbar_init(&mma_bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_slot;
  const int row = tid & 127, ch = tid >> 7;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  constexpr uint32_t ID = idesc_bf16(128, OZ_N, false);
  const int nkh = A.cplx ? 2 : 1, nnh = A.cplx ? 2 : 1;
  const int rounds = nkh * nnh;   // (nh, kh), kh fastest
  // the rounds of this CTA: tiles blockIdx.x, blockIdx.x + gridDim.x, ...
  auto load_round = [&](long long tile, int nh, int kh) {
    mbar_expect_tx(&ld_bar, (uint32_t)(PASS_BYTES + OZ_S * BH));
    bulk_copy(smem_u32(sA), A.pa + ((size_t)tile * 2 + kh) * PASS_BYTES, PASS_BYTES, &ld_bar);
    bulk_copy(smem_u32(sB), A.pb + (size_t)(nh * 2 + kh) * OZ_S * BH, OZ_S * BH, &ld_bar);
  };
  long long tile = blockIdx.x;
  int q = 0;   // round within the tile
  if (tid == 0 && tile < A.tiles) load_round(tile, 0, 0);
  int it = 0;
  bool loads_out = tile < A.tiles, mma_out = false;
  while (tile < A.tiles) {
    const int nh = q / nkh, kh = q % nkh;
    bool ok = mbar_wait(&ld_bar, (uint32_t)(it & 1), &s_fail);
    if (__syncthreads_or(!ok)) { s_fail = 1; break; }
    loads_out = false;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int d = 0; d < OZ_S; ++d)
#pragma unroll 1
        for (int s = 0; s <= d; ++s) {
          const int t = d - s;
#pragma unroll
          for (int ks = 0; ks < OZ_K / 16; ++ks)
            mma_bf16(taddr + d * OZ_N, sdesc(smem_u32(sA + s * PL) + ks * 32), sdesc(smem_u32(sB + t * BH) + ks * 32),
                     ID, (kh == 0 && s == 0 && ks == 0) ? 0u : 1u);
        }
      mma_commit(&mma_bar);
    }
    mma_out = true;
    ok = mbar_wait(&mma_bar, (uint32_t)(it & 1), &s_fail);
    if (__syncthreads_or(!ok)) { s_fail = 1; break; }
    mma_out = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ++it;
    // next round (this tile's next (nh, kh), or the CTA's next tile): its copies run during the epilogue
    const long long cur_tile = tile;
    ++q;
    if (q == rounds) { q = 0; tile += gridDim.x; }
    if (tid == 0 && tile < A.tiles) load_round(tile, q / nkh, q % nkh);
    loads_out = tile < A.tiles;
    if (kh == nkh - 1) {
      // ---- epilogue of (cur_tile, nh): 32 columns of one row per thread
      const long long grow = cur_tile * 128 + row;
      const int E = A.ea[cur_tile * 128 + row];
      if (tid < OZ_N) Fexp[tid] = A.eb[nh * 64 + tid];
      __syncthreads();
#pragma unroll
      for (int g = 0; g < OZ_C / 16; ++g) {
        const int c0 = ch * OZ_C + 16 * g;
        float lo[16];
        {
          float v[16];
          tmem_ld16(taddr + lane_base + 6 * OZ_N + c0, v);
#pragma unroll
          for (int c = 0; c < 16; ++c) lo[c] = v[c];
#pragma unroll
          for (int d = 5; d >= 4; --d) {
            tmem_ld16(taddr + lane_base + d * OZ_N + c0, v);
#pragma unroll
            for (int c = 0; c < 16; ++c) lo[c] = __fmaf_rn(lo[c], 0.0078125f, v[c]);
          }
        }
        f2 S[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) S[c] = f2{__fmul_rn(lo[c], 3.7252902984619141e-09f), 0.0f};   // 2^-28
#pragma unroll 1
        for (int d = 3; d >= 0; --d) {
          float v[16];
          tmem_ld16(taddr + lane_base + d * OZ_N + c0, v);
          const float w = __int_as_float((127 - 7 * d) << 23);
#pragma unroll
          for (int c = 0; c < 16; ++c) S[c] = f2_add(S[c], f2{__fmul_rn(v[c], w), 0.0f});
        }
        if (grow < A.n) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int col = c0 + c;
            if (col >= A.nv) continue;
            const int sc = E + Fexp[col] - 14;
            const double val = f_scaled(S[c].h, sc) + f_scaled(S[c].l, sc);
            if (A.cplx) {
              double* xr = reinterpret_cast<double*>(A.X) + 2 * ((size_t)grow * A.ldx + col);
              xr[nh] = val;
            } else {
              reinterpret_cast<double*>(A.X)[(size_t)grow * A.ldx + col] = val;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  if (tid == 0 && s_fail) {
    if (mma_out) mbar_wait_drain(&mma_bar, (uint32_t)(it & 1));
    if (loads_out) mbar_wait_drain(&ld_bar, (uint32_t)(it & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) atomicExch(A.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(OZ_TCOLS) : "memory");
}

// S from the partial sums of all blocks: Re S = D[i][j] + D[nv+i][nv+j], Im S = D[i][nv+j] - D[nv+i][j]
template <typename S>
__global__ void k_gram_oz_reduce(const double* part, int nbx, int nv, S* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nv) return;
  const int i = t / nv, j = t % nv;
  auto P = [&](int h, int b, int row, int col) { return part[(((size_t)h * nbx + b) * 128 + row) * OZ_N + col]; };
  double re = 0.0, im = 0.0;
  for (int b = 0; b < nbx; ++b) {
    if constexpr (sizeof(S) == sizeof(cd)) {
      re += P(0, b, i, j) + P(1, b, nv + i, j);
      im += P(1, b, i, j) - P(0, b, nv + i, j);
    } else {
      re += P(0, b, i, j);
    }
  }
  if constexpr (sizeof(S) == sizeof(cd)) out[t] = mkc(re, im);
  else out[t] = re;
}

}  // namespace

// out = X^+ W (nv x nv) on the tensor cores; *done = false when the shape is not covered (nv > 64)
template <typename S>
int gram_ozaki(oefe_ctx* c, const S* X, int ldx, const S* W, int ldw, int64_t n, int nv, S* out, bool* done) {
  *done = false;
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  if (nv > OZ_N || n <= 0) return OEFE_OK;
  const int halves = CPLX ? 2 : 1;
  const int nbx = std::max(1, c->num_sms / halves);
  const long long passes = (n + OZ_K - 1) / OZ_K;
  auto a256 = [](size_t x) { return ((x + 255) / 256) * 256; };
  const size_t pl_bytes = a256((size_t)passes * PASS_BYTES), ex_bytes = a256((size_t)passes * 128 * sizeof(int));
  const size_t pt_bytes = a256((size_t)halves * nbx * 128 * OZ_N * sizeof(double));
  const size_t need = 2 * pl_bytes + 2 * ex_bytes + pt_bytes;
  if (c->ozpart_bytes < need) {
    cudaStreamSynchronize(c->stream);
    dev_free(c->d_ozpart);
    c->d_ozpart = nullptr;
    c->ozpart_bytes = 0;
    OEFE_TRY(dev_alloc(c, &c->d_ozpart, need));
    c->ozpart_bytes = need;
  }
  unsigned char* base = (unsigned char*)c->d_ozpart;
  unsigned char* pa = base;
  unsigned char* pbp = base + pl_bytes;
  int* ea = (int*)(base + 2 * pl_bytes);
  int* eb = (int*)(base + 2 * pl_bytes + ex_bytes);
  double* part = (double*)(base + 2 * pl_bytes + 2 * ex_bytes);
  const size_t dsm = (size_t)128 * 65 * sizeof(unsigned long long);
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_oz_digits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
  DigArgs D{X, ldx, n, nv, CPLX, false, pa, ea};
  OEFE_COUNTED k_oz_digits<<<(unsigned)passes, DG_T, dsm, c->stream>>>(D);
  D = DigArgs{W, ldw, n, nv, CPLX, true, pbp, eb};
  OEFE_COUNTED k_oz_digits<<<(unsigned)passes, DG_T, dsm, c->stream>>>(D);
  OzArgs A;
  A.pa = pa;
  A.ea = ea;
  A.pb = pbp;
  A.eb = eb;
  A.passes = passes;
  A.passes_per_cta = (passes + nbx - 1) / nbx;
  A.cplx = CPLX;
  A.nv = nv;
  A.part = part;
  A.err = c->d_status + 2;   // its own word: the Cholesky kernels report through word 0
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  dim3 grid(nbx, halves);
  OEFE_COUNTED k_gram_oz<<<grid, OZ_T, OZ_SMEM, c->stream>>>(A);
  OEFE_COUNTED k_gram_oz_reduce<S><<<(nv * nv + 255) / 256, 256, 0, c->stream>>>(part, nbx, nv, out);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  int flag = 0;
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (flag) {
    cudaMemsetAsync(c->d_status + 2, 0, sizeof(int), c->stream);
    c->err = "gram: a tensor-core wait timed out";
    return OEFE_ERR_TIMEOUT;
  }
  *done = true;
  return OEFE_OK;
}

template int gram_ozaki<double>(oefe_ctx*, const double*, int, const double*, int, int64_t, int, double*, bool*);
template int gram_ozaki<cd>(oefe_ctx*, const cd*, int, const cd*, int, int64_t, int, cd*, bool*);

// X[0:n] <- X G (G = C, or C^+ of a lower triangular C when herm) on the tensor cores; *done =
// false when the shape is not covered (nv > 64)
template <typename S>
int rotate_ozaki(oefe_ctx* c, S* X, int ldx, int64_t n, int nv, const S* C, bool herm, bool* done) {
  *done = false;
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  if (nv > OZ_N || n <= 0) return OEFE_OK;
  const long long tiles = (n + 127) / 128;
  auto a256 = [](size_t x) { return ((x + 255) / 256) * 256; };
  const size_t pa_bytes = a256((size_t)tiles * 2 * PASS_BYTES), ea_bytes = a256((size_t)tiles * 128 * sizeof(int));
  const size_t pb_bytes = a256((size_t)4 * OZ_S * BH), eb_bytes = 256 + 128 * sizeof(int);
  const size_t need = pa_bytes + ea_bytes + pb_bytes + eb_bytes;
  if (c->ozpart_bytes < need) {
    cudaStreamSynchronize(c->stream);
    dev_free(c->d_ozpart);
    c->d_ozpart = nullptr;
    c->ozpart_bytes = 0;
    OEFE_TRY(dev_alloc(c, &c->d_ozpart, need));
    c->ozpart_bytes = need;
  }
  unsigned char* base = (unsigned char*)c->d_ozpart;
  unsigned char* pa = base;
  int* ea = (int*)(base + pa_bytes);
  unsigned char* pb = base + pa_bytes + ea_bytes;
  int* eb = (int*)(pb + pb_bytes);
  const size_t dsm = (size_t)128 * 129 * sizeof(unsigned long long);
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_oz_rot_digits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
  RotDigArgs D{X, ldx, n, nv, CPLX, pa, ea};
  OEFE_COUNTED k_oz_rot_digits<<<(unsigned)tiles, DG_T, dsm, c->stream>>>(D);
  OEFE_COUNTED k_oz_rot_bdigits<S><<<1, 128, 0, c->stream>>>(C, nv, herm, pb, eb);
  RotArgs A;
  A.pa = pa;
  A.ea = ea;
  A.pb = pb;
  A.eb = eb;
  A.tiles = tiles;
  A.n = n;
  A.nv = nv;
  A.cplx = CPLX;
  A.X = X;
  A.ldx = ldx;
  A.err = c->d_status + 2;
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_rot_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM));
  const int grid = (int)std::min<long long>(tiles, c->num_sms);
  OEFE_COUNTED k_rot_oz<<<grid, OZ_T, OZ_SMEM, c->stream>>>(A);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  int flag = 0;
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (flag) {
    cudaMemsetAsync(c->d_status + 2, 0, sizeof(int), c->stream);
    c->err = "rotate: a tensor-core wait timed out";
    return OEFE_ERR_TIMEOUT;
  }
  *done = true;
  return OEFE_OK;
}

template int rotate_ozaki<double>(oefe_ctx*, double*, int, int64_t, int, const double*, bool, bool*);
template int rotate_ozaki<cd>(oefe_ctx*, cd*, int, int64_t, int, const cd*, bool, bool*);
