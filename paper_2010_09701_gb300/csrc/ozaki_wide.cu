// FP64-class Gram matrices and rotations of wide vector blocks (more than the 64 vectors the
// plane-based kernels of ozaki_gram.cu take) on the tensor cores, with the same exact bf16 digit
// slicing (the Ozaki scheme): every operand value is cut into 7 digits of 7 bits under a common
// exponent per operand row and K chunk, the 28 digit products of levels d = s + t <= 6 are
// accumulated exactly in FP32 in tensor memory (7 accumulators of 64 columns), and the levels are
// combined in FP32 pairs, scaled by exact powers of two and summed over the chunks in pairs.
//
// Unlike the plane-based kernels, the digits are cut inside the MMA kernels into shared memory
// (nothing is staged in global memory but the small rotation matrix's digits), so wide blocks need
// no digit planes the size of the operands. One round = one K chunk of 64 real entries for one
// tile of 128 operand rows and 64 output columns: 112 MMAs (M 128, N 64, K 16).
//
//   Gram S = X^+ W: real form A = [Re X | Im X]^T (2 nv operand rows, nv for real data), B = [Re W |
//   Im W] (2 nv columns); K = the rows of the blocks in passes of 64. A CTA takes one (128-row,
//   64-column) tile of D = A B over a range of passes; D's partial sums are combined afterwards:
//   Re S = D[i][j] + D[nv+i][nv+j], Im S = D[i][nv+j] - D[nv+i][j].
//
//   Rotation X <- X G: A = rows of X, a K chunk = 64 columns (real) or [Re | Im] of 32 complex
//   columns; B = the matching rows of the real form of G for 64 output columns (the real parts, or
//   the imaginary parts, of 64 complex output columns). A CTA takes whole tiles of 128 rows, the K
//   chunks outermost (the A digits of a chunk cut once for all output blocks), every output block's
//   FP32-pair partial sums in a staging area, so the in-place update never reads a row it has
//   written.
//
// Every wait is bounded; on a timeout the CTA raises the error flag, lets its copies and MMAs in
// flight land, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "oefe_internal.h"
#include "pair_dev.cuh"
#include "tcgen05_dev.cuh"
#include "ozaki_dev.cuh"

namespace {

constexpr int WT = 256;                 // threads per CTA
constexpr int WK = 64;                  // real K entries per round (one 128-byte swizzle row of bf16)
constexpr int WN = 64;                  // output columns per round
constexpr int PLA = 128 * 128;          // bytes of one A digit plane: 128 operand rows x 64 bf16
constexpr int PLB = WN * 128;           // bytes of one B digit plane: 64 rows x 64 bf16
constexpr size_t WSMEM = 1024 + (size_t)OZ_S * PLA + (size_t)OZ_S * PLB;
constexpr int WTCOLS = 512;             // tensor-memory columns (7 x 64 used)
// the FP32 accumulation of a level (at most OZ_S digit pairs, products at most 2^14) over the
// WK entries of a round stays exact
static_assert((long long)OZ_S * WK * (1LL << 14) <= (1LL << 24), "level sums must be exact in FP32");

__device__ __forceinline__ int bexp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// the 7 digits of two consecutive K entries (kk, kk + 1) of operand row r into the planes at base
__device__ __forceinline__ void put_pair(unsigned char* base, int plane_bytes, int r, int kk, double v0, double v1,
                                         int E) {
  float c0[OZ_S], c1[OZ_S];
  digits7((unsigned long long)__double_as_longlong(v0), E, c0);
  digits7((unsigned long long)__double_as_longlong(v1), E, c1);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s)
    *reinterpret_cast<__nv_bfloat162*>(base + (size_t)s * plane_bytes + swz(r, kk)) = __floats2bfloat162_rn(c0[s], c1[s]);
}

// thread 0: the digit products of levels d = s + t <= 6 into accumulator d
__device__ __forceinline__ void issue_round(uint32_t taddr, uint32_t sA, uint32_t sB) {
  constexpr uint32_t ID = idesc_bf16(128, WN, false);
#pragma unroll 1
  for (int d = 0; d < OZ_S; ++d)
#pragma unroll 1
    for (int s = 0; s <= d; ++s) {
      const int t = d - s;
#pragma unroll
      for (int ks = 0; ks < WK / 16; ++ks)
        mma_bf16(taddr + d * WN, sdesc(sA + s * PLA + ks * 32), sdesc(sB + t * PLB + ks * 32), ID,
                 (s == 0 && ks == 0) ? 0u : 1u);
    }
}

// the levels of (row, 32 columns ch*32 ..) combined and added to the running pair sums R:
// levels 6..4 by FP32 Horner steps in units of level 4, levels 3..0 in pairs, scaled by
// 2^(E + F_col - 14) (exact powers of two)
__device__ __forceinline__ void add_levels(uint32_t taddr, uint32_t lane_base, int ch, int E, const int* Fexp,
                                           f2* R) {
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int c0 = ch * 32 + 16 * g;
    float lo[16];
    {
      float v[16];
      tmem_ld16(taddr + lane_base + 6 * WN + c0, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) lo[c] = v[c];
#pragma unroll
      for (int d = 5; d >= 4; --d) {
        tmem_ld16(taddr + lane_base + d * WN + c0, v);
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
      tmem_ld16(taddr + lane_base + d * WN + c0, v);
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
}

__device__ __forceinline__ void tmem_alloc_cta(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(WTCOLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free_cta(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(WTCOLS) : "memory");
}

// operand value of the Gram's real form: index ra < nv the real part of column ra, nv <= ra < 2 nv
// the imaginary part of column ra - nv (complex), zero beyond
__device__ __forceinline__ double gram_op(const void* M, int ld, long long g, int ra, int nv, bool cplx) {
  if (!cplx) return ra < nv ? reinterpret_cast<const double*>(M)[g * ld + ra] : 0.0;
  if (ra < nv) return reinterpret_cast<const cd*>(M)[g * ld + ra].x;
  if (ra < 2 * nv) return reinterpret_cast<const cd*>(M)[g * ld + ra - nv].y;
  return 0.0;
}

struct WGramArgs {
  const void* X;
  int ldx;
  const void* W;
  int ldw;
  long long n;
  int nv;
  bool cplx;
  int nI, nJ;                // tiles of 128 A rows and 64 B columns of D
  bool upper;                // symmetric result: only the tiles (I, J >= 2 I) that meet the upper triangle
  long long passes, ppc;     // passes of 64 rows, passes per CTA
  double* part;              // [block][I][J][128][64]
  int* err;
};

__global__ void __launch_bounds__(WT, 1) k_gram_wide(const WGramArgs A) {
  extern __shared__ __align__(1024) unsigned char wz_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)wz_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + OZ_S * PLA;
  __shared__ int sE[128], Fexp[WN];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tmem_alloc_cta(&tmem_slot);
  if (tid == 0) {
    mbar_init(&mma_bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_slot;
  int I = blockIdx.y / A.nJ, J = blockIdx.y % A.nJ;
  if (A.upper) {   // blockIdx.y enumerates the tiles with J >= 2 I row by row
    int y = blockIdx.y;
    I = 0;
    while (y >= A.nJ - 2 * I) {
      y -= A.nJ - 2 * I;
      ++I;
    }
    J = 2 * I + y;
  }
  const long long pb = (long long)blockIdx.x * A.ppc, pe = min(A.passes, pb + A.ppc);
  const int row = tid & 127, ch = tid >> 7;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  f2 R[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) R[j] = f2{0.0f, 0.0f};
  int it = 0;
  bool mma_out = false;
  for (long long p = pb; p < pe; ++p, ++it) {
    const long long g0 = p * 64;
    const int ng = (int)min(64ll, A.n - g0);
    // digits: threads 0..127 one A operand row each, threads 128..191 one B operand column each,
    // over the pass's 64 rows (a warp's loads of one row are consecutive columns)
    if (tid < 192) {
      const bool isA = tid < 128;
      const int r = isA ? tid : tid - 128;
      const int ra = isA ? I * 128 + r : J * WN + r;
      const void* M = isA ? A.X : A.W;
      const int ld = isA ? A.ldx : A.ldw;
      // register u holds K entry (u + 2 s) mod 64, s = (r / 8) mod 4: at the store of register pair q
      // the 32 lanes of a warp (rows with 8 values of r mod 8, 4 of s) write 32 different banks
      const int sh = 2 * ((r >> 3) & 3);
      double v[64];
      int mex = 0;
#pragma unroll
      for (int u = 0; u < 64; ++u) {
        const int kk = (u + sh) & 63;
        v[u] = kk < ng ? gram_op(M, ld, g0 + kk, ra, A.nv, A.cplx) : 0.0;
        mex = max(mex, bexp(v[u]));
      }
      const int E = mex ? mex - 1022 : 0;
      unsigned char* base = isA ? sA : sB;
      const int pbytes = isA ? PLA : PLB;
#pragma unroll
      for (int q = 0; q < 32; ++q) put_pair(base, pbytes, r, (2 * q + sh) & 63, v[2 * q], v[2 * q + 1], E);
      if (isA) sE[r] = E;
      else Fexp[r] = E;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue_round(taddr, smem_u32(sA), smem_u32(sB));
      mma_commit(&mma_bar);
    }
    mma_out = true;
    const bool ok = mbar_wait(&mma_bar, (uint32_t)(it & 1), &s_fail);
    if (__syncthreads_or(!ok)) { s_fail = 1; break; }
    mma_out = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    add_levels(taddr, lane_base, ch, sE[row], Fexp, R);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (tid == 0 && s_fail && mma_out) mbar_wait_drain(&mma_bar, (uint32_t)(it & 1));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (!s_fail) {
    double* out = A.part + ((((size_t)blockIdx.x * A.nI + I) * A.nJ + J) * 128 + row) * WN + ch * 32;
#pragma unroll
    for (int j = 0; j < 32; ++j) out[j] = f2_to(R[j]);
  }
  if (s_fail && tid == 0) atomicExch(A.err, 1);
  if (warp == 0) tmem_free_cta(taddr);
}

// S from the partial sums of all blocks (real form combined for complex data)
template <typename S>
__global__ void k_gram_wide_reduce(const double* part, int nbx, int nI, int nJ, int nv, bool upper, S* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nv) return;
  // upper (real symmetric result): entry (i, j) below the diagonal is entry (j, i), which lies in a
  // computed tile (column tile j / 64 >= 2 (row tile i / 128) whenever i <= j)
  const int i = upper ? min(t / nv, t % nv) : t / nv, j = upper ? max(t / nv, t % nv) : t % nv;
  auto D = [&](int ra, int rb) {
    double s = 0.0;
    for (int b = 0; b < nbx; ++b)
      s += part[((((size_t)b * nI + ra / 128) * nJ + rb / WN) * 128 + ra % 128) * WN + rb % WN];
    return s;
  };
  if constexpr (sizeof(S) == sizeof(cd)) out[t] = mkc(D(i, j) + D(nv + i, nv + j), D(i, nv + j) - D(nv + i, j));
  else out[t] = D(i, j);
}

// ------------------------------------------------------------------ rotation X <- X G
// A K entry kk of chunk kc: real data column kc * 64 + kk; complex data [Re | Im] of the columns
// kc * 32 + (kk mod 32)
__device__ __forceinline__ double rot_op(const void* X, int ldx, long long g, int kc, int kk, int nv, bool cplx) {
  if (!cplx) {
    const int j = kc * 64 + kk;
    return j < nv ? reinterpret_cast<const double*>(X)[g * ldx + j] : 0.0;
  }
  const int j = kc * 32 + (kk & 31);
  if (j >= nv) return 0.0;
  const cd v = reinterpret_cast<const cd*>(X)[g * ldx + j];
  return kk < 32 ? v.x : v.y;
}

// digits of the real form of G for every (K chunk, output block), one thread per output column:
// planes [(kc, ob)][digit][64 columns][64 k], exponents [(kc, ob)][64]. G[k][j] = herm ?
// (k <= j ? conj(C[j][k]) : 0) : C[k][j]. Output block ob: real data columns ob * 64 ..; complex
// data the real (nh = 0) or imaginary (nh = 1) parts of columns (ob / 2) * 64 ..
template <typename S>
__global__ void k_rot_wide_bdigits(const S* C, int nv, bool herm, int nkc, int nob, unsigned char* planes, int* exps) {
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nkc * nob * WN) return;
  const int n = (int)(t % WN), ob = (int)((t / WN) % nob), kc = (int)(t / ((long long)WN * nob));
  auto G = [&](int k, int j) -> cd {
    if (k >= nv || j >= nv) return mkc(0, 0);
    if (herm) {
      if (k > j) return mkc(0, 0);
      if constexpr (CPLX) return cconj(C[(size_t)j * nv + k]);
      else return mkc(C[(size_t)j * nv + k], 0.0);
    }
    if constexpr (CPLX) return C[(size_t)k * nv + j];
    else return mkc(C[(size_t)k * nv + j], 0.0);
  };
  auto Bv = [&](int kk) -> double {
    if (!CPLX) return G(kc * 64 + kk, ob * WN + n).x;
    const int nh = ob & 1, col = (ob >> 1) * WN + n;
    const cd g = G(kc * 32 + (kk & 31), col);
    if (kk < 32) return nh == 0 ? g.x : g.y;   // Re X rows
    return nh == 0 ? -g.y : g.x;              // Im X rows
  };
  int mex = 0;
  for (int kk = 0; kk < WK; ++kk) mex = max(mex, bexp(Bv(kk)));
  const int E = mex ? mex - 1022 : 0;
  const size_t blk = (size_t)kc * nob + ob;
  exps[blk * WN + n] = E;
  for (int kp = 0; kp < WK / 2; ++kp)
    put_pair(planes + blk * OZ_S * PLB, PLB, n, 2 * kp, Bv(2 * kp), Bv(2 * kp + 1), E);
}

struct WRotArgs {
  void* X;
  int ldx;
  long long n;
  int nv;
  bool cplx;
  int nkc, nob;
  bool herm;                 // G upper triangular: K chunks past an output block's columns are zero
  const unsigned char* bpl;  // B digit planes per (kc, ob)
  const int* bex;            // B exponents per (kc, ob)
  float2* stage;             // per CTA: [ob][128 rows][64 columns] FP32-pair partial sums
  int* err;
};

// K chunk kc contributes to output block ob (an upper triangular G has no entries in the chunks past
// the block's last column)
__device__ __forceinline__ bool rot_active(const WRotArgs& A, int kc, int ob) {
  return !A.herm || kc < (A.cplx ? 2 * (ob >> 1) + 2 : ob + 1);
}

// Per tile of 128 rows the K chunks run outermost: the A digits of a chunk are cut once (a warp per
// 16 rows, a lane per pair of K entries: coalesced loads, a row's exponent by one warp reduction)
// and serve every output block the chunk contributes to; each (chunk, block) round's combined
// levels are added to the block's FP32-pair partial sums staged per CTA (the first chunk stores),
// and the tile's rows of X are rewritten from the stage once every chunk is done.
__global__ void __launch_bounds__(WT, 1) k_rot_wide(const WRotArgs A) {
  extern __shared__ __align__(1024) unsigned char wz_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)wz_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + OZ_S * PLA;
  __shared__ int sE[128], Fexp[WN];
  __shared__ uint64_t b_bar, mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc_cta(&tmem_slot);
  if (tid == 0) {
    mbar_init(&b_bar, 1);
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
  float2* stage = A.stage + (size_t)blockIdx.x * A.nob * 128 * WN;
  double* Xd = reinterpret_cast<double*>(A.X);
  const long long ldr = (long long)A.ldx * (A.cplx ? 2 : 1);
  const long long tiles = (A.n + 127) / 128;
  long long it = 0;   // rounds so far: the phase of both barriers
  bool b_out = false, mma_out = false;
  for (long long tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x) {
    const long long r0 = tile * 128;
    const int nr = (int)min(128ll, A.n - r0);
    for (int kc = 0; kc < A.nkc && !s_fail; ++kc) {
      {   // A digits of the chunk: warp w takes rows 16 w .. 16 w + 15, lane l the K entries 2 l, 2 l + 1
        double v[32];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = warp * 16 + i;
          const bool ok = r < nr;
          v[2 * i] = ok ? rot_op(A.X, A.ldx, r0 + r, kc, 2 * lane, A.nv, A.cplx) : 0.0;
          v[2 * i + 1] = ok ? rot_op(A.X, A.ldx, r0 + r, kc, 2 * lane + 1, A.nv, A.cplx) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = warp * 16 + i;
          const int mex = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(bexp(v[2 * i]), bexp(v[2 * i + 1])));
          const int E = mex ? mex - 1022 : 0;
          if (lane == 0) sE[r] = E;
          put_pair(sA, PLA, r, 2 * lane, v[2 * i], v[2 * i + 1], E);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      for (int ob = 0; ob < A.nob; ++ob, ++it) {
        if (!rot_active(A, kc, ob)) { --it; continue; }
        const size_t blk = (size_t)kc * A.nob + ob;
        if (tid < WN) Fexp[tid] = A.bex[blk * WN + tid];
        if (tid == 0) {   // the round's B digits, then its 112 MMAs
          mbar_expect_tx(&b_bar, (uint32_t)(OZ_S * PLB));
          bulk_copy(smem_u32(sB), A.bpl + blk * OZ_S * PLB, (uint32_t)(OZ_S * PLB), &b_bar);
          b_out = true;
          if (mbar_wait(&b_bar, (uint32_t)(it & 1), &s_fail)) {
            b_out = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_round(taddr, smem_u32(sA), smem_u32(sB));
            mma_commit(&mma_bar);
          } else {
            s_fail = 1;
          }
        }
        __syncthreads();
        if (s_fail) break;
        mma_out = true;
        const bool ok = mbar_wait(&mma_bar, (uint32_t)(it & 1), &s_fail);
        if (__syncthreads_or(!ok)) { s_fail = 1; break; }
        mma_out = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        f2 R[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) R[j] = f2{0.0f, 0.0f};
        add_levels(taddr, lane_base, ch, sE[row], Fexp, R);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        // the block's partial sums of (row, 32 columns ch 32 ..): 256 contiguous bytes per thread
        float4* st = reinterpret_cast<float4*>(stage + ((size_t)ob * 128 + row) * WN + ch * 32);
        if (kc == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) st[j] = make_float4(R[2 * j].h, R[2 * j].l, R[2 * j + 1].h, R[2 * j + 1].l);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float4 o = st[j];
            const f2 a = f2_add(f2{o.x, o.y}, R[2 * j]), b = f2_add(f2{o.z, o.w}, R[2 * j + 1]);
            st[j] = make_float4(a.h, a.l, b.h, b.l);
          }
        }
        __syncthreads();
      }
    }
    if (s_fail) break;
    // every chunk of the tile is done: its rows of X from the stage (a thread per real of a row)
    for (int ob = 0; ob < A.nob; ++ob)
      for (int t = tid; t < nr * WN; t += WT) {
        const int r = t / WN, col = t % WN;
        const float2 v = stage[((size_t)ob * 128 + r) * WN + col];
        const double x = f2_to(f2{v.x, v.y});
        if (!A.cplx) {
          const int c = ob * WN + col;
          if (c < A.nv) Xd[(r0 + r) * ldr + c] = x;
        } else {
          const int c = (ob >> 1) * WN + col;
          if (c < A.nv) Xd[(r0 + r) * ldr + 2 * c + (ob & 1)] = x;
        }
      }
    __syncthreads();
  }
  if (tid == 0 && s_fail) {
    if (mma_out) mbar_wait_drain(&mma_bar, (uint32_t)(it & 1));
    if (b_out) mbar_wait_drain(&b_bar, (uint32_t)(it & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) atomicExch(A.err, 1);
  if (warp == 0) tmem_free_cta(taddr);
}

int grow_ozpart(oefe_ctx* c, size_t need) {
  if (c->ozpart_bytes >= need) return OEFE_OK;
  cudaStreamSynchronize(c->stream);
  dev_free(c->d_ozpart);
  c->d_ozpart = nullptr;
  c->ozpart_bytes = 0;
  OEFE_TRY(dev_alloc(c, &c->d_ozpart, need));
  c->ozpart_bytes = need;
  return OEFE_OK;
}

int finish_wide(oefe_ctx* c, const char* what) {
  OEFE_CUDA_TRY(c, cudaGetLastError());
  int flag = 0;
  OEFE_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  OEFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (flag) {
    cudaMemsetAsync(c->d_status + 2, 0, sizeof(int), c->stream);
    c->err = std::string(what) + ": a tensor-core wait timed out";
    return OEFE_ERR_TIMEOUT;
  }
  return OEFE_OK;
}

}  // namespace

// out = X^+ W (nv x nv) on the tensor cores, any nv; herm: the result is known to be Hermitian
// (real data: only the tiles meeting the upper triangle run, the rest is mirrored)
template <typename S>
int gram_ozaki_wide(oefe_ctx* c, const S* X, int ldx, const S* W, int ldw, int64_t n, int nv, S* out, bool herm) {
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  const int NA = CPLX ? 2 * nv : nv;
  const int nI = (NA + 127) / 128, nJ = (NA + WN - 1) / WN;
  const bool upper = herm && !CPLX;
  int ntile = nI * nJ;
  if (upper) {
    ntile = 0;
    for (int I = 0; I < nI; ++I) ntile += std::max(0, nJ - 2 * I);
  }
  const long long passes = std::max<long long>(1, (n + 63) / 64);
  const int nbx = (int)std::max<long long>(1, std::min<long long>(passes, c->num_sms / std::max(1, ntile)));
  const long long ppc = (passes + nbx - 1) / nbx;
  const size_t need = (size_t)nbx * nI * nJ * 128 * WN * sizeof(double);
  OEFE_TRY(grow_ozpart(c, need));
  WGramArgs A;
  A.X = X;
  A.ldx = ldx;
  A.W = W;
  A.ldw = ldw;
  A.n = n;
  A.nv = nv;
  A.cplx = CPLX;
  A.nI = nI;
  A.nJ = nJ;
  A.upper = upper;
  A.passes = passes;
  A.ppc = ppc;
  A.part = (double*)c->d_ozpart;
  A.err = c->d_status + 2;
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_gram_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WSMEM));
  dim3 grid(nbx, ntile);
  OEFE_COUNTED k_gram_wide<<<grid, WT, WSMEM, c->stream>>>(A);
  OEFE_COUNTED k_gram_wide_reduce<S><<<(nv * nv + 255) / 256, 256, 0, c->stream>>>(A.part, nbx, nI, nJ, nv, upper, out);
  return finish_wide(c, "gram");
}

// X[0:n] <- X G (G = C, or C^+ of a lower triangular C when herm) on the tensor cores, any nv
template <typename S>
int rotate_ozaki_wide(oefe_ctx* c, S* X, int ldx, int64_t n, int nv, const S* C, bool herm) {
  constexpr bool CPLX = sizeof(S) == sizeof(cd);
  const int nkc = CPLX ? (nv + 31) / 32 : (nv + 63) / 64;
  const int nob = CPLX ? 2 * ((nv + WN - 1) / WN) : (nv + WN - 1) / WN;
  const long long tiles = (n + 127) / 128;
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, c->num_sms));
  auto a256 = [](size_t x) { return ((x + 255) / 256) * 256; };
  const size_t pl_bytes = a256((size_t)nkc * nob * OZ_S * PLB), ex_bytes = a256((size_t)nkc * nob * WN * sizeof(int));
  const size_t st_bytes = a256((size_t)grid * nob * 128 * WN * sizeof(float2));
  OEFE_TRY(grow_ozpart(c, pl_bytes + ex_bytes + st_bytes));
  unsigned char* base = (unsigned char*)c->d_ozpart;
  WRotArgs A;
  A.X = X;
  A.ldx = ldx;
  A.n = n;
  A.nv = nv;
  A.cplx = CPLX;
  A.nkc = nkc;
  A.nob = nob;
  A.herm = herm;
  A.bpl = base;
  A.bex = (const int*)(base + pl_bytes);
  A.stage = (float2*)(base + pl_bytes + ex_bytes);
  A.err = c->d_status + 2;
  const long long nb = (long long)nkc * nob * WN;
  OEFE_COUNTED k_rot_wide_bdigits<S><<<(unsigned)((nb + 127) / 128), 128, 0, c->stream>>>(C, nv, herm, nkc, nob, base,
                                                                                           (int*)(base + pl_bytes));
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_rot_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WSMEM));
  OEFE_COUNTED k_rot_wide<<<grid, WT, WSMEM, c->stream>>>(A);
  return finish_wide(c, "rotate");
}

template int gram_ozaki_wide<double>(oefe_ctx*, const double*, int, const double*, int, int64_t, int, double*, bool);
template int gram_ozaki_wide<cd>(oefe_ctx*, const cd*, int, const cd*, int, int64_t, int, cd*, bool);
template int rotate_ozaki_wide<double>(oefe_ctx*, double*, int, int64_t, int, const double*, bool);
template int rotate_ozaki_wide<cd>(oefe_ctx*, cd*, int, int64_t, int, const cd*, bool);
