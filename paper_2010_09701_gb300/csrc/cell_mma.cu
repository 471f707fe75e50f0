// Cell products Z_e = H^O_e X_e on the 5th-generation tensor cores (tcgen05).
//
// Precision: BF16x3. The cell matrices are stored split, H = H_hi + H_lo with
// H_hi = bf16(H), H_lo = bf16(H - H_hi); the gathered vectors are split the
// same way on the fly, and Z = H_hi X_hi + H_hi X_lo + H_lo X_hi is
// accumulated in FP32 in tensor memory (the dropped H_lo X_lo term and the
// split residuals are ~2^-17 relative).
//
// Complex arithmetic with real MMAs: Z_r = H_r X_r - H_i X_i and
// Z_i = H_r X_i + H_i X_r, the minus sign through the instruction
// descriptor's A-negate bit, into two N = 64 accumulators per M tile.
//
// One CTA per (cell, block of 64 vectors). M tiles of 128 rows, K tiles of 64
// (128-byte rows, 128B swizzle), two pipeline stages: the loads of iteration
// i overlap the MMAs of iteration i-1; every stage's reuse waits on the
// mbarrier its MMAs commit to. Every wait is bounded; on a timeout the CTA
// raises the error flag, drains and frees its tensor memory, and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "oefe_internal.h"

namespace {

constexpr int MT = 128;          // rows per M tile
constexpr int KT = 64;           // K per tile (bf16: 128 bytes per row)
constexpr int THREADS = 256;
constexpr long long WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on a phase of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::f16, BF16 x BF16 -> F32, K-major A and B
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool negA) {
  return (1u << 4)                 // D format F32
         | (1u << 7)               // A format BF16
         | (1u << 10)              // B format BF16
         | ((negA ? 1u : 0u) << 13)
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
  static_assert(N == 16 || N == 32, "16 or 32 columns");
  if constexpr (N == 32) tmem_ld32(taddr, v);
  else tmem_ld16(taddr, v);
}

// byte offset of element (row, k) of a K-major 128B-swizzled bf16 tile (128-byte rows)
__device__ __forceinline__ uint32_t swz(int row, int k) {
  const int byte = k * 2;
  return (uint32_t)(row * 128 + ((((byte >> 4) ^ (row & 7)) & 7) << 4) + (byte & 15));
}

// One (cell, vector block) tile: Z_e[:, v0:v0+NB] = H_e X_e[:, v0:v0+NB].
// g is the CTA's running pipeline iteration count (mbarrier phases continue
// across tiles); every tile ends with all its MMAs complete and its
// accumulators read, so the next tile starts on free stages.
template <bool CPLX, int NB>
__device__ __forceinline__ void mma_tile(const __nv_bfloat16* __restrict__ He, const float* __restrict__ X, int ldx,
                                         int nv, int v0, int e, const int* __restrict__ cell_nodes,
                                         const int* __restrict__ act_off, const int* __restrict__ act_idx, int nloc,
                                         int npad, int64_t nh, float* __restrict__ Z, unsigned char* sA,
                                         unsigned char* sB, uint64_t* bars, uint32_t taddr, int& g, int* s_fail) {
  constexpr int PLANES = CPLX ? 4 : 2;             // (Hr_hi, Hr_lo, Hi_hi, Hi_lo) or (H_hi, H_lo)
  constexpr int NB_ROWS = CPLX ? 2 * NB : NB;      // B^T rows: [X_r | X_i] or X
  constexpr int A_PLANE = MT * 128;                // bytes per A plane tile
  constexpr int A_STAGE = PLANES * A_PLANE;
  constexpr int B_PART = NB_ROWS * 128;            // bytes per B split part
  constexpr int B_STAGE = 2 * B_PART;              // hi, lo
  constexpr int MCOLS = CPLX ? 2 * NB : NB;        // accumulator columns per M tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ne = act_off[e + 1] - act_off[e];
  const int naug = nloc + ne;
  const int mt = npad / MT, ktn = npad / KT;
  const int nit = mt * ktn;
  const int g0 = g;
  int issued = 0;
  for (int it = 0; it < nit; ++it) {
    const int gi = g0 + it;
    const int kt = it / mt, m = it % mt, s = gi & 1;
    if (it >= 2) {
      if (!mbar_wait(&bars[s], ((gi - 2) >> 1) & 1)) *s_fail = 1;
    }
    __syncthreads();
    if (*s_fail) break;
    {  // A tiles of (kt, m): PLANES x 128 rows x 8 chunks of 16 bytes into the swizzled stage
      const uint32_t a0 = smem_u32(sA + s * A_STAGE);
      for (int c = tid; c < PLANES * MT * 8; c += THREADS) {
        const int p = c / (MT * 8), r = (c / 8) % MT, ch = c % 8;
        // tile-contiguous storage: [K tile][M tile][plane][128 rows][64 columns]
        const __nv_bfloat16* src = He + ((((size_t)kt * mt + m) * PLANES + p) * MT + r) * KT + ch * 8;
        cp_async16(a0 + p * A_PLANE + r * 128 + (((ch ^ (r & 7)) & 7) << 4), src);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if (m == 0) {  // B tile of kt: gather the cell's rows, split to bf16 hi / lo
      unsigned char* b0 = sB + (kt & 1) * B_STAGE;
      for (int idx = tid; idx < KT * NB; idx += THREADS) {
        const int kk = idx / NB, v = idx % NB;
        const int r = kt * KT + kk;
        float xr = 0.f, xi = 0.f;
        if (r < naug && v0 + v < nv) {
          const int64_t row = r < nloc ? (int64_t)cell_nodes[(size_t)e * nloc + r] : nh + act_idx[act_off[e] + r - nloc];
          if (CPLX) {
            const float2 x = reinterpret_cast<const float2*>(X)[row * ldx + v0 + v];
            xr = x.x;
            xi = x.y;
          } else {
            xr = X[row * ldx + v0 + v];
          }
        }
        const __nv_bfloat16 rh = __float2bfloat16_rn(xr);
        const __nv_bfloat16 rl = __float2bfloat16_rn(xr - __bfloat162float(rh));
        *reinterpret_cast<__nv_bfloat16*>(b0 + swz(v, kk)) = rh;
        *reinterpret_cast<__nv_bfloat16*>(b0 + B_PART + swz(v, kk)) = rl;
        if (CPLX) {
          const __nv_bfloat16 ih = __float2bfloat16_rn(xi);
          const __nv_bfloat16 il = __float2bfloat16_rn(xi - __bfloat162float(ih));
          *reinterpret_cast<__nv_bfloat16*>(b0 + swz(NB + v, kk)) = ih;
          *reinterpret_cast<__nv_bfloat16*>(b0 + B_PART + swz(NB + v, kk)) = il;
        }
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_base = smem_u32(sA + s * A_STAGE);
      const uint32_t b_base = smem_u32(sB + (kt & 1) * B_STAGE);
      const uint32_t dcol = taddr + m * MCOLS;
      constexpr uint32_t ID = idesc_bf16(MT, NB, false);
      constexpr uint32_t IDN = idesc_bf16(MT, NB, true);
#pragma unroll
      for (int ks = 0; ks < KT / 16; ++ks) {
        const uint32_t koff = ks * 32;
        const uint32_t first = (kt == 0 && ks == 0) ? 0u : 1u;
        if (CPLX) {
          const uint64_t Arh = sdesc(a_base + 0 * A_PLANE + koff), Arl = sdesc(a_base + 1 * A_PLANE + koff);
          const uint64_t Aih = sdesc(a_base + 2 * A_PLANE + koff), Ail = sdesc(a_base + 3 * A_PLANE + koff);
          const uint64_t Xrh = sdesc(b_base + koff), Xih = sdesc(b_base + NB * 128 + koff);
          const uint64_t Xrl = sdesc(b_base + B_PART + koff), Xil = sdesc(b_base + B_PART + NB * 128 + koff);
          const uint32_t Dr = dcol, Di = dcol + NB;
          // Z_r += H_r X_r - H_i X_i
          mma_bf16(Dr, Arh, Xrh, ID, first);
          mma_bf16(Dr, Arh, Xrl, ID, 1);
          mma_bf16(Dr, Arl, Xrh, ID, 1);
          mma_bf16(Dr, Aih, Xih, IDN, 1);
          mma_bf16(Dr, Aih, Xil, IDN, 1);
          mma_bf16(Dr, Ail, Xih, IDN, 1);
          // Z_i += H_r X_i + H_i X_r
          mma_bf16(Di, Arh, Xih, ID, first);
          mma_bf16(Di, Arh, Xil, ID, 1);
          mma_bf16(Di, Arl, Xih, ID, 1);
          mma_bf16(Di, Aih, Xrh, ID, 1);
          mma_bf16(Di, Aih, Xrl, ID, 1);
          mma_bf16(Di, Ail, Xrh, ID, 1);
        } else {
          const uint64_t Ah = sdesc(a_base + koff), Al = sdesc(a_base + A_PLANE + koff);
          const uint64_t Bh = sdesc(b_base + koff), Bl = sdesc(b_base + B_PART + koff);
          mma_bf16(dcol, Ah, Bh, ID, first);
          mma_bf16(dcol, Ah, Bl, ID, 1);
          mma_bf16(dcol, Al, Bh, ID, 1);
        }
      }
      mma_commit(&bars[s]);
    }
    issued = it + 1;
  }
  if (issued > 0) {  // drain: the last committed group implies all earlier ones
    const int last = g0 + issued - 1;
    if (!mbar_wait(&bars[last & 1], (last >> 1) & 1)) *s_fail = 1;
  }
  g = g0 + issued;
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!*s_fail && issued == nit) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31; the two warpgroups split the vector columns
    constexpr int HC = NB / 2;
    const int q = warp & 3, h = warp >> 2;
    for (int m = 0; m < mt; ++m) {
      const int row = m * MT + 32 * q + lane;
      const uint32_t tl = taddr + ((uint32_t)(32 * q) << 16) + m * MCOLS + HC * h;
      float re[HC], im[HC];
      tmem_ld<HC>(tl, re);
      if (CPLX) tmem_ld<HC>(tl + NB, im);
      if (row < naug) {
        float* zr = Z + ((size_t)e * npad + row) * (size_t)nv * (CPLX ? 2 : 1);
#pragma unroll
        for (int j = 0; j < HC; ++j) {
          const int v = v0 + HC * h + j;
          if (v < nv) {
            if (CPLX) {
              zr[2 * v] = re[j];
              zr[2 * v + 1] = im[j];
            } else {
              zr[v] = re[j];
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
}

template <bool CPLX, int NB>
struct MmaCfg {
  static constexpr int PLANES = CPLX ? 4 : 2;
  static constexpr int NB_ROWS = CPLX ? 2 * NB : NB;
  static constexpr int SMEM = 1024 + 2 * PLANES * MT * 128 + 2 * 2 * NB_ROWS * 128;
  static constexpr int TCOLS_NEED = 4 * (CPLX ? 2 * NB : NB);   // up to 4 M tiles
  static constexpr int TCOLS = TCOLS_NEED <= 128 ? 128 : TCOLS_NEED <= 256 ? 256 : 512;
};

__device__ __forceinline__ uint32_t cta_setup(uint64_t* bars, uint32_t* tmem_slot, int* s_fail, int tcols) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *tmem_slot;
}

__device__ __forceinline__ void cta_teardown(uint32_t taddr, int tcols, const int* s_fail, int* err) {
  if (*s_fail && threadIdx.x == 0) atomicExch(err, 1);
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(tcols) : "memory");
}

// one CTA per (cell, vector block)
template <bool CPLX, int NB>
__global__ void __launch_bounds__(THREADS, 1)
    k_cell_mma(const __nv_bfloat16* __restrict__ Hb, const float* __restrict__ X, int ldx, int nv,
               const int* __restrict__ cell_nodes, const int* __restrict__ act_off, const int* __restrict__ act_idx,
               int nloc, int npad, int64_t nh, float* __restrict__ Z, int* __restrict__ err) {
  using Cfg = MmaCfg<CPLX, NB>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const uint32_t taddr = cta_setup(bars, &tmem_slot, &s_fail, Cfg::TCOLS);
  const int e = blockIdx.x;
  int g = 0;
  mma_tile<CPLX, NB>(Hb + (size_t)e * Cfg::PLANES * npad * npad, X, ldx, nv, blockIdx.y * NB, e, cell_nodes, act_off,
                     act_idx, nloc, npad, nh, Z, smem, smem + 2 * Cfg::PLANES * MT * 128, bars, taddr, g, &s_fail);
  cta_teardown(taddr, Cfg::TCOLS, &s_fail, err);
}

// persistent: all (k, cell, vector block) tiles of a batch of k-points
template <bool CPLX, int NB>
__global__ void __launch_bounds__(THREADS, 1)
    k_cell_mma_multi(const MmaK* __restrict__ ks, int nk, long long ntiles, const int* __restrict__ cell_nodes,
                     const int* __restrict__ act_off, const int* __restrict__ act_idx, int nloc, int npad, int ncells,
                     int64_t nh, int* __restrict__ err) {
  using Cfg = MmaCfg<CPLX, NB>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const uint32_t taddr = cta_setup(bars, &tmem_slot, &s_fail, Cfg::TCOLS);
  int g = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int k = 0;
    while (k + 1 < nk && ks[k + 1].tile0 <= t) ++k;
    const MmaK P = ks[k];
    const __nv_bfloat16* Hk = (const __nv_bfloat16*)P.H;
    const long long r = t - P.tile0;
    const int e = (int)(r / P.vblocks), vb = (int)(r % P.vblocks);
    mma_tile<CPLX, NB>(Hk + (size_t)e * Cfg::PLANES * npad * npad, P.X, P.ldx, P.nv, vb * NB, e, cell_nodes, act_off,
                       act_idx, nloc, npad, nh, P.Z, smem, smem + 2 * Cfg::PLANES * MT * 128, bars, taddr, g, &s_fail);
    if (s_fail) break;
  }
  cta_teardown(taddr, Cfg::TCOLS, &s_fail, err);
}

}  // namespace

size_t cell_mma_smem(bool cplx, int nb) {
  if (cplx) return nb == 64 ? MmaCfg<true, 64>::SMEM : MmaCfg<true, 32>::SMEM;
  return nb == 64 ? MmaCfg<false, 64>::SMEM : MmaCfg<false, 32>::SMEM;
}

static int check_npad(oefe_ctx* c) {
  if (c->npad % MT != 0 || c->npad > 4 * MT) {
    c->err = "tensor path needs npad a multiple of 128 and at most 512";
    return OEFE_ERR_ARG;
  }
  return OEFE_OK;
}

template <bool CPLX, int NB>
static int launch_one(oefe_ctx* c, const void* H, const void* X, int ldx, int nv, void* Z, cudaStream_t st) {
  const size_t smem = MmaCfg<CPLX, NB>::SMEM;
  dim3 grid(c->ncells, (nv + NB - 1) / NB);
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_mma<CPLX, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  OEFE_COUNTED k_cell_mma<CPLX, NB><<<grid, THREADS, smem, st>>>((const __nv_bfloat16*)H, (const float*)X, ldx, nv, c->d_cell_nodes,
                                                    c->d_act_off, c->d_act_idx, c->nloc, c->npad, c->nh, (float*)Z,
                                                    c->d_status);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

int launch_cell_mma_ptrs(oefe_ctx* c, const void* H, const void* X, int ldx, int nv, void* Z, bool cplx, int nb,
                         cudaStream_t st) {
  OEFE_TRY(check_npad(c));
  if (cplx) return nb == 64 ? launch_one<true, 64>(c, H, X, ldx, nv, Z, st) : launch_one<true, 32>(c, H, X, ldx, nv, Z, st);
  return nb == 64 ? launch_one<false, 64>(c, H, X, ldx, nv, Z, st) : launch_one<false, 32>(c, H, X, ldx, nv, Z, st);
}

int launch_cell_mma(oefe_ctx* c, const KData& K, const void* X, int ldx, int nv, bool cplx, void* Z) {
  OEFE_TRY(check_npad(c));
  if (!K.Hbf) { c->err = "BF16x3 cell matrices were not stored"; return OEFE_ERR_STATE; }
  const int ik = (int)(&K - c->kd.data());
  // the three-part split runs on the TMA kernel only
  if ((c->use_tma || K.bf_parts == 3) && c->d_tmaps && ik >= 0 && ik < c->n_tmaps) {
    MmaK k0;
    k0.H = K.Hbf;
    k0.X = (const float*)X;
    k0.Z = (float*)Z;
    k0.ldx = ldx;
    k0.nv = nv;
    k0.vblocks = (nv + 63) / 64;
    k0.tile0 = 0;
    const long long nt = (long long)c->ncells * k0.vblocks;
    return launch_cell_mma_tma(c, (const char*)c->d_tmaps + (size_t)ik * tensor_map_bytes(), nullptr, &k0, 1, nt, cplx,
                               K.bf_parts, (int)std::min<long long>(nt, c->num_sms), c->stream);
  }
  if (K.bf_parts != 2) { c->err = "tensor path: the split cell matrices have no tensor maps"; return OEFE_ERR_STATE; }
  if (cplx) return launch_one<true, 64>(c, K.Hbf, X, ldx, nv, Z, c->stream);
  return launch_one<false, 64>(c, K.Hbf, X, ldx, nv, Z, c->stream);
}

template <bool CPLX, int NB>
static int launch_multi_t(oefe_ctx* c, const MmaK* d_ks, int nk, long long ntiles, int grid, cudaStream_t st) {
  const size_t smem = MmaCfg<CPLX, NB>::SMEM;
  OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_mma_multi<CPLX, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
  OEFE_COUNTED k_cell_mma_multi<CPLX, NB><<<grid, THREADS, smem, st>>>(d_ks, nk, ntiles, c->d_cell_nodes, c->d_act_off,
                                                          c->d_act_idx, c->nloc, c->npad, c->ncells, c->nh,
                                                          c->d_status);
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}

int launch_cell_mma_multi(oefe_ctx* c, const MmaK* d_ks, int nk, long long ntiles, bool cplx, int nb, int grid,
                          cudaStream_t st) {
  OEFE_TRY(check_npad(c));
  if (cplx) return nb == 64 ? launch_multi_t<true, 64>(c, d_ks, nk, ntiles, grid, st)
                            : launch_multi_t<true, 32>(c, d_ks, nk, ntiles, grid, st);
  return nb == 64 ? launch_multi_t<false, 64>(c, d_ks, nk, ntiles, grid, st)
                  : launch_multi_t<false, 32>(c, d_ks, nk, ntiles, grid, st);
}
