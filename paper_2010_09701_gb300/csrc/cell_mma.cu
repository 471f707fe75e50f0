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
constexpr int NBV = 64;          // vectors per CTA
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

// byte offset of element (row, k) of a K-major 128B-swizzled bf16 tile (128-byte rows)
__device__ __forceinline__ uint32_t swz(int row, int k) {
  const int byte = k * 2;
  return (uint32_t)(row * 128 + ((((byte >> 4) ^ (row & 7)) & 7) << 4) + (byte & 15));
}

template <bool CPLX>
__global__ void __launch_bounds__(THREADS, 1)
    k_cell_mma(const __nv_bfloat16* __restrict__ Hb, const float* __restrict__ X, int ldx, int nv,
               const int* __restrict__ cell_nodes, const int* __restrict__ act_off, const int* __restrict__ act_idx,
               int nloc, int npad, int64_t nh, float* __restrict__ Z, int* __restrict__ err) {
  constexpr int PLANES = CPLX ? 4 : 2;             // (Hr_hi, Hr_lo, Hi_hi, Hi_lo) or (H_hi, H_lo)
  constexpr int NB_ROWS = CPLX ? 2 * NBV : NBV;    // B^T rows: [X_r | X_i] or X
  constexpr int A_PLANE = MT * 128;                // bytes per A plane tile
  constexpr int A_STAGE = PLANES * A_PLANE;
  constexpr int B_PART = NB_ROWS * 128;            // bytes per B split part
  constexpr int B_STAGE = 2 * B_PART;              // hi, lo
  constexpr int TCOLS = CPLX ? 512 : 256;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + 2 * A_STAGE;
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = blockIdx.x;
  const int v0 = blockIdx.y * NBV;
  const int ne = act_off[e + 1] - act_off[e];
  const int naug = nloc + ne;
  const int mt = npad / MT, ktn = npad / KT;
  const int nit = mt * ktn;
  const int mcols = CPLX ? 2 * NBV : NBV;          // accumulator columns per M tile

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_slot;
  const __nv_bfloat16* He = Hb + (size_t)e * PLANES * npad * npad;
  const int64_t* dummy = nullptr;
  (void)dummy;

  int issued = 0;  // MMA groups committed (iterations)
  for (int it = 0; it < nit; ++it) {
    const int kt = it / mt, m = it % mt, s = it & 1;
    if (it >= 2) {
      if (!mbar_wait(&bars[s], ((it - 2) >> 1) & 1)) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    // A tiles of (kt, m): PLANES x 128 rows x 8 chunks of 16 bytes, async copies into the swizzled stage
    {
      const uint32_t a0 = smem_u32(sA + s * A_STAGE);
      for (int c = tid; c < PLANES * MT * 8; c += THREADS) {
        const int p = c / (MT * 8), r = (c / 8) % MT, ch = c % 8;
        const __nv_bfloat16* src = He + ((size_t)p * npad + m * MT + r) * npad + kt * KT + ch * 8;
        cp_async16(a0 + p * A_PLANE + r * 128 + (((ch ^ (r & 7)) & 7) << 4), src);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // B tile of kt (first M tile only): gather the cell's rows, split to bf16 hi/lo
    if (m == 0) {
      unsigned char* b0 = sB + (kt & 1) * B_STAGE;
      for (int idx = tid; idx < KT * NBV; idx += THREADS) {
        const int kk = idx / NBV, v = idx % NBV;
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
          *reinterpret_cast<__nv_bfloat16*>(b0 + swz(NBV + v, kk)) = ih;
          *reinterpret_cast<__nv_bfloat16*>(b0 + B_PART + swz(NBV + v, kk)) = il;
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
      const uint32_t dcol = taddr + m * mcols;
      constexpr uint32_t ID = idesc_bf16(MT, NBV, false);
      constexpr uint32_t IDN = idesc_bf16(MT, NBV, true);
#pragma unroll
      for (int ks = 0; ks < KT / 16; ++ks) {
        const uint32_t koff = ks * 32;
        const uint32_t first = (kt == 0 && ks == 0) ? 0u : 1u;
        if (CPLX) {
          const uint64_t Arh = sdesc(a_base + 0 * A_PLANE + koff), Arl = sdesc(a_base + 1 * A_PLANE + koff);
          const uint64_t Aih = sdesc(a_base + 2 * A_PLANE + koff), Ail = sdesc(a_base + 3 * A_PLANE + koff);
          const uint64_t Xrh = sdesc(b_base + koff), Xih = sdesc(b_base + NBV * 128 + koff);
          const uint64_t Xrl = sdesc(b_base + B_PART + koff), Xil = sdesc(b_base + B_PART + NBV * 128 + koff);
          const uint32_t Dr = dcol, Di = dcol + NBV;
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
  // drain: wait for the last committed group (it implies all earlier ones)
  if (issued > 0) {
    const int last = issued - 1;
    if (!mbar_wait(&bars[last & 1], (last >> 1) & 1)) s_fail = 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_fail && issued == nit) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31; the two warpgroups split the vector columns
    const int q = warp & 3, h = warp >> 2;
    for (int m = 0; m < mt; ++m) {
      const int row = m * MT + 32 * q + lane;
      const uint32_t tl = taddr + ((uint32_t)(32 * q) << 16) + m * mcols + 32 * h;
      float re[32], im[32];
      tmem_ld32(tl, re);
      if (CPLX) tmem_ld32(tl + NBV, im);
      if (row < naug) {
        float* zr = Z + ((size_t)e * npad + row) * (size_t)nv * (CPLX ? 2 : 1);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int v = v0 + 32 * h + j;
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
  if (s_fail && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS) : "memory");
  }
}

}  // namespace

size_t cell_mma_smem(bool cplx) {
  const int planes = cplx ? 4 : 2;
  const int nbrows = cplx ? 2 * NBV : NBV;
  return 1024 + 2 * (size_t)planes * MT * 128 + 2 * 2 * (size_t)nbrows * 128;
}

int launch_cell_mma(oefe_ctx* c, const KData& K, const void* X, int ldx, int nv, bool cplx, void* Z) {
  if (c->npad % MT != 0 || c->npad > 4 * MT) {
    c->err = "tensor path needs npad a multiple of 128 and at most 512";
    return OEFE_ERR_ARG;
  }
  if (!K.Hbf) { c->err = "BF16x3 cell matrices were not stored"; return OEFE_ERR_STATE; }
  const size_t smem = cell_mma_smem(cplx);
  dim3 grid(c->ncells, (nv + NBV - 1) / NBV);
  if (cplx) {
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_mma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_cell_mma<true><<<grid, THREADS, smem, c->stream>>>((const __nv_bfloat16*)K.Hbf, (const float*)X, ldx, nv,
                                                         c->d_cell_nodes, c->d_act_off, c->d_act_idx, c->nloc,
                                                         c->npad, c->nh, (float*)Z, c->d_status);
  } else {
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(k_cell_mma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_cell_mma<false><<<grid, THREADS, smem, c->stream>>>((const __nv_bfloat16*)K.Hbf, (const float*)X, ldx, nv,
                                                          c->d_cell_nodes, c->d_act_off, c->d_act_idx, c->nloc,
                                                          c->npad, c->nh, (float*)Z, c->d_status);
  }
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}
