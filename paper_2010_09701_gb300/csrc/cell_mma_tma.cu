// Warp-specialized tensor-core cell products (tcgen05 + TMA), BF16x3.
//
// Same arithmetic as k_cell_mma (cell_mma.cu): Z_e = H_e X_e with the cell
// matrices stored as bf16 hi / lo planes, the vectors split on the fly,
// Z = H_hi X_hi + H_hi X_lo + H_lo X_hi accumulated in FP32 in tensor memory,
// complex products as real MMAs with the A-negate bit.
//
// Roles (one persistent CTA per SM, looping over (k, cell, vector block) tiles):
//   warp 0      TMA producer: the cell-matrix tile of every (K tile, M tile) as
//               2-plane boxes (hi, lo of the real part, then of the imaginary
//               part) into a ring of 32 KB shared-memory stages;
//   warp 1      MMA issuer (one thread): waits for a full A stage (and B stage),
//               issues the MMAs, commits to the stage's "empty" barriers;
//   warps 2-5   gather producers: rows of X for every K tile, split to bf16;
//   warps 6-9   epilogue: tensor memory -> registers -> per-cell products, one
//               M tile at a time, so the next tile's MMAs into an M tile start
//               as soon as that M tile has been drained.
// Every mbarrier wait is bounded; on a timeout the CTA raises the error flag,
// lets the other roles drain, waits for its copies in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "oefe_internal.h"
#include "tcgen05_dev.cuh"

namespace {

constexpr int MT = 128;     // rows per M tile
constexpr int KT = 64;      // K per tile (bf16: 128 bytes per row)
constexpr int NBV = 64;     // vectors per tile (complex; real data also 128, the NVT parameter)
constexpr int THREADS = 320;
constexpr int MAXPAD = 4 * MT;  // largest npad

// Shared-memory plan per (complex, bf16 parts): NPART planes per A stage (one part of the cell
// matrix: real or imaginary) and per B stage (the split vectors); the three-part split trades an A
// stage and half of the epilogue staging for the larger stages.
template <bool CPLX, int NPART, int NVT = NBV>
struct TmaCfg {
  static constexpr int SA = NPART == 2 ? 3 : 2;        // A ring stages
  static constexpr int SB = 2;                         // B ring stages
  static constexpr int ER = NPART == 2 ? 32 : 16;      // epilogue rows staged per round, per warp
  static constexpr int NB_ROWS = CPLX ? 2 * NBV : NVT;
  static constexpr int A_PLANE = MT * 128;
  static constexpr int A_STAGE = NPART * A_PLANE;
  static constexpr int B_PART = NB_ROWS * 128;
  static constexpr int B_STAGE = NPART * B_PART;
  static constexpr int STG = ER * 256;
  static constexpr size_t SMEM = 1024 + (size_t)SA * A_STAGE + (size_t)SB * B_STAGE + 4 * (size_t)STG;
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// barrier among the 128 gather threads (named barrier 1) that also ORs a flag over them, so that
// all of them take the same exit decision
__device__ __forceinline__ bool gather_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

struct TmaArgs {
  const CUtensorMap* maps;  // one per k-point, in global memory
  const MmaK* ks;           // per-k parameters in global memory, or null: use k0
  MmaK k0;
  int nk;
  long long ntiles;
  const int* cell_nodes;
  const int* act_off;
  const int* act_idx;
  int nloc, npad;
  int64_t nh;
  int* err;
};

// M tiles (128 rows) and K tiles (64 columns) a cell's matrix occupies: the rest of the npad x npad
// block is zero padding, which no role loads, multiplies or drains
__device__ __forceinline__ void cell_tiles(const TmaArgs& A, int e, int mt, int ktn, int* mte, int* kte) {
  const int naug = A.nloc + A.act_off[e + 1] - A.act_off[e];
  *mte = min(mt, (naug + MT - 1) / MT);
  *kte = min(ktn, (naug + KT - 1) / KT);
}

// tile t of the CTA's sequence -> (k, cell, vector block)
__device__ __forceinline__ MmaK kparams(const TmaArgs& A, int k) { return A.ks ? A.ks[k] : A.k0; }

__device__ __forceinline__ void decode_tile(const TmaArgs& A, long long t, int* k, int* e, int* vb) {
  int kk = 0;
  if (A.ks)
    while (kk + 1 < A.nk && A.ks[kk + 1].tile0 <= t) ++kk;
  const MmaK P = kparams(A, kk);
  const long long r = t - P.tile0;
  *k = kk;
  *e = (int)(r / P.vblocks);
  *vb = (int)(r % P.vblocks);
}

// MERGE (complex only): the real part of the cell matrix multiplies [Re X | Im X] in one N = 128
// MMA instead of two N = 64 ones (fewer tensor instructions; which is faster depends on the split,
// so the autotuner chooses)
// NVT (real data only): vectors per tile, 64 or 128; with 128 a cell's matrix streams once for
// twice the vectors (one N = 128 MMA per product, 128 tensor-memory columns per M tile)
template <bool CPLX, int NPART, bool MERGE, int NVT = NBV>
__global__ void __launch_bounds__(THREADS, 1) k_cell_mma_tma(const TmaArgs A) {
  static_assert(NVT == NBV || (!CPLX && NVT == 2 * NBV), "128-vector tiles are for real data");
  using Cfg = TmaCfg<CPLX, NPART, NVT>;
  constexpr int SA = Cfg::SA, SB = Cfg::SB, STG = Cfg::STG;
  constexpr int HALVES = CPLX ? 2 : 1;   // A stages per (K tile, M tile)
  constexpr int A_PLANE = Cfg::A_PLANE;
  constexpr int A_STAGE = Cfg::A_STAGE;
  constexpr int B_PART = Cfg::B_PART;
  constexpr int B_STAGE = Cfg::B_STAGE;
  constexpr int MCOLS = CPLX ? 2 * NBV : NVT;
  constexpr int TCOLS = (CPLX || NVT == 2 * NBV) ? 512 : 256;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + SA * A_STAGE;
  unsigned char* sE = sB + SB * B_STAGE;   // epilogue staging, one STG block per epilogue warp
  __shared__ uint64_t a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], acc_full[4], acc_empty[4], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_fail;
  __shared__ int s_rows[2][MAXPAD];   // gathered rows of the current / next tile (gather warps)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = A.npad / MT, ktn = A.npad / KT;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(&b_full[s], 128);
      mbar_init(&b_empty[s], 1);
    }
    for (int m = 0; m < 4; ++m) {
      mbar_init(&acc_full[m], 1);
      mbar_init(&acc_empty[m], 128);
    }
    mbar_init(&mma_done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      long long ga = 0;
      for (int k = 0; k < A.nk; ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&A.maps[k]) : "memory");
      for (long long t = blockIdx.x; t < A.ntiles && !s_fail; t += gridDim.x) {
        int k, e, vb, mte, kte;
        decode_tile(A, t, &k, &e, &vb);
        cell_tiles(A, e, mt, ktn, &mte, &kte);
        for (int it = 0; it < mte * kte * HALVES && !s_fail; ++it, ++ga) {
          const int h = it % HALVES, kt = it / (HALVES * mte), m = (it / HALVES) % mte;
          const int s = (int)(ga % SA);
          const long long u = ga / SA;
          if (u >= 1 && !mbar_wait(&a_empty[s], (uint32_t)((u - 1) & 1), &s_fail)) break;
          mbar_expect_tx(&a_full[s], A_STAGE);
          // one contiguous block of NPART planes: (cell, K tile, M tile, real or imaginary part)
          const int chunk = ((e * ktn + kt) * mt + m) * HALVES + h;
          tma_load_3d(smem_u32(sA + s * A_STAGE), &A.maps[k], 0, 0, NPART == 2 ? chunk : chunk * NPART, &a_full[s]);
        }
      }
      // drain: every issued load lands before the CTA leaves
      for (long long g = (ga > SA ? ga - SA : 0); g < ga; ++g) mbar_wait_drain(&a_full[g % SA], (uint32_t)((g / SA) & 1));
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      long long ga = 0, gb = 0;
      int use[4] = {0, 0, 0, 0};   // tiles so far whose products went to M tile m
      bool ok = true;
      for (long long t = blockIdx.x; t < A.ntiles && ok && !s_fail; t += gridDim.x) {
        int k, e, vb, mte, kte;
        decode_tile(A, t, &k, &e, &vb);
        cell_tiles(A, e, mt, ktn, &mte, &kte);
        for (int it = 0; it < mte * kte && ok; ++it) {
          const int kt = it / mte, m = it % mte;
          const int sb = (int)((gb + kt) % SB);
          if (kt == 0 && use[m] >= 1 && !mbar_wait(&acc_empty[m], (uint32_t)((use[m] - 1) & 1), &s_fail)) {
            ok = false;
            break;
          }
          if (m == 0 && !mbar_wait(&b_full[sb], (uint32_t)(((gb + kt) / SB) & 1), &s_fail)) { ok = false; break; }
          const uint32_t b_base = smem_u32(sB + sb * B_STAGE);
          const uint32_t dcol = taddr + m * MCOLS;
          constexpr uint32_t ID = idesc_bf16(MT, CPLX ? NBV : NVT, false);
          constexpr uint32_t IDN = idesc_bf16(MT, NBV, true);
          constexpr uint32_t ID2 = idesc_bf16(MT, 2 * NBV, false);   // [Re | Im] in one N = 128 MMA
          for (int h = 0; h < HALVES; ++h, ++ga) {
            const int s = (int)(ga % SA);
            if (!mbar_wait(&a_full[s], (uint32_t)((ga / SA) & 1), &s_fail)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_base = smem_u32(sA + s * A_STAGE);
            // the products of the split: (hi, hi), (hi, lo), (lo, hi) for two parts; for three parts
            // also (hi, lo), (mid, mid), (lo, hi) with mid in the middle: all pairs of order <= 2
            constexpr int NPROD = NPART == 2 ? 3 : 6;
            constexpr int PA[6] = {0, 0, 1, 0, 1, 2};
            constexpr int PX[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
            for (int ks = 0; ks < KT / 16; ++ks) {
              const uint32_t koff = ks * 32;
              if (!CPLX) {
#pragma unroll
                for (int pi = 0; pi < NPROD; ++pi)
                  mma_bf16(dcol, sdesc(a_base + PA[pi] * A_PLANE + koff), sdesc(b_base + PX[pi] * B_PART + koff), ID,
                           (pi == 0 && kt == 0 && ks == 0) ? 0u : 1u);
              } else if (h == 0 && MERGE) {   // real part: [Re Z | Im Z] += Re H [Re X | Im X]
#pragma unroll
                for (int pi = 0; pi < NPROD; ++pi)
                  mma_bf16(dcol, sdesc(a_base + PA[pi] * A_PLANE + koff), sdesc(b_base + PX[pi] * B_PART + koff), ID2,
                           (pi == 0 && kt == 0 && ks == 0) ? 0u : 1u);
              } else {
                // one accumulator at a time: Re Z then Im Z
                //   real part of H:       Re Z += Re H Re X,  Im Z += Re H Im X
                //   imaginary part of H:  Re Z -= Im H Im X,  Im Z += Im H Re X
#pragma unroll
                for (int acc = 0; acc < 2; ++acc) {
                  const uint32_t D = dcol + acc * NBV;
                  const uint32_t xoff = (h == 0 ? acc : 1 - acc) * NBV * 128;
                  const uint32_t idesc = (h == 1 && acc == 0) ? IDN : ID;
#pragma unroll
                  for (int pi = 0; pi < NPROD; ++pi)
                    mma_bf16(D, sdesc(a_base + PA[pi] * A_PLANE + koff), sdesc(b_base + PX[pi] * B_PART + xoff + koff),
                             idesc, (h == 0 && pi == 0 && kt == 0 && ks == 0) ? 0u : 1u);
                }
              }
            }
            mma_commit(&a_empty[s]);
          }
          if (!ok) break;
          if (m == mte - 1) mma_commit(&b_empty[sb]);
          if (kt == kte - 1) mma_commit(&acc_full[m]);
        }
        for (int m = 0; m < mte; ++m) ++use[m];
        gb += kte;
      }
      // every MMA issued has completed before the tensor memory is released
      if (ga > 0) {
        mma_commit(&mma_done);
        mbar_wait_drain(&mma_done, 0);
      }
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- gather producers
    const int gt = tid - 64;  // 0 .. 127
    long long gb = 0;
    int tg = 0;
    for (long long t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
      int k, e, vb;
      decode_tile(A, t, &k, &e, &vb);
      const MmaK P = kparams(A, k);
      const int ne = A.act_off[e + 1] - A.act_off[e];
      const int naug = A.nloc + ne;
      const int v0 = vb * NVT;
      int mte, kte;
      cell_tiles(A, e, mt, ktn, &mte, &kte);
      // the tile's row map, once per tile, double-buffered; the barrier publishes it and takes
      // the exit decision on a failure uniformly over the gather threads
      int* rows = s_rows[tg & 1];
      for (int r = gt; r < naug; r += 128)
        rows[r] = r < A.nloc ? A.cell_nodes[(size_t)e * A.nloc + r] : (int)(A.nh + A.act_idx[A.act_off[e] + r - A.nloc]);
      ++tg;
      if (gather_bar_or(s_fail != 0)) break;
      for (int kt = 0; kt < kte && !s_fail; ++kt, ++gb) {
        const int sb = (int)(gb % SB);
        const long long u = gb / SB;
        if (u >= 1 && !mbar_wait(&b_empty[sb], (uint32_t)((u - 1) & 1), &s_fail)) break;
        unsigned char* b0 = sB + sb * B_STAGE;
        // each thread owns one vector column v and the row pairs (kk, kk+1) p = r0 + TPV w of the
        // K tile (TPV threads per vector: 16 pairs each for 64-vector tiles, 32 for 128); all the
        // thread's loads of a K tile are issued together so their latencies overlap, and each pair
        // is written to shared memory as one packed bf16x2 word per plane
        constexpr int TPV = 128 / NVT;
        const int v = gt % NVT, r0 = gt / NVT;          // r0 in [0, TPV)
        constexpr int BATCH = KT / (2 * TPV);           // pairs per batch: all the thread's loads in flight
        const bool vok = v0 + v < P.nv;
#pragma unroll 1
        for (int j0 = 0; j0 < KT / (2 * TPV); j0 += BATCH) {
          float2 xv[2 * BATCH];
#pragma unroll
          for (int u = 0; u < 2 * BATCH; ++u) {
            const int kk = 2 * (r0 + TPV * (j0 + (u >> 1))) + (u & 1);
            const int r = kt * KT + kk;
            xv[u] = make_float2(0.f, 0.f);
            if (r < naug && vok) {
              const int64_t row = rows[r];
              if (CPLX) xv[u] = __ldg(reinterpret_cast<const float2*>(P.X) + row * P.ldx + v0 + v);
              else xv[u].x = __ldg(P.X + row * P.ldx + v0 + v);
            }
          }
#pragma unroll
          for (int w = 0; w < BATCH; ++w) {
            const int kk = 2 * (r0 + TPV * (j0 + w));   // even: the pair shares one 4-byte word
            const float2 x0 = xv[2 * w], x1 = xv[2 * w + 1];
            // NPART-way split of the pair: part s = bf16 of what the earlier parts left (the
            // differences are exact in FP32, so three parts hold an FP32 value exactly)
            float ra = x0.x, rb = x1.x;
#pragma unroll
            for (int s = 0; s < NPART; ++s) {
              const __nv_bfloat162 ps = __floats2bfloat162_rn(ra, rb);
              *reinterpret_cast<__nv_bfloat162*>(b0 + s * B_PART + swz(v, kk)) = ps;
              ra -= __low2float(ps);
              rb -= __high2float(ps);
            }
            if (CPLX) {
              float ia = x0.y, ib = x1.y;
#pragma unroll
              for (int s = 0; s < NPART; ++s) {
                const __nv_bfloat162 ps = __floats2bfloat162_rn(ia, ib);
                *reinterpret_cast<__nv_bfloat162*>(b0 + s * B_PART + swz(NBV + v, kk)) = ps;
                ia -= __low2float(ps);
                ib -= __high2float(ps);
              }
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&b_full[sb]);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;
    int use[4] = {0, 0, 0, 0};   // tiles so far whose M tile m was drained
    for (long long t = blockIdx.x; t < A.ntiles && !s_fail; t += gridDim.x) {
      int k, e, vb, mte, kte;
      decode_tile(A, t, &k, &e, &vb);
      cell_tiles(A, e, mt, ktn, &mte, &kte);
      const MmaK P = kparams(A, k);
      const int ne = A.act_off[e + 1] - A.act_off[e];
      const int naug = A.nloc + ne;
      const int v0 = vb * NVT;
      bool ok = true;
      for (int m = 0; m < mte; ++m) {
        if (!mbar_wait(&acc_full[m], (uint32_t)(use[m] & 1), &s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m * MT + 32 * q + lane;
        for (int h = 0; h < (CPLX ? 2 : NVT / 32); ++h) {
          const uint32_t tl0 = taddr + ((uint32_t)(32 * q) << 16) + m * MCOLS + 32 * h;
          float re[32], im[32];
          tmem_ld32(tl0, re);
          if (CPLX) tmem_ld32(tl0 + NBV, im);
          const int vb0 = v0 + 32 * h;
          const bool full = CPLX ? ((P.nv & 1) == 0 && vb0 + 32 <= P.nv) : ((P.nv & 3) == 0 && vb0 + 32 <= P.nv);
          if (full) {
            // stage the warp's rows (ER at a time) x 32 values in shared memory (16-byte chunks,
            // XOR-swizzled by row), then write whole row segments: 256 contiguous bytes per row
            // (complex), 128 (real)
            constexpr int CPR = CPLX ? 16 : 8;      // 16-byte chunks per row segment
            constexpr int RPI = 32 / CPR;           // rows per store instruction
            constexpr int ER = Cfg::ER;
            unsigned char* st = sE + q * STG;
#pragma unroll
            for (int round = 0; round < 32 / ER; ++round) {
              if (lane / ER == round) {
                const int sl = lane % ER;              // staging row of this lane
#pragma unroll
                for (int j = 0; j < CPR; ++j) {
                  const float4 v = CPLX ? make_float4(re[2 * j], im[2 * j], re[2 * j + 1], im[2 * j + 1])
                                        : make_float4(re[4 * j], re[4 * j + 1], re[4 * j + 2], re[4 * j + 3]);
                  *reinterpret_cast<float4*>(st + sl * (CPR * 16) + ((j ^ (sl & (CPR - 1))) << 4)) = v;
                }
              }
              __syncwarp();
              const int ch = lane % CPR, rsub = lane / CPR;
#pragma unroll
              for (int i = 0; i < ER; i += RPI) {
                const int rl = i + rsub;                     // staging row
                const int grow = m * MT + 32 * q + round * ER + rl;
                if (rl < ER && grow < naug) {
                  const float4 v =
                      *reinterpret_cast<const float4*>(st + rl * (CPR * 16) + ((ch ^ (rl & (CPR - 1))) << 4));
                  float* zr = P.Z + ((size_t)e * A.npad + grow) * (size_t)P.nv * (CPLX ? 2 : 1);
                  *reinterpret_cast<float4*>(zr + (CPLX ? 2 : 1) * vb0 + 4 * ch) = v;
                }
              }
              __syncwarp();
            }
          } else if (row < naug) {
            float* zr = P.Z + ((size_t)e * A.npad + row) * (size_t)P.nv * (CPLX ? 2 : 1);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int v = vb0 + j;
              if (v < P.nv) {
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
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&acc_empty[m]);
        ++use[m];
      }
      if (!ok) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) atomicExch(A.err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

size_t cell_mma_tma_smem(bool cplx, int parts, int nvt) {
  if (!cplx && nvt == 2 * NBV) return parts == 3 ? TmaCfg<false, 3, 2 * NBV>::SMEM : TmaCfg<false, 2, 2 * NBV>::SMEM;
  if (parts == 3) return cplx ? TmaCfg<true, 3>::SMEM : TmaCfg<false, 3>::SMEM;
  return cplx ? TmaCfg<true, 2>::SMEM : TmaCfg<false, 2>::SMEM;
}

// Tensor map of one k-point's split cell matrices, stored tile-contiguous ([cell][K tile][M tile]
// [plane][128][64]): one box = the bf16 parts of the real or of the imaginary part of one
// (K tile, M tile).
int make_cell_tmap(oefe_ctx* c, const KData& K, void* map_out) {
  auto fn = encode_fn();
  if (!fn) { c->err = "cuTensorMapEncodeTiled is not available"; return OEFE_ERR_CUDA; }
  const int parts = K.bf_parts;
  if (parts != 2 && parts != 3) { c->err = "tensor map: no split cell matrices"; return OEFE_ERR_STATE; }
  const int planes = (K.cplx ? 2 : 1) * parts;
  const cuuint64_t nplanes = (cuuint64_t)c->ncells * (c->npad / KT) * (c->npad / MT) * planes;
  // two parts: (column, row of a plane pair, chunk), box (64, 256, 1); three parts: (column, row,
  // plane), box (64, 128, 3) (a box dimension holds at most 256)
  const cuuint64_t dims[3] = {(cuuint64_t)KT, (cuuint64_t)MT * (parts == 2 ? 2 : 1), parts == 2 ? nplanes / 2 : nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)KT * 2, (cuuint64_t)MT * KT * 2 * (parts == 2 ? 2 : 1)};
  const cuuint32_t box[3] = {KT, (cuuint32_t)MT * (parts == 2 ? 2 : 1), parts == 2 ? 1u : 3u};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  const CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, K.Hbf, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    c->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return OEFE_ERR_CUDA;
  }
  std::memcpy(map_out, &m, sizeof(CUtensorMap));
  return OEFE_OK;
}

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

int launch_cell_mma_tma(oefe_ctx* c, const void* d_maps, const MmaK* d_ks, const MmaK* k0, int nk, long long ntiles,
                        bool cplx, int parts, int grid, cudaStream_t st, int nvt) {
  if (parts != 2 && parts != 3) { c->err = "tensor path: the split cell matrices were not stored"; return OEFE_ERR_STATE; }
  if (nvt != NBV && (cplx || nvt != 2 * NBV)) { c->err = "tensor path: 64 vectors per tile, or 128 for real data"; return OEFE_ERR_ARG; }
  if (c->npad % MT != 0 || c->npad > 4 * MT) {
    c->err = "tensor path needs npad a multiple of 128 and at most 512";
    return OEFE_ERR_ARG;
  }
  TmaArgs A;
  A.maps = (const CUtensorMap*)d_maps;
  A.ks = d_ks;
  if (k0) A.k0 = *k0;
  A.nk = nk;
  A.ntiles = ntiles;
  A.cell_nodes = c->d_cell_nodes;
  A.act_off = c->d_act_off;
  A.act_idx = c->d_act_idx;
  A.nloc = c->nloc;
  A.npad = c->npad;
  A.nh = c->nh;
  A.err = c->d_status;
  const size_t smem = cell_mma_tma_smem(cplx, parts, nvt);
  auto go = [&](auto kern) -> int {
    OEFE_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    OEFE_COUNTED kern<<<grid, THREADS, smem, st>>>(A);
    return OEFE_OK;
  };
  // merged real-part MMAs: the tuned choice, else on (measured faster for both splits)
  const bool merge = c->tune_merge >= 0 ? c->tune_merge != 0 : true;
  if (!cplx && nvt == 2 * NBV)
    OEFE_TRY(parts == 3 ? go(k_cell_mma_tma<false, 3, false, 2 * NBV>) : go(k_cell_mma_tma<false, 2, false, 2 * NBV>));
  else if (!cplx) OEFE_TRY(parts == 3 ? go(k_cell_mma_tma<false, 3, false>) : go(k_cell_mma_tma<false, 2, false>));
  else if (parts == 3) OEFE_TRY(merge ? go(k_cell_mma_tma<true, 3, true>) : go(k_cell_mma_tma<true, 3, false>));
  else OEFE_TRY(merge ? go(k_cell_mma_tma<true, 2, true>) : go(k_cell_mma_tma<true, 2, false>));
  OEFE_CUDA_TRY(c, cudaGetLastError());
  return OEFE_OK;
}
