// Digit slicing of FP64 values for the exact tensor-core products of the Gram matrices and
// rotations (the Ozaki scheme with bf16 digits): the digits of a value under a common exponent, the
// exact rescaling of an FP32 partial sum to FP64, and the bulk copy into shared memory.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tcgen05_dev.cuh"

namespace {

constexpr int OZ_S = 7;             // digits per value

// Y = trunc(x 2^(49-E)) from the bits of x by integer operations only (|x| < 2^E; subnormals
// count as zero), then the digits: c0 signed, the rest non-negative (two's complement split)
__device__ __forceinline__ void digits7(unsigned long long b, int E, float c[OZ_S]) {
  const int ex = (int)((b >> 52) & 0x7FF);
  const int sh = 1026 - ex + E;                         // >= 4 since |x| < 2^E
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long ya = (ex == 0 || sh >= 64) ? 0ull : (mant >> sh);
  const long long Y = (b >> 63) ? -(long long)ya : (long long)ya;
  // small integers to float without a conversion instruction: 2^23 + m as bits, minus 2^23
  const int top = (int)(Y >> 42) + 128;                 // c0 + 128 in [0, 255]
  c[0] = __fsub_rn(__int_as_float(0x4B000000 | top), 8388736.0f);   // 2^23 + 128
#pragma unroll
  for (int s = 1; s < OZ_S; ++s)
    c[s] = __fsub_rn(__int_as_float(0x4B000000 | (int)((Y >> (42 - 7 * s)) & 127)), 8388608.0f);
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// x 2^sc as a double (exact): the float's sign and fraction with the exponent rebased, by integer
// operations (IEEE 754 binary32 and binary64 layouts); zero, subnormal, infinite or NaN x and a
// result outside the normal range go through ldexp
__device__ __forceinline__ double f_scaled(float x, int sc) {
  const unsigned int b = __float_as_uint(x);
  const int ef = (int)((b >> 23) & 0xFFu);
  const int e = ef - 127 + 1023 + sc;
  if (ef == 0 || ef == 255 || e < 1 || e > 2046) return ldexp((double)x, sc);
  const unsigned long long bits = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)e << 52) |
                                  ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

}  // namespace
