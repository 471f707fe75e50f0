// FP64-class arithmetic on the FP32 pipe: a value is an unevaluated sum h + l of two FP32 numbers
// (|l| <= ulp(h) / 2, about 48 significant bits), the "double-length" arithmetic of Dekker (1971).
// A multiply-add takes the exact product of the high parts by FMA (Dekker's product in its FMA
// form), adds the cross terms, and adds the result to the accumulator's high part exactly by
// Knuth's two-sum; the rounding errors collect in the accumulator's low part. Twelve FP32
// operations per multiply-add: on a GPU that issues FP32 at 64 times its FP64 rate this is about
// five times the throughput of an FP64 FMA. Every operation is written with the _rn intrinsics so
// that the compiler neither contracts nor reassociates the error-free steps.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace {

// 8-byte aligned, so that a pair moves as one 64-bit load or store (two 32-bit accesses to
// interleaved words would take twice the shared-memory wavefronts)
struct alignas(8) f2 {
  float h, l;
};

// accumulator: h holds the running sum, l the collected rounding errors (normalized by f2_fin)
struct alignas(8) f2acc {
  float h, l;
};

__device__ __forceinline__ f2 f2_from(double x) {
  const float h = __double2float_rn(x);
  return f2{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double f2_to(f2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{-a.h, -a.l}; }

// s += a b
__device__ __forceinline__ void f2_mac(f2acc& s, f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);  // exact: a.h b.h = p + e
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float t = __fadd_rn(s.h, p);  // two-sum: s.h + p = t + er exactly
  const float bp = __fsub_rn(t, s.h);
  const float er = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(er, e));
}

__device__ __forceinline__ f2 f2_fin(f2acc s) {
  const float h = __fadd_rn(s.h, s.l);  // fast two-sum (|s.h| >= |s.l|)
  return f2{h, __fsub_rn(s.l, __fsub_rn(h, s.h))};
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const float t = __fadd_rn(a.h, b.h);
  const float bp = __fsub_rn(t, a.h);
  const float er = __fadd_rn(__fsub_rn(a.h, __fsub_rn(t, bp)), __fsub_rn(b.h, bp));
  return f2_fin(f2acc{t, __fadd_rn(er, __fadd_rn(a.l, b.l))});
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2acc s{0.0f, 0.0f};
  f2_mac(s, a, b);
  return f2_fin(s);
}

// ---- one interface over FP64 and pairs, for kernels written once for both
template <typename V>
struct AccOf;
template <>
struct AccOf<double> {
  using type = double;
};
template <>
struct AccOf<f2> {
  using type = f2acc;
};

template <typename V>
__device__ __forceinline__ V v_from(double x);
template <>
__device__ __forceinline__ double v_from<double>(double x) { return x; }
template <>
__device__ __forceinline__ f2 v_from<f2>(double x) { return f2_from(x); }

__device__ __forceinline__ double v_to(double a) { return a; }
__device__ __forceinline__ double v_to(f2 a) { return f2_to(a); }
__device__ __forceinline__ double v_neg(double a) { return -a; }
__device__ __forceinline__ f2 v_neg(f2 a) { return f2_neg(a); }
__device__ __forceinline__ void v_mac(double& s, double a, double b) { s = fma(a, b, s); }
__device__ __forceinline__ void v_mac(f2acc& s, f2 a, f2 b) { f2_mac(s, a, b); }
__device__ __forceinline__ double v_fin(double s) { return s; }
__device__ __forceinline__ f2 v_fin(f2acc s) { return f2_fin(s); }
__device__ __forceinline__ double v_mul(double a, double b) { return a * b; }
__device__ __forceinline__ f2 v_mul(f2 a, f2 b) { return f2_mul(a, b); }
__device__ __forceinline__ double v_add(double a, double b) { return a + b; }
__device__ __forceinline__ f2 v_add(f2 a, f2 b) { return f2_add(a, b); }
template <typename V>
__device__ __forceinline__ typename AccOf<V>::type v_zero() {
  return typename AccOf<V>::type{};
}

// sum_{i < n} a(i) b(i). Pairs: two independent accumulators (even and odd terms), so that the
// dependent two-sum chains of consecutive terms overlap; FP64: one FMA chain.
template <typename V, typename FA, typename FB>
__device__ __forceinline__ V v_dot(int n, FA a, FB b) {
  if constexpr (std::is_same<V, double>::value) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(a(i), b(i), s);
    return s;
  } else {
    f2acc s0{0.0f, 0.0f}, s1{0.0f, 0.0f};
    int i = 0;
    for (; i + 1 < n; i += 2) {
      f2_mac(s0, a(i), b(i));
      f2_mac(s1, a(i + 1), b(i + 1));
    }
    if (i < n) f2_mac(s0, a(i), b(i));
    return f2_add(f2_fin(s0), f2_fin(s1));
  }
}

}  // namespace
