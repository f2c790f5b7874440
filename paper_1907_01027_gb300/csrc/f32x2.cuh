// Float-float ("f32x2") arithmetic, the precision of the residual sweeps of the mixed-precision solve.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2: 48 significant bits in
// float's exponent range.  The operations are built from three error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and e with a + b = s + e exactly, 6 additions;
//   FastTwoSum (Dekker 1971): the same in 3 additions when |a| >= |b| or a = 0;
//   TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p), a b = p + e exactly.
// A sum adds the low parts to the TwoSum error of the high parts and renormalises once; a product adds the
// cross terms hi_a lo_b + lo_a hi_b to the TwoProd error.  The error of each operation is a few units of 2^-48
// of the operands' magnitudes (|a| + |b| for a sum), against 2^-53 in double: enough for a residual that must
// be right to 1e-8 of its reference, and all of it runs on the FP32 pipe, which on this GPU issues 64 times the
// FP64 pipe's instructions per cycle.
//
// The additions and the products that feed the transformations use the _rn intrinsics, which the compiler never
// contracts into fused multiply-adds: a contraction would break the exactness the transformations rely on.
#pragma once
#include <cuda_runtime.h>
#include <cmath>

namespace lmdg {

using ::fabs;
using ::fma;

struct __align__(8) f2 {
  float hi, lo;
  f2() = default;
  __host__ __device__ constexpr f2(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr f2(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ constexpr f2(float h, float l) : hi(h), lo(l) {}
  // rounded to the nearest float, then the remainder rounded (exact when the double has at most 48 bits)
  __host__ __device__ constexpr explicit f2(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  return s;
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return f2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.hi, -a.lo); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
  float e;
  const float s = two_sum(a.hi, b.hi, e);
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return a + (-b); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 operator*(f2 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 operator*(float a, f2 b) { return b * a; }
// a b + c with one renormalisation
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float t;
  const float s = two_sum(p, c.hi, t);
  return fast_two_sum(s, __fadd_rn(t, __fadd_rn(e, c.lo)));
}
// 1 / x: one Newton step r + r (1 - x r) from the hardware approximation r of 1 / hi (relative error about
// 2^-23, so the step leaves about 2^-46); the residual 1 - x r is formed with fused multiply-adds, in which it
// is exact to float rounding of its own (small) magnitude.
__device__ __forceinline__ f2 rcp(f2 x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
  const float e = fmaf(-x.lo, r, fmaf(-x.hi, r, 1.0f));
  return fast_two_sum(r, __fmul_rn(e, r));
}
__device__ __forceinline__ f2 operator/(f2 a, f2 b) { return a * rcp(b); }
__device__ __forceinline__ f2 &operator+=(f2 &a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2 &operator-=(f2 &a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2 &operator*=(f2 &a, f2 b) { return a = a * b; }
__device__ __forceinline__ f2 fabs(f2 a) {
  const unsigned m = __float_as_uint(a.hi) & 0x80000000u;
  return f2(__uint_as_float(__float_as_uint(a.hi) ^ m), __uint_as_float(__float_as_uint(a.lo) ^ m));
}

// host conversion of a double (setup data)
inline f2 f2_from_double(double v) {
  const float h = (float)v;
  return f2(h, (float)(v - (double)h));
}

template <typename T> struct is_f2 { static constexpr bool value = false; };
template <> struct is_f2<f2> { static constexpr bool value = true; };

}  // namespace lmdg
