// Double-float arithmetic for the FP64 steps of the solver: FP64 storage, FP32 arithmetic.
//
// GB300 executes about two FP64 fused multiply-adds per clock per SM against 128 FP32 ones, so
// the solver's high-precision operator applies (reliable updates, source preparation S_L and
// reconstruction S_R) run in "double-float": a value is the unevaluated sum hi + lo of two FP32
// numbers, about 48 significant bits. The operations are the error-free transformations of Knuth
// (TwoSum), Dekker (FastTwoSum) and the exact product through a fused multiply-add, combined as in
// the double-double arithmetic of Hida, Li and Bailey ("Algorithms for quad-double precision
// floating point arithmetic", 2001) with FP32 in place of FP64; additions use the faster variant
// whose error is bounded relative to |a| + |b| (no cancellation-sensitive sums occur inside the
// operator; the solver's cancelling difference b - A y is taken in FP64 afterwards).
//
// Loads and stores convert between FP64 and the float pair with integer operations only, so no
// instruction of a double-float kernel runs on the FP64 pipe. Range: magnitudes below 2^-126 load
// as zero and the low word is dropped below 2^-74 (the operator's fields are far from both).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace wf {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // from a compile-time or host value (FP64 arithmetic: not for device hot loops)
  __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df64(int i) : df64((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// (s, e) with s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}
// (s, e) with s + e = a + b exactly, for |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  df64 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // exact low part of a.hi * b.hi
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df64 r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
// a * b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
using ::fma;

// FP64 -> float pair by integer operations: hi takes the sign, the exponent and the leading 23
// fraction bits; lo the remaining 29 fraction bits, scaled by 2^(e - 1075)
__device__ __forceinline__ df64 df_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu);
  const int fe = e - 1023 + 127;
  if (fe <= 0) return df64(0.f, 0.f);
  const unsigned hb = sgn | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rem = (unsigned)(b & 0x1fffffffu);
  float lo = 0.f;
  const int le = e - 1075 + 127;
  if (le > 0 && rem) {
    // exact conversion of the 29-bit integer rem in two 23-bit pieces (2^23 + x trick)
    const float f_lo = __uint_as_float(0x4B000000u | (rem & 0x7fffffu)) - 8388608.f;
    const float f_hi = __uint_as_float(0x4B000000u | (rem >> 23)) - 8388608.f;
    lo = fmaf(f_hi, 8388608.f, f_lo) * __uint_as_float((unsigned)le << 23);
    lo = __uint_as_float(__float_as_uint(lo) | sgn);
  }
  return df64(__uint_as_float(hb), lo);
}

// float pair -> FP64 by integer operations: both significands aligned to hi's exponent in a 64-bit
// integer, added, renormalised to 53 bits (truncating)
__device__ __forceinline__ double df_to_double(df64 v) {
  const unsigned hb = __float_as_uint(v.hi), lb = __float_as_uint(v.lo);
  const int eh = (int)((hb >> 23) & 0xffu), el = (int)((lb >> 23) & 0xffu);
  if (eh == 0) {
    if (el == 0) return 0.0;
    // lo alone (a normal FP32 value): exact re-encoding
    const unsigned long long bits = ((unsigned long long)(lb & 0x80000000u) << 32) |
                                    ((unsigned long long)(el - 127 + 1023) << 52) |
                                    ((unsigned long long)(lb & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
  }
  long long H = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;  // units of 2^(eh - 179)
  if (hb & 0x80000000u) H = -H;
  long long Lv = 0;
  if (el != 0) {
    const unsigned long long ml = (lb & 0x7fffffu) | 0x800000u;
    int sh = el - eh + 29;  // lo in units of 2^(eh - 179)
    if (sh > 8) sh = 8;     // a well-formed pair has |lo| <= ulp(hi): sh <= 6
    const unsigned long long m = sh >= 0 ? (ml << sh) : (sh > -64 ? (ml >> -sh) : 0ull);
    Lv = (lb & 0x80000000u) ? -(long long)m : (long long)m;
  }
  long long S = H + Lv;
  if (S == 0) return 0.0;
  const unsigned long long sg = S < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long A = (unsigned long long)(S < 0 ? -S : S);
  const int p = 63 - __clzll((long long)A);  // leading bit position
  if (p > 52)
    A >>= (p - 52);
  else
    A <<= (52 - p);
  const long long E = (long long)eh + p + 844;  // biased FP64 exponent of A * 2^(eh - 179 + p - 52)
  const unsigned long long bits = sg | ((unsigned long long)E << 52) | (A & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

}  // namespace wf
