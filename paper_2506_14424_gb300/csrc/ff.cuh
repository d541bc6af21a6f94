// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two IEEE binary32 numbers with |lo| <= ulp(hi)/2, about 48
// significant bits. Built from the error-free transformations of Knuth
// (TwoSum), Dekker (FastTwoSum) and the FMA-based TwoProduct, as in Hida, Li
// and Bailey, "Algorithms for quad-double precision floating point
// arithmetic" (2001). Every step uses the explicitly rounded intrinsics
// (__fadd_rn, __fmul_rn, __fmaf_rn) so that the compiler can neither contract
// nor reassociate them.
//
// On this GPU the FP32 pipe issues 75x more operations per cycle than the
// FP64 pipe, so FP64-accurate operator applies run faster in this format
// (~10-20 FP32 operations per multiply-add) than in native FP64.
#pragma once
#include <cuda_runtime.h>

namespace sipg {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ff(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ constexpr ff(int v) : hi(float(v)), lo(0.0f) {}
  // split of a binary64 value: hi = RN(d), lo = RN(d - hi) (d - hi is exact)
  __device__ explicit ff(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
};

__device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff(s, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);          // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { a = a + b; return a; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { a = a * b; return a; }
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
// a / b by one Newton correction of the FP32 quotient (used off the hot path)
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - b * ff(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

// Dot-product accumulator: sum_j m_j x_j with exact products and a lazily
// normalised low word (one renormalisation at the end).
template <typename T>
struct Acc {
  T s = T(0);
  __device__ __forceinline__ void add(T m, T x) { s += m * x; }
  __device__ __forceinline__ T get() const { return s; }
};
template <>
struct Acc<ff> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(ff m, ff x) {
    const float p = __fmul_rn(m.hi, x.hi);
    float e = __fmaf_rn(m.hi, x.hi, -p);
    e = __fmaf_rn(m.hi, x.lo, e);
    e = __fmaf_rn(m.lo, x.hi, e);
    const ff s = two_sum(hi, p);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, e));
  }
  __device__ __forceinline__ ff get() const { return fast_two_sum(hi, lo); }
};

// storage <-> compute conversions
template <typename TC, typename TS>
__device__ __forceinline__ TC load_as(TS v) { return TC(v); }
template <>
__device__ __forceinline__ ff load_as<ff, double>(double v) { return ff(v); }
template <typename TS, typename TC>
__device__ __forceinline__ TS store_as(TC v) { return TS(v); }
template <>
__device__ __forceinline__ double store_as<double, ff>(ff v) { return to_double(v); }

}  // namespace sipg

namespace sipg {
template <typename T>
__device__ __forceinline__ T from_double(double d) { return T(d); }
template <>
__device__ __forceinline__ ff from_double<ff>(double d) { return ff(d); }
}  // namespace sipg
