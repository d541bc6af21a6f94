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

struct __align__(8) ff {  // the layout of float2: (hi, lo)
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

// ---- the same conversions with integer instructions, for streaming kernels.
// The FP64 pipe of this GPU issues about 1.5 instructions per cycle per SM,
// and ff(double) / to_double put three instructions on it (two F2F, one
// DADD), which bounds a kernel with little arithmetic per value far below
// HBM speed. split_double gives the same bits as ff(double) (hi = RN(d),
// lo = RN(d - hi), both round-to-nearest-even) by assembling them from the
// fields of d wherever hi and lo are normal floats (|d| in [2^-70, 2^127));
// elsewhere (zero, tiny, huge, inf, nan) it takes the hardware path.
// join_double gives the bits of to_double with one FP64 addition.
__device__ __forceinline__ ff split_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned E = (unsigned)(b >> 52) & 0x7FFu;
  if (E < 1023u - 70u || E > 1023u + 126u) return ff(d);
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  // top 23 mantissa bits: bits 51..29 of b = bits 19..0 of hi32 and 31..29 of lo32
  unsigned hib = sgn | ((E - 1023u + 127u) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
  const unsigned R = lo32 & 0x1FFFFFFFu;  // the 29 bits below hi's last bit
  const bool up = R > 0x10000000u || (R == 0x10000000u && (hib & 1u));
  hib += up ? 1u : 0u;  // a mantissa carry moves into the exponent, as it should
  const unsigned mag = up ? 0x20000000u - R : R;  // |d - hi| in units of 2^(E-1075)
  if (mag == 0u) return ff(__uint_as_float(hib), 0.0f);
  const int p = 31 - __clz(mag);  // leading bit of mag, 0..28
  unsigned q;
  if (p > 23) {  // round mag to 24 significant bits, nearest even
    const int sh = p - 23;
    q = mag >> sh;
    const unsigned rem = mag & ((1u << sh) - 1u), half = 1u << (sh - 1);
    q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
  } else {
    q = mag << (23 - p);
  }
  const unsigned ex = (unsigned)((int)E - 1075 + p + 127);
  const unsigned lsg = up ? sgn ^ 0x80000000u : sgn;
  const unsigned lob = lsg | ((ex << 23) + (q - 0x800000u));  // q = 2^24 carries into the exponent
  return ff(__uint_as_float(hib), __uint_as_float(lob));
}

// exact binary32 -> binary64 by re-biasing the exponent (normal floats and zero)
__device__ __forceinline__ double widen_float(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned a = b & 0x7FFFFFFFu;
  if (a == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  if (a - 0x00800000u >= 0x7F000000u) return (double)f;  // subnormal, inf, nan
  return __hiloint2double((int)((b & 0x80000000u) | (((a >> 23) + 896u) << 20) | ((a & 0x7FFFFFu) >> 3)),
                          (int)(a << 29));
}

__device__ __forceinline__ double join_double(ff a) { return widen_float(a.hi) + widen_float(a.lo); }

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
// storage <-> compute conversions of the streaming kernels (integer split)
template <typename TC, typename TS>
__device__ __forceinline__ TC stream_load(TS v) { return TC(v); }
template <>
__device__ __forceinline__ ff stream_load<ff, double>(double v) { return split_double(v); }
template <typename TS, typename TC>
__device__ __forceinline__ TS stream_store(TC v) { return TS(v); }
template <>
__device__ __forceinline__ double stream_store<double, ff>(ff v) { return join_double(v); }

template <typename T>
__device__ __forceinline__ T from_double(double d) { return T(d); }
template <>
__device__ __forceinline__ ff from_double<ff>(double d) { return ff(d); }
}  // namespace sipg
