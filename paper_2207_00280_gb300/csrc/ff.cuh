// ff.cuh -- float-float arithmetic for the FP64_DF forms of the kernels.
//
// A value is hi + lo, two FP32 numbers (about 48 significant bits); products
// use the exact FMA error term (Dekker/Kahan), sums Knuth's two-sum with a
// renormalisation; every multiply-add runs on the FP32 pipes, which GB300
// issues 64 times faster than FP64 ones.  Inputs stay double in memory
// (store_t) and are split with integer instructions (to_compute), results are
// written back as double (to_store).  Dot products use mac/fin: the exact
// two-sum of the high products and one error term, renormalised once.
#pragma once
#include <cstdint>

namespace iga {

struct ff {
  float hi, lo;
  ff() = default;
  __device__ __forceinline__ ff(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit ff(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
};
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = p + e;
  return ff(s, e - (s - p));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  const float l = err + a.lo + b.lo;
  const float h = s + l;
  return ff(h, l - (h - s));
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) {
  a = a + b;
  return a;
}

// x as hi + lo without FP64 arithmetic: hi = x with its mantissa cut to 24
// bits (exact in FP32), lo = the remaining 29 bits as an integer, converted
// (rounded to 24 bits) and scaled by 2^(e - 1075), both normal FP32 numbers
// for biased exponents e in [949, 1150] (2^-74 <= |x| < 2^128).  Zeros and
// values outside that range take the exact FP64 conversion.
__device__ __forceinline__ ff split_d(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex < 949 || ex > 1150) return ff(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned mh = (unsigned)((b >> 29) & 0x7fffffu);
  const float h = __uint_as_float(sgn | ((unsigned)(ex - 896) << 23) | mh);
  const unsigned ml = (unsigned)(b & 0x1fffffffu);
  const float l = __uint2float_rn(ml) * __uint_as_float((unsigned)(ex - 948) << 23);
  return ff(h, sgn ? -l : l);
}

// Dot products: mac(a, x, y) accumulates x * y into a; fin(a) is the value.
// For ff the accumulator keeps the exact two-sum of the high products in hi
// and every low-order term in lo, renormalised once by fin, so the
// loop-carried dependence is one FP32 add.
template <typename T> __device__ __forceinline__ void mac(T& a, T x, T y) { a += x * y; }
template <typename T> __device__ __forceinline__ T fin(T a) { return a; }
template <> __device__ __forceinline__ void mac<ff>(ff& a, ff x, ff y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  const float s = a.hi + p;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (p - bb);
  a.hi = s;
  a.lo += err + e;
}
template <> __device__ __forceinline__ ff fin<ff>(ff a) {
  const float h = a.hi + a.lo;
  return ff(h, a.lo - (h - a.hi));
}

template <typename T> struct store_of { using type = T; };
template <> struct store_of<ff> { using type = double; };
template <typename T> using store_t = typename store_of<T>::type;

template <typename T> __device__ __forceinline__ T to_compute(store_t<T> x) { return x; }
template <> __device__ __forceinline__ ff to_compute<ff>(double x) { return split_d(x); }
template <typename T> __device__ __forceinline__ T from_double(double x) { return (T)x; }
template <> __device__ __forceinline__ ff from_double<ff>(double x) { return split_d(x); }
template <typename T> __device__ __forceinline__ store_t<T> to_store(T x) { return x; }
template <> __device__ __forceinline__ double to_store<ff>(ff x) { return (double)x.hi + (double)x.lo; }

// The double equal to float f, by integer instructions for normal numbers
// and zeros (sign, exponent rebiased from 127 to 1023, mantissa shifted to
// the top of 52 bits); subnormal, infinite and NaN values take the
// conversion instruction.  The same value as (double)f.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u <= 253u)
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu)),
                            (int)(u << 29));
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}

// to_store with the two exact conversions of a float-float done by integer
// instructions and one FP64 addition left (the same double).  For kernels
// whose FP64 pipe also carries other work (the adjoint's FP64 partial sums);
// where issue slots are the limit, to_store's conversion instructions cost less.
template <typename T> __device__ __forceinline__ store_t<T> to_store_int(T x) { return to_store<T>(x); }
template <> __device__ __forceinline__ double to_store_int<ff>(ff x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

}  // namespace iga
