// Double-single arithmetic on the device and the global loads / stores of
// nodal values for the apply kernels (included by fine.cu and dim3.cu).
#pragma once

#include "kernels.h"

namespace th {

// ----------------------------------------------------- double-single arithmetic
// Error-free transformations of Knuth (two_sum) and Dekker (fast_two_sum, the
// FMA form of two_prod); the rounded intrinsics keep the compiler from
// contracting or reassociating the steps.  Relative error of +, * about 2^-47.
__device__ __forceinline__ ds ds_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ds(s, e);
}
__device__ __forceinline__ ds ds_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return ds(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ds operator+(ds a, ds b) {
  const ds s = ds_two_sum(a.h, b.h);
  return ds_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ds operator-(ds a) { return ds(-a.h, -a.l); }
__device__ __forceinline__ ds operator-(ds a, ds b) { return a + (-b); }
__device__ __forceinline__ ds operator*(ds a, ds b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return ds_fast_two_sum(p, e);
}
__device__ __forceinline__ ds& operator+=(ds& a, ds b) { return a = a + b; }
__device__ __forceinline__ ds fmadd(ds a, ds b, ds c) { return c + a * b; }
__device__ __forceinline__ ds& operator-=(ds& a, ds b) { return a = a - b; }

// Unnormalised double-single accumulator: s takes the rounded products and
// sums, c the exact rounding errors (Knuth's two-sum for the additions,
// Dekker's product through FMA for the multiplications).  A term costs 12
// FP32 operations against 18 for a normalised ds multiply-add; the pair is
// normalised once, at the end (ds_of).
struct dsacc {
  float s, c;
};
__device__ __forceinline__ void acc_prod(dsacc& a, ds x, ds y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  const float t = __fadd_rn(a.s, p);
  const float z = __fsub_rn(t, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(p, z));
  a.c = __fadd_rn(a.c, __fadd_rn(err, e));
  a.s = t;
}
// the accumulated value as a normalised ds number
__device__ __forceinline__ ds ds_of(const dsacc& a) { return ds_two_sum(a.s, a.c); }

// Multiply-accumulate chains of the apply kernels: plain T for FP32 / FP64
// (the expressions of those kernels unchanged), the unnormalised pair for ds.
template <typename T>
struct MacAcc {
  using type = T;
};
template <>
struct MacAcc<ds> {
  using type = dsacc;
};
template <typename T>
__device__ __forceinline__ void mac(T& acc, T a, T b) {  // acc += a b
  acc += a * b;
}
__device__ __forceinline__ void mac(dsacc& acc, ds a, ds b) { acc_prod(acc, a, b); }
template <typename T>
__device__ __forceinline__ void mac_fma(T& acc, T a, T b) {  // acc = fma(a, b, acc)
  acc = fmadd(a, b, acc);
}
__device__ __forceinline__ void mac_fma(dsacc& acc, ds a, ds b) { acc_prod(acc, a, b); }
template <typename T>
__device__ __forceinline__ T mac_val(const T& a) {
  return a;
}
__device__ __forceinline__ ds mac_val(const dsacc& a) { return ds_of(a); }

// Exact split of a double into h (its leading 24 significant bits, truncated)
// and l (the remaining 29 bits rounded to 24) with integer operations only;
// magnitudes below 2^-126 (and l below the float range) flush to zero.
__device__ __forceinline__ ds ds_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32);
  const unsigned sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  const int ef = e - 1023 + 127;
  if (ef <= 0) return ds(0.f, 0.f);
  if (ef >= 255) return ds(__uint_as_float(sign | 0x7f800000u | ((hi32 & 0xfffffu) ? 0x400000u : 0u)), 0.f);
  const unsigned frac23 = (unsigned)((b >> 29) & 0x7fffffu);
  const float h = __uint_as_float(sign | ((unsigned)ef << 23) | frac23);
  const unsigned low = (unsigned)(b & 0x1fffffffu);
  if (low == 0) return ds(h, 0.f);
  const unsigned fb = __float_as_uint(__uint2float_rn(low));  // low * 2^(e - 1075), rescaled below
  const int ne = (int)((fb >> 23) & 0xffu) + (e - 1075);
  const float l = ne > 0 ? __uint_as_float(sign | ((unsigned)ne << 23) | (fb & 0x7fffffu)) : 0.f;
  return ds(h, l);
}

// float -> double by its bit pattern (integer operations only: the FP64 pipe
// of this GPU is 1/64 of the FP32 rate); subnormal floats become zero
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu, m = e == 0u ? 0u : (u & 0x7fffffu);
  const unsigned ed = e == 0u ? 0u : (e == 255u ? 2047u : e + 896u);
  return __hiloint2double((int)((u & 0x80000000u) | (ed << 20) | (m >> 3)), (int)((m & 7u) << 29));
}

// Global loads and stores of nodal values: FP64 / FP32 as stored; for the
// double-single apply the inputs are FP64 vectors and the output is FP32.
template <typename T>
struct NodeIO {
  using C = typename Cx<T>::t;
  static __device__ __forceinline__ C ld(const C* p, size_t i) { return p[i]; }
  static __device__ __forceinline__ void st(C* p, size_t i, C v) { p[i] = v; }
};
template <>
struct NodeIO<ds> {
  static __device__ __forceinline__ cds ld(const cds* p, size_t i) {
    const double2 d = reinterpret_cast<const double2*>(p)[i];
    cds c;
    c.x = ds_from_double(d.x);
    c.y = ds_from_double(d.y);
    return c;
  }
  static __device__ __forceinline__ void st(cds* p, size_t i, cds v) {
    reinterpret_cast<float2*>(p)[i] = make_float2(__fadd_rn(v.x.h, v.x.l), __fadd_rn(v.y.h, v.y.l));
  }
};

}  // namespace th
