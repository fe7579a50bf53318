// Double-float arithmetic on the FP32 pipes for the df64 type (dg_internal.h).
//
// A value is hi + lo with two FP32 numbers. The operations are built from two error-free
// transformations:
//   TwoSum(a, b) = (s, e) with s = fl(a + b) and s + e = a + b exactly, in six
//     additions and no branch (Knuth, TAOCP Vol. 2, Sec. 4.2.2, Theorem B);
//   FastTwoSum(a, b) for |a| >= |b|, the same in three additions (Dekker, Numer. Math.
//     18 (1971), 224-242);
// and the fused multiply-add, which gives the rounding error of a product exactly:
// a b - fl(a b) = fma(a, b, -fl(a b)).
// Products keep the cross terms hi_a lo_b and lo_a hi_b and drop lo_a lo_b (2^-48
// relative); sums add the low parts after a TwoSum of the high parts (the "sloppy"
// double-double addition). The result has a relative error of a few 2^-48 per operation,
// and in a cancelling sum an absolute error of a few 2^-48 times the operands.
//
// Every step uses the round-to-nearest intrinsics (__fadd_rn, __fsub_rn, __fmul_rn),
// which the compiler never contracts into an FMA or reassociates: a contraction would
// break the exactness of the transformations.
#pragma once
#include "dg_internal.h"

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// exact product of the high parts plus the two cross terms, as an unnormalised (p, e)
__device__ __forceinline__ void df_prod(const df64 &a, const df64 &b, float &p, float &e) {
  p = __fmul_rn(a.hi, b.hi);
  e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
}

__device__ __forceinline__ df64 operator*(const df64 &a, const df64 &b) {
  float p, e;
  df_prod(a, b, p, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64 operator+(const df64 &a, const df64 &b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(const df64 &a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(const df64 &a, const df64 &b) { return a + (-b); }
__device__ __forceinline__ df64 &operator*=(df64 &a, const df64 &b) { return a = a * b; }

// a b + c with one normalisation: the product's error term joins the low parts
__device__ __forceinline__ df64 fma(const df64 &a, const df64 &b, const df64 &c) {
  float p, e;
  df_prod(a, b, p, e);
  const df64 s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// a / b: the FP32 quotient of the high parts, corrected once by the quotient of the
// double-float remainder a - q b (Dekker 1971, Sec. 8), about 2^-46 relative.
__device__ __forceinline__ df64 operator/(const df64 &a, const df64 &b) {
  const float q = __fdiv_rn(a.hi, b.hi);
  const df64 r = a - b * df64(q, 0.f);
  return df_fast_two_sum(q, __fdiv_rn(r.hi, b.hi));
}

// sqrt(a) for a >= 0: the FP32 root s of the high part and one Newton correction
// (a - s^2) / (2 s) with the exact square (Karp and Markstein, ACM TOMS 23 (1997)).
__device__ __forceinline__ df64 sqrt(const df64 &a) {
  if (!(a.hi > 0.f)) return df64(0.f, 0.f);
  const float s = __fsqrt_rn(a.hi);
  const df64 r = a - df64(s, 0.f) * df64(s, 0.f);
  return df_fast_two_sum(s, __fdiv_rn(r.hi, __fadd_rn(s, s)));
}

// Accumulator of a contraction sum_j a_j b_j. For double and float it is the plain FMA
// chain (the same instructions as writing the chain out). For df64 it keeps a running
// FP32 high sum s, updated by TwoSum with each exact high product, and one FP32 sum c of
// everything below it: the products' rounding errors, the cross terms hi_a lo_b and
// lo_a hi_b, and the TwoSum errors. It normalises once at the end: 12 FP32 operations
// per term instead of 15 for a chain of double-float FMAs. The error terms are about
// 2^-24 of the products, so summing them in FP32 keeps the 2^-48 relative accuracy.
template <typename T>
struct Acc {
  T v;
  __device__ __forceinline__ void init(const T &a, const T &b) { v = a * b; }
  __device__ __forceinline__ void set(const T &x) { v = x; }
  __device__ __forceinline__ void add(const T &a, const T &b) { v = fma(a, b, v); }
  __device__ __forceinline__ T get() const { return v; }
};

template <>
struct Acc<df64> {
  float s, c;
  __device__ __forceinline__ void init(const df64 &a, const df64 &b) {
    s = __fmul_rn(a.hi, b.hi);
    c = fmaf(a.hi, b.hi, -s);
    c = fmaf(a.hi, b.lo, c);
    c = fmaf(a.lo, b.hi, c);
  }
  __device__ __forceinline__ void set(const df64 &x) { s = x.hi; c = x.lo; }
  __device__ __forceinline__ void add(const df64 &a, const df64 &b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    const df64 t = df_two_sum(s, p);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, e));
    c = fmaf(a.hi, b.lo, c);
    c = fmaf(a.lo, b.hi, c);
  }
  __device__ __forceinline__ df64 get() const { return df_fast_two_sum(s, c); }
};

// Store of a value computed in T to a T buffer, or of a double-float value to an FP64 one.
template <typename T>
__device__ __forceinline__ void store_to(T *p, const T &v) { *p = v; }
__device__ __forceinline__ void store_to(df64 *p, const df64 &v) { *p = v; }
__device__ __forceinline__ void store_to(double *p, const df64 &v) { *p = (double)v.hi + (double)v.lo; }

// Conversions of the FP64 input and output vectors (identity for double and float).
template <typename T>
__device__ __forceinline__ T io_in(io_t<T> v) { return v; }
template <>
__device__ __forceinline__ df64 io_in<df64>(double v) {
  const float h = __double2float_rn(v);
  return df64(h, __double2float_rn(v - (double)h));
}
template <typename T>
__device__ __forceinline__ io_t<T> io_out(T v) { return v; }
__device__ __forceinline__ double io_out(df64 v) { return (double)v.hi + (double)v.lo; }

// Accumulator of a dot product at FP64-class accuracy. For FP32 values it runs on the FP32
// pipes: each product a b enters as its rounded value p = fl(a b), added to the high sum
// by TwoSum, and as its exact rounding error fma(a, b, -p), added with the TwoSum error to
// an FP32 low sum; value() = hi + lo in FP64 (about 44 significant bits after thousands of
// terms, against 24 for an FP32 sum). For FP64 values it is one FP64 FMA per product.
template <typename T>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s = fma((double)a, (double)b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const df64 t = df_two_sum(hi, p);
    hi = t.hi;
    lo = __fadd_rn(lo, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ void add4(float4 a, float4 b) {
    add(a.x, b.x);
    add(a.y, b.y);
    add(a.z, b.z);
    add(a.w, b.w);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
