// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  On this GPU
// FP32 runs 61 times faster than FP64, so pipe-bound FP64 kernels can run
// their arithmetic in pairs of FP32 instead.
//
// The operations are the classical error-free transformations: Knuth's
// TwoSum (the rounding error of a + b, exact for any a, b), Dekker's
// Fast-TwoSum renormalisation (exact when |a| >= |b|) and the FMA form of the
// product error (fma(a, b, -fl(a b)) is the exact rounding error of a b).
// Every step uses the explicitly rounded intrinsics, so the compiler cannot
// contract or reassociate them.  Addition ("sloppy" variant: the two low
// parts are added once) and multiplication each cost 8-10 FP32 operations;
// their relative error is a small multiple of 2^-48 except when the high
// parts of a sum cancel, where the error stays a small multiple of 2^-48
// times the operands.
#pragma once

#include <cuda_runtime.h>

namespace mgdg {

struct df64 {
  float hi, lo;
  __host__ __device__ df64() {}
  __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ df64(int v) : hi((float)v), lo(0.f) {}
  __device__ df64(float v) : hi(v), lo(0.f) {}
  // nearest pair to an FP64 value (FP64 arithmetic; constants fold at compile time)
  __device__ df64(double v) {
#ifdef __CUDA_ARCH__
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
#endif
  }
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// Inner products sum_k a_k b_k: a plain multiply-add chain for FP64 / FP32;
// for double-float the compensated dot product in the style of Ogita, Rump
// and Oishi ("Dot2"): the running sum s and one compensation term c, each
// product split exactly (FMA) and each addition by TwoSum, renormalised once
// at the end -- about 12 FP32 operations per term instead of 18 for a
// renormalised multiply and add, with the same order of accuracy.
template <typename T>
struct Acc {
  T v;
  __device__ __forceinline__ void init(T a, T b) { v = a * b; }
  __device__ __forceinline__ void add(T a, T b) { v += a * b; }
  __device__ __forceinline__ void add(T a) { v += a; }
  __device__ __forceinline__ T get() const { return v; }
};

template <>
struct Acc<df64> {
  float s, c;
  __device__ __forceinline__ void init(df64 a, df64 b) {
    s = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -s);
    e = __fmaf_rn(a.hi, b.lo, e);
    c = __fmaf_rn(a.lo, b.hi, e);
  }
  __device__ __forceinline__ void add(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df64 t = df_two_sum(s, p);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ void add(df64 a) {
    const df64 t = df_two_sum(s, a.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, a.lo));
  }
  __device__ __forceinline__ df64 get() const { return df_fast_two_sum(s, c); }
};

// Nearest double-float to x and back (these conversions use the FP64 pipe).
__device__ __forceinline__ df64 df_from_double(double x) { return df64(x); }

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a; }

}  // namespace mgdg
