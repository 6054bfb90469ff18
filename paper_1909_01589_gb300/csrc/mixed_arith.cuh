// Arithmetic traits for the evaluation kernels that run on the FP32 pipe.
//
// Ar<df>    double-float (hi + lo), about 48 significant bits: the
//           LRDMC_PRECISION_DF64 mode, accurate to FP64 parity.
// Ar<float> plain IEEE single precision: the LRDMC_PRECISION_FP32 mode
//           (mixed precision: the evaluation in FP32, while inverse Slater
//           matrices, Sherman-Morrison updates, weights and reconfiguration
//           stay in FP64).
// Both expose the same operation names so one templated evaluation serves
// both modes. Constants are kept as double-floats; Ar<float> reads their
// high parts.
#pragma once
#include "df64.cuh"

namespace lrdmc {

template <class R>
struct Ar;

template <>
struct Ar<df> {
  typedef df T;
  static __device__ __forceinline__ df zero() { return df_make(0.0f, 0.0f); }
  static __device__ __forceinline__ df one() { return df_make(1.0f, 0.0f); }
  static __device__ __forceinline__ df inf() { return df_make(INFINITY, 0.0f); }
  static __device__ __forceinline__ df c(const df& x) { return x; }
  static __device__ __forceinline__ df store(const df& x) { return x; }
  static __device__ __forceinline__ df from_double(double x) { return df_from_double(x); }
  static __device__ __forceinline__ double to_double(df x) { return df_to_double(x); }
  // add and sub use the one-two_sum addition (error ~2^-44 of |a| + |b|):
  // every sum the evaluation forms is compared against the FP64 reference
  // relative to the magnitude of its terms, which this bound respects; the
  // primitives that need the exact-cancellation form (the exp range
  // reduction) call df_add / df_sub directly
  static __device__ __forceinline__ df add(df a, df b) { return df_add_fast(a, b); }
  static __device__ __forceinline__ df add_fast(df a, df b) { return df_add_fast(a, b); }
  static __device__ __forceinline__ df sub(df a, df b) { return df_sub_fast(a, b); }
  static __device__ __forceinline__ df sub_fast(df a, df b) { return df_sub_fast(a, b); }
  static __device__ __forceinline__ df add_f(df a, float b) { return df_add_f(a, b); }
  static __device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }
  static __device__ __forceinline__ df mul_f(df a, float b) { return df_mul_f(a, b); }
  static __device__ __forceinline__ df sqr(df a) { return df_sqr(a); }
  static __device__ __forceinline__ df div(df a, df b) { return df_div(a, b); }
  static __device__ __forceinline__ df rcp(df a) { return df_rcp(a); }
  static __device__ __forceinline__ df sqrt(df a) { return df_sqrt(a); }
  static __device__ __forceinline__ df neg(df a) { return df_neg(a); }
  static __device__ __forceinline__ df half(df a) { return df_make(0.5f * a.hi, 0.5f * a.lo); }
  static __device__ __forceinline__ df exp(df a, const ExpConsts& K, const float2* tab) { return df_exp(a, K, tab); }
  static __device__ __forceinline__ df log(df a, const ExpConsts& K, const float2* tab) { return df_log(a, K, tab); }
  static __device__ __forceinline__ float approx(df a) { return a.hi; }
  static __device__ __forceinline__ bool positive(df a) { return a.hi > 0.0f; }
  static __device__ __forceinline__ bool lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
  static __device__ __forceinline__ df shfl(df v, int src)
  {
    return df_make(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
  }
  static __device__ __forceinline__ df shfl_up(df v, int o)
  {
    return df_make(__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o));
  }
  static __device__ __forceinline__ df shfl_xor(df v, int o)
  {
    return df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
  }
};

template <>
struct Ar<float> {
  typedef float T;
  static __device__ __forceinline__ float zero() { return 0.0f; }
  static __device__ __forceinline__ float one() { return 1.0f; }
  static __device__ __forceinline__ float inf() { return INFINITY; }
  static __device__ __forceinline__ float c(const df& x) { return x.hi; }
  static __device__ __forceinline__ df store(float x) { return df_make(x, 0.0f); }
  static __device__ __forceinline__ float from_double(double x) { return (float)x; }
  static __device__ __forceinline__ double to_double(float x) { return (double)x; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float add_fast(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float sub_fast(float a, float b) { return a - b; }
  static __device__ __forceinline__ float add_f(float a, float b) { return a + b; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float mul_f(float a, float b) { return a * b; }
  static __device__ __forceinline__ float sqr(float a) { return a * a; }
  static __device__ __forceinline__ float div(float a, float b) { return a / b; }
  static __device__ __forceinline__ float rcp(float a) { return 1.0f / a; }
  static __device__ __forceinline__ float sqrt(float a) { return sqrtf(a); }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float half(float a) { return 0.5f * a; }
  static __device__ __forceinline__ float exp(float a, const ExpConsts&, const float2*) { return expf(a); }
  static __device__ __forceinline__ float log(float a, const ExpConsts&, const float2*) { return logf(a); }
  static __device__ __forceinline__ float approx(float a) { return a; }
  static __device__ __forceinline__ bool positive(float a) { return a > 0.0f; }
  static __device__ __forceinline__ bool lt(float a, float b) { return a < b; }
  static __device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  static __device__ __forceinline__ float shfl_up(float v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
  static __device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
};

}  // namespace lrdmc
