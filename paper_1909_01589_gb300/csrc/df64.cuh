// Double-float arithmetic on the FP32 pipe: a value is hi + lo with two
// floats, |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 executes FP64 at 1/69 of its FP32 rate, so the hot loops of the
// projection run in this representation and reach the accuracy FP64 parity
// needs (relative error ~1e-14) at a fraction of the FP64 pipe time.
//
// Methods (all error-free transformations use round-to-nearest FP32 and the
// fused multiply-add; intrinsics __fadd_rn / __fmul_rn keep the compiler
// from contracting or reassociating them):
//   two_sum        Knuth, The Art of Computer Programming vol. 2 (1969)
//   fast_two_sum   Dekker, "A floating-point technique for extending the
//                  available precision", Numer. Math. 18 (1971)
//   two_prod       the FMA form of Dekker's product (exact a*b - fl(a*b))
//   add / mul      the double-float operations of Dekker (1971) with the
//                  accurate-addition ordering of Hida, Li and Bailey's
//                  double-double library (ARITH 2001)
//   div, sqrt      one Newton correction of an FP32 seed (Karp and
//                  Markstein, ACM TOMS 23 (1997))
//   exp            Tang's table-driven method (ACM TOMS 15 (1989)):
//                  x = (64 n + j) ln2/64 + r, |r| <= ln2/128,
//                  e^x = 2^n 2^(j/64) e^r with a short Taylor series.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Functions with long bodies (exp, log, sqrt, division) are kept out of
// line in device code when LRDMC_DF_OUTLINE is defined, trading call
// overhead for a smaller instruction footprint.
#if defined(__CUDA_ARCH__) && defined(LRDMC_DF_OUTLINE)
#define DF_HEAVY __host__ __device__ __noinline__
#else
#define DF_HEAVY __host__ __device__ __forceinline__
#endif

namespace lrdmc {

struct df {
  float hi, lo;
};

__host__ __device__ __forceinline__ df df_make(float h, float l)
{
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#define DF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) fmaf((a), (b), (c))
#endif

// |a| >= |b| (or a == 0): s + e == a + b exactly.
__host__ __device__ __forceinline__ df fast_two_sum(float a, float b)
{
  float s = DF_ADD(a, b);
  float e = DF_SUB(b, DF_SUB(s, a));
  return df_make(s, e);
}

__host__ __device__ __forceinline__ df two_sum(float a, float b)
{
  float s = DF_ADD(a, b);
  float bb = DF_SUB(s, a);
  float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
  return df_make(s, e);
}

__host__ __device__ __forceinline__ df two_prod(float a, float b)
{
  float p = DF_MUL(a, b);
  float e = DF_FMA(a, b, -p);
  return df_make(p, e);
}

__host__ __device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

__host__ __device__ __forceinline__ df df_add(df a, df b)
{
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  float e = DF_ADD(s.lo, t.hi);
  df u = fast_two_sum(s.hi, e);
  e = DF_ADD(u.lo, t.lo);
  return fast_two_sum(u.hi, e);
}

__host__ __device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Cheaper addition for operands whose sum is used with an absolute error
// of about 2^-44 (|a| + |b|) (distances, Jastrow terms): one two_sum.
__host__ __device__ __forceinline__ df df_add_fast(df a, df b)
{
  df s = two_sum(a.hi, b.hi);
  float e = DF_ADD(s.lo, DF_ADD(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__host__ __device__ __forceinline__ df df_sub_fast(df a, df b) { return df_add_fast(a, df_neg(b)); }

__host__ __device__ __forceinline__ df df_add_f(df a, float b)
{
  df s = two_sum(a.hi, b);
  float e = DF_ADD(s.lo, a.lo);
  return fast_two_sum(s.hi, e);
}

__host__ __device__ __forceinline__ df df_mul(df a, df b)
{
  df p = two_prod(a.hi, b.hi);
  float e = DF_FMA(a.hi, b.lo, p.lo);
  e = DF_FMA(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}

__host__ __device__ __forceinline__ df df_mul_f(df a, float b)
{
  df p = two_prod(a.hi, b);
  float e = DF_FMA(a.lo, b, p.lo);
  return fast_two_sum(p.hi, e);
}

__host__ __device__ __forceinline__ df df_sqr(df a)
{
  df p = two_prod(a.hi, a.hi);
  float e = DF_FMA(DF_ADD(a.hi, a.hi), a.lo, p.lo);
  return fast_two_sum(p.hi, e);
}

// a * b + c
__host__ __device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

__host__ __device__ __forceinline__ float f_rcp_approx(float x)
{
#ifdef __CUDA_ARCH__
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}

__host__ __device__ __forceinline__ float f_rsqrt_approx(float x)
{
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}

// a / b: FP32 quotient q1, then one correction q2 = (a - b q1) / b. The
// remainder a_hi - b_hi q1 comes from one FMA (exact up to one rounding of a
// quantity ~2^-22 a_hi), plus a_lo - b_lo q1 (relative error ~2^-44).
DF_HEAVY df df_div(df a, df b)
{
  float r = f_rcp_approx(b.hi);
  float q1 = DF_MUL(a.hi, r);
  float rem = DF_FMA(-q1, b.hi, a.hi);
  rem = DF_ADD(rem, DF_FMA(-q1, b.lo, a.lo));
  float q2 = DF_MUL(rem, r);
  return fast_two_sum(q1, q2);
}

// 1 / b
__host__ __device__ __forceinline__ df df_rcp(df b) { return df_div(df_make(1.0f, 0.0f), b); }

// sqrt(a), a >= 0: s = a_hi rsqrt(a_hi), corrected by the residual
// a - s^2 (one FMA, plus a_lo) times 1/(2s) (relative error ~2^-44).
DF_HEAVY df df_sqrt(df a)
{
  if (!(a.hi > 0.0f)) return df_make(0.0f, 0.0f);
  float y = f_rsqrt_approx(a.hi);
  float s = DF_MUL(a.hi, y);
  float res = DF_ADD(DF_FMA(-s, s, a.hi), a.lo);
  float c = DF_MUL(res, DF_MUL(0.5f, y));
  return fast_two_sum(s, c);
}

// Constants of the exponential: ln2/64 split in two floats and 64/ln2.
struct ExpConsts {
  float ln2_64_hi, ln2_64_lo;
  float inv_ln2_64;
  float pad;
};

// Table of 2^(j/64), j = 0..63, as double-floats (x = hi, y = lo).
struct ExpTable {
  ExpConsts K;
  float2 t[64];
};

// e^a for a in about [-87, 88]; 0 below, +inf above. tab: the table.
DF_HEAVY df df_exp(df a, const ExpConsts& K, const float2* tab)
{
  if (a.hi < -87.0f) return df_make(0.0f, 0.0f);
  if (a.hi > 88.0f) return df_make(INFINITY, 0.0f);
  float mf = rintf(DF_MUL(a.hi, K.inv_ln2_64));
  int m = (int)mf;
  // r = a - m ln2/64, exact product of the float m with the split constant
  df p = two_prod(mf, K.ln2_64_hi);
  p.lo = DF_FMA(mf, K.ln2_64_lo, p.lo);
  df r = df_sub(a, p);
  // e^r = 1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720), |r| <= ln2/128
  float x = r.hi;
  float tail = DF_FMA(x, 1.0f / 720.0f, 1.0f / 120.0f);
  tail = DF_FMA(x, tail, 1.0f / 24.0f);
  tail = DF_FMA(x, tail, 1.0f / 6.0f);
  tail = DF_MUL(DF_MUL(DF_MUL(x, x), x), tail);
  df r2 = df_sqr(r);
  r2.hi = DF_MUL(r2.hi, 0.5f);
  r2.lo = DF_MUL(r2.lo, 0.5f);
  df e = df_add_fast(r, r2);  // r2 = r^2/2 <= |r| ln2/256: no cancellation
  e = df_add_f(e, tail);
  e = df_add_f(e, 1.0f);
  int j = m & 63;
  int n = (m - j) >> 6;
  const float2 tj = tab[j];
  e = df_mul(e, df_make(tj.x, tj.y));
  // scale by 2^n in two steps so that intermediate factors stay normal
  int n1 = n >> 1, n2 = n - n1;
#ifdef __CUDA_ARCH__
  float s1 = __int_as_float((n1 + 127) << 23), s2 = __int_as_float((n2 + 127) << 23);
#else
  float s1 = ldexpf(1.0f, n1), s2 = ldexpf(1.0f, n2);
#endif
  return df_make(DF_MUL(DF_MUL(e.hi, s1), s2), DF_MUL(DF_MUL(e.lo, s1), s2));
}

// log(a), a > 0: FP32 seed y0, then one Newton step y0 + a e^(-y0) - 1.
DF_HEAVY df df_log(df a, const ExpConsts& K, const float2* tab)
{
  float y0 = logf(a.hi);
  df t = df_mul(a, df_exp(df_make(-y0, 0.0f), K, tab));
  t = df_add_f(t, -1.0f);
  return df_add_f(t, y0);
}

// sin(pi x) and cos(pi x) for a double-float x in about [0, 2]: x = (n +
// r)/2 with integer n and |r| <= 1/2, theta = r pi/2 (|theta| <= pi/4),
// Taylor series of sin and cos in theta^2 to degree 15 and 16 (truncation
// below 5e-16), then the quadrant n mod 4. inv_fact[k] = 1/k! and half_pi
// as double-floats.
DF_HEAVY void df_sincospi(df x, const df* inv_fact, df half_pi, df* s_out, df* c_out)
{
  df t = df_make(DF_ADD(x.hi, x.hi), DF_ADD(x.lo, x.lo));
  float n = rintf(t.hi);
  df r = df_add_f(t, -n);
  df th = df_mul(r, half_pi);
  df z = df_sqr(th);
  df ps = df_neg(inv_fact[15]);
  for (int j = 6; j >= 0; --j) {
    df cj = inv_fact[2 * j + 1];
    ps = df_add_fast(df_mul(ps, z), (j & 1) ? df_neg(cj) : cj);
  }
  df sn = df_mul(th, ps);
  df pc = inv_fact[16];
  for (int j = 7; j >= 0; --j) {
    df cj = inv_fact[2 * j];
    pc = df_add_fast(df_mul(pc, z), (j & 1) ? df_neg(cj) : cj);
  }
  const int q = ((int)n) & 3;
  df so = sn, co = pc;
  if (q == 1) { so = pc; co = df_neg(sn); }
  else if (q == 2) { so = df_neg(sn); co = df_neg(pc); }
  else if (q == 3) { so = df_neg(pc); co = sn; }
  *s_out = so;
  *c_out = co;
}

// Conversions (each touches the FP64 pipe: use them outside inner loops).
__host__ __device__ __forceinline__ df df_from_double(double d)
{
  float h = (float)d;
  float l = (float)(d - (double)h);
  return df_make(h, l);
}

__host__ __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace lrdmc
