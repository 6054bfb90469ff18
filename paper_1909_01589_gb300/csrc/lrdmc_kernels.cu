// CUDA kernels (sm_103a) of the LRDMC hot path.
//
// One warp owns one walker at a time. Shared memory holds the walker's
// positions, inverse Slater matrices, lattice rotation, the P jump rates of
// its cached evaluation, per-electron work vectors and (double-float mode)
// the electron-pair and electron-nucleus caches of the evaluation; the MO
// coefficients are staged once per block. The lanes split the P lattice
// moves of an evaluation, the electrons of the local energy, the orbitals
// and matrix entries of the Sherman-Morrison update, and the rows of the
// Gauss-Jordan inverse. The evaluation runs in IEEE double, in double-float
// on the FP32 pipe, or in single precision (the kernels' template argument
// carries the arithmetic and whether the neural pair term is set); inverses,
// updates, weights and reconfiguration stay in IEEE double. Kernels:
//   k_init      start configurations -> inverses, first rotation
//   k_eval_all  evaluate every walker (after a change of lattice)
//   k_interval  one interval tau of continuous-time projection per walker,
//               walkers fetched dynamically by the warps (ragged jump counts)
//   k_comb_sums, k_comb_parents  reconfiguration: running weight sums, comb
//               parents, trace entry, order of the next interval
//   k_evaluate  stateless evaluation of given configurations (and the
//               variant with static scratch, k_evaluate_static)
//   k_base_terms  gradients and local energies without the neural term
// The population is double-buffered: k_interval gathers the record of
// parent[s] from the source buffer, so reconfiguration needs no copy pass.
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <mutex>

#include "lrdmc_internal.h"
#include "mixed_arith.cuh"

namespace lrdmc {

#define FULL_MASK 0xffffffffu

// ----------------------------------------------------------------------------
// Counter-based random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
// SC'11), key (seed, 0), counter (slot, interval, iteration, tag).
// Inlining of the large, once-per-jump or rarely executed parts of the
// interval loop (tuning switches; the default inlines everything):
//   LRDMC_NOINLINE_COLD  the Gauss-Jordan recompute (every few intervals)
//   LRDMC_NOINLINE_JUMP  the Sherman-Morrison update and the new rotation
//   LRDMC_NOINLINE_EL    the local-energy parts of an evaluation
#ifdef LRDMC_NOINLINE_COLD
#define LRDMC_COLD __noinline__
#else
#define LRDMC_COLD
#endif
#ifdef LRDMC_NOINLINE_JUMP
#define LRDMC_JUMP __noinline__
#define LRDMC_JUMP_INLINE __noinline__
#else
#define LRDMC_JUMP
#define LRDMC_JUMP_INLINE __forceinline__
#endif
#ifdef LRDMC_NOINLINE_EL
#define LRDMC_EL __noinline__
#else
#define LRDMC_EL
#endif

// ----------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

__device__ __forceinline__ double to_u01(uint64_t bits)
{
  return ((double)(bits >> 12) + 0.5) * 0x1.0p-52;
}

__device__ __forceinline__ void draw_uniforms(uint64_t seed, uint64_t slot, uint64_t k, uint64_t m,
                                              uint64_t tag, double u[4])
{
  uint64_t c[4] = {slot, k, m, tag};
  philox4x64_10(c, seed, 0ull);
#pragma unroll
  for (int j = 0; j < 4; ++j) u[j] = to_u01(c[j]);
}

// The same uniform ((bits >> 12) + 1/2) 2^-52 = N 2^-53, N = 2 (bits >> 12)
// + 1 < 2^53, as a double-float built with integer operations only (no FP64
// pipe): the 24 bits below N's leading bit give hi exactly, the remaining
// low bits (at most 29) give lo, so the relative error is below 2^-47 for
// every uniform, however small.
__device__ __forceinline__ df df_u01(uint64_t bits)
{
  const uint64_t N = ((bits >> 12) << 1) | 1ull;
  const int sh = (63 - __clzll((long long)N)) - 23;  // shift that leaves 24 bits
  const uint64_t top = sh >= 0 ? (N >> sh) : (N << (-sh));
  const uint64_t rem = sh > 0 ? (N - (top << sh)) : 0ull;
  const float hi = (float)(uint32_t)top * __int_as_float((127 + sh - 53) << 23);
  const float lo = (float)(uint32_t)rem * 0x1.0p-53f;
  return fast_two_sum(hi, lo);
}

// A single-precision uniform from the top 24 bits, in (0, 1).
__device__ __forceinline__ float f_u01(uint64_t bits)
{
  return ((float)(uint32_t)(bits >> 40) + 0.5f) * 0x1.0p-24f;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src)
{
  uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src), hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
  return ((uint64_t)hi << 32) | lo;
}

// Uniformly random rotation (Shoemake's unit quaternion from three uniforms).
__device__ void rotation_matrix(double u1, double u2, double u3, double* R)
{
  double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
  double sa, ca, sb, cb;
  sincospi(2.0 * u2, &sa, &ca);
  sincospi(2.0 * u3, &sb, &cb);
  double x = s1 * sa, y = s1 * ca, z = s2 * sb, w = s2 * cb;
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - z * w);       R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);       R[7] = 2.0 * (y * z + x * w);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// The same rotation from the three uniforms of bits[0..2], with the work
// spread over the warp: lanes 0-3 evaluate sqrt(1-u1), sqrt(u1),
// sincospi(2 u2) and sincospi(2 u3), lanes 0-8 then form one entry of R
// each. FP64 mode: IEEE double (the same operations as rotation_matrix).
// DF64 mode: double-float (the FP32 pipe), accurate to ~1e-15. FP32 mode:
// single precision. All lanes must call it; R (double) goes to shared memory.
template <int PREC>
__device__ LRDMC_JUMP_INLINE void rotation_matrix_warp(const uint64_t* bits, double* R, int lane, const SysDev& S)
{
  double x, y, z, w;
  if (PREC == LRDMC_PRECISION_FP32) {
    float a = 0.0f, c = 0.0f;
    if (lane == 0) a = sqrtf(1.0f - f_u01(bits[0]));
    else if (lane == 1) a = sqrtf(f_u01(bits[0]));
    else if (lane == 2) sincospif(2.0f * f_u01(bits[1]), &a, &c);
    else if (lane == 3) sincospif(2.0f * f_u01(bits[2]), &a, &c);
    float s1 = __shfl_sync(FULL_MASK, a, 0), s2 = __shfl_sync(FULL_MASK, a, 1);
    float sa = __shfl_sync(FULL_MASK, a, 2), ca = __shfl_sync(FULL_MASK, c, 2);
    float sb = __shfl_sync(FULL_MASK, a, 3), cb = __shfl_sync(FULL_MASK, c, 3);
    float qx = s1 * sa, qy = s1 * ca, qz = s2 * sb, qw = s2 * cb;
    float v = 0.0f;
    switch (lane) {
      case 0: v = 1.0f - 2.0f * (qy * qy + qz * qz); break;
      case 1: v = 2.0f * (qx * qy - qz * qw); break;
      case 2: v = 2.0f * (qx * qz + qy * qw); break;
      case 3: v = 2.0f * (qx * qy + qz * qw); break;
      case 4: v = 1.0f - 2.0f * (qx * qx + qz * qz); break;
      case 5: v = 2.0f * (qy * qz - qx * qw); break;
      case 6: v = 2.0f * (qx * qz - qy * qw); break;
      case 7: v = 2.0f * (qy * qz + qx * qw); break;
      case 8: v = 1.0f - 2.0f * (qx * qx + qy * qy); break;
      default: break;
    }
    if (lane < 9) R[lane] = (double)v;
    return;
  }
  if (PREC == LRDMC_PRECISION_DF64) {
    // lanes 0 and 1: sqrt(1 - u1) and sqrt(u1); lanes 2 and 3: sincospi of
    // 2 u2 and 2 u3 - one pass each, the operand chosen per lane
    df a = df_make(0.0f, 0.0f), c = df_make(0.0f, 0.0f);
    if (lane < 2) {
      const df u = df_u01(bits[0]);
      a = df_sqrt(lane == 0 ? df_add_f(df_neg(u), 1.0f) : u);
    } else if (lane < 4) {
      df_sincospi(df_mul_f(df_u01(bits[lane - 1]), 2.0f), S.D.inv_fact, S.D.half_pi, &a, &c);
    }
    typedef Ar<df> A;
    df s1 = A::shfl(a, 0), s2 = A::shfl(a, 1), sa = A::shfl(a, 2), ca = A::shfl(c, 2);
    df sb = A::shfl(a, 3), cb = A::shfl(c, 3);
    const df q[4] = {df_mul(s1, sa), df_mul(s1, ca), df_mul(s2, sb), df_mul(s2, cb)};  // x, y, z, w
    // entry (row, col) = lane: delta + 2 (s1 q[a] q[b] + s2 q[c] q[d]); the
    // operand indices and signs of the nine entries, packed per lane
    //   R00 = 1 - 2(yy + zz)  R01 = 2(xy - zw)  R02 = 2(xz + yw)
    //   R10 = 2(xy + zw)  R11 = 1 - 2(xx + zz)  R12 = 2(yz - xw)
    //   R20 = 2(xz - yw)  R21 = 2(yz + xw)  R22 = 1 - 2(xx + yy)
    const int L = lane < 9 ? lane : 0;
    const unsigned long long ka = 0x10100001ull, kb = 0x22201211ull;
    const unsigned long long kc = 0x101022122ull, kd = 0x133323332ull;
    const unsigned ia = (ka >> (4 * L)) & 0xF, ib = (kb >> (4 * L)) & 0xF;
    const unsigned ic = (kc >> (4 * L)) & 0xF, id = (kd >> (4 * L)) & 0xF;
    const bool diag = L == 0 || L == 4 || L == 8;
    const bool minus2 = L == 1 || L == 5 || L == 6;
    auto pick = [&](unsigned k) { return k == 0 ? q[0] : k == 1 ? q[1] : k == 2 ? q[2] : q[3]; };
    df t1 = df_mul(pick(ia), pick(ib)), t2 = df_mul(pick(ic), pick(id));
    df v;
    if (diag) v = df_add_f(df_mul_f(df_add(t1, t2), -2.0f), 1.0f);
    else v = df_mul_f(minus2 ? df_sub(t1, t2) : df_add(t1, t2), 2.0f);
    if (lane < 9) R[lane] = df_to_double(v);
    return;
  }
  {
    double a = 0.0, c = 0.0;
    const double u1 = to_u01(bits[0]);
    if (lane == 0) a = sqrt(1.0 - u1);
    else if (lane == 1) a = sqrt(u1);
    else if (lane == 2) sincospi(2.0 * to_u01(bits[1]), &a, &c);
    else if (lane == 3) sincospi(2.0 * to_u01(bits[2]), &a, &c);
    double s1 = __shfl_sync(FULL_MASK, a, 0), s2 = __shfl_sync(FULL_MASK, a, 1);
    double sa = __shfl_sync(FULL_MASK, a, 2), ca = __shfl_sync(FULL_MASK, c, 2);
    double sb = __shfl_sync(FULL_MASK, a, 3), cb = __shfl_sync(FULL_MASK, c, 3);
    x = s1 * sa; y = s1 * ca; z = s2 * sb; w = s2 * cb;
  }
  double v = 0.0;
  switch (lane) {
    case 0: v = 1.0 - 2.0 * (y * y + z * z); break;
    case 1: v = 2.0 * (x * y - z * w); break;
    case 2: v = 2.0 * (x * z + y * w); break;
    case 3: v = 2.0 * (x * y + z * w); break;
    case 4: v = 1.0 - 2.0 * (x * x + z * z); break;
    case 5: v = 2.0 * (y * z - x * w); break;
    case 6: v = 2.0 * (x * z - y * w); break;
    case 7: v = 2.0 * (y * z + x * w); break;
    case 8: v = 1.0 - 2.0 * (x * x + y * y); break;
    default: break;
  }
  if (lane < 9) R[lane] = v;
}

// ----------------------------------------------------------------------------
// Warp helpers.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

// Chunked inclusive scan of T[0..P): chunks of 32 in order, a Hillis-Steele
// scan inside each chunk plus the running total of the previous chunks.
// Returns the total (identical in every lane). When pick != nullptr, *pick
// receives the smallest c with target < C_c (or -1), and *last the largest c
// with T_c > 0 (or -1).
__device__ double warp_scan(const double* T, int P, int lane, double target, int* pick, int* last)
{
  double carry = 0.0;
  int p = -1, lp = -1;
  for (int base = 0; base < P; base += 32) {
    int c = base + lane;
    double t = (c < P) ? T[c] : 0.0;
    double v = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double y = __shfl_up_sync(FULL_MASK, v, o);
      if (lane >= o) v += y;
    }
    double C = carry + v;
    if (pick) {
      unsigned hit = __ballot_sync(FULL_MASK, (c < P) && (target < C));
      if (p < 0 && hit) p = base + __ffs(hit) - 1;
      unsigned pos = __ballot_sync(FULL_MASK, (c < P) && (t > 0.0));
      if (pos) lp = base + 31 - __clz(pos);
    }
    carry = __shfl_sync(FULL_MASK, C, 31);
  }
  if (pick) { *pick = p; *last = lp; }
  return carry;
}

// ----------------------------------------------------------------------------
// Atomic orbitals: chi = S(d) R(|d|), d = r - R_centre, S a real solid
// harmonic of degree l, R Slater r^m exp(-zeta r) or a Gaussian contraction.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double int_pow(double r, int m)
{
  double p = 1.0;
  for (int j = 0; j < m; ++j) p *= r;
  return p;
}

// Radial value R, R'/r and R''. e is exp(-zeta r) for Slater shells.
__device__ __forceinline__ void radial(const ShellDev& sh, double r, double e, double& R, double& R1,
                                       double& R2, bool der)
{
  if (sh.kind == 0) {
    double pw = (sh.m_int >= 0) ? int_pow(r, sh.m_int) : pow(r, sh.m);
    R = pw * e;
    if (der) {
      double t = sh.m / r - sh.zeta;
      R1 = t * R / r;
      R2 = (t * t - sh.m / (r * r)) * R;
    }
  } else {
    double r2 = r * r;
    R = 0.0; R1 = 0.0; R2 = 0.0;
    for (int p = 0; p < sh.n_prim; ++p) {
      double al = sh.alpha[p];
      double g = sh.coef[p] * exp(-al * r2);
      R += g;
      if (der) {
        R1 += -2.0 * al * g;
        R2 += (4.0 * al * al * r2 - 2.0 * al) * g;
      }
    }
  }
}

// Solid harmonics of degree l at d and their gradients.
__device__ __forceinline__ int solid(int l, const double d[3], double S[5], double gS[5][3], bool der)
{
  if (l == 0) {
    S[0] = 1.0;
    if (der) { gS[0][0] = gS[0][1] = gS[0][2] = 0.0; }
    return 1;
  }
  if (l == 1) {
    S[0] = d[0]; S[1] = d[1]; S[2] = d[2];
    if (der) {
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int k = 0; k < 3; ++k) gS[f][k] = (f == k) ? 1.0 : 0.0;
    }
    return 3;
  }
  S[0] = d[0] * d[1];
  S[1] = d[1] * d[2];
  S[2] = d[2] * d[0];
  S[3] = d[0] * d[0] - d[1] * d[1];
  S[4] = 2.0 * d[2] * d[2] - d[0] * d[0] - d[1] * d[1];
  if (der) {
    gS[0][0] = d[1];        gS[0][1] = d[0];        gS[0][2] = 0.0;
    gS[1][0] = 0.0;         gS[1][1] = d[2];        gS[1][2] = d[1];
    gS[2][0] = d[2];        gS[2][1] = 0.0;         gS[2][2] = d[0];
    gS[3][0] = 2.0 * d[0];  gS[3][1] = -2.0 * d[1]; gS[3][2] = 0.0;
    gS[4][0] = -2.0 * d[0]; gS[4][1] = -2.0 * d[1]; gS[4][2] = 4.0 * d[2];
  }
  return 5;
}

// Sum_mu v[mu] chi_mu(p): the determinant ratio when v is the projected
// inverse column of the moving electron.
__device__ double ao_dot(const SysDev& S, const double* v, double px, double py, double pz)
{
  double acc = 0.0;
  int prev_c = -1;
  double d[3] = {0, 0, 0}, r = 0.0, e = 0.0;
  for (int q = 0; q < S.n_shell; ++q) {
    const ShellDev& sh = S.sh[q];
    if (sh.center != prev_c) {
      prev_c = sh.center;
      d[0] = px - S.nuc[prev_c][0];
      d[1] = py - S.nuc[prev_c][1];
      d[2] = pz - S.nuc[prev_c][2];
      r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    if (sh.kind == 0 && !sh.same_exp) e = exp(-sh.zeta * r);
    double R, R1, R2, Sv[5], gS[5][3];
    radial(sh, r, e, R, R1, R2, false);
    int nf = solid(sh.l, d, Sv, gS, false);
    double part = 0.0;
    for (int f = 0; f < nf; ++f) part += v[sh.ao_offset + f] * Sv[f];
    acc += part * R;
  }
  return acc;
}

// Sum_mu v[mu] chi_mu, grad chi_mu, lap chi_mu at p.
__device__ void ao_dot_der(const SysDev& S, const double* v, const double* p, double& val,
                           double g[3], double& lap)
{
  val = 0.0; g[0] = g[1] = g[2] = 0.0; lap = 0.0;
  int prev_c = -1;
  double d[3] = {0, 0, 0}, r = 0.0, e = 0.0;
  for (int q = 0; q < S.n_shell; ++q) {
    const ShellDev& sh = S.sh[q];
    if (sh.center != prev_c) {
      prev_c = sh.center;
      d[0] = p[0] - S.nuc[prev_c][0];
      d[1] = p[1] - S.nuc[prev_c][1];
      d[2] = p[2] - S.nuc[prev_c][2];
      r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    if (sh.kind == 0 && !sh.same_exp) e = exp(-sh.zeta * r);
    double R, R1, R2, Sv[5], gS[5][3];
    radial(sh, r, e, R, R1, R2, true);
    int nf = solid(sh.l, d, Sv, gS, true);
    double radlap = R2 + 2.0 * (sh.l + 1) * R1;
    for (int f = 0; f < nf; ++f) {
      double c = v[sh.ao_offset + f];
      val += c * Sv[f] * R;
#pragma unroll
      for (int k = 0; k < 3; ++k) g[k] += c * (R * gS[f][k] + Sv[f] * R1 * d[k]);
      lap += c * Sv[f] * radlap;
    }
  }
}

// chi_mu(p) for all AOs into out[n_ao].
__device__ void ao_values(const SysDev& S, const double* p, double* out)
{
  int prev_c = -1;
  double d[3] = {0, 0, 0}, r = 0.0, e = 0.0;
  for (int q = 0; q < S.n_shell; ++q) {
    const ShellDev& sh = S.sh[q];
    if (sh.center != prev_c) {
      prev_c = sh.center;
      d[0] = p[0] - S.nuc[prev_c][0];
      d[1] = p[1] - S.nuc[prev_c][1];
      d[2] = p[2] - S.nuc[prev_c][2];
      r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    if (sh.kind == 0 && !sh.same_exp) e = exp(-sh.zeta * r);
    double R, R1, R2, Sv[5], gS[5][3];
    radial(sh, r, e, R, R1, R2, false);
    int nf = solid(sh.l, d, Sv, gS, false);
    for (int f = 0; f < nf; ++f) out[sh.ao_offset + f] = Sv[f] * R;
  }
}

// ----------------------------------------------------------------------------
// Jastrow factor.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int spin_of(const SysDev& S, int i) { return i < S.n_up ? 0 : 1; }

// Neural pair term, tabulated: the cell of r (uniform in sqrt(r) on
// [0, r_cut)) holds r_k, 1/w_k and c_0..c_5; g = sum_q c_q t^q with
// t = (r - r_k)/w_k (Horner), 0 from r_cut on. The cell index is taken in
// single precision: next to a cell edge either neighbour's polynomial
// agrees with the other to second order at the edge, so the choice is
// immaterial.
__device__ __forceinline__ int nj_ch_ee(const SysDev& S, int i, int j) { return spin_of(S, i) == spin_of(S, j) ? 0 : 1; }

__device__ __forceinline__ const double* nj_cell(const SysDev& S, int c, double r)
{
  int k = (int)(sqrtf((float)r) * S.nj_scale_f[c]);
  k = min(max(k, 0), S.nj_cells - 1);
  return S.nj_tab + ((size_t)c * S.nj_cells + k) * 8;
}

__device__ __forceinline__ double nj_value(const SysDev& S, int c, double r)
{
  if (!(r < S.nj_rcut[c])) return 0.0;
  const double* e = nj_cell(S, c, r);
  const double t = (r - __ldg(e)) * __ldg(e + 1);
  double v = __ldg(e + 7);
#pragma unroll
  for (int q = 6; q >= 2; --q) v = fma(v, t, __ldg(e + q));
  return v;
}

__device__ __forceinline__ void nj_value3(const SysDev& S, int c, double r, double& g, double& g1, double& g2)
{
  g = 0.0; g1 = 0.0; g2 = 0.0;
  if (!(r < S.nj_rcut[c])) return;
  const double* e = nj_cell(S, c, r);
  const double iw = __ldg(e + 1), t = (r - __ldg(e)) * iw;
  const double c0 = __ldg(e + 2), c1 = __ldg(e + 3), c2 = __ldg(e + 4), c3 = __ldg(e + 5), c4 = __ldg(e + 6),
               c5 = __ldg(e + 7);
  g = c0 + t * (c1 + t * (c2 + t * (c3 + t * (c4 + t * c5))));
  const double d1 = c1 + t * (2.0 * c2 + t * (3.0 * c3 + t * (4.0 * c4 + t * 5.0 * c5)));
  const double d2 = 2.0 * c2 + t * (6.0 * c3 + t * (12.0 * c4 + t * 20.0 * c5));
  g1 = d1 * iw;
  g2 = d2 * iw * iw;
}

// sum_{j != i} u_ee(|p - r_j|) + sum_I u_en(|p - R_I|).
template <bool NJ>
__device__ double jastrow_terms(const SysDev& S, const double* sx, int i, double px, double py,
                                double pz)
{
  double acc = 0.0;
  const int si = spin_of(S, i);
  for (int j = 0; j < S.N; ++j) {
    if (j == i) continue;
    double dx = px - sx[3 * j], dy = py - sx[3 * j + 1], dz = pz - sx[3 * j + 2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double c = (spin_of(S, j) == si) ? S.c_par : S.c_anti;
    acc += c * r / (1.0 + S.b_ee * r);
    if (NJ) acc += nj_value(S, nj_ch_ee(S, i, j), r);
  }
  for (int I = 0; I < S.n_nuc; ++I) {
    double dx = px - S.nuc[I][0], dy = py - S.nuc[I][1], dz = pz - S.nuc[I][2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    acc -= S.en_b1[I] * r / (1.0 + S.en_b2 * r);
    if (NJ) acc += nj_value(S, 2 + S.nj_species[I], r);
  }
  return acc;
}

// p at a point: nearest heavy nucleus, Eq. 3 (Gaussian) or Eq. 2 (Pade).
__device__ __forceinline__ double p_weight(const SysDev& S, const LatDev& L, double px, double py,
                                           double pz)
{
  double best = INFINITY;
  for (int I = 0; I < S.n_nuc; ++I) {
    if (!S.heavy[I]) continue;
    double dx = px - S.nuc[I][0], dy = py - S.nuc[I][1], dz = pz - S.nuc[I][2];
    double d2 = dx * dx + dy * dy + dz * dz;
    best = fmin(best, d2);
  }
  if (L.pkind == 0) return exp(-best * L.p_coef);
  return 1.0 / (1.0 + L.p_coef * best);
}

// ----------------------------------------------------------------------------
// Per-warp shared-memory views.
// ----------------------------------------------------------------------------
struct WarpMem {
  double* x;    // [N][3]
  double* A;    // inverse up [nu][nu] then down [nd][nd]
  double* R;    // [9]
  double* T;    // [P_max]
  double* v;    // [N][n_ao]
  double* Ssum; // [N]
  df* xd;       // [N][3]      double-float copies for the DF64 evaluation
  df* vd;       // [N][n_ao]   (aliases v)
  df* Sd;       // [N]         (aliases Ssum)
  df* Rd;       // [12]
  df* pc;       // [n_pc][pcw] pair cache: |r_a - r_b|^2, e_k . (r_a - r_b) (a < b) and, with
                //   pcw = 8, the pair's Jastrow terms u, u'/r, u'' + 2u'/r and 1/r
  df* enc;      // [N][n_nuc][8] electron-nucleus cache: d, |d|^2, e_k . d
  double* scr;  // scratch
  int n_pc;     // pairs in the cache (0: no cache)
  int pcw;      // double-floats per cached pair
};

__device__ __forceinline__ WarpMem warp_mem(const Layout& Lo, const SysDev& S, double* base)
{
  WarpMem m;
  m.x = base;
  m.A = m.x + 3 * Lo.N;
  m.R = m.A + Lo.nu * Lo.nu + Lo.nd * Lo.nd;
  m.T = m.R + 12;
  m.v = m.T + Lo.P_max;
  m.Ssum = m.v + Lo.N * S.n_ao;
  // the FP64 evaluation uses v and Ssum, the FP32-pipe evaluations their
  // double-float images vd and Sd: one precision runs per launch, so they
  // share the storage
  m.vd = reinterpret_cast<df*>(m.v);
  m.Sd = reinterpret_cast<df*>(m.Ssum);
  m.xd = reinterpret_cast<df*>(m.Ssum + Lo.N);
  m.Rd = m.xd + 3 * Lo.N;
  m.pc = m.Rd + 12;
  m.enc = m.pc + Lo.pcw * Lo.n_pc;
  m.scr = reinterpret_cast<double*>(m.enc + (Lo.enc ? 8 * Lo.N * S.n_nuc : 0));
  m.n_pc = Lo.n_pc;
  m.pcw = Lo.pcw;
  return m;
}

// Block-shared tables: MO coefficients (double, then a float copy), then
// the 2^(j/64) table.
struct BlockMem {
  double* C;
  df* Cd;
  float* Cf;
  float2* tab;
};

__device__ __forceinline__ BlockMem block_mem(const SysDev& S, double* smem)
{
  BlockMem b;
  const int nc = S.n_ao * S.n_mo;
  b.C = smem;
  b.Cd = reinterpret_cast<df*>(smem + nc);
  b.Cf = reinterpret_cast<float*>(smem + 2 * nc);
  b.tab = reinterpret_cast<float2*>(smem + 2 * nc + (nc + 1) / 2);
  return b;
}

// ----------------------------------------------------------------------------
// Inverse Slater matrix of one spin block by Gauss-Jordan elimination with
// partial pivoting (warp-cooperative). A[l][m] = phi_m(r_l); the inverse is
// stored as Ainv[m][l]. Returns false for a singular matrix (below).
// ----------------------------------------------------------------------------
// With resid (nullable), first the residual of the inverse the block holds
// (the Sherman-Morrison-updated one): max |sum_m A[l][m] Ainv[m][q] -
// delta_lq| over the block, where A is the Slater matrix at the current
// positions; *resid becomes the larger of itself and that residual (the
// same value in every lane).
__device__ LRDMC_COLD bool warp_inverse(const SysDev& S, const double* sC, const double* sx, int spin,
                             double* Ainv, double* scr, int lane, double* resid = nullptr)
{
  const int n = spin == 0 ? S.n_up : S.n_dn;
  if (n == 0) return true;
  const int off = spin == 0 ? 0 : S.n_up;
  const int w2 = 2 * n;
  double* M = scr;                 // [n][2n]
  double* chi = scr + n * w2;      // [n][n_ao]
  for (int l = lane; l < n; l += 32) {
    ao_values(S, &sx[3 * (off + l)], &chi[l * S.n_ao]);
    for (int m = 0; m < n; ++m) {
      double a = 0.0;
      for (int mu = 0; mu < S.n_ao; ++mu) a += sC[mu * S.n_mo + m] * chi[l * S.n_ao + mu];
      M[l * w2 + m] = a;
      M[l * w2 + n + m] = (m == l) ? 1.0 : 0.0;
    }
  }
  __syncwarp();
  if (resid) {
    double r = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) {
      const int l = idx / n, q = idx % n;
      double a = (l == q) ? -1.0 : 0.0;
      for (int m = 0; m < n; ++m) a += M[l * w2 + m] * Ainv[m * n + q];
      r = fmax(r, fabs(a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(FULL_MASK, r, o));
    *resid = fmax(*resid, r);
  }
  // Singular Slater matrix: two equal-spin electrons on one point (the
  // determinant vanishes by antisymmetry; elimination would leave a residual
  // row of rounding size, not an exact zero), or a pivot that is zero or not
  // finite. No relative pivot threshold is applied: the orbitals of a heavy
  // atom span many orders of magnitude (a 1s value at a valence electron),
  // so pivots far below the largest entry of their column are legitimate,
  // and rounding noise amplified by that scale spread cannot be told apart
  // from a small genuine pivot.
  int coincide = 0;
  for (int pr = lane; pr < n * n; pr += 32) {
    const int l = pr / n, q = pr % n;
    if (q <= l) continue;
    const double* a = &sx[3 * (off + l)];
    const double* c = &sx[3 * (off + q)];
    coincide |= (a[0] == c[0] && a[1] == c[1] && a[2] == c[2]);
  }
  if (__any_sync(FULL_MASK, coincide)) return false;
  bool ok = true;
  for (int col = 0; col < n && ok; ++col) {
    // pivot row: largest |M[r][col]| for r >= col, lowest r on ties
    double best = -1.0;
    int br = col;
    for (int r = col + lane; r < n; r += 32) {
      double a = fabs(M[r * w2 + col]);
      if (a > best) { best = a; br = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(FULL_MASK, best, o);
      int orr = __shfl_xor_sync(FULL_MASK, br, o);
      if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; }
    }
    if (!(best > 0.0) || !isfinite(best)) { ok = false; break; }
    if (br != col) {
      for (int j = lane; j < w2; j += 32) {
        double t = M[col * w2 + j];
        M[col * w2 + j] = M[br * w2 + j];
        M[br * w2 + j] = t;
      }
      __syncwarp();
    }
    double inv = 1.0 / M[col * w2 + col];
    __syncwarp();
    for (int j = lane; j < w2; j += 32) M[col * w2 + j] *= inv;
    __syncwarp();
    for (int r = lane; r < n; r += 32) {
      if (r == col) continue;
      double f = M[r * w2 + col];
      if (f != 0.0)
        for (int j = 0; j < w2; ++j) M[r * w2 + j] -= f * M[col * w2 + j];
    }
    __syncwarp();
  }
  if (ok) {
    for (int idx = lane; idx < n * n; idx += 32) {
      int m = idx / n, l = idx % n;
      Ainv[m * n + l] = M[m * w2 + n + l];
    }
  }
  __syncwarp();
  return ok;
}

// ----------------------------------------------------------------------------
// One evaluation of all P lattice moves out of the walker's configuration
// (Eq. 1 lattice, fixed-node rates) and of its continuous local energy.
// On return sT holds T_c, b and el are warp-uniform. ratio_out (global,
// nullable) receives psi_G(x')/psi_G(x) for every move.
// ----------------------------------------------------------------------------
template <bool NJ>
__device__ void warp_eval(const SysDev& S, const double* sC, const LatDev& L, const WarpMem& wm,
                          int lane, double* ratio_out, double& b, double& el, double* grad_out = nullptr,
                          bool moves = true)
{
  const int N = S.N, nao = S.n_ao, nu = S.n_up;
  // projected inverse columns: v[i][mu] = sum_m C[mu][m] Ainv_sigma[m][l_i]
  for (int idx = lane; idx < N * nao; idx += 32) {
    int i = idx / nao, mu = idx % nao;
    int spin = i < nu ? 0 : 1, l = i < nu ? i : i - nu, n = spin ? S.n_dn : nu;
    const double* A = spin ? wm.A + nu * nu : wm.A;
    double acc = 0.0;
    for (int m = 0; m < n; ++m) acc += sC[mu * S.n_mo + m] * A[m * n + l];
    wm.v[idx] = acc;
  }
  __syncwarp();
  // local energy: lanes over electrons
  double part = 0.0;
  for (int i = lane; i < N; i += 32) {
    const double* ri = &wm.x[3 * i];
    double val, gD[3], lD;
    ao_dot_der(S, &wm.v[i * nao], ri, val, gD, lD);
    double gJ[3] = {0.0, 0.0, 0.0}, lJ = 0.0, Ssum = 0.0, V = 0.0;
    const int si = spin_of(S, i);
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double d0 = ri[0] - wm.x[3 * j], d1 = ri[1] - wm.x[3 * j + 1], d2 = ri[2] - wm.x[3 * j + 2];
      double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      double c = (spin_of(S, j) == si) ? S.c_par : S.c_anti;
      double inv = 1.0 / (1.0 + S.b_ee * r);
      double u1 = c * inv * inv;
      double u2 = -2.0 * S.b_ee * c * inv * inv * inv;
      double ir = 1.0 / r;
      Ssum += c * r * inv;
      if (NJ) {
        double g, g1, g2;
        nj_value3(S, nj_ch_ee(S, i, j), r, g, g1, g2);
        u1 += g1; u2 += g2; Ssum += g;
      }
      gJ[0] += u1 * d0 * ir; gJ[1] += u1 * d1 * ir; gJ[2] += u1 * d2 * ir;
      lJ += u2 + 2.0 * u1 * ir;
      if (j > i && S.ee_on) V += ir;
    }
    for (int I = 0; I < S.n_nuc; ++I) {
      double d0 = ri[0] - S.nuc[I][0], d1 = ri[1] - S.nuc[I][1], d2 = ri[2] - S.nuc[I][2];
      double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      double b1 = S.en_b1[I];
      double inv = 1.0 / (1.0 + S.en_b2 * r);
      double u1 = -b1 * inv * inv;
      double u2 = 2.0 * S.en_b2 * b1 * inv * inv * inv;
      double ir = 1.0 / r;
      Ssum -= b1 * r * inv;
      if (NJ) {
        double g, g1, g2;
        nj_value3(S, 2 + S.nj_species[I], r, g, g1, g2);
        u1 += g1; u2 += g2; Ssum += g;
      }
      gJ[0] += u1 * d0 * ir; gJ[1] += u1 * d1 * ir; gJ[2] += u1 * d2 * ir;
      lJ += u2 + 2.0 * u1 * ir;
      V -= S.Z[I] * ir;
    }
    wm.Ssum[i] = Ssum;
    if (grad_out)
      for (int k = 0; k < 3; ++k) grad_out[3 * i + k] = gD[k] + gJ[k];
    double lap = lD + 2.0 * (gD[0] * gJ[0] + gD[1] * gJ[1] + gD[2] * gJ[2]) + lJ +
                 gJ[0] * gJ[0] + gJ[1] * gJ[1] + gJ[2] * gJ[2];
    part += -0.5 * lap + V;
  }
  el = warp_sum(part) + S.V_nn;
  __syncwarp();
  if (!moves) {
    b = 0.0;
    return;
  }
  // the P lattice moves: lanes over candidates
  const int G = L.G, per_e = 6 * G, P = N * per_e;
  for (int c = lane; c < P; c += 32) {
    int i = c / per_e, rem = c - i * per_e, g = rem / 6, k = (rem % 6) >> 1;
    double sign = (c & 1) ? -1.0 : 1.0;
    double h = g ? L.ap : L.a;
    double ex = wm.R[k], ey = wm.R[3 + k], ez = wm.R[6 + k];
    const double* ri = &wm.x[3 * i];
    double px = ri[0] + sign * h * ex, py = ri[1] + sign * h * ey, pz = ri[2] + sign * h * ez;
    double rdet = ao_dot(S, &wm.v[i * nao], px, py, pz);
    double dJ = jastrow_terms<NJ>(S, wm.x, i, px, py, pz) - wm.Ssum[i];
    double rho = rdet * exp(dJ);
    double w = 1.0;
    if (G == 2) {
      double hh = 0.5 * h;
      double pm = p_weight(S, L, ri[0] + sign * hh * ex, ri[1] + sign * hh * ey, ri[2] + sign * hh * ez);
      w = g ? 1.0 - pm : pm;
    }
    double T = rho > 0.0 ? w * (g ? L.inv2ap2 : L.inv2a2) * rho : 0.0;
    wm.T[c] = T;
    if (ratio_out) ratio_out[c] = rho;
  }
  __syncwarp();
  b = warp_scan(wm.T, P, lane, 0.0, nullptr, nullptr);
}

// ----------------------------------------------------------------------------
// The evaluation on the FP32 pipe, templated on the number type NT:
//   NT = df    double-float (LRDMC_PRECISION_DF64), accurate to FP64 parity;
//   NT = float single precision (LRDMC_PRECISION_FP32), the mixed mode.
// Inputs are converted once per evaluation (positions, rotation, projected
// inverse columns) and kept as double-floats in shared memory (the FP32 mode
// reads their high parts); every lattice move and the local energy are
// computed in NT; rates stay in NT (stored as double-floats), the local
// energy is converted to double.
// ----------------------------------------------------------------------------
template <class NT>
__device__ __forceinline__ NT dot3(NT a0, NT a1, NT a2)
{
  typedef Ar<NT> A;
  return A::add_fast(A::add_fast(A::sqr(a0), A::sqr(a1)), A::sqr(a2));
}

// Slater radial part r^m e^(-zeta r) (e given) or a Gaussian contraction.
template <class NT>
__device__ __forceinline__ NT radial_value_m(const SysDev& S, const ShellDev& sh, const DfShell& dsh, NT r, NT r2,
                                             NT e, const BlockMem& bm)
{
  typedef Ar<NT> A;
  if (sh.kind == 0) {
    if (sh.m_int >= 0) {
      NT pw = A::one();
      for (int j = 0; j < sh.m_int; ++j) pw = A::mul(pw, r);
      return A::mul(pw, e);
    }
    NT lr = A::log(r, S.D.exp.K, bm.tab);
    return A::mul(A::exp(A::mul(A::c(dsh.m), lr), S.D.exp.K, bm.tab), e);
  }
  NT acc = A::zero();
  for (int p = 0; p < sh.n_prim; ++p)
    acc = A::add(acc, A::mul(A::c(dsh.coef[p]),
                             A::exp(A::neg(A::mul(A::c(dsh.alpha[p]), r2)), S.D.exp.K, bm.tab)));
  return acc;
}

template <class NT>
__device__ __forceinline__ int solid_m(int l, const NT d[3], NT Sv[5])
{
  typedef Ar<NT> A;
  if (l == 0) {
    Sv[0] = A::one();
    return 1;
  }
  if (l == 1) {
    Sv[0] = d[0]; Sv[1] = d[1]; Sv[2] = d[2];
    return 3;
  }
  NT xx = A::sqr(d[0]), yy = A::sqr(d[1]), zz = A::sqr(d[2]);
  Sv[0] = A::mul(d[0], d[1]);
  Sv[1] = A::mul(d[1], d[2]);
  Sv[2] = A::mul(d[2], d[0]);
  Sv[3] = A::sub(xx, yy);
  Sv[4] = A::sub(A::add(zz, zz), A::add(xx, yy));
  return 5;
}

// Per nucleus I (one distance each): the determinant ratio
// sum_mu v[mu] chi_mu(p) over the shells centred on I, and the e-n Jastrow
// -sum_I b1_I r/(1 + b2 r).
// The neural pair term in NT arithmetic (same table, double-float copy).
template <class NT>
__device__ __forceinline__ const df* nj_cell_m(const SysDev& S, int c, float rf)
{
  int k = (int)(sqrtf(rf) * S.nj_scale_f[c]);
  k = min(max(k, 0), S.nj_cells - 1);
  return S.nj_tab_df + ((size_t)c * S.nj_cells + k) * 8;
}

__device__ __forceinline__ void nj_load(const df* e, df E[8])
{
  const float4* q = reinterpret_cast<const float4*>(e);
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float4 v = __ldg(q + h);
    E[2 * h] = df_make(v.x, v.y);
    E[2 * h + 1] = df_make(v.z, v.w);
  }
}

template <class NT>
__device__ __forceinline__ NT nj_value_m(const SysDev& S, int c, NT r)
{
  typedef Ar<NT> A;
  const float rf = A::approx(r);
  if (!(rf < S.nj_rcut_f[c])) return A::zero();
  df E[8];
  nj_load(nj_cell_m<NT>(S, c, rf), E);
  const NT t = A::mul(A::sub(r, A::c(E[0])), A::c(E[1]));
  if (sizeof(NT) == sizeof(df)) {
    // the cubic to quintic terms are below 1e-5 of the value on these narrow
    // cells (c_q ~ w^q g^(q)/q!), so single precision carries them to well
    // below the double-float rounding of the sum; the low orders in NT
    const float tf = A::approx(t);
    const float hi = fmaf(fmaf(E[7].hi, tf, E[6].hi), tf, E[5].hi);
    NT v = A::add(A::c(E[4]), A::mul_f(t, hi));
    v = A::add(A::mul(v, t), A::c(E[3]));
    return A::add(A::mul(v, t), A::c(E[2]));
  }
  NT v = A::c(E[7]);
#pragma unroll
  for (int q = 6; q >= 2; --q) v = A::add(A::mul(v, t), A::c(E[q]));
  return v;
}

template <class NT>
__device__ __forceinline__ void nj_value3_m(const SysDev& S, int c, NT r, NT& g, NT& g1, NT& g2)
{
  typedef Ar<NT> A;
  g = A::zero(); g1 = A::zero(); g2 = A::zero();
  const float rf = A::approx(r);
  if (!(rf < S.nj_rcut_f[c])) return;
  df E[8];
  nj_load(nj_cell_m<NT>(S, c, rf), E);
  const NT iw = A::c(E[1]);
  const NT t = A::mul(A::sub(r, A::c(E[0])), iw);
  const NT c1 = A::c(E[3]), c2 = A::c(E[4]), c3 = A::c(E[5]), c4 = A::c(E[6]), c5 = A::c(E[7]);
  NT v = c5, d1 = A::mul_f(c5, 5.0f), d2 = A::mul_f(c5, 20.0f);
  v = A::add(A::mul(v, t), c4);
  v = A::add(A::mul(v, t), c3);
  v = A::add(A::mul(v, t), c2);
  v = A::add(A::mul(v, t), c1);
  g = A::add(A::mul(v, t), A::c(E[2]));
  d1 = A::add(A::mul(d1, t), A::mul_f(c4, 4.0f));
  d1 = A::add(A::mul(d1, t), A::mul_f(c3, 3.0f));
  d1 = A::add(A::mul(d1, t), A::mul_f(c2, 2.0f));
  d1 = A::add(A::mul(d1, t), c1);
  d2 = A::add(A::mul(d2, t), A::mul_f(c4, 12.0f));
  d2 = A::add(A::mul(d2, t), A::mul_f(c3, 6.0f));
  d2 = A::add(A::mul(d2, t), A::mul_f(c2, 2.0f));
  g1 = A::mul(d1, iw);
  g2 = A::mul(d2, A::sqr(iw));
}

// One nucleus's part of a lattice move: the e-n Jastrow terms (Pade and,
// when set, neural) into jen and the basis functions centred on it,
// contracted with the projected inverse column v, into rdet. d = r' - R_I,
// r2 = |d|^2.
template <class NT, bool NJ>
__device__ __forceinline__ void nucleus_term_m(const SysDev& S, const df* v, int I, const NT d[3], NT r2,
                                               const BlockMem& bm, NT& rdet, NT& jen)
{
  typedef Ar<NT> A;
  NT r = A::sqrt(r2);
  if (S.en_b1[I] != 0.0)
    jen = A::sub(jen, A::div(A::mul(A::c(S.D.en_b1[I]), r), A::add_f(A::mul(A::c(S.D.en_b2), r), 1.0f)));
  if (NJ) jen = A::add(jen, nj_value_m<NT>(S, 2 + S.nj_species[I], r));
  NT e = A::zero();
  for (int q = S.nuc_shell_begin[I]; q < S.nuc_shell_begin[I + 1]; ++q) {
    const ShellDev& sh = S.sh[q];
    const DfShell& dsh = S.D.sh[q];
    if (sh.kind == 0 && !sh.same_exp) e = A::exp(A::neg(A::mul(A::c(dsh.zeta), r)), S.D.exp.K, bm.tab);
    NT Rv = radial_value_m<NT>(S, sh, dsh, r, r2, e, bm);
    NT part;
    if (sh.l == 0) {
      part = A::c(v[sh.ao_offset]);
    } else {
      NT Sv[5];
      int nf = solid_m<NT>(sh.l, d, Sv);
      part = A::zero();
      for (int f = 0; f < nf; ++f) part = A::add(part, A::mul(A::c(v[sh.ao_offset + f]), Sv[f]));
    }
    rdet = A::add(rdet, A::mul(part, Rv));
  }
}

template <class NT, bool NJ>
__device__ void nucleus_terms_m(const SysDev& S, const df* v, const NT p[3], const BlockMem& bm, NT& rdet, NT& jen)
{
  typedef Ar<NT> A;
  rdet = A::zero();
  jen = A::zero();
  for (int I = 0; I < S.n_nuc; ++I) {
    NT d[3] = {A::sub_fast(p[0], A::c(S.D.nuc[I][0])), A::sub_fast(p[1], A::c(S.D.nuc[I][1])),
               A::sub_fast(p[2], A::c(S.D.nuc[I][2]))};
    nucleus_term_m<NT, NJ>(S, v, I, d, dot3<NT>(d[0], d[1], d[2]), bm, rdet, jen);
  }
}

// The electron-nucleus cache of one evaluation: for electron i and nucleus
// I, d = r_i - R_I, |d|^2 and e_k . d on the rotated axes (8 double-floats,
// the last unused). A move r_i -> r_i + h e_k has r' - R_I = d + h e_k,
// |r' - R_I|^2 = |d|^2 + 2 h (e_k . d) + h^2, and its bond midpoint
// |d|^2 + h (e_k . d) + h^2/4.
template <class NT>
__device__ void fill_en_cache(const SysDev& S, const WarpMem& wm, int lane)
{
  typedef Ar<NT> A;
  const int n = S.N * S.n_nuc;
  for (int q = lane; q < n; q += 32) {
    const int i = q / S.n_nuc, I = q - i * S.n_nuc;
    NT d[3];
    for (int k = 0; k < 3; ++k) d[k] = A::sub_fast(A::c(wm.xd[3 * i + k]), A::c(S.D.nuc[I][k]));
    df* e = &wm.enc[8 * q];
    for (int k = 0; k < 3; ++k) e[k] = A::store(d[k]);
    e[3] = A::store(dot3<NT>(d[0], d[1], d[2]));
    for (int k = 0; k < 3; ++k)
      e[4 + k] = A::store(A::add(A::add(A::mul(A::c(wm.Rd[k]), d[0]), A::mul(A::c(wm.Rd[3 + k]), d[1])),
                                 A::mul(A::c(wm.Rd[6 + k]), d[2])));
  }
}

// All nuclei's parts of a move from the cache, and (double grid) the
// squared distance of the bond midpoint from the nearest heavy nucleus.
template <class NT, bool NJ>
__device__ __forceinline__ void nucleus_terms_cached_m(const SysDev& S, const df* v, const df* en, int k, NT h,
                                                       const NT he[3], NT h2, const BlockMem& bm, NT& rdet,
                                                       NT& jen, NT& mid2)
{
  typedef Ar<NT> A;
  rdet = A::zero();
  jen = A::zero();
  mid2 = A::inf();
  const NT h2q = A::mul_f(h2, 0.25f);
  for (int I = 0; I < S.n_nuc; ++I) {
    const df* e = &en[8 * I];
    const NT hp = A::mul(h, A::c(e[4 + k]));
    const NT D = A::c(e[3]);
    NT d[3] = {A::add(A::c(e[0]), he[0]), A::add(A::c(e[1]), he[1]), A::add(A::c(e[2]), he[2])};
    nucleus_term_m<NT, NJ>(S, v, I, d, A::add(A::add(D, A::mul_f(hp, 2.0f)), h2), bm, rdet, jen);
    if (S.heavy[I]) {
      NT m2 = A::add(A::add(D, hp), h2q);
      if (A::lt(m2, mid2)) mid2 = m2;
    }
  }
}

// p from the squared distance to the nearest heavy nucleus: Eq. 3
// (Gaussian) or Eq. 2 (Pade).
template <class NT>
__device__ __forceinline__ NT p_from_d2_m(const SysDev& S, const LatDev& L, NT best, const BlockMem& bm)
{
  typedef Ar<NT> A;
  if (L.pkind == 0) return A::exp(A::neg(A::mul(best, A::c(L.p_coef_df))), S.D.exp.K, bm.tab);
  return A::rcp(A::add_f(A::mul(A::c(L.p_coef_df), best), 1.0f));
}

// Index of the electron pair (a, b), a < b, in the pair cache.
__device__ __forceinline__ int pair_index(int N, int a, int b) { return a * N - a * (a + 1) / 2 + (b - a - 1); }

// The pair cache of one evaluation: for every pair a < b, D = |r_a - r_b|^2
// and P_k = e_k . (r_a - r_b) on the evaluation's rotated axes. A lattice
// move r_i -> r_i + h e_k then has |r' - r_j|^2 = D + 2 h s P_k + h^2, with
// s = +1 for i = a and -1 for i = b.
template <class NT, bool NJ>
__device__ void fill_pair_cache(const SysDev& S, const WarpMem& wm, int lane)
{
  typedef Ar<NT> A;
  const int N = S.N;
  for (int q = lane; q < wm.n_pc; q += 32) {
    int a = 0, base = 0;
    while (base + (N - 1 - a) <= q) { base += N - 1 - a; ++a; }
    const int b = a + 1 + (q - base);
    NT d[3];
    for (int k = 0; k < 3; ++k) d[k] = A::sub_fast(A::c(wm.xd[3 * a + k]), A::c(wm.xd[3 * b + k]));
    df* e = &wm.pc[wm.pcw * q];
    const NT D = dot3<NT>(d[0], d[1], d[2]);
    e[0] = A::store(D);
    for (int k = 0; k < 3; ++k) {
      NT pk = A::add(A::add(A::mul(A::c(wm.Rd[k]), d[0]), A::mul(A::c(wm.Rd[3 + k]), d[1])),
                     A::mul(A::c(wm.Rd[6 + k]), d[2]));
      e[1 + k] = A::store(pk);
    }
    if ((wm.pcw == 8 && wm.n_pc > 0 && NJ)) {
      // with the neural term, the pair's Jastrow terms for the local energy
      // (Pade plus neural): u, u'/r, u'' + 2 u'/r, and 1/r (with the Pade
      // factor alone, evaluating them inside the local energy is faster)
      const NT rr = A::sqrt(D);
      const NT bb = A::c(S.D.b_ee);
      const NT c = (spin_of(S, a) == spin_of(S, b)) ? A::c(S.D.c_par) : A::c(S.D.c_anti);
      const NT inv = A::rcp(A::add_f(A::mul(bb, rr), 1.0f));
      const NT inv2 = A::sqr(inv);
      NT u = A::mul(A::mul(c, rr), inv);
      NT u1 = A::mul(c, inv2);
      NT u2 = A::mul_f(A::mul(A::mul(bb, c), A::mul(inv2, inv)), -2.0f);
      if (NJ) {
        NT g, g1, g2;
        nj_value3_m<NT>(S, nj_ch_ee(S, a, b), rr, g, g1, g2);
        u1 = A::add(u1, g1); u2 = A::add(u2, g2); u = A::add(u, g);
      }
      const NT irr = A::rcp(rr);
      const NT u1ir = A::mul(u1, irr);
      e[4] = A::store(u);
      e[5] = A::store(u1ir);
      e[6] = A::store(A::add(u2, A::mul_f(u1ir, 2.0f)));
      e[7] = A::store(irr);
    }
  }
}

// num and den times the power of two that brings den (positive, normal,
// below 2^127) into [1, 2): exact, so num/den keeps its value bit for bit.
__device__ __forceinline__ void pow2_rescale(float& num, float& den)
{
  const float s = __int_as_float((254 - ((__float_as_int(den) >> 23) & 0xff)) << 23);
  num *= s;
  den *= s;
}

__device__ __forceinline__ void pow2_rescale(df& num, df& den)
{
  const float s = __int_as_float((254 - ((__float_as_int(den.hi) >> 23) & 0xff)) << 23);
  num.hi *= s;
  num.lo *= s;
  den.hi *= s;
  den.lo *= s;
}

// sum_{j != i} u_ee(|r_i + h e_k - r_j|) from the pair cache (h carries
// the sign of the move, h2 = h^2); the Pade terms as one running fraction.
template <class NT, bool NJ>
__device__ NT jastrow_ee_cached_m(const SysDev& S, const df* pc, int pcw, int i, int k, NT h, NT h2)
{
  typedef Ar<NT> A;
  NT num = A::zero(), den = A::one(), nn = A::zero();
  const int si = spin_of(S, i), N = S.N;
  const NT b = A::c(S.D.b_ee), cp = A::c(S.D.c_par), ca = A::c(S.D.c_anti);
  // 2h s for the partners after i (s = +1) and before i (s = -1): scaling by
  // a power of two is exact
  const NT h2p = A::mul_f(h, 2.0f), h2m = A::neg(h2p);
  // pair (j, i), j < i, sits at j N - j (j + 1)/2 + (i - j - 1), which grows by
  // N - j - 2 from j to j + 1; pair (i, j), j > i, at q0 + (j - i - 1)
  int q = i - 1;  // pair (0, i)
  for (int j = 0; j < N; ++j) {
    if (j == i) {
      q = pair_index(N, i, i + 1);  // the next partner's pair (unused when i = N - 1)
      continue;
    }
    const df* e = &pc[pcw * q];
    const NT hp = A::mul(j > i ? h2p : h2m, A::c(e[1 + k]));
    // |r' - r_j|^2 = D + 2 h s P_k + h^2: the cheap addition suffices (its
    // error ~2^-44 (D + |2hP| + h^2) is far below what the ratios resolve)
    NT r = A::sqrt(A::add_fast(A::add_fast(A::c(e[0]), hp), h2));
    NT c = (spin_of(S, j) == si) ? cp : ca;
    NT dj = A::add_f(A::mul(b, r), 1.0f);
    num = A::add_fast(A::mul(num, dj), A::mul(A::mul(c, r), den));
    den = A::mul(den, dj);
    if (NJ) nn = A::add(nn, nj_value_m<NT>(S, nj_ch_ee(S, i, j), r));
    q += (j < i) ? N - j - 2 : 1;
    if ((j & 15) == 15) pow2_rescale(num, den);  // every 16 partners, as in jastrow_ee_m
  }
  return A::add(A::div(num, den), nn);
}

// sum_{j != i} u_ee(|p - r_j|): the Pade terms c r/(1 + b r) (all of one
// sign) are summed as one running fraction num/den, so one division serves
// all partners. Every 16 partners pow2_rescale brings den back into [1, 2):
// the product of the (1 + b r) would otherwise leave the float exponent
// range (about 3.4e38) that double-floats and floats share, as 47 partners
// a few bohr away do; 16 factors fit while their geometric mean stays
// below 200.
template <class NT, bool NJ>
__device__ NT jastrow_ee_m(const SysDev& S, const df* xd, int i, const NT p[3])
{
  typedef Ar<NT> A;
  NT num = A::zero(), den = A::one(), nn = A::zero();
  const int si = spin_of(S, i);
  const NT b = A::c(S.D.b_ee), cp = A::c(S.D.c_par), ca = A::c(S.D.c_anti);
  for (int j = 0; j < S.N; ++j) {
    if (j == i) continue;
    NT d0 = A::sub_fast(p[0], A::c(xd[3 * j])), d1 = A::sub_fast(p[1], A::c(xd[3 * j + 1])),
       d2 = A::sub_fast(p[2], A::c(xd[3 * j + 2]));
    NT r = A::sqrt(dot3<NT>(d0, d1, d2));
    NT c = (spin_of(S, j) == si) ? cp : ca;
    NT dj = A::add_f(A::mul(b, r), 1.0f);
    num = A::add_fast(A::mul(num, dj), A::mul(A::mul(c, r), den));
    den = A::mul(den, dj);
    if (NJ) nn = A::add(nn, nj_value_m<NT>(S, nj_ch_ee(S, i, j), r));
    if ((j & 15) == 15) pow2_rescale(num, den);
  }
  return A::add(A::div(num, den), nn);
}

template <class NT>
__device__ __forceinline__ NT p_weight_m(const SysDev& S, const LatDev& L, const NT m[3], const BlockMem& bm)
{
  typedef Ar<NT> A;
  NT best = A::inf();
  for (int I = 0; I < S.n_nuc; ++I) {
    if (!S.heavy[I]) continue;
    NT d0 = A::sub_fast(m[0], A::c(S.D.nuc[I][0])), d1 = A::sub_fast(m[1], A::c(S.D.nuc[I][1])),
       d2 = A::sub_fast(m[2], A::c(S.D.nuc[I][2]));
    NT d2s = dot3<NT>(d0, d1, d2);
    if (A::lt(d2s, best)) best = d2s;
  }
  if (L.pkind == 0) return A::exp(A::neg(A::mul(best, A::c(L.p_coef_df))), S.D.exp.K, bm.tab);
  return A::rcp(A::add_f(A::mul(A::c(L.p_coef_df), best), 1.0f));
}

template <class NT>
__device__ __forceinline__ NT warp_sum_m(NT v)
{
  typedef Ar<NT> A;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = A::add(v, A::shfl_xor(v, o));
  return v;
}

// Chunked inclusive scan of the rates (as warp_scan) in NT.
template <class NT>
__device__ NT warp_scan_m(const df* T, int P, int lane, NT target, int* pick, int* last)
{
  typedef Ar<NT> A;
  NT carry = A::zero();
  int p = -1, lp = -1;
  for (int base = 0; base < P; base += 32) {
    int c = base + lane;
    NT t = (c < P) ? A::c(T[c]) : A::zero();
    NT v = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      NT y = A::shfl_up(v, o);
      if (lane >= o) v = A::add(v, y);
    }
    NT C = A::add(carry, v);
    if (pick) {
      unsigned hit = __ballot_sync(FULL_MASK, (c < P) && A::lt(target, C));
      if (p < 0 && hit) p = base + __ffs(hit) - 1;
      unsigned pos = __ballot_sync(FULL_MASK, (c < P) && A::positive(t));
      if (pos) lp = base + 31 - __clz(pos);
    }
    carry = A::shfl(C, 31);
  }
  if (pick) { *pick = p; *last = lp; }
  return carry;
}

// Partial sums of the local energy of electron i over the shell units, the
// partners (the t-th electron other than i) and the nuclei whose index is
// congruent to part modulo L.
template <class NT>
struct ElParts {
  NT gD[3], lD, gJ[3], lJ, S, V;
};

template <class NT>
__device__ __forceinline__ void el_zero(ElParts<NT>& o)
{
  typedef Ar<NT> A;
  o.lD = A::zero(); o.lJ = A::zero(); o.S = A::zero(); o.V = A::zero();
  for (int k = 0; k < 3; ++k) { o.gD[k] = A::zero(); o.gJ[k] = A::zero(); }
}

template <class NT, bool NJ, bool PC = true>
__device__ LRDMC_EL void el_parts_m(const SysDev& S, const WarpMem& wm, int i, int part, int L, const BlockMem& bm,
                           ElParts<NT>& o)
{
  typedef Ar<NT> A;
  const int nao = S.n_ao;
  const df* v = &wm.vd[i * nao];
  const NT ri[3] = {A::c(wm.xd[3 * i]), A::c(wm.xd[3 * i + 1]), A::c(wm.xd[3 * i + 2])};
  el_zero<NT>(o);
  // basis: gradient and Laplacian contracted with v. The shells' units
  // (single shells, or groups sharing one Slater exponential) are dealt to
  // the parts, and each part loops over its own units only, so that the
  // parts' shells run side by side on their lanes (a loop over all shells
  // with the others' skipped would run them one after the other).
  int prev_c = -1;
  NT d[3] = {A::zero(), A::zero(), A::zero()}, r = A::zero(), r2 = A::zero(), ir = A::zero(), e = A::zero();
  for (int gi = part; gi < S.n_grp; gi += L)
  for (int q = S.grp_first[gi]; q < S.grp_first[gi + 1]; ++q) {
    const ShellDev& sh = S.sh[q];
    const DfShell& dsh = S.D.sh[q];
    const bool first = q == S.grp_first[gi];
    if (sh.center != prev_c) {
      prev_c = sh.center;
      d[0] = A::sub_fast(ri[0], A::c(S.D.nuc[prev_c][0]));
      d[1] = A::sub_fast(ri[1], A::c(S.D.nuc[prev_c][1]));
      d[2] = A::sub_fast(ri[2], A::c(S.D.nuc[prev_c][2]));
      r2 = dot3<NT>(d[0], d[1], d[2]);
      r = A::sqrt(r2);
      ir = A::rcp(r);
    }
    if (sh.kind == 0 && (first || !sh.same_exp)) e = A::exp(A::neg(A::mul(A::c(dsh.zeta), r)), S.D.exp.K, bm.tab);
    NT Rv, R1, R2;
    if (sh.kind == 0) {
      Rv = radial_value_m<NT>(S, sh, dsh, r, r2, e, bm);
      NT t = A::sub(A::mul(A::c(dsh.m), ir), A::c(dsh.zeta));
      R1 = A::mul(A::mul(t, Rv), ir);
      R2 = A::mul(A::sub(A::sqr(t), A::mul(A::c(dsh.m), A::sqr(ir))), Rv);
    } else {
      Rv = A::zero(); R1 = A::zero(); R2 = A::zero();
      for (int p = 0; p < sh.n_prim; ++p) {
        NT al = A::c(dsh.alpha[p]);
        NT g = A::mul(A::c(dsh.coef[p]), A::exp(A::neg(A::mul(al, r2)), S.D.exp.K, bm.tab));
        Rv = A::add(Rv, g);
        NT m2a = A::mul_f(al, -2.0f);
        R1 = A::add(R1, A::mul(m2a, g));
        NT four_a2r2 = A::mul_f(A::mul(A::sqr(al), r2), 4.0f);
        R2 = A::add(R2, A::mul(A::add(four_a2r2, m2a), g));
      }
    }
    NT Sv[5];
    int nf = solid_m<NT>(sh.l, d, Sv);
    NT radlap = A::add(R2, A::mul_f(R1, 2.0f * (sh.l + 1)));
    for (int f = 0; f < nf; ++f) {
      NT cc = A::c(v[sh.ao_offset + f]);
      NT cS = A::mul(cc, Sv[f]);
      // grad S of the solid harmonics
      NT gS[3];
      if (sh.l == 0) { gS[0] = A::zero(); gS[1] = A::zero(); gS[2] = A::zero(); }
      else if (sh.l == 1) { gS[0] = A::zero(); gS[1] = A::zero(); gS[2] = A::zero(); gS[f] = A::one(); }
      else {
        switch (f) {
          case 0: gS[0] = d[1]; gS[1] = d[0]; gS[2] = A::zero(); break;
          case 1: gS[0] = A::zero(); gS[1] = d[2]; gS[2] = d[1]; break;
          case 2: gS[0] = d[2]; gS[1] = A::zero(); gS[2] = d[0]; break;
          case 3: gS[0] = A::mul_f(d[0], 2.0f); gS[1] = A::mul_f(d[1], -2.0f); gS[2] = A::zero(); break;
          default: gS[0] = A::mul_f(d[0], -2.0f); gS[1] = A::mul_f(d[1], -2.0f); gS[2] = A::mul_f(d[2], 4.0f); break;
        }
      }
      NT cSR1 = A::mul(cS, R1);
      NT cR = A::mul(cc, Rv);
      for (int k = 0; k < 3; ++k) o.gD[k] = A::add(o.gD[k], A::add(A::mul(cR, gS[k]), A::mul(cSR1, d[k])));
      o.lD = A::add(o.lD, A::mul(cS, radlap));
    }
  }
  // e-e pairs: the N - 1 partners of i (j = t, skipping i) dealt evenly
  // to the parts
  const int si = spin_of(S, i);
  const NT b = A::c(S.D.b_ee);
  if (PC && sizeof(NT) == sizeof(df) && (wm.pcw == 8 && wm.n_pc > 0 && NJ)) {
    // every pair's terms come from the pair cache (evaluated once per pair)
    for (int t = part; t < S.N - 1; t += L) {
      const int j = t < i ? t : t + 1;
      const df* e = &wm.pc[8 * pair_index(S.N, min(i, j), max(i, j))];
      NT d0 = A::sub_fast(ri[0], A::c(wm.xd[3 * j])), d1 = A::sub_fast(ri[1], A::c(wm.xd[3 * j + 1])),
         d2 = A::sub_fast(ri[2], A::c(wm.xd[3 * j + 2]));
      const NT u1ir = A::c(e[5]);
      o.gJ[0] = A::add(o.gJ[0], A::mul(u1ir, d0));
      o.gJ[1] = A::add(o.gJ[1], A::mul(u1ir, d1));
      o.gJ[2] = A::add(o.gJ[2], A::mul(u1ir, d2));
      o.lJ = A::add(o.lJ, A::c(e[6]));
      o.S = A::add(o.S, A::c(e[4]));
      if (j > i && S.ee_on) o.V = A::add(o.V, A::c(e[7]));
    }
  } else
  for (int t = part; t < S.N - 1; t += L) {
    const int j = t < i ? t : t + 1;
    NT d0 = A::sub_fast(ri[0], A::c(wm.xd[3 * j])), d1 = A::sub_fast(ri[1], A::c(wm.xd[3 * j + 1])),
       d2 = A::sub_fast(ri[2], A::c(wm.xd[3 * j + 2]));
    NT rr = A::sqrt(dot3<NT>(d0, d1, d2));
    NT c = (spin_of(S, j) == si) ? A::c(S.D.c_par) : A::c(S.D.c_anti);
    NT inv = A::rcp(A::add_f(A::mul(b, rr), 1.0f));
    NT inv2 = A::sqr(inv);
    NT u1 = A::mul(c, inv2);
    NT u2 = A::mul_f(A::mul(A::mul(b, c), A::mul(inv2, inv)), -2.0f);
    o.S = A::add(o.S, A::mul(A::mul(c, rr), inv));
    if (NJ) {
      NT g, g1, g2;
      nj_value3_m<NT>(S, nj_ch_ee(S, i, j), rr, g, g1, g2);
      u1 = A::add(u1, g1); u2 = A::add(u2, g2); o.S = A::add(o.S, g);
    }
    NT irr = A::rcp(rr);
    NT u1ir = A::mul(u1, irr);
    o.gJ[0] = A::add(o.gJ[0], A::mul(u1ir, d0));
    o.gJ[1] = A::add(o.gJ[1], A::mul(u1ir, d1));
    o.gJ[2] = A::add(o.gJ[2], A::mul(u1ir, d2));
    o.lJ = A::add(o.lJ, A::add(u2, A::mul_f(u1ir, 2.0f)));
    if (j > i && S.ee_on) o.V = A::add(o.V, irr);
  }
  // e-n terms
  for (int I = part; I < S.n_nuc; I += L) {
    NT d0 = A::sub_fast(ri[0], A::c(S.D.nuc[I][0])), d1 = A::sub_fast(ri[1], A::c(S.D.nuc[I][1])),
       d2 = A::sub_fast(ri[2], A::c(S.D.nuc[I][2]));
    NT rr = A::sqrt(dot3<NT>(d0, d1, d2));
    NT b1 = A::c(S.D.en_b1[I]), b2 = A::c(S.D.en_b2);
    NT inv = A::rcp(A::add_f(A::mul(b2, rr), 1.0f));
    NT inv2 = A::sqr(inv);
    NT u1 = A::neg(A::mul(b1, inv2));
    NT u2 = A::mul_f(A::mul(A::mul(b2, b1), A::mul(inv2, inv)), 2.0f);
    o.S = A::sub(o.S, A::mul(A::mul(b1, rr), inv));
    if (NJ) {
      NT g, g1, g2;
      nj_value3_m<NT>(S, 2 + S.nj_species[I], rr, g, g1, g2);
      u1 = A::add(u1, g1); u2 = A::add(u2, g2); o.S = A::add(o.S, g);
    }
    NT irr = A::rcp(rr);
    NT u1ir = A::mul(u1, irr);
    o.gJ[0] = A::add(o.gJ[0], A::mul(u1ir, d0));
    o.gJ[1] = A::add(o.gJ[1], A::mul(u1ir, d1));
    o.gJ[2] = A::add(o.gJ[2], A::mul(u1ir, d2));
    o.lJ = A::add(o.lJ, A::add(u2, A::mul_f(u1ir, 2.0f)));
    o.V = A::sub(o.V, A::mul(A::c(S.D.Z[I]), irr));
  }
}

template <class NT>
__device__ __forceinline__ void el_combine(ElParts<NT>& o, int src, bool take)
{
  typedef Ar<NT> A;
  NT t;
#define ELC(field)            \
  t = A::shfl(o.field, src);  \
  if (take) o.field = A::add(o.field, t);
  ELC(lD) ELC(lJ) ELC(S) ELC(V)
  ELC(gD[0]) ELC(gD[1]) ELC(gD[2]) ELC(gJ[0]) ELC(gJ[1]) ELC(gJ[2])
#undef ELC
}

template <class NT>
__device__ __forceinline__ NT el_local(const ElParts<NT>& o)
{
  typedef Ar<NT> A;
  NT dot = A::add(A::add(A::mul(o.gD[0], o.gJ[0]), A::mul(o.gD[1], o.gJ[1])), A::mul(o.gD[2], o.gJ[2]));
  NT gg = A::add(A::add(A::sqr(o.gJ[0]), A::sqr(o.gJ[1])), A::sqr(o.gJ[2]));
  NT lap = A::add(A::add(o.lD, A::mul_f(dot, 2.0f)), A::add(o.lJ, gg));
  return A::add(A::mul_f(lap, -0.5f), o.V);
}

// One lattice move c of an evaluation (Eq. 1 lattice, fixed-node rate): the
// determinant and Jastrow ratios at the displaced position, p at the bond
// midpoint on the double grid, the rate T_c into Td[c]. Reads the
// evaluation's shared-memory state (projected inverse columns, positions,
// rotation, caches and the Jastrow sums Sd of its local-energy pass).
template <class NT, bool NJ, bool NC>
__device__ __forceinline__ void candidate_m(const SysDev& S, const LatDev& L, const WarpMem& wm, const BlockMem& bm,
                                            int c, df* Td, double* ratio_out)
{
  typedef Ar<NT> A;
  const int nao = S.n_ao;
  const int G = L.G, per_e = 6 * G;
  constexpr bool kUsePairCache = sizeof(NT) == sizeof(df) && !NC;
  {
    const int i = c / per_e, rem = c - i * per_e, g = rem / 6, k = (rem % 6) >> 1;
    NT h = g ? A::c(L.ap_df) : A::c(L.a_df);
    if (c & 1) h = A::neg(h);
    const NT e0 = A::c(wm.Rd[k]), e1 = A::c(wm.Rd[3 + k]), e2 = A::c(wm.Rd[6 + k]);
    NT rdet, jen, jee, pm = A::one();
    if (kUsePairCache) {
      // the caches pay in double-float arithmetic only (single precision
      // recomputes a distance faster than it reads it back)
      const NT h2 = A::sqr(h);
      const NT he[3] = {A::mul(h, e0), A::mul(h, e1), A::mul(h, e2)};
      NT mid2;
      nucleus_terms_cached_m<NT, NJ>(S, &wm.vd[i * nao], &wm.enc[8 * i * S.n_nuc], k, h, he, h2, bm, rdet, jen,
                                 mid2);
      if (wm.n_pc) {
        jee = jastrow_ee_cached_m<NT, NJ>(S, wm.pc, wm.pcw, i, k, h, h2);
      } else {
        const NT p[3] = {A::add(A::c(wm.xd[3 * i]), he[0]), A::add(A::c(wm.xd[3 * i + 1]), he[1]),
                         A::add(A::c(wm.xd[3 * i + 2]), he[2])};
        jee = jastrow_ee_m<NT, NJ>(S, wm.xd, i, p);
      }
      if (G == 2) pm = p_from_d2_m<NT>(S, L, mid2, bm);
    } else {
      const NT ri[3] = {A::c(wm.xd[3 * i]), A::c(wm.xd[3 * i + 1]), A::c(wm.xd[3 * i + 2])};
      const NT p[3] = {A::add(ri[0], A::mul(h, e0)), A::add(ri[1], A::mul(h, e1)), A::add(ri[2], A::mul(h, e2))};
      nucleus_terms_m<NT, NJ>(S, &wm.vd[i * nao], p, bm, rdet, jen);
      jee = jastrow_ee_m<NT, NJ>(S, wm.xd, i, p);
      if (G == 2) {
        const NT hh = A::half(h);
        const NT mid[3] = {A::add(ri[0], A::mul(hh, e0)), A::add(ri[1], A::mul(hh, e1)),
                           A::add(ri[2], A::mul(hh, e2))};
        pm = p_weight_m<NT>(S, L, mid, bm);
      }
    }
    NT dJ = A::sub(A::add(jee, jen), A::c(wm.Sd[i]));
    NT rho = A::mul(rdet, A::exp(dJ, S.D.exp.K, bm.tab));
    NT w = A::one();
    if (G == 2) w = g ? A::add_f(A::neg(pm), 1.0f) : pm;
    NT T = A::zero();
    if (A::positive(rho)) T = A::mul(A::mul(w, g ? A::c(L.inv2ap2_df) : A::c(L.inv2a2_df)), rho);
    Td[c] = A::store(T);
    if (ratio_out) ratio_out[c] = A::to_double(rho);
  }
}

// The first part of an evaluation: projected inverse columns, converted
// positions and rotation, the caches, then the local energy (into el) and
// the Jastrow sums Sd of every electron. The moves read all of it.
// 1: the FP32 mode's local energy in double-float (the lattice moves stay in
// single precision); 0: all of its evaluation in single precision.
#ifndef LRDMC_FP32_EL_DF
#define LRDMC_FP32_EL_DF 1
#endif
template <class NT, bool NJ, bool NC>
__device__ __forceinline__ void eval_prelude_m(const SysDev& S, const double* sC, const LatDev& L, const WarpMem& wm,
                                               int lane, double& el)
{
  typedef Ar<NT> A;
  const int N = S.N, nao = S.n_ao, nu = S.n_up;
  const BlockMem bm = block_mem(S, const_cast<double*>(sC));
  // projected inverse columns (FP64, or FP32 in the mixed mode), then
  // converted with the positions. The mixed mode converts the inverse
  // blocks to float once (scratch), not once per use: each conversion from
  // double runs on the FP64 pipe
  // The FP32 mode can take its local energy in double-float (LRDMC_FP32_EL_DF,
  // on by default): the projected columns, positions and rotation are then
  // formed as in the double-float mode, and only the lattice moves run in
  // single precision (they read the double-float values' leading floats).
  constexpr bool kElDf = sizeof(NT) == sizeof(float) && LRDMC_FP32_EL_DF;
  constexpr bool kFloatProj = sizeof(NT) == sizeof(float) && !kElDf;
  typedef typename std::conditional<kElDf, df, NT>::type ET;
  typedef Ar<ET> AE;
  const float* Af = reinterpret_cast<const float*>(wm.scr);
  if (kFloatProj) {
    for (int j = lane; j < nu * nu + S.n_dn * S.n_dn; j += 32) reinterpret_cast<float*>(wm.scr)[j] = (float)wm.A[j];
    __syncwarp();
  }
  for (int idx = lane; idx < N * nao; idx += 32) {
    int i = idx / nao, mu = idx % nao;
    int spin = i < nu ? 0 : 1, l = i < nu ? i : i - nu, n = spin ? S.n_dn : nu;
    const double* Am = spin ? wm.A + nu * nu : wm.A;
    if (kFloatProj) {
      const float* Amf = spin ? Af + nu * nu : Af;
      float acc = 0.0f;
      for (int m = 0; m < n; ++m) acc += bm.Cf[mu * S.n_mo + m] * Amf[m * n + l];
      wm.vd[idx] = df_make(acc, 0.0f);
    } else {
      double acc = 0.0;
      for (int m = 0; m < n; ++m) acc += sC[mu * S.n_mo + m] * Am[m * n + l];
      wm.vd[idx] = AE::store(AE::from_double(acc));
    }
  }
  for (int j = lane; j < 3 * N; j += 32) wm.xd[j] = AE::store(AE::from_double(wm.x[j]));
  if (lane < 9) wm.Rd[lane] = AE::store(AE::from_double(wm.R[lane]));
  __syncwarp();
  // the caches pay in double-float arithmetic only, and exist only when
  // the system's layout has room for them (NC is set otherwise: the
  // kernels of such systems carry no cached code)
  constexpr bool kUsePairCache = sizeof(NT) == sizeof(df) && !NC;
  if (kUsePairCache) {
    fill_pair_cache<NT, NJ>(S, wm, lane);
    fill_en_cache<NT>(S, wm, lane);
    __syncwarp();
  }
  // local energy: Lp lanes per electron share its shells, electrons and nuclei
  constexpr bool kPC = sizeof(NT) == sizeof(df) && !NC;  // the pair cache holds the pairs' terms
  ET epart = AE::zero();
  if (N <= 32) {
    const int Lp = 32 / N;
    const int i = lane % N, part = lane / N;
    const bool act = lane < N * Lp;
    ElParts<ET> o;
    if (act) el_parts_m<ET, NJ, kPC>(S, wm, i, part, Lp, bm, o);
    else el_zero<ET>(o);
    for (int pp = 1; pp < Lp; ++pp) {
      int src = lane + pp * N;
      el_combine<ET>(o, src < 32 ? src : lane, part == 0 && src < N * Lp);
    }
    if (part == 0 && act) {
      wm.Sd[i] = AE::store(o.S);
      epart = el_local<ET>(o);
    }
  } else {
    for (int i = lane; i < N; i += 32) {
      ElParts<ET> o;
      el_parts_m<ET, NJ, kPC>(S, wm, i, 0, 1, bm, o);
      wm.Sd[i] = AE::store(o.S);
      epart = AE::add(epart, el_local<ET>(o));
    }
  }
  ET etot = warp_sum_m<ET>(epart);
  el = AE::to_double(etot) + S.V_nn;
  __syncwarp();
}

template <class NT, bool NJ, bool NC, bool MOVES = true>
__device__ void warp_eval_m(const SysDev& S, const double* sC, const LatDev& L, const WarpMem& wm, int lane,
                            double* ratio_out, double& b, df& bdf, double& el)
{
  typedef Ar<NT> A;
  const int N = S.N;
  const BlockMem bm = block_mem(S, const_cast<double*>(sC));
  eval_prelude_m<NT, NJ, NC>(S, sC, L, wm, lane, el);
  if (!MOVES) {  // local energy and Jastrow sums only (the caller forms the moves)
    b = 0.0;
    bdf = A::store(A::zero());
    return;
  }
  // the P lattice moves
  const int G = L.G, per_e = 6 * G, P = N * per_e;
  df* Td = reinterpret_cast<df*>(wm.T);  // rates stay in NT, stored as double-floats
  for (int c = lane; c < P; c += 32) candidate_m<NT, NJ, NC>(S, L, wm, bm, c, Td, ratio_out);
  __syncwarp();
  NT btot = warp_scan_m<NT>(Td, P, lane, A::zero(), nullptr, nullptr);
  bdf = A::store(btot);
  b = A::to_double(btot);
}

template <int PREC, bool NJ, bool NC>
__device__ __forceinline__ void warp_eval_any(const SysDev& S, const double* sC, const LatDev& L,
                                              const WarpMem& wm, int lane, double* ratio_out, double& b,
                                              df& bdf, double& el)
{
  if (PREC == LRDMC_PRECISION_DF64) {
    warp_eval_m<df, NJ, NC>(S, sC, L, wm, lane, ratio_out, b, bdf, el);
  } else if (PREC == LRDMC_PRECISION_FP32) {
    warp_eval_m<float, NJ, true>(S, sC, L, wm, lane, ratio_out, b, bdf, el);
  } else {
    warp_eval<NJ>(S, sC, L, wm, lane, ratio_out, b, el);
    bdf = df_make(0.0f, 0.0f);
  }
}

// ----------------------------------------------------------------------------
// Sherman-Morrison update for electron i moving to p (warp-cooperative):
// y_n = sum_m phi_m(p) Ainv[m][n], ratio = y_l,
// Ainv[m][n] -= Ainv[m][l] (y_n - delta_nl) / ratio.
// ----------------------------------------------------------------------------
// chi_mu(p) for all AOs in double-float, one lane per shell, written back
// as doubles.
__device__ void ao_values_df_lanes(const SysDev& S, const double* p, double* out, int lane, const BlockMem& bm)
{
  typedef Ar<df> A;
  df pd[3] = {df_from_double(p[0]), df_from_double(p[1]), df_from_double(p[2])};
  // one shell per lane (at most 32 shells), each with its own centre
  // distance and exponential: all shells side by side
  for (int q = lane; q < S.n_shell; q += 32) {
    const ShellDev& sh = S.sh[q];
    const DfShell& dsh = S.D.sh[q];
    df d[3];
    d[0] = df_sub_fast(pd[0], S.D.nuc[sh.center][0]);
    d[1] = df_sub_fast(pd[1], S.D.nuc[sh.center][1]);
    d[2] = df_sub_fast(pd[2], S.D.nuc[sh.center][2]);
    const df r2 = dot3<df>(d[0], d[1], d[2]);
    const df r = df_sqrt(r2);
    df e = A::zero();
    if (sh.kind == 0) e = df_exp(df_neg(df_mul(dsh.zeta, r)), S.D.exp.K, bm.tab);
    df Rv = radial_value_m<df>(S, sh, dsh, r, r2, e, bm);
    df Sv[5];
    int nf = solid_m<df>(sh.l, d, Sv);
    for (int f = 0; f < nf; ++f) out[sh.ao_offset + f] = df_to_double(df_mul(Sv[f], Rv));
  }
}

// chi_mu(p) for all AOs in double-float into out (df), one lane per shell.
__device__ void ao_values_df_out(const SysDev& S, const df* pd, df* out, int lane, const BlockMem& bm)
{
  typedef Ar<df> A;
  // one shell per lane (at most 32 shells), each with its own centre
  // distance and exponential: all shells side by side
  for (int q = lane; q < S.n_shell; q += 32) {
    const ShellDev& sh = S.sh[q];
    const DfShell& dsh = S.D.sh[q];
    df d[3];
    d[0] = df_sub_fast(pd[0], S.D.nuc[sh.center][0]);
    d[1] = df_sub_fast(pd[1], S.D.nuc[sh.center][1]);
    d[2] = df_sub_fast(pd[2], S.D.nuc[sh.center][2]);
    const df r2 = dot3<df>(d[0], d[1], d[2]);
    const df r = df_sqrt(r2);
    df e = A::zero();
    if (sh.kind == 0) e = df_exp(df_neg(df_mul(dsh.zeta, r)), S.D.exp.K, bm.tab);
    df Rv = radial_value_m<df>(S, sh, dsh, r, r2, e, bm);
    df Sv[5];
    int nf = solid_m<df>(sh.l, d, Sv);
    for (int f = 0; f < nf; ++f) out[sh.ao_offset + f] = df_mul(Sv[f], Rv);
  }
}

// Sherman-Morrison update in double-float arithmetic (the FP32 mode): the
// orbitals at the new position, y = phi A^-1, ratio = y_l, and
// the rank-one update, with the spin block read from and written back to
// its IEEE-double copy. pd: the new position as a double-float.
__device__ LRDMC_JUMP bool warp_sm_update_df(const SysDev& S, const BlockMem& bm, const WarpMem& wm, int i, const df* pd,
                                  int lane)
{
  const int nu = S.n_up;
  const int spin = i < nu ? 0 : 1, l = i < nu ? i : i - nu, n = spin ? S.n_dn : nu;
  double* A = spin ? wm.A + nu * nu : wm.A;
  df* chi = reinterpret_cast<df*>(wm.scr);  // [n_ao]
  df* phi = chi + S.n_ao;                   // [n]
  df* y = phi + n;                          // [n]
  df* Ad = y + n;                           // [n][n]
  ao_values_df_out(S, pd, chi, lane, bm);
  for (int idx = lane; idx < n * n; idx += 32) Ad[idx] = df_from_double(A[idx]);
  __syncwarp();
  for (int m = lane; m < n; m += 32) {
    df a = df_make(0.0f, 0.0f);
    for (int mu = 0; mu < S.n_ao; ++mu) a = df_add(a, df_mul(bm.Cd[mu * S.n_mo + m], chi[mu]));
    phi[m] = a;
  }
  __syncwarp();
  for (int q = lane; q < n; q += 32) {
    df a = df_make(0.0f, 0.0f);
    for (int m = 0; m < n; ++m) a = df_add(a, df_mul(phi[m], Ad[m * n + q]));
    y[q] = a;
  }
  __syncwarp();
  const df ratio = y[l];
  if (ratio.hi == 0.0f) return false;
  const df inv = df_rcp(ratio);
  for (int idx = lane; idx < n * n; idx += 32) {
    int m = idx / n, q = idx % n;
    df yq = (q == l) ? df_add_f(y[q], -1.0f) : y[q];
    A[idx] = df_to_double(df_sub(Ad[idx], df_mul(Ad[m * n + l], df_mul(yq, inv))));
  }
  __syncwarp();
  return true;
}

template <int PREC>
__device__ LRDMC_JUMP bool warp_sm_update(const SysDev& S, const double* sC, const WarpMem& wm, int i,
                               const double* p, int lane)
{
  const int nu = S.n_up;
  const int spin = i < nu ? 0 : 1, l = i < nu ? i : i - nu, n = spin ? S.n_dn : nu;
  double* A = spin ? wm.A + nu * nu : wm.A;
  double* chi = wm.scr;            // [n_ao]
  double* phi = chi + S.n_ao;      // [n]
  double* y = phi + n;             // [n]
  double* col = y + n;             // [n]
  if (PREC != LRDMC_PRECISION_FP64) ao_values_df_lanes(S, p, chi, lane, block_mem(S, const_cast<double*>(sC)));
  else if (lane == 0) ao_values(S, p, chi);
  __syncwarp();
  for (int m = lane; m < n; m += 32) {
    double a = 0.0;
    for (int mu = 0; mu < S.n_ao; ++mu) a += sC[mu * S.n_mo + m] * chi[mu];
    phi[m] = a;
  }
  __syncwarp();
  for (int q = lane; q < n; q += 32) {
    double a = 0.0;
    for (int m = 0; m < n; ++m) a += phi[m] * A[m * n + q];
    y[q] = a;
    col[q] = A[q * n + l];
  }
  __syncwarp();
  double ratio = y[l];
  if (ratio == 0.0) return false;
  double inv = 1.0 / ratio;
  for (int idx = lane; idx < n * n; idx += 32) {
    int m = idx / n, q = idx % n;
    A[idx] -= col[m] * ((y[q] - (q == l ? 1.0 : 0.0)) * inv);
  }
  __syncwarp();
  return true;
}

// ----------------------------------------------------------------------------
// Record load / store.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void load_record(const Layout& Lo, const double* rec, const WarpMem& wm,
                                            int lane, double& b, double& el)
{
  for (int j = lane; j < 3 * Lo.N; j += 32) wm.x[j] = rec[Lo.off_x + j];
  for (int j = lane; j < Lo.nu * Lo.nu + Lo.nd * Lo.nd; j += 32) wm.A[j] = rec[Lo.off_au + j];
  for (int j = lane; j < 9; j += 32) wm.R[j] = rec[Lo.off_R + j];
  for (int j = lane; j < Lo.P_max; j += 32) wm.T[j] = rec[Lo.off_T + j];
  b = rec[Lo.off_b];
  el = rec[Lo.off_el];
  __syncwarp();
}

__device__ __forceinline__ void store_record(const Layout& Lo, double* rec, const WarpMem& wm,
                                             int lane, double b, double el)
{
  __syncwarp();
  for (int j = lane; j < 3 * Lo.N; j += 32) rec[Lo.off_x + j] = wm.x[j];
  for (int j = lane; j < Lo.nu * Lo.nu + Lo.nd * Lo.nd; j += 32) rec[Lo.off_au + j] = wm.A[j];
  for (int j = lane; j < 9; j += 32) rec[Lo.off_R + j] = wm.R[j];
  for (int j = lane; j < Lo.P_max; j += 32) rec[Lo.off_T + j] = wm.T[j];
  if (lane == 0) {
    rec[Lo.off_b] = b;
    rec[Lo.off_el] = el;
  }
}

__device__ __forceinline__ void stage_coefficients(const SysDev& S, double* sC)
{
  BlockMem bm = block_mem(S, sC);
  for (int j = threadIdx.x; j < S.n_ao * S.n_mo; j += blockDim.x) {
    sC[j] = S.C[j];
    bm.Cd[j] = df_from_double(S.C[j]);
    bm.Cf[j] = (float)S.C[j];
  }
  for (int j = threadIdx.x; j < 64; j += blockDim.x) bm.tab[j] = S.D.exp.t[j];
  __syncthreads();
}

// ----------------------------------------------------------------------------
// Kernels.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_init(const __grid_constant__ SysDev S, const Layout Lo, const PopDev P, const double* x0)
{
  extern __shared__ double smem[];
  double* sC = smem;
  stage_coefficients(S, sC);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int s = blockIdx.x * kWarpsPerBlock + wib;
  if (s >= P.W) return;
  WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
  for (int j = lane; j < 3 * Lo.N; j += 32) wm.x[j] = x0[(size_t)s * 3 * Lo.N + j];
  for (int j = lane; j < Lo.P_max; j += 32) wm.T[j] = 0.0;
  __syncwarp();
  bool ok = warp_inverse(S, sC, wm.x, 0, wm.A, wm.scr, lane);
  ok = ok && warp_inverse(S, sC, wm.x, 1, wm.A + Lo.nu * Lo.nu, wm.scr, lane);
  if (!ok && lane == 0) atomicOr(P.err, kErrSingular);
  if (lane == 0) {
    double u[4];
    draw_uniforms(P.seed, (uint64_t)s, kIntervalInit, 0, kTagRot, u);
    rotation_matrix(u[0], u[1], u[2], wm.R);
    P.parent[s] = s;
    P.order[s] = s;
  }
  store_record(Lo, P.rec_src + (size_t)s * Lo.rec, wm, lane, NAN, NAN);
}

template <int PREC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_eval_all(const __grid_constant__ SysDev S, const Layout Lo, const LatDev L, const PopDev P)
{
  constexpr int PR = PREC & 3;         // the arithmetic (LRDMC_PRECISION_*)
  constexpr bool NJ = (PREC & 8) != 0;  // the neural pair term is set
  constexpr bool NC = (PREC & 4) != 0;  // the layout has no evaluation caches
  extern __shared__ double smem[];
  double* sC = smem;
  stage_coefficients(S, sC);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int s = blockIdx.x * kWarpsPerBlock + wib;
  if (s >= P.W) return;
  WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
  double* rec = P.rec_src + (size_t)s * Lo.rec;
  double b, el;
  df bdf;
  load_record(Lo, rec, wm, lane, b, el);
  warp_eval_any<PR, NJ, NC>(S, sC, L, wm, lane, nullptr, b, bdf, el);
  if (!isfinite(el) || !isfinite(b)) {
    if (lane == 0) atomicOr(P.err, kErrNonFinite);
  }
  store_record(Lo, rec, wm, lane, b, el);
}

// ----------------------------------------------------------------------------
// Tail helpers of the interval kernel. Walkers make Poisson-distributed
// numbers of jumps, so at the end of an interval most warps of a block have
// no walker left while a few still run one. A warp whose fetch finds the
// queue empty attaches to a warp of its block that still runs a walker and,
// in every evaluation that warp publishes (projected columns, caches, local
// energy and Jastrow sums ready), takes chunks of 32 of its lattice moves.
// Owner and helpers run the same inlined move code (one loop of the kernel
// serves both roles), so a rate has the same bits whoever computes it and
// no second copy of the move code competes for the instruction cache. Every
// wait is bounded (kTeamSpin polls with a short sleep); one that runs out
// sets kErrTimeout in the error word and gives up, reported to the host as
// LRDMC_ERR_TIMEOUT, never a hang.
// ----------------------------------------------------------------------------
constexpr int kMaxIntervalWarps = 16;
struct TeamSlot {
  int attach;  // bit 31: closed to helpers; bits 0-30: helpers attached
  int pub;     // published evaluation (generation << 4 | participants), or kTeamRelease
  int next;    // next chunk of moves of the published evaluation
  int done;    // helpers finished with the published evaluation
  int gen;     // the owner's generation counter
  int pad[3];
};
constexpr int kTeamClosed = (int)0x80000000;
constexpr int kTeamRelease = -1;
constexpr int kTeamSpin = 1 << 22;

__device__ __forceinline__ int ld_vol(const int* p) { return *(const volatile int*)p; }

// Owner, after the evaluation's first part: the number of helpers taking
// part (0: alone; a helper that attaches later joins at the next one).
__device__ __forceinline__ int team_publish(TeamSlot* t, int lane)
{
  int nh = 0;
  if (lane == 0) {
    nh = ld_vol(&t->attach);
    nh = nh < 0 ? 0 : (nh > 15 ? 15 : nh);
  }
  nh = __shfl_sync(FULL_MASK, nh, 0);
  if (nh == 0) return 0;
  __threadfence_block();  // this lane's writes of the evaluation state
  __syncwarp();
  if (lane == 0) {
    const int g = t->gen + 1;
    t->gen = g;
    t->next = 0;
    t->done = 0;
    __threadfence_block();
    atomicExch(&t->pub, (g << 4) | nh);
  }
  __syncwarp();
  return nh;
}

// The moves of an evaluation in chunks of 32: alone (t == nullptr) in
// order, or taken in turn from t->next by the owner and its helpers.
template <class NT, bool NJ, bool NC>
__device__ __forceinline__ void chunked_moves(const SysDev& S, const LatDev& L, const WarpMem& wm, const BlockMem& bm,
                                              TeamSlot* t, int P, int lane)
{
  df* Td = reinterpret_cast<df*>(wm.T);
  // chunks of 16 moves in a team (more helpers take part in a small
  // system's moves; measured 3 % faster than 32 on the bench workload)
#ifndef LRDMC_TEAM_CHUNK
#define LRDMC_TEAM_CHUNK 16
#endif
  const int cs = t ? LRDMC_TEAM_CHUNK : 32;
  for (int c0 = 0;; c0 += 32) {
    if (t) {
      int c = 0;
      if (lane == 0) c = atomicAdd(&t->next, cs);
      c0 = __shfl_sync(FULL_MASK, c, 0);
    }
    if (c0 >= P) break;
    if (lane < cs && c0 + lane < P) candidate_m<NT, NJ, NC>(S, L, wm, bm, c0 + lane, Td, nullptr);
  }
  if (t) __threadfence_block();
  __syncwarp();
}

// Owner: wait until the nh helpers of the published evaluation are done.
__device__ __forceinline__ void team_wait_helpers(TeamSlot* t, int nh, int lane, int* err)
{
  if (lane == 0) {
    int it = 0;
    while (ld_vol(&t->done) < nh && ++it < kTeamSpin) __nanosleep(32);
    if (it >= kTeamSpin) atomicOr(err, kErrTimeout);
    __threadfence_block();
  }
  __syncwarp();
}

// Owner, when its walker's interval is over: close the slot and release
// the helpers attached to it.
__device__ __forceinline__ void team_close(TeamSlot* t, int lane)
{
  if (lane == 0) {
    atomicOr(&t->attach, kTeamClosed);
    atomicExch(&t->pub, kTeamRelease);
  }
  __syncwarp();
}

__device__ __forceinline__ void team_open(TeamSlot* t, int lane)
{
  if (lane == 0) {
    t->pub = 0;
    __threadfence_block();
    atomicExch(&t->attach, 0);
  }
  __syncwarp();
}

// Helper: attach to the open slot of the block with the fewest helpers;
// returns the owner's warp (or -1: no warp of the block runs a walker) and
// the helper's index among that owner's helpers.
__device__ __forceinline__ int team_attach(TeamSlot* slots, int nw, int wib, int lane, int& kidx)
{
  int o = -1, kk = 0;
  if (lane == 0) {
    for (int tries = 0; tries < 64 && o < 0; ++tries) {
      int best = -1, bc = 0x7fffffff;
      for (int q = 0; q < nw; ++q) {
        const int a = ld_vol(&slots[q].attach);
        if (q == wib || a < 0) continue;  // itself, or closed (bit 31)
        if (a < bc) { bc = a; best = q; }
      }
      if (best < 0) break;
      if (atomicCAS(&slots[best].attach, bc, bc + 1) == bc) { o = best; kk = bc; }
    }
  }
  kidx = __shfl_sync(FULL_MASK, kk, 0);
  return __shfl_sync(FULL_MASK, o, 0);
}

// Helper: wait for an evaluation of its owner it takes part in (returns
// its generation), a release (-1) or a timeout (-2, reported).
__device__ __forceinline__ int team_wait_publication(TeamSlot* t, int kidx, int last, int lane, int* err)
{
  int g = 0;
  if (lane == 0) {
    int it = 0;
    for (;;) {
      const int pub = ld_vol(&t->pub);
      if (pub == kTeamRelease) { g = -1; break; }
      if ((pub >> 4) > last && kidx < (pub & 15)) { g = pub >> 4; break; }
      if (++it >= kTeamSpin) { g = -2; atomicOr(err, kErrTimeout); break; }
      __nanosleep(64);
    }
    __threadfence_block();
  }
  g = __shfl_sync(FULL_MASK, g, 0);
  __syncwarp();  // orders lane 0's observation before every lane's reads
  return g;
}

__shared__ TeamSlot g_team[kMaxIntervalWarps];

// Per-warp state of the interval loop that the move code does not need: it
// lives in shared memory (written by lane 0, read by the whole warp after a
// __syncwarp), so that the registers of the move code are the same as in a
// loop without helpers.
struct WarpState {
  double tau_left, logw, b, el;
  unsigned long long m;
  df bdf;
  int s, jumps, finish;
  int owner, kidx, last;
};
__shared__ WarpState g_ws[kMaxIntervalWarps];

// The interval loop of the FP32-pipe evaluations (double-float and FP32):
// each warp is an owner while it runs a walker (the same steps, draws and
// arithmetic as the loop of the FP64 mode below), then a helper of the
// warps of its block that still run one.
template <class NT, int PR, bool NJ, bool NC>
__device__ __forceinline__ void interval_team(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P,
                                              double* sC, uint64_t k, bool recompute, int lane, int wib)
{
  typedef Ar<NT> A;
  const int P_moves = S.N * 6 * L.G;
  const BlockMem bm = block_mem(S, sC);
  TeamSlot* mine = &g_team[wib];
  WarpState& st = g_ws[wib];
  enum { kNeed, kOwner, kSearch, kHelper, kDone };
  int mode = kNeed;
  for (;;) {
    if (mode == kNeed) {
      int idx = 0;
      if (lane == 0) idx = atomicAdd(P.counter, 1);
      idx = __shfl_sync(FULL_MASK, idx, 0);
      if (idx >= P.W) {
        // out of walkers: a kernel launched after this one with programmatic
        // stream serialization (the pipelined batch) may start on the SMs
        // this block frees
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        mode = P.helpers ? kSearch : kDone;
      } else {
        if (P.helpers) team_open(mine, lane);
        const int s = bounded(P.order[idx], P.W, P.err);
        const WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
        double b, el;
        load_record(Lo, P.rec_src + (size_t)bounded(P.parent[s], P.W, P.err) * Lo.rec, wm, lane, b, el);
        if (recompute) {
          double rs = 0.0;
          bool ok = warp_inverse(S, sC, wm.x, 0, wm.A, wm.scr, lane, &rs);
          ok = ok && warp_inverse(S, sC, wm.x, 1, wm.A + Lo.nu * Lo.nu, wm.scr, lane, &rs);
          if (!ok && lane == 0) atomicOr(P.err, kErrSingular);
          if (lane == 0 && isfinite(rs)) atomicMax(P.resid, (unsigned long long)__double_as_longlong(rs));
        }
        if (lane == 0) {
          st.s = s;
          st.b = b;
          st.el = el;
          st.bdf = df_from_double(b);
          st.tau_left = P.tau;
          st.logw = 0.0;
          st.jumps = 0;
          st.m = 0;
          st.finish = 0;
        }
        __syncwarp();
        mode = kOwner;
      }
    }
    if (mode == kDone) break;
    int target = wib, nh = 0;
    if (mode == kOwner) {
      const WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
      const double b = st.b, el = st.el, tau_left = st.tau_left;
      const df bdf = st.bdf;
      bool over = st.finish != 0;
      double t = 0.0, logw = st.logw;
      uint64_t b0[4], b1[4];
      if (!over) {
        // both draws of this iteration at once: even lanes compute the
        // (waiting time, heat bath) block, odd lanes the rotation block
        uint64_t cb[4] = {(uint64_t)st.s, k, (uint64_t)st.m, (lane & 1) ? kTagRot : kTagTimeHB};
        philox4x64_10(cb, P.seed, 0ull);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          b0[j] = shfl_u64(cb[j], 0);
          b1[j] = shfl_u64(cb[j], 1);
        }
        if (PR == LRDMC_PRECISION_DF64)
          t = b > 0.0 ? df_to_double(df_div(df_neg(df_log(df_u01(b0[0]), S.D.exp.K, bm.tab)), bdf)) : INFINITY;
        else
          t = b > 0.0 ? (double)(-logf(f_u01(b0[0])) / bdf.hi) : INFINITY;
        if (t >= tau_left) {
          logw -= tau_left * (el - P.e_trial);
          over = true;
        }
      }
      int i = 0, pick = -1;
      if (!over) {
        logw -= t * (el - P.e_trial);
        // heat bath over the cached rates
        int lastc;
        if (PR == LRDMC_PRECISION_DF64)
          warp_scan_m<df>(reinterpret_cast<const df*>(wm.T), P_moves, lane, df_mul(df_u01(b0[1]), bdf), &pick,
                          &lastc);
        else
          warp_scan_m<float>(reinterpret_cast<const df*>(wm.T), P_moves, lane, f_u01(b0[1]) * bdf.hi, &pick,
                             &lastc);
        if (pick < 0) pick = lastc;
        if (pick < 0) {  // no allowed move: cannot happen with b > 0
          if (lane == 0) atomicOr(P.err, kErrNonFinite);
          over = true;
        }
      }
      double pnew[3];
      if (!over) {
        const int per_e = 6 * L.G;
        i = pick / per_e;
        const int rem = pick - i * per_e, g = rem / 6, kx = (rem % 6) >> 1;
        const double sign = (pick & 1) ? -1.0 : 1.0, h = g ? L.ap : L.a;
#pragma unroll
        for (int d = 0; d < 3; ++d) pnew[d] = wm.x[3 * i + d] + sign * h * wm.R[3 * d + kx];
        bool sm_ok;
        if (PR != LRDMC_PRECISION_FP32) {
          // the parity modes keep the update in IEEE double: near a node the
          // update amplifies rounding by the condition number of the Slater
          // matrix, and a double-float update (2^-48) parts trajectories
          // from the FP64 reference in rare walkers
          sm_ok = warp_sm_update<PR>(S, sC, wm, i, pnew, lane);
        } else {
          // the new position as a double-float (the shared-memory
          // double-float copies of x and R belong to the last evaluation,
          // which for the first jump of an interval may have been another
          // walker's)
          df pd[3] = {df_from_double(pnew[0]), df_from_double(pnew[1]), df_from_double(pnew[2])};
          sm_ok = warp_sm_update_df(S, bm, wm, i, pd, lane);
        }
        if (!sm_ok) {
          if (lane == 0) atomicOr(P.err, kErrSingular);
          over = true;
        }
      }
      if (over) {
        if (P.helpers) team_close(mine, lane);
        store_record(Lo, P.rec_dst + (size_t)st.s * Lo.rec, wm, lane, b, el);
        if (lane == 0) {
          const int s = st.s;
          P.logw[s] = logw;
          P.wgt[s] = exp(logw);
          P.el_end[s] = el;
          P.jumps[s] = st.jumps;
        }
        __syncwarp();
        mode = kNeed;
        continue;
      }
      if (lane == 0) {
        st.logw = logw;
        st.tau_left = tau_left - t;
      }
      if (lane < 3) wm.x[3 * i + lane] = pnew[lane];
      __syncwarp();
      rotation_matrix_warp<PR>(b1, wm.R, lane, S);
      __syncwarp();
      double eln;
      eval_prelude_m<NT, NJ, NC>(S, sC, L, wm, lane, eln);
      if (lane == 0) st.el = eln;
      if (P.helpers) nh = team_publish(mine, lane);
    } else {
      if (mode == kSearch) {
        int kidx;
        const int o = team_attach(g_team, blockDim.x >> 5, wib, lane, kidx);
        if (o < 0) {
          mode = kDone;
          continue;
        }
        if (lane == 0) {
          st.owner = bounded(o, blockDim.x >> 5, P.err);
          st.kidx = kidx;
          st.last = 0;
        }
        __syncwarp();
        mode = kHelper;
      }
      const int gw = team_wait_publication(&g_team[st.owner], st.kidx, st.last, lane, P.err);
      if (gw == -2) {
        mode = kDone;
        continue;
      }
      if (gw == -1) {
        mode = kSearch;
        continue;
      }
      if (lane == 0) st.last = gw;
      target = st.owner;
    }
    // the moves of the target walker's evaluation: one copy of the move
    // code for the owner alone, the owner with helpers, and the helpers
    {
      const WarpMem twm = warp_mem(Lo, S, sC + Lo.head + target * Lo.smem_warp);
      chunked_moves<NT, NJ, NC>(S, L, twm, bm, (mode == kHelper || nh > 0) ? &g_team[target] : nullptr, P_moves,
                                lane);
    }
    if (mode == kHelper) {
      if (lane == 0) atomicAdd(&g_team[target].done, 1);
      __syncwarp();
      continue;
    }
    if (nh > 0) team_wait_helpers(mine, nh, lane, P.err);
    const NT btot = warp_scan_m<NT>(reinterpret_cast<const df*>(warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp).T),
                                    P_moves, lane, A::zero(), nullptr, nullptr);
    const double b = A::to_double(btot);
    if (lane == 0) {
      st.bdf = A::store(btot);
      st.b = b;
      st.jumps = st.jumps + 1;
      int fin = 0;
      if (!isfinite(st.el) || !isfinite(b)) {
        atomicOr(P.err, kErrNonFinite);
        fin = 1;
      }
      if (st.m + 1 >= (unsigned long long)kMaxItersPerInterval) {
        atomicOr(P.err, kErrIters);
        fin = 1;
      }
      st.finish = fin;
      st.m = st.m + 1;
    }
    __syncwarp();
  }
}

// One interval of length tau for every walker slot (continuous-time
// projection of the cited LRDMC method): wait for an exponential time of
// rate b_x, decrease log w by (E_L - E_T) times the time spent, and at the
// end of the wait jump to move c with probability T_c / b_x.
#ifndef LRDMC_INTERVAL_MIN_BLOCKS
#define LRDMC_INTERVAL_MIN_BLOCKS 1
#endif
template <int PREC>
__global__ void __launch_bounds__(kMaxIntervalWarps * 32, LRDMC_INTERVAL_MIN_BLOCKS)
k_interval(const __grid_constant__ SysDev S, const Layout Lo, const LatDev L, const PopDev P)
{
  constexpr int PR = PREC & 3;         // the arithmetic (LRDMC_PRECISION_*)
  constexpr bool NJ = (PREC & 8) != 0;  // the neural pair term is set
  constexpr bool NC = (PREC & 4) != 0;  // the layout has no evaluation caches
  extern __shared__ double smem[];
  double* sC = smem;
  // interval k from the device counter (advanced by k_comb_parents); the inverse
  // Slater matrices are recomputed at the start of every recompute_every-th
  // interval
  const uint64_t k = *P.kdev;
  const bool recompute = k > 0 && P.recompute_every > 0 && k % (uint64_t)P.recompute_every == 0;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (PR != LRDMC_PRECISION_FP64 && lane == 0) {
    g_team[wib].attach = kTeamClosed;
    g_team[wib].pub = 0;
    g_team[wib].next = 0;
    g_team[wib].done = 0;
    g_team[wib].gen = 0;
  }
  stage_coefficients(S, sC);  // ends with __syncthreads
  if constexpr (PR != LRDMC_PRECISION_FP64) {
    if (PR == LRDMC_PRECISION_DF64) interval_team<df, PR, NJ, NC>(S, Lo, L, P, sC, k, recompute, lane, wib);
    else interval_team<float, PR, NJ, true>(S, Lo, L, P, sC, k, recompute, lane, wib);
  } else {
    // the FP64 mode: every warp alone
    WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
    const int P_moves = S.N * 6 * L.G;
    const BlockMem bm = block_mem(S, sC);
    for (;;) {
      int idx = 0;
      if (lane == 0) idx = atomicAdd(P.counter, 1);
      idx = __shfl_sync(FULL_MASK, idx, 0);
      if (idx >= P.W) {
        // out of walkers: a kernel launched after this one with programmatic
        // stream serialization (the pipelined batch) may start on the SMs
        // this block frees
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        break;
      }
      const int s = bounded(P.order[idx], P.W, P.err);
      const int src = bounded(P.parent[s], P.W, P.err);
      double b, el;
      load_record(Lo, P.rec_src + (size_t)src * Lo.rec, wm, lane, b, el);
      df bdf = df_from_double(b);
      if (recompute) {
        double rs = 0.0;
        bool ok = warp_inverse(S, sC, wm.x, 0, wm.A, wm.scr, lane, &rs);
        ok = ok && warp_inverse(S, sC, wm.x, 1, wm.A + Lo.nu * Lo.nu, wm.scr, lane, &rs);
        if (!ok && lane == 0) atomicOr(P.err, kErrSingular);
        if (lane == 0 && isfinite(rs)) atomicMax(P.resid, (unsigned long long)__double_as_longlong(rs));
      }
      double tau_left = P.tau, logw = 0.0;
      int jumps = 0;
      for (uint64_t m = 0;; ++m) {
        // both draws of this iteration at once: even lanes compute the
        // (waiting time, heat bath) block, odd lanes the rotation block
        uint64_t cb[4] = {(uint64_t)s, k, m, (lane & 1) ? kTagRot : kTagTimeHB};
        philox4x64_10(cb, P.seed, 0ull);
        uint64_t b0[4], b1[4];
  #pragma unroll
        for (int j = 0; j < 4; ++j) {
          b0[j] = shfl_u64(cb[j], 0);
          b1[j] = shfl_u64(cb[j], 1);
        }
        double t;
        if (PR == LRDMC_PRECISION_DF64)
          t = b > 0.0 ? df_to_double(df_div(df_neg(df_log(df_u01(b0[0]), S.D.exp.K, bm.tab)), bdf)) : INFINITY;
        else if (PR == LRDMC_PRECISION_FP32)
          t = b > 0.0 ? (double)(-logf(f_u01(b0[0])) / bdf.hi) : INFINITY;
        else
          t = b > 0.0 ? -log(to_u01(b0[0])) / b : INFINITY;
        if (t >= tau_left) {
          logw -= tau_left * (el - P.e_trial);
          break;
        }
        logw -= t * (el - P.e_trial);
        tau_left -= t;
        // heat bath over the cached rates
        int pick, last;
        if (PR == LRDMC_PRECISION_DF64)
          warp_scan_m<df>(reinterpret_cast<const df*>(wm.T), P_moves, lane, df_mul(df_u01(b0[1]), bdf), &pick, &last);
        else if (PR == LRDMC_PRECISION_FP32)
          warp_scan_m<float>(reinterpret_cast<const df*>(wm.T), P_moves, lane, f_u01(b0[1]) * bdf.hi, &pick, &last);
        else
          warp_scan(wm.T, P_moves, lane, to_u01(b0[1]) * b, &pick, &last);
        if (pick < 0) pick = last;
        if (pick < 0) {  // no allowed move: cannot happen with b > 0
          if (lane == 0) atomicOr(P.err, kErrNonFinite);
          break;
        }
        const int per_e = 6 * L.G;
        const int i = pick / per_e, rem = pick - i * per_e, g = rem / 6, kx = (rem % 6) >> 1;
        const double sign = (pick & 1) ? -1.0 : 1.0, h = g ? L.ap : L.a;
        double pnew[3];
  #pragma unroll
        for (int d = 0; d < 3; ++d) pnew[d] = wm.x[3 * i + d] + sign * h * wm.R[3 * d + kx];
        bool sm_ok;
        if (PR != LRDMC_PRECISION_FP32) {
          // the parity modes keep the update in IEEE double: near a node the
          // update amplifies rounding by the condition number of the Slater
          // matrix, and a double-float update (2^-48) parts trajectories from
          // the FP64 reference in rare walkers
          sm_ok = warp_sm_update<PR>(S, sC, wm, i, pnew, lane);
        } else {
          // the new position as a double-float (the shared-memory double-float
          // copies of x and R belong to the last evaluation, which for the
          // first jump of an interval may have been another walker's)
          df pd[3] = {df_from_double(pnew[0]), df_from_double(pnew[1]), df_from_double(pnew[2])};
          sm_ok = warp_sm_update_df(S, bm, wm, i, pd, lane);
        }
        if (!sm_ok) {
          if (lane == 0) atomicOr(P.err, kErrSingular);
          break;
        }
        if (lane < 3) wm.x[3 * i + lane] = pnew[lane];
        __syncwarp();
        rotation_matrix_warp<PR>(b1, wm.R, lane, S);
        __syncwarp();
        warp_eval_any<PR, NJ, NC>(S, sC, L, wm, lane, nullptr, b, bdf, el);
        ++jumps;
        if (!isfinite(el) || !isfinite(b)) {
          if (lane == 0) atomicOr(P.err, kErrNonFinite);
          break;
        }
        if (m + 1 >= (uint64_t)kMaxItersPerInterval) {
          if (lane == 0) atomicOr(P.err, kErrIters);
          break;
        }
      }
      store_record(Lo, P.rec_dst + (size_t)s * Lo.rec, wm, lane, b, el);
      if (lane == 0) {
        P.logw[s] = logw;
        P.wgt[s] = exp(logw);
        P.el_end[s] = el;
        P.jumps[s] = jumps;
      }
      __syncwarp();
    }
    // Launched early behind another system's interval kernel (pipelined
    // batch): this grid does not read that kernel's results, but it finishes
    // only after that kernel has, so that work after the chain in the stream
    // sees every kernel of the chain complete. Without a prerequisite grid
    // the wait returns at once.
  }
  if (threadIdx.x == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Reconfiguration at the end of interval k, spread over G blocks of
// kCombThreads threads; block g owns the R = ceil(W/G) slots from g R. Its
// FP64 work (running sums, comb targets and comparisons) used to run on one
// SM, whose FP64 pipe took 38 us for 4096 walkers. Two kernels:
//   k_comb_sums     per block: running weight sums of its slots from the
//                   block's start (P.cum) and the block's totals (weights,
//                   w E_L, jumps)
//   k_comb_parents  per block: the block offsets off[g] (the same sequential
//                   sum in every block), the comb parents of its slots, and
//                   the next interval's processing order of its slots; the
//                   last block to finish writes the trace entry and clears
//                   the counters.
// Running sums: within a block, lane i of the first kCombLanes lanes sums
// its consecutive slots from zero (l_i(s)), and O_0 = 0, O_{i+1} = O_i +
// l_i(last slot of i) sequentially; c(s) = O_i + l_i(s). Over the blocks
// off[0] = 0, off[g+1] = off[g] + c(last slot of g), and C_s = off[g] +
// c(s). Each boundary repeats the rounding of the sum that ends the previous
// part, so C is non-decreasing (rounding is monotone, weights are >= 0) and
// slot t's parent is well defined: the smallest s with
// (t + xi) C_{W-1} / W < C_s, else W - 1. The sequential parts are kept
// short (FP64 additions have a long latency on this GPU): kCombLanes lanes
// per block, a few dozen blocks.
//
// Processing order of the next interval, longest expected first: a slot's
// number of jumps is about tau times the total rate b of the walker it
// receives. Each block sorts its slots by that b (64 buckets over the
// block's range, descending), and the blocks' sorted lists are dealt round
// robin into P.order: the r-th slot of every block comes before the
// (r+1)-th of any. The blocks are samples of the population, so this is
// close to a global sort, with no pass over the whole population. The order
// affects no result, only the tail of the next interval.
constexpr int kCombLanes = 16;

__device__ __forceinline__ int comb_slots(int W, int G) { return (W + G - 1) / G; }

__global__ void __launch_bounds__(kCombThreads) k_comb_sums(const PopDev P)
{
  // the parents kernel is launched behind this one with programmatic stream
  // serialization; its blocks may take their SMs now and wait for this grid
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int NW = kCombThreads / 32;
  __shared__ double s_e[NW], s_tot[kCombLanes];
  __shared__ long long s_j[NW];
  const int W = P.W, G = gridDim.x, g = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int R = comb_slots(W, G);
  const int b0 = min(W, g * R), b1 = min(W, b0 + R);
  // the block's totals other than the weights: every thread
  double swe = 0.0;
  long long sj = 0;
  for (int s = b0 + t; s < b1; s += kCombThreads) {
    swe += P.wgt[s] * P.el_end[s];
    sj += P.jumps[s];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    swe += __shfl_xor_sync(FULL_MASK, swe, o);
    sj += __shfl_xor_sync(FULL_MASK, sj, o);
  }
  if (lane == 0) { s_e[wid] = swe; s_j[wid] = sj; }
  // the running sums: the first kCombLanes lanes, each a run of slots
  const int per = (b1 - b0 + kCombLanes - 1) / kCombLanes;
  const int lo = min(b1, b0 + t * per), hi = min(b1, lo + per);
  if (t < kCombLanes) {
    double l = 0.0;
    for (int s = lo; s < hi; ++s) l += P.wgt[s];
    s_tot[t] = l;
  }
  __syncthreads();
  if (t == 0) {
    double o = 0.0;
    for (int i = 0; i < kCombLanes; ++i) {
      const double ti = s_tot[i];
      s_tot[i] = o;
      o += ti;
    }
    P.part[g].w = o;  // = c(last slot of the block): the last lane with slots ends there
  }
  if (t == 32) {  // fixed-order sums of the warps' totals
    double es = 0.0;
    long long js = 0;
    for (int q = 0; q < NW; ++q) {
      es += s_e[q];
      js += s_j[q];
    }
    P.part[g].swe = es;
    P.part[g].jumps = js;
  }
  __syncthreads();
  if (t < kCombLanes) {
    const double O = s_tot[t];
    double c = 0.0;
    for (int s = lo; s < hi; ++s) {
      c += P.wgt[s];
      P.cum[s] = O + c;
    }
  }
}

// Running sum C_s of the comb: from shared memory when the population's sums
// were staged there, else off[block of s] + P.cum[s] (the same number).
__device__ __forceinline__ double comb_C(const double* s_cum, const double* s_off, const double* cum, int R, int s,
                                        bool in_smem)
{
  return in_smem ? s_cum[s] : s_off[s / R] + __ldcg(cum + s);
}

// Adds one to the shared counter of bucket q for every lane of the warp
// (lanes with q < 0 take no part) and returns this lane's old count plus
// its rank among the lanes with the same q: one shared-memory atomic per
// distinct bucket of the warp instead of one per lane.
__device__ __forceinline__ int bucket_take(int* cnt, int q, int lane)
{
  const unsigned peers = __match_any_sync(FULL_MASK, q);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader && q >= 0) base = atomicAdd(&cnt[q], __popc(peers));
  base = __shfl_sync(FULL_MASK, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// Position in P.order of the r-th slot (in the block's sorted order) of
// block g: the blocks hold R slots but for a shorter last non-empty block
// (Rl slots) and empty ones after it (Gn non-empty blocks); the first Rl
// ranks of all Gn blocks come first, round robin, then the further ranks of
// the Gn - 1 full blocks. A bijection of the slots onto 0..W-1.
__device__ __forceinline__ int comb_order_pos(int g, int r, int Gn, int Rl)
{
  return r < Rl ? r * Gn + g : Rl * Gn + (r - Rl) * (Gn - 1) + g;
}

__global__ void __launch_bounds__(kCombThreads) k_comb_parents(const PopDev P, const double* rec_next,
                                                              int rec_stride, int off_b)
{
  extern __shared__ double s_cum[];  // the running sums C_s (W <= kReconfigSmemW)
  __shared__ double s_off[kMaxCombBlocks + 1];
  __shared__ double s_pw[kMaxCombBlocks];
  __shared__ float s_lo[kCombThreads / 32], s_hi[kCombThreads / 32];
  __shared__ int s_cnt[64];
  __shared__ int s_last;
  const int W = P.W, G = gridDim.x, g = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int R = comb_slots(W, G);
  const bool in_smem = W <= kReconfigSmemW;
  // everything below reads the sums kernel's results
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const uint64_t k = *P.kdev;
  if (t < 64) s_cnt[t] = 0;
  for (int h = t; h < G; h += kCombThreads) s_pw[h] = __ldcg(&P.part[h].w);
  __syncthreads();
  if (t == 0) {
    double o = 0.0;
    for (int h = 0; h < G; ++h) {
      s_off[h] = o;
      o += s_pw[h];
    }
    s_off[G] = o;
  }
  __syncthreads();
  if (in_smem) {
    constexpr int U = 8;
    for (int s0 = 0; s0 < W; s0 += U * kCombThreads) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + u * kCombThreads + t;
        v[u] = s < W ? __ldcg(P.cum + s) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + u * kCombThreads + t;
        if (s < W) s_cum[s] = s_off[s / R] + v[u];
      }
    }
    __syncthreads();
  }
  const double total = s_off[G];
  double uu[4];
  draw_uniforms(P.seed, kSlotGlobal, k, 0, kTagComb, uu);
  const double xi = uu[0];
  // t -> (t + xi) total / W; for W a power of two the product with 1/W is
  // the same number as the quotient (an exact scaling)
  const bool w_pow2 = (W & (W - 1)) == 0;
  const double inv_w = 1.0 / (double)W;
  const int b0 = min(W, g * R), b1 = min(W, b0 + R);
  const int chunk = (b1 - b0 + kCombThreads - 1) / kCombThreads;
  const int lo = min(b1, b0 + t * chunk), hi = min(b1, lo + chunk);
  // The targets grow with the slot, so the parents do too: a thread searches
  // for its first slot's parent, then steps forward from the previous one
  // (up to 8 steps, else a search over the rest), with the same comparisons.
  // The rate b of each slot's parent goes to the slot's bq byte's place in
  // shared memory (as a float, in the dynamic area after the sums).
  float* s_b = reinterpret_cast<float*>(s_cum + (in_smem ? W : 0));
  int a = 0;
  float bmin = INFINITY, bmax = -INFINITY;
  for (int tt = lo; tt < hi; ++tt) {
    const double num = ((double)tt + xi) * total;
    const double target = w_pow2 ? num * inv_w : num / (double)W;
    int steps = 0;
    while (tt > lo && steps < 8 && a < W - 1 && !(target < comb_C(s_cum, s_off, P.cum, R, a, in_smem))) {
      ++a;
      ++steps;
    }
    if (tt == lo || (steps == 8 && a < W - 1 && !(target < comb_C(s_cum, s_off, P.cum, R, a, in_smem)))) {
      int bnd = W - 1;
      while (a < bnd) {
        const int mid = (a + bnd) >> 1;
        if (target < comb_C(s_cum, s_off, P.cum, R, mid, in_smem)) bnd = mid; else a = mid + 1;
      }
    }
    a = bounded(a, W, P.err);
    P.parent[tt] = a;
    const float bt = (float)rec_next[(size_t)a * rec_stride + off_b];
    s_b[bounded(tt - b0, R, P.err)] = bt;
    bmin = fminf(bmin, bt);
    bmax = fmaxf(bmax, bt);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bmin = fminf(bmin, __shfl_xor_sync(FULL_MASK, bmin, o));
    bmax = fmaxf(bmax, __shfl_xor_sync(FULL_MASK, bmax, o));
  }
  if (lane == 0) { s_lo[wid] = bmin; s_hi[wid] = bmax; }
  __syncthreads();
  // the block's slots by bucket of b, descending: counts, bases, positions
  float gmin = INFINITY, gmax = -INFINITY;
  for (int q = 0; q < kCombThreads / 32; ++q) {
    gmin = fminf(gmin, s_lo[q]);
    gmax = fmaxf(gmax, s_hi[q]);
  }
  const float scale = (gmax > gmin) ? 64.0f / (gmax - gmin) : 0.0f;
  const int n = b1 - b0;
  const int rounds = (n + kCombThreads - 1) / kCombThreads;  // warp-uniform
  for (int i = 0; i < rounds; ++i) {
    const int j = i * kCombThreads + t;
    int q = -1;
    if (j < n) {
      q = (int)((s_b[j] - gmin) * scale);
      q = 63 - min(63, max(0, q));
    }
    bucket_take(s_cnt, q, lane);
  }
  __syncthreads();
  if (t < 32) {  // exclusive scan of the 64 bucket counts (two per lane)
    const int c0 = s_cnt[2 * t], c1 = s_cnt[2 * t + 1];
    int incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL_MASK, incl, o);
      if (lane >= o) incl += y;
    }
    const int ex = incl - c0 - c1;
    s_cnt[2 * t] = ex;
    s_cnt[2 * t + 1] = ex + c0;
  }
  __syncthreads();
  const int Gn = (W + R - 1) / R;  // blocks with slots
  const int Rl = W - (Gn - 1) * R;  // slots of the last of them
  for (int i = 0; i < rounds; ++i) {
    const int j = i * kCombThreads + t;
    int q = -1;
    if (j < n) {
      q = (int)((s_b[j] - gmin) * scale);
      q = 63 - min(63, max(0, q));
    }
    const int r = bucket_take(s_cnt, q, lane);
    if (j < n) P.order[bounded(comb_order_pos(g, r, Gn, Rl), W, P.err)] = b0 + j;
  }
  // the last block to finish writes the trace entry
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(P.ticket, 1) == G - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (t < 32) {  // fixed-order sums over the blocks' totals
    double swe = 0.0;
    long long sj = 0;
    for (int h = t; h < G; h += 32) {
      swe += __ldcg(&P.part[h].swe);
      sj += __ldcg(&P.part[h].jumps);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      swe += __shfl_xor_sync(FULL_MASK, swe, o);
      sj += __shfl_xor_sync(FULL_MASK, sj, o);
    }
    if (t == 0) {
      const uint64_t kt = bounded(k, P.trace_cap, P.err);  // the trace slot
      P.trace[kt] = swe / total;
      P.trace[P.trace_cap + kt] = total / (double)W;
      P.trace[2 * P.trace_cap + kt] = (double)sj / (double)W;
      // the Sherman-Morrison residual measured at this interval's recompute
      // (-1: no recompute at this interval), then cleared for the next one
      const bool recomputed = k > 0 && P.recompute_every > 0 && k % (uint64_t)P.recompute_every == 0;
      P.trace[3 * P.trace_cap + kt] = recomputed ? __longlong_as_double((long long)*P.resid) : -1.0;
      *P.resid = 0ull;
      *P.moves += (unsigned long long)sj;
      *P.counter = 0;
      *P.ticket = 0;
      // every block has read k before taking its ticket: advance it
      *P.kdev = k + 1;
    }
  }
}

// Stateless evaluation of configuration c (one warp): inverses from x, then
// one evaluation of every lattice move and of the local energy. Returns
// false, with no output written, for a singular Slater matrix. The body of
// k_evaluate and of k_evaluate_static, which differ only in where they
// report that.
template <int PREC>
__device__ __forceinline__ bool evaluate_config(const SysDev& S, const Layout& Lo, const LatDev& L, const double* sC,
                                                int c, int lane, int wib, const double* x, const double* rot,
                                                double* ratio, double* T, double* b_out, double* el_out)
{
  constexpr int PR = PREC & 3;         // the arithmetic (LRDMC_PRECISION_*)
  constexpr bool NJ = (PREC & 8) != 0;  // the neural pair term is set
  constexpr bool NC = (PREC & 4) != 0;  // the layout has no evaluation caches
  WarpMem wm = warp_mem(Lo, S, const_cast<double*>(sC) + Lo.head + wib * Lo.smem_warp);
  for (int j = lane; j < 3 * Lo.N; j += 32) wm.x[j] = x[(size_t)c * 3 * Lo.N + j];
  for (int j = lane; j < 9; j += 32) wm.R[j] = rot[(size_t)c * 9 + j];
  __syncwarp();
  bool ok = warp_inverse(S, sC, wm.x, 0, wm.A, wm.scr, lane);
  ok = ok && warp_inverse(S, sC, wm.x, 1, wm.A + Lo.nu * Lo.nu, wm.scr, lane);
  if (!ok) return false;
  const int P = S.N * 6 * L.G;
  double b, el;
  df bdf;
  warp_eval_any<PR, NJ, NC>(S, sC, L, wm, lane, ratio ? ratio + (size_t)c * P : nullptr, b, bdf, el);
  if (T)
    for (int j = lane; j < P; j += 32)
      T[(size_t)c * P + j] = (PR != LRDMC_PRECISION_FP64) ? df_to_double(reinterpret_cast<const df*>(wm.T)[j])
                                                            : wm.T[j];
  if (lane == 0) {
    if (b_out) b_out[c] = b;
    if (el_out) el_out[c] = el;
  }
  return true;
}

// Stateless evaluation of given configurations (one warp per configuration).
template <int PREC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_evaluate(const __grid_constant__ SysDev S, const Layout Lo, const LatDev L, int n,
           const double* x, const double* rot, double* ratio, double* T, double* b_out,
           double* el_out, int* err)
{
  extern __shared__ double smem[];
  double* sC = smem;
  stage_coefficients(S, sC);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.x * kWarpsPerBlock + wib;
  if (c >= n) return;
  if (!evaluate_config<PREC>(S, Lo, L, sC, c, lane, wib, x, rot, ratio, T, b_out, el_out) && lane == 0)
    atomicOr(err, kErrSingular);
}

// ----------------------------------------------------------------------------
// Host launchers.
// ----------------------------------------------------------------------------
static df split_ld(long double x)
{
  float h = (float)x;
  float l = (float)(x - (long double)h);
  return df_make(h, l);
}

void fill_df_constants(SysDev& S)
{
  DfSys& D = S.D;
  for (int I = 0; I < S.n_nuc; ++I) {
    for (int k = 0; k < 3; ++k) D.nuc[I][k] = split_ld(S.nuc[I][k]);
    D.Z[I] = split_ld(S.Z[I]);
    D.en_b1[I] = split_ld(S.en_b1[I]);
  }
  D.b_ee = split_ld(S.b_ee);
  D.c_par = split_ld(S.c_par);
  D.c_anti = split_ld(S.c_anti);
  D.en_b2 = split_ld(S.en_b2);
  for (int q = 0; q < S.n_shell; ++q) {
    D.sh[q].m = split_ld(S.sh[q].m);
    D.sh[q].zeta = split_ld(S.sh[q].zeta);
    for (int p = 0; p < kMaxPrim; ++p) {
      D.sh[q].alpha[p] = split_ld(S.sh[q].alpha[p]);
      D.sh[q].coef[p] = split_ld(S.sh[q].coef[p]);
    }
  }
  // Tang's table: 2^(j/64) and ln2/64, from long double arithmetic
  const long double ln2 = logl(2.0L);
  df c = split_ld(ln2 / 64.0L);
  D.exp.K.ln2_64_hi = c.hi;
  D.exp.K.ln2_64_lo = c.lo;
  D.exp.K.inv_ln2_64 = (float)(64.0L / ln2);
  D.exp.K.pad = 0.0f;
  for (int j = 0; j < 64; ++j) {
    df t = split_ld(exp2l((long double)j / 64.0L));
    D.exp.t[j] = make_float2(t.hi, t.lo);
  }
  long double f = 1.0L;
  for (int k = 0; k < 18; ++k) {
    if (k > 0) f *= (long double)k;
    D.inv_fact[k] = split_ld(1.0L / f);
  }
  D.half_pi = split_ld(2.0L * atanl(1.0L));
}

void fill_lattice_df(LatDev& L)
{
  L.a_df = split_ld(L.a);
  L.ap_df = split_ld(L.ap);
  L.inv2a2_df = split_ld(L.inv2a2);
  L.inv2ap2_df = split_ld(L.inv2ap2);
  L.p_coef_df = split_ld(L.p_coef);
}

static_assert(sizeof(SysDev) + sizeof(Layout) + sizeof(LatDev) + sizeof(PopDev) + 64 < 32764,
              "kernel parameters exceed the 32 KB limit");

Layout make_layout(const SysDev& S, bool caches)
{
  Layout Lo;
  Lo.N = S.N;
  Lo.nu = S.n_up;
  Lo.nd = S.n_dn;
  Lo.P_max = 12 * S.N;
  Lo.off_x = 0;
  Lo.off_au = 3 * S.N;
  Lo.off_ad = Lo.off_au + S.n_up * S.n_up;
  Lo.off_R = Lo.off_ad + S.n_dn * S.n_dn;
  Lo.off_T = Lo.off_R + 9;
  Lo.off_b = Lo.off_T + Lo.P_max;
  Lo.off_el = Lo.off_b + 1;
  Lo.rec = (Lo.off_el + 1 + 3) & ~3;
  const int n = S.n_up;
  int scr = 2 * n * n + n * S.n_ao;          // Gauss-Jordan + orbital rows
  int scr_sm = S.n_ao + 3 * n + n * n;       // Sherman-Morrison (FP64 or double-float)
  if (scr_sm > scr) scr = scr_sm;
  // The caches of the double-float evaluation (omitted when caches is false):
  // the electron-nucleus cache (8 df per electron and nucleus), and the pair
  // cache up to 24 electrons (beyond, its 4 df per pair would cost blocks
  // per SM), with room for the pair's Jastrow terms up to 12 electrons (used
  // with the neural term: the local energy then evaluates every pair once)
  Lo.n_pc = (caches && S.N <= 24) ? S.N * (S.N - 1) / 2 : 0;
  Lo.pcw = S.N <= 12 ? 8 : 4;
  Lo.enc = caches ? 1 : 0;
  Lo.smem_warp = 3 * S.N + S.n_up * S.n_up + S.n_dn * S.n_dn + 12 + Lo.P_max + S.N * S.n_ao + S.N +
                 (3 * S.N + 12) + Lo.pcw * Lo.n_pc + (Lo.enc ? 8 * S.N * S.n_nuc : 0) + scr;
  Lo.smem_warp = (Lo.smem_warp + 1) & ~1;
  Lo.head = ((2 * S.n_ao * S.n_mo + (S.n_ao * S.n_mo + 1) / 2 + 64) + 1) & ~1;
  Lo.smem_block_bytes = (int)sizeof(double) * (Lo.head + kWarpsPerBlock * Lo.smem_warp);
  return Lo;
}

static cudaError_t set_smem(const void* fn, int bytes)
{
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return cudaSuccess;
}

cudaError_t launch_init(const SysDev& S, const Layout& Lo, const PopDev& P, const double* x0,
                        cudaStream_t st)
{
  cudaError_t e = set_smem((const void*)k_init, Lo.smem_block_bytes);
  if (e != cudaSuccess) return e;
  int blocks = (P.W + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_init<<<blocks, kWarpsPerBlock * 32, Lo.smem_block_bytes, st>>>(S, Lo, P, x0);
  return cudaGetLastError();
}

// Kernel variant of a system: the arithmetic in bits 0-1 of the template
// argument, bit 2 for a double-float system whose layout has no evaluation
// caches, the neural pair term in bit 3 (kernels without a feature carry
// none of its code).
constexpr int kNoCacheBit = 4;
constexpr int kNjBit = 8;

#define LRDMC_DISPATCH_NJ(S, BASE, ...)                                            \
  do {                                                                             \
    if ((S).nj_on != 0) { constexpr int V = (BASE) | kNjBit; __VA_ARGS__; }        \
    else { constexpr int V = (BASE); __VA_ARGS__; }                                \
  } while (0)

#define LRDMC_DISPATCH(S, Lo, ...)                                                 \
  do {                                                                             \
    if ((S).precision == LRDMC_PRECISION_DF64) {                                   \
      if ((Lo).enc) LRDMC_DISPATCH_NJ(S, LRDMC_PRECISION_DF64, __VA_ARGS__);       \
      else LRDMC_DISPATCH_NJ(S, LRDMC_PRECISION_DF64 | kNoCacheBit, __VA_ARGS__);  \
    } else if ((S).precision == LRDMC_PRECISION_FP32) {                            \
      LRDMC_DISPATCH_NJ(S, LRDMC_PRECISION_FP32, __VA_ARGS__);                     \
    } else {                                                                       \
      LRDMC_DISPATCH_NJ(S, LRDMC_PRECISION_FP64, __VA_ARGS__);                     \
    }                                                                              \
  } while (0)

template <int PREC>
static cudaError_t launch_eval_all_t(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P,
                                     cudaStream_t st)
{
  cudaError_t e = set_smem((const void*)k_eval_all<PREC>, Lo.smem_block_bytes);
  if (e != cudaSuccess) return e;
  int blocks = (P.W + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_eval_all<PREC><<<blocks, kWarpsPerBlock * 32, Lo.smem_block_bytes, st>>>(S, Lo, L, P);
  return cudaGetLastError();
}

cudaError_t launch_eval_all(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P,
                            cudaStream_t st)
{
  LRDMC_DISPATCH(S, Lo, return launch_eval_all_t<V>(S, Lo, L, P, st));
  return cudaErrorInvalidValue;
}

static int sm_count_current()
{
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return 152;
  return n;
}

// Warps per block of the interval kernel: 16 (so that the warps of an SM,
// one block, can help one another at the end of an interval), halved while
// the population cannot give every warp of every SM a walker or the block's
// shared memory does not fit; at least the other kernels' four.
int interval_warps(const Layout& Lo, int W)
{
  const int sms = sm_count_current();
  int w = kMaxIntervalWarps;
  while (w > kWarpsPerBlock &&
         ((int)sizeof(double) * (Lo.head + w * Lo.smem_warp) > kMaxSmemBlock || W < sms * w))
    w >>= 1;
  return w;
}

static int interval_smem(const Layout& Lo, int w) { return (int)sizeof(double) * (Lo.head + w * Lo.smem_warp); }

// Persistent grid of the interval kernel: as many blocks as fit on the GPU
// at once (occupancy for this system's shared memory), at most one warp per
// walker.
template <int PREC>
static cudaError_t interval_occupancy(const Layout& Lo, int w, int* blocks)
{
  int per_sm = 0;
  cudaError_t e = set_smem((const void*)k_interval<PREC>, interval_smem(Lo, w));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interval<PREC>, w * 32, interval_smem(Lo, w));
  *blocks = (per_sm < 1 ? 1 : per_sm) * sm_count_current();
  return e;
}

int interval_default_blocks(const SysDev& S, const Layout& Lo, int W)
{
  int b = 0;
  const int w = interval_warps(Lo, W);
  LRDMC_DISPATCH(S, Lo, interval_occupancy<V>(Lo, w, &b));
  return b;
}

template <int PREC>
static cudaError_t launch_interval_t(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P,
                                     int blocks, int carveout, bool pdl, cudaStream_t st)
{
  static int cached_blocks = -1, cached_smem = -1;
  const int w = interval_warps(Lo, P.W);
  const int smem = interval_smem(Lo, w);
  cudaError_t e = set_smem((const void*)k_interval<PREC>, smem);
  if (e != cudaSuccess) return e;
  if (blocks <= 0) {
    if (cached_smem != smem) {
      e = interval_occupancy<PREC>(Lo, w, &cached_blocks);
      if (e != cudaSuccess) return e;
      cached_smem = smem;
    }
    blocks = cached_blocks;
  }
  const int need = (P.W + w - 1) / w;
  if (blocks > need) blocks = need;
  if (carveout < 0 && !pdl) {
    k_interval<PREC><<<blocks, w * 32, smem, st>>>(S, Lo, L, P);
    return cudaGetLastError();
  }
  // the same launch with launch attributes: a preferred shared-memory
  // carveout for this launch only (kernels of different systems sharing the
  // SMs then ask for the same L1/shared split), and programmatic stream
  // serialization (this kernel may start once every block of the previous
  // kernel in the stream has run out of walkers)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(w * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (carveout >= 0) {
    attr[na].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[na].val.sharedMemCarveout = (unsigned)carveout;
    ++na;
  }
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, k_interval<PREC>, S, Lo, L, P);
}

cudaError_t launch_interval(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P, int blocks,
                            cudaStream_t st, int carveout, bool pdl)
{
  LRDMC_DISPATCH(S, Lo, return launch_interval_t<V>(S, Lo, L, P, blocks, carveout, pdl, st));
  return cudaErrorInvalidValue;
}

int comb_blocks(int W)
{
  // at least 256 slots per block (short sequential sums over the blocks),
  // at most kMaxCombBlocks blocks
  const int R = std::max(kCombThreads, (W + kMaxCombBlocks - 1) / kMaxCombBlocks);
  return std::max(1, (W + R - 1) / R);
}

cudaError_t launch_reconfig(const PopDev& P, const Layout& Lo, cudaStream_t st)
{
  const int G = comb_blocks(P.W);
  const int R = (P.W + G - 1) / G;
  // the running sums (up to kReconfigSmemW walkers), then a float per slot
  // of the block
  const int smem = (P.W <= kReconfigSmemW ? (int)sizeof(double) * P.W : 0) + (int)sizeof(float) * R;
  // the attribute always takes the largest size, so systems of different
  // populations (and batches captured in one graph) never lower it
  cudaError_t e = set_smem((const void*)k_comb_parents, kCombSmemMax);
  if (e != cudaSuccess) return e;
  if (smem > kCombSmemMax) return cudaErrorInvalidValue;
  k_comb_sums<<<G, kCombThreads, 0, st>>>(P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kCombThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_comb_parents, P, (const double*)P.rec_dst, Lo.rec, Lo.off_b);
}

// Base terms of the neural objective: grad_i log|psi_G| and E_L of every
// configuration in IEEE double, one warp per configuration (the caller
// passes the system with the neural term switched off).
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_base_terms(const __grid_constant__ SysDev S, const Layout Lo, int n, const double* x, double* grad,
             double* e, int* err)
{
  extern __shared__ double smem[];
  double* sC = smem;
  stage_coefficients(S, sC);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int s = blockIdx.x * kWarpsPerBlock + wib;
  if (s >= n) return;
  WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
  for (int j = lane; j < 3 * Lo.N; j += 32) wm.x[j] = x[(size_t)s * 3 * Lo.N + j];
  __syncwarp();
  bool ok = warp_inverse(S, sC, wm.x, 0, wm.A, wm.scr, lane);
  ok = ok && warp_inverse(S, sC, wm.x, 1, wm.A + Lo.nu * Lo.nu, wm.scr, lane);
  if (!ok) {
    if (lane == 0) atomicOr(err, kErrSingular);
    for (int j = lane; j < 3 * Lo.N; j += 32) grad[(size_t)s * 3 * Lo.N + j] = NAN;
    if (lane == 0) e[s] = NAN;
    return;
  }
  LatDev L{};
  L.G = 1;
  double b, el;
  warp_eval<false>(S, sC, L, wm, lane, nullptr, b, el, grad + (size_t)s * 3 * Lo.N, false);
  if (lane == 0) e[s] = el;
}

cudaError_t launch_base_terms(const SysDev& S, const Layout& Lo, int n, const double* x, double* grad,
                              double* e_out, int* err, cudaStream_t st)
{
  if (n <= 0) return cudaSuccess;
  cudaError_t e = set_smem((const void*)k_base_terms, Lo.smem_block_bytes);
  if (e != cudaSuccess) return e;
  const int blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_base_terms<<<blocks, kWarpsPerBlock * 32, Lo.smem_block_bytes, st>>>(S, Lo, n, x, grad, e_out, err);
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_evaluate_t(const SysDev& S, const Layout& Lo, const LatDev& L, int n, const double* x,
                                     const double* rot, double* ratio, double* T, double* b, double* el, int* err,
                                     cudaStream_t st)
{
  const int blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  cudaError_t e = set_smem((const void*)k_evaluate<PREC>, Lo.smem_block_bytes);
  if (e != cudaSuccess) return e;
  k_evaluate<PREC><<<blocks, kWarpsPerBlock * 32, Lo.smem_block_bytes, st>>>(S, Lo, L, n, x, rot, ratio, T, b, el,
                                                                            err);
  return cudaGetLastError();
}

cudaError_t launch_evaluate(const SysDev& S, const Layout& Lo, const LatDev& L, int n,
                            const double* x, const double* rot, double* ratio, double* T,
                            double* b, double* el, int* err, cudaStream_t st)
{
  LRDMC_DISPATCH(S, Lo, return launch_evaluate_t<V>(S, Lo, L, n, x, rot, ratio, T, b, el, err, st));
  return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------------------
// Tensor-core form of the orbital contraction (tcgen05, FP32 mode).
//
// The literal contraction of the displaced positions' basis values with the
// MO coefficients, phi_m(r'_c) = sum_mu chi_mu(r'_c) C[mu][m], as a GEMM on
// the fifth-generation tensor cores: one CTA of four warps evaluates four
// configurations in lock step; per round every lane computes the basis
// values of one lattice move (FP32) and writes them, split into bfloat16
// high and low parts, as one row of a 128-row A tile in shared memory;
// thread 0 issues D = A_hi B_hi + A_hi B_lo + A_lo B_hi (B = C^T split the
// same way; three bf16 products carry about 16 significant bits) into a
// 128 x 32 FP32 accumulator in tensor memory; each warp reads its 32 rows
// back (tcgen05.ld) and finishes its moves: the determinant ratio
// sum_m phi_m Ainv[m][l_i] (FP32), the Jastrow ratio and the rate, as the
// FP32 mode's projected form does. Shared-memory operands use the
// canonical K-major layout without swizzle: 8 x 16-byte core matrices,
// adjacent in K at LBO = 128 bytes, 8-row groups at SBO = 16 Kp bytes.
// Every wait on the MMA's mbarrier is bounded; a wait that runs out sets
// kErrTimeout, waits once more (bounded) and frees the tensor memory.
// ----------------------------------------------------------------------------
constexpr int kTcRows = 128;    // A tile rows: 4 warps x 32 moves
constexpr int kTcN = 32;        // accumulator columns (orbitals, padded)
constexpr int kTcCols = 32;     // tensor-memory columns allocated
constexpr int kTcSpin = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(const void* base, uint32_t lbo, uint32_t sbo)
{
  uint64_t d = (uint64_t)((smem_u32(base) & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100-class tensor cores; no swizzle, base offset 0
  return d;
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, N, M.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N)
{
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar)
{
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count)
{
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* mbar, uint32_t parity)
{
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the MMA barrier (kTcSpin polls, a short
// sleep between them: well under a second); false when it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity)
{
  for (int it = 0; it < kTcSpin; ++it) {
    if (mbar_test_wait(mbar, parity)) return true;
    __nanosleep(20);
  }
  return false;
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v)
{
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// x as bfloat16 high part plus the bfloat16 of the remainder (round to
// nearest even both times): x - hi - lo is about 2^-17 |x|.
__device__ __forceinline__ void bf16_split(float x, uint16_t& hi, uint16_t& lo)
{
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

// Byte offset of element (row, k) in a K-major tile without swizzle.
__device__ __forceinline__ uint32_t tc_off(int row, int k, int Kp)
{
  return (uint32_t)((row >> 3) * (Kp * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Writes one row of the A tiles, value by value in K order.
struct TcRowWriter {
  char* hi;
  char* lo;
  int row, Kp, k;
  __device__ __forceinline__ void put(float v)
  {
    uint16_t h, l;
    bf16_split(v, h, l);
    const uint32_t o = tc_off(row, k, Kp);
    *reinterpret_cast<uint16_t*>(hi + o) = h;
    *reinterpret_cast<uint16_t*>(lo + o) = l;
    ++k;
  }
  // zeros up to Kp (the padding of K, or a whole inactive row)
  __device__ __forceinline__ void finish()
  {
    while (k < Kp) put(0.0f);
  }
};

// Basis values chi_mu(p) of every AO (FP32, in AO order) into the row
// writer, and the electron-nucleus Jastrow terms into jen.
template <bool NJ>
__device__ __forceinline__ void tc_basis_row(const SysDev& S, const float p[3], const BlockMem& bm, TcRowWriter& w,
                                             float& jen)
{
  typedef Ar<float> A;
  jen = 0.0f;
  for (int I = 0; I < S.n_nuc; ++I) {
    const float d[3] = {p[0] - S.D.nuc[I][0].hi, p[1] - S.D.nuc[I][1].hi, p[2] - S.D.nuc[I][2].hi};
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float r = sqrtf(r2);
    if (S.en_b1[I] != 0.0) jen -= S.D.en_b1[I].hi * r / (S.D.en_b2.hi * r + 1.0f);
    if (NJ) jen += nj_value_m<float>(S, 2 + S.nj_species[I], r);
    float e = 0.0f;
    for (int q = S.nuc_shell_begin[I]; q < S.nuc_shell_begin[I + 1]; ++q) {
      const ShellDev& sh = S.sh[q];
      const DfShell& dsh = S.D.sh[q];
      if (sh.kind == 0 && !sh.same_exp) e = expf(-dsh.zeta.hi * r);
      const float Rv = radial_value_m<float>(S, sh, dsh, r, r2, e, bm);
      float Sv[5];
      const int nf = solid_m<float>(sh.l, d, Sv);
      w.k = sh.ao_offset;
      for (int f = 0; f < nf; ++f) w.put(Sv[f] * Rv);
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_evaluate_tc(const __grid_constant__ SysDev S, const Layout Lo, const LatDev L, int n, const double* x,
              const double* rot, double* ratio, double* T, double* b_out, double* el_out, int* err, int Kp,
              int tile_off)
{
  constexpr bool NJ = (PREC & 8) != 0;
  typedef Ar<float> A;
  extern __shared__ double smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  double* sC = smem;
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  char* tiles = reinterpret_cast<char*>(smem) + tile_off;
  const int tileA = kTcRows * Kp * 2, tileB = kTcN * Kp * 2;
  char* Ah = tiles;
  char* Al = Ah + tileA;
  char* Bh = Al + tileA;
  char* Bl = Bh + tileB;
  stage_coefficients(S, sC);
  const BlockMem bm = block_mem(S, sC);
  // B = C^T (orbital m, AO k), split into bfloat16 high and low parts
  for (int idx = tid; idx < kTcN * Kp; idx += blockDim.x) {
    const int m = idx / Kp, k = idx - m * Kp;
    const float v = (m < S.n_mo && k < S.n_ao) ? (float)S.C[k * S.n_mo + m] : 0.0f;
    uint16_t h, l;
    bf16_split(v, h, l);
    const uint32_t o = tc_off(m, k, Kp);
    *reinterpret_cast<uint16_t*>(Bh + o) = h;
    *reinterpret_cast<uint16_t*>(Bl + o) = l;
  }
  if (wib == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_tmem)), "r"(kTcCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&s_mbar, 1);
    s_bad = 0;
  }
  fence_async_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  // this warp's configuration: inverses, then the local energy and the
  // Jastrow sums of the FP32 evaluation
  const int c = blockIdx.x * kWarpsPerBlock + wib;
  WarpMem wm = warp_mem(Lo, S, sC + Lo.head + wib * Lo.smem_warp);
  bool ok = c < n;
  double b = 0.0, el = 0.0;
  df bdf;
  if (ok) {
    for (int j = lane; j < 3 * Lo.N; j += 32) wm.x[j] = x[(size_t)c * 3 * Lo.N + j];
    for (int j = lane; j < 9; j += 32) wm.R[j] = rot[(size_t)c * 9 + j];
    __syncwarp();
    ok = warp_inverse(S, sC, wm.x, 0, wm.A, wm.scr, lane);
    ok = ok && warp_inverse(S, sC, wm.x, 1, wm.A + Lo.nu * Lo.nu, wm.scr, lane);
    if (!ok && lane == 0) atomicOr(err, kErrSingular);
    if (ok) warp_eval_m<float, NJ, true, false>(S, sC, L, wm, lane, nullptr, b, bdf, el);
  }
  const int N = S.N, G = L.G, per_e = 6 * G, P = N * per_e;
  const int rounds = (P + 31) / 32;
  df* Td = reinterpret_cast<df*>(wm.T);
  const uint32_t idesc = tc_idesc_bf16(kTcRows, kTcN);
  uint32_t phase = 0;
  for (int rd = 0; rd < rounds; ++rd) {
    const int cand = rd * 32 + lane;
    const bool act = ok && cand < P;
    TcRowWriter w;
    w.hi = Ah;
    w.lo = Al;
    w.row = wib * 32 + lane;
    w.Kp = Kp;
    w.k = 0;
    float jsum = 0.0f, pm = 1.0f;
    int i = 0, g = 0;
    if (act) {
      i = cand / per_e;
      const int rem = cand - i * per_e, k = (rem % 6) >> 1;
      g = rem / 6;
      float h = g ? L.ap_df.hi : L.a_df.hi;
      if (cand & 1) h = -h;
      const float e0 = wm.Rd[k].hi, e1 = wm.Rd[3 + k].hi, e2 = wm.Rd[6 + k].hi;
      const float ri[3] = {wm.xd[3 * i].hi, wm.xd[3 * i + 1].hi, wm.xd[3 * i + 2].hi};
      const float p[3] = {ri[0] + h * e0, ri[1] + h * e1, ri[2] + h * e2};
      float jen;
      tc_basis_row<NJ>(S, p, bm, w, jen);
      jsum = jastrow_ee_m<float, NJ>(S, wm.xd, i, p) + jen;
      if (G == 2) {
        const float hh = 0.5f * h;
        const float mid[3] = {ri[0] + hh * e0, ri[1] + hh * e1, ri[2] + hh * e2};
        pm = p_weight_m<float>(S, L, mid, bm);
      }
    }
    w.finish();
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int kk = 0; kk < Kp / 16; ++kk) {
        const uint32_t off = (uint32_t)kk * 256;
        const uint64_t ah = tc_desc(Ah + off, 128, Kp * 16), al = tc_desc(Al + off, 128, Kp * 16);
        const uint64_t bh = tc_desc(Bh + off, 128, Kp * 16), bl = tc_desc(Bl + off, 128, Kp * 16);
        tc_mma(tmem, ah, bh, idesc, kk > 0);
        tc_mma(tmem, ah, bl, idesc, 1);
        tc_mma(tmem, al, bh, idesc, 1);
      }
      tc_commit(&s_mbar);
    }
    if (!mbar_wait_bounded(&s_mbar, phase)) s_bad = 1;
    phase ^= 1u;
    __syncthreads();
    if (s_bad) break;
    tc_fence_after();
    float phi[32];
    tc_ld32(tmem + ((uint32_t)(wib * 32) << 16), phi);
    if (act) {
      const int nu = S.n_up, spin = i < nu ? 0 : 1, l = i < nu ? i : i - nu, ns = spin ? S.n_dn : nu;
      const double* Am = spin ? wm.A + nu * nu : wm.A;
      float rdet = 0.0f;
#pragma unroll
      for (int m = 0; m < kTcN; ++m)
        if (m < ns) rdet += phi[m] * (float)Am[m * ns + l];
      const float rho = rdet * expf(jsum - wm.Sd[i].hi);
      float wgt = 1.0f;
      if (G == 2) wgt = g ? 1.0f - pm : pm;
      float Tc = 0.0f;
      if (rho > 0.0f) Tc = wgt * (g ? L.inv2ap2_df.hi : L.inv2a2_df.hi) * rho;
      Td[cand] = A::store(Tc);
      if (ratio) ratio[(size_t)c * P + cand] = (double)rho;
    }
    tc_fence_before();
    __syncthreads();  // every lane has read the accumulator and the A tiles are free
  }
  if (s_bad) {
    // the MMA barrier did not complete in time: report, wait once more for
    // the tensor core to finish with this CTA's memory, then free it
    if (tid == 0) {
      atomicOr(err, kErrTimeout);
      mbar_wait_bounded(&s_mbar, phase ^ 1u);
    }
    __syncthreads();
  } else if (ok) {
    __syncwarp();
    const float btot = warp_scan_m<float>(Td, P, lane, 0.0f, nullptr, nullptr);
    b = (double)btot;
    if (T)
      for (int j = lane; j < P; j += 32) T[(size_t)c * P + j] = (double)Td[j].hi;
    if (lane == 0) {
      if (b_out) b_out[c] = b;
      if (el_out) el_out[c] = el;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wib == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols) : "memory");
  }
}

// Shared memory of the tensor-core evaluation: the evaluation's own layout,
// then (128-byte aligned) the A and B tiles in both parts.
static int tc_tile_offset(const Layout& Lo) { return (Lo.smem_block_bytes + 127) & ~127; }
static int tc_smem_bytes(const Layout& Lo, int Kp) { return tc_tile_offset(Lo) + 2 * (kTcRows + kTcN) * Kp * 2; }

int evaluate_tc_smem_bytes(const SysDev& S, const Layout& Lo)
{
  const int Kp = (S.n_ao + 15) & ~15;
  return tc_smem_bytes(Lo, Kp);
}

cudaError_t launch_evaluate_tc(const SysDev& S, const Layout& Lo, const LatDev& L, int n, const double* x,
                               const double* rot, double* ratio, double* T, double* b, double* el, int* err,
                               cudaStream_t st)
{
  if (n <= 0) return cudaSuccess;
  const int Kp = (S.n_ao + 15) & ~15;
  const int bytes = tc_smem_bytes(Lo, Kp);
  const int blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  cudaError_t e;
  if (S.nj_on) {
    e = set_smem((const void*)k_evaluate_tc<LRDMC_PRECISION_FP32 | kNjBit>, bytes);
    if (e != cudaSuccess) return e;
    k_evaluate_tc<LRDMC_PRECISION_FP32 | kNjBit><<<blocks, kWarpsPerBlock * 32, bytes, st>>>(
        S, Lo, L, n, x, rot, ratio, T, b, el, err, Kp, tc_tile_offset(Lo));
  } else {
    e = set_smem((const void*)k_evaluate_tc<LRDMC_PRECISION_FP32>, bytes);
    if (e != cudaSuccess) return e;
    k_evaluate_tc<LRDMC_PRECISION_FP32><<<blocks, kWarpsPerBlock * 32, bytes, st>>>(
        S, Lo, L, n, x, rot, ratio, T, b, el, err, Kp, tc_tile_offset(Lo));
  }
  return cudaGetLastError();
}


// ----------------------------------------------------------------------------
// Evaluation that allocates nothing (lrdmc_evaluate_static).
//
// Some callers cannot allocate device memory at the moment they evaluate:
// code that runs inside another framework's fixed memory budget (a caching
// allocator that has reserved the device), processes that forbid any
// allocation after start-up, or callers that must not synchronise the
// device the way cudaMalloc and cudaFree can. This variant of k_evaluate
// keeps its scratch - a summary status word and one status word per
// configuration - in the file-scope device array below instead of memory
// from cudaMalloc. Every GPU that loads the library holds the array
// (64 + LRDMC_STATIC_EVAL_MAX ints, 1 MiB) until the process exits. All
// calls share it: calls that overlap on the GPU race on it.
// ----------------------------------------------------------------------------
static __device__ __align__(256) int g_eval_scratch[64 + LRDMC_STATIC_EVAL_MAX];

template <int PREC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_evaluate_static(const __grid_constant__ SysDev S, const Layout Lo, const LatDev L, int n,
                  const double* x, const double* rot, double* ratio, double* T, double* b_out,
                  double* el_out, int* scratch)
{
  extern __shared__ double smem[];
  double* sC = smem;
  stage_coefficients(S, sC);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.x * kWarpsPerBlock + wib;
  if (c >= n) return;
  // word 64 + c: status of configuration c; word 0: OR of all statuses
  if (!evaluate_config<PREC>(S, Lo, L, sC, c, lane, wib, x, rot, ratio, T, b_out, el_out) && lane == 0) {
    scratch[64 + c] = kErrSingular;
    atomicOr(&scratch[0], kErrSingular);
  }
}

// Device address of g_eval_scratch, looked up once per device with that
// device current (host code must not pass the symbol itself: in host code
// it names a host-side stand-in, not device memory).
static int* g_eval_scratch_ptr[64];
static std::mutex g_eval_scratch_mu;

static cudaError_t eval_scratch_address(int** out)
{
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_eval_scratch_mu);
  if (!g_eval_scratch_ptr[dev]) {
    int* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_eval_scratch);
    if (e != cudaSuccess) return e;
    g_eval_scratch_ptr[dev] = p;
  }
  *out = g_eval_scratch_ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_evaluate_static(const SysDev& S, const Layout& Lo, const LatDev& L, int n,
                                   const double* x, const double* rot, double* ratio, double* T,
                                   double* b, double* el, int* summary, int* first_bad, cudaStream_t st)
{
  if (first_bad) *first_bad = -1;
  if (n < 0 || n > LRDMC_STATIC_EVAL_MAX) return cudaErrorInvalidValue;
  int* scratch = nullptr;
  cudaError_t e = eval_scratch_address(&scratch);
  if (e != cudaSuccess) return e;
  // the summary word and the statuses of this call start at zero
  e = cudaMemsetAsync(scratch, 0, sizeof(int) * (64 + (size_t)n), st);
  if (e != cudaSuccess) return e;
  const int blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  LRDMC_DISPATCH(S, Lo, {
    e = set_smem((const void*)k_evaluate_static<V>, Lo.smem_block_bytes);
    if (e != cudaSuccess) return e;
    if (blocks > 0)
      k_evaluate_static<V><<<blocks, kWarpsPerBlock * 32, Lo.smem_block_bytes, st>>>(S, Lo, L, n, x, rot, ratio,
                                                                                    T, b, el, scratch);
  });
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(summary, scratch, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || *summary == 0 || !first_bad) return e;
  // a configuration failed: find the first one from the per-configuration
  // words, in chunks through a fixed host buffer (no allocation)
  int chunk[1024];
  for (int c0 = 0; c0 < n; c0 += 1024) {
    const int m = n - c0 < 1024 ? n - c0 : 1024;
    e = cudaMemcpyAsync(chunk, scratch + 64 + c0, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int j = 0; j < m; ++j)
      if (chunk[j] != 0) {
        *first_bad = c0 + j;
        return cudaSuccess;
      }
  }
  return cudaSuccess;
}

}  // namespace lrdmc
