// Neural pair term of the Jastrow factor: the host-side table that the
// projection interpolates, and the training kernels of the variance
// objective (forward with radial derivatives, per-configuration assembly,
// backward to the parameters).
//
// The term (declared in include/lrdmc.h): g_c(r) = m(r, c) s(r / r_cut_c),
// m = w3 . silu(W2 silu(W1 z + b1) + b2) + b3, z = [r^2/(r^2 + ell_k^2),
// one-hot(c)], s(t) = 1 - 10t^3 + 15t^4 - 6t^5. Radial derivatives are
// carried forward through the layers as chains (value, d/dr, d2/dr2):
// a linear layer maps each chain by the same matrix (the bias only the
// value), an activation maps (z, z', z'') to (silu z, silu'(z) z',
// silu''(z) z'^2 + silu'(z) z'').
//
// Training arithmetic is FP32 with the parameters staged in shared memory
// (bfloat16-rounded when the spec asks for it); one warp evaluates one
// pair, lane l owning hidden units l and l + 32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lrdmc_internal.h"

namespace lrdmc {

// ----------------------------------------------------------------------------
// Host: parameters, rounding and the interpolation table.
// ----------------------------------------------------------------------------
int nj_n_params(int n_feat, int n_ch, int hidden)
{
  const int D = n_feat + n_ch, H = hidden;
  return H * D + H + H * H + H + H + 1;
}

float nj_bf16(float x)
{
  // round to nearest bfloat16, ties to even, on the float32 bit pattern
  uint32_t u;
  memcpy(&u, &x, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  float y;
  memcpy(&y, &u, 4);
  return y;
}

namespace {

struct HostNet {
  int F, C, H, D;
  std::vector<double> ell2, rcut, W1, b1, W2, b2, w3;
  double b3;
};

HostNet host_net(const lrdmc_nj_spec& sp, const float* params)
{
  HostNet n;
  n.F = sp.n_feat; n.C = sp.n_ch; n.H = sp.hidden; n.D = n.F + n.C;
  for (int f = 0; f < n.F; ++f) n.ell2.push_back(sp.ell[f] * sp.ell[f]);
  for (int c = 0; c < n.C; ++c) n.rcut.push_back(sp.r_cut[c]);
  auto val = [&](int idx) { return (double)(sp.bf16 ? nj_bf16(params[idx]) : params[idx]); };
  int o = 0;
  const int H = n.H, D = n.D;
  for (int q = 0; q < H * D; ++q) n.W1.push_back(val(o++));
  for (int q = 0; q < H; ++q) n.b1.push_back(val(o++));
  for (int q = 0; q < H * H; ++q) n.W2.push_back(val(o++));
  for (int q = 0; q < H; ++q) n.b2.push_back(val(o++));
  for (int q = 0; q < H; ++q) n.w3.push_back(val(o++));
  n.b3 = val(o++);
  return n;
}

void silu_chain_d(double z, double z1, double z2, double& a, double& a1, double& a2)
{
  const double sg = 1.0 / (1.0 + exp(-z));
  const double d1 = sg * (1.0 + z * (1.0 - sg));
  const double d2 = sg * (1.0 - sg) * (2.0 + z * (1.0 - 2.0 * sg));
  a = z * sg;
  a1 = d1 * z1;
  a2 = d2 * z1 * z1 + d1 * z2;
}

// g_c(r), g', g'' in IEEE double
void host_radial(const HostNet& n, int c, double r, double& g, double& g1, double& g2)
{
  const double rc = n.rcut[c];
  g = g1 = g2 = 0.0;
  if (!(r < rc)) return;
  std::vector<double> x0(n.D, 0.0), x1(n.D, 0.0), x2(n.D, 0.0);
  for (int f = 0; f < n.F; ++f) {
    const double l2 = n.ell2[f], den = r * r + l2;
    x0[f] = r * r / den;
    x1[f] = 2.0 * r * l2 / (den * den);
    x2[f] = 2.0 * l2 * (l2 - 3.0 * r * r) / (den * den * den);
  }
  x0[n.F + c] = 1.0;
  std::vector<double> h(n.H), h1(n.H), h2(n.H), k(n.H), k1(n.H), k2(n.H);
  for (int u = 0; u < n.H; ++u) {
    double z = n.b1[u], z1 = 0.0, z2 = 0.0;
    for (int f = 0; f < n.D; ++f) {
      const double w = n.W1[u * n.D + f];
      z += w * x0[f]; z1 += w * x1[f]; z2 += w * x2[f];
    }
    silu_chain_d(z, z1, z2, h[u], h1[u], h2[u]);
  }
  for (int u = 0; u < n.H; ++u) {
    double z = n.b2[u], z1 = 0.0, z2 = 0.0;
    for (int v = 0; v < n.H; ++v) {
      const double w = n.W2[u * n.H + v];
      z += w * h[v]; z1 += w * h1[v]; z2 += w * h2[v];
    }
    silu_chain_d(z, z1, z2, k[u], k1[u], k2[u]);
  }
  double m = n.b3, m1 = 0.0, m2 = 0.0;
  for (int u = 0; u < n.H; ++u) { m += n.w3[u] * k[u]; m1 += n.w3[u] * k1[u]; m2 += n.w3[u] * k2[u]; }
  const double t = r / rc;
  const double s = 1.0 - t * t * t * (10.0 - t * (15.0 - 6.0 * t));
  const double s1 = -30.0 * t * t * (1.0 - t) * (1.0 - t) / rc;
  const double s2 = -60.0 * t * (1.0 - t) * (1.0 - 2.0 * t) / (rc * rc);
  g = m * s;
  g1 = m1 * s + m * s1;
  g2 = m2 * s + 2.0 * m1 * s1 + m * s2;
}

}  // namespace

// Per channel and cell k: r_k, 1/w_k and the coefficients c_0..c_5 (in
// t = (r - r_k)/w_k) of the quintic that matches (g, w g', w^2 g'') at both
// ends of the cell. With D = p1 - p0:
//   c0 = p0, c1 = d0, c2 = s0/2,
//   c3 = 10 D - 6 d0 - 4 d1 - (3 s0 - s1)/2,
//   c4 = -15 D + 8 d0 + 7 d1 + (3 s0 - 2 s1)/2,
//   c5 = 6 D - 3 d0 - 3 d1 - (s0 - s1)/2.
void nj_build_table(const lrdmc_nj_spec& sp, const float* params, std::vector<double>& tab)
{
  const HostNet net = host_net(sp, params);
  const int n = sp.n_cells;
  tab.assign((size_t)sp.n_ch * n * 8, 0.0);
  std::vector<double> G(n + 1), G1(n + 1), G2(n + 1), R(n + 1);
  for (int c = 0; c < sp.n_ch; ++c) {
    const double rc = sp.r_cut[c];
    for (int k = 0; k <= n; ++k) {
      const double q = (double)k / n;
      R[k] = rc * q * q;
      host_radial(net, c, R[k], G[k], G1[k], G2[k]);
    }
    for (int k = 0; k < n; ++k) {
      const double w = R[k + 1] - R[k];
      const double p0 = G[k], d0 = w * G1[k], s0 = w * w * G2[k];
      const double p1 = G[k + 1], d1 = w * G1[k + 1], s1 = w * w * G2[k + 1];
      const double D = p1 - p0;
      double* e = &tab[((size_t)c * n + k) * 8];
      e[0] = R[k];
      e[1] = 1.0 / w;
      e[2] = p0;
      e[3] = d0;
      e[4] = 0.5 * s0;
      e[5] = 10.0 * D - 6.0 * d0 - 4.0 * d1 - 0.5 * (3.0 * s0 - s1);
      e[6] = -15.0 * D + 8.0 * d0 + 7.0 * d1 + 0.5 * (3.0 * s0 - 2.0 * s1);
      e[7] = 6.0 * D - 3.0 * d0 - 3.0 * d1 - 0.5 * (s0 - s1);
    }
  }
}

// ----------------------------------------------------------------------------
// Device: training kernels.
// ----------------------------------------------------------------------------
constexpr int kNjH = LRDMC_NJ_HIDDEN;
constexpr int kNjMaxF = LRDMC_NJ_MAX_FEAT;
constexpr int kNjMaxC = LRDMC_NJ_MAX_CH;
constexpr int kNjWarps = 4;
static_assert(kNjH == 64, "lanes own hidden units l and l + 32");

// Shared-memory image of the parameters (float, bf16-rounded if asked):
// W1T [D][H] (transposed), b1, W2T [H][H] (transposed, forward), W2 [H][H]
// (row-major, backward), b2, w3, b3; then the pair table and the per-warp
// chain buffers.
struct NjSmem {
  float* W1T; float* b1; float* W2T; float* W2; float* b2; float* w3; float* b3;
  int* pairs;      // [n_pairs]: i | j << 8 | channel << 16 (j = nucleus for e-n)
  float4* chain;   // [warps][H] per-warp broadcast buffer
};

__host__ __device__ inline int nj_smem_floats(int D, int n_pairs)
{
  return D * kNjH + kNjH + 2 * kNjH * kNjH + 2 * kNjH + 1 + 3 /*pad*/ + n_pairs + 4 * kNjWarps * kNjH + 4;
}

__device__ inline NjSmem nj_stage(const NjGeom& G, const NjNetDev& N, const float* params, float* sm)
{
  NjSmem m;
  const int D = N.D, H = kNjH;
  m.W1T = sm;
  m.b1 = m.W1T + D * H;
  m.W2T = m.b1 + H;
  m.W2 = m.W2T + H * H;
  m.b2 = m.W2 + H * H;
  m.w3 = m.b2 + H;
  m.b3 = m.w3 + H;
  m.pairs = reinterpret_cast<int*>(m.b3 + 4);
  const int np = G.n_pairs;
  uintptr_t a = reinterpret_cast<uintptr_t>(m.pairs + np);
  a = (a + 15) & ~(uintptr_t)15;
  m.chain = reinterpret_cast<float4*>(a);
  auto rd = [&](int idx) { float v = params[idx]; return N.bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v; };
  const int oW1 = 0, ob1 = H * D, oW2 = ob1 + H, ob2 = oW2 + H * H, ow3 = ob2 + H, ob3 = ow3 + H;
  for (int q = threadIdx.x; q < H * D; q += blockDim.x) {
    const int u = q / D, f = q % D;
    m.W1T[f * H + u] = rd(oW1 + q);
  }
  for (int q = threadIdx.x; q < H * H; q += blockDim.x) {
    const int u = q / H, v = q % H;
    const float w = rd(oW2 + q);
    m.W2[q] = w;
    m.W2T[v * H + u] = w;
  }
  for (int q = threadIdx.x; q < H; q += blockDim.x) {
    m.b1[q] = rd(ob1 + q);
    m.b2[q] = rd(ob2 + q);
    m.w3[q] = rd(ow3 + q);
  }
  if (threadIdx.x == 0) m.b3[0] = rd(ob3);
  // pair table: electron pairs i < j, then electron-nucleus pairs i-major
  const int N_e = G.N, n_ee = N_e * (N_e - 1) / 2;
  for (int q = threadIdx.x; q < np; q += blockDim.x) {
    int i, j, c;
    if (q < n_ee) {
      // invert q = i N - i (i + 1)/2 + (j - i - 1)
      i = 0;
      int base = 0;
      while (base + (N_e - 1 - i) <= q) { base += N_e - 1 - i; ++i; }
      j = i + 1 + (q - base);
      c = ((i < G.n_up) == (j < G.n_up)) ? 0 : 1;
    } else {
      const int r = q - n_ee;
      i = r / G.n_nuc;
      j = r % G.n_nuc;
      c = 2 + G.species[j];
    }
    m.pairs[q] = i | (j << 8) | (c << 16);
  }
  __syncthreads();
  return m;
}

__device__ __forceinline__ void silu3(float z, float& a, float& d1, float& d2, float& d3)
{
  const float sg = 1.0f / (1.0f + expf(-z));
  const float sp = sg * (1.0f - sg);       // sigma'
  const float u = 1.0f - 2.0f * sg;
  a = z * sg;
  d1 = sg * (1.0f + z * (1.0f - sg));     // silu'
  d2 = sp * (2.0f + z * u);               // silu''
  d3 = sp * (u * (3.0f + z * u) - 2.0f * z * sp);  // silu'''
}

// Geometry of pair q of configuration cfg: radius, unit vector (from i to
// the partner: r_i - r_j or r_i - R_I), electrons and channel.
struct PairGeo {
  float r, e[3];
  int i, j, c, is_en;
};

__device__ __forceinline__ PairGeo pair_geo(const NjGeom& G, const NjSmem& m, const double* x, size_t cfg, int q)
{
  PairGeo p;
  const int code = m.pairs[q];
  p.i = code & 0xFF;
  p.j = (code >> 8) & 0xFF;
  p.c = code >> 16;
  p.is_en = p.c >= 2;
  const double* xi = x + (cfg * G.N + p.i) * 3;
  double d[3];
  if (p.is_en) {
    for (int k = 0; k < 3; ++k) d[k] = xi[k] - G.nuc[p.j][k];
  } else {
    const double* xj = x + (cfg * G.N + p.j) * 3;
    for (int k = 0; k < 3; ++k) d[k] = xi[k] - xj[k];
  }
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  p.r = (float)r;
  for (int k = 0; k < 3; ++k) p.e[k] = (float)(d[k] / r);
  return p;
}

// Features and their radial derivatives (radial part only; the channel code
// is constant).
__device__ __forceinline__ void features(const NjNetDev& N, float r, float f0[kNjMaxF], float f1[kNjMaxF],
                                         float f2[kNjMaxF])
{
#pragma unroll
  for (int f = 0; f < kNjMaxF; ++f) {
    if (f < N.F) {
      const float l2 = N.ell2[f], r2 = r * r, den = r2 + l2, id = 1.0f / den;
      f0[f] = r2 * id;
      f1[f] = 2.0f * r * l2 * id * id;
      f2[f] = 2.0f * l2 * (l2 - 3.0f * r2) * id * id * id;
    } else {
      f0[f] = 0.0f; f1[f] = 0.0f; f2[f] = 0.0f;
    }
  }
}

// Cut-off factor s(r/r_c) and its radial derivatives.
__device__ __forceinline__ void cutoff(float r, float rc, float& s, float& s1, float& s2)
{
  const float t = r / rc;
  if (t >= 1.0f) { s = 0.0f; s1 = 0.0f; s2 = 0.0f; return; }
  s = 1.0f - t * t * t * (10.0f - t * (15.0f - 6.0f * t));
  s1 = -30.0f * t * t * (1.0f - t) * (1.0f - t) / rc;
  s2 = -60.0f * t * (1.0f - t) * (1.0f - 2.0f * t) / (rc * rc);
}

// The two layers for the warp's pair; lane l computes units l and l + 32.
// On return: z1 chains of layer 1 (own units), the layer-1 activations of
// all units in the warp buffer, the z2 chains of layer 2 (own units).
struct Fwd {
  float z[2], z1[2], z2[2];   // layer 1 pre-activation chains
  float y[2], y1[2], y2[2];   // layer 2 pre-activation chains
};

__device__ __forceinline__ void fwd_layers(const NjNetDev& N, const NjSmem& m, float4* buf, int lane, int c,
                                           const float f0[kNjMaxF], const float f1[kNjMaxF],
                                           const float f2[kNjMaxF], Fwd& o)
{
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int u = lane + 32 * h;
    float z = m.b1[u] + m.W1T[(N.F + c) * kNjH + u], z1 = 0.0f, z2 = 0.0f;
#pragma unroll
    for (int f = 0; f < kNjMaxF; ++f) {
      if (f < N.F) {
        const float w = m.W1T[f * kNjH + u];
        z = fmaf(w, f0[f], z); z1 = fmaf(w, f1[f], z1); z2 = fmaf(w, f2[f], z2);
      }
    }
    o.z[h] = z; o.z1[h] = z1; o.z2[h] = z2;
    float a, d1, d2, d3;
    silu3(z, a, d1, d2, d3);
    buf[u] = make_float4(a, d1 * z1, d2 * z1 * z1 + d1 * z2, 0.0f);
  }
  __syncwarp();
  float y[2] = {m.b2[lane], m.b2[lane + 32]}, y1[2] = {0.0f, 0.0f}, y2[2] = {0.0f, 0.0f};
#pragma unroll 8
  for (int v = 0; v < kNjH; ++v) {
    const float4 a = buf[v];
    const float w0 = m.W2T[v * kNjH + lane], w1 = m.W2T[v * kNjH + lane + 32];
    y[0] = fmaf(w0, a.x, y[0]); y1[0] = fmaf(w0, a.y, y1[0]); y2[0] = fmaf(w0, a.z, y2[0]);
    y[1] = fmaf(w1, a.x, y[1]); y1[1] = fmaf(w1, a.y, y1[1]); y2[1] = fmaf(w1, a.z, y2[1]);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) { o.y[h] = y[h]; o.y1[h] = y1[h]; o.y2[h] = y2[h]; }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// g, g', g'' of every pair of every configuration.
__global__ void __launch_bounds__(kNjWarps * 32)
k_nj_pairs_fwd(const __grid_constant__ NjGeom G, const __grid_constant__ NjNetDev N, const float* params, int n,
               const double* x, float* pair_out)
{
  extern __shared__ float4 nj_smem4[];
  const NjSmem m = nj_stage(G, N, params, reinterpret_cast<float*>(nj_smem4));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float4* buf = m.chain + wib * kNjH;
  const long long total = (long long)n * G.n_pairs;
  for (long long p = (long long)blockIdx.x * kNjWarps + wib; p < total; p += (long long)gridDim.x * kNjWarps) {
    const size_t cfg = (size_t)(p / G.n_pairs);
    const int q = (int)(p % G.n_pairs);
    const PairGeo pg = pair_geo(G, m, x, cfg, q);
    float f0[kNjMaxF], f1[kNjMaxF], f2[kNjMaxF];
    features(N, pg.r, f0, f1, f2);
    Fwd o;
    fwd_layers(N, m, buf, lane, pg.c, f0, f1, f2, o);
    float mv = 0.0f, m1 = 0.0f, m2 = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float a, d1, d2, d3;
      silu3(o.y[h], a, d1, d2, d3);
      const float w = m.w3[lane + 32 * h];
      mv = fmaf(w, a, mv);
      m1 = fmaf(w, d1 * o.y1[h], m1);
      m2 = fmaf(w, d2 * o.y1[h] * o.y1[h] + d1 * o.y2[h], m2);
    }
    mv = warp_sum_f(mv) + m.b3[0];
    m1 = warp_sum_f(m1);
    m2 = warp_sum_f(m2);
    if (lane == 0) {
      float s, s1, s2;
      cutoff(pg.r, N.rcut[pg.c], s, s1, s2);
      float* out = pair_out + (size_t)p * 3;
      out[0] = mv * s;
      out[1] = m1 * s + mv * s1;
      out[2] = m2 * s + 2.0f * m1 * s1 + mv * s2;
    }
    __syncwarp();
  }
}

// Per configuration (one warp): G_i, L_i, J, E_L and q = a + G, in fixed
// summation order.
__global__ void __launch_bounds__(128)
k_nj_assemble(const __grid_constant__ NjGeom G, int n, const double* x, const double* grad_base,
              const double* e_base, const float* pair_out, float* el_out, float* j_out, float* q_out)
{
  const int lane = threadIdx.x & 31;
  const long long cfg = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (cfg >= n) return;
  const int N_e = G.N, n_ee = N_e * (N_e - 1) / 2;
  const float* po = pair_out + (size_t)cfg * G.n_pairs * 3;
  const double* xc = x + (size_t)cfg * N_e * 3;
  float part = 0.0f, jsum = 0.0f;
  for (int q = lane; q < G.n_pairs; q += 32) jsum += po[3 * q];
  for (int i = lane; i < N_e; i += 32) {
    float Gi[3] = {0.0f, 0.0f, 0.0f}, Li = 0.0f;
    for (int j = 0; j < N_e; ++j) {
      if (j == i) continue;
      const int a = min(i, j), b = max(i, j);
      const int q = a * N_e - a * (a + 1) / 2 + (b - a - 1);
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = xc[3 * i + k] - xc[3 * j + k];
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const float g1 = po[3 * q + 1], g2 = po[3 * q + 2], rf = (float)r;
      for (int k = 0; k < 3; ++k) Gi[k] += g1 * (float)(d[k] / r);
      Li += g2 + 2.0f * g1 / rf;
    }
    for (int I = 0; I < G.n_nuc; ++I) {
      const int q = n_ee + i * G.n_nuc + I;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = xc[3 * i + k] - G.nuc[I][k];
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const float g1 = po[3 * q + 1], g2 = po[3 * q + 2], rf = (float)r;
      for (int k = 0; k < 3; ++k) Gi[k] += g1 * (float)(d[k] / r);
      Li += g2 + 2.0f * g1 / rf;
    }
    const double* a = grad_base + ((size_t)cfg * N_e + i) * 3;
    float dot = 0.0f, gg = 0.0f;
    for (int k = 0; k < 3; ++k) {
      const float ak = (float)a[k];
      dot += ak * Gi[k];
      gg += Gi[k] * Gi[k];
      q_out[((size_t)cfg * N_e + i) * 3 + k] = ak + Gi[k];
    }
    part += 2.0f * dot + gg + Li;
  }
  part = warp_sum_f(part);
  jsum = warp_sum_f(jsum);
  if (lane == 0) {
    el_out[cfg] = (float)(e_base[cfg] - 0.5 * (double)part);
    j_out[cfg] = jsum;
  }
}

// Backward: per pair, the upstream derivatives with respect to g, g', g''
// from d_el and d_j of its configuration, then reverse through the cut-off,
// the output layer and both activations (the derivative chains included).
// Every sum runs in a fixed order, so the gradient is the same bits from
// run to run: each warp accumulates layers 2 and 3 in registers and layer 1
// in its own shared-memory slice (a lane owns its hidden units), the warps
// are added in warp order, and each block writes its sums to partials
// [blockIdx.x][n_params] for k_nj_grad_reduce.
__global__ void __launch_bounds__(kNjWarps * 32, 2)
k_nj_pairs_bwd(const __grid_constant__ NjGeom G, const __grid_constant__ NjNetDev N, const float* params, int n,
               const double* x, const float* qv, const float* d_el, const float* d_j, float* partials)
{
  extern __shared__ float4 nj_smem4[];
  const NjSmem m = nj_stage(G, N, params, reinterpret_cast<float*>(nj_smem4));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float4* buf = m.chain + wib * kNjH;
  float4* dbuf = m.chain + (kNjWarps + wib) * kNjH;
  const int D = N.D;
  const int H = kNjH, oW1 = 0, ob1 = H * D, oW2 = ob1 + H, ob2 = oW2 + H * H, ow3 = ob2 + H, ob3 = ow3 + H;
  const int np = ob3 + 1;
  // block accumulator of the gradient, then one layer-1 slice per warp
  // (W1 and b1, the first ob1 + H entries of the parameter vector)
  float* acc = reinterpret_cast<float*>(m.chain + 2 * kNjWarps * kNjH);
  const int np1 = ob1 + H;
  float* acc1 = acc + np;
  float* my1 = acc1 + wib * np1;
  for (int t = threadIdx.x; t < np; t += blockDim.x) acc[t] = 0.0f;
  for (int t = threadIdx.x; t < kNjWarps * np1; t += blockDim.x) acc1[t] = 0.0f;
  __syncthreads();
  float gW2[2][kNjH];
  float gb2[2] = {0.0f, 0.0f}, gw3[2] = {0.0f, 0.0f};
  float gb3 = 0.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int v = 0; v < kNjH; ++v) gW2[h][v] = 0.0f;
  const long long total = (long long)n * G.n_pairs;
  for (long long p = (long long)blockIdx.x * kNjWarps + wib; p < total; p += (long long)gridDim.x * kNjWarps) {
    const size_t cfg = (size_t)(p / G.n_pairs);
    const int q = (int)(p % G.n_pairs);
    const PairGeo pg = pair_geo(G, m, x, cfg, q);
    // upstream derivatives
    const float de = d_el[cfg], dj = d_j[cfg];
    const float* qi = qv + (cfg * G.N + pg.i) * 3;
    float dg1, dg2;
    if (pg.is_en) {
      const float qe = qi[0] * pg.e[0] + qi[1] * pg.e[1] + qi[2] * pg.e[2];
      dg1 = de * (-qe - 1.0f / pg.r);
      dg2 = -0.5f * de;
    } else {
      const float* qj = qv + (cfg * G.N + pg.j) * 3;
      const float qe = (qi[0] - qj[0]) * pg.e[0] + (qi[1] - qj[1]) * pg.e[1] + (qi[2] - qj[2]) * pg.e[2];
      dg1 = de * (-qe - 2.0f / pg.r);
      dg2 = -de;
    }
    float s, s1, s2;
    cutoff(pg.r, N.rcut[pg.c], s, s1, s2);
    const float dm = dj * s + dg1 * s1 + dg2 * s2;
    const float dm1 = dg1 * s + 2.0f * dg2 * s1;
    const float dm2 = dg2 * s;
    // forward recomputation
    float f0[kNjMaxF], f1[kNjMaxF], f2[kNjMaxF];
    features(N, pg.r, f0, f1, f2);
    Fwd o;
    fwd_layers(N, m, buf, lane, pg.c, f0, f1, f2, o);
    gb3 += dm;  // counted on every lane; lane 0's value is used
    // output layer and layer-2 activation
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = lane + 32 * h;
      float a, d1, d2, d3;
      silu3(o.y[h], a, d1, d2, d3);
      const float k1 = d1 * o.y1[h], k2 = d2 * o.y1[h] * o.y1[h] + d1 * o.y2[h];
      gw3[h] += dm * a + dm1 * k1 + dm2 * k2;
      const float w = m.w3[u];
      const float dh = w * dm, dh1 = w * dm1, dh2 = w * dm2;
      const float dz = dh * d1 + dh1 * d2 * o.y1[h] + dh2 * (d3 * o.y1[h] * o.y1[h] + d2 * o.y2[h]);
      const float dz1 = dh1 * d1 + 2.0f * dh2 * d2 * o.y1[h];
      const float dz2 = dh2 * d1;
      gb2[h] += dz;
#pragma unroll
      for (int v = 0; v < kNjH; ++v) {
        const float4 av = buf[v];
        gW2[h][v] = fmaf(dz, av.x, fmaf(dz1, av.y, fmaf(dz2, av.z, gW2[h][v])));
      }
      dbuf[u] = make_float4(dz, dz1, dz2, 0.0f);
    }
    __syncwarp();
    // layer-1 activations: da = W2^T dz (chains), then through silu
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = lane + 32 * h;
      float da = 0.0f, da1 = 0.0f, da2 = 0.0f;
#pragma unroll 8
      for (int u = 0; u < kNjH; ++u) {
        const float4 d = dbuf[u];
        const float w = m.W2[u * kNjH + v];
        da = fmaf(w, d.x, da); da1 = fmaf(w, d.y, da1); da2 = fmaf(w, d.z, da2);
      }
      float a, d1, d2, d3;
      silu3(o.z[h], a, d1, d2, d3);
      const float z1 = o.z1[h], z2 = o.z2[h];
      const float dz = da * d1 + da1 * d2 * z1 + da2 * (d3 * z1 * z1 + d2 * z2);
      const float dz1 = da1 * d1 + 2.0f * da2 * d2 * z1;
      const float dz2 = da2 * d1;
      // hidden unit v belongs to this lane alone within the warp's slice
      my1[ob1 + v] += dz;
      my1[oW1 + v * D + N.F + pg.c] += dz;
#pragma unroll
      for (int f = 0; f < kNjMaxF; ++f)
        if (f < N.F) my1[oW1 + v * D + f] += dz * f0[f] + dz1 * f1[f] + dz2 * f2[f];
    }
    __syncwarp();
  }
  // block reduction in warp order (a lane owns output units u, so the adds
  // of one warp touch distinct entries), layer 1 from the warp slices
  __syncthreads();
  for (int w = 0; w < kNjWarps; ++w) {
    if (wib == w) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int u = lane + 32 * h;
#pragma unroll
        for (int v = 0; v < kNjH; ++v) acc[oW2 + u * H + v] += gW2[h][v];
        acc[ob2 + u] += gb2[h];
        acc[ow3 + u] += gw3[h];
      }
      if (lane == 0) acc[ob3] += gb3;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < np1; t += blockDim.x) {
    float a = 0.0f;
    for (int w = 0; w < kNjWarps; ++w) a += acc1[w * np1 + t];
    acc[t] = a;
  }
  __syncthreads();
  float* out = partials + (size_t)blockIdx.x * np;
  for (int t = threadIdx.x; t < np; t += blockDim.x) out[t] = acc[t];
}

// grad[t] = sum over the backward blocks of partials[b][t], in block order.
__global__ void k_nj_grad_reduce(const float* partials, int blocks, int np, float* grad)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  float a = 0.0f;
  for (int b = 0; b < blocks; ++b) a += partials[(size_t)b * np + t];
  grad[t] = a;
}

static int nj_smem_bytes(const NjGeom& G, const NjNetDev& N, bool backward)
{
  // staging image and one chain buffer per warp; the backward pass adds a
  // second chain buffer per warp and the block's gradient accumulator
  int f = nj_smem_floats(N.D, G.n_pairs);
  if (backward) f += 4 * kNjWarps * kNjH + nj_n_params(N.F, N.C, kNjH) + kNjWarps * (kNjH * N.D + kNjH);
  return (int)sizeof(float) * f;
}

static int nj_grid(const void* fn, int smem)
{
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kNjWarps * 32, smem);
  return sms * (per > 0 ? per : 1);
}

cudaError_t launch_nj_forward(const NjGeom& G, const NjNetDev& N, const float* params, int n, const double* x,
                              const double* grad_base, const double* e_base, float* el, float* j, float* q,
                              float* pair_out, cudaStream_t st)
{
  if (n <= 0) return cudaSuccess;
  const int smem = nj_smem_bytes(G, N, false);
  cudaError_t e = cudaFuncSetAttribute((const void*)k_nj_pairs_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n * G.n_pairs;
  long long blocks = nj_grid((const void*)k_nj_pairs_fwd, smem);
  blocks = std::min(blocks, (total + kNjWarps - 1) / kNjWarps);
  k_nj_pairs_fwd<<<(int)blocks, kNjWarps * 32, smem, st>>>(G, N, params, n, x, pair_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nj_assemble<<<(n + 3) / 4, 128, 0, st>>>(G, n, x, grad_base, e_base, pair_out, el, j, q);
  return cudaGetLastError();
}

int nj_backward_max_blocks(const NjGeom& G, const NjNetDev& N)
{
  const int smem = nj_smem_bytes(G, N, true);
  if (cudaFuncSetAttribute((const void*)k_nj_pairs_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return -1;
  return nj_grid((const void*)k_nj_pairs_bwd, smem);
}

cudaError_t launch_nj_backward(const NjGeom& G, const NjNetDev& N, const float* params, int n, const double* x,
                               const float* q, const float* d_el, const float* d_j, float* grad, float* partials,
                               int max_blocks, cudaStream_t st)
{
  const int np = nj_n_params(N.F, N.C, kNjH);
  if (n <= 0) return cudaMemsetAsync(grad, 0, sizeof(float) * np, st);
  const int smem = nj_smem_bytes(G, N, true);
  cudaError_t e = cudaFuncSetAttribute((const void*)k_nj_pairs_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n * G.n_pairs;
  long long blocks = std::min((long long)max_blocks, (total + kNjWarps - 1) / kNjWarps);
  k_nj_pairs_bwd<<<(int)blocks, kNjWarps * 32, smem, st>>>(G, N, params, n, x, q, d_el, d_j, partials);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nj_grad_reduce<<<(np + 255) / 256, 256, 0, st>>>(partials, (int)blocks, np, grad);
  return cudaGetLastError();
}

}  // namespace lrdmc
