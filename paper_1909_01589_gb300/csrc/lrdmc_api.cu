// C ABI of the LRDMC library (declared in include/lrdmc.h): argument
// checks, the host-side double-grid parameters (S-13, Eq. 4, 6, 7), the
// device workspace layout and the launch sequence of one projection step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lrdmc_internal.h"

using namespace lrdmc;

// NVTX ranges around the entry points that launch GPU work, so that a
// profiler's timeline shows the library's calls by name (header-only NVTX
// v3: without a profiler attached a range costs a branch).
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace


struct lrdmc_system_s {
  SysDev S;
  Layout Lo;
  double Zmax;
  int iZmax;
  // population
  int W = 0;
  int trace_cap = 0;
  uint64_t seed = 0;
  double tau = 0.0, e_trial = 0.0;
  int recompute_every = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* rec[2] = {nullptr, nullptr};
  int cur = 0;
  PopDev P;
  uint64_t k = 0;
  bool have_pop = false;
  bool have_eval = false;
  LatDev eval_lat;
  int eval_prec = LRDMC_PRECISION_DF64;  // arithmetic of the cached rates (their storage format)
  int* err_host = nullptr;  // pinned
  int* eval_err = nullptr;  // device error word of lrdmc_evaluate
  // kernel timing (lrdmc_set_profiling)
  bool profiling = false;
  std::vector<cudaEvent_t> events;  // 4 per step: interval start/stop, reconfig start/stop
  size_t ev_used = 0;               // events recorded since the last collection
  bool pending = false;             // steps enqueued since the last synchronisation
  double t_interval_ms = 0.0, t_reconfig_ms = 0.0;
  long long n_interval = 0, n_reconfig = 0;
  std::string last_error;
  int blocks = 0;  // persistent grid of the interval kernel (0 = occupancy default)
  int helpers = 1;  // tail helpers of the interval kernel (lrdmc_set_tail_helpers)
  uint64_t version = 0;  // bumped whenever kernel arguments change (batches re-capture)
  // neural pair term (lrdmc_set_neural_jastrow)
  double* nj_tab = nullptr;
  df* nj_tab_df = nullptr;
  int* base_err = nullptr;
  // per-block partial gradients of lrdmc_nj_backward (grown on demand)
  float* nj_partials = nullptr;
  size_t nj_partials_n = 0;
};

static const char* g_static_error = "";

static lrdmc_status fail(lrdmc_system_t s, lrdmc_status st, const std::string& msg)
{
  if (s) s->last_error = msg;
  else g_static_error = "invalid system handle";
  return st;
}

static lrdmc_status cuda_fail(lrdmc_system_t s, cudaError_t e, const char* where)
{
  return fail(s, LRDMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ----------------------------------------------------------------------------
// Double-grid parameters.
// ----------------------------------------------------------------------------

// S-13: r_c(a, Z) = beta (kappa alpha^-2 + 1) / (alpha^-2 + 1) Z^(-5/7),
// alpha^-2 = (a Z)^2.
static double rc_s13(double a, double Z, double beta, double kappa)
{
  const double aZ2 = (a * Z) * (a * Z);
  return beta * (kappa * aZ2 + 1.0) / (aZ2 + 1.0) * pow(Z, -5.0 / 7.0);
}

// Slater's screening rules for a neutral atom: occupied subshells in
// Madelung order, grouped as (ns,np) or (nd) or (nf); returns per group the
// electron count, n* and the exponent (Z - s)/n*.
struct SlaterGroup {
  int n, kind, occ;  // kind 0 = s/p group, 2 = d, 3 = f
  double nstar, zeta;
};

static std::vector<SlaterGroup> slater_groups(int Z)
{
  static const int order_n[] = {1, 2, 2, 3, 3, 4, 3, 4, 5, 4, 5, 6, 4, 5, 6, 7, 5, 6, 7};
  static const int order_l[] = {0, 0, 1, 0, 1, 0, 2, 1, 0, 2, 1, 0, 3, 2, 1, 0, 3, 2, 1};
  // group list in Slater's left-to-right order
  std::vector<SlaterGroup> g;
  auto rank = [](int n, int kind) {  // position in Slater's ordering
    return n * 10 + (kind == 0 ? 0 : kind);
  };
  int left = Z;
  for (unsigned f = 0; f < sizeof(order_n) / sizeof(int) && left > 0; ++f) {
    int cap = 4 * order_l[f] + 2, put = left < cap ? left : cap;
    int kind = order_l[f] < 2 ? 0 : order_l[f];
    bool found = false;
    for (auto& q : g)
      if (q.n == order_n[f] && q.kind == kind) { q.occ += put; found = true; }
    if (!found) g.push_back({order_n[f], kind, put, 0.0, 0.0});
    left -= put;
  }
  // sort by Slater's ordering
  for (size_t i = 0; i < g.size(); ++i)
    for (size_t j = i + 1; j < g.size(); ++j)
      if (rank(g[j].n, g[j].kind) < rank(g[i].n, g[i].kind)) std::swap(g[i], g[j]);
  static const double nstar_of[] = {0, 1.0, 2.0, 3.0, 3.7, 4.0, 4.2, 4.2};
  for (size_t i = 0; i < g.size(); ++i) {
    double s = (g[i].occ - 1) * (g[i].n == 1 ? 0.30 : 0.35);
    for (size_t j = 0; j < g.size(); ++j) {
      if (j == i) continue;
      if (g[i].kind == 0) {
        int dn = g[i].n - g[j].n;
        if (dn == 1) s += 0.85 * g[j].occ;
        else if (dn >= 2) s += 1.00 * g[j].occ;
      } else if (j < i) {
        s += 1.00 * g[j].occ;
      }
    }
    g[i].nstar = nstar_of[g[i].n];
    g[i].zeta = (Z - s) / g[i].nstar;
  }
  return g;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Eq. 7: N_core(r_c) = int 4 pi r^2 rho_eff(r) exp(-r^2/(2 r_c^2)) dr with
// rho_eff from Slater's effective orbitals (normalised r^(n*-1) e^(-zeta r)).
// Composite 24-point Gauss-Legendre on 240 panels clustered towards r = 0.
static double n_core(int Z, double rc)
{
  auto g = slater_groups(Z);
  double zmin = 1e300;
  for (auto& q : g) zmin = fmin(zmin, q.zeta);
  std::vector<double> gx, gw;
  gauss_legendre(24, gx, gw);
  const double rmax = 90.0 / zmin;
  const int panels = 240;
  double total = 0.0;
  for (int p = 0; p < panels; ++p) {
    double t0 = (double)p / panels, t1 = (double)(p + 1) / panels;
    double r0 = rmax * t0 * t0, r1 = rmax * t1 * t1;
    double half = 0.5 * (r1 - r0), mid = 0.5 * (r1 + r0);
    for (int i = 0; i < 24; ++i) {
      double r = mid + half * gx[i];
      double f = 0.0;
      for (auto& q : g) {
        double lognorm = (2.0 * q.nstar + 1.0) * log(2.0 * q.zeta) - lgamma(2.0 * q.nstar + 1.0);
        f += q.occ * exp(lognorm + 2.0 * q.nstar * log(r) - 2.0 * q.zeta * r);
      }
      if (rc > 0.0 && isfinite(rc)) f *= exp(-r * r / (2.0 * rc * rc));
      total += half * gw[i] * f;
    }
  }
  return total;
}

static lrdmc_status lattice_from(lrdmc_system_t s, double a, const lrdmc_spacing_fn* sp, LatDev& L)
{
  if (!(a > 0.0) || !isfinite(a)) return fail(s, LRDMC_ERR_ARG, "lattice spacing a must be > 0");
  if (!sp) return fail(s, LRDMC_ERR_ARG, "spacing function is NULL");
  memset(&L, 0, sizeof(L));
  L.a = a;
  L.inv2a2 = 0.5 / (a * a);
  double ratio = 1.0, rc = 0.0;
  switch (sp->kind) {
    case LRDMC_SINGLE:
      L.G = 1;
      L.ap = a;
      L.inv2ap2 = L.inv2a2;
      fill_lattice_df(L);
      return LRDMC_OK;
    case LRDMC_DOUBLE_THIS_WORK: {
      if (!(sp->beta > 0.0) || !(sp->kappa > 0.0)) return fail(s, LRDMC_ERR_ARG, "beta and kappa must be > 0");
      if (s->iZmax < 1 || fabs(s->Zmax - s->iZmax) > 1e-12)
        return fail(s, LRDMC_ERR_ARG, "THIS_WORK needs an integer Z_max (Slater's rules)");
      rc = rc_s13(a, s->Zmax, sp->beta, sp->kappa);
      double nc = n_core(s->iZmax, rc);
      ratio = sqrt((s->Zmax - nc) / nc);
      L.pkind = 0;
      break;
    }
    case LRDMC_DOUBLE_PREVIOUS:
      rc = s->Zmax / 2.0;
      ratio = sqrt(s->Zmax * s->Zmax / 4.0 + 1.0);
      L.pkind = 1;
      break;
    case LRDMC_DOUBLE_EXPLICIT:
      if (!(sp->rc > 0.0) || !(sp->aprime_over_a > 0.0)) return fail(s, LRDMC_ERR_ARG, "explicit r_c and a'/a must be > 0");
      rc = sp->rc;
      ratio = sp->aprime_over_a;
      L.pkind = 0;
      break;
    default:
      return fail(s, LRDMC_ERR_ARG, "unknown spacing kind");
  }
  if (!isfinite(ratio) || !(ratio > 0.0)) return fail(s, LRDMC_ERR_ARG, "a'/a is not finite and positive");
  L.G = 2;
  L.ap = a * ratio;
  L.inv2ap2 = 0.5 / (L.ap * L.ap);
  L.rc = rc;
  L.p_coef = (L.pkind == 0) ? 1.0 / (2.0 * rc * rc) : rc * rc;
  fill_lattice_df(L);
  return LRDMC_OK;
}

static bool same_lattice(const LatDev& x, const LatDev& y)
{
  return x.a == y.a && x.ap == y.ap && x.G == y.G && x.pkind == y.pkind && x.rc == y.rc;
}

// ----------------------------------------------------------------------------
// C ABI.
// ----------------------------------------------------------------------------
extern "C" {

lrdmc_status lrdmc_create_system(int n_nuc, const double* nuc_xyz, const double* Z, int n_up,
                                 int n_dn, const lrdmc_shell* shells, int n_shells,
                                 const double* mo_coeff, int n_ao, int n_mo,
                                 const lrdmc_jastrow* jas, lrdmc_system_t* out)
{
  if (!out) return LRDMC_ERR_ARG;
  *out = nullptr;
  if (n_nuc < 1 || n_nuc > kMaxNuc || !nuc_xyz || !Z || !shells || !mo_coeff || !jas) {
    g_static_error = "create_system: bad nuclei or NULL input";
    return LRDMC_ERR_ARG;
  }
  if (n_up < 1 || n_dn < 0 || n_dn > n_up || n_up > kMaxSpin || n_mo < n_up || n_mo > kMaxMO ||
      n_ao < 1 || n_ao > kMaxAO || n_shells < 1 || n_shells > kMaxShell) {
    g_static_error = "create_system: sizes beyond the limits of lrdmc.h";
    return LRDMC_ERR_ARG;
  }
  // every number the kernels read is finite, every charge positive, and no
  // two nuclei coincide (V_nn would be infinite)
  bool finite = std::isfinite(jas->b_ee) && std::isfinite(jas->c_par) && std::isfinite(jas->c_anti) &&
                std::isfinite(jas->en_b2);
  for (int I = 0; I < n_nuc; ++I) {
    finite = finite && Z[I] > 0.0 && std::isfinite(Z[I]) && std::isfinite(jas->en_b1[I]);
    for (int d = 0; d < 3; ++d) finite = finite && std::isfinite(nuc_xyz[3 * I + d]);
  }
  for (int q = 0; q < n_ao * n_mo; ++q) finite = finite && std::isfinite(mo_coeff[q]);
  if (!finite) {
    g_static_error = "create_system: non-finite coordinates, charges, Jastrow or MO coefficients, or a charge <= 0";
    return LRDMC_ERR_ARG;
  }
  for (int I = 0; I < n_nuc; ++I)
    for (int J = I + 1; J < n_nuc; ++J)
      if (nuc_xyz[3 * I] == nuc_xyz[3 * J] && nuc_xyz[3 * I + 1] == nuc_xyz[3 * J + 1] &&
          nuc_xyz[3 * I + 2] == nuc_xyz[3 * J + 2]) {
        g_static_error = "create_system: two nuclei at one point";
        return LRDMC_ERR_ARG;
      }
  lrdmc_system_t s = new lrdmc_system_s();
  SysDev& S = s->S;
  memset(&S, 0, sizeof(S));
  S.n_nuc = n_nuc;
  S.n_up = n_up;
  S.n_dn = n_dn;
  S.N = n_up + n_dn;
  S.n_shell = n_shells;
  S.n_ao = n_ao;
  S.n_mo = n_mo;
  S.ee_on = jas->ee_on ? 1 : 0;
  double zmax = 0.0;
  for (int I = 0; I < n_nuc; ++I) {
    for (int d = 0; d < 3; ++d) S.nuc[I][d] = nuc_xyz[3 * I + d];
    S.Z[I] = Z[I];
    S.en_b1[I] = jas->en_b1[I];
    zmax = fmax(zmax, Z[I]);
  }
  for (int I = 0; I < n_nuc; ++I) S.heavy[I] = (Z[I] == zmax) ? 1 : 0;
  s->Zmax = zmax;
  s->iZmax = (int)lround(zmax);
  S.b_ee = jas->b_ee;
  S.c_par = jas->c_par;
  S.c_anti = jas->c_anti;
  S.en_b2 = jas->en_b2;
  double vnn = 0.0;
  for (int I = 0; I < n_nuc; ++I)
    for (int J = I + 1; J < n_nuc; ++J) {
      double dx = S.nuc[I][0] - S.nuc[J][0], dy = S.nuc[I][1] - S.nuc[J][1], dz = S.nuc[I][2] - S.nuc[J][2];
      vnn += Z[I] * Z[J] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  S.V_nn = vnn;
  // shells are stored sorted by centre (stable); AOs follow the sorted
  // shells, so the MO coefficient rows are permuted to match
  int order[kMaxShell];
  {
    int n = 0;
    for (int I = 0; I < n_nuc; ++I) {
      S.nuc_shell_begin[I] = n;
      for (int q = 0; q < n_shells; ++q)
        if (shells[q].center == I) order[n++] = q;
    }
    S.nuc_shell_begin[n_nuc] = n;
    if (n != n_shells) {
      delete s;
      g_static_error = "create_system: invalid shell centre";
      return LRDMC_ERR_ARG;
    }
  }
  int user_off[kMaxShell];
  {
    int o = 0;
    for (int q = 0; q < n_shells; ++q) {
      user_off[q] = o;
      o += 2 * shells[q].l + 1;
    }
  }
  int off = 0;
  for (int qs = 0; qs < n_shells; ++qs) {
    const int q = order[qs];
    const lrdmc_shell& in = shells[q];
    ShellDev& sh = S.sh[qs];
    if (in.center < 0 || in.center >= n_nuc || in.l < 0 || in.l > 2 || (in.kind != 0 && in.kind != 1) ||
        (in.kind == 1 && (in.n_prim < 1 || in.n_prim > kMaxPrim)) ||
        (in.kind == 0 && !(in.zeta > 0.0)) || (in.kind == 0 && in.n_eff - 1.0 - in.l < 0.0)) {
      delete s;
      g_static_error = "create_system: invalid shell";
      return LRDMC_ERR_ARG;
    }
    sh.center = in.center;
    sh.l = in.l;
    sh.kind = in.kind;
    sh.n_prim = in.kind == 1 ? in.n_prim : 0;
    sh.ao_offset = off;
    sh.m = in.n_eff - 1.0 - in.l;
    sh.zeta = in.zeta;
    double mr = nearbyint(sh.m);
    sh.m_int = (in.kind == 0 && fabs(sh.m - mr) == 0.0 && mr <= 8.0) ? (int)mr : -1;
    for (int p = 0; p < kMaxPrim; ++p) {
      sh.alpha[p] = in.alpha[p];
      sh.coef[p] = in.coef[p];
    }
    const lrdmc_shell* prev = qs > 0 ? &shells[order[qs - 1]] : nullptr;
    sh.same_exp = (prev && in.kind == 0 && prev->kind == 0 && prev->center == in.center && prev->zeta == in.zeta)
                      ? 1 : 0;
    off += 2 * in.l + 1;
  }
  if (off != n_ao) {
    delete s;
    g_static_error = "create_system: n_ao differs from the shells' 2l+1 count";
    return LRDMC_ERR_ARG;
  }
  // the local energy's parts per electron (32 / N lanes, one beyond 32
  // electrons) deal out single shells when they outnumber the shells
  const int el_parts = S.N <= 32 ? 32 / S.N : 1;
  S.n_grp = 0;
  for (int qs = 0; qs < n_shells; ++qs)
    if (n_shells <= el_parts || !(S.sh[qs].kind == 0 && S.sh[qs].same_exp)) S.grp_first[S.n_grp++] = qs;
  S.grp_first[S.n_grp] = n_shells;
  for (int qs = 0; qs < n_shells; ++qs) {
    const int q = order[qs];
    for (int f = 0; f < 2 * shells[q].l + 1; ++f)
      for (int m = 0; m < n_mo; ++m)
        S.C[(S.sh[qs].ao_offset + f) * n_mo + m] = mo_coeff[(user_off[q] + f) * n_mo + m];
  }
  S.precision = LRDMC_PRECISION_DF64;
  fill_df_constants(S);
  // one block holds kWarpsPerBlock walkers in shared memory; without room
  // for the evaluation caches the system runs without them, and a system
  // that does not fit even then is rejected
  s->Lo = make_layout(S, true);
  if (s->Lo.smem_block_bytes > kMaxSmemBlock) s->Lo = make_layout(S, false);
  if (s->Lo.smem_block_bytes > kMaxSmemBlock) {
    static std::string msg;
    msg = "create_system: " + std::to_string(S.N) + " electrons with " + std::to_string(n_ao) +
          " AOs need " + std::to_string(s->Lo.smem_block_bytes / 1024) + " KB of shared memory per block of " +
          std::to_string(kWarpsPerBlock) + " walkers (at most " + std::to_string(kMaxSmemBlock / 1024) + " KB)";
    g_static_error = msg.c_str();
    delete s;
    return LRDMC_ERR_ARG;
  }
  *out = s;
  return LRDMC_OK;
}

lrdmc_status lrdmc_spacing_params(lrdmc_system_t s, double a, const lrdmc_spacing_fn* sp,
                                  double* aprime_over_a, double* rc)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  LatDev L;
  lrdmc_status st = lattice_from(s, a, sp, L);
  if (st != LRDMC_OK) return st;
  if (aprime_over_a) *aprime_over_a = (L.G == 2) ? L.ap / a : 1.0;
  if (rc) *rc = L.rc;
  return LRDMC_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsPlan {
  size_t rec, parent, order, logw, wgt, el, jumps, cum, part, trace, moves, err, counter, kdev, resid, ticket,
      total;
};

static WsPlan plan_ws(const Layout& Lo, int W, int cap)
{
  WsPlan p;
  size_t o = 0;
  p.rec = o; o += align256(sizeof(double) * (size_t)W * Lo.rec) * 2;
  p.parent = o; o += align256(sizeof(int) * (size_t)W);
  p.order = o; o += align256(sizeof(int) * (size_t)W);
  p.logw = o; o += align256(sizeof(double) * (size_t)W);
  p.wgt = o; o += align256(sizeof(double) * (size_t)W);
  p.el = o; o += align256(sizeof(double) * (size_t)W);
  p.jumps = o; o += align256(sizeof(int) * (size_t)W);
  p.cum = o; o += align256(sizeof(double) * (size_t)W);
  p.part = o; o += align256(sizeof(CombPart) * kMaxCombBlocks);
  p.trace = o; o += align256(sizeof(double) * 4 * (size_t)cap);
  // six words cleared together at initialisation
  p.moves = o; o += 256;
  p.err = o; o += 256;
  p.counter = o; o += 256;
  p.kdev = o; o += 256;
  p.resid = o; o += 256;
  p.ticket = o; o += 256;
  p.total = o;
  return p;
}

lrdmc_status lrdmc_workspace_bytes(lrdmc_system_t s, int n_walkers, int cap, size_t* bytes)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (n_walkers < 1 || n_walkers > kMaxWalkers || cap < 1 || !bytes)
    return fail(s, LRDMC_ERR_ARG, "workspace_bytes: bad sizes");
  *bytes = plan_ws(s->Lo, n_walkers, cap).total;
  return LRDMC_OK;
}

static lrdmc_status read_error_word(lrdmc_system_t s)
{
  cudaError_t e = cudaMemcpyAsync(s->err_host, s->P.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "error word read");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  int w = *s->err_host;
  if (w & kErrSingular) return fail(s, LRDMC_ERR_SINGULAR, "singular Slater matrix or zero update ratio");
  if (w & kErrNonFinite) return fail(s, LRDMC_ERR_NONFINITE, "non-finite local energy or rate");
  if (w & kErrIters) return fail(s, LRDMC_ERR_TIMEOUT, "an interval exceeded its iteration limit");
  if (w & kErrTimeout) return fail(s, LRDMC_ERR_TIMEOUT, "a bounded wait of the interval kernel's tail helpers ran out");
  if (w & kErrBounds) return fail(s, LRDMC_ERR_BOUNDS, "a checked walker index was out of range");
  return LRDMC_OK;
}

lrdmc_status lrdmc_init_walkers(lrdmc_system_t s, int W, const double* x0, uint64_t seed, double tau,
                                double e_trial, int recompute_every, int cap, void* workspace,
                                size_t ws_bytes, void* stream)
{
  NvtxRange nvtx("lrdmc_init_walkers");
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (W < 1 || cap < 1 || !x0 || !workspace) return fail(s, LRDMC_ERR_ARG, "init_walkers: bad arguments");
  if (W > kMaxWalkers) return fail(s, LRDMC_ERR_ARG, "init_walkers: more than LRDMC_MAX_WALKERS walkers");
  if (!(tau > 0.0) || !isfinite(tau) || !isfinite(e_trial) || recompute_every < 0)
    return fail(s, LRDMC_ERR_ARG, "init_walkers: tau must be > 0, recompute_every >= 0");
  if (((uintptr_t)workspace & 255) != 0) return fail(s, LRDMC_ERR_ARG, "init_walkers: workspace not 256-byte aligned");
  WsPlan p = plan_ws(s->Lo, W, cap);
  if (ws_bytes < p.total) return fail(s, LRDMC_ERR_ARG, "init_walkers: workspace too small");
  if (!s->err_host) {
    cudaError_t e = cudaMallocHost((void**)&s->err_host, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(s, e, "pinned error word");
  }
  s->W = W;
  s->trace_cap = cap;
  s->seed = seed;
  s->tau = tau;
  s->e_trial = e_trial;
  s->recompute_every = recompute_every;
  s->stream = (cudaStream_t)stream;
  s->ws = (char*)workspace;
  s->ws_bytes = ws_bytes;
  size_t recb = align256(sizeof(double) * (size_t)W * s->Lo.rec);
  s->rec[0] = (double*)(s->ws + p.rec);
  s->rec[1] = (double*)(s->ws + p.rec + recb);
  s->cur = 0;
  PopDev& P = s->P;
  P.parent = (int*)(s->ws + p.parent);
  P.order = (int*)(s->ws + p.order);
  P.logw = (double*)(s->ws + p.logw);
  P.wgt = (double*)(s->ws + p.wgt);
  P.el_end = (double*)(s->ws + p.el);
  P.jumps = (int*)(s->ws + p.jumps);
  P.cum = (double*)(s->ws + p.cum);
  P.part = (CombPart*)(s->ws + p.part);
  P.ticket = (int*)(s->ws + p.ticket);
  P.trace = (double*)(s->ws + p.trace);
  P.moves = (unsigned long long*)(s->ws + p.moves);
  P.err = (int*)(s->ws + p.err);
  P.counter = (int*)(s->ws + p.counter);
  P.kdev = (unsigned long long*)(s->ws + p.kdev);
  P.resid = (unsigned long long*)(s->ws + p.resid);
  P.recompute_every = recompute_every;
  P.W = W;
  P.trace_cap = cap;
  P.seed = seed;
  P.tau = tau;
  P.e_trial = e_trial;
  P.helpers = s->helpers;
  // moves, err, counter, kdev, resid, ticket
  cudaError_t e = cudaMemsetAsync(s->ws + p.moves, 0, 6 * 256, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "workspace clear");
  e = cudaMemsetAsync(P.logw, 0, sizeof(double) * W, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.wgt, 0, sizeof(double) * W, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.jumps, 0, sizeof(int) * W, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "workspace clear");
  // stage x0 (host or device memory) in the second record buffer
  double* stage = s->rec[1];
  e = cudaMemcpyAsync(stage, x0, sizeof(double) * (size_t)W * 3 * s->S.N, cudaMemcpyDefault, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "x0 copy");
  P.rec_src = s->rec[0];
  P.rec_dst = s->rec[1];
  e = launch_init(s->S, s->Lo, P, stage, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "k_init launch");
  s->k = 0;
  s->have_pop = true;
  s->have_eval = false;
  s->version++;
  return read_error_word(s);
}

lrdmc_status lrdmc_step(lrdmc_system_t s, int n_steps, double a, const lrdmc_spacing_fn* sp)
{
  NvtxRange nvtx("lrdmc_step");
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "step before init_walkers");
  if (n_steps < 0) return fail(s, LRDMC_ERR_ARG, "n_steps < 0");
  if (s->k + (uint64_t)n_steps > (uint64_t)s->trace_cap)
    return fail(s, LRDMC_ERR_ARG, "step: the trace would exceed trace_capacity");
  LatDev L;
  lrdmc_status st = lattice_from(s, a, sp, L);
  if (st != LRDMC_OK) return st;
  cudaError_t e;
  if (s->profiling) {
    while (s->events.size() < s->ev_used + 4 * (size_t)n_steps) {
      cudaEvent_t ev;
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(s, e, "profiling event");
      s->events.push_back(ev);
    }
  }
  PopDev P = s->P;
  if (!s->have_eval || !same_lattice(L, s->eval_lat)) {
    P.rec_src = s->rec[s->cur];
    P.rec_dst = s->rec[1 - s->cur];
    e = launch_eval_all(s->S, s->Lo, L, P, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "k_eval_all launch");
    s->have_eval = true;
    s->eval_lat = L;
    s->eval_prec = s->S.precision;
  }
  for (int n = 0; n < n_steps; ++n) {
    P.rec_src = s->rec[s->cur];
    P.rec_dst = s->rec[1 - s->cur];
    cudaEvent_t* ev = nullptr;
    if (s->profiling) {
      ev = &s->events[s->ev_used];
      s->ev_used += 4;
    }
    if (ev) cudaEventRecord(ev[0], s->stream);
    e = launch_interval(s->S, s->Lo, L, P, s->blocks, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "k_interval launch");
    if (ev) {
      cudaEventRecord(ev[1], s->stream);
      cudaEventRecord(ev[2], s->stream);
    }
    e = launch_reconfig(P, s->Lo, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "reconfiguration launch");
    if (ev) cudaEventRecord(ev[3], s->stream);
    s->cur = 1 - s->cur;
    s->k++;
  }
  // the error word travels to pinned host memory behind the step's kernels;
  // it is examined at the next synchronising call
  e = cudaMemcpyAsync(s->err_host, s->P.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "error word read");
  s->pending = true;
  return LRDMC_OK;
}

// Waits for the stream, folds the recorded kernel events into the timing
// totals and reports the device error word.
static lrdmc_status sync_system(lrdmc_system_t s)
{
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  for (size_t n = 0; n + 3 < s->ev_used; n += 4) {
    float a_ms = 0.f, b_ms = 0.f;
    cudaEventElapsedTime(&a_ms, s->events[n], s->events[n + 1]);
    cudaEventElapsedTime(&b_ms, s->events[n + 2], s->events[n + 3]);
    s->t_interval_ms += a_ms;
    s->t_reconfig_ms += b_ms;
    s->n_interval += 1;
    s->n_reconfig += 1;
  }
  s->ev_used = 0;
  if (!s->pending) return LRDMC_OK;
  s->pending = false;
  int w = *s->err_host;
  if (w & kErrSingular) return fail(s, LRDMC_ERR_SINGULAR, "singular Slater matrix or zero update ratio");
  if (w & kErrNonFinite) return fail(s, LRDMC_ERR_NONFINITE, "non-finite local energy or rate");
  if (w & kErrIters) return fail(s, LRDMC_ERR_TIMEOUT, "an interval exceeded its iteration limit");
  if (w & kErrTimeout) return fail(s, LRDMC_ERR_TIMEOUT, "a bounded wait of the interval kernel's tail helpers ran out");
  if (w & kErrBounds) return fail(s, LRDMC_ERR_BOUNDS, "a checked walker index was out of range");
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_energy_trace(lrdmc_system_t s, double* e_out, double* w_out, double* j_out,
                                    int max_n, int* n_written)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "trace before init_walkers");
  lrdmc_status ss = sync_system(s);
  if (ss != LRDMC_OK) return ss;
  int n = (int)((uint64_t)max_n < s->k ? (uint64_t)max_n : s->k);
  if (n < 0) n = 0;
  double* outs[3] = {e_out, w_out, j_out};
  for (int r = 0; r < 3; ++r) {
    if (!outs[r] || n == 0) continue;
    cudaError_t e = cudaMemcpyAsync(outs[r], s->P.trace + (size_t)r * s->trace_cap, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "trace copy");
  }
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  if (n_written) *n_written = n;
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_energy_trace_async(lrdmc_system_t s, int first, int n, double* e_out, double* w_out,
                                          double* j_out)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "trace before init_walkers");
  if (first < 0 || n < 0 || (uint64_t)first + (uint64_t)n > s->k)
    return fail(s, LRDMC_ERR_ARG, "energy_trace_async: entries beyond the intervals stepped");
  double* outs[3] = {e_out, w_out, j_out};
  for (int r = 0; r < 3; ++r) {
    if (!outs[r] || n == 0) continue;
    cudaError_t e = cudaMemcpyAsync(outs[r], s->P.trace + (size_t)r * s->trace_cap + first, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "trace copy");
  }
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_residual_trace(lrdmc_system_t s, double* resid, int max_n, int* n_written)
{
  if (!s || !resid) return fail(s, LRDMC_ERR_ARG, "residual_trace: NULL");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "residual trace before init_walkers");
  lrdmc_status ss = sync_system(s);
  if (ss != LRDMC_OK) return ss;
  int n = (int)((uint64_t)max_n < s->k ? (uint64_t)max_n : s->k);
  if (n < 0) n = 0;
  if (n > 0) {
    cudaError_t e = cudaMemcpyAsync(resid, s->P.trace + (size_t)3 * s->trace_cap, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "residual trace copy");
  }
  if (n_written) *n_written = n;
  return LRDMC_OK;
}

lrdmc_status lrdmc_get_walkers(lrdmc_system_t s, double* x, double* el, double* b, double* T,
                               double* logw_pre, int* jumps_pre, int* parent)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "get_walkers before init_walkers");
  lrdmc_status ss = sync_system(s);
  if (ss != LRDMC_OK) return ss;
  const int W = s->W;
  const Layout& Lo = s->Lo;
  std::vector<double> rec((size_t)W * Lo.rec);
  std::vector<int> par(W);
  cudaError_t e = cudaMemcpyAsync(rec.data(), s->rec[s->cur], sizeof(double) * rec.size(),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(par.data(), s->P.parent, sizeof(int) * W, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && logw_pre)
    e = cudaMemcpyAsync(logw_pre, s->P.logw, sizeof(double) * W, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && jumps_pre)
    e = cudaMemcpyAsync(jumps_pre, s->P.jumps, sizeof(int) * W, cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "walker copy");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
  const int P = s->have_eval ? s->S.N * 6 * s->eval_lat.G : 0;
  for (int t = 0; t < W; ++t) {
    const double* r = &rec[(size_t)par[t] * Lo.rec];
    if (x) memcpy(&x[(size_t)t * 3 * Lo.N], r + Lo.off_x, sizeof(double) * 3 * Lo.N);
    if (el) el[t] = r[Lo.off_el];
    if (b) b[t] = r[Lo.off_b];
    if (T && P) {
      if (s->eval_prec != LRDMC_PRECISION_FP64) {
        // rates cached as double-floats (two floats per slot)
        const float* f = reinterpret_cast<const float*>(r + Lo.off_T);
        for (int c = 0; c < P; ++c) T[(size_t)t * P + c] = (double)f[2 * c] + (double)f[2 * c + 1];
      } else {
        memcpy(&T[(size_t)t * P], r + Lo.off_T, sizeof(double) * P);
      }
    }
  }
  if (parent) memcpy(parent, par.data(), sizeof(int) * W);
  return LRDMC_OK;
}

lrdmc_status lrdmc_moves(lrdmc_system_t s, long long* moves)
{
  if (!s || !moves) return fail(s, LRDMC_ERR_ARG, "moves: NULL");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "moves before init_walkers");
  lrdmc_status ss = sync_system(s);
  if (ss != LRDMC_OK) return ss;
  unsigned long long m = 0;
  cudaError_t e = cudaMemcpyAsync(&m, s->P.moves, sizeof(m), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "moves copy");
  *moves = (long long)m;
  return LRDMC_OK;
}

lrdmc_status lrdmc_evaluate(lrdmc_system_t s, int n, const double* x, const double* rot, double a,
                            const lrdmc_spacing_fn* sp, double* ratio, double* T, double* b,
                            double* el, void* stream)
{
  NvtxRange nvtx("lrdmc_evaluate");
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (n < 0 || (n > 0 && (!x || !rot))) return fail(s, LRDMC_ERR_ARG, "evaluate: bad arguments");
  if (n == 0) return LRDMC_OK;
  LatDev L;
  lrdmc_status st = lattice_from(s, a, sp, L);
  if (st != LRDMC_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!s->eval_err) e = cudaMalloc((void**)&s->eval_err, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(s, e, "evaluate error word");
  if (!s->err_host) e = cudaMallocHost((void**)&s->err_host, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(s, e, "pinned error word");
  e = cudaMemsetAsync(s->eval_err, 0, sizeof(int), cs);
  if (e == cudaSuccess) e = launch_evaluate(s->S, s->Lo, L, n, x, rot, ratio, T, b, el, s->eval_err, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->err_host, s->eval_err, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(s, e, "evaluate");
  int h = *s->err_host;
  if (h & kErrSingular) return fail(s, LRDMC_ERR_SINGULAR, "evaluate: singular Slater matrix");
  return LRDMC_OK;
}

lrdmc_status lrdmc_evaluate_tc(lrdmc_system_t s, int n, const double* x, const double* rot, double a,
                               const lrdmc_spacing_fn* sp, double* ratio, double* T, double* b, double* el,
                               void* stream)
{
  NvtxRange nvtx("lrdmc_evaluate_tc");
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (n < 0 || (n > 0 && (!x || !rot))) return fail(s, LRDMC_ERR_ARG, "evaluate_tc: bad arguments");
  if (s->S.n_mo > 32) return fail(s, LRDMC_ERR_ARG, "evaluate_tc: more than 32 orbitals per spin");
  if (evaluate_tc_smem_bytes(s->S, s->Lo) > kMaxSmemBlock)
    return fail(s, LRDMC_ERR_ARG, "evaluate_tc: the block's shared memory with the tensor-core tiles exceeds " +
                                      std::to_string(kMaxSmemBlock / 1024) + " KB");
  if (n == 0) return LRDMC_OK;
  LatDev L;
  lrdmc_status st = lattice_from(s, a, sp, L);
  if (st != LRDMC_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!s->eval_err) e = cudaMalloc((void**)&s->eval_err, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(s, e, "evaluate error word");
  if (!s->err_host) e = cudaMallocHost((void**)&s->err_host, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(s, e, "pinned error word");
  e = cudaMemsetAsync(s->eval_err, 0, sizeof(int), cs);
  if (e == cudaSuccess) e = launch_evaluate_tc(s->S, s->Lo, L, n, x, rot, ratio, T, b, el, s->eval_err, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->err_host, s->eval_err, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(s, e, "evaluate_tc");
  int h = *s->err_host;
  if (h & kErrTimeout) return fail(s, LRDMC_ERR_TIMEOUT, "evaluate_tc: the tensor-core barrier wait ran out");
  if (h & kErrSingular) return fail(s, LRDMC_ERR_SINGULAR, "evaluate_tc: singular Slater matrix");
  return LRDMC_OK;
}

lrdmc_status lrdmc_evaluate_static(lrdmc_system_t s, int n, const double* x, const double* rot,
                                   double a, const lrdmc_spacing_fn* sp, double* ratio, double* T,
                                   double* b, double* el, void* stream)
{
  NvtxRange nvtx("lrdmc_evaluate_static");
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (n < 0 || (n > 0 && (!x || !rot))) return fail(s, LRDMC_ERR_ARG, "evaluate_static: bad arguments");
  if (n > LRDMC_STATIC_EVAL_MAX)
    return fail(s, LRDMC_ERR_ARG, "evaluate_static: n_configs exceeds LRDMC_STATIC_EVAL_MAX (" +
                                      std::to_string(LRDMC_STATIC_EVAL_MAX) + "); split the batch");
  if (n == 0) return LRDMC_OK;
  LatDev L;
  lrdmc_status st = lattice_from(s, a, sp, L);
  if (st != LRDMC_OK) return st;
  int summary = 0, first_bad = -1;
  cudaError_t e = launch_evaluate_static(s->S, s->Lo, L, n, x, rot, ratio, T, b, el, &summary, &first_bad,
                                         (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "evaluate_static");
  if (summary & kErrSingular)
    return fail(s, LRDMC_ERR_SINGULAR, "evaluate_static: singular Slater matrix (first at configuration " +
                                           std::to_string(first_bad) + ")");
  return LRDMC_OK;
}

// Checkpoint file: magic, sizes, counters, then the current record buffer,
// parents, trace and the moves counter.
static const uint64_t kMagic = 0x4C52444D43303032ull;  // "LRDMC002" (four trace columns)

lrdmc_status lrdmc_save(lrdmc_system_t s, const char* path)
{
  if (!s || !path) return fail(s, LRDMC_ERR_ARG, "save: NULL");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "save before init_walkers");
  lrdmc_status ss = sync_system(s);
  if (ss != LRDMC_OK) return ss;
  const int W = s->W;
  std::vector<double> rec((size_t)W * s->Lo.rec), trace(4 * (size_t)s->trace_cap);
  std::vector<int> par(W);
  unsigned long long moves = 0;
  cudaError_t e = cudaMemcpyAsync(rec.data(), s->rec[s->cur], sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(par.data(), s->P.parent, sizeof(int) * W, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(trace.data(), s->P.trace, sizeof(double) * trace.size(), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&moves, s->P.moves, sizeof(moves), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "save copy");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(s, LRDMC_ERR_ARG, std::string("save: cannot open ") + path);
  int64_t hdr[8] = {(int64_t)kMagic, W, s->Lo.rec, s->trace_cap, (int64_t)s->k, s->have_eval ? 1 : 0,
                    s->eval_prec, 0};
  bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&s->eval_lat, sizeof(LatDev), 1, f) == 1 &&
            fwrite(rec.data(), sizeof(double), rec.size(), f) == rec.size() &&
            fwrite(par.data(), sizeof(int), W, f) == (size_t)W &&
            fwrite(trace.data(), sizeof(double), trace.size(), f) == trace.size() &&
            fwrite(&moves, sizeof(moves), 1, f) == 1;
  fclose(f);
  return ok ? LRDMC_OK : fail(s, LRDMC_ERR_ARG, "save: write failed");
}

lrdmc_status lrdmc_load(lrdmc_system_t s, const char* path)
{
  if (!s || !path) return fail(s, LRDMC_ERR_ARG, "load: NULL");
  if (!s->have_pop) return fail(s, LRDMC_ERR_STATE, "load needs an initialised population of the same size");
  lrdmc_status ss = sync_system(s);
  if (ss != LRDMC_OK) return ss;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(s, LRDMC_ERR_ARG, std::string("load: cannot open ") + path);
  int64_t hdr[8];
  LatDev L;
  bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && fread(&L, sizeof(LatDev), 1, f) == 1;
  if (!ok || hdr[0] != (int64_t)kMagic || hdr[1] != s->W || hdr[2] != s->Lo.rec || hdr[3] != s->trace_cap) {
    fclose(f);
    return fail(s, LRDMC_ERR_ARG, "load: file does not match this population");
  }
  const int W = s->W;
  std::vector<double> rec((size_t)W * s->Lo.rec), trace(4 * (size_t)s->trace_cap);
  std::vector<int> par(W);
  unsigned long long moves = 0;
  ok = fread(rec.data(), sizeof(double), rec.size(), f) == rec.size() &&
       fread(par.data(), sizeof(int), W, f) == (size_t)W &&
       fread(trace.data(), sizeof(double), trace.size(), f) == trace.size() &&
       fread(&moves, sizeof(moves), 1, f) == 1;
  fclose(f);
  if (!ok) return fail(s, LRDMC_ERR_ARG, "load: truncated file");
#ifndef LRDMC_BOUNDS  // the bounds-checked build leaves them to the kernels' checks
  for (int t = 0; t < W; ++t)
    if (par[t] < 0 || par[t] >= W) return fail(s, LRDMC_ERR_ARG, "load: corrupt parent index");
#endif
  s->cur = 0;
  cudaError_t e = cudaMemcpyAsync(s->rec[0], rec.data(), sizeof(double) * rec.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->P.parent, par.data(), sizeof(int) * W, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->P.trace, trace.data(), sizeof(double) * trace.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->P.moves, &moves, sizeof(moves), cudaMemcpyHostToDevice, s->stream);
  const unsigned long long kload = (unsigned long long)hdr[4];
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->P.kdev, &kload, sizeof(kload), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "load copy");
  s->k = (uint64_t)hdr[4];
  s->version++;
  s->have_eval = hdr[5] != 0 && hdr[6] == s->S.precision;
  s->eval_prec = (int)hdr[6];
  s->eval_lat = L;
  return LRDMC_OK;
}

lrdmc_status lrdmc_set_precision(lrdmc_system_t s, int precision)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (precision != LRDMC_PRECISION_FP64 && precision != LRDMC_PRECISION_DF64 && precision != LRDMC_PRECISION_FP32)
    return fail(s, LRDMC_ERR_ARG, "set_precision: unknown precision");
  if (precision != s->S.precision) s->have_eval = false;  // cached rates change format
  s->S.precision = precision;
  s->version++;
  return LRDMC_OK;
}

lrdmc_status lrdmc_set_profiling(lrdmc_system_t s, int on)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  s->profiling = on != 0;
  return LRDMC_OK;
}

lrdmc_status lrdmc_sync(lrdmc_system_t s)
{
  NvtxRange nvtx("lrdmc_sync");
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (!s->have_pop) return LRDMC_OK;
  return sync_system(s);
}

lrdmc_status lrdmc_kernel_times(lrdmc_system_t s, double* interval_ms, double* reconfig_ms,
                                long long* interval_launches, long long* reconfig_launches, int reset)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (s->have_pop) {
    lrdmc_status ss = sync_system(s);
    if (ss != LRDMC_OK) return ss;
  }
  if (interval_ms) *interval_ms = s->t_interval_ms;
  if (reconfig_ms) *reconfig_ms = s->t_reconfig_ms;
  if (interval_launches) *interval_launches = s->n_interval;
  if (reconfig_launches) *reconfig_launches = s->n_reconfig;
  if (reset) {
    s->t_interval_ms = s->t_reconfig_ms = 0.0;
    s->n_interval = s->n_reconfig = 0;
  }
  return LRDMC_OK;
}

// ---------------------------------------------------------------------------
// Neural pair term.
// ---------------------------------------------------------------------------
static bool nj_spec_ok(lrdmc_system_t s, const lrdmc_nj_spec* sp, std::string& why)
{
  if (!sp) { why = "spec is NULL"; return false; }
  if (sp->n_feat < 1 || sp->n_feat > LRDMC_NJ_MAX_FEAT || !sp->ell) { why = "n_feat out of range"; return false; }
  for (int f = 0; f < sp->n_feat; ++f)
    if (!(sp->ell[f] > 0.0) || !isfinite(sp->ell[f])) { why = "ell must be positive and finite"; return false; }
  if (sp->n_ch < 2 || sp->n_ch > LRDMC_NJ_MAX_CH || !sp->r_cut) { why = "n_ch out of range"; return false; }
  for (int c = 0; c < sp->n_ch; ++c)
    if (!(sp->r_cut[c] > 0.0) || !isfinite(sp->r_cut[c])) { why = "r_cut must be positive and finite"; return false; }
  if (!sp->species) { why = "species is NULL"; return false; }
  for (int I = 0; I < s->S.n_nuc; ++I)
    if (sp->species[I] < 0 || 2 + sp->species[I] >= sp->n_ch) { why = "species out of range"; return false; }
  if (sp->hidden != LRDMC_NJ_HIDDEN) { why = "hidden must equal LRDMC_NJ_HIDDEN"; return false; }
  if (sp->n_cells < 1 || sp->n_cells > LRDMC_NJ_MAX_CELLS) { why = "n_cells out of range"; return false; }
  return true;
}

static NjGeom nj_geom(lrdmc_system_t s, const lrdmc_nj_spec* sp)
{
  NjGeom G{};
  G.N = s->S.N;
  G.n_up = s->S.n_up;
  G.n_nuc = s->S.n_nuc;
  G.n_pairs = G.N * (G.N - 1) / 2 + G.N * G.n_nuc;
  for (int I = 0; I < G.n_nuc; ++I) {
    for (int k = 0; k < 3; ++k) G.nuc[I][k] = s->S.nuc[I][k];
    G.species[I] = sp->species[I];
  }
  return G;
}

static NjNetDev nj_net(const lrdmc_nj_spec* sp)
{
  NjNetDev N{};
  N.F = sp->n_feat;
  N.C = sp->n_ch;
  N.D = N.F + N.C;
  N.bf16 = sp->bf16 != 0;
  for (int f = 0; f < N.F; ++f) N.ell2[f] = (float)(sp->ell[f] * sp->ell[f]);
  for (int c = 0; c < N.C; ++c) N.rcut[c] = (float)sp->r_cut[c];
  return N;
}

int lrdmc_nj_n_params(const lrdmc_nj_spec* sp)
{
  if (!sp || sp->n_feat < 1 || sp->n_feat > LRDMC_NJ_MAX_FEAT || sp->n_ch < 2 || sp->n_ch > LRDMC_NJ_MAX_CH ||
      sp->hidden != LRDMC_NJ_HIDDEN)
    return 0;
  return nj_n_params(sp->n_feat, sp->n_ch, sp->hidden);
}

lrdmc_status lrdmc_set_neural_jastrow(lrdmc_system_t s, const lrdmc_nj_spec* sp, const float* params)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (!sp) {
    s->S.nj_on = 0;
    s->have_eval = false;
    s->version++;
    return LRDMC_OK;
  }
  std::string why;
  if (!nj_spec_ok(s, sp, why)) return fail(s, LRDMC_ERR_ARG, "set_neural_jastrow: " + why);
  if (!params) return fail(s, LRDMC_ERR_ARG, "set_neural_jastrow: params is NULL");
  const int np = nj_n_params(sp->n_feat, sp->n_ch, sp->hidden);
  for (int q = 0; q < np; ++q)
    if (!isfinite(params[q])) return fail(s, LRDMC_ERR_ARG, "set_neural_jastrow: non-finite parameter");
  std::vector<double> tab;
  nj_build_table(*sp, params, tab);
  for (double v : tab)
    if (!isfinite(v)) return fail(s, LRDMC_ERR_NONFINITE, "set_neural_jastrow: non-finite table entry");
  std::vector<df> tdf(tab.size());
  for (size_t q = 0; q < tab.size(); ++q) {
    const float hi = (float)tab[q];
    tdf[q] = df_make(hi, (float)(tab[q] - (double)hi));
  }
  if (s->nj_tab) cudaFree(s->nj_tab);
  if (s->nj_tab_df) cudaFree(s->nj_tab_df);
  s->nj_tab = nullptr;
  s->nj_tab_df = nullptr;
  s->S.nj_on = 0;
  cudaError_t e = cudaMalloc((void**)&s->nj_tab, sizeof(double) * tab.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->nj_tab_df, sizeof(df) * tdf.size());
  if (e == cudaSuccess) e = cudaMemcpy(s->nj_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->nj_tab_df, tdf.data(), sizeof(df) * tdf.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(s, e, "set_neural_jastrow upload");
  s->S.nj_tab = s->nj_tab;
  s->S.nj_tab_df = s->nj_tab_df;
  s->S.nj_cells = sp->n_cells;
  for (int c = 0; c < sp->n_ch; ++c) {
    s->S.nj_rcut[c] = sp->r_cut[c];
    s->S.nj_rcut_f[c] = (float)sp->r_cut[c];
    s->S.nj_scale_f[c] = (float)(sp->n_cells / sqrt(sp->r_cut[c]));
  }
  for (int I = 0; I < s->S.n_nuc; ++I) s->S.nj_species[I] = sp->species[I];
  s->S.nj_on = 1;
  s->have_eval = false;
  s->version++;
  return LRDMC_OK;
}

lrdmc_status lrdmc_base_terms(lrdmc_system_t s, int n, const double* x, double* grad_out, double* e_out,
                              void* stream)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (n < 0 || (n > 0 && (!x || !grad_out || !e_out))) return fail(s, LRDMC_ERR_ARG, "base_terms: bad arguments");
  if (n == 0) return LRDMC_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!s->base_err) e = cudaMalloc((void**)&s->base_err, sizeof(int));
  if (e == cudaSuccess && !s->err_host) e = cudaMallocHost((void**)&s->err_host, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(s, e, "base_terms error word");
  SysDev S = s->S;
  S.nj_on = 0;  // the base terms exclude the neural term
  e = cudaMemsetAsync(s->base_err, 0, sizeof(int), cs);
  if (e == cudaSuccess) e = launch_base_terms(S, s->Lo, n, x, grad_out, e_out, s->base_err, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->err_host, s->base_err, sizeof(int), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(s, e, "base_terms");
  if (*s->err_host & kErrSingular) return fail(s, LRDMC_ERR_SINGULAR, "base_terms: singular Slater matrix");
  return LRDMC_OK;
}

lrdmc_status lrdmc_nj_forward(lrdmc_system_t s, const lrdmc_nj_spec* sp, const float* params, int n,
                              const double* x, const double* grad_base, const double* e_base, float* el_out,
                              float* j_out, float* q_out, float* pair_out, void* stream)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  std::string why;
  if (!nj_spec_ok(s, sp, why)) return fail(s, LRDMC_ERR_ARG, "nj_forward: " + why);
  if (n < 0 || (n > 0 && (!params || !x || !grad_base || !e_base || !el_out || !j_out || !q_out || !pair_out)))
    return fail(s, LRDMC_ERR_ARG, "nj_forward: bad arguments");
  cudaError_t e = launch_nj_forward(nj_geom(s, sp), nj_net(sp), params, n, x, grad_base, e_base, el_out, j_out,
                                    q_out, pair_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "nj_forward");
  return LRDMC_OK;
}

lrdmc_status lrdmc_nj_backward(lrdmc_system_t s, const lrdmc_nj_spec* sp, const float* params, int n,
                               const double* x, const float* q, const float* d_el, const float* d_j,
                               float* grad_out, void* stream)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  std::string why;
  if (!nj_spec_ok(s, sp, why)) return fail(s, LRDMC_ERR_ARG, "nj_backward: " + why);
  if (n < 0 || !grad_out || (n > 0 && (!params || !x || !q || !d_el || !d_j)))
    return fail(s, LRDMC_ERR_ARG, "nj_backward: bad arguments");
  const NjGeom G = nj_geom(s, sp);
  const NjNetDev N = nj_net(sp);
  const int max_blocks = nj_backward_max_blocks(G, N);
  if (max_blocks <= 0) return cuda_fail(s, cudaGetLastError(), "nj_backward: grid size");
  const size_t need = (size_t)max_blocks * (size_t)nj_n_params(N.F, N.C, LRDMC_NJ_HIDDEN);
  if (need > s->nj_partials_n) {
    if (s->nj_partials) cudaFree(s->nj_partials);  // synchronises: no earlier call still reads it
    s->nj_partials = nullptr;
    s->nj_partials_n = 0;
    cudaError_t ea = cudaMalloc((void**)&s->nj_partials, sizeof(float) * need);
    if (ea != cudaSuccess) return cuda_fail(s, ea, "nj_backward: scratch");
    s->nj_partials_n = need;
  }
  cudaError_t e = launch_nj_backward(G, N, params, n, x, q, d_el, d_j, grad_out, s->nj_partials, max_blocks,
                                     (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "nj_backward");
  return LRDMC_OK;
}

// ---------------------------------------------------------------------------
// Persistent grid size and batches of systems.
// ---------------------------------------------------------------------------
lrdmc_status lrdmc_set_interval_blocks(lrdmc_system_t s, int blocks)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (blocks < 0) return fail(s, LRDMC_ERR_ARG, "set_interval_blocks: blocks < 0");
  s->blocks = blocks;
  s->version++;
  return LRDMC_OK;
}

lrdmc_status lrdmc_interval_blocks(lrdmc_system_t s, int* current, int* occupancy_default)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (current) *current = s->blocks;
  if (occupancy_default) *occupancy_default = interval_default_blocks(s->S, s->Lo, s->W > 0 ? s->W : 1 << 30);
  return LRDMC_OK;
}

lrdmc_status lrdmc_set_tail_helpers(lrdmc_system_t s, int on)
{
  if (!s) return fail(s, LRDMC_ERR_ARG, "");
  if (on != 0 && on != 1) return fail(s, LRDMC_ERR_ARG, "set_tail_helpers: on must be 0 or 1");
  s->helpers = on;
  s->P.helpers = on;
  s->version++;
  return LRDMC_OK;
}

}  // extern "C"

struct lrdmc_batch_s {
  std::vector<lrdmc_system_t> sys;
  std::vector<LatDev> lat;
  std::vector<int> group;  // systems of one group run concurrently; groups run in order
  uint64_t group_version = 0;
  int carveout = -1;       // shared-memory carveout of the batched interval launches (-1: default)
  int pipelined = 0;       // 1: interval kernels chained on one stream with programmatic serialization
  std::vector<cudaStream_t> branch;  // one per system, owned
  std::vector<cudaEvent_t> join, ready;
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  struct Graph {
    uint64_t parity;
    std::vector<uint64_t> versions;
    uint64_t group_version;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  std::string last_error;
};

static lrdmc_status bfail(lrdmc_batch_t b, lrdmc_status st, const std::string& msg)
{
  if (b) b->last_error = msg;
  return st;
}

static lrdmc_status bcuda(lrdmc_batch_t b, cudaError_t e, const char* where)
{
  return bfail(b, LRDMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static void batch_release(lrdmc_batch_t b)
{
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  for (cudaStream_t st : b->branch) if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->join) if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : b->ready) if (ev) cudaEventDestroy(ev);
  if (b->main) cudaStreamDestroy(b->main);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
}

// One step of every system as one graph. The groups run in increasing
// group number; within a group, a fork on the batch stream, per system on
// its own branch stream the interval kernel, the reconfiguration kernel and
// the copy of its error word, then a join.
static cudaError_t capture_step(lrdmc_batch_t b, cudaGraphExec_t* out)
{
  cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaError_t first = cudaSuccess;
  if (b->pipelined) {
    // every system's interval kernel on the batch stream in group order (then
    // index order), each after the first launched with programmatic stream
    // serialization: it starts on the SMs that the previous system's blocks
    // free as they run out of walkers. Each kernel finishes only after its
    // predecessor (griddepcontrol.wait at its end), so the reconfiguration
    // kernels, launched normally after the chain, see every interval done.
    std::vector<size_t> seq(b->sys.size());
    for (size_t i = 0; i < seq.size(); ++i) seq[i] = i;
    std::stable_sort(seq.begin(), seq.end(), [&](size_t x, size_t y) { return b->group[x] < b->group[y]; });
    for (size_t q = 0; q < seq.size() && first == cudaSuccess; ++q) {
      lrdmc_system_t s = b->sys[seq[q]];
      PopDev P = s->P;
      P.rec_src = s->rec[s->cur];
      P.rec_dst = s->rec[1 - s->cur];
      first = launch_interval(s->S, s->Lo, b->lat[seq[q]], P, s->blocks, b->main, b->carveout, q > 0);
    }
    for (size_t q = 0; q < seq.size() && first == cudaSuccess; ++q) {
      lrdmc_system_t s = b->sys[seq[q]];
      PopDev P = s->P;
      P.rec_src = s->rec[s->cur];
      P.rec_dst = s->rec[1 - s->cur];
      first = launch_reconfig(P, s->Lo, b->main);
      if (first == cudaSuccess)
        first = cudaMemcpyAsync(s->err_host, s->P.err, sizeof(int), cudaMemcpyDeviceToHost, b->main);
    }
  }
  std::vector<int> order(b->group);
  std::sort(order.begin(), order.end());
  order.erase(std::unique(order.begin(), order.end()), order.end());
  if (b->pipelined) order.clear();
  for (int grp : order) {
    if (first == cudaSuccess) first = cudaEventRecord(b->fork, b->main);
    for (size_t i = 0; i < b->sys.size() && first == cudaSuccess; ++i) {
      if (b->group[i] != grp) continue;
      lrdmc_system_t s = b->sys[i];
      PopDev P = s->P;
      P.rec_src = s->rec[s->cur];
      P.rec_dst = s->rec[1 - s->cur];
      first = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
      if (first == cudaSuccess)
        first = launch_interval(s->S, s->Lo, b->lat[i], P, s->blocks, b->branch[i], b->carveout);
      if (first == cudaSuccess) first = launch_reconfig(P, s->Lo, b->branch[i]);
      if (first == cudaSuccess)
        first = cudaMemcpyAsync(s->err_host, s->P.err, sizeof(int), cudaMemcpyDeviceToHost, b->branch[i]);
      if (first == cudaSuccess) first = cudaEventRecord(b->join[i], b->branch[i]);
      if (first == cudaSuccess) first = cudaStreamWaitEvent(b->main, b->join[i], 0);
    }
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->main, &g);
  if (first != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return first;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

extern "C" {

lrdmc_status lrdmc_batch_create(lrdmc_system_t* systems, int n, const double* a, const lrdmc_spacing_fn* spacing,
                                lrdmc_batch_t* out)
{
  if (!out) return LRDMC_ERR_ARG;
  *out = nullptr;
  if (!systems || !a || !spacing || n < 1 || n > 64) return LRDMC_ERR_ARG;
  lrdmc_batch_t b = new lrdmc_batch_s();
  for (int i = 0; i < n; ++i) {
    lrdmc_system_t s = systems[i];
    if (!s || !s->have_pop) {
      delete b;
      return LRDMC_ERR_STATE;
    }
    for (int j = 0; j < i; ++j)
      if (systems[j] == s) {
        delete b;
        return LRDMC_ERR_ARG;
      }
    LatDev L;
    if (lattice_from(s, a[i], &spacing[i], L) != LRDMC_OK) {
      delete b;
      return LRDMC_ERR_ARG;
    }
    b->sys.push_back(s);
    b->lat.push_back(L);
    b->group.push_back(0);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  b->branch.assign(n, nullptr);
  b->join.assign(n, nullptr);
  b->ready.assign(n, nullptr);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    batch_release(b);
    delete b;
    return LRDMC_ERR_CUDA;
  }
  *out = b;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_step(lrdmc_batch_t b, int n_steps)
{
  NvtxRange nvtx("lrdmc_batch_step");
  if (!b) return LRDMC_ERR_ARG;
  if (n_steps < 0) return bfail(b, LRDMC_ERR_ARG, "batch_step: n_steps < 0");
  const size_t n = b->sys.size();
  for (size_t i = 0; i < n; ++i) {
    lrdmc_system_t s = b->sys[i];
    if (!s->have_pop) return bfail(b, LRDMC_ERR_STATE, "batch_step: a system has no population");
    if (s->k + (uint64_t)n_steps > (uint64_t)s->trace_cap)
      return bfail(b, LRDMC_ERR_ARG, "batch_step: the trace of system " + std::to_string(i) + " would overflow");
  }
  if (n_steps == 0) return LRDMC_OK;
  // the first evaluation of a population (or after a lattice change) on the
  // system's own stream, then the batch stream waits for every system
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    lrdmc_system_t s = b->sys[i];
    if (!s->have_eval || !same_lattice(b->lat[i], s->eval_lat)) {
      PopDev P = s->P;
      P.rec_src = s->rec[s->cur];
      P.rec_dst = s->rec[1 - s->cur];
      e = launch_eval_all(s->S, s->Lo, b->lat[i], P, s->stream);
      if (e != cudaSuccess) break;
      s->have_eval = true;
      s->eval_lat = b->lat[i];
      s->eval_prec = s->S.precision;
    }
    e = cudaEventRecord(b->ready[i], s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->ready[i], 0);
  }
  if (e != cudaSuccess) return bcuda(b, e, "batch_step: preparation");
  for (int step = 0; step < n_steps; ++step) {
    uint64_t parity = 0;
    for (size_t i = 0; i < n; ++i) parity |= (uint64_t)b->sys[i]->cur << i;
    cudaGraphExec_t exec = nullptr;
    for (auto& g : b->graphs) {
      if (g.parity != parity || g.group_version != b->group_version) continue;
      bool same = true;
      for (size_t i = 0; i < n; ++i) same = same && g.versions[i] == b->sys[i]->version;
      if (same) { exec = g.exec; break; }
    }
    if (!exec) {
      // drop graphs of stale kernel arguments, then capture this parity
      std::vector<lrdmc_batch_s::Graph> keep;
      for (auto& g : b->graphs) {
        bool same = g.group_version == b->group_version;
        for (size_t i = 0; i < n; ++i) same = same && g.versions[i] == b->sys[i]->version;
        if (same) keep.push_back(g); else cudaGraphExecDestroy(g.exec);
      }
      b->graphs = keep;
      e = capture_step(b, &exec);
      if (e != cudaSuccess) return bcuda(b, e, "batch_step: graph capture");
      lrdmc_batch_s::Graph g;
      g.parity = parity;
      g.group_version = b->group_version;
      g.exec = exec;
      for (size_t i = 0; i < n; ++i) g.versions.push_back(b->sys[i]->version);
      b->graphs.push_back(g);
    }
    e = cudaGraphLaunch(exec, b->main);
    if (e != cudaSuccess) return bcuda(b, e, "batch_step: graph launch");
    for (size_t i = 0; i < n; ++i) {
      lrdmc_system_t s = b->sys[i];
      s->cur = 1 - s->cur;
      s->k++;
      s->pending = true;
    }
  }
  // later work on each system's own stream follows the batch
  e = cudaEventRecord(b->done, b->main);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->sys[i]->stream, b->done, 0);
  if (e != cudaSuccess) return bcuda(b, e, "batch_step: join");
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_sync(lrdmc_batch_t b)
{
  if (!b) return LRDMC_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(b->main);
  if (e != cudaSuccess) return bcuda(b, e, "batch_sync");
  for (size_t i = 0; i < b->sys.size(); ++i) {
    lrdmc_status st = sync_system(b->sys[i]);
    if (st != LRDMC_OK) return bfail(b, st, "system " + std::to_string(i) + ": " + b->sys[i]->last_error);
  }
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_set_groups(lrdmc_batch_t b, const int* group)
{
  if (!b) return LRDMC_ERR_ARG;
  if (!group) return bfail(b, LRDMC_ERR_ARG, "batch_set_groups: NULL");
  for (size_t i = 0; i < b->sys.size(); ++i)
    if (group[i] < 0) return bfail(b, LRDMC_ERR_ARG, "batch_set_groups: negative group");
  for (size_t i = 0; i < b->sys.size(); ++i) b->group[i] = group[i];
  b->group_version++;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_set_carveout(lrdmc_batch_t b, int carveout)
{
  if (!b) return LRDMC_ERR_ARG;
  if (carveout < -1 || carveout > 100) return bfail(b, LRDMC_ERR_ARG, "batch_set_carveout: -1 or 0..100");
  b->carveout = carveout;
  b->group_version++;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_set_pipelined(lrdmc_batch_t b, int on)
{
  if (!b) return LRDMC_ERR_ARG;
  if (on != 0 && on != 1) return bfail(b, LRDMC_ERR_ARG, "batch_set_pipelined: on must be 0 or 1");
  b->pipelined = on;
  b->group_version++;
  return LRDMC_OK;
}

lrdmc_status lrdmc_batch_stream(lrdmc_batch_t b, void** stream)
{
  if (!b || !stream) return LRDMC_ERR_ARG;
  *stream = (void*)b->main;
  return LRDMC_OK;
}

const char* lrdmc_batch_last_error(lrdmc_batch_t b) { return b ? b->last_error.c_str() : g_static_error; }

void lrdmc_batch_destroy(lrdmc_batch_t b)
{
  if (!b) return;
  cudaStreamSynchronize(b->main);
  batch_release(b);
  delete b;
}

const char* lrdmc_last_error(lrdmc_system_t s) { return s ? s->last_error.c_str() : g_static_error; }

int lrdmc_build_flags(void) { return kBuildFlags; }

void lrdmc_destroy(lrdmc_system_t s)
{
  if (!s) return;
  if (s->err_host) cudaFreeHost(s->err_host);
  if (s->eval_err) cudaFree(s->eval_err);
  if (s->nj_tab) cudaFree(s->nj_tab);
  if (s->nj_tab_df) cudaFree(s->nj_tab_df);
  if (s->base_err) cudaFree(s->base_err);
  if (s->nj_partials) cudaFree(s->nj_partials);
  for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
  delete s;
}

}  // extern "C"
