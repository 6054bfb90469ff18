/*
 * Plain FP64 CPU oracle for LRDMC with the single and the double ("smart")
 * lattice of Nakano, Maezono and Sorella, arXiv:1909.01589.
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's shared library. The
 * product library does not include, link or call anything here, and nothing
 * here comes from the product.
 *
 * The oracle is written for reading, not for speed. Every function follows
 * one passage of the paper or of the method it cites (lattice regularization
 * of Casula, Filippi and Sorella, PRL 95, 100201 (2005), "2005CAS" below):
 *   - double-grid parameters: Eq. 2, 3, 4, 5, 6, 7 and S-13;
 *   - the double-grid lattice Laplacian: Eq. 1;
 *   - the fixed-node lattice Hamiltonian, its off-diagonal elements and the
 *     sign-flip term, continuous-time projection and walker reconfiguration:
 *     the cited LRDMC method (2005CAS and the Becca-Sorella text).
 * Where the paper is silent the choices are documented at the function.
 * Determinant ratios go the plain route (orbitals first, then the dot with
 * a column of the inverse Slater matrix); no factorisation tricks.
 */
#include "lrdmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* =========================================================================
 * 1. Double-grid parameters.
 * ========================================================================= */

/* S-13: r_c(a, Z) = beta * (kappa alpha^-2 + 1) / (alpha^-2 + 1) * Z^(-5/7),
 * with alpha = 1/(a Z) (so alpha^-2 = (a Z)^2). The Z^(-5/7) law is Eq. 10
 * and the text after it; beta = 0.75 and kappa = 2.5 in the paper. */
double orc_rc_this_work(double a, double Z, double beta, double kappa)
{
  double inv_alpha2 = (a * Z) * (a * Z);
  return beta * (kappa * inv_alpha2 + 1.0) / (inv_alpha2 + 1.0) * pow(Z, -5.0 / 7.0);
}

/* Slater's rules (Slater 1930, cited for the effective model of Eq. 7):
 * the electrons of a neutral atom fill subshells in Madelung order and are
 * grouped as [1s][2s2p][3s3p][3d][4s4p][4d][4f][5s5p][5d][5f][6s6p]...
 * For an electron of an (ns,np) group the other electrons of its group
 * screen 0.35 each (0.30 within 1s), electrons of principal shell n-1 screen
 * 0.85 each, and deeper shells 1.00 each. For an (nd) or (nf) group the
 * other electrons of its group screen 0.35 and every group to its left
 * screens 1.00. zeta = (Z - s) / n*, with n* = 1, 2, 3, 3.7, 4.0, 4.2.
 * Returns the number of occupied groups. */
int orc_slater_groups(int Z, int* n_out, int* type_out, double* neff_out,
                      double* zeta_out, int* occ_out, int max_groups)
{
  /* Madelung filling order as (n, l) */
  static const int fill_n[] = {1, 2, 2, 3, 3, 4, 3, 4, 5, 4, 5, 6, 4, 5, 6, 7, 5, 6, 7};
  static const int fill_l[] = {0, 0, 1, 0, 1, 0, 2, 1, 0, 2, 1, 0, 3, 2, 1, 0, 3, 2, 1};
  /* Slater group order: (n, type) with type 0 = s/p, 2 = d, 3 = f */
  static const int grp_n[] = {1, 2, 3, 3, 4, 4, 4, 5, 5, 5, 6, 6, 7};
  static const int grp_t[] = {0, 0, 0, 2, 0, 2, 3, 0, 2, 3, 0, 2, 0};
  static const double nstar[] = {0.0, 1.0, 2.0, 3.0, 3.7, 4.0, 4.2, 4.2};
  const int n_groups_all = (int)(sizeof(grp_n) / sizeof(grp_n[0]));
  int occ[16] = {0};
  int left = Z;
  for (int f = 0; f < (int)(sizeof(fill_n) / sizeof(fill_n[0])) && left > 0; ++f) {
    int cap = 2 * (2 * fill_l[f] + 1);
    int put = left < cap ? left : cap;
    int type = fill_l[f] <= 1 ? 0 : fill_l[f];
    for (int g = 0; g < n_groups_all; ++g)
      if (grp_n[g] == fill_n[f] && grp_t[g] == type) occ[g] += put;
    left -= put;
  }
  int out = 0;
  for (int g = 0; g < n_groups_all; ++g) {
    if (occ[g] == 0) continue;
    double s = 0.0;
    for (int h = 0; h < n_groups_all; ++h) {
      if (occ[h] == 0) continue;
      int others = (h == g) ? occ[h] - 1 : occ[h];
      if (h == g) {
        s += others * ((grp_n[g] == 1) ? 0.30 : 0.35);
      } else if (grp_t[g] == 0) {
        if (grp_n[h] == grp_n[g] - 1) s += others * 0.85;
        else if (grp_n[h] < grp_n[g] - 1) s += others * 1.00;
      } else {
        if (h < g) s += others * 1.00;
      }
    }
    if (out < max_groups) {
      n_out[out] = grp_n[g];
      type_out[out] = grp_t[g];
      neff_out[out] = nstar[grp_n[g]];
      zeta_out[out] = ((double)Z - s) / nstar[grp_n[g]];
      occ_out[out] = occ[g];
    }
    ++out;
  }
  return out;
}

/* Eq. 7: N_core(r_c) = int_0^inf dr 4 pi r^2 rho_eff(r) exp(-r^2 / (2 r_c^2)),
 * with rho_eff the density of Slater's effective model: each group holds occ
 * electrons in the normalised radial function
 * R(r) = N r^(n*-1) exp(-zeta r), N^2 = (2 zeta)^(2 n* + 1) / Gamma(2 n* + 1).
 * Plain composite Simpson rule on [0, r_max], r_max = 80 / zeta_min. */
double orc_ncore(int Z, double rc)
{
  int n[16], type[16], occ[16];
  double neff[16], zeta[16];
  int ng = orc_slater_groups(Z, n, type, neff, zeta, occ, 16);
  double zmin = 1e300;
  for (int g = 0; g < ng; ++g) if (zeta[g] < zmin) zmin = zeta[g];
  const double rmax = 80.0 / zmin;
  const int M = 400000; /* even number of intervals */
  const double h = rmax / M;
  double sum = 0.0;
  for (int j = 0; j <= M; ++j) {
    double r = j * h;
    double f = 0.0;
    for (int g = 0; g < ng; ++g) {
      double norm2 = pow(2.0 * zeta[g], 2.0 * neff[g] + 1.0) / tgamma(2.0 * neff[g] + 1.0);
      f += occ[g] * norm2 * pow(r, 2.0 * neff[g]) * exp(-2.0 * zeta[g] * r);
    }
    if (rc > 0.0 && isfinite(rc)) f *= exp(-r * r / (2.0 * rc * rc));
    double wgt = (j == 0 || j == M) ? 1.0 : ((j % 2) ? 4.0 : 2.0);
    sum += wgt * f;
  }
  return sum * h / 3.0;
}

/* Eq. 6 with r_c from S-13: a'/a = sqrt((Z - N_core) / N_core). */
double orc_aprime_over_a_this_work(int Z, double a, double beta, double kappa)
{
  double rc = orc_rc_this_work(a, (double)Z, beta, kappa);
  double nc = orc_ncore(Z, rc);
  return sqrt(((double)Z - nc) / nc);
}

/* Eq. 4 (the earlier choice, used with the Pade p of Eq. 2 and r_c = Z/2):
 * a'/a = sqrt(Z^2/4 + 1). */
double orc_aprime_over_a_previous(double Z) { return sqrt(Z * Z / 4.0 + 1.0); }

/* Eq. 5: 1/speedup = N_core/Z + (N_valence/Z) (a'/a)^-2, N_valence = Z - N_core. */
double orc_speedup(double Z, double n_core, double aprime_over_a)
{
  double inv = n_core / Z + (Z - n_core) / Z / (aprime_over_a * aprime_over_a);
  return 1.0 / inv;
}

/* =========================================================================
 * 2. Counter-based random numbers and the lattice rotation.
 * ========================================================================= */

/* Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11): ten rounds of
 * (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
 * c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), with the key advanced by
 * the Weyl constants between rounds. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    unsigned __int128 p0 = (unsigned __int128)M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A double strictly inside (0, 1): the top 52 bits plus one half, times
 * 2^-52. Every value (j + 1/2) 2^-52 is exact, the largest is 1 - 2^-53. */
double orc_uniform(uint64_t bits) { return ((double)(bits >> 12) + 0.5) * 0x1.0p-52; }

/* Uniformly random rotation from three uniforms: the unit quaternion
 * q = (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2,
 *      sqrt(u1) sin 2 pi u3,   sqrt(u1) cos 2 pi u3) = (x, y, z, w)
 * (Shoemake, Graphics Gems III, 1992), turned into the rotation matrix. */
void orc_rotation(double u1, double u2, double u3, double R[9])
{
  double s1 = sqrt(1.0 - u1), s2 = sqrt(u1);
  double x = s1 * sin(2.0 * M_PI * u2), y = s1 * cos(2.0 * M_PI * u2);
  double z = s2 * sin(2.0 * M_PI * u3), w = s2 * cos(2.0 * M_PI * u3);
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - z * w);       R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);       R[7] = 2.0 * (y * z + x * w);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* =========================================================================
 * 3. The trial function psi_G(x) = det_up * det_dn * exp(J(x)).
 * ========================================================================= */

struct orc_system {
  int n_nuc;
  double R[ORC_MAX_NUC][3];
  double Z[ORC_MAX_NUC];
  int n_up, n_dn, N;
  int n_shell;
  int* sh_center; int* sh_l; int* sh_kind; int* sh_nprim;
  double* sh_neff; double* sh_zeta; double* prim_alpha; double* prim_coef;
  int n_ao, n_mo;
  double* C; /* [n_ao][n_mo] */
  double b_ee, c_par, c_anti, en_b2;
  double en_b1[ORC_MAX_NUC];
  int ee_on;
  /* optional neural pair term (section 3b) */
  int nj_ch, nj_cells;
  double nj_rcut[ORC_NJ_MAX_CH];
  int nj_species[ORC_MAX_NUC];
  double* nj_nodes; /* [ch][cells + 1][3]: g, g', g'' at the nodes, or NULL */
};

orc_system* orc_system_create(int n_nuc, const double* nuc_xyz, const double* Z,
                              int n_up, int n_dn,
                              int n_shell, const int* sh_center, const int* sh_l,
                              const int* sh_kind, const int* sh_nprim,
                              const double* sh_neff, const double* sh_zeta,
                              const double* prim_alpha, const double* prim_coef,
                              int n_ao, int n_mo, const double* C,
                              double b_ee, double c_par, double c_anti,
                              const double* en_b1, double en_b2, int ee_on)
{
  if (n_nuc < 1 || n_nuc > ORC_MAX_NUC || n_up < n_dn || n_dn < 0 || n_up < 1) return NULL;
  if (n_mo < n_up) return NULL;
  orc_system* s = (orc_system*)calloc(1, sizeof(orc_system));
  s->n_nuc = n_nuc;
  for (int I = 0; I < n_nuc; ++I) {
    for (int d = 0; d < 3; ++d) s->R[I][d] = nuc_xyz[3 * I + d];
    s->Z[I] = Z[I];
    s->en_b1[I] = en_b1 ? en_b1[I] : 0.0;
  }
  s->n_up = n_up; s->n_dn = n_dn; s->N = n_up + n_dn;
  s->n_shell = n_shell;
  s->sh_center = (int*)malloc(sizeof(int) * n_shell);
  s->sh_l = (int*)malloc(sizeof(int) * n_shell);
  s->sh_kind = (int*)malloc(sizeof(int) * n_shell);
  s->sh_nprim = (int*)malloc(sizeof(int) * n_shell);
  s->sh_neff = (double*)malloc(sizeof(double) * n_shell);
  s->sh_zeta = (double*)malloc(sizeof(double) * n_shell);
  s->prim_alpha = (double*)malloc(sizeof(double) * n_shell * ORC_MAX_PRIM);
  s->prim_coef = (double*)malloc(sizeof(double) * n_shell * ORC_MAX_PRIM);
  int count = 0;
  for (int q = 0; q < n_shell; ++q) {
    s->sh_center[q] = sh_center[q]; s->sh_l[q] = sh_l[q]; s->sh_kind[q] = sh_kind[q];
    s->sh_nprim[q] = sh_nprim[q]; s->sh_neff[q] = sh_neff[q]; s->sh_zeta[q] = sh_zeta[q];
    for (int p = 0; p < ORC_MAX_PRIM; ++p) {
      s->prim_alpha[q * ORC_MAX_PRIM + p] = prim_alpha[q * ORC_MAX_PRIM + p];
      s->prim_coef[q * ORC_MAX_PRIM + p] = prim_coef[q * ORC_MAX_PRIM + p];
    }
    count += 2 * sh_l[q] + 1;
  }
  if (count != n_ao) { orc_system_destroy(s); return NULL; }
  s->n_ao = n_ao; s->n_mo = n_mo;
  s->C = (double*)malloc(sizeof(double) * n_ao * n_mo);
  memcpy(s->C, C, sizeof(double) * n_ao * n_mo);
  s->b_ee = b_ee; s->c_par = c_par; s->c_anti = c_anti; s->en_b2 = en_b2; s->ee_on = ee_on;
  return s;
}

void orc_system_destroy(orc_system* s)
{
  if (!s) return;
  free(s->nj_nodes);
  free(s->sh_center); free(s->sh_l); free(s->sh_kind); free(s->sh_nprim);
  free(s->sh_neff); free(s->sh_zeta); free(s->prim_alpha); free(s->prim_coef);
  free(s->C); free(s);
}

int orc_n_ao(const orc_system* s) { return s->n_ao; }

/* Atomic orbitals chi_mu(r) = S(d) R(|d|), d = r - R_center, with S a real
 * solid harmonic of degree l (l = 0: 1; l = 1: x, y, z; l = 2: xy, yz, zx,
 * x^2 - y^2, 2z^2 - x^2 - y^2) and R either a Slater radial part
 * r^(n-1-l) exp(-zeta r) or a contraction sum_p c_p exp(-alpha_p r^2).
 * Derivatives use x.grad S = l S and lap S = 0:
 *   grad chi = R grad S + S (R'/r) d,   lap chi = S (R'' + 2 (l+1) R'/r). */
void orc_ao_values(const orc_system* s, const double r[3], double* chi, double* grad, double* lap)
{
  int mu = 0;
  for (int q = 0; q < s->n_shell; ++q) {
    const int l = s->sh_l[q];
    const double* c = s->R[s->sh_center[q]];
    double d[3] = {r[0] - c[0], r[1] - c[1], r[2] - c[2]};
    double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Rv, R1, R2; /* R, R'/r, R'' */
    if (s->sh_kind[q] == 0) {
      double m = s->sh_neff[q] - 1.0 - l;
      double zeta = s->sh_zeta[q];
      Rv = pow(rr, m) * exp(-zeta * rr);
      R1 = (m / rr - zeta) * Rv / rr;
      R2 = ((m / rr - zeta) * (m / rr - zeta) - m / (rr * rr)) * Rv;
    } else {
      Rv = 0.0; R1 = 0.0; R2 = 0.0;
      for (int p = 0; p < s->sh_nprim[q]; ++p) {
        double al = s->prim_alpha[q * ORC_MAX_PRIM + p];
        double e = s->prim_coef[q * ORC_MAX_PRIM + p] * exp(-al * rr * rr);
        Rv += e;
        R1 += -2.0 * al * e;
        R2 += (4.0 * al * al * rr * rr - 2.0 * al) * e;
      }
    }
    double S[5], gS[5][3];
    int nf = 2 * l + 1;
    memset(gS, 0, sizeof(gS));
    if (l == 0) {
      S[0] = 1.0;
    } else if (l == 1) {
      for (int k = 0; k < 3; ++k) { S[k] = d[k]; gS[k][k] = 1.0; }
    } else {
      S[0] = d[0] * d[1]; gS[0][0] = d[1]; gS[0][1] = d[0];
      S[1] = d[1] * d[2]; gS[1][1] = d[2]; gS[1][2] = d[1];
      S[2] = d[2] * d[0]; gS[2][2] = d[0]; gS[2][0] = d[2];
      S[3] = d[0] * d[0] - d[1] * d[1]; gS[3][0] = 2.0 * d[0]; gS[3][1] = -2.0 * d[1];
      S[4] = 2.0 * d[2] * d[2] - d[0] * d[0] - d[1] * d[1];
      gS[4][0] = -2.0 * d[0]; gS[4][1] = -2.0 * d[1]; gS[4][2] = 4.0 * d[2];
    }
    for (int f = 0; f < nf; ++f, ++mu) {
      chi[mu] = S[f] * Rv;
      if (grad)
        for (int k = 0; k < 3; ++k) grad[3 * mu + k] = Rv * gS[f][k] + S[f] * R1 * d[k];
      if (lap) lap[mu] = S[f] * (R2 + 2.0 * (l + 1) * R1);
    }
  }
}

/* phi_m(r) = sum_mu C[mu][m] chi_mu(r) for m < n_orb. */
static void orbitals(const orc_system* s, const double* chi, int n_orb, double* phi)
{
  for (int m = 0; m < n_orb; ++m) {
    double v = 0.0;
    for (int mu = 0; mu < s->n_ao; ++mu) v += s->C[mu * s->n_mo + m] * chi[mu];
    phi[m] = v;
  }
}

static int spin_of(const orc_system* s, int i) { return i < s->n_up ? 0 : 1; }
static int local_index(const orc_system* s, int i) { return i < s->n_up ? i : i - s->n_up; }
static int spin_count(const orc_system* s, int spin) { return spin == 0 ? s->n_up : s->n_dn; }

/* Slater matrix of one spin block: A[l][m] = phi_m(r_l). */
static void slater_matrix(const orc_system* s, const double* x, int spin, double* A)
{
  int n = spin_count(s, spin), off = spin == 0 ? 0 : s->n_up;
  double* chi = (double*)malloc(sizeof(double) * s->n_ao);
  for (int l = 0; l < n; ++l) {
    orc_ao_values(s, &x[3 * (off + l)], chi, NULL, NULL);
    orbitals(s, chi, n, &A[l * n]);
  }
  free(chi);
}

/* Gaussian elimination with partial pivoting: returns 0 on success, the
 * inverse in Ainv (may be NULL), log|det| and the sign of det. */
static int lu_inverse(int n, const double* A_in, double* Ainv, double* log_abs, double* sign)
{
  double* A = (double*)malloc(sizeof(double) * n * n);
  double* X = (double*)malloc(sizeof(double) * n * n);
  memcpy(A, A_in, sizeof(double) * n * n);
  for (int i = 0; i < n * n; ++i) X[i] = 0.0;
  for (int i = 0; i < n; ++i) X[i * n + i] = 1.0;
  double la = 0.0, sg = 1.0;
  int rc = 0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
    if (A[piv * n + col] == 0.0) { rc = 1; break; }
    if (piv != col) {
      for (int k = 0; k < n; ++k) {
        double t = A[col * n + k]; A[col * n + k] = A[piv * n + k]; A[piv * n + k] = t;
        t = X[col * n + k]; X[col * n + k] = X[piv * n + k]; X[piv * n + k] = t;
      }
      sg = -sg;
    }
    double p = A[col * n + col];
    la += log(fabs(p));
    if (p < 0) sg = -sg;
    for (int r = col + 1; r < n; ++r) {
      double f = A[r * n + col] / p;
      for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
      for (int k = 0; k < n; ++k) X[r * n + k] -= f * X[col * n + k];
    }
  }
  if (rc == 0 && Ainv) {
    /* back substitution: U Y = X */
    for (int col = n - 1; col >= 0; --col) {
      for (int k = 0; k < n; ++k) {
        double v = X[col * n + k];
        for (int j = col + 1; j < n; ++j) v -= A[col * n + j] * Ainv[j * n + k];
        Ainv[col * n + k] = v / A[col * n + col];
      }
    }
  }
  if (log_abs) *log_abs = la;
  if (sign) *sign = sg;
  free(A); free(X);
  return rc;
}

/* =========================================================================
 * 3b. Optional neural pair term of the Jastrow factor.
 *
 * J_NN(x) = sum_{i<j} g_{c(i,j)}(r_ij) + sum_{i,I} g_{2+species(I)}(r_iI),
 * channel 0 for equal-spin electron pairs, 1 for opposite spins, 2+s for the
 * electron-nucleus pairs of nucleus species s. Each g_c is the quintic
 * Hermite interpolant of a radial network on the nodes
 * r_k = r_cut (k/n)^2, k = 0..n: in cell k, with t = (r - r_k)/w_k and
 * w_k = r_{k+1} - r_k, it is the degree-5 polynomial that takes the node
 * values g, w g', w^2 g'' at t = 0 and t = 1 (so g is twice continuously
 * differentiable); g = 0 for r >= r_cut. The node data come from the
 * network (oracle/neural.py); this file only interpolates.
 * ========================================================================= */
int orc_system_set_neural(orc_system* s, int n_ch, int n_cells, const double* r_cut,
                          const int* species, const double* nodes)
{
  free(s->nj_nodes);
  s->nj_nodes = NULL;
  s->nj_ch = 0;
  if (n_ch == 0) return 0;
  if (n_ch < 2 || n_ch > ORC_NJ_MAX_CH || n_cells < 1) return 1;
  for (int I = 0; I < s->n_nuc; ++I)
    if (species[I] < 0 || 2 + species[I] >= n_ch) return 1;
  for (int c = 0; c < n_ch; ++c)
    if (!(r_cut[c] > 0.0)) return 1;
  s->nj_ch = n_ch;
  s->nj_cells = n_cells;
  for (int c = 0; c < n_ch; ++c) s->nj_rcut[c] = r_cut[c];
  for (int I = 0; I < s->n_nuc; ++I) s->nj_species[I] = species[I];
  size_t len = (size_t)n_ch * (n_cells + 1) * 3;
  s->nj_nodes = (double*)malloc(sizeof(double) * len);
  memcpy(s->nj_nodes, nodes, sizeof(double) * len);
  return 0;
}

/* g_c(r), g_c'(r), g_c''(r) by the quintic Hermite basis on [0, 1]:
 *   H0 = 1 - 10t^3 + 15t^4 - 6t^5   (value at 0)
 *   H1 = t - 6t^3 + 8t^4 - 3t^5     (first derivative at 0)
 *   H2 = (t^2 - 3t^3 + 3t^4 - t^5)/2 (second derivative at 0)
 *   H3 = 10t^3 - 15t^4 + 6t^5       (value at 1)
 *   H4 = -4t^3 + 7t^4 - 3t^5        (first derivative at 1)
 *   H5 = (t^3 - 2t^4 + t^5)/2       (second derivative at 1) */
void orc_neural_pair(const orc_system* s, int c, double r, double* g, double* g1, double* g2)
{
  *g = 0.0; *g1 = 0.0; *g2 = 0.0;
  if (!s->nj_nodes || c < 0 || c >= s->nj_ch) return;
  const double rc = s->nj_rcut[c];
  const int n = s->nj_cells;
  if (!(r < rc)) return;
  int k = (int)floor(sqrt(r / rc) * n);
  if (k < 0) k = 0;
  if (k > n - 1) k = n - 1;
  double r0 = rc * ((double)k / n) * ((double)k / n);
  double r1 = rc * ((double)(k + 1) / n) * ((double)(k + 1) / n);
  double w = r1 - r0, t = (r - r0) / w;
  const double* A = &s->nj_nodes[((size_t)c * (n + 1) + k) * 3];
  const double* B = A + 3;
  double f[6] = {A[0], w * A[1], w * w * A[2], B[0], w * B[1], w * w * B[2]};
  double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
  double H[6] = {1 - 10 * t3 + 15 * t4 - 6 * t5, t - 6 * t3 + 8 * t4 - 3 * t5,
                 0.5 * (t2 - 3 * t3 + 3 * t4 - t5), 10 * t3 - 15 * t4 + 6 * t5,
                 -4 * t3 + 7 * t4 - 3 * t5, 0.5 * (t3 - 2 * t4 + t5)};
  double D1[6] = {-30 * t2 + 60 * t3 - 30 * t4, 1 - 18 * t2 + 32 * t3 - 15 * t4,
                  0.5 * (2 * t - 9 * t2 + 12 * t3 - 5 * t4), 30 * t2 - 60 * t3 + 30 * t4,
                  -12 * t2 + 28 * t3 - 15 * t4, 0.5 * (3 * t2 - 8 * t3 + 5 * t4)};
  double D2[6] = {-60 * t + 180 * t2 - 120 * t3, -36 * t + 96 * t2 - 60 * t3,
                  0.5 * (2 - 18 * t + 36 * t2 - 20 * t3), 60 * t - 180 * t2 + 120 * t3,
                  -24 * t + 84 * t2 - 60 * t3, 0.5 * (6 * t - 24 * t2 + 20 * t3)};
  double v = 0.0, d1 = 0.0, d2 = 0.0;
  for (int q = 0; q < 6; ++q) { v += f[q] * H[q]; d1 += f[q] * D1[q]; d2 += f[q] * D2[q]; }
  *g = v;
  *g1 = d1 / w;
  *g2 = d2 / (w * w);
}

/* Pade pair functions of the Jastrow factor, u(r) = c r / (1 + b r), plus
 * the neural pair term when one is set. pair_ee / pair_en return u, du/dr
 * and d2u/dr2. */
static void pair_ee(const orc_system* s, int i, int j, double r, double* u, double* u1, double* u2)
{
  int same = spin_of(s, i) == spin_of(s, j);
  double c = same ? s->c_par : s->c_anti;
  double den = 1.0 + s->b_ee * r;
  *u = c * r / den;
  *u1 = c / (den * den);
  *u2 = -2.0 * s->b_ee * c / (den * den * den);
  if (s->nj_nodes) {
    double g, g1, g2;
    orc_neural_pair(s, same ? 0 : 1, r, &g, &g1, &g2);
    *u += g; *u1 += g1; *u2 += g2;
  }
}
static void pair_en(const orc_system* s, int I, double r, double* u, double* u1, double* u2)
{
  double den = 1.0 + s->en_b2 * r;
  *u = -s->en_b1[I] * r / den;
  *u1 = -s->en_b1[I] / (den * den);
  *u2 = 2.0 * s->en_b2 * s->en_b1[I] / (den * den * den);
  if (s->nj_nodes) {
    double g, g1, g2;
    orc_neural_pair(s, 2 + s->nj_species[I], r, &g, &g1, &g2);
    *u += g; *u1 += g1; *u2 += g2;
  }
}
static double u_ee(const orc_system* s, int i, int j, double r)
{
  double u, u1, u2;
  pair_ee(s, i, j, r, &u, &u1, &u2);
  return u;
}
static double u_en(const orc_system* s, int I, double r)
{
  double u, u1, u2;
  pair_en(s, I, r, &u, &u1, &u2);
  return u;
}
static double dist(const double* p, const double* q)
{
  double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

/* J(x) = sum_{i<j} u_ee(r_ij) + sum_i sum_I u_en(r_iI). */
static double jastrow(const orc_system* s, const double* x)
{
  double J = 0.0;
  for (int i = 0; i < s->N; ++i) {
    for (int j = i + 1; j < s->N; ++j) J += u_ee(s, i, j, dist(&x[3 * i], &x[3 * j]));
    for (int I = 0; I < s->n_nuc; ++I) J += u_en(s, I, dist(&x[3 * i], s->R[I]));
  }
  return J;
}

/* log|psi_G(x)| and its sign from the two determinants (by elimination) and
 * the Jastrow factor: the brute-force value of the trial function. */
int orc_log_psi(const orc_system* s, const double* x, double* log_abs, double* sign)
{
  double total = 0.0, sg = 1.0;
  for (int spin = 0; spin < 2; ++spin) {
    int n = spin_count(s, spin);
    if (n == 0) continue;
    double* A = (double*)malloc(sizeof(double) * n * n);
    slater_matrix(s, x, spin, A);
    double la, sgn;
    int rc = lu_inverse(n, A, NULL, &la, &sgn);
    free(A);
    if (rc) { *log_abs = -INFINITY; *sign = 0.0; return 1; }
    total += la; sg *= sgn;
  }
  *log_abs = total + jastrow(s, x);
  *sign = sg;
  return 0;
}

int orc_inverses(const orc_system* s, const double* x, double* Ainv_up, double* Ainv_dn)
{
  int rc = 0;
  for (int spin = 0; spin < 2; ++spin) {
    int n = spin_count(s, spin);
    if (n == 0) continue;
    double* A = (double*)malloc(sizeof(double) * n * n);
    slater_matrix(s, x, spin, A);
    rc |= lu_inverse(n, A, spin == 0 ? Ainv_up : Ainv_dn, NULL, NULL);
    free(A);
  }
  return rc;
}

/* Continuous-space kinetic and potential terms at x:
 *   lap psi_G / psi_G = sum_i [ lap_i D/D + 2 (grad_i D/D).(grad_i J)
 *                               + lap_i J + |grad_i J|^2 ],
 * with grad_i D/D = sum_m grad phi_m(r_i) Ainv[m][l_i] (same for lap), and
 * V = sum_{i<j} 1/r_ij - sum_{i,I} Z_I / r_iI + sum_{I<J} Z_I Z_J / R_IJ. */
static void laplacian_terms(const orc_system* s, const double* x, const double* Ainv_up,
                            const double* Ainv_dn, double* lap_over_psi, double* V_out,
                            double* grad_log_psi)
{
  const int nao = s->n_ao;
  double* chi = (double*)malloc(sizeof(double) * nao);
  double* g = (double*)malloc(sizeof(double) * nao * 3);
  double* lp = (double*)malloc(sizeof(double) * nao);
  double total = 0.0, V = 0.0;
  for (int i = 0; i < s->N; ++i) {
    int spin = spin_of(s, i), l = local_index(s, i), n = spin_count(s, spin);
    const double* Ainv = spin == 0 ? Ainv_up : Ainv_dn;
    orc_ao_values(s, &x[3 * i], chi, g, lp);
    /* orbital gradients and Laplacians, then the dot with column l of Ainv */
    double gD[3] = {0, 0, 0}, lD = 0.0;
    for (int m = 0; m < n; ++m) {
      double gphi[3] = {0, 0, 0}, lphi = 0.0;
      for (int mu = 0; mu < nao; ++mu) {
        double c = s->C[mu * s->n_mo + m];
        for (int k = 0; k < 3; ++k) gphi[k] += c * g[3 * mu + k];
        lphi += c * lp[mu];
      }
      double a = Ainv[m * n + l];
      for (int k = 0; k < 3; ++k) gD[k] += gphi[k] * a;
      lD += lphi * a;
    }
    /* Jastrow gradient and Laplacian for electron i */
    double gJ[3] = {0, 0, 0}, lJ = 0.0;
    for (int j = 0; j < s->N; ++j) {
      if (j == i) continue;
      double r = dist(&x[3 * i], &x[3 * j]);
      double u, u1, u2;
      pair_ee(s, i, j, r, &u, &u1, &u2);
      for (int k = 0; k < 3; ++k) gJ[k] += u1 * (x[3 * i + k] - x[3 * j + k]) / r;
      lJ += u2 + 2.0 * u1 / r;
      if (j > i && s->ee_on) V += 1.0 / r;
    }
    for (int I = 0; I < s->n_nuc; ++I) {
      double r = dist(&x[3 * i], s->R[I]);
      double u, u1, u2;
      pair_en(s, I, r, &u, &u1, &u2);
      for (int k = 0; k < 3; ++k) gJ[k] += u1 * (x[3 * i + k] - s->R[I][k]) / r;
      lJ += u2 + 2.0 * u1 / r;
      V -= s->Z[I] / r;
    }
    if (grad_log_psi)
      for (int k = 0; k < 3; ++k) grad_log_psi[3 * i + k] = gD[k] + gJ[k];
    total += lD + 2.0 * (gD[0] * gJ[0] + gD[1] * gJ[1] + gD[2] * gJ[2]) + lJ
             + gJ[0] * gJ[0] + gJ[1] * gJ[1] + gJ[2] * gJ[2];
  }
  for (int I = 0; I < s->n_nuc; ++I)
    for (int J = I + 1; J < s->n_nuc; ++J) V += s->Z[I] * s->Z[J] / dist(s->R[I], s->R[J]);
  free(chi); free(g); free(lp);
  *lap_over_psi = total;
  *V_out = V;
}

void orc_laplacian_terms(const orc_system* s, const double* x, const double* Ainv_up,
                         const double* Ainv_dn, double* lap_over_psi, double* V_out)
{
  laplacian_terms(s, x, Ainv_up, Ainv_dn, lap_over_psi, V_out, NULL);
}

/* grad_i log|psi_G(x)| = grad_i D/D + grad_i J for every electron ([N][3]). */
void orc_grad_log_psi(const orc_system* s, const double* x, const double* Ainv_up,
                      const double* Ainv_dn, double* grad)
{
  double lap, V;
  laplacian_terms(s, x, Ainv_up, Ainv_dn, &lap, &V, grad);
}

/* E_L(x) = -1/2 lap psi_G / psi_G + V(x). The lattice-regularized local
 * energy of psi_G with the fixed-node H^a equals this continuous value,
 * because V^a = V + (Delta^{a,a'} psi_G - lap psi_G) / (2 psi_G) by
 * construction in the cited method. */
double orc_local_energy(const orc_system* s, const double* x, const double* Ainv_up,
                        const double* Ainv_dn)
{
  double lap, V;
  orc_laplacian_terms(s, x, Ainv_up, Ainv_dn, &lap, &V);
  return -0.5 * lap + V;
}

/* Sherman-Morrison update of one spin block when electron l moves to r_new:
 * y_n = sum_m phi_m(r_new) Ainv[m][n], ratio = y_l,
 * Ainv'[m][n] = Ainv[m][n] - Ainv[m][l] (y_n - delta_nl) / ratio. */
int orc_sm_update(const orc_system* s, int spin, double* Ainv, int l, const double r_new[3],
                  double* ratio_out)
{
  int n = spin_count(s, spin);
  double* chi = (double*)malloc(sizeof(double) * s->n_ao);
  double* phi = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  double* col = (double*)malloc(sizeof(double) * n);
  orc_ao_values(s, r_new, chi, NULL, NULL);
  orbitals(s, chi, n, phi);
  for (int q = 0; q < n; ++q) {
    double v = 0.0;
    for (int m = 0; m < n; ++m) v += phi[m] * Ainv[m * n + q];
    y[q] = v;
  }
  double ratio = y[l];
  int rc = (ratio == 0.0) ? 1 : 0;
  if (!rc) {
    for (int m = 0; m < n; ++m) col[m] = Ainv[m * n + l];
    for (int m = 0; m < n; ++m)
      for (int q = 0; q < n; ++q)
        Ainv[m * n + q] -= col[m] * (y[q] - (q == l ? 1.0 : 0.0)) / ratio;
  }
  if (ratio_out) *ratio_out = ratio;
  free(chi); free(phi); free(y); free(col);
  return rc;
}

/* =========================================================================
 * 4. The lattice: Eq. 1 with p(r) from Eq. 2 or Eq. 3.
 * ========================================================================= */

int orc_n_candidates(const orc_system* s, int G) { return s->N * G * 6; }

/* p(r) at a point: R_c is the nucleus closest to r among the heaviest ones
 * (for a polyatomic system only the atoms with Z = Z_max count). Eq. 3
 * (Gaussian, r_c a length): exp(-|r - R_c|^2 / (2 r_c^2)). Eq. 2 (Pade,
 * r_c an inverse length, r_c = Z/2 with Eq. 4): 1 / (1 + r_c^2 |r - R_c|^2). */
double orc_p(const orc_system* s, const orc_lattice* L, const double r[3])
{
  double zmax = 0.0;
  for (int I = 0; I < s->n_nuc; ++I) if (s->Z[I] > zmax) zmax = s->Z[I];
  double best = INFINITY;
  for (int I = 0; I < s->n_nuc; ++I) {
    if (s->Z[I] != zmax) continue;
    double dx = r[0] - s->R[I][0], dy = r[1] - s->R[I][1], dz = r[2] - s->R[I][2];
    double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 < best) best = d2;
  }
  if (L->pkind == 0) return exp(-best / (2.0 * L->rc * L->rc));
  return 1.0 / (1.0 + L->rc * L->rc * best);
}

/* One evaluation of every lattice move out of configuration x.
 * Eq. 1 with the finite-difference form of the cited method: for electron
 * i, spacing h and rotated axis e_k,
 *   Delta^{h,q}_i f(x) = sum_k h^-2 [ q(r_i + h e_k/2) (f(x_i^{+h,k}) - f(x))
 *                                   + q(r_i - h e_k/2) (f(x_i^{-h,k}) - f(x)) ],
 * and Delta^{a,a'}_i = Delta^{a,p}_i + Delta^{a',1-p}_i (single grid: p = 1).
 * The off-diagonal element of H^a to the neighbour x' is -w/(2 h^2), with
 * w = p(mid) on the a grid and 1 - p(mid) on the a' grid. Fixed node with
 * sign flip (gamma = 0): moves with psi_G(x')/psi_G(x) < 0 are removed from
 * the off-diagonal part. The importance-sampled jump rate to x' is
 *   T(x' <- x) = w / (2 h^2) * max(psi_G(x') / psi_G(x), 0),
 * and b_x = sum of all T is the total rate of leaving x.
 * Outputs: ratio[c] = psi_G(x'_c)/psi_G(x), w[c], T[c], *b, *EL. */
void orc_lattice_eval(const orc_system* s, const orc_lattice* L, const double* x,
                      const double* Ainv_up, const double* Ainv_dn, const double* R,
                      double* ratio, double* w, double* T, double* b, double* EL)
{
  const int N = s->N, G = L->G;
  double* chi = (double*)malloc(sizeof(double) * s->n_ao);
  double* phi = (double*)malloc(sizeof(double) * (s->n_up > 0 ? s->n_up : 1));
  double bsum = 0.0;
  for (int i = 0; i < N; ++i) {
    int spin = spin_of(s, i), l = local_index(s, i), n = spin_count(s, spin);
    const double* Ainv = spin == 0 ? Ainv_up : Ainv_dn;
    for (int g = 0; g < G; ++g) {
      double h = (g == 0) ? L->a : L->ap;
      for (int k = 0; k < 3; ++k) {
        double e[3] = {R[0 * 3 + k], R[1 * 3 + k], R[2 * 3 + k]};
        for (int sg = 0; sg < 2; ++sg) {
          double sign = sg == 0 ? 1.0 : -1.0;
          int c = ((i * G + g) * 3 + k) * 2 + sg;
          double rn[3], mid[3];
          for (int d = 0; d < 3; ++d) {
            rn[d] = x[3 * i + d] + sign * h * e[d];
            mid[d] = x[3 * i + d] + sign * (0.5 * h) * e[d];
          }
          /* determinant ratio: orbitals at the new position, then the dot
           * with column l of the inverse Slater matrix */
          orc_ao_values(s, rn, chi, NULL, NULL);
          orbitals(s, chi, n, phi);
          double rdet = 0.0;
          for (int m = 0; m < n; ++m) rdet += phi[m] * Ainv[m * n + l];
          /* Jastrow ratio: the terms of J that involve electron i */
          double dJ = 0.0;
          for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            dJ += u_ee(s, i, j, dist(rn, &x[3 * j])) - u_ee(s, i, j, dist(&x[3 * i], &x[3 * j]));
          }
          for (int I = 0; I < s->n_nuc; ++I)
            dJ += u_en(s, I, dist(rn, s->R[I])) - u_en(s, I, dist(&x[3 * i], s->R[I]));
          double rho = rdet * exp(dJ);
          double wc = 1.0;
          if (G == 2) {
            double pm = orc_p(s, L, mid);
            wc = (g == 0) ? pm : 1.0 - pm;
          }
          double Tc = rho > 0.0 ? wc / (2.0 * h * h) * rho : 0.0;
          if (ratio) ratio[c] = rho;
          if (w) w[c] = wc;
          if (T) T[c] = Tc;
          bsum += Tc;
        }
      }
    }
  }
  free(chi); free(phi);
  if (b) *b = bsum;
  if (EL) *EL = orc_local_energy(s, x, Ainv_up, Ainv_dn);
}

/* =========================================================================
 * 5. Walkers, continuous-time projection and reconfiguration.
 *
 * The paper defines the lattice Hamiltonian H^a (the "Boosting the
 * double-grid LRDMC" paragraph of the main text: Eq. 1 with p of Eq. 2 or
 * Eq. 3, and a' of Eq. 4 or Eq. 6). It leaves the projection itself to the
 * LRDMC literature it cites with Eq. 1 (Casula, Filippi and Sorella, 2005;
 * Becca and Sorella, 2017). That projection is continuous-time Green's
 * function Monte Carlo with heat-bath jumps, the fixed node with sign flip,
 * and population control. The functions below write those steps out in
 * their plain form, one walker at a time:
 *  - run_interval: waiting times, weights and heat-bath jumps;
 *  - orc_heat_bath;
 *  - orc_sm_update: the Sherman-Morrison rank-one update;
 *  - reconfigure and orc_comb: the comb.
 * ========================================================================= */

struct orc_pop {
  orc_system* s;
  int W, P_cap;
  uint64_t seed;
  double tau, e_trial;
  int recompute_every;
  double* x; double* Aup; double* Adn; double* rot; double* T;
  double* b; double* EL; double* logw; int* jumps;
  /* values of the last finished interval, before reconfiguration */
  double* logw_pre; int* jumps_pre; int* parent;
  double* margin_w; double margin_comb;
  double* margin_teeth;  /* per new slot t: distance of tooth t from its bin's edges */
  int have_eval; orc_lattice eval_lat; int P;
  uint64_t k;
  int n_trace, cap_trace;
  double* tr_e; double* tr_w; double* tr_j;
  long long moves;
  int err;
};


/* Heat-bath choice among the lattice moves: the smallest c with
 * u * b < C_c, C_c = sum_{c' <= c} T_c' summed in candidate order; b is the
 * total rate (the same sequential sum). *margin receives the smallest
 * |u b - C_c| / b over the moves with T_c > 0 (the distance of the decision
 * from a bin edge). Returns -1 only when every T_c is zero. */
int orc_heat_bath(const double* T, int P, double b, double u, double* margin)
{
  double target = u * b, C = 0.0, mg = INFINITY;
  int chosen = -1, last_pos = -1;
  for (int c = 0; c < P; ++c) {
    if (!(T[c] > 0.0)) continue;
    C += T[c];
    last_pos = c;
    double mc = fabs(target - C) / b;
    if (mc < mg) mg = mc;
    if (chosen < 0 && target < C) chosen = c;
  }
  if (chosen < 0) chosen = last_pos;
  if (margin) *margin = mg;
  return chosen;
}

/* Comb (systematic) resampling of a population with weights wt[0..W-1]:
 * C_s = sum_{s' <= s} wt_s' in slot order; new slot t takes the parent s
 * whose bin [C_{s-1}, C_s) holds (t + xi) * C_{W-1} / W. Every walker gets
 * floor or ceil of W wt_s / sum(wt) copies, exactly that many on average
 * over xi. *margin receives the smallest distance of a tooth from the edges
 * of its bin, relative to the total weight; margin_teeth[t] (nullable) the
 * same distance for tooth t alone. */
void orc_comb(int W, const double* wt, double xi, int* parent, double* margin, double* margin_teeth)
{
  double* C = (double*)malloc(sizeof(double) * W);
  double sumw = 0.0, mg = INFINITY;
  for (int s = 0; s < W; ++s) { sumw += wt[s]; C[s] = sumw; }
  double total = C[W - 1];
  int s_ptr = 0;
  for (int t = 0; t < W; ++t) {
    double target = ((double)t + xi) * total / (double)W;
    while (s_ptr < W - 1 && !(target < C[s_ptr])) ++s_ptr;
    parent[t] = s_ptr;
    double mt = fabs(target - C[s_ptr]) / total;
    if (s_ptr > 0) {
      double m2 = fabs(target - C[s_ptr - 1]) / total;
      if (m2 < mt) mt = m2;
    }
    if (mt < mg) mg = mt;
    if (margin_teeth) margin_teeth[t] = mt;
  }
  if (margin) *margin = mg;
  free(C);
}

#define MAX_ITERS_PER_INTERVAL 1000000
static const uint64_t TAG_TIME_HB = 0, TAG_ROT = 1, TAG_COMB = 2;
static const uint64_t SLOT_GLOBAL = 0xFFFFFFFFFFFFFFFFULL;
static const uint64_t K_INIT = 0xFFFFFFFFFFFFFFFFULL;

static void draw4(const orc_pop* p, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t tag, double u[4])
{
  uint64_t ctr[4] = {c0, c1, c2, tag}, key[2] = {p->seed, 0}, o[4];
  orc_philox4x64(ctr, key, o);
  for (int j = 0; j < 4; ++j) u[j] = orc_uniform(o[j]);
}

orc_pop* orc_pop_create(orc_system* s, int W, const double* x0, uint64_t seed,
                        double tau, double e_trial, int recompute_every)
{
  if (!s || W < 1 || !(tau > 0.0)) return NULL;
  orc_pop* p = (orc_pop*)calloc(1, sizeof(orc_pop));
  int N = s->N, nu = s->n_up, nd = s->n_dn;
  p->s = s; p->W = W; p->seed = seed; p->tau = tau; p->e_trial = e_trial;
  p->recompute_every = recompute_every;
  p->P_cap = N * 12;
  p->x = (double*)malloc(sizeof(double) * W * N * 3);
  p->Aup = (double*)malloc(sizeof(double) * W * nu * nu);
  p->Adn = (double*)malloc(sizeof(double) * W * (nd > 0 ? nd * nd : 1));
  p->rot = (double*)malloc(sizeof(double) * W * 9);
  p->T = (double*)calloc((size_t)W * p->P_cap, sizeof(double));
  p->b = (double*)calloc(W, sizeof(double));
  p->EL = (double*)calloc(W, sizeof(double));
  p->logw = (double*)calloc(W, sizeof(double));
  p->jumps = (int*)calloc(W, sizeof(int));
  p->logw_pre = (double*)calloc(W, sizeof(double));
  p->jumps_pre = (int*)calloc(W, sizeof(int));
  p->parent = (int*)calloc(W, sizeof(int));
  p->margin_w = (double*)calloc(W, sizeof(double));
  p->margin_teeth = (double*)calloc(W, sizeof(double));
  memcpy(p->x, x0, sizeof(double) * W * N * 3);
  for (int w = 0; w < W; ++w) {
    p->parent[w] = w;
    if (orc_inverses(s, &p->x[w * N * 3], &p->Aup[w * nu * nu], nd > 0 ? &p->Adn[w * nd * nd] : NULL))
      p->err = 3;
    /* rotation of the first evaluation: counter (slot, k = all ones, 0, TAG_ROT) */
    double u[4];
    draw4(p, (uint64_t)w, K_INIT, 0, TAG_ROT, u);
    orc_rotation(u[0], u[1], u[2], &p->rot[w * 9]);
  }
  p->cap_trace = 1024;
  p->tr_e = (double*)malloc(sizeof(double) * p->cap_trace);
  p->tr_w = (double*)malloc(sizeof(double) * p->cap_trace);
  p->tr_j = (double*)malloc(sizeof(double) * p->cap_trace);
  return p;
}

void orc_pop_destroy(orc_pop* p)
{
  if (!p) return;
  free(p->x); free(p->Aup); free(p->Adn); free(p->rot); free(p->T); free(p->b); free(p->EL);
  free(p->logw); free(p->jumps); free(p->logw_pre); free(p->jumps_pre); free(p->parent);
  free(p->margin_w); free(p->margin_teeth); free(p->tr_e); free(p->tr_w); free(p->tr_j); free(p);
}

static void eval_walker(orc_pop* p, const orc_lattice* L, int w)
{
  const orc_system* s = p->s;
  int N = s->N, nu = s->n_up, nd = s->n_dn;
  orc_lattice_eval(s, L, &p->x[w * N * 3], &p->Aup[w * nu * nu],
                   nd > 0 ? &p->Adn[w * nd * nd] : NULL, &p->rot[w * 9],
                   NULL, NULL, &p->T[(size_t)w * p->P_cap], &p->b[w], &p->EL[w]);
}

/* Apply lattice move c: electron i goes to r_i + sign h e_k, with a
 * Sherman-Morrison update of its spin block. */
static int apply_move(orc_pop* p, const orc_lattice* L, int w, int c)
{
  const orc_system* s = p->s;
  int N = s->N, nu = s->n_up, nd = s->n_dn, G = L->G;
  int sg = c % 2, k = (c / 2) % 3, g = (c / 6) % G, i = c / (6 * G);
  double h = (g == 0) ? L->a : L->ap, sign = sg == 0 ? 1.0 : -1.0;
  const double* R = &p->rot[w * 9];
  double* xi = &p->x[(w * N + i) * 3];
  double rn[3];
  for (int d = 0; d < 3; ++d) rn[d] = xi[d] + sign * h * R[d * 3 + k];
  int spin = spin_of(s, i);
  double* Ainv = spin == 0 ? &p->Aup[w * nu * nu] : &p->Adn[w * nd * nd];
  double ratio;
  int rc = orc_sm_update(s, spin, Ainv, local_index(s, i), rn, &ratio);
  for (int d = 0; d < 3; ++d) xi[d] = rn[d];
  return rc;
}

/* One interval of length tau for walker w (continuous-time Green's function
 * Monte Carlo of the cited method): the walker waits at x for an
 * exponentially distributed time of rate b_x, its log-weight decreases by
 * (E_L(x) - E_T) times the time spent, and at the end of the wait it jumps
 * to candidate c with probability T_c / b_x (heat bath). Uniforms come from
 * Philox with counter (slot, interval k, iteration m, tag). */
static void run_interval(orc_pop* p, const orc_lattice* L, int w, uint64_t k)
{
  double tau_left = p->tau, margin = INFINITY;
  const int P = p->P;
  double* T = &p->T[(size_t)w * p->P_cap];
  uint64_t m = 0;
  p->logw[w] = 0.0;
  p->jumps[w] = 0;
  for (;;) {
    double u[4];
    draw4(p, (uint64_t)w, k, m, TAG_TIME_HB, u);
    double xi = u[0], uh = u[1];
    double t = p->b[w] > 0.0 ? -log(xi) / p->b[w] : INFINITY;
    double mt = fabs(t - tau_left) / p->tau;
    if (mt < margin) margin = mt;
    if (t >= tau_left) {
      p->logw[w] -= tau_left * (p->EL[w] - p->e_trial);
      break;
    }
    p->logw[w] -= t * (p->EL[w] - p->e_trial);
    tau_left -= t;
    double mhb;
    int chosen = orc_heat_bath(T, P, p->b[w], uh, &mhb);
    if (mhb < margin) margin = mhb;
    if (apply_move(p, L, w, chosen)) p->err = 3;
    draw4(p, (uint64_t)w, k, m, TAG_ROT, u);
    orc_rotation(u[0], u[1], u[2], &p->rot[w * 9]);
    eval_walker(p, L, w);
    if (!isfinite(p->EL[w]) || !isfinite(p->b[w])) { p->err = 4; break; }
    ++m;
    p->jumps[w] += 1;
    if (m > MAX_ITERS_PER_INTERVAL) { p->err = 5; break; }
  }
  p->margin_w[w] = margin;
}

static int same_lattice(const orc_lattice* a, const orc_lattice* b)
{
  return a->a == b->a && a->G == b->G && (a->G == 1 || (a->ap == b->ap && a->pkind == b->pkind && a->rc == b->rc));
}

/* Reconfiguration at the end of interval k (fixed population, comb /
 * systematic resampling): w_s = exp(log w_s); the trace gets
 * e_k = sum_s w_s E_L(x_s) / sum_s w_s, wbar_k = mean w and the mean number of
 * jumps; new slot t takes the parent s whose cumulative-weight bin
 * [C_{s-1}, C_s) holds (t + xi) * C_{W-1} / W, xi one uniform per interval;
 * every weight is then reset to 1. */
static void reconfigure(orc_pop* p, uint64_t k)
{
  const orc_system* s = p->s;
  const int W = p->W, N = s->N, nu = s->n_up, nd = s->n_dn;
  double* wt = (double*)malloc(sizeof(double) * W);
  double sumw = 0.0, sumwe = 0.0, sumj = 0.0;
  for (int w = 0; w < W; ++w) {
    wt[w] = exp(p->logw[w]);
    sumw += wt[w];
    sumwe += wt[w] * p->EL[w];
    sumj += p->jumps[w];
    p->logw_pre[w] = p->logw[w];
    p->jumps_pre[w] = p->jumps[w];
  }
  if (p->n_trace == p->cap_trace) {
    p->cap_trace *= 2;
    p->tr_e = (double*)realloc(p->tr_e, sizeof(double) * p->cap_trace);
    p->tr_w = (double*)realloc(p->tr_w, sizeof(double) * p->cap_trace);
    p->tr_j = (double*)realloc(p->tr_j, sizeof(double) * p->cap_trace);
  }
  p->tr_e[p->n_trace] = sumwe / sumw;
  p->tr_w[p->n_trace] = sumw / W;
  p->tr_j[p->n_trace] = sumj / W;
  p->n_trace++;
  double u[4];
  draw4(p, SLOT_GLOBAL, k, 0, TAG_COMB, u);
  orc_comb(W, wt, u[0], p->parent, &p->margin_comb, p->margin_teeth);
  /* gather the parents' state into the new slots */
  const int P = p->P_cap;
  double* x = (double*)malloc(sizeof(double) * W * N * 3);
  double* Au = (double*)malloc(sizeof(double) * W * nu * nu);
  double* Ad = (double*)malloc(sizeof(double) * W * (nd > 0 ? nd * nd : 1));
  double* R = (double*)malloc(sizeof(double) * W * 9);
  double* T = (double*)malloc(sizeof(double) * (size_t)W * P);
  double* b = (double*)malloc(sizeof(double) * W);
  double* EL = (double*)malloc(sizeof(double) * W);
  for (int t = 0; t < W; ++t) {
    int q = p->parent[t];
    memcpy(&x[t * N * 3], &p->x[q * N * 3], sizeof(double) * N * 3);
    memcpy(&Au[t * nu * nu], &p->Aup[q * nu * nu], sizeof(double) * nu * nu);
    if (nd > 0) memcpy(&Ad[t * nd * nd], &p->Adn[q * nd * nd], sizeof(double) * nd * nd);
    memcpy(&R[t * 9], &p->rot[q * 9], sizeof(double) * 9);
    memcpy(&T[(size_t)t * P], &p->T[(size_t)q * P], sizeof(double) * P);
    b[t] = p->b[q];
    EL[t] = p->EL[q];
  }
  free(p->x); free(p->Aup); free(p->Adn); free(p->rot); free(p->T); free(p->b); free(p->EL);
  p->x = x; p->Aup = Au; p->Adn = Ad; p->rot = R; p->T = T; p->b = b; p->EL = EL;
  for (int w = 0; w < W; ++w) { p->logw[w] = 0.0; p->jumps[w] = 0; }
  free(wt);
}

int orc_pop_step(orc_pop* p, const orc_lattice* L, int n_steps, int n_threads)
{
  const orc_system* s = p->s;
  const int W = p->W, N = s->N, nu = s->n_up, nd = s->n_dn;
  if (L->G != 1 && L->G != 2) return 1;
  if (n_threads < 1) n_threads = 1;
  /* (re-)evaluate with the stored rotations when the lattice changed */
  if (!p->have_eval || !same_lattice(L, &p->eval_lat)) {
    p->P = orc_n_candidates(s, L->G);
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1)
    for (int w = 0; w < W; ++w) eval_walker(p, L, w);
    p->have_eval = 1;
    p->eval_lat = *L;
  }
  for (int step = 0; step < n_steps && !p->err; ++step) {
    uint64_t k = p->k;
    if (k > 0 && p->recompute_every > 0 && k % (uint64_t)p->recompute_every == 0) {
      for (int w = 0; w < W; ++w)
        if (orc_inverses(s, &p->x[w * N * 3], &p->Aup[w * nu * nu], nd > 0 ? &p->Adn[w * nd * nd] : NULL))
          p->err = 3;
    }
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1)
    for (int w = 0; w < W; ++w) run_interval(p, L, w, k);
    for (int w = 0; w < W; ++w) p->moves += p->jumps[w];
    reconfigure(p, k);
    p->k++;
  }
  return p->err;
}

int orc_pop_trace(const orc_pop* p, double* e, double* wbar, double* mean_jumps, int max_n)
{
  int n = p->n_trace < max_n ? p->n_trace : max_n;
  for (int j = 0; j < n; ++j) {
    if (e) e[j] = p->tr_e[j];
    if (wbar) wbar[j] = p->tr_w[j];
    if (mean_jumps) mean_jumps[j] = p->tr_j[j];
  }
  return n;
}

void orc_pop_walkers(const orc_pop* p, double* x, double* EL, double* b, double* T,
                     double* logw_pre, int* jumps_pre, int* parent)
{
  const int W = p->W, N = p->s->N;
  if (x) memcpy(x, p->x, sizeof(double) * W * N * 3);
  if (EL) memcpy(EL, p->EL, sizeof(double) * W);
  if (b) memcpy(b, p->b, sizeof(double) * W);
  if (T)
    for (int w = 0; w < W; ++w)
      memcpy(&T[(size_t)w * p->P], &p->T[(size_t)w * p->P_cap], sizeof(double) * p->P);
  if (logw_pre) memcpy(logw_pre, p->logw_pre, sizeof(double) * W);
  if (jumps_pre) memcpy(jumps_pre, p->jumps_pre, sizeof(int) * W);
  if (parent) memcpy(parent, p->parent, sizeof(int) * W);
}

void orc_pop_margins(const orc_pop* p, double* margin_walker, double* margin_comb, double* margin_teeth)
{
  if (margin_teeth) memcpy(margin_teeth, p->margin_teeth, sizeof(double) * p->W);
  if (margin_walker) memcpy(margin_walker, p->margin_w, sizeof(double) * p->W);
  if (margin_comb) *margin_comb = p->margin_comb;
}

long long orc_pop_moves(const orc_pop* p) { return p->moves; }
int orc_pop_error(const orc_pop* p) { return p->err; }
