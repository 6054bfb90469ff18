/*
 * Plain FP64 CPU oracle for lattice-regularized diffusion Monte Carlo (LRDMC)
 * with the single-grid and the double-grid ("smart") lattice of Nakano,
 * Maezono and Sorella, arXiv:1909.01589.
 *
 * TEST INFRASTRUCTURE ONLY. This header and lrdmc_oracle.c are used by the
 * test suite, by the smoke check and by the CPU-baseline leg of the
 * benchmark. The product library never includes, links or calls them, and
 * they include nothing from the product.
 *
 * Conventions shared by every function below:
 *  - lengths in bohr, energies in hartree, all arithmetic in IEEE double;
 *  - electron configurations x are [N][3] row-major, electrons
 *    0..n_up-1 are spin up, n_up..N-1 spin down;
 *  - a lattice rotation is a 3x3 row-major matrix whose column k is the
 *    rotated axis e_k;
 *  - A_sigma[l][m] = phi_m(r_l) (row = electron of that spin, column =
 *    orbital), inverses are stored row-major as Ainv[m][l];
 *  - candidate c of a configuration is ordered electron-major, then grid
 *    (a before a'), then axis (x, y, z), then sign (+ before -):
 *        c = ((i*G + g)*3 + k)*2 + (sign < 0).
 */
#ifndef LRDMC_ORACLE_H
#define LRDMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_NUC 16
#define ORC_MAX_PRIM 16
#define ORC_NJ_MAX_CH 8

/* ---- parameters of the double grid (Eq. 2-10, S-12..S-14) ---- */
double orc_rc_this_work(double a, double Z, double beta, double kappa);
int    orc_slater_groups(int Z, int* n, int* l_max, double* n_eff,
                         double* zeta, int* occ, int max_groups);
double orc_ncore(int Z, double rc);
double orc_aprime_over_a_this_work(int Z, double a, double beta, double kappa);
double orc_aprime_over_a_previous(double Z);
double orc_speedup(double Z, double n_core, double aprime_over_a);

/* ---- counter-based generator (Philox4x64-10, Salmon et al., SC'11) and the
 *      random lattice rotation (Shoemake's uniform quaternion) ---- */
void   orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double orc_uniform(uint64_t bits);
void   orc_rotation(double u1, double u2, double u3, double R[9]);

/* ---- the trial function psi_G = det_up * det_dn * exp(J) (Slater-Jastrow,
 *      Pade Jastrow factor); E_L = -lap psi_G / (2 psi_G) + V ---- */
typedef struct orc_system orc_system;
orc_system* orc_system_create(int n_nuc, const double* nuc_xyz, const double* Z,
                              int n_up, int n_dn,
                              int n_shell, const int* sh_center, const int* sh_l,
                              const int* sh_kind, const int* sh_nprim,
                              const double* sh_neff, const double* sh_zeta,
                              const double* prim_alpha, const double* prim_coef,
                              int n_ao, int n_mo, const double* C,
                              double b_ee, double c_par, double c_anti,
                              const double* en_b1, double en_b2, int ee_on);
void   orc_system_destroy(orc_system* s);
int    orc_n_ao(const orc_system* s);
void   orc_ao_values(const orc_system* s, const double r[3], double* chi,
                     double* grad /*[n_ao][3] or NULL*/, double* lap /* or NULL */);
int    orc_log_psi(const orc_system* s, const double* x, double* log_abs, double* sign);
int    orc_inverses(const orc_system* s, const double* x, double* Ainv_up, double* Ainv_dn);
void   orc_laplacian_terms(const orc_system* s, const double* x, const double* Ainv_up,
                           const double* Ainv_dn, double* lap_over_psi, double* V);
double orc_local_energy(const orc_system* s, const double* x, const double* Ainv_up,
                        const double* Ainv_dn);
void   orc_grad_log_psi(const orc_system* s, const double* x, const double* Ainv_up,
                        const double* Ainv_dn, double* grad /*[N][3]*/);

/* ---- optional neural pair term (tabulated, quintic Hermite) ---- */
int    orc_system_set_neural(orc_system* s, int n_ch, int n_cells, const double* r_cut,
                             const int* species /*[n_nuc]*/,
                             const double* nodes /*[n_ch][n_cells+1][3]*/);
void   orc_neural_pair(const orc_system* s, int channel, double r, double* g, double* g1,
                       double* g2);
int    orc_sm_update(const orc_system* s, int spin, double* Ainv, int l,
                     const double r_new[3], double* ratio);

/* ---- the lattice (Eq. 1 with p from Eq. 2 or Eq. 3) ---- */
typedef struct {
  double a;        /* small spacing                                    */
  double ap;       /* large spacing a' (ignored when G == 1)           */
  int    G;        /* 1 = single grid, 2 = double grid                 */
  int    pkind;    /* 0 = Gaussian p (Eq. 3), 1 = Pade p (Eq. 2)       */
  double rc;       /* r_c: a length for Eq. 3, an inverse length Eq. 2 */
} orc_lattice;

int    orc_n_candidates(const orc_system* s, int G);
double orc_p(const orc_system* s, const orc_lattice* L, const double r[3]);
void   orc_lattice_eval(const orc_system* s, const orc_lattice* L, const double* x,
                        const double* Ainv_up, const double* Ainv_dn, const double* R,
                        double* ratio, double* w, double* T, double* b, double* EL);

/* ---- heat bath and comb: the jump choice and the population control of
 *      the LRDMC projection cited with Eq. 1 ---- */
int    orc_heat_bath(const double* T, int P, double b, double u, double* margin);
void   orc_comb(int W, const double* wt, double xi, int* parent, double* margin, double* margin_teeth);

/* ---- the walker population and the continuous-time projection with H^a
 *      (Eq. 1; the method cited with it) ---- */
typedef struct orc_pop orc_pop;
orc_pop* orc_pop_create(orc_system* s, int W, const double* x0, uint64_t seed,
                        double tau, double e_trial, int recompute_every);
void   orc_pop_destroy(orc_pop* p);
int    orc_pop_step(orc_pop* p, const orc_lattice* L, int n_steps, int n_threads);
int    orc_pop_trace(const orc_pop* p, double* e, double* wbar, double* mean_jumps, int max_n);
void   orc_pop_walkers(const orc_pop* p, double* x, double* EL, double* b, double* T,
                       double* logw_pre, int* jumps_pre, int* parent);
void   orc_pop_margins(const orc_pop* p, double* margin_walker, double* margin_comb,
                       double* margin_teeth);
long long orc_pop_moves(const orc_pop* p);
int    orc_pop_error(const orc_pop* p);

#ifdef __cplusplus
}
#endif
#endif
