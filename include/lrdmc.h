/*
 * lrdmc.h - C ABI of the GB300 (sm_103a) library for lattice-regularized
 * diffusion Monte Carlo with the single-grid and the double-grid ("smart")
 * lattice of Nakano, Maezono and Sorella, "Speeding up the ab initio
 * diffusion Monte Carlo by a smart lattice regularization", arXiv:1909.01589.
 *
 * What the library computes, per walker and per walker-move:
 *   - the lattice moves of every electron, r_i -> r_i +- h e_k on a randomly
 *     rotated lattice, with h = a and (double grid) h = a', Eq. 1;
 *   - p at each bond midpoint from Eq. 3 (this work) or Eq. 2 (previous),
 *     with r_c and a'/a from S-13 and Eq. 6 / Eq. 7, or from Eq. 4;
 *   - psi_G(x')/psi_G(x) at every move for a Slater-Jastrow trial function,
 *     the fixed-node jump rates T = w/(2h^2) max(ratio, 0) and the local
 *     energy (the LRDMC method the paper builds on, Casula, Filippi and
 *     Sorella, PRL 95, 100201 (2005));
 *   - continuous-time projection: waiting time, weight, heat-bath jump and
 *     Sherman-Morrison update of the inverse Slater matrix, and comb
 *     reconfiguration of the population at the end of every interval tau.
 *
 * Conventions for every entry point:
 *   - lengths in bohr, energies in hartree, all floating point in IEEE
 *     double (FP64);
 *   - configurations are [N][3] row-major, electrons 0..n_up-1 spin up;
 *   - a rotation is a 3x3 row-major matrix whose column k is the axis e_k;
 *   - candidate (lattice move) c is ordered electron-major, then grid
 *     (a before a'), axis (x, y, z), sign (+ before -):
 *         c = ((i*G + g)*3 + k)*2 + (sign < 0),   P = 6 G N moves;
 *   - every function returns a status and never aborts; on failure
 *     lrdmc_last_error() describes the cause;
 *   - device pointers are plain CUDA device addresses (e.g. from PyTorch),
 *     owned by the caller; host pointers are ordinary host memory, owned by
 *     the caller; the library copies what it needs during the call;
 *   - a stream is borrowed, never destroyed; all work of a system is
 *     ordered on the stream given to lrdmc_init_walkers.
 * Random numbers: Philox4x64-10 (Salmon et al., SC'11) keyed by (seed, 0),
 * counter (walker slot, interval k, iteration m, tag); uniforms are
 * ((bits >> 12) + 1/2) 2^-52.
 */
#ifndef LRDMC_H
#define LRDMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LRDMC_API __attribute__((visibility("default")))
#else
#define LRDMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define LRDMC_MAX_NUC 8
#define LRDMC_MAX_SHELL 32
#define LRDMC_MAX_PRIM 8
#define LRDMC_MAX_AO 64
#define LRDMC_MAX_SPIN 32 /* electrons per spin */

typedef struct lrdmc_system_s* lrdmc_system_t;

typedef enum {
  LRDMC_OK = 0,
  LRDMC_ERR_ARG = 1,       /* invalid argument or size beyond the limits    */
  LRDMC_ERR_CUDA = 2,      /* a CUDA call failed                            */
  LRDMC_ERR_SINGULAR = 3,  /* singular Slater matrix or zero update ratio   */
  LRDMC_ERR_NONFINITE = 4, /* non-finite local energy or rate               */
  LRDMC_ERR_TIMEOUT = 5,   /* an interval exceeded its iteration limit      */
  LRDMC_ERR_STATE = 6,     /* call out of order (e.g. step before init)     */
  LRDMC_ERR_BOUNDS = 7     /* a checked index was out of range (only in a
                              build with -DLRDMC_BOUNDS, see
                              lrdmc_build_flags)                            */
} lrdmc_status;

/* Build flags of the loaded library (lrdmc_build_flags). */
#define LRDMC_BUILD_BOUNDS 1 /* compiled with -DLRDMC_BOUNDS                */

/* Lattice spacing function, Eq. 1-7 and S-13. */
typedef enum {
  LRDMC_SINGLE = 0,           /* single grid, p = 1                          */
  LRDMC_DOUBLE_THIS_WORK = 1, /* Gaussian p (Eq. 3), r_c from S-13, a'/a Eq. 6 */
  LRDMC_DOUBLE_PREVIOUS = 2,  /* Pade p (Eq. 2) with r_c = Z/2, a'/a Eq. 4   */
  LRDMC_DOUBLE_EXPLICIT = 3   /* Gaussian p with the given r_c and a'/a      */
} lrdmc_spacing_kind;

typedef struct {
  int kind;             /* lrdmc_spacing_kind                                  */
  double beta;          /* S-13 prefactor (0.75 in the paper), THIS_WORK only  */
  double kappa;         /* S-13 f(a) constant (2.5 in the paper), THIS_WORK   */
  double rc;            /* r_c, EXPLICIT only                                 */
  double aprime_over_a; /* a'/a, EXPLICIT only                               */
} lrdmc_spacing_fn;

/* One shell of atomic orbitals: 2l+1 real solid harmonics S (l = 0: 1;
 * l = 1: x, y, z; l = 2: xy, yz, zx, x^2-y^2, 2z^2-x^2-y^2) times a radial
 * part, kind 0 (Slater): r^(n_eff-1-l) exp(-zeta r); kind 1 (contracted
 * Gaussian): sum_p coef[p] exp(-alpha[p] r^2). */
typedef struct {
  int center; /* nucleus index                 */
  int l;      /* 0, 1 or 2                      */
  int kind;   /* 0 = Slater, 1 = Gaussian       */
  int n_prim; /* primitives (kind 1)            */
  double n_eff;
  double zeta;
  double alpha[LRDMC_MAX_PRIM];
  double coef[LRDMC_MAX_PRIM];
} lrdmc_shell;

/* Pade Jastrow factor J = sum_{i<j} c r_ij/(1 + b_ee r_ij)
 *   (c = c_par for equal spins, c_anti otherwise)
 *   - sum_{i,I} en_b1[I] r_iI/(1 + en_b2 r_iI);
 * ee_on = 0 drops the electron-electron Coulomb repulsion (test systems). */
typedef struct {
  double b_ee, c_par, c_anti, en_b2;
  double en_b1[LRDMC_MAX_NUC];
  int ee_on;
} lrdmc_jastrow;

/* Creates a system: nuclei [n_nuc][3] and charges Z [n_nuc], n_up >= n_dn
 * electrons, shells (AOs numbered shell by shell), MO coefficients C
 * [n_ao][n_mo] row-major shared by both spins (spin down uses the first
 * n_dn columns), Jastrow parameters. All inputs are host memory, copied.
 * Limits: n_nuc <= LRDMC_MAX_NUC, n_shell <= LRDMC_MAX_SHELL,
 * n_ao <= LRDMC_MAX_AO, n_up <= LRDMC_MAX_SPIN, n_mo >= n_up; and the
 * shared memory of one block of four walkers (positions, inverse Slater
 * matrices, rates, projected inverse columns and scratch, which grow as
 * N^2 and N n_ao) must fit in 227 KB. A system whose block fits only
 * without the double-float evaluation caches is laid out without them
 * (same results, slower double-float evaluation): e.g. 48 electrons on 8
 * centres with 42 AOs. 64 electrons with 62 AOs do not fit at all; such
 * systems fail with LRDMC_ERR_ARG and a message giving the size. So do
 * non-finite coordinates, Jastrow parameters or MO coefficients, a charge
 * that is not positive, and two nuclei at one point. No GPU work. */
LRDMC_API lrdmc_status lrdmc_create_system(int n_nuc, const double* nuc_xyz, const double* Z,
                                 int n_up, int n_dn, const lrdmc_shell* shells, int n_shells,
                                 const double* mo_coeff, int n_ao, int n_mo,
                                 const lrdmc_jastrow* jastrow, lrdmc_system_t* out);

/* Double-grid parameters for spacing a: a'/a and r_c (S-13 with Eq. 6 and
 * Eq. 7 for THIS_WORK, Eq. 4 with r_c = Z_max/2 for PREVIOUS; for a
 * polyatomic system from the heaviest atom, as the paper's section on large
 * systems prescribes). N_core of Eq. 7 uses Slater's-rule densities. Host
 * computation, no GPU. For SINGLE returns a'/a = 1, r_c = 0. */
LRDMC_API lrdmc_status lrdmc_spacing_params(lrdmc_system_t sys, double a, const lrdmc_spacing_fn* spacing,
                                  double* aprime_over_a, double* rc);

/* Device workspace bytes needed by lrdmc_init_walkers for n_walkers (1 to
 * LRDMC_MAX_WALKERS) and a trace of trace_capacity intervals. */
#define LRDMC_MAX_WALKERS 4194304
LRDMC_API lrdmc_status lrdmc_workspace_bytes(lrdmc_system_t sys, int n_walkers, int trace_capacity,
                                   size_t* bytes);

/* Starts a population of n_walkers (1 to LRDMC_MAX_WALKERS) at
 * configurations x0 [n_walkers][N][3] (host or device memory; copied). workspace is caller-owned device memory
 * of at least lrdmc_workspace_bytes(), 256-byte aligned, held by the system
 * until lrdmc_destroy or the next init. tau is the reconfiguration
 * interval, e_trial the energy shift of the log-weights, recompute_every the
 * number of intervals between full recomputations of the inverse Slater
 * matrices (0 = never). stream is a cudaStream_t (NULL = default stream).
 * Fails with LRDMC_ERR_SINGULAR if a start configuration has a singular
 * Slater matrix: two electrons of one spin on the same point, or a zero or
 * non-finite pivot in the elimination. */
LRDMC_API lrdmc_status lrdmc_init_walkers(lrdmc_system_t sys, int n_walkers, const double* x0,
                                uint64_t seed, double tau, double e_trial, int recompute_every,
                                int trace_capacity, void* workspace, size_t workspace_bytes,
                                void* stream);

/* Projects the population through n_steps intervals of length tau with
 * lattice spacing a and the given spacing function: per walker the
 * continuous-time loop (waiting time of rate b_x, weight exp(-t (E_L -
 * e_trial)), heat-bath jump, Sherman-Morrison update, new rotation and
 * evaluation of all P moves), then comb reconfiguration and one trace entry
 * per interval. Asynchronous: the call enqueues the kernels and a copy of
 * the device error word on the stream and returns; errors raised by the
 * kernels (singular matrix, non-finite energy, iteration limit) are
 * reported by the next synchronising call (lrdmc_sync and every read-back
 * function). Fails at once with LRDMC_ERR_ARG when the trace would exceed
 * its capacity. */
LRDMC_API lrdmc_status lrdmc_step(lrdmc_system_t sys, int n_steps, double a, const lrdmc_spacing_fn* spacing);

/* Waits for the system's stream and reports any error the enqueued steps
 * raised. */
LRDMC_API lrdmc_status lrdmc_sync(lrdmc_system_t sys);

/* Copies the trace to host arrays (each nullable, length >= max_n): e_k =
 * weighted mean local energy at the end of interval k, wbar_k = mean weight
 * exp(-int (E_L - e_trial) dt), mean_jumps_k. *n_written = min(max_n, k). */
LRDMC_API lrdmc_status lrdmc_get_energy_trace(lrdmc_system_t sys, double* e, double* wbar,
                                    double* mean_jumps, int max_n, int* n_written);

/* Enqueues, on the system's stream and without waiting, the copy of trace
 * entries [first, first + n) into host arrays e, wbar and mean_jumps (each
 * nullable, length >= n; the same quantities as lrdmc_get_energy_trace).
 * The copies run behind every step enqueued before the call, so entries
 * first .. first + n - 1 must belong to intervals already enqueued
 * (first + n <= the number of intervals stepped), else LRDMC_ERR_ARG. The
 * host arrays must stay valid until the next synchronising call (lrdmc_sync
 * or a read-back function), after which they hold the values; with pinned
 * host memory the copies are asynchronous, with pageable memory the CUDA
 * runtime may complete them before returning. Kernel errors are reported by
 * that synchronising call, as for lrdmc_step. */
LRDMC_API lrdmc_status lrdmc_get_energy_trace_async(lrdmc_system_t sys, int first, int n, double* e,
                                                    double* wbar, double* mean_jumps);

/* The Sherman-Morrison residual of every interval so far (not a step of
 * the paper's method: a diagnostic of the cited LRDMC implementation's
 * rank-one inverse updates). At the start of an interval whose inverse
 * Slater matrices are rebuilt (k > 0, k a multiple of recompute_every), the
 * kernel first measures, for every walker and spin block, max |sum_m
 * A[l][m] Ainv[m][q] - delta_lq| of the inverse the updates carried, A the
 * Slater matrix at the current positions; resid[k] is the largest over the
 * population, and -1 at intervals without a rebuild. Same count and
 * synchronisation as lrdmc_get_energy_trace. */
LRDMC_API lrdmc_status lrdmc_get_residual_trace(lrdmc_system_t sys, double* resid, int max_n, int* n_written);

/* Copies the population to host arrays (each nullable): positions
 * [W][N][3], E_L [W], b [W] and rates T [W][P] of the cached evaluation,
 * the pre-reconfiguration log-weights and jump counts [W] of the last
 * interval and the comb's parent indices [W]. Synchronises the stream. */
LRDMC_API lrdmc_status lrdmc_get_walkers(lrdmc_system_t sys, double* x, double* el, double* b, double* T,
                               double* logw_pre, int* jumps_pre, int* parent);

/* Total number of walker-moves (jumps, each with one evaluation of all P
 * moves) made by lrdmc_step since init. */
LRDMC_API lrdmc_status lrdmc_moves(lrdmc_system_t sys, long long* moves);

/* One evaluation of all P lattice moves for n_configs independent
 * configurations (no population state): x [n][N][3] and rotations
 * rot [n][9] are device inputs; ratio [n][P] (psi_G(x')/psi_G(x)),
 * T [n][P], b [n] and el [n] are device outputs (each nullable except
 * none of x, rot). Inverse Slater matrices are computed from x. */
LRDMC_API lrdmc_status lrdmc_evaluate(lrdmc_system_t sys, int n_configs, const double* x, const double* rot,
                            double a, const lrdmc_spacing_fn* spacing, double* ratio, double* T,
                            double* b, double* el, void* stream);

/* The same evaluation with the orbital contraction on the tensor cores, the
 * mixed-precision form of the basis x MO product the method needs at every
 * displaced position (Eq. 1 lattice moves; the determinant ratio
 * psi(x')/psi(x) of the cited LRDMC method): per lattice move the basis
 * values chi_mu(r') are computed in FP32, split into bfloat16 high and low
 * parts, and phi_m(r') = sum_mu chi_mu(r') C[mu][m] is formed by tcgen05
 * MMAs (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation in tensor
 * memory, about 16 significant bits) for 128 moves of four configurations
 * at a time; the determinant ratio sum_m phi_m Ainv[m][l], the Jastrow
 * ratio, p, the rates and the local energy are the FP32 mode's
 * (LRDMC_PRECISION_FP32, whatever the system's precision setting). Same
 * arguments, layouts and outputs as lrdmc_evaluate. Requires at most 32
 * orbitals per spin and room for the operand tiles in one block's shared
 * memory (LRDMC_ERR_ARG otherwise). LRDMC_ERR_TIMEOUT if a bounded wait for
 * the tensor core runs out; LRDMC_ERR_SINGULAR for a singular Slater
 * matrix. Synchronises the stream. */
LRDMC_API lrdmc_status lrdmc_evaluate_tc(lrdmc_system_t sys, int n_configs, const double* x, const double* rot,
                                         double a, const lrdmc_spacing_fn* spacing, double* ratio, double* T,
                                         double* b, double* el, void* stream);

/* Evaluation that allocates nothing. The paper has no counterpart: this
 * is a service for callers that cannot call cudaMalloc when they evaluate -
 * code running inside another framework's reserved memory budget,
 * processes that forbid device allocation after start-up, or callers that
 * must not let an allocation synchronise the device. Same inputs, outputs
 * and results as lrdmc_evaluate, whose error word comes from cudaMalloc;
 * here the scratch (a summary status word and one status word per
 * configuration) lives in a static device array of 64 + LRDMC_STATIC_EVAL_MAX
 * ints (about 1 MiB) that every GPU loading the library holds until the
 * process exits. n_configs above LRDMC_STATIC_EVAL_MAX is rejected with
 * LRDMC_ERR_ARG. The first call on a device looks up the array's device
 * address (once per device, with that device current). The call clears
 * the words it uses, then
 * synchronises the stream to read the summary word; when it reports
 * LRDMC_ERR_SINGULAR, lrdmc_last_error names the first configuration whose
 * status word is set. All calls share the
 * array and it keeps the last call's contents: calls that overlap on the
 * GPU (other threads, other streams) race on it. No cudaMalloc, cudaFree
 * or other device allocation happens in this call. */
#define LRDMC_STATIC_EVAL_MAX 262144
LRDMC_API lrdmc_status lrdmc_evaluate_static(lrdmc_system_t sys, int n_configs, const double* x,
                                             const double* rot, double a, const lrdmc_spacing_fn* spacing,
                                             double* ratio, double* T, double* b, double* el,
                                             void* stream);

/* Writes / reads the population (positions, inverses, rotations, cached
 * evaluation, parents, interval counter, trace) to / from a file. load
 * fails with LRDMC_ERR_ARG for a file of another population size or
 * layout, a truncated file, or (default build) a parent index outside
 * [0, W); a bounds-checked build (lrdmc_build_flags) leaves the parent
 * indices to the kernels' checks, which report LRDMC_ERR_BOUNDS at the next
 * lrdmc_sync. */
LRDMC_API lrdmc_status lrdmc_save(lrdmc_system_t sys, const char* path);
LRDMC_API lrdmc_status lrdmc_load(lrdmc_system_t sys, const char* path);

/* Arithmetic of the evaluation kernels. LRDMC_PRECISION_FP64 runs every
 * step in IEEE double on the FP64 pipe. LRDMC_PRECISION_DF64 (default)
 * evaluates the lattice moves and the local energy in double-float
 * arithmetic on the FP32 pipe (pairs of floats, about 48 significant bits,
 * relative error ~1e-14; GB300 runs FP64 at 1/69 of its FP32 rate) and
 * keeps the inverse Slater matrices, Sherman-Morrison updates, weights,
 * and reconfiguration in IEEE double. Values below about 1e-30 lose
 * low-order bits in double-float (their contribution to any sum is then
 * negligible); arguments of exp below -87 give 0. LRDMC_PRECISION_FP32 is
 * the mixed-precision mode: the lattice moves (ratios and rates), waiting
 * time and heat bath in IEEE single precision (ratios to ~1e-6 relative),
 * the local energy in double-float (a single-precision local energy's
 * rare large errors near the nuclei inflated the weights' variance), and
 * FP64 kept for the inverse Slater matrices (updates and periodic
 * recomputation), weights and reconfiguration; its results are not
 * FP64-parity results but statistically equivalent ones. Takes effect at
 * the next lrdmc_step / lrdmc_evaluate call. */
#define LRDMC_PRECISION_FP64 0
#define LRDMC_PRECISION_DF64 1
#define LRDMC_PRECISION_FP32 2
LRDMC_API lrdmc_status lrdmc_set_precision(lrdmc_system_t sys, int precision);

/* Kernel timing for measurement. With profiling on, lrdmc_step brackets
 * every launch of its interval kernel and of its reconfiguration kernel
 * with CUDA events on the system's stream and accumulates their durations
 * (read after the step's final synchronisation). lrdmc_kernel_times returns
 * the accumulated milliseconds and launch counts (each nullable) and, if
 * reset != 0, clears them. Profiling is off after init. */
LRDMC_API lrdmc_status lrdmc_set_profiling(lrdmc_system_t sys, int on);
LRDMC_API lrdmc_status lrdmc_kernel_times(lrdmc_system_t sys, double* interval_ms, double* reconfig_ms,
                                          long long* interval_launches, long long* reconfig_launches,
                                          int reset);

/* -------------------------------------------------------------------------
 * Neural pair term of the Jastrow factor. The paper's guiding functions are
 * fixed (JSD/JAGP); this term is an addition that leaves the lattice method
 * itself unchanged, because the lattice Laplacian needs only values of
 * psi_G at the displaced points:
 *   J_NN(x) = sum_{i<j} g_{c(i,j)}(r_ij) + sum_{i,I} g_{2+species[I]}(r_iI),
 * channel c = 0 for equal-spin electron pairs, 1 for opposite spins,
 * 2 + s for an electron with a nucleus of species s;
 *   g_c(r) = m(r, c) s(r / r_cut[c]),  s(t) = 1 - 10t^3 + 15t^4 - 6t^5 (t < 1), 0 beyond,
 *   m = w3 . silu(W2 silu(W1 z + b1) + b2) + b3,
 *   z = [r^2 / (r^2 + ell_k^2) for k < n_feat, one-hot(c)].
 * Every feature is flat at r = 0 and s'(0) = 0, so g'(0) = 0: the Pade
 * factor keeps the cusp conditions. Parameters are one float32 vector,
 * row-major: W1 [hidden][n_feat + n_ch], b1 [hidden], W2 [hidden][hidden],
 * b2 [hidden], w3 [hidden], b3 [1]. With bf16 = 1 every parameter enters
 * as its bfloat16 rounding (to nearest, ties to even).
 * ---------------------------------------------------------------------- */
#define LRDMC_NJ_MAX_CH 8
#define LRDMC_NJ_MAX_FEAT 12
#define LRDMC_NJ_HIDDEN 64
#define LRDMC_NJ_MAX_CELLS 8192
typedef struct {
  int n_feat;           /* 1..LRDMC_NJ_MAX_FEAT                          */
  const double* ell;    /* [n_feat] feature lengths (bohr, > 0)          */
  int n_ch;             /* 2 + number of nucleus species, <= LRDMC_NJ_MAX_CH */
  const double* r_cut;  /* [n_ch] cut-off radius per channel (bohr, > 0) */
  const int* species;   /* [n_nuc] species of every nucleus, 0..n_ch-3   */
  int hidden;           /* must equal LRDMC_NJ_HIDDEN                    */
  int bf16;             /* 1: bfloat16-rounded parameters                */
  int n_cells;          /* table cells per channel, 1..LRDMC_NJ_MAX_CELLS */
} lrdmc_nj_spec;

/* Number of parameters of a spec (0 for an invalid spec). */
LRDMC_API int lrdmc_nj_n_params(const lrdmc_nj_spec* spec);

/* Installs the term in the projection and in every evaluation (params:
 * host float32, copied); spec = NULL removes it. The projection uses the
 * quintic Hermite interpolant of each g_c on the nodes r_k = r_cut (k/n)^2,
 * k = 0..n (n = n_cells): the node values g, g', g'' are computed here, in
 * IEEE double, from the parameters, and each cell holds the degree-5
 * polynomial that matches them at both ends, so the term is twice
 * continuously differentiable and the local energy stays continuous.
 * Host work plus one upload of 128 n_ch n_cells bytes; synchronous. Takes
 * effect at the next step or evaluation (a cached evaluation of the
 * population is recomputed). */
LRDMC_API lrdmc_status lrdmc_set_neural_jastrow(lrdmc_system_t sys, const lrdmc_nj_spec* spec,
                                                const float* params);

/* Base terms of the variance objective, in IEEE double: for every
 * configuration x [n][N][3] (device), grad_out [n][N][3] = grad_i log|psi_G|
 * and e_out [n] = E_L of the trial function WITHOUT the neural term
 * (whether or not one is installed). Device outputs; synchronises the
 * stream; LRDMC_ERR_SINGULAR for a singular configuration. */
LRDMC_API lrdmc_status lrdmc_base_terms(lrdmc_system_t sys, int n, const double* x, double* grad_out,
                                        double* e_out, void* stream);

/* Training forward pass, FP32 arithmetic, the network's exact radial
 * derivatives (no table). For every configuration x [n][N][3] with base
 * terms grad_base [n][N][3], e_base [n] (from lrdmc_base_terms):
 *   E_L = e_base - 1/2 sum_i [2 a_i . G_i + |G_i|^2 + L_i],  J = J_NN(x),
 * a_i = grad_base_i, G_i = grad_i J_NN, L_i = lap_i J_NN. Writes el_out [n],
 * j_out [n] and q_out [n][N][3] = a + G (float32; lrdmc_nj_backward reads
 * it) and pair_out [n][n_pairs][3] = g, g', g'' of every pair
 * (n_pairs = N(N-1)/2 + N n_nuc, electron pairs i < j first, row-major,
 * then electron-nucleus pairs i-major). params: device float32. All
 * pointers device; asynchronous on stream. */
LRDMC_API lrdmc_status lrdmc_nj_forward(lrdmc_system_t sys, const lrdmc_nj_spec* spec, const float* params,
                                        int n, const double* x, const double* grad_base,
                                        const double* e_base, float* el_out, float* j_out, float* q_out,
                                        float* pair_out, void* stream);

/* Training backward pass: grad_out (float32 [n_params], overwritten) =
 * d/dparams of sum_x (d_el[x] E_L(x) + d_j[x] J(x)), from the q of the
 * matching forward call; derivatives are taken with respect to the values
 * the network computes with (the bfloat16 roundings when spec->bf16).
 * Every sum runs in a fixed order, so equal inputs give the same bits.
 * The per-block partial sums go to device scratch the system owns (grid
 * size x n_params floats, allocated at the first call, grown if needed,
 * freed by lrdmc_destroy): backward calls on one system must not run
 * concurrently. All pointers device; asynchronous on stream. */
LRDMC_API lrdmc_status lrdmc_nj_backward(lrdmc_system_t sys, const lrdmc_nj_spec* spec, const float* params,
                                         int n, const double* x, const float* q, const float* d_el,
                                         const float* d_j, float* grad_out, void* stream);

/* -------------------------------------------------------------------------
 * Persistent grid size and batches of systems.
 *
 * The interval kernel runs a persistent grid whose warps fetch walkers
 * through an atomic counter. By default the grid holds as many blocks as fit
 * on the GPU for the system's shared-memory footprint;
 * lrdmc_set_interval_blocks overrides that (0 restores the default) and
 * lrdmc_interval_blocks reports the current and default sizes. The grid
 * size never changes results, only how the GPU is shared.
 * ---------------------------------------------------------------------- */
LRDMC_API lrdmc_status lrdmc_set_interval_blocks(lrdmc_system_t sys, int blocks);
LRDMC_API lrdmc_status lrdmc_interval_blocks(lrdmc_system_t sys, int* current, int* occupancy_default);

/* Tail helpers (on = 1, the default; 0 = off). Not a step of the paper's
 * method: a schedule of the interval kernel. Jump counts per interval are
 * Poisson-distributed, so near the end of an interval most warps have no
 * walker left while a few still run one. With helpers on, a warp whose
 * fetch finds no walker takes chunks of the lattice moves of a walker that
 * another warp of its block still runs; blocks hold up to 16 warps (one per
 * SM), fewer for small populations. Double-float and FP32 evaluation; the
 * FP64 mode runs every warp alone. The rates, and so every result, are bit
 * for bit the same either way. Every wait between warps is bounded; one
 * that runs out is reported as LRDMC_ERR_TIMEOUT. Takes effect at the next
 * step. */
LRDMC_API lrdmc_status lrdmc_set_tail_helpers(lrdmc_system_t sys, int on);

/* A batch projects several systems (different atoms, electron counts and
 * spacings) together. Every step is one CUDA graph: per execution group
 * (lrdmc_batch_set_groups) a fork, then per system of the group on its own
 * stream its interval kernel, its reconfiguration kernel and the copy of
 * its error word, then a join. The systems' persistent grids run
 * concurrently and share the GPU in proportion to their grid sizes. Graphs
 * are captured on first use (one per parity of the double-buffered
 * populations) and captured again when a system's kernel arguments change
 * (precision, neural term, grid size, init, load). Each system keeps its
 * own population, trace and results: a batched step gives bit for bit the
 * results of the same step made with lrdmc_step. n_systems <= 64; every
 * system must have a population; a[i] and spacing[i] are system i's
 * lattice. The batch borrows the systems (destroy it first); its streams
 * are its own, and each system's stream waits for the batch after every
 * batch_step. Asynchronous; lrdmc_batch_sync waits and reports the first
 * system error. */
typedef struct lrdmc_batch_s* lrdmc_batch_t;
LRDMC_API lrdmc_status lrdmc_batch_create(lrdmc_system_t* systems, int n_systems, const double* a,
                                          const lrdmc_spacing_fn* spacing, lrdmc_batch_t* out);
LRDMC_API lrdmc_status lrdmc_batch_step(lrdmc_batch_t batch, int n_steps);
LRDMC_API lrdmc_status lrdmc_batch_sync(lrdmc_batch_t batch);
/* Execution groups: group[i] >= 0 for every system; the systems of one
 * group run concurrently and the groups run one after another in
 * increasing group number, all inside the step's graph (default: one
 * group). Takes effect at the next batch_step (the graphs are captured
 * again). Results do not depend on the grouping. */
LRDMC_API lrdmc_status lrdmc_batch_set_groups(lrdmc_batch_t batch, const int* group);
/* Preferred shared-memory share (percent of the unified L1/shared storage,
 * 0..100, or -1 for the driver's default) of the batched interval launches:
 * kernels of different systems on one SM run together only under one
 * L1/shared split. A launch attribute of the batch's launches; lrdmc_step
 * is unaffected. Takes effect at the next batch_step. */
LRDMC_API lrdmc_status lrdmc_batch_set_carveout(lrdmc_batch_t batch, int carveout);
/* Pipelined schedule (on = 1; 0, the default, is the fork/join schedule
 * above). Every system's interval kernel runs on the batch stream in group
 * order (systems of equal group in index order), each after the first
 * launched with programmatic stream serialization: its blocks start on the
 * SMs that the previous system's blocks free once its walker queue is
 * empty, so one system's end-of-interval tail overlaps the next system's
 * start; the reconfiguration kernels follow the chain. Results do not
 * depend on the schedule. Takes effect at the next batch_step. */
LRDMC_API lrdmc_status lrdmc_batch_set_pipelined(lrdmc_batch_t batch, int on);
/* The batch's own stream (a cudaStream_t), for timing with events. */
LRDMC_API lrdmc_status lrdmc_batch_stream(lrdmc_batch_t batch, void** stream);
LRDMC_API const char* lrdmc_batch_last_error(lrdmc_batch_t batch);
LRDMC_API void lrdmc_batch_destroy(lrdmc_batch_t batch);

/* Last error message of the system (static string if sys is NULL). */
LRDMC_API const char* lrdmc_last_error(lrdmc_system_t sys);

/* Build flags of this library: LRDMC_BUILD_BOUNDS when it was compiled
 * with -DLRDMC_BOUNDS. In that build every walker-level index the kernels
 * read from device memory or derive from it (processing order, comb
 * parents and order positions, trace slots, helper teams) is checked
 * against its array; an index out of range sets a device error word and is
 * replaced by 0, so the access stays in bounds, and the next
 * synchronising call (lrdmc_sync) fails with LRDMC_ERR_BOUNDS. Results are
 * otherwise the default build's. Needs no GPU; never fails. */
LRDMC_API int lrdmc_build_flags(void);

/* Releases the system (not the caller's workspace or stream). */
LRDMC_API void lrdmc_destroy(lrdmc_system_t sys);

#ifdef __cplusplus
}
#endif
#endif /* LRDMC_H */
