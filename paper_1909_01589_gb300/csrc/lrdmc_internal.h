// Internal interface between the C-ABI host code (lrdmc_api.cu) and the
// CUDA kernels (lrdmc_kernels.cu). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/lrdmc.h"
#include "df64.cuh"

namespace lrdmc {

constexpr int kMaxNuc = LRDMC_MAX_NUC;
constexpr int kMaxShell = LRDMC_MAX_SHELL;
constexpr int kMaxPrim = LRDMC_MAX_PRIM;
constexpr int kMaxAO = LRDMC_MAX_AO;
constexpr int kMaxSpin = LRDMC_MAX_SPIN;
constexpr int kMaxMO = LRDMC_MAX_SPIN;
constexpr int kMaxNjCh = LRDMC_NJ_MAX_CH;
constexpr int kWarpsPerBlock = 4;
constexpr int kMaxItersPerInterval = 1 << 20;

// Error bits of the device error word.
constexpr int kErrSingular = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrIters = 4;
constexpr int kErrTimeout = 8;  // a bounded wait ran out (tail helpers of the interval kernel, tensor-core barrier)
constexpr int kErrBounds = 16;  // a checked index was out of range (bounds-checked builds only)

#ifdef LRDMC_BOUNDS
constexpr int kBuildFlags = LRDMC_BUILD_BOUNDS;
#else
constexpr int kBuildFlags = 0;
#endif

// The walker-level indices that the kernels read from device memory or
// derive from it (processing order, parents, comb order positions, trace
// slots, helper teams) pass through bounded(i, n, err). In a build with
// -DLRDMC_BOUNDS an index outside [0, n) sets kErrBounds in the error word
// and becomes 0, so the access stays inside its array and the host reports
// LRDMC_ERR_BOUNDS; in the default build it is the index unchanged.
template <class I>
__device__ __forceinline__ I bounded(I i, long long n, int* err)
{
#ifdef LRDMC_BOUNDS
  if ((unsigned long long)(long long)i >= (unsigned long long)n) {
    atomicOr(err, kErrBounds);
    return I(0);
  }
#else
  (void)n;
  (void)err;
#endif
  return i;
}

// Philox counter tags.
constexpr uint64_t kTagTimeHB = 0;
constexpr uint64_t kTagRot = 1;
constexpr uint64_t kTagComb = 2;
constexpr uint64_t kSlotGlobal = 0xFFFFFFFFFFFFFFFFull;
constexpr uint64_t kIntervalInit = 0xFFFFFFFFFFFFFFFFull;

struct ShellDev {
  int center, l, kind, n_prim;
  int ao_offset;
  int m_int;       // Slater power r^m as an integer (>= 0), or -1 for pow()
  int same_exp;    // 1: same centre and Slater exponent as the previous shell
  int pad;
  double m;        // n_eff - 1 - l
  double zeta;
  double alpha[kMaxPrim];
  double coef[kMaxPrim];
};

// Double-float copies of the constants the double-float evaluation reads
// (split on the host so that no kernel converts them on the FP64 pipe).
struct DfShell {
  df m, zeta;
  df alpha[kMaxPrim], coef[kMaxPrim];
};

struct DfSys {
  df nuc[kMaxNuc][3];
  df Z[kMaxNuc];
  df en_b1[kMaxNuc];
  df b_ee, c_par, c_anti, en_b2;
  DfShell sh[kMaxShell];
  ExpTable exp;
  df inv_fact[18];  // 1/k!, k = 0..17 (series of sin and cos)
  df half_pi;
};

// Trial function and Hamiltonian constants, passed by value as a kernel
// parameter (__grid_constant__); the MO coefficients are staged in shared
// memory by every block.
struct SysDev {
  int n_nuc, n_up, n_dn, N;
  int n_shell, n_ao, n_mo, ee_on;
  double nuc[kMaxNuc][3];
  double Z[kMaxNuc];
  double en_b1[kMaxNuc];
  int heavy[kMaxNuc];  // 1 for the nuclei with Z = Z_max (centres of p)
  int nuc_shell_begin[kMaxNuc + 1];  // shells are sorted by centre: [begin[I], begin[I+1])
  double b_ee, c_par, c_anti, en_b2;
  double V_nn;
  ShellDev sh[kMaxShell];
  // units of consecutive shells that the parts of an electron's local
  // energy deal out (unit g is shells [grp_first[g], grp_first[g + 1])):
  // every shell alone when there are no more shells than parts (each then
  // forms its own exponential), else groups sharing one Slater exponential
  // (a shell with same_exp joins the group of the shell before it)
  int n_grp;
  int grp_first[kMaxShell + 1];
  double C[kMaxAO * kMaxMO];  // [n_ao][n_mo]
  int precision;  // LRDMC_PRECISION_FP64 or LRDMC_PRECISION_DF64
  // neural pair term of the Jastrow factor, tabulated: channel c, cell k
  // (uniform in sqrt(r) on [0, r_cut_c)) holds r_k, 1/w_k and the
  // coefficients c_0..c_5 of g_c = sum_q c_q t^q, t = (r - r_k)/w_k
  int nj_on;
  int nj_cells;
  const double* nj_tab;   // [n_ch][nj_cells][8]
  const df* nj_tab_df;    // the same as double-floats
  double nj_rcut[kMaxNjCh];
  float nj_rcut_f[kMaxNjCh];
  float nj_scale_f[kMaxNjCh];  // nj_cells / sqrt(r_cut_c)
  int nj_species[kMaxNuc];     // e-n channel of nucleus I is 2 + nj_species[I]
  DfSys D;
};

struct LatDev {
  double a, ap;     // spacings a and a'
  double inv2a2;    // 1 / (2 a^2)
  double inv2ap2;   // 1 / (2 a'^2)
  double rc;        // r_c (Gaussian: length, Pade: inverse length)
  double p_coef;    // Gaussian: 1/(2 r_c^2); Pade: r_c^2
  int G;            // 1 single grid, 2 double grid
  int pkind;        // 0 Gaussian (Eq. 3), 1 Pade (Eq. 2)
  // the same values as double-floats
  df a_df, ap_df, inv2a2_df, inv2ap2_df, p_coef_df;
};

// Walker record layout (doubles) in the double-buffered population.
struct Layout {
  int N, nu, nd, P_max;
  int off_x, off_au, off_ad, off_R, off_T, off_b, off_el;
  int rec;  // doubles per record (multiple of 4)
  int head;       // doubles of shared memory per block before the warp regions
  int smem_warp;  // doubles of shared memory per warp
  int smem_block_bytes;
  int n_pc;       // electron pairs with a cached distance and projections (0: no cache)
  int pcw;        // double-floats per cached pair: 4 (distance, projections) or 8 (+ Jastrow pair terms)
  int enc;        // 1: the electron-nucleus cache (and the pair cache, if any) is in the layout
};

// Shared-memory layout of a system; caches = false leaves out the
// evaluation caches (for systems that would not fit otherwise).
Layout make_layout(const SysDev& S, bool caches);
// Largest dynamic shared memory of one block on sm_100-class GPUs (227 KB),
// less 2 KB for the kernels' static shared memory (the interval kernel's
// per-warp loop state and tail-helper slots, 1.7 KB).
constexpr int kMaxSmemBlock = 232448 - 2048;

// Populations up to this many walkers keep the comb's running sums in the
// shared memory of every block of the reconfiguration (8 bytes each).
constexpr int kReconfigSmemW = 16384;
// Reconfiguration grid: blocks of kCombThreads threads, each owning at
// least kCombThreads consecutive slots, at most kMaxCombBlocks blocks; the
// largest dynamic shared memory of its second kernel (the running sums of
// up to kReconfigSmemW walkers, or a float per slot of a block).
constexpr int kCombThreads = 256;
constexpr int kMaxCombBlocks = 128;
constexpr int kCombSmemMax = 200 * 1024;
// Largest population (the reconfiguration's per-block slots fit its shared
// memory with room to spare).
constexpr int kMaxWalkers = LRDMC_MAX_WALKERS;
int comb_blocks(int W);

// Totals of one block of the reconfiguration.
struct CombPart {
  double w;          // sum of the block's weights (its last running sum)
  double swe;        // sum of w E_L
  long long jumps;   // sum of jumps
};

struct PopDev {
  double* rec_src;
  double* rec_dst;
  int* parent;
  int* order;  // processing order of the slots (longest expected interval first)
  double* logw;
  double* wgt;  // exp(logw) of the last interval, written with logw
  double* el_end;
  int* jumps;
  double* cum;  // running weight sums of the comb, relative to the start of each reconfiguration block
  CombPart* part;       // [kMaxCombBlocks] totals of the reconfiguration blocks
  int* ticket;          // reconfiguration blocks finished (zero between reconfigurations)
  double* trace;  // [4][cap]: e_k, mean weight, mean jumps, Sherman-Morrison residual at the recompute
  // largest Sherman-Morrison residual of the current interval's recompute,
  // as the bits of a non-negative double (atomicMax orders them as doubles)
  unsigned long long* resid;
  unsigned long long* moves;
  int* err;
  int* counter;
  // interval counter k on the device: the interval kernel reads it (Philox
  // counters, the recompute decision), the reconfiguration kernel reads it
  // (comb uniform, trace slot) and advances it, so a captured step replays
  // correctly
  unsigned long long* kdev;
  int recompute_every;
  int W;
  int trace_cap;
  uint64_t seed;
  double tau, e_trial;
  // 1: in the FP32-pipe evaluations, warps of the interval kernel that run
  // out of walkers help the warps of their block that still run one
  int helpers;
};

void fill_df_constants(SysDev& S);
void fill_lattice_df(LatDev& L);

cudaError_t launch_init(const SysDev& S, const Layout& Lo, const PopDev& P, const double* x0,
                        cudaStream_t st);
cudaError_t launch_eval_all(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P,
                            cudaStream_t st);
// carveout: preferred shared-memory share of the L1/shared storage for this
// launch in percent (cudaLaunchAttributePreferredSharedMemoryCarveout), or
// -1 for the default; pdl: launch with programmatic stream serialization
// (may start while the previous kernel in the stream drains its walkers)
cudaError_t launch_interval(const SysDev& S, const Layout& Lo, const LatDev& L, const PopDev& P, int blocks,
                            cudaStream_t st, int carveout = -1, bool pdl = false);
cudaError_t launch_reconfig(const PopDev& P, const Layout& Lo, cudaStream_t st);
// Occupancy-default persistent grid of the interval kernel for a population
// of W walkers (blocks of interval_warps(S, Lo, W) warps).
int interval_default_blocks(const SysDev& S, const Layout& Lo, int W);
int interval_warps(const Layout& Lo, int W);
cudaError_t launch_evaluate(const SysDev& S, const Layout& Lo, const LatDev& L, int n,
                            const double* x, const double* rot, double* ratio, double* T,
                            double* b, double* el, int* err, cudaStream_t st);

// Neural pair term: geometry and network shape for the training kernels.
struct NjGeom {
  int N, n_up, n_nuc, n_pairs;  // n_pairs = N(N-1)/2 + N n_nuc
  double nuc[kMaxNuc][3];
  int species[kMaxNuc];
};
struct NjNetDev {
  int F, C, D, bf16;  // features, channels, F + C, bfloat16 parameters
  float ell2[LRDMC_NJ_MAX_FEAT];
  float rcut[kMaxNjCh];
};

int nj_n_params(int n_feat, int n_ch, int hidden);
float nj_bf16(float x);
void nj_build_table(const lrdmc_nj_spec& spec, const float* params, std::vector<double>& tab);
cudaError_t launch_nj_forward(const NjGeom& G, const NjNetDev& N, const float* params, int n, const double* x,
                              const double* grad_base, const double* e_base, float* el, float* j, float* q,
                              float* pair_out, cudaStream_t st);
// Grid size of the backward kernel (its per-block partial gradients need
// that many times n_params floats of scratch); -1 on a CUDA error.
int nj_backward_max_blocks(const NjGeom& G, const NjNetDev& N);
cudaError_t launch_nj_backward(const NjGeom& G, const NjNetDev& N, const float* params, int n, const double* x,
                               const float* q, const float* d_el, const float* d_j, float* grad, float* partials,
                               int max_blocks, cudaStream_t st);

cudaError_t launch_base_terms(const SysDev& S, const Layout& Lo, int n, const double* x, double* grad,
                              double* e, int* err, cudaStream_t st);

// Evaluation with the orbital contraction on the tensor cores (FP32 mode
// arithmetic; bf16x3 operands, FP32 accumulation in tensor memory); its
// shared memory per block, and the launch. err receives kErrSingular and
// kErrTimeout bits.
int evaluate_tc_smem_bytes(const SysDev& S, const Layout& Lo);
cudaError_t launch_evaluate_tc(const SysDev& S, const Layout& Lo, const LatDev& L, int n, const double* x,
                               const double* rot, double* ratio, double* T, double* b, double* el, int* err,
                               cudaStream_t st);

cudaError_t launch_evaluate_static(const SysDev& S, const Layout& Lo, const LatDev& L, int n,
                                   const double* x, const double* rot, double* ratio, double* T,
                                   double* b, double* el, int* summary, int* first_bad, cudaStream_t st);

}  // namespace lrdmc
