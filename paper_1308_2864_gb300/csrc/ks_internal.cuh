// Internal declarations shared by the translation units of the library.
#pragma once

#include <initializer_list>
#include <cuda_runtime.h>
#include <cstddef>
#include <array>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "ks.h"

namespace ks {

// ---------------------------------------------------------------- errors
ks_status set_error(ks_status st, const char *fmt, ...);
ks_status cuda_error(cudaError_t e, const char *where);

#define KS_CUDA_TRY(call)                                              \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return ::ks::cuda_error(e_, #call);         \
  } while (0)

#define KS_TRY(call)                                                   \
  do {                                                                 \
    ks_status s_ = (call);                                             \
    if (s_ != KS_OK) return s_;                                        \
  } while (0)

// Device status word values beyond ks_status (bit flags are not used: the
// first error wins).
constexpr int kDevOk = 0;

// Spin limit of every device-side wait (about a second with the back-off
// used); after it the waiting block records KS_ETIMEOUT and returns.
// FP32 phase: iterations without a 0.1 % improvement of the best ||D||_M
// after which the phase ends (its rounding floor reached).
constexpr int kStallWindow = 500;
constexpr long long kSpinLimit = 1LL << 22;

// ---------------------------------------------------------------- grid
// Workspace of the software grid barrier used by cooperative kernels.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// Launch geometry of the cooperative CG kernel.
constexpr int kCgThreads = 256;

// Threads of generic one-dimensional kernels.
constexpr int kThreads = 256;

// Gram / update tiles (FP64): 64 x 64 output tile, 256 threads, 4 x 4 each.
constexpr int kTile = 64;
constexpr int kTileK = 16;

// ---------------------------------------------------------------- state
// Scalars kept on the device (indices into Problem::scal).
enum Scalar : int {
  SC_EKIN = 0,     // (f/2) sum X . KX
  SC_EEXT,         // h^3 sum Vext rho
  SC_EH,           // variational Hartree energy
  SC_EXC,          // h^3 sum rho eps_xc
  SC_ETF,          // h^3 sum C_TF rho^(5/3) (orbital-free model; follows SC_EXC)
  SC_EII,          // ion-ion energy
  SC_DNORM2,       // ||D||_M^2
  SC_BB_SS,        // tr(dX^T M dX)
  SC_BB_SY,        // tr(dX^T M dD)
  SC_BB_YY,        // tr(dD^T M dD)
  SC_ORTHO,        // ||X^T M X - I||_F^2
  SC_CG_ITERS,     // iterations of the last CG solve (as double)
  SC_COUNT = 16
};

struct Problem {
  // geometry and sizes
  int N = 0, n = 0, p = 0, natoms = 0, xc = 0;
  double L = 0, h = 0, rc = 0, occ = 0, cg_tol = 0;
  // kinetic model: kin_w multiplies (occ/2) tr(X^T K X) (1, or mu of the
  // TFW functional); ctf is the Thomas-Fermi constant (0 for orbitals)
  int kinetic = KS_KIN_ORBITALS;
  double kin_w = 1.0, ctf = 0.0;
  int mass = KS_MASS_CONSISTENT;     // KS_MASS_LUMPED: M = h^3 I
  double cg_tol_phase = 0;         // > 0: Hartree tolerance of the running FP32 phase
  int cg_maxit = 0;
  std::vector<double> atoms_host;  // natoms x 4: x, y, z, Z
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sms = 0;
  int cg_blocks = 0;               // cooperative grid of the CG kernel

  // n-vectors
  double *vext = nullptr, *rho = nullptr, *vH = nullptr, *veff = nullptr;
  double *rho_b = nullptr;         // density of the base X_b (FP32 phase, increment form)
  double *veff_b = nullptr;        // V_eff at the base X_b
  double *zero_n = nullptr;        // n zeros (V_eff = 0: the kinetic part f K X alone)
  double *cg_r = nullptr, *cg_pa = nullptr, *cg_pb = nullptr, *cg_q = nullptr;
  double *cg_z = nullptr;          // preconditioned residual
  double *cg_rho_prev = nullptr;   // density of the last Hartree solve (its right-hand side)
  bool cg_inc_ok = false;          // cg_r = b_last - K vH: the next warm solve needs no stencil
  int cg_inc_count = 0;            // incremental starts since the last full residual
  float *cg_t1 = nullptr, *cg_t2 = nullptr;  // sine-transform work (FP32)
  float *dst_phi = nullptr, *dst_kap = nullptr, *dst_mu = nullptr;
  int cg_precond = 1;
  int use_tc = 1;                  // FP32-phase tensor cores: 0 never, 1 for wide products, 2 always
  int use_oz = 0;                  // FP64 Grams on the tensor cores by digit splitting: 0 never,
                                   // 1 when both sides have >= 48 columns, 2 always
  int *oz_emax = nullptr;          // column exponents of the split operands
  unsigned char *oz_img = nullptr; // split coefficients of the FP64 tensor-core update
  int *oz_rowexp = nullptr;        // row exponents of the update's A (n)
  int oz_emax_len = 0;
  int use_tma = 1;                 // TMA plane staging in the stencils (when the layout allows)
  bool vH_valid = false;           // warm start available
  int rho_block = -1;              // block whose iterate's density P.rho already holds (-1: none)

  // n x p blocks (FP64 capacity plus 256 bytes; the FP32 phase keeps a second
  // FP32 block in the upper half, at byte offset half_off, 256-byte aligned)
  static constexpr int kNBlocks = 13;
  double *blk[kNBlocks] = {};
  size_t half_off = 0;

  // p x p work (all FP64)
  double *pp = nullptr;            // pool of small matrices
  float *cf = nullptr;             // 3 p^2: FP32 copies of the update coefficients
  float *rt32 = nullptr;           // 2 p^2: FP32 copies of D^T M D and X^T M D (increment form)
  float *tc_img = nullptr;         // coefficient image of the tensor-core update
  size_t tc_img_len = 0;
  size_t pp_len = 0;

  // reductions
  double *partials = nullptr;      // Gram partial tiles and block partial sums
  size_t partials_len = 0;
  double *scal = nullptr;          // device scalars (SC_*)
  double *scal_host = nullptr;     // pinned mirror
  double *atoms_dev = nullptr;
  double *thomas_w = nullptr;      // N pivots of the 1-D mass solve
  GridBarrier *bar = nullptr;
  unsigned int *red_counter = nullptr;  // last-block reduction counter (rests at 0)
  int *dstatus = nullptr;          // device status word
  int *dstatus_host = nullptr;     // pinned mirror

  // State of the last ConOptM phase (for ks_state_save / resume): slot
  // indices of the current/previous/trial blocks and the line-search scalars.
  struct RunState {
    bool valid = false;
    int elem = 8;                  // bytes per element of the phase's blocks
    int retraction = 0;
    int first_k = 0, k = 0;        // iteration offset of the phase, iterations in it
    int have_prev = 0;
    double C = 0, Q = 1, E = 0, dnorm2 = 0, ss = 0, sy = 0, yy = 0, best = 0;
    double last_tau = 0;           // last accepted step (carried into the FP64 polish)
    int last_improve = 0;
    int ix[3] = {0, 1, 2}, imx[3] = {3, 4, 5}, iex[2] = {6, 7}, id[2] = {9, 10}, imd[2] = {11, 12};
    // FP32 phase in increment form: X = X_b + delta, with the base's kinetic
    // energy T_b (the base blocks live in the upper halves of B_MX0..2)
    int split = 0;
    int since_rebase = 0;          // accepted iterations since the base was refreshed
    double T_b = 0;
  } state;

  // last mixed-precision phase
  int mixed_iters = 0;
  double mixed_dnorm = 0, mixed_E = 0;

  // last evaluation
  double last_parts[5] = {0, 0, 0, 0, 0};
  double last_E = 0;
  int last_cg_iters = 0;

  size_t bytes = 0;
};

size_t problem_bytes(int N, int p, int sms);
// Checks every field of a problem description on the host (no device call);
// KS_EINVAL with the reason recorded, else KS_OK.
ks_status validate_desc(const ks_problem_desc *d);

// ---------------------------------------------------------------- profiling
enum ProfClass : int {
  KP_DENSITY = 0, KP_CG, KP_POTENTIAL, KP_HAMILTONIAN, KP_MASS, KP_MASS_INV,
  KP_GRAM, KP_COMBINE, KP_SMALL, KP_REDUCE, KP_SETUP, KP_OTHER
};
// Counts `nlaunch` kernel launches and, when timing is on, brackets the
// scope's launches with CUDA events on `s`.
// `flops` and `bytes` are the algorithmic work of the launch (minimal
// arithmetic and DRAM traffic), summed per class while timing is on.
struct ProfScope {
  ProfScope(cudaStream_t s, int cls, double flops = 0.0, double bytes = 0.0, int nlaunch = 1);
  ~ProfScope();
  cudaStream_t stream;
  int cls;
  void *a;
};
// Accumulate the timings of completed launches (call after a stream sync).
void prof_collect();
// Per-launch timing switched on (no graph capture while it is).
bool prof_enabled();
// Adjust the launch counter (graph replays add their kernels; a capture
// removes the launches it recorded, which did not run).
void count_launches(long long delta);

// ---------------------------------------------------------------- kernels
// ks_setup.cu
ks_status launch_setup(Problem &P);
// ks_density.cu: rho_k = f sum_i X_ki^2 (X FP64 or FP32, rho FP64)
template <typename T>
ks_status launch_density(Problem &P, const T *X, double *rho);
// Increment form: rho = rho_b + f sum_i d_i (2 xb_i + d_i) (d, xb FP32 n x p)
ks_status launch_density_inc(Problem &P, const float *d, const float *xb, const double *rho_b,
                             double *rho);
// ks_split.cu: elementwise kernels of the increment form (n x p blocks)
// out = (hi + lo) + d in FP64
ks_status launch_split_join(Problem &P, const float *hi, const float *lo, const float *d,
                            double *out);
// hi = fl32(x), lo = fl32(x - hi)
ks_status launch_split_hilo(Problem &P, const double *x, float *hi, float *lo);
// out = a + s b (FP32)
ks_status launch_axpy_f32(Problem &P, const float *a, float s, const float *b, float *out);
// x += d (x FP64, d FP32)
ks_status launch_add_f64_f32(Problem &P, double *x, const float *d);
// out = A + s I (p x p); out may be A
ks_status launch_add_identity(Problem &P, const double *A, double s, double *out);
// C = alpha op(A) op(B) + beta C (p x p FP64, op = transpose when the flag is set;
// C must not alias A or B)
ks_status launch_small_gemm(Problem &P, int ta, const double *A, int tb, const double *B,
                            double alpha, double beta, double *C);
// out = A + s B (p x p; out may be A or B)
ks_status launch_add_pp(Problem &P, const double *A, double s, const double *B, double *out);
// out = X + Y + Y^T (p x p; out must not alias Y)
ks_status launch_sym_add(Problem &P, const double *X, const double *Y, double *out);
// out = R - (T + T^T) / tau (p x p)
ks_status launch_qr_exact_gram(Problem &P, const double *R, const double *T, double tau,
                               double *out);
// ks_cg.cu: K v = 4 pi h^3 rho; v in/out (warm if warm), r out
ks_status launch_cg(Problem &P, const double *rho, double *v, double *r, bool warm);
ks_status launch_sine_setup(Problem &P);
int cg_grid_blocks(int sms, int n, int N);
ks_status launch_gram_oz(Problem &P, const double *A, int pa, const double *B, int qb,
                         int *emax, double *part, int chunks);
int gram_oz_chunks(const Problem &P, int pa, int qb);
size_t oz_image_bytes(int p);
bool combine_oz_applies(const Problem &P, int k1, int k2, int q);
ks_status launch_combine_oz(Problem &P, const double *A1, int k1, const double *C1,
                            const double *A2, int k2, const double *C2, double alpha, double beta,
                            const double *Bm, double *out, int q);
size_t cg_dynamic_smem(int N);
// ks_xc.cu: veff = vext + vH + v_xc(rho); energy partials; reduction helpers
ks_status launch_potential(Problem &P, const double *rho, const double *vH, const double *r,
                           double *veff, bool with_hartree, bool fp32_xc = false);
ks_status launch_reduce(Problem &P, const double *partials, int nchan, int nb, double *out,
                        double scale = 1.0);
// Blocks of the grid-stride reduction kernels (their partials are nchan x this).
int reduce_blocks(const Problem &P, long long work);
// ks_stencil.cu (T = double or float; sums always returned in FP64)
template <typename T>
ks_status launch_hamiltonian(Problem &P, const T *X, const double *veff, T *EX, T *MX,
                             double *ekin_out);
template <typename T>
ks_status launch_mass(Problem &P, const T *X, T *MX);
// Increment form (FP32 phase with X = X_b + d): the change of the gradient
// from the base, e = f K d + 2 f h^3 (Diag(veff - veff_b) xb + Diag(veff) d),
// Md = M d (may be null), and the kinetic energy change from the base,
// sum d . (f K X_b + (f/2) K d) with f K X_b = eb - 2 f h^3 veff_b xb, into
// *dkin_out.  xb = fl32(X_b), eb = fl32(E_X at X_b with veff_b) (f = occ, or
// mu occ for TFW).
ks_status launch_hamiltonian_inc(Problem &P, const float *d, const double *veff,
                                 const double *veff_b, const float *xb, const float *eb,
                                 float *e, float *Md, double *dkin_out);
// MD = M D; dnorm2 = sum D.MD; with prev != null also the BB traces.
template <typename T>
struct BBPrevT { const T *X, *MX, *D, *MD; };
template <typename T>
ks_status launch_mass_dots(Problem &P, const T *D, T *MD, const T *X, const T *MX,
                           const BBPrevT<T> *prev, double *out4);
// ks_minv.cu: G = M^{-1} E (+ add, folded into the last sweep, when given)
template <typename T>
ks_status launch_mass_inverse(Problem &P, const T *E, T *G, const T *add = nullptr);
// ks_blas.cu
// out (pa x qb, FP64) = A^T B with A n x pa, B n x qb (row-major, ld = pa, qb)
template <typename T>
ks_status launch_gram(Problem &P, const T *A, int pa, const T *B, int qb, double *out);
// FP32: out = A1^T B1 + A2^T B2 (one pass when the pipelined kernel applies;
// otherwise two Grams, tmp a p x p scratch matrix)
ks_status launch_gram_pair(Problem &P, const float *A1, const float *B1, const float *A2,
                           const float *B2, int pa, int qb, double *out, double *tmp);
// FP32: out1 = A1^T B, out2 = A2^T B (B read once when the kernel applies);
// out32 (optional, 2 pa qb floats): FP32 copies of out1 then out2
ks_status launch_gram_dual(Problem &P, const float *A1, const float *A2, const float *B, int pa,
                           int qb, double *out1, double *out2, float *out32 = nullptr);
// out (n x q) = alpha (A1 C1 + A2 C2) + beta Bm (A2/Bm may be null);
// C1 k1 x q, C2 k2 x q (FP64).  out must not alias A1, A2 or Bm.
template <typename T>
ks_status launch_combine(Problem &P, const T *A1, int k1, const double *C1, const T *A2, int k2,
                         const double *C2, double alpha, double beta, const T *Bm, T *out, int q);
// Function attributes of the update kernels (once per problem creation).
ks_status configure_blas_kernels();
// out = A1 C1 + A2 C2 + A3 C3 and out2 = add2 + out (FP32 n x q, q <= 64,
// k1 + k2 + k3 <= 192, C FP64) in one pass; combine3_f32_applies says when.
// With rho set (q = p; out the increment delta, add2 the base X_b) the same
// pass writes rho = rho_b + f sum delta (2 X_b + delta) of X_b + delta.
bool combine3_f32_applies(const Problem &P, int k1, int k2, int k3, int q);
ks_status launch_combine3_f32(Problem &P, const float *A1, int k1, const double *C1,
                              const float *A2, int k2, const double *C2, const float *A3, int k3,
                              const double *C3, float *out, const float *add2, float *out2, int q,
                              const double *rho_b = nullptr, double *rho = nullptr,
                              bool images_ready = false);
// Increment form, QR step: from FP32 copies of R = D^T M D and T = X^T M D
// (rt32: R then T, p x p each) the factor L L^T = I - tau (T + T^T) +
// tau^2 R as deviations from I in FP32; writes the FP32 coefficients
// [L^{-T} - I; L^{-T}; -tau L^{-T}] of launch_combine3_f32 to P.cf
// (images_ready).
bool qr_factor_dev_applies(const Problem &P);
ks_status launch_qr_factor_dev(Problem &P, const float *rt32, double tau);
// elementwise precision conversion of an n x p block
ks_status launch_convert(Problem &P, const double *in, float *out);
ks_status launch_convert(Problem &P, const float *in, double *out);
// sum of squares of (O - I) for a p x p O
ks_status launch_ortho_err(Problem &P, const double *O, double *out);
// ks_small.cu: small dense FP64 algebra in one CTA
// QR step: R = I + tau^2 DMD (or R = O when DMD is null); L L^T = R;
// C = L^{-T}; writes C1 = C and C2 = -tau C.
ks_status launch_qr_factor(Problem &P, const double *DMD, const double *O, double tau,
                           double *C1, double *C2);
// Cayley step: builds N = [[A, O], [-B, -S]], solves (I + tau/2 N) P = [O; -S]
// and writes C1 = I - tau P2 (p x p), C2 = -tau P1 (p x p), both for
// X+ = X C1 + G C2.  A = X^T E_X, S = E_X^T X, B = E_X^T G, O = X^T M X.
ks_status launch_cayley_factor(Problem &P, const double *A, const double *S, const double *B,
                               const double *O, double tau, double *C1, double *C2);
// Function attributes of the small kernels (once per problem creation).
ks_status configure_small_kernels();
// ks_tc.cu: FP32 Gram on the tensor cores (partials per chunk, FP64)
ks_status configure_tc_kernels();
// Narrow updates (q <= 64, K <= 192) on the tensor cores (three TF32
// products per term, ks_set_tensor_cores mode 3): out = s1 A1 C1 + s2 A2 C2
// + s3 A3 C3 with FP32 coefficient matrices (k_i x q, row-major; a null C_i
// is the identity, so a whole matrix can be added), out2 = A3 + out (k3 = q,
// each operand's columns in whole stages of 32) and, with rho, the
// increment-form density rho = rho_b + f sum out (2 A3 + out).  applies:
// mode, q, the operand widths ks (multiples of 4, at most 6 stages of 32
// in all) and 16-byte alignment of ptrs.
bool combine_tc64_applies(const Problem &P, int q, std::initializer_list<int> ks,
                          std::initializer_list<const void *> ptrs);
ks_status launch_combine_tc64(Problem &P, int q, const float *A1, int k1, const float *C1,
                              float s1, const float *A2, int k2, const float *C2, float s2,
                              const float *A3, int k3, const float *C3, float s3, float *out,
                              float *out2, const double *rho_b, double *rho);
size_t tc_image_floats(int p);
int gram_tc_chunks(const Problem &P, int pa, int qb);
ks_status launch_gram_tc(Problem &P, const float *A, int pa, const float *B, int qb,
                         double *part, int chunks);
ks_status launch_combine_tc(Problem &P, const float *A1, int k1, const double *C1,
                            const float *A2, int k2, const double *C2, double alpha, double beta,
                            const float *Bm, float *out, int q);
// Transpose a p x p matrix into out.
ks_status launch_transpose(Problem &P, const double *A, double *out);

// Index of the n x p blocks in Problem::blk.
enum Block { B_X0 = 0, B_X1, B_X2, B_MX0, B_MX1, B_MX2, B_EX0, B_EX1, B_G, B_D0, B_D1, B_MD0, B_MD1 };

// Offsets (in units of p*p) of the small matrices in the pp pool; the first
// 6 p^2 are scratch of the factor kernels.
// S_XMD .. S_DS: the FP32 phase in increment form (X^T M D, work, S_b and
// S - S_b).
enum Small { S_WORK = 0, S_S = 6, S_DMD, S_O, S_A, S_B, S_C1, S_C2, S_T, S_XMD, S_E1, S_E2, S_E3,
             S_SB, S_DS, S_COUNT };

// Slack of the Armijo test for the rounding of the energy sums: in the FP64
// phase a trial is not rejected for a rise below 4 eps sum |E_parts| (near
// convergence the required decrease rho1 tau ||D||^2 falls below the
// rounding of E, and an exact-arithmetic test would backtrack at random);
// the FP32 phase keeps the strict test, so that it stalls and hands over.
template <typename T>
inline double armijo_slack(const double *parts) {
  if (sizeof(T) != 8) return 0.0;
  double a = 0.0;
  for (int i = 0; i < 5; ++i) a += parts[i] < 0 ? -parts[i] : parts[i];
  return 4.0 * 2.220446049250313e-16 * a;
}

// ---------------------------------------------------------------- batch
// A job table of independent systems advanced together (ks_batch_*): every
// launch of a step covers all jobs whose active flag is set.  Each job keeps
// its buffers in its own Problem; BJob is the device-side view of them plus
// the job's launch geometry.
struct BJob {
  int N, p;
  long long n;
  double h, occ, h3, cg_tol;
  int xc, cg_maxit, cg_precond;
  void *blk[Problem::kNBlocks];
  double *vext, *rho, *vH, *veff, *cg_r;
  double *pp;                      // small matrices, same layout as Problem::pp
  float *cf;                       // FP32 copies of update coefficients (2 p^2)
  double *partials;
  unsigned int *red_counter;
  double *thomas_w;
  double *scal;                    // this job's row of the batch scalar table (SC_COUNT)
  int *status;                     // this job's entry of the batch status table
  double qc[8];                    // Q1 stencil classes k0, kf, ke, kc, m0, mf, me, mc
  float qcf[9];                    // k0, ke, kc, m0, mf, me, mc, occ, 2 occ h^3 in FP32
  int st_zseg, st_tiles_x, st_tiles_y, st_chunks, st_nb;   // stencil geometry (job's PC class)
  int pot_nb;                      // potential blocks (grid-stride)
  int gram_chunks;                 // row chunks of the Grams
  long long gram_rows_per;
  int comb_nb;                     // blocks of the narrow update
};

// Block maps of the batched launches: prefix sums over jobs of the blocks
// each job takes in a launch family.
enum BMap {
  BM_DENSITY = 0, BM_POTENTIAL, BM_ST4, BM_ST8, BM_ST16, BM_ST32, BM_THOMAS, BM_GRAM_SMALL,
  BM_GRAM_MID, BM_GRAM_TILED, BM_GRAM_REDUCE, BM_CG_NODES, BM_CG_PLANES, BM_COMB_NARROW, BM_COMB_TILED, BM_COEF, BM_COPY, BM_COUNT
};

// Launch shapes of the batched kernels that the autotuner chooses.
struct BatchTuning {
  int gram_rows = 4096;            // Gram rows per chunk (block)
  int comb_per_thread = 8;         // narrow update: outputs per thread
  int pot_per_thread = 4;          // potential: nodes per thread
  int st_planes = 0;               // stencil planes per block (0: default geometry)
};

struct Batch {
  int J = 0, sms = 0, maxN = 0, maxp = 0;
  BatchTuning tune;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<ks_problem *> probs;
  std::vector<BJob> jobs_host;
  BJob *jobs_dev = nullptr;
  int *maps_dev = nullptr;         // BM_COUNT x (J + 1)
  std::vector<int> maps_host;
  unsigned char *active_dev = nullptr, *active_host = nullptr;   // launch mask (pinned mirror)
  double *tau_dev = nullptr, *tau_host = nullptr;                // per-job step (pinned mirror)
  double *scal_dev = nullptr, *scal_host = nullptr;              // J x SC_COUNT
  int *status_dev = nullptr, *status_host = nullptr;             // J
  void *cg_args_dev = nullptr;     // J CgArgs (Hartree PCG of each job)
  void *cg_state_dev = nullptr;    // J per-job PCG scalars
  double *cg_tolw_dev = nullptr, *cg_tolw_host = nullptr;   // per job (tolerance, warm)
  unsigned int *cg_counters = nullptr;                      // per-job last-block counters
  int *cg_remaining_dev = nullptr, *cg_remaining_host = nullptr;
  std::vector<unsigned char> warm; // per job: a previous Hartree potential exists
  char *ring_host = nullptr;       // pinned staging ring of the small uploads
  size_t ring_bytes = 0, ring_used = 0;
  // CUDA graphs of the step sequences, keyed by sequence kind, precision and
  // block slots; value: executable graph and the kernel launches it holds
  bool use_graphs = true;
  std::map<std::array<int, 14>, std::pair<cudaGraphExec_t, long long>> graphs;
  size_t bytes = 0;
  const int *map(int m) const { return maps_dev + (size_t)m * (J + 1); }
  int total(int m) const { return maps_host[(size_t)m * (J + 1) + J]; }
};

// Device: the job whose block range [start[j], start[j+1]) holds block b.
__device__ __forceinline__ int batch_job_of(const int *start, int J, int b) {
  int lo = 0, hi = J;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Batched launches (slots index BJob::blk, -1 = none; sm* are offsets in
// units of p^2 into BJob::pp).  ks_density.cu, ks_cg.cu, ks_xc.cu,
// ks_stencil.cu, ks_minv.cu, ks_blas.cu, ks_small.cu.
template <typename T>
ks_status batch_density(Batch &B, int sX);
ks_status batch_cg(Batch &B, double tol);
ks_status batch_cg_upload(Batch &B, double tol);
ks_status batch_cg_launch(Batch &B, int iters);
ks_status batch_cg_continue(Batch &B);
ks_status batch_cg_setup(Batch &B);
ks_status batch_potential(Batch &B, bool fp32_xc);
template <typename T>
ks_status batch_hamiltonian(Batch &B, int sX, int sEX, int sMX);
template <typename T>
ks_status batch_mass(Batch &B, int sX, int sMX);
template <typename T>
ks_status batch_mass_dots(Batch &B, int sD, int sMD, int sX, int sMX, int sXp, int sMXp, int sDp,
                          int sMDp);
ks_status batch_stencil_geometry(Batch &B);
template <typename T>
ks_status batch_mass_inverse(Batch &B, int sE, int sG);
template <typename T>
ks_status batch_gram(Batch &B, int sA, int sB, int smOut);
template <typename T>
ks_status batch_combine(Batch &B, int sA1, int smC1, int sA2, int smC2, double alpha, double beta,
                        int sBm, int sOut);
template <typename Tin, typename Tout>
ks_status batch_convert(Batch &B, int sIn, int sOut);
ks_status batch_ortho_err(Batch &B, int smO);
ks_status batch_qr_factor(Batch &B, int smDMD, int smO, bool with_tau, int smC1, int smC2);

}  // namespace ks

struct ks_problem {
  ks::Problem P;
};
