/*
 * ks.h -- C ABI of the GB300 library for direct Kohn-Sham energy
 * minimisation on the generalised Stiefel manifold X^T M X = I.
 *
 * Method: Zhang, Zhu, Wen, Zhou, "Gradient type optimization methods for
 * electronic structure calculations".  The problem is Eq. opt (minimise the
 * discretised KS energy subject to orthonormal orbitals, Sec. 3), with the
 * mass-matrix constraint of the finite-element model (Eq. disOFinf, handled
 * by the substitution y = B^{1/2} c of Eq. OFDFT-y).  The iteration is
 * Alg. ConOptM: projected gradient (Eq. def-nablaE), a Cholesky-QR
 * (Eq. QR, Alg. ChQR) or Cayley (Eq. WY3) retraction, Barzilai-Borwein steps
 * (Eq. bb-1) and the nonmonotone Armijo search (Eq. NMLS-Armijo).
 *
 * Discretisation: Q1 finite elements on a cube of side L with N interior
 * nodes per edge (h = L/(N+1)) and zero Dirichlet boundary values; stiffness
 * K and consistent mass M are the 27-point trilinear operators.  Orbitals
 * are stored row-major n x p (n = N^3, node index k = (iz*N + iy)*N + ix,
 * orbital index fastest), FP64, densely packed (leading dimension p).
 *
 * Conventions for every call:
 *   - the return value is a ks_status; no call aborts the process;
 *   - pointers documented as DEVICE point to memory of the current CUDA
 *     device that the caller owns; the library never frees them;
 *   - work is issued on the problem's stream; calls that return host values
 *     synchronise that stream before returning;
 *   - a problem object is not thread-safe and must be used from one host
 *     thread at a time;
 *   - on failure the caller's output buffers are left unchanged except where
 *     a call says otherwise, and ks_last_error_string() describes the error.
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KS_OK = 0,
  KS_EINVAL = 1,      /* invalid argument */
  KS_ENOMEM = 2,      /* device allocation failed */
  KS_ECUDA = 3,       /* CUDA runtime error */
  KS_ENOCONV = 4,     /* Hartree CG or the outer iteration hit its limit */
  KS_ENOTPD = 5,      /* Cholesky of a Gram matrix met a non-positive pivot */
  KS_ESINGULAR = 6,   /* the Cayley system I + tau/2 V^T U is singular */
  KS_ENAN = 7,        /* a non-finite value appeared */
  KS_ETIMEOUT = 8,    /* a bounded device-side wait gave up */
  KS_EAGAIN = 9       /* ks_server_poll: the job has not finished yet */
} ks_status;

/* Opaque problem handle; owns all device workspace of one system. */
typedef struct ks_problem ks_problem;

enum { KS_XC_SLATER = 0, KS_XC_SLATER_PZ81 = 1 };
enum { KS_FP64 = 0, KS_MIXED = 1 };
enum { KS_QR = 0, KS_CAYLEY = 1 };
enum { KS_KIN_ORBITALS = 0, KS_KIN_TFW = 1 };
enum { KS_MASS_CONSISTENT = 0, KS_MASS_LUMPED = 1 };

/* One discretised KS system (Eq. EKS discretised, Sec. 2.3). */
typedef struct {
  int N;              /* interior nodes per edge (2 .. 2048, with N^3 p <= 2^31 - 1) */
  double L;           /* cube side in bohr */
  int natoms;         /* number of pseudo-atoms (>= 0) */
  const double *R;    /* HOST, 3*natoms positions (x, y, z) in bohr; copied */
  const double *Z;    /* HOST, natoms valence charges; copied */
  double rc;          /* erf radius of -Z erf(r/rc)/r (0.5) */
  int p;              /* number of orbitals (>= 1) */
  double occ;         /* occupation per orbital (2) */
  int xc;             /* KS_XC_SLATER or KS_XC_SLATER_PZ81 */
  double cg_tol;      /* Hartree CG: ||r||_2 <= cg_tol ||b||_2 (1e-10) */
  int cg_maxit;       /* Hartree CG iteration limit */
  int precision;      /* KS_FP64 or KS_MIXED; informative only: the precision of a
                         minimisation is chosen by ks_opts.precision */
  void *stream;       /* cudaStream_t to issue work on; NULL = library-owned */
  int cg_precond;     /* 1: precondition the Hartree CG with the FP32 sine-basis inverse
                         of K (default); 0: plain CG */
  int kinetic;        /* KS_KIN_ORBITALS (0): the Kohn-Sham kinetic energy (occ/2) tr(X^T K X).
                         KS_KIN_TFW (1): the orbital-free model of Sec. 2.2 with the
                         Thomas-Fermi-von Weizsaecker functional of Eq. TFW; p must be 1,
                         X is the amplitude c with rho = occ c^2 (occ = the electron count),
                         c^T M c = 1 (Eq. disOFinf), and the kinetic energy is
                         mu (occ/2) c^T K c + h^3 sum C_TF rho^(5/3),
                         C_TF = (3/10) (3 pi^2)^(2/3) */
  double mu;          /* KS_KIN_TFW: weight of the von Weizsaecker term (>= 0; 1 = full) */
  int mass;           /* metric of the constraint X^T M X = I: KS_MASS_CONSISTENT (0), the Q1
                         mass matrix; KS_MASS_LUMPED (1), its row sums M = h^3 I, under which
                         the nodal density integrates to exactly occ * p electrons (the form
                         the orbital-free model needs: a consistent-mass amplitude that
                         oscillates node to node carries up to 27 times the electrons in the
                         nodal density).  The stiffness K is the Q1 one in both. */
} ks_problem_desc;

/* Parameters of Alg. ConOptM (the paper fixes none of their values). */
typedef struct {
  int retraction;     /* KS_QR or KS_CAYLEY (KS_QR) */
  double gtol;        /* stop when ||D||_M <= gtol (1e-6) */
  int maxit;          /* iteration limit (300) */
  double tau0;        /* first step and reset value (1e-3) */
  double rho1;        /* Armijo constant, < 1/2 (1e-4) */
  double delta;       /* backtracking factor (0.1) */
  double eta;         /* nonmonotone weight (0.85) */
  double tau_min;     /* BB clamp (1e-10) */
  double tau_max;     /* BB clamp (1e10) */
  int max_backtrack;  /* backtracks per iteration before accepting (10) */
  double ortho_tol;   /* re-orthonormalise when ||X^T M X - I||_F > ortho_tol (1e-12) */
  int ortho_every;    /* QR path: check ||X^T M X - I|| every this many iterations (20) */
  int verbose;        /* > 0: print E, ||D||_M and tau to stderr every `verbose` iterations (0) */
  int precision;      /* KS_FP64, or KS_MIXED: an FP32 phase, then an FP64 polish to gtol.
                         The FP32 phase carries the iterate as an FP64 base plus FP32
                         increments (fp32_increment = 1, below) and runs to gtol itself; with
                         fp32_increment = 0 it holds FP32 orbital blocks until ||D||_M <=
                         polish_gtol (or no progress for stall_iters iterations), evaluates
                         eps_xc and v_xc in FP32 and solves the Hartree CG to mixed_cg_tol.
                         The energy sums and p x p algebra are FP64 in every form (KS_FP64) */
  double polish_gtol; /* switch from the FP32 phase to the FP64 polish (1e-4) */
  int stall_iters;    /* 1: the FP32 phase also ends when it stagnates, i.e. the mean of
                         df_k = |E_{k-1} - E_k| / (|E_{k-1}| + 1) over the last three
                         iterations falls below stall_df (the stagnation measure of
                         Sec. 4.1), or the best ||D||_M has not improved by 0.1 % for 500
                         iterations (the FP32 rounding floor of systems whose energy is so
                         large that df never falls that far); 0: it ends only at
                         polish_gtol or maxit (1) */
  double stall_df;    /* stagnation threshold of the FP32 phase (1e-11) */
  int resume;         /* 1: continue from the state of the last ks_minimize on this problem
                         or from ks_state_load (X_inout is then output only); maxit counts
                         all iterations including those before the checkpoint.
                         ks_energy_grad, ks_retract, ks_orthonormalize and ks_minimize_host
                         work in the blocks that hold the state and discard it (0) */
  double mixed_cg_tol; /* KS_MIXED: Hartree CG tolerance during the FP32 phase, clamped to
                          [cg_tol, 1e-3]; FP32 orbitals carry about 1e-7 relative
                          error, so a tighter solve buys nothing there (1e-7).  The FP64
                          polish uses cg_tol. */
  int fp64_split;     /* 1: for this call, FP64 Grams and updates with at least 48 columns run on
                         the tensor cores by exact digit splitting (ks_set_fp64_emulation 1);
                         2: all of them; 0: the problem's own setting (0).  ks_batch_minimize
                         ignores it (the batched kernels do not split) */
  int fp32_increment; /* KS_MIXED: 1: the FP32 phase carries X = X_b + delta, an FP64 base
                         (refreshed every 32 iterations, M-orthonormalised in FP64) plus an
                         FP32 increment; the density, kinetic energy and retraction are
                         formed on the increment and the rest of the energy from the FP64
                         density (FP64 xc, Hartree to cg_tol), so its rounding scales with
                         |delta|.  The gradient is formed the same way (E_X, the Gram
                         E_X^T X and D as FP64 values at the base plus FP32 increments), so
                         the phase runs to gtol itself, or until ||D||_M has not improved by
                         0.1 % for 50000 iterations (stall_iters = 1); the FP64 polish then
                         confirms gtol; polish_gtol, stall_df and mixed_cg_tol do not apply.
                         0: the FP32 phase on an FP32 iterate (stops at its rounding floor,
                         ||D||_M ~ 1e-3 on large systems) (1).  ks_batch_minimize ignores
                         it */
} ks_opts;

typedef struct {
  double E;           /* total energy (hartree) at the returned X */
  double gradnorm;    /* ||D||_M at the returned X */
  double ortho_err;   /* ||X^T M X - I||_F at the returned X */
  double E_parts[5];  /* kinetic, external, Hartree, exchange-correlation, ion-ion */
  int iters;          /* outer iterations taken */
  int cg_iters_total; /* Hartree CG iterations over the whole run */
  int backtracks;     /* total backtracking steps */
  int status;         /* ks_status of the run (KS_ENOCONV when maxit was hit) */
  double seconds;     /* wall time of the call */
  int mixed_iters;    /* KS_MIXED: iterations of the FP32 phase */
  double mixed_gradnorm; /* KS_MIXED: ||D||_M at the end of the FP32 phase */
  double mixed_E;     /* KS_MIXED: energy at the end of the FP32 phase */
} ks_result;

/* Defaults listed in ks_opts. */
void ks_opts_default(ks_opts *opts);

/* Create a problem: copies the geometry, allocates all device workspace,
 * tabulates the external potential (sum of -Z erf(r/rc)/r) and the ion-ion
 * energy (Eq. EKS, E_II).  *out is NULL on failure.  The description is
 * checked on the host before any device call: 2 <= N <= 2048, L > 0,
 * 1 <= p <= N^3, N^3 p <= 2^31 - 1 (32-bit entry indices), natoms >= 0 with R and Z given when natoms > 0, rc > 0,
 * known xc, precision, mass and kinetic values, cg_tol > 0, cg_maxit >= 1,
 * and for KS_KIN_TFW p = 1 and a finite mu >= 0; KS_EINVAL otherwise. */
ks_status ks_problem_create(const ks_problem_desc *desc, ks_problem **out);
ks_status ks_problem_destroy(ks_problem *prob);

/* Bytes of device memory ks_problem_create would allocate (for admission);
 * 0 for an invalid description. */
size_t ks_problem_bytes(const ks_problem_desc *desc);

/* Energy and derivative at X (Eq. EKS discretised; E_X = dE/dX, the
 * paper's H(X)X of Eq. "partial deriv" with the occupation factor):
 *   X   DEVICE n x p (need not be M-orthonormal for E and EX)
 *   E   HOST, receives the total energy
 *   EX  DEVICE n x p or NULL, receives dE/dX
 *   D   DEVICE n x p or NULL, receives the projected gradient
 *       D = M^{-1} E_X - X (E_X^T X) (Eq. def-nablaE in the M metric)
 *   gradnorm  HOST or NULL, receives ||D||_M = sqrt(tr(D^T M D))
 * The Hartree solve is warm-started from the previous call's potential. */
ks_status ks_energy_grad(ks_problem *prob, const double *X, double *E,
                         double *EX, double *D, double *gradnorm);

/* Energy parts of the last evaluation: kinetic, external, Hartree,
 * exchange-correlation, ion-ion (HOST array of 5). */
ks_status ks_energy_parts(ks_problem *prob, double parts[5]);

/* One retraction step from an M-orthonormal X along -D (Eqs. QR or WY3):
 *   kind  KS_QR or KS_CAYLEY
 *   X     DEVICE n x p, M-orthonormal
 *   EX    DEVICE n x p, dE/dX at X (e.g. from ks_energy_grad)
 *   tau   step size
 *   Xout  DEVICE n x p, must not alias X or EX
 * Returns KS_ENOTPD / KS_ESINGULAR when the small system cannot be solved. */
ks_status ks_retract(ks_problem *prob, int kind, const double *X, const double *EX,
                     double tau, double *Xout);

/* X <- X L^{-T} with X^T M X = L L^T, applied twice (Cholesky QR in the M
 * inner product, Alg. ChQR).  X is DEVICE n x p, updated in place; when X^T M X
 * is not positive definite (dependent or zero columns) returns KS_ENOTPD and
 * leaves X unchanged. */
ks_status ks_orthonormalize(ks_problem *prob, double *X);

/* Alg. ConOptM from X_inout (DEVICE n x p, any full-rank block; it is
 * M-orthonormalised first).  On return X_inout holds the last accepted
 * iterate, also when the status is KS_ENOCONV. */
ks_status ks_minimize(ks_problem *prob, double *X_inout, const ks_opts *opts,
                      ks_result *result);

/* Same as ks_minimize with X_inout in HOST memory: the initial block is
 * copied to the device and the result copied back inside the call. */
ks_status ks_minimize_host(ks_problem *prob, double *X_inout_host, const ks_opts *opts,
                           ks_result *result);

/* Uniform refinement (Alg. AdpConOptM with every element refined and a fixed
 * number of levels, Sec. 4.3).  Nested grids have N' = 2N + 1 interior nodes
 * (spacing h/2, fine node 2i+1 = coarse node i).
 *
 * ks_prolong: Xf = (P1 x P1 x P1) Xc, the fine nodal values of the coarse
 * Q1 (trilinear) field.  P1 carries weight 1 to coinciding nodes and 1/2 to
 * midpoints; values beyond the ends are zero (Dirichlet).
 *   Xc: DEVICE, Nc^3 x p, row-major (orbital fastest).
 *   Xf: DEVICE, (2 Nc + 1)^3 x p.  Caller-owned; must not overlap Xc.
 *   stream: cudaStream_t, or NULL for the legacy default stream.
 * Returns KS_EINVAL for Nc outside [1, 1023], p < 1, null or overlapping
 * pointers.  The call is asynchronous on `stream`. */
ks_status ks_prolong(int Nc, int p, const double *Xc, double *Xf, void *stream);
ks_status ks_prolong_f32(int Nc, int p, const float *Xc, float *Xf, void *stream);

/* Alg. ConOptM on the grids N_l = (desc->N + 1) / 2^(levels-1-l) - 1,
 * l = 0 .. levels-1, ending at desc->N.  Each level gets its own problem with
 * the same geometry (desc with N replaced).
 *   X0_host: HOST, the initial block on the coarsest grid (N_0^3 x p).
 *   Levels l > 0 start from the prolongation of level l-1's final iterate.
 *   Coarser levels stop at ||D||_M <= coarse_gtol.  A coarse level that
 *     reaches opts->maxit still seeds the next.
 *   The finest level runs to opts->gtol.
 *   level_results: HOST, `levels` entries, one ks_result per level.
 *   X_host_out: HOST (N^3 x p), or NULL; receives the finest level's final
 *     block.
 * Requires a valid desc (the checks of ks_problem_create), (desc->N + 1)
 * divisible by 2^(levels-1) and N_0 >= 2; KS_EINVAL otherwise, before any
 * device call.  Returns the finest level's status, or the first error.  All
 * device memory is freed before return. */
ks_status ks_minimize_refine(const ks_problem_desc *desc, int levels, const double *X0_host,
                             const ks_opts *opts, double coarse_gtol, double *X_host_out,
                             ks_result *level_results);

/* Checkpoint of the minimiser (line-search scalars, current and previous
 * iterates with their M products, gradients, the Hartree potential and the
 * Hartree solver's last residual and right-hand side) after
 * the last iteration of the last ks_minimize call.  ks_state_bytes returns
 * the size needed (0 when there is nothing to save); ks_state_save writes it
 * to a HOST buffer; ks_state_load restores it into a problem with the same N
 * and p, after which ks_minimize with opts.resume = 1 continues the run.  With
 * the FP64 path the continued run is bitwise identical to an uninterrupted
 * one (all reductions have a fixed order). */
size_t ks_state_bytes(ks_problem *prob);
ks_status ks_state_save(ks_problem *prob, void *host_buf, size_t bytes);
ks_status ks_state_load(ks_problem *prob, const void *host_buf, size_t bytes);

/* Kernels this library has launched in this process so far. */
unsigned long long ks_kernel_launches(void);

/* Bounds-checked build.  Compiled with -DKS_DEBUG_BOUNDS (the build's
 * KS_DEBUG_BOUNDS=1), the hot-path kernels -- stencils, density, M^{-1}
 * sweeps, Grams and updates, the Hartree solver's passes, the p x p factor
 * and the tensor-core update -- test each computed global and shared-memory
 * index before the access it guards; an index out of range skips the access
 * and is counted instead of faulting.  Returns 1 in such a build, 0
 * otherwise.  *count (when not NULL) receives the number of out-of-range
 * indices caught since the last call (always 0 in a normal build), *file and
 * *line the source file and line of the first one (NULL, 0 when none); the
 * record is then cleared.  Synchronises the device in a checked build. */
int ks_debug_bounds(unsigned long long *count, const char **file, int *line);

/* Optional timing of the library's kernels by class with CUDA events on the
 * launching stream.  ks_profile_start() clears the totals and switches
 * timing on; ks_profile_stop() waits for the recorded events, switches
 * timing off and returns per class the summed milliseconds and the number
 * of timed launch groups (HOST arrays of KS_PROF_CLASSES, either may be
 * NULL).  Classes, in order: density, hartree_cg, potential, hamiltonian,
 * mass, mass_inverse, gram, combine, small_factor, reduce, setup, other. */
#define KS_PROF_CLASSES 12
ks_status ks_profile_start(void);
ks_status ks_profile_stop(double ms[KS_PROF_CLASSES], long long counts[KS_PROF_CLASSES]);
const char *ks_profile_class_name(int cls);
/* Algorithmic work of the launches timed since ks_profile_start, per class:
 * floating-point operations (an FMA counts 2) and minimal DRAM bytes (each
 * input block read once, each output block written once). */
ks_status ks_profile_work(double flops[KS_PROF_CLASSES], double bytes[KS_PROF_CLASSES]);

/* ------------------------------------------------------------------ serving
 * A server runs minimisation jobs (one KS system each) with continuous
 * batching: jobs are admitted in arrival order as soon as a slot is free and
 * their device memory (ks_problem_bytes plus the n x p block) fits in the
 * HBM budget; each admitted job runs on its own stream and host worker, so
 * admitted jobs overlap on the device, and a finishing job immediately
 * makes room for the next.  Jobs share no device state and every reduction
 * has a fixed order, so a job's result does not depend on what else runs.
 * The server is thread-safe; it uses the CUDA device current at creation. */
typedef struct ks_server ks_server;

typedef struct {
  int queued;                 /* jobs waiting for admission */
  int running;                /* jobs admitted and not finished */
  int peak_running;           /* maximum of running so far */
  unsigned long long completed;
  size_t bytes_in_use;        /* device bytes of the running jobs */
  size_t peak_bytes_in_use;   /* maximum of bytes_in_use so far (<= budget) */
  size_t budget;
} ks_server_counters;

/* max_slots: concurrent jobs (1..256); hbm_budget_bytes: admission limit. */
ks_status ks_server_create(size_t hbm_budget_bytes, int max_slots, ks_server **out);

/* Queue one job; desc->stream is ignored (each job gets its own stream), desc
 * geometry and X0_host (HOST n x p initial block) are copied; opts may be NULL
 * (defaults).  Returns KS_ENOMEM when the job alone exceeds the budget. */
ks_status ks_server_submit(ks_server *srv, const ks_problem_desc *desc, const ks_opts *opts,
                           const double *X0_host, uint64_t *job_id);

/* Result of a job: KS_EAGAIN while it is queued or running (wait = 0), or
 * blocks until it finishes (wait != 0).  On completion fills res, X_host
 * (HOST n x p, may be NULL) and latency_s (submit to finish, may be NULL),
 * then forgets the job (a job can be collected once: when several threads
 * wait on the same id, one collects it and the others get KS_EINVAL). */
ks_status ks_server_poll(ks_server *srv, uint64_t job_id, int wait, ks_result *res,
                         double *X_host, double *latency_s);

ks_status ks_server_stats(ks_server *srv, ks_server_counters *out);

/* Waits for running jobs, drops queued ones, joins the workers.  No other
 * call on srv may run concurrently with it or follow it. */
ks_status ks_server_destroy(ks_server *srv);

/* ---------------------------------------------------------------------------
 * Batched job table.  The paper minimises one system at a time; this is the
 * throughput form for many small independent systems: Alg. ConOptM (QR
 * retraction, Prop. 3.1) runs for every job of the table in lockstep
 * iterations, and each step of an iteration (density, Hartree CG, potential,
 * stencils, M^{-1}, Grams, updates, p x p factors) is ONE kernel launch over
 * all jobs that are still iterating.  Every job keeps its own step size,
 * nonmonotone line search, convergence test and iteration count; a job that
 * backtracks repeats its trial while the others wait; a job that converges
 * (or fails) drops out of the launches.  Per-job results agree with
 * ks_minimize on the same system up to the order of floating-point sums.
 *
 * Limits: p <= 104 per job; njobs <= the number of CG blocks that fit on the
 * device at once (several hundred on GB300); KS_QR only. */
typedef struct ks_batch ks_batch;

/* descs: njobs systems (stream fields ignored); stream: cudaStream_t for all
 * work (NULL = library-owned).  Allocates every job's device state.  Every
 * description is checked first (the checks of ks_problem_create, p <= 104,
 * orbital kinetic energy, consistent mass): KS_EINVAL before any device call. */
ks_status ks_batch_create(const ks_problem_desc *descs, int njobs, void *stream, ks_batch **out);

/* Device bytes held by the batch. */
size_t ks_batch_bytes(const ks_batch *batch);

/* 1 (default): the step sequences of an iteration (trial step + energy,
 * projection) run as CUDA graphs captured on first use per block-rotation
 * state and replayed (a captured energy evaluation holds three Hartree CG
 * iterations; jobs that need more continue outside the graph); 0: plain
 * launches.  Both give the same results bitwise.  Graphs are not used while
 * ks_profile_start timing is on. */
ks_status ks_batch_set_graphs(ks_batch *batch, int enable);

/* Autotuner of the batched launch shapes: times candidates of the Gram rows
 * per block (1024..16384), the update's outputs per thread (2..16), the
 * potential's nodes per thread (1..8) and the stencil's planes per block
 * (default, 8..64) on this job table and keeps the fastest of each (out, may
 * be NULL: the four choices).  Overwrites the jobs' device blocks (call it
 * before ks_batch_minimize).  A tuned batch gives each job a decomposition
 * chosen from the whole table's timings, so results agree with an untuned
 * run up to the order of sums only. */
ks_status ks_batch_autotune(ks_batch *batch, int out[4]);

/* Minimise every job from X_inout[j] (HOST, n_j x p_j row-major FP64; the
 * result overwrites it).  opts as for ks_minimize (retraction must be KS_QR;
 * KS_MIXED runs the FP32 phase for all jobs, then the FP64 polish for the
 * jobs that reached polish_gtol or stagnated); results: njobs entries.
 * results may be NULL; results[j].ortho_err is not computed (-1) and
 * results[j].seconds is the whole call's wall time.  Returns KS_OK when every
 * job converged, KS_ENOCONV when some did not (see results[j].status),
 * another code when the batch could not run. */
ks_status ks_batch_minimize(ks_batch *batch, double *const *X_inout, const ks_opts *opts,
                            ks_result *results);

ks_status ks_batch_destroy(ks_batch *batch);

/* Text of the last error on the calling thread ("" if none). */
const char *ks_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* KS_H */
