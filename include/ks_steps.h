/*
 * ks_steps.h -- one C entry point per step of the iteration, for callers that
 * compose their own driver and for step-by-step verification.  Each
 * ks_step_* call runs on the problem's stream with the problem's sizes
 * (n = N^3 nodes, p orbitals), synchronises it before returning, and follows
 * the conventions of ks.h (ks_status return value; DEVICE pointers are owned
 * by the caller; outputs must not alias inputs).  ks_gram_noalloc at the end
 * only enqueues (see its comment).
 */
#ifndef KS_STEPS_H
#define KS_STEPS_H

#include "ks.h"

#ifdef __cplusplus
extern "C" {
#endif

/* External potential sum_a -Z_a erf(|r - R_a|/rc)/|r - R_a| on the nodes
 * (E_ext of Eq. EKS).  vext: DEVICE n. */
ks_status ks_step_vext(ks_problem *prob, double *vext);

/* Ion-ion energy E_II of Eq. EKS (HOST scalar). */
ks_status ks_step_eii(ks_problem *prob, double *eii);

/* rho_k = f sum_i X_ki^2 (Sec. 2.3, rho(X) = diag(X X^T)).
 * X: DEVICE n x p; rho: DEVICE n. */
ks_status ks_step_density(ks_problem *prob, const double *X, double *rho);

/* Hartree potential by conjugate gradients on K vH = 4 pi h^3 rho (the
 * discrete L^+ rho of Sec. 2.3), stopping at ||r|| <= cg_tol ||b||.
 *   rho    DEVICE n
 *   vH     DEVICE n, in/out: the start vector when warm != 0, else ignored
 *   resid  DEVICE n or NULL, receives r = 4 pi h^3 rho - K vH
 *   iters  HOST or NULL, receives the iteration count
 * Returns KS_ENOCONV when cg_maxit is reached. */
ks_status ks_step_hartree(ks_problem *prob, const double *rho, double *vH, int warm,
                          double *resid, int *iters);

/* V_eff = Vext + vH + v_xc(rho) (+ v_TF = (5/3) C_TF rho^(2/3) for the
 * KS_KIN_TFW model) and the energies (HOST, 4): h^3 sum Vext rho,
 * 1/2 h^3 sum vH rho + vH.resid/(8 pi), h^3 sum rho eps_xc(rho), and the
 * Thomas-Fermi energy h^3 sum C_TF rho^(5/3) (0 for KS_KIN_ORBITALS).  resid
 * may be NULL (treated as zero).  rho, vH, veff: DEVICE n. */
ks_status ks_step_potential(ks_problem *prob, const double *rho, const double *vH,
                            const double *resid, double *veff, double energies[4]);

/* E_X = w f K X + 2 f h^3 Diag(veff) X, MX = M X (DEVICE n x p or NULL) and
 * the kinetic energy w (f/2) tr(X^T K X) (HOST), with w = 1 (KS_KIN_ORBITALS)
 * or mu (KS_KIN_TFW: the von Weizsaecker term). */
ks_status ks_step_hamiltonian(ks_problem *prob, const double *X, const double *veff,
                              double *EX, double *MX, double *kinetic);

/* FP32 form of ks_step_hamiltonian used by the mixed-precision phase: X, EX,
 * MX DEVICE n x p FP32 (MX may be NULL), veff DEVICE n FP64 (rounded to FP32
 * once per node), kinetic HOST FP64 (FP32 terms, FP64 block sums). */
ks_status ks_step_hamiltonian_f32(ks_problem *prob, const float *X, const double *veff,
                                  float *EX, float *MX, double *kinetic);

/* MX = M X with the problem's mass (consistent Q1, or h^3 I when lumped).
 * DEVICE n x p. */
ks_status ks_step_mass(ks_problem *prob, const double *X, double *MX);

/* G = M^{-1} E (consistent mass: three tridiagonal line sweeps; lumped:
 * h^-3 E).  DEVICE n x p; G must not alias E. */
ks_status ks_step_mass_inverse(ks_problem *prob, const double *E, double *G);

/* out = A^T B: A DEVICE n x pa, B DEVICE n x qb, out DEVICE pa x qb
 * (1 <= pa, qb <= p). */
ks_status ks_step_gram(ks_problem *prob, const double *A, int pa, const double *B, int qb,
                       double *out);

/* Tensor-core use of the FP32 phase: 0 never, 1 (default) for products of
 * at least 256 x 256 columns, 2 always (pa, qb, q > 8 for the Gram, q > 32
 * for the update), 3 as 1 plus the narrow updates (q <= 64, q a multiple
 * of 4, K <= 192, 16-byte-aligned blocks: the retraction's update and the
 * projected gradient at p <= 64) with three TF32 products per term. */
ks_status ks_set_tensor_cores(ks_problem *prob, int mode);

/* FP64 Grams A^T B and updates A1 C1 + A2 C2 (ks_step_gram, ks_step_combine and
 * every FP64 product of a minimisation) on the tensor cores by error-free
 * splitting.  Each FP64 entry becomes 8 signed digits below the largest
 * exponent of its line: 6-bit digits (48 bits) below its Gram column's,
 * 7-bit digits (56 bits) below its update row's (A) or column's (C).  Every
 * digit product is exact in a BF16 MMA whose FP32 accumulation stays exact
 * (512-row chunks for the Gram, K <= 128 for the update); digit pairs of
 * weight below 2^(-8 b) are not formed, and the digit groups are combined
 * exactly before one FP64 rounding.  Truncating an entry a_k of a line with
 * largest magnitude amax loses less than 2^-47 amax (Gram) or 2^-55 amax
 * (update), so an entry of A^T B differs from the exact sum by about
 * 2^-47 (max|a| sum|b_k| + max|b| sum|a_k|) plus one rounding, and an update
 * entry by about 2^-55 (max_k|a_k| sum|c_k| + max_k|c_k| sum|a_k|) plus the
 * roundings of alpha, beta and Bm; FP64 summation gives ~K 2^-53 sum|a_k b_k|.
 *   mode 0: never (default);
 *   mode 1: Grams whose operands both have at least 48 columns, and updates
 *     with K <= 128 and at least 48 output columns;
 *   mode 2: always (updates with K <= 128).
 * KS_EINVAL for other modes. */
ks_status ks_set_fp64_emulation(ks_problem *prob, int mode);

/* Plane staging of the 27-point stencils: 1 (default) TMA tile loads into a
 * shared-memory ring when the row pitch p * element size and the block's
 * base address are multiples of 16 bytes, 0 plain loads always.  Both give
 * the same sums in the same order. */
ks_status ks_set_tma(ks_problem *prob, int mode);

/* FP32 Gram of the mixed-precision phase, out = A^T B in FP64 (A: DEVICE
 * n x pa FP32, B: DEVICE n x qb FP32, 1 <= pa, qb <= p).  When
 * ks_set_tensor_cores selects them (by default for pa, qb >= 256) it runs on
 * the tensor cores with three TF32 products per term (hi.hi + hi.lo +
 * lo.hi, about 2^-21 relative error per product); otherwise on the FP32
 * pipes.  FP32 accumulation within a chunk of rows; chunks summed in FP64. */
ks_status ks_step_gram_f32(ks_problem *prob, const float *A, int pa, const float *B, int qb,
                           double *out);

/* FP32 update of the mixed-precision phase, out = alpha (A1 C1 + A2 C2) +
 * beta Bm with FP32 blocks A1 (n x k1), A2 (n x k2 or NULL), Bm (n x q or NULL),
 * out (n x q) and FP64 C1 (k1 x q), C2 (k2 x q), all DEVICE.  C1, C2 are
 * rounded to FP32 once per call.  For q > 32 it runs on the tensor cores
 * when ks_set_tensor_cores selects them (three TF32 products per term). */
ks_status ks_step_combine_f32(ks_problem *prob, const float *A1, int k1, const double *C1,
                              const float *A2, int k2, const double *C2, double alpha,
                              double beta, const float *Bm, float *out, int q);

/* out = alpha (A1 C1 + A2 C2) + beta Bm: A1 DEVICE n x k1, C1 DEVICE k1 x q,
 * A2 DEVICE n x k2 or NULL, C2 DEVICE k2 x q, Bm DEVICE n x q or NULL,
 * out DEVICE n x q (1 <= k1, k2, q <= p). */
ks_status ks_step_combine(ks_problem *prob, const double *A1, int k1, const double *C1,
                          const double *A2, int k2, const double *C2, double alpha,
                          double beta, const double *Bm, double *out, int q);

/* Self-test of the bounded device waits.  Every device-side wait of the
 * library (the software grid barrier of the cooperative kernels, the
 * mbarrier waits of the TMA and tensor-core pipelines) gives up after a fixed
 * number of polls, records KS_ETIMEOUT in the launch's status word and
 * returns.  The probe runs the grid barrier in a one-block launch while the
 * barrier expects two blocks, so its wait expires.
 *   stream   cudaStream_t, or NULL for the legacy default stream
 *   status   HOST, receives the status the probe recorded (KS_ETIMEOUT when
 *            the bound works)
 *   seconds  HOST or NULL, wall time of the call (about a second)
 * Returns KS_OK when the probe ran and the context is still usable. */
ks_status ks_selftest_wait_timeout(void *stream, int *status, double *seconds);

/* Peak-rate probe of the FMA pipes, the denominator of the roofline of the
 * FP64 n p^2 contractions (Grams and updates of Sec. 3, rows of Alg. ConOptM)
 * and of the FP32 SIMT kernels.  Enqueues one kernel of `blocks` blocks of
 * 256 threads on `stream`; each thread updates a 4 x 4 block of accumulators
 * with the outer product of two register 4-vectors `iters` times (16
 * independent FMA chains) with no memory traffic.  The caller times the
 * launch (e.g. with events on the same stream); nothing is synchronised here.
 *   fp64    nonzero: FP64 FMAs; zero: FP32 FMAs
 *   blocks  grid size (a multiple of the SM count keeps every SM busy)
 *   iters   rounds of 16 FMAs per thread (rounded up to a multiple of 4)
 *   stream  cudaStream_t, or NULL for the legacy default stream
 *   sink    DEVICE, at least `blocks` doubles; written only under a condition
 *           the recurrence never meets, so its contents stay as they are
 *   flops   HOST, receives the flop count of the launch (2 per FMA)
 * Returns KS_EINVAL for null pointers or non-positive sizes. */
ks_status ks_probe_fma(int fp64, int blocks, int iters, void *stream, double *sink,
                       double *flops);

/* Allocation-free variant of ks_step_gram, for callers that cannot call
 * cudaMalloc: a host process whose device memory is owned by its own
 * allocator or reserved up front under a fixed budget (a serving process that
 * must not grow past what it reserved), code running inside another library's
 * callback where calling into the CUDA allocator is not allowed, and
 * latency-bound loops that must not pay for an allocation.  It needs no
 * ks_problem (ks_problem_create allocates) and calls no allocating routine:
 * the per-chunk partial sums live in a file-scope device array of 2^21
 * doubles (16 MiB) that every GPU which loads the library holds until the
 * process exits.  The paper has no counterpart.
 *   A    DEVICE n x pa (row-major, FP64)
 *   B    DEVICE n x qb (row-major, FP64)
 *   out  DEVICE pa x qb, receives A^T B
 *   stream  cudaStream_t to issue on (NULL = legacy default stream)
 * Requires pa * qb <= 2^21 (returns KS_EINVAL otherwise).  The first call on a
 * device looks up the array's device address for that device (with it
 * current, a runtime query besides the launches) and keeps it for the life
 * of the process; do not use this entry point after a cudaDeviceReset in the
 * same process (the kept address would be stale).
 * The call only enqueues work: the result is ready when `stream` reaches it.
 * All calls in the process share the one array and every call overwrites all
 * of it that it reads, so calls whose executions overlap on the GPU (for
 * example on two streams at once) race and must be serialised by the
 * caller. */
ks_status ks_gram_noalloc(const double *A, int pa, const double *B, int qb, long long n,
                          double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KS_STEPS_H */
