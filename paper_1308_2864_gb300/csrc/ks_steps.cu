// Per-step entry points (include/ks_steps.h): thin wrappers that run one
// kernel of the iteration on caller-provided buffers and synchronise.
#include "ks_internal.cuh"
#include "ks_steps.h"

using namespace ks;

namespace {

ks_status finish(Problem &P) {
  int st = 0;
  KS_CUDA_TRY(cudaMemcpyAsync(P.dstatus_host, P.dstatus, sizeof(int), cudaMemcpyDeviceToHost,
                              P.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  st = *P.dstatus_host;
  if (st != KS_OK) {
    KS_CUDA_TRY(cudaMemsetAsync(P.dstatus, 0, sizeof(int), P.stream));
    KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
    return set_error((ks_status)st, "device status %d", st);
  }
  return KS_OK;
}

ks_status read_scalars(Problem &P, int first, int count, double *out) {
  KS_CUDA_TRY(cudaMemcpyAsync(out, P.scal + first, count * sizeof(double), cudaMemcpyDeviceToHost,
                              P.stream));
  return finish(P);
}

}  // namespace

extern "C" {

ks_status ks_step_vext(ks_problem *kp, double *vext) {
  if (!kp || !vext) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  KS_CUDA_TRY(cudaMemcpyAsync(vext, P.vext, (size_t)P.n * sizeof(double), cudaMemcpyDeviceToDevice,
                              P.stream));
  return finish(P);
}

ks_status ks_step_eii(ks_problem *kp, double *eii) {
  if (!kp || !eii) return set_error(KS_EINVAL, "null argument");
  return read_scalars(kp->P, SC_EII, 1, eii);
}

ks_status ks_step_density(ks_problem *kp, const double *X, double *rho) {
  if (!kp || !X || !rho) return set_error(KS_EINVAL, "null argument");
  KS_TRY(launch_density(kp->P, X, rho));
  return finish(kp->P);
}

ks_status ks_step_hartree(ks_problem *kp, const double *rho, double *vH, int warm, double *resid,
                          int *iters) {
  if (!kp || !rho || !vH) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  double *r = resid ? resid : P.cg_r;
  KS_TRY(launch_cg(P, rho, vH, r, warm != 0));
  P.cg_inc_ok = false;     // the caller's vH and residual, not the loop's
  double it = 0;
  KS_CUDA_TRY(cudaMemcpyAsync(&it, P.scal + SC_CG_ITERS, sizeof(double), cudaMemcpyDeviceToHost,
                              P.stream));
  ks_status st = finish(P);
  if (iters) *iters = (int)it;
  return st;
}

ks_status ks_step_potential(ks_problem *kp, const double *rho, const double *vH,
                            const double *resid, double *veff, double energies[4]) {
  if (!kp || !rho || !vH || !veff) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  const double *r = resid;
  if (!r) {
    KS_CUDA_TRY(cudaMemsetAsync(P.cg_q, 0, (size_t)P.n * sizeof(double), P.stream));
    r = P.cg_q;
  }
  KS_TRY(launch_potential(P, rho, vH, r, veff, true));
  double e[4];
  KS_TRY(read_scalars(P, SC_EEXT, 4, e));
  if (energies)
    for (int i = 0; i < 4; ++i) energies[i] = e[i];
  return KS_OK;
}

ks_status ks_step_hamiltonian(ks_problem *kp, const double *X, const double *veff, double *EX,
                              double *MX, double *kinetic) {
  if (!kp || !X || !veff || !EX) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  KS_TRY(launch_hamiltonian(P, X, veff, EX, MX, P.scal + SC_EKIN));
  double k = 0;
  KS_TRY(read_scalars(P, SC_EKIN, 1, &k));
  if (kinetic) *kinetic = k;
  return KS_OK;
}

ks_status ks_step_hamiltonian_f32(ks_problem *kp, const float *X, const double *veff, float *EX,
                                  float *MX, double *kinetic) {
  if (!kp || !X || !veff || !EX) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  KS_TRY(launch_hamiltonian<float>(P, X, veff, EX, MX, P.scal + SC_EKIN));
  double k = 0;
  KS_TRY(read_scalars(P, SC_EKIN, 1, &k));
  if (kinetic) *kinetic = k;
  return KS_OK;
}

ks_status ks_step_mass(ks_problem *kp, const double *X, double *MX) {
  if (!kp || !X || !MX) return set_error(KS_EINVAL, "null argument");
  KS_TRY(launch_mass(kp->P, X, MX));
  return finish(kp->P);
}

ks_status ks_step_mass_inverse(ks_problem *kp, const double *E, double *G) {
  if (!kp || !E || !G) return set_error(KS_EINVAL, "null argument");
  if (E == G) return set_error(KS_EINVAL, "output aliases input");
  KS_TRY(launch_mass_inverse(kp->P, E, G));
  return finish(kp->P);
}

ks_status ks_step_gram(ks_problem *kp, const double *A, int pa, const double *B, int qb,
                       double *out) {
  if (!kp || !A || !B || !out) return set_error(KS_EINVAL, "null argument");
  if (pa < 1 || qb < 1 || pa > kp->P.p || qb > kp->P.p) return set_error(KS_EINVAL, "bad sizes");
  KS_TRY(launch_gram(kp->P, A, pa, B, qb, out));
  return finish(kp->P);
}

ks_status ks_set_tensor_cores(ks_problem *kp, int mode) {
  if (!kp || mode < 0 || mode > 3) return set_error(KS_EINVAL, "bad argument");
  kp->P.use_tc = mode;
  return KS_OK;
}

ks_status ks_set_fp64_emulation(ks_problem *kp, int mode) {
  if (!kp || mode < 0 || mode > 2) return set_error(KS_EINVAL, "bad argument");
  kp->P.use_oz = mode;
  return KS_OK;
}

ks_status ks_set_tma(ks_problem *kp, int mode) {
  if (!kp || mode < 0 || mode > 1) return set_error(KS_EINVAL, "bad argument");
  kp->P.use_tma = mode;
  return KS_OK;
}

ks_status ks_step_gram_f32(ks_problem *kp, const float *A, int pa, const float *B, int qb,
                           double *out) {
  if (!kp || !A || !B || !out) return set_error(KS_EINVAL, "null argument");
  if (pa < 1 || qb < 1 || pa > kp->P.p || qb > kp->P.p) return set_error(KS_EINVAL, "bad sizes");
  KS_TRY(launch_gram<float>(kp->P, A, pa, B, qb, out));
  return finish(kp->P);
}

ks_status ks_step_combine(ks_problem *kp, const double *A1, int k1, const double *C1,
                          const double *A2, int k2, const double *C2, double alpha, double beta,
                          const double *Bm, double *out, int q) {
  if (!kp || !A1 || !C1 || !out) return set_error(KS_EINVAL, "null argument");
  const int p = kp->P.p;
  if (k1 < 1 || k1 > p || q < 1 || q > p || (A2 && (k2 < 1 || k2 > p || !C2)))
    return set_error(KS_EINVAL, "bad sizes");
  if (out == A1 || out == A2 || out == Bm) return set_error(KS_EINVAL, "output aliases input");
  KS_TRY(launch_combine(kp->P, A1, k1, C1, A2, k2, C2, alpha, beta, Bm, out, q));
  return finish(kp->P);
}

ks_status ks_step_combine_f32(ks_problem *kp, const float *A1, int k1, const double *C1,
                              const float *A2, int k2, const double *C2, double alpha, double beta,
                              const float *Bm, float *out, int q) {
  if (!kp || !A1 || !C1 || !out) return set_error(KS_EINVAL, "null argument");
  const int p = kp->P.p;
  if (k1 < 1 || k1 > p || q < 1 || q > p || (A2 && (k2 < 1 || k2 > p || !C2)))
    return set_error(KS_EINVAL, "bad sizes");
  if (out == A1 || out == A2 || out == Bm) return set_error(KS_EINVAL, "output aliases input");
  KS_TRY(launch_combine<float>(kp->P, A1, k1, C1, A2, k2, C2, alpha, beta, Bm, out, q));
  return finish(kp->P);
}

}  // extern "C"
