// The C ABI (include/ks.h): problem lifetime, energy and gradient, one
// retraction step, M-orthonormalisation and the Alg. ConOptM driver.
//
// Host code here only sequences kernels and takes the scalar decisions of
// the line search (Eq. NMLS-Armijo) and of the Barzilai-Borwein step
// (Eq. bb-1) from device-computed traces; every array operation runs in the
// kernels of this library.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>

#include "ks_internal.cuh"

namespace ks {

namespace {
thread_local char g_err[512] = "";
}

ks_status set_error(ks_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

ks_status cuda_error(cudaError_t e, const char *where) {
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation)
    return set_error(KS_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
  return set_error(KS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}


static size_t gram_partials_len(int p, int sms) {
  const size_t tiles = (size_t)((p + kTile - 1) / kTile) * ((p + kTile - 1) / kTile);
  size_t len = ((size_t)4 * sms + tiles) * kTile * kTile;
  // tensor-core Grams (p >= 256): one 128 x 256 tile per SM, p^2 per chunk
  const size_t tc_tiles = (size_t)((p + 127) / 128) * ((p + 255) / 256);
  const size_t tc = ((sms + tc_tiles - 1) / tc_tiles) * (size_t)p * p;
  if (p >= 256 && tc > len) len = tc;
  return len;
}

size_t problem_bytes(int N, int p, int sms) {
  const size_t n = (size_t)N * N * N;
  size_t b = 13 * n * sizeof(double) + 2 * n * sizeof(float);         // n-vectors
  b += ((size_t)N * N + 2 * N) * sizeof(float);                      // sine basis
  b += (size_t)Problem::kNBlocks * (n * p * sizeof(double) + 256);    // n x p blocks
  b += (size_t)S_COUNT * p * p * sizeof(double);                      // small matrices
  b += (size_t)5 * p * p * sizeof(float);                             // FP32 coefficients, Grams
  b += tc_image_floats(p) * sizeof(float);                            // tensor-core image
  b += (size_t)(2 * p + 128) * sizeof(int);                           // split exponents
  b += oz_image_bytes(p);                                             // split coefficients
  b += n * sizeof(int);                                               // row exponents
  size_t part = gram_partials_len(p, sms);
  const size_t red = (size_t)4 * 8 * sms;
  const size_t cg = (size_t)4 * 2 * sms;
  if (red > part) part = red;
  if (cg > part) part = cg;
  b += part * sizeof(double);
  b += SC_COUNT * sizeof(double) + (size_t)N * sizeof(double) + 4096;
  return b;
}

ks_status validate_desc(const ks_problem_desc *d) {
  if (!d) return set_error(KS_EINVAL, "null description");
  if (d->N < 2 || d->N > 2048) return set_error(KS_EINVAL, "N = %d out of range [2, 2048]", d->N);
  if (!(d->L > 0.0)) return set_error(KS_EINVAL, "L must be positive");
  if (d->p < 1 || (long long)d->p > (long long)d->N * d->N * d->N)
    return set_error(KS_EINVAL, "p = %d out of range", d->p);
  // node and entry indices of an n x p block are 32-bit (2^31 - 1 FP64
  // entries per block is already 223 GB for the 13 blocks of a problem)
  if ((long long)d->N * d->N * d->N * d->p > 0x7fffffffLL)
    return set_error(KS_EINVAL, "n p = %lld entries exceeds 2^31 - 1",
                     (long long)d->N * d->N * d->N * d->p);
  if (d->natoms < 0 || (d->natoms > 0 && (!d->R || !d->Z)))
    return set_error(KS_EINVAL, "bad atom arrays");
  if (!(d->rc > 0.0)) return set_error(KS_EINVAL, "rc must be positive");
  if (d->xc != KS_XC_SLATER && d->xc != KS_XC_SLATER_PZ81) return set_error(KS_EINVAL, "bad xc");
  if (d->precision != KS_FP64 && d->precision != KS_MIXED)
    return set_error(KS_EINVAL, "bad precision");
  if (!(d->cg_tol > 0.0) || d->cg_maxit < 1) return set_error(KS_EINVAL, "bad CG parameters");
  if (d->mass != KS_MASS_CONSISTENT && d->mass != KS_MASS_LUMPED)
    return set_error(KS_EINVAL, "bad mass model");
  if (d->kinetic != KS_KIN_ORBITALS && d->kinetic != KS_KIN_TFW)
    return set_error(KS_EINVAL, "bad kinetic model");
  if (d->kinetic == KS_KIN_TFW) {
    if (d->p != 1) return set_error(KS_EINVAL, "the TFW model takes one amplitude (p = 1)");
    if (!(d->mu >= 0.0) || !std::isfinite(d->mu))
      return set_error(KS_EINVAL, "TFW weight mu must be finite and >= 0");
  }
  return KS_OK;
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// problem's stream), so creating and destroying problems does not
// synchronise the device while other problems run on other streams.
static void free_problem(Problem &P) {
  cudaStream_t s = P.stream;
  auto f = [s](void *q) { if (q) cudaFreeAsync(q, s); };
  f(P.vext); f(P.rho); f(P.vH); f(P.veff); f(P.rho_b); f(P.veff_b); f(P.zero_n); f(P.cg_r); f(P.cg_pa); f(P.cg_pb); f(P.cg_q);
  f(P.cg_z); f(P.cg_rho_prev); f(P.cg_t1); f(P.cg_t2); f(P.dst_phi); f(P.dst_kap); f(P.dst_mu);
  for (auto &b : P.blk) f(b);
  f(P.pp); f(P.cf); f(P.rt32); f(P.tc_img); f(P.oz_emax); f(P.oz_img); f(P.oz_rowexp); f(P.partials); f(P.scal); f(P.atoms_dev); f(P.thomas_w); f(P.bar); f(P.red_counter); f(P.dstatus);
  delete[] P.scal_host;
  delete[] P.dstatus_host;
  P.scal_host = nullptr;
  P.dstatus_host = nullptr;
  if (s) cudaStreamSynchronize(s);
  cudaGetLastError();
  if (P.own_stream && P.stream) cudaStreamDestroy(P.stream);
}

template <typename T>
static ks_status dalloc(T **ptr, size_t count, Problem &P) {
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : sizeof(T);
  cudaError_t e = cudaMallocAsync((void **)ptr, bytes, P.stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
  P.bytes += bytes;
  return KS_OK;
}

static double *sm(Problem &P, int which) { return P.pp + (size_t)which * P.p * P.p; }

// Copy device scalars and the status word to the host and wait.
static ks_status sync_scalars(Problem &P) {
  KS_CUDA_TRY(cudaMemcpyAsync(P.scal_host, P.scal, SC_COUNT * sizeof(double),
                              cudaMemcpyDeviceToHost, P.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(P.dstatus_host, P.dstatus, sizeof(int), cudaMemcpyDeviceToHost,
                              P.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  prof_collect();
  const int st = *P.dstatus_host;
  if (st != KS_OK) {
    KS_CUDA_TRY(cudaMemsetAsync(P.dstatus, 0, sizeof(int), P.stream));
    switch (st) {
      case KS_ENOCONV: return set_error(KS_ENOCONV, "Hartree CG did not reach its tolerance");
      case KS_ENOTPD: return set_error(KS_ENOTPD, "Cholesky met a non-positive pivot");
      case KS_ESINGULAR: return set_error(KS_ESINGULAR, "Cayley system is singular");
      case KS_ENAN: return set_error(KS_ENAN, "non-finite value in the Hartree CG");
      case KS_ETIMEOUT: return set_error(KS_ETIMEOUT, "device grid barrier timed out");
      default: return set_error(KS_ECUDA, "device status %d", st);
    }
  }
  return KS_OK;
}

// ---------------------------------------------------------------- phases
// Typed view of the n x p block `b` (blocks hold FP64 capacity; the mixed
// phase stores FP32 values in them).
template <typename T>
static T *blk(Problem &P, int b) { return reinterpret_cast<T *>(P.blk[b]); }

// Energy at X: density, Hartree CG (warm-started when a previous potential
// exists), potential and energy sums, Hamiltonian stencil (E_X, M X).
template <typename T>
static ks_status evaluate(Problem &P, const T *X, T *EX, T *MX, double *E) {
  P.rho_block = -1;
  KS_TRY(launch_density<T>(P, X, P.rho));
  KS_TRY(launch_cg(P, P.rho, P.vH, P.cg_r, P.vH_valid));
  KS_TRY(launch_potential(P, P.rho, P.vH, P.cg_r, P.veff, true, sizeof(T) == 4));
  KS_TRY(launch_hamiltonian<T>(P, X, P.veff, EX, MX, P.scal + SC_EKIN));
  ks_status st = sync_scalars(P);
  if (st != KS_OK) {
    P.vH_valid = false;
    return st;
  }
  P.vH_valid = true;
  const double *s = P.scal_host;
  P.last_parts[0] = s[SC_EKIN] + s[SC_ETF];
  P.last_parts[1] = s[SC_EEXT];
  P.last_parts[2] = s[SC_EH];
  P.last_parts[3] = s[SC_EXC];
  P.last_parts[4] = s[SC_EII];
  P.last_cg_iters = (int)s[SC_CG_ITERS];
  P.last_E = s[SC_EKIN] + s[SC_ETF] + s[SC_EEXT] + s[SC_EH] + s[SC_EXC] + s[SC_EII];
  if (!std::isfinite(P.last_E)) return set_error(KS_ENAN, "non-finite energy");
  *E = P.last_E;
  return KS_OK;
}

struct Traces {
  double dnorm2 = 0, ss = 0, sy = 0, yy = 0;
};

// Projected gradient at X (Eq. def-nablaE in the M metric):
// G = M^{-1} E_X, S = E_X^T X, D = G - X S, MD = M D, ||D||_M^2, the BB
// traces against `prev`, and the Grams the retraction needs.
template <typename T>
static ks_status project(Problem &P, int retraction, const T *X, const T *EX, const T *MX, T *D,
                         T *MD, const BBPrevT<T> *prev, Traces *tr) {
  const int p = P.p;
  T *G = blk<T>(P, B_G);
  KS_TRY(launch_mass_inverse<T>(P, EX, G));
  KS_TRY(launch_gram<T>(P, EX, p, X, p, sm(P, S_S)));
  KS_TRY(launch_combine<T>(P, X, p, sm(P, S_S), nullptr, 0, nullptr, -1.0, 1.0, G, D, p));
  KS_TRY(launch_mass_dots<T>(P, D, MD, X, MX, prev, P.scal + SC_DNORM2));
  if (retraction == KS_QR) {
    KS_TRY(launch_gram<T>(P, D, p, MD, p, sm(P, S_DMD)));
  } else {
    KS_TRY(launch_transpose(P, sm(P, S_S), sm(P, S_A)));
    KS_TRY(launch_gram<T>(P, EX, p, G, p, sm(P, S_B)));
    KS_TRY(launch_gram<T>(P, X, p, MX, p, sm(P, S_O)));
  }
  KS_TRY(sync_scalars(P));
  tr->dnorm2 = P.scal_host[SC_DNORM2];
  if (prev) {
    tr->ss = P.scal_host[SC_BB_SS];
    tr->sy = P.scal_host[SC_BB_SY];
    tr->yy = P.scal_host[SC_BB_YY];
  }
  if (!std::isfinite(tr->dnorm2)) return set_error(KS_ENAN, "non-finite gradient norm");
  return KS_OK;
}

// X+ from X along -D with step tau (uses the Grams left by project()).
template <typename T>
static ks_status retract(Problem &P, int retraction, const T *X, const T *D, double tau,
                         T *Xout) {
  const int p = P.p;
  if (retraction == KS_QR) {
    KS_TRY(launch_qr_factor(P, sm(P, S_DMD), nullptr, tau, sm(P, S_C1), sm(P, S_C2)));
    KS_TRY(launch_combine<T>(P, X, p, sm(P, S_C1), D, p, sm(P, S_C2), 1.0, 0.0, nullptr, Xout, p));
  } else {
    KS_TRY(launch_cayley_factor(P, sm(P, S_A), sm(P, S_S), sm(P, S_B), sm(P, S_O), tau,
                                sm(P, S_C1), sm(P, S_C2)));
    KS_TRY(launch_combine<T>(P, X, p, sm(P, S_C1), blk<T>(P, B_G), p, sm(P, S_C2), 1.0, 0.0,
                             nullptr, Xout, p));
  }
  return KS_OK;
}

// Cholesky QR in the M inner product, `passes` times; X is updated in place
// (tmp is an n x p scratch block, MX receives M X of the result).  The Gram
// and the factor are FP64 in both precisions.
template <typename T>
static ks_status orthonormalize(Problem &P, T *X, T *tmp, T *MX, int passes) {
  const int p = P.p;
  for (int k = 0; k < passes; ++k) {
    KS_TRY(launch_mass<T>(P, X, MX));
    KS_TRY(launch_gram<T>(P, X, p, MX, p, sm(P, S_O)));
    KS_TRY(launch_qr_factor(P, nullptr, sm(P, S_O), 0.0, sm(P, S_C1), nullptr));
    KS_TRY(launch_combine<T>(P, X, p, sm(P, S_C1), nullptr, 0, nullptr, 1.0, 0.0, nullptr, tmp, p));
    KS_CUDA_TRY(cudaMemcpyAsync(X, tmp, (size_t)P.n * p * sizeof(T), cudaMemcpyDeviceToDevice,
                                P.stream));
  }
  KS_TRY(launch_mass<T>(P, X, MX));
  return sync_scalars(P);
}

// ||X^T M X - I||_F
template <typename T>
static ks_status ortho_error(Problem &P, const T *X, const T *MX, double *err) {
  KS_TRY(launch_gram<T>(P, X, P.p, MX, P.p, sm(P, S_T)));
  KS_TRY(launch_ortho_err(P, sm(P, S_T), P.scal + SC_ORTHO));
  KS_TRY(sync_scalars(P));
  *err = std::sqrt(P.scal_host[SC_ORTHO]);
  return KS_OK;
}

// tau_{k,1} = ss/|sy| on odd k, tau_{k,2} = |sy|/yy on even k (Eq. bb-1),
// reset to tau0 when not a positive finite number, then clamped.
static double bb_step(int k, const Traces &t, const ks_opts &o) {
  double num, den;
  if (k % 2 == 1) { num = t.ss; den = std::fabs(t.sy); }
  else { num = std::fabs(t.sy); den = t.yy; }
  if (!(den > 0.0) || !std::isfinite(num) || !std::isfinite(den)) return o.tau0;
  double tau = num / den;
  if (!std::isfinite(tau) || tau <= 0.0) return o.tau0;
  if (tau < o.tau_min) tau = o.tau_min;
  if (tau > o.tau_max) tau = o.tau_max;
  return tau;
}

struct PhaseResult {
  double E = 0, dnorm = 0;
  double last_tau = 0;             // last accepted step
  int iters = 0, cg = 0, backtracks = 0;
  bool stalled = false;
};

// One run of Alg. ConOptM in storage precision T from the block Xstart
// (copied in, then M-orthonormalised) -- or, when `resume` is set, from the
// state left in P.state by an earlier run or by ks_state_load -- until
// ||D||_M <= gtol, `maxit` iterations in total, or (stall > 0) stagnation:
// the energy measure of Sec. 4.1 below o.stall_df, or no 0.1 % improvement of
// the best ||D||_M for kStallWindow iterations.  The final iterate
// is copied to Xend and the loop state is kept in P.state.
template <typename T>
static ks_status run_phase(Problem &P, const T *Xstart, T *Xend, const ks_opts &o, double gtol,
                           int maxit, int stall, int first_k, double ortho_tol, bool resume,
                           PhaseResult *out, double tau_first = 0.0) {
  const int p = P.p;
  const size_t bytes = (size_t)P.n * p * sizeof(T);
  Problem::RunState &S = P.state;
  int ix[3] = {B_X0, B_X1, B_X2};        // cur, prev, trial
  int imx[3] = {B_MX0, B_MX1, B_MX2};
  int iex[2] = {B_EX0, B_EX1};           // cur, trial
  int id[2] = {B_D0, B_D1};              // cur, prev
  int imd[2] = {B_MD0, B_MD1};
  auto X = [&](int s) { return blk<T>(P, ix[s]); };
  auto MX = [&](int s) { return blk<T>(P, imx[s]); };
  auto EX = [&](int s) { return blk<T>(P, iex[s]); };
  auto D = [&](int s) { return blk<T>(P, id[s]); };
  auto MD = [&](int s) { return blk<T>(P, imd[s]); };

  double E = 0, C = 0, Q = 1.0, best = 0;
  int k = 0, last_improve = 0, cg_total = 0;
  bool have_prev = false;
  Traces tr;
  if (resume) {
    for (int i = 0; i < 3; ++i) { ix[i] = S.ix[i]; imx[i] = S.imx[i]; }
    for (int i = 0; i < 2; ++i) { iex[i] = S.iex[i]; id[i] = S.id[i]; imd[i] = S.imd[i]; }
    first_k = S.first_k;
    k = S.k;
    E = S.E; C = S.C; Q = S.Q; best = S.best; last_improve = S.last_improve;
    out->last_tau = S.last_tau;
    have_prev = S.have_prev != 0;
    P.vH_valid = true;
    // regenerates D, MD, the small matrices and the traces exactly (all
    // reductions have a fixed order)
    BBPrevT<T> prev{X(1), MX(1), D(1), MD(1)};
    KS_TRY(project<T>(P, S.retraction, X(0), EX(0), MX(0), D(0), MD(0),
                      have_prev ? &prev : nullptr, &tr));
  } else {
    KS_CUDA_TRY(cudaMemcpyAsync(X(0), Xstart, bytes, cudaMemcpyDeviceToDevice, P.stream));
    KS_TRY(orthonormalize<T>(P, X(0), X(2), MX(0), 2));
    KS_TRY(evaluate<T>(P, X(0), EX(0), MX(0), &E));
    cg_total = P.last_cg_iters;
    KS_TRY(project<T>(P, o.retraction, X(0), EX(0), MX(0), D(0), MD(0), nullptr, &tr));
    C = E;
    best = std::sqrt(std::fmax(tr.dnorm2, 0.0));
  }
  const int k0 = k;
  int backtracks = 0;
  bool stalled = false;
  double df[3] = {1.0, 1.0, 1.0}, Eprev = E;
  auto save_state = [&]() {
    S.valid = true;
    S.elem = (int)sizeof(T);
    S.split = 0;
    S.retraction = o.retraction;
    S.first_k = first_k;
    S.k = k;
    S.have_prev = have_prev ? 1 : 0;
    S.C = C; S.Q = Q; S.E = E; S.best = best; S.last_improve = last_improve;
    S.last_tau = out->last_tau;
    S.dnorm2 = tr.dnorm2; S.ss = tr.ss; S.sy = tr.sy; S.yy = tr.yy;
    for (int i = 0; i < 3; ++i) { S.ix[i] = ix[i]; S.imx[i] = imx[i]; }
    for (int i = 0; i < 2; ++i) { S.iex[i] = iex[i]; S.id[i] = id[i]; S.imd[i] = imd[i]; }
  };
  save_state();
  while (std::sqrt(std::fmax(tr.dnorm2, 0.0)) > gtol && first_k + k < maxit) {
    double tau = have_prev ? bb_step(first_k + k, tr, o) : (tau_first > 0.0 ? tau_first : o.tau0);
    int h = 0;
    double Et = 0;
    bool forced = false;
    for (;;) {
      KS_TRY(retract<T>(P, o.retraction, X(0), D(0), tau, X(2)));
      KS_TRY(evaluate<T>(P, X(2), EX(1), MX(2), &Et));
      cg_total += P.last_cg_iters;
      const bool ok = Et <= C - o.rho1 * tau * tr.dnorm2 + armijo_slack<T>(P.last_parts);
      if (ok || h == o.max_backtrack) {
        forced = !ok;
        break;
      }
      tau *= o.delta;
      ++h;
    }
    backtracks += h;
    out->last_tau = tau;
    const double Qn = o.eta * Q + 1.0;
    C = (o.eta * Q * C + Et) / Qn;
    Q = Qn;
    // FP64: a trial accepted without meeting the test restarts the nonmonotone
    // reference at its energy (C = E, Q = 1; C_k >= E_k still holds), so that
    // a reference left below the current energy cannot reject every later
    // step.  The FP32 phase keeps the reference: there a run of rejected steps
    // at its rounding floor freezes the energy, which ends the phase through
    // the stagnation measure.
    if (forced && sizeof(T) == 8) {
      C = Et;
      Q = 1.0;
    }
    // accept: prev <- cur, cur <- trial
    std::swap(ix[1], ix[0]);
    std::swap(ix[0], ix[2]);
    std::swap(imx[1], imx[0]);
    std::swap(imx[0], imx[2]);
    std::swap(iex[0], iex[1]);
    std::swap(id[0], id[1]);
    std::swap(imd[0], imd[1]);
    E = Et;
    ++k;
    bool reortho = false;
    // the Cayley path checks every iteration (Sec. 4.1); the QR path every
    // ortho_every iterations (every 5 in the FP32 phase, whose rounding
    // drifts faster), and every iteration for one amplitude (p = 1: the check
    // is one dot product, and the factor of Prop. 3.1 assumes c^T M c = 1,
    // which an amplitude carrying all the electrons needs to the last bits)
    const int every = p == 1 ? 1 : (sizeof(T) == 4 ? std::min(o.ortho_every, 5) : o.ortho_every);
    if (o.retraction == KS_CAYLEY || (every > 0 && (first_k + k) % every == 0)) {
      double oerr = 0;
      KS_TRY(ortho_error<T>(P, X(0), MX(0), &oerr));
      reortho = oerr > ortho_tol;
    }
    if (reortho) {
      KS_TRY(orthonormalize<T>(P, X(0), X(2), MX(0), 1));
      KS_TRY(evaluate<T>(P, X(0), EX(0), MX(0), &E));
      cg_total += P.last_cg_iters;
    }
    BBPrevT<T> prev{X(1), MX(1), D(1), MD(1)};
    KS_TRY(project<T>(P, o.retraction, X(0), EX(0), MX(0), D(0), MD(0), &prev, &tr));
    have_prev = true;
    const double dn = std::sqrt(std::fmax(tr.dnorm2, 0.0));
    bool stop = false;
    // energy stagnation measure of Sec. 4.1: df_k = |E_{k-1} - E_k| / (|E_{k-1}| + 1),
    // averaged over the last three iterations
    df[k % 3] = std::fabs(Eprev - E) / (std::fabs(Eprev) + 1.0);
    Eprev = E;
    if (dn < 0.999 * best) {
      best = dn;
      last_improve = k;
    }
    if (stall > 0 && k - k0 >= 3 &&
        ((df[0] + df[1] + df[2]) / 3.0 < o.stall_df || k - last_improve >= kStallWindow)) {
      stalled = true;
      stop = true;
    }
    save_state();
    if (o.verbose > 0 && (first_k + k) % o.verbose == 0)
      fprintf(stderr, "ks_minimize[%s]: k=%d E=%.12f |D|=%.3e tau=%.3e h=%d cg=%d\n",
              sizeof(T) == 8 ? "fp64" : "fp32", first_k + k, E, dn, tau, h, P.last_cg_iters);
    if (stop) break;
  }
  KS_CUDA_TRY(cudaMemcpyAsync(Xend, X(0), bytes, cudaMemcpyDeviceToDevice, P.stream));
  out->E = E;
  out->dnorm = std::sqrt(std::fmax(tr.dnorm2, 0.0));
  out->iters = k - k0;
  out->cg = cg_total;
  out->backtracks = backtracks;
  out->stalled = stalled;
  return KS_OK;
}

// ---------------------------------------------------------------- increment form
// FP32 phase that carries its iterate as X = X_b + delta: an FP64 base X_b,
// held as two FP32 blocks hi + lo, and an FP32 increment delta.  At the base
// everything is evaluated in FP64 -- energy, density rho_b, potential V_b,
// gradient E_b = E_X(X_b), the Gram S_b = E_b^T X_b and the projected
// gradient D_b = M^{-1} E_b - X_b S_b (Eq. def-nablaE) -- and between
// refreshes only increments are formed in FP32:
//   rho = rho_b + f sum delta (2 X_b + delta)
//   T   = T_b + sum delta . (f K X_b + (f/2) K delta)   (compensated sum)
//   E_ext, E_H, E_xc from rho in FP64 (FP64 xc, Hartree CG to cg_tol)
//   e   = E_X - E_b = f K delta + 2 f h^3 (Diag(V - V_b) X_b + Diag(V) delta)
//   dS  = S - S_b = E_b^T delta + e^T X
//   D   = D_b + M^{-1} e - delta S_b - X dS
// so every FP32 rounding scales with |delta|, |e| or ||D||, never with |X|
// or |E_X|: the energies the line search compares and the direction it takes
// stay as accurate as FP64 ones far below the FP32 rounding of the orbitals.
// The retraction forms delta+ = X_b (A - I) + delta A + D B (retract_split).
// Every kRebaseEvery accepted iterations the base absorbs the increment in
// FP64 (and is re-M-orthonormalised when it has drifted).
//
// Storage: the iterate blocks hold delta in their lower half and the FP32
// copy X32 = fl32(X_b + delta) in their upper half; the E_X blocks hold e;
// the upper halves of B_MX0, B_MX1, B_MX2 and B_G hold hi, lo, fl32(E_b) and
// fl32(D_b); rho_b, V_b are n-vectors and S_b is a p x p matrix.
#ifndef KS_REBASE_EVERY
#define KS_REBASE_EVERY 32
#endif
namespace {
constexpr int kRebaseEvery = KS_REBASE_EVERY;
constexpr double kSplitOrthoTol = 1e-13;
constexpr int kSplitStallWindow = 50000;
}  // namespace

static float *lower32(Problem &P, int b) { return reinterpret_cast<float *>(P.blk[b]); }
static float *upper32(Problem &P, int b) {
  return reinterpret_cast<float *>(reinterpret_cast<char *>(P.blk[b]) + P.half_off);
}
static float *base_hi(Problem &P) { return upper32(P, B_MX0); }
static float *base_lo(Problem &P) { return upper32(P, B_MX1); }
static float *base_eb(Problem &P) { return upper32(P, B_MX2); }
static float *base_db(Problem &P) { return upper32(P, B_G); }

// Energy at X_b + delta (delta in the lower half of block bx), the gradient
// increment e and M delta.
static ks_status evaluate_split(Problem &P, int bx, float *e, float *Md, double *E) {
  const float *d = lower32(P, bx);
  // the retraction's update pass may already have formed the trial's density
  if (P.rho_block != bx) KS_TRY(launch_density_inc(P, d, base_hi(P), P.rho_b, P.rho));
  P.rho_block = -1;
  KS_TRY(launch_cg(P, P.rho, P.vH, P.cg_r, P.vH_valid));
  KS_TRY(launch_potential(P, P.rho, P.vH, P.cg_r, P.veff, true, false));
  KS_TRY(launch_hamiltonian_inc(P, d, P.veff, P.veff_b, base_hi(P), base_eb(P), e, Md,
                                P.scal + SC_EKIN));
  ks_status st = sync_scalars(P);
  if (st != KS_OK) {
    P.vH_valid = false;
    return st;
  }
  P.vH_valid = true;
  const double *s = P.scal_host;
  const double ekin = P.state.T_b + s[SC_EKIN];
  P.last_parts[0] = ekin + s[SC_ETF];
  P.last_parts[1] = s[SC_EEXT];
  P.last_parts[2] = s[SC_EH];
  P.last_parts[3] = s[SC_EXC];
  P.last_parts[4] = s[SC_EII];
  P.last_cg_iters = (int)s[SC_CG_ITERS];
  P.last_E = ekin + s[SC_ETF] + s[SC_EEXT] + s[SC_EH] + s[SC_EXC] + s[SC_EII];
  if (!std::isfinite(P.last_E)) return set_error(KS_ENAN, "non-finite energy");
  *E = P.last_E;
  return KS_OK;
}

// Projected gradient at the iterate of block bx (delta and X32) with
// gradient increment e and M delta: D = D_b + M^{-1} e - delta S_b - X dS,
// S = S_b + dS, the BB traces on the increments (X_b is common to both
// iterates), and the Grams the retraction needs: R = D^T M D, T = X^T M D,
// and for Cayley A = S^T, B = E_X^T G = E_X^T D + S S, O = I.
static ks_status project_split(Problem &P, int retraction, int bx, const float *e,
                               const float *Md, float *D, float *MD, const BBPrevT<float> *prev,
                               Traces *tr) {
  const int p = P.p;
  float *Gi = lower32(P, B_G);
  const float *X32 = upper32(P, bx), *d = lower32(P, bx);
  KS_TRY(launch_mass_inverse<float>(P, e, Gi, base_db(P)));                // D_b + M^{-1} e
  // dS = E_b^T delta + e^T X
  KS_TRY(launch_gram_pair(P, base_eb(P), d, e, X32, p, p, sm(P, S_DS), sm(P, S_E1)));
  KS_TRY(launch_add_pp(P, sm(P, S_SB), 1.0, sm(P, S_DS), sm(P, S_S)));      // S
  KS_TRY(launch_combine<float>(P, d, p, sm(P, S_SB), X32, p, sm(P, S_DS), -1.0, 1.0, Gi, D, p));
  KS_TRY(launch_mass_dots<float>(P, D, MD, d, Md, prev, P.scal + SC_DNORM2));
  KS_TRY(launch_gram_dual(P, D, X32, MD, p, p, sm(P, S_DMD), sm(P, S_XMD),  // D^T MD, X^T MD
                          P.rt32));
  if (retraction != KS_QR) {
    KS_TRY(launch_transpose(P, sm(P, S_S), sm(P, S_A)));
    // E_X^T D = E_b^T D + e^T D
    KS_TRY(launch_gram_pair(P, base_eb(P), D, e, D, p, p, sm(P, S_B), sm(P, S_E1)));
    KS_TRY(launch_small_gemm(P, 0, sm(P, S_S), 0, sm(P, S_S), 1.0, 1.0, sm(P, S_B)));  // + S S
    // X^T M X = I up to the increment's rounding
    KS_CUDA_TRY(cudaMemsetAsync(sm(P, S_O), 0, (size_t)p * p * sizeof(double), P.stream));
    KS_TRY(launch_add_identity(P, sm(P, S_O), 1.0, sm(P, S_O)));
  }
  KS_TRY(sync_scalars(P));
  tr->dnorm2 = P.scal_host[SC_DNORM2];
  if (prev) {
    tr->ss = P.scal_host[SC_BB_SS];
    tr->sy = P.scal_host[SC_BB_SY];
    tr->yy = P.scal_host[SC_BB_YY];
  }
  if (!std::isfinite(tr->dnorm2)) return set_error(KS_ENAN, "non-finite gradient norm");
  return KS_OK;
}

// Trial increment in block bt from the iterate in block bx along -D (QR) or
// along the Cayley curve, with its FP32 copy X32 = X_b + delta+.  Both steps
// are written on the basis [X, D], X+ = X A + D B, and A, B are
// right-multiplied by L^{-T} with L L^T = Y^T M Y formed exactly from
// X^T M X = I, T = X^T M D and R = D^T M D (p x p Grams):
//   QR:     A = I, B = -tau I; Y^T M Y = I - tau (T + T^T) + tau^2 R
//           (Alg. ChQR with the explicit Y^T M Y).
//   Cayley: X+ = X C1 + G C2 (Eq. WY3) with G = D + X S gives A = C1 + S C2,
//           B = C2; Y^T M Y = A^T A + A^T T B + B^T T^T A + B^T R B.
// The first-order term matters here.  With a drift eta = X^T M X - I the
// projected gradient has X^T M D = -eta S, and Prop. 3.1's I + tau^2 R
// would carry eta into the trial as eta + tau (eta S + S eta): growth by
// about 1 + 2 tau ||S|| per step (the Lagrange multipliers reach ~27 per
// orbital on the 64^3 system, about 100x over the 32 steps between
// refreshes), and an energy error of order tr(Lambda eta) that the line
// search sees.  With the measured T the trial keeps X^T M X - I = eta.  The
// increment is then delta+ = X_b (A - I) + delta A + D B, with A - I formed
// in FP64.
static ks_status retract_split(Problem &P, int retraction, int bx, const float *D, double tau,
                               int bt) {
  const int p = P.p;
  const size_t pp = (size_t)p * p * sizeof(double);
  const double *Ac, *Bc;
  float *dt = lower32(P, bt), *xt = upper32(P, bt);
  P.rho_block = -1;
  if (retraction == KS_QR && qr_factor_dev_applies(P) && combine3_f32_applies(P, p, p, p, p)) {
    // the factor as deviations from I in FP32 (with the coefficient image),
    // then one pass: delta+, its FP32 copy X_b + delta+ and the trial's density
    KS_TRY(launch_qr_factor_dev(P, P.rt32, tau));
    KS_TRY(launch_combine3_f32(P, base_hi(P), p, sm(P, S_T), lower32(P, bx), p, sm(P, S_C1), D,
                               p, sm(P, S_C2), dt, base_hi(P), xt, p, P.rho_b, P.rho, true));
    P.rho_block = bt;
    return KS_OK;
  }
  if (retraction == KS_QR) {
    KS_TRY(launch_qr_exact_gram(P, sm(P, S_DMD), sm(P, S_XMD), tau, sm(P, S_E1)));
    KS_TRY(launch_qr_factor(P, sm(P, S_E1), nullptr, tau, sm(P, S_C1), sm(P, S_C2)));
    Ac = sm(P, S_C1);
    Bc = sm(P, S_C2);
  } else {
    double *A = sm(P, S_C1), *B = sm(P, S_C2);
    double *E1 = sm(P, S_E1), *E2 = sm(P, S_E2), *E3 = sm(P, S_E3);
    KS_TRY(launch_cayley_factor(P, sm(P, S_A), sm(P, S_S), sm(P, S_B), sm(P, S_O), tau, E1, B));
    KS_CUDA_TRY(cudaMemcpyAsync(A, E1, pp, cudaMemcpyDeviceToDevice, P.stream));
    KS_TRY(launch_small_gemm(P, 0, sm(P, S_S), 0, B, 1.0, 1.0, A));        // A = C1 + S C2
    KS_TRY(launch_small_gemm(P, 0, sm(P, S_XMD), 0, B, 1.0, 0.0, E2));     // T B
    KS_TRY(launch_small_gemm(P, 1, A, 0, E2, 1.0, 0.0, E1));               // A^T T B
    KS_TRY(launch_small_gemm(P, 0, sm(P, S_DMD), 0, B, 1.0, 0.0, E3));     // R B
    KS_TRY(launch_small_gemm(P, 1, B, 0, E3, 1.0, 0.0, E2));               // B^T R B
    KS_TRY(launch_small_gemm(P, 1, A, 0, A, 1.0, 1.0, E2));                // + A^T A
    KS_TRY(launch_sym_add(P, E2, E1, E3));                                 // Y^T M Y
    KS_TRY(launch_qr_factor(P, nullptr, E3, 0.0, E1, nullptr));            // L^{-T}
    KS_TRY(launch_small_gemm(P, 0, A, 0, E1, 1.0, 0.0, E3));               // A L^{-T}
    KS_TRY(launch_small_gemm(P, 0, B, 0, E1, 1.0, 0.0, E2));               // B L^{-T}
    Ac = E3;
    Bc = E2;
  }
  KS_TRY(launch_add_identity(P, Ac, -1.0, sm(P, S_T)));
  if (combine3_f32_applies(P, p, p, p, p)) {
    // one pass: delta+, its FP32 copy X_b + delta+ and the trial's density
    KS_TRY(launch_combine3_f32(P, base_hi(P), p, sm(P, S_T), lower32(P, bx), p, Ac, D, p, Bc, dt,
                               base_hi(P), xt, p, P.rho_b, P.rho));
    P.rho_block = bt;
    return KS_OK;
  }
  // X_b (A - I) + D B into the trial's upper half, then delta A added
  KS_TRY(launch_combine<float>(P, base_hi(P), p, sm(P, S_T), D, p, Bc, 1.0, 0.0, nullptr, xt, p));
  KS_TRY(launch_combine<float>(P, lower32(P, bx), p, Ac, nullptr, 0, nullptr, 1.0, 1.0, xt, dt,
                               p));
  return launch_axpy_f32(P, base_hi(P), 1.0f, dt, xt);
}

// The base absorbs the increment of block bx (gradient increment in block
// bex, M delta in bmx): X_b <- X_b + delta, formed in FP64 in block b64 and
// evaluated there in FP64 (energy *E, rho_b, V_b, E_b, T_b; the Hartree
// solve warm-started), re-M-orthonormalised when ||X_b^T M X_b - I||_F >
// kSplitOrthoTol (X_b <- X_b L^{-T}, applied as the small correction
// X_b (L^{-T} - I) formed in FP32, then evaluated again), then S_b and D_b
// are formed in FP64 (scratch: blocks bex and B_G), delta, M delta and e
// become 0, and the previous increment (block bxp, M delta in bmxp; -1: none)
// is re-expressed against the new base.  scratch: a free FP32 n x p block.
static ks_status rebase_split(Problem &P, int bx, int bmx, int bex, int bxp, int bmxp, int b64,
                              float *scratch, double *E) {
  const int p = P.p;
  double *xb = P.blk[b64];
  double *w1 = P.blk[bex];     // E_b, then D_b
  double *w2 = P.blk[B_G];     // M X_b, then M^{-1} E_b
  KS_TRY(launch_split_join(P, base_hi(P), base_lo(P), lower32(P, bx), xb));
  for (int pass = 0; pass < 2; ++pass) {
    KS_TRY(evaluate<double>(P, xb, w1, w2, E));
    KS_TRY(launch_gram<double>(P, xb, p, w2, p, sm(P, S_O)));
    KS_TRY(launch_ortho_err(P, sm(P, S_O), P.scal + SC_ORTHO));
    KS_TRY(sync_scalars(P));
    if (pass == 1 || std::sqrt(P.scal_host[SC_ORTHO]) <= kSplitOrthoTol) break;
    KS_TRY(launch_qr_factor(P, nullptr, sm(P, S_O), 0.0, sm(P, S_C1), nullptr));
    KS_TRY(launch_add_identity(P, sm(P, S_C1), -1.0, sm(P, S_T)));
    KS_TRY(launch_combine<float>(P, upper32(P, bx), p, sm(P, S_T), nullptr, 0, nullptr, 1.0, 0.0,
                                 nullptr, scratch, p));
    KS_TRY(launch_add_f64_f32(P, xb, scratch));
  }
  P.state.T_b = P.scal_host[SC_EKIN];
  KS_CUDA_TRY(cudaMemcpyAsync(P.rho_b, P.rho, (size_t)P.n * sizeof(double),
                              cudaMemcpyDeviceToDevice, P.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(P.veff_b, P.veff, (size_t)P.n * sizeof(double),
                              cudaMemcpyDeviceToDevice, P.stream));
  // S_b = E_b^T X_b and D_b = M^{-1} E_b - X_b S_b in FP64
  KS_TRY(launch_mass_inverse<double>(P, w1, w2));
  KS_TRY(launch_gram<double>(P, w1, p, xb, p, sm(P, S_SB)));
  KS_TRY(launch_convert(P, w1, base_eb(P)));
  KS_TRY(launch_combine<double>(P, xb, p, sm(P, S_SB), nullptr, 0, nullptr, -1.0, 1.0, w2, w1, p));
  KS_TRY(launch_convert(P, w1, base_db(P)));
  KS_TRY(launch_split_hilo(P, xb, base_hi(P), base_lo(P)));
  if (bxp >= 0) {
    KS_TRY(launch_axpy_f32(P, lower32(P, bxp), -1.0f, lower32(P, bx), lower32(P, bxp)));
    KS_TRY(launch_axpy_f32(P, lower32(P, bmxp), -1.0f, lower32(P, bmx), lower32(P, bmxp)));
  }
  const size_t b32 = (size_t)P.n * p * sizeof(float);
  KS_CUDA_TRY(cudaMemsetAsync(lower32(P, bx), 0, b32, P.stream));
  KS_CUDA_TRY(cudaMemsetAsync(lower32(P, bmx), 0, b32, P.stream));
  KS_CUDA_TRY(cudaMemsetAsync(lower32(P, bex), 0, b32, P.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(upper32(P, bx), base_hi(P), b32, cudaMemcpyDeviceToDevice,
                              P.stream));
  P.state.since_rebase = 0;
  return KS_OK;
}

// Alg. ConOptM in the increment form from the FP64 block Xstart (copied,
// then M-orthonormalised in FP64) -- or, with `resume`, from the saved
// state -- until ||D||_M <= gtol, maxit iterations in total, or (stall > 0)
// no 0.1 % improvement of the best ||D||_M for kStallWindow iterations (the
// limit of the FP32 direction).  The final X = X_b + delta is written to
// Xend in FP64.  The line search treats the energies like FP64 ones
// (rounding slack and restart of the reference after a forced acceptance).
static ks_status run_phase_split(Problem &P, const double *Xstart, double *Xend,
                                 const ks_opts &o, double gtol, int maxit, int stall,
                                 bool resume, PhaseResult *out) {
  const int p = P.p;
  Problem::RunState &S = P.state;
  int ix[3] = {B_X0, B_X1, B_X2};
  int imx[3] = {B_MX0, B_MX1, B_MX2};
  int iex[2] = {B_EX0, B_EX1};
  int id[2] = {B_D0, B_D1};
  int imd[2] = {B_MD0, B_MD1};
  auto MD_ = [&](int s) { return lower32(P, imx[s]); };
  auto EX = [&](int s) { return lower32(P, iex[s]); };   // gradient increments e
  auto D = [&](int s) { return lower32(P, id[s]); };
  auto MDd = [&](int s) { return lower32(P, imd[s]); };
  double E = 0, C = 0, Q = 1.0, best = 0;
  int k = 0, last_improve = 0, cg_total = 0;
  bool have_prev = false;
  Traces tr;
  P.cg_tol_phase = 0.0;
  if (resume) {
    for (int i = 0; i < 3; ++i) { ix[i] = S.ix[i]; imx[i] = S.imx[i]; }
    for (int i = 0; i < 2; ++i) { iex[i] = S.iex[i]; id[i] = S.id[i]; imd[i] = S.imd[i]; }
    k = S.k;
    E = S.E; C = S.C; Q = S.Q; best = S.best; last_improve = S.last_improve;
    out->last_tau = S.last_tau;
    have_prev = S.have_prev != 0;
    P.vH_valid = true;
    BBPrevT<float> prev{lower32(P, ix[1]), MD_(1), D(1), MDd(1)};
    KS_TRY(project_split(P, S.retraction, ix[0], EX(0), MD_(0), D(0), MDd(0),
                         have_prev ? &prev : nullptr, &tr));
  } else {
    // FP64 start: X_b = CholQR2(Xstart) in block ix[2], delta = 0
    double *x64 = P.blk[ix[2]];
    KS_CUDA_TRY(cudaMemcpyAsync(x64, Xstart, (size_t)P.n * p * sizeof(double),
                                cudaMemcpyDeviceToDevice, P.stream));
    KS_TRY(orthonormalize<double>(P, x64, P.blk[iex[1]], P.blk[B_G], 2));
    KS_TRY(launch_split_hilo(P, x64, base_hi(P), base_lo(P)));
    KS_CUDA_TRY(cudaMemsetAsync(lower32(P, ix[0]), 0, (size_t)P.n * p * sizeof(float),
                                P.stream));
    KS_CUDA_TRY(cudaMemcpyAsync(upper32(P, ix[0]), base_hi(P), (size_t)P.n * p * sizeof(float),
                                cudaMemcpyDeviceToDevice, P.stream));
    KS_TRY(rebase_split(P, ix[0], imx[0], iex[0], -1, -1, ix[2], MD_(2), &E));
    cg_total = P.last_cg_iters;
    KS_TRY(project_split(P, o.retraction, ix[0], EX(0), MD_(0), D(0), MDd(0), nullptr, &tr));
    C = E;
    best = std::sqrt(std::fmax(tr.dnorm2, 0.0));
    S.since_rebase = 0;
  }
  const int k0 = k;
  int backtracks = 0;
  bool stalled = false;
  auto save_state = [&]() {
    S.valid = true;
    S.elem = 4;
    S.split = 1;
    S.retraction = o.retraction;
    S.first_k = 0;
    S.k = k;
    S.have_prev = have_prev ? 1 : 0;
    S.C = C; S.Q = Q; S.E = E; S.best = best; S.last_improve = last_improve;
    S.last_tau = out->last_tau;
    S.dnorm2 = tr.dnorm2; S.ss = tr.ss; S.sy = tr.sy; S.yy = tr.yy;
    for (int i = 0; i < 3; ++i) { S.ix[i] = ix[i]; S.imx[i] = imx[i]; }
    for (int i = 0; i < 2; ++i) { S.iex[i] = iex[i]; S.id[i] = id[i]; S.imd[i] = imd[i]; }
  };
  save_state();
  while (std::sqrt(std::fmax(tr.dnorm2, 0.0)) > gtol && k < maxit) {
    double tau = have_prev ? bb_step(k, tr, o) : o.tau0;
    int h = 0;
    double Et = 0;
    bool forced = false;
    for (;;) {
      KS_TRY(retract_split(P, o.retraction, ix[0], D(0), tau, ix[2]));
      KS_TRY(evaluate_split(P, ix[2], EX(1), MD_(2), &Et));
      cg_total += P.last_cg_iters;
      const bool ok = Et <= C - o.rho1 * tau * tr.dnorm2 + armijo_slack<double>(P.last_parts);
      if (ok || h == o.max_backtrack) {
        forced = !ok;
        break;
      }
      tau *= o.delta;
      ++h;
    }
    backtracks += h;
    out->last_tau = tau;
    const double Qn = o.eta * Q + 1.0;
    C = (o.eta * Q * C + Et) / Qn;
    Q = Qn;
    if (forced) {
      C = Et;
      Q = 1.0;
    }
    std::swap(ix[1], ix[0]);
    std::swap(ix[0], ix[2]);
    std::swap(imx[1], imx[0]);
    std::swap(imx[0], imx[2]);
    std::swap(iex[0], iex[1]);
    std::swap(id[0], id[1]);
    std::swap(imd[0], imd[1]);
    E = Et;
    ++k;
    if (++S.since_rebase >= kRebaseEvery) {
      // the base absorbs the increment (an FP64 evaluation at the same point)
      KS_TRY(rebase_split(P, ix[0], imx[0], iex[0], ix[1], imx[1], ix[2], MD_(2), &E));
      cg_total += P.last_cg_iters;
    }
    BBPrevT<float> prev{lower32(P, ix[1]), MD_(1), D(1), MDd(1)};
    KS_TRY(project_split(P, o.retraction, ix[0], EX(0), MD_(0), D(0), MDd(0), &prev, &tr));
    have_prev = true;
    const double dn = std::sqrt(std::fmax(tr.dnorm2, 0.0));
    if (dn < 0.999 * best) {
      best = dn;
      last_improve = k;
    }
    // the direction is accurate to FP32 rounding relative to ||D||, so the
    // phase has no floor above gtol to detect: only a run whose best ||D||
    // stays put for kSplitStallWindow iterations (far longer than the
    // plateaus of the BB iteration on slowly converging systems) hands over
    bool stop = false;
    if (stall > 0 && k - last_improve >= kSplitStallWindow) {
      stalled = true;
      stop = true;
    }
    save_state();
    if (o.verbose > 0 && k % o.verbose == 0)
      fprintf(stderr, "ks_minimize[fp32+base]: k=%d E=%.12f |D|=%.3e tau=%.3e h=%d cg=%d\n", k, E,
              dn, tau, h, P.last_cg_iters);
    if (stop) break;
  }
  KS_TRY(launch_split_join(P, base_hi(P), base_lo(P), lower32(P, ix[0]), Xend));
  out->E = E;
  out->dnorm = std::sqrt(std::fmax(tr.dnorm2, 0.0));
  out->iters = k - k0;
  out->cg = cg_total;
  out->backtracks = backtracks;
  out->stalled = stalled;
  return KS_OK;
}

static ks_status minimize_device(Problem &P, double *X_inout, const ks_opts &o, ks_result *res,
                                 bool resume) {
  const auto t0 = std::chrono::steady_clock::now();
  PhaseResult fr;
  int iters = 0, cg = 0, backtracks = 0;
  const bool resume_fp32 = resume && P.state.elem == 4;
  bool resume_fp64 = resume && P.state.elem == 8;
  int done = resume ? P.state.first_k + P.state.k : 0;   // iterations before this call
  double polish_tau = 0.0;
  if (o.precision == KS_MIXED && (!resume || resume_fp32)) {
    PhaseResult mr;
    const bool inc = resume ? P.state.split != 0 : o.fp32_increment != 0;
    bool limit_hit = false;
    if (inc) {
      // FP32 phase in increment form (X = X_b + delta), to gtol or until the
      // FP32 direction stops improving; the result is written to X_inout in
      // FP64
      const ks_status pst = run_phase_split(P, X_inout, X_inout, o, o.gtol, o.maxit,
                                            o.stall_iters, resume_fp32, &mr);
      KS_TRY(pst);
      P.mixed_iters = P.state.k;
      limit_hit = P.mixed_iters >= o.maxit && !mr.stalled && mr.dnorm > o.gtol;
    } else {
      // FP32 phase (Hartree, energy sums and p x p algebra stay FP64), then
      // an FP64 polish from its last iterate.
      float *xs = blk<float>(P, B_G);
      if (!resume) KS_TRY(launch_convert(P, X_inout, xs));
      P.cg_tol_phase = o.mixed_cg_tol > P.cg_tol ? std::fmin(o.mixed_cg_tol, 1e-3) : 0.0;
      const ks_status pst = run_phase<float>(P, xs, xs, o, std::fmax(o.polish_gtol, o.gtol),
                                             o.maxit, o.stall_iters, 0,
                                             std::fmax(o.ortho_tol, 1e-5), resume_fp32, &mr);
      P.cg_tol_phase = 0.0;
      KS_TRY(pst);
      P.mixed_iters = P.state.first_k + P.state.k;
      double *xd = blk<double>(P, B_MD1);
      KS_TRY(launch_convert(P, xs, xd));
      KS_CUDA_TRY(cudaMemcpyAsync(X_inout, xd, (size_t)P.n * P.p * sizeof(double),
                                  cudaMemcpyDeviceToDevice, P.stream));
      limit_hit = P.mixed_iters >= o.maxit && !mr.stalled &&
                  mr.dnorm > std::fmax(o.polish_gtol, o.gtol);
    }
    iters += mr.iters;
    cg += mr.cg;
    backtracks += mr.backtracks;
    polish_tau = mr.last_tau;
    P.mixed_dnorm = mr.dnorm;
    P.mixed_E = mr.E;
    done = P.mixed_iters;
    resume_fp64 = false;
    if (limit_hit) {
      // iteration limit inside the FP32 phase: no polish; the FP32 state
      // stays resumable and X_inout holds the FP32 iterate in FP64
      if (res) {
        res->E = mr.E;
        res->gradnorm = mr.dnorm;
        res->ortho_err = -1.0;
        for (int i = 0; i < 5; ++i) res->E_parts[i] = P.last_parts[i];
        res->iters = iters;
        res->cg_iters_total = cg;
        res->backtracks = backtracks;
        res->status = KS_ENOCONV;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        res->mixed_iters = P.mixed_iters;
        res->mixed_gradnorm = P.mixed_dnorm;
        res->mixed_E = P.mixed_E;
      }
      KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
      return set_error(KS_ENOCONV, "iteration limit reached in the FP32 phase");
    }
  } else if (resume && o.precision != KS_MIXED && P.state.elem != 8) {
    return set_error(KS_EINVAL, "saved state is from an FP32 phase; resume it with KS_MIXED");
  }
  // the polish continues with the FP32 phase's last accepted step instead
  // of restarting from tau0
  KS_TRY(run_phase<double>(P, X_inout, X_inout, o, o.gtol, o.maxit, 0, done, o.ortho_tol,
                           resume_fp64, &fr, polish_tau));
  iters += fr.iters;
  cg += fr.cg;
  backtracks += fr.backtracks;
  const ks_status status = fr.dnorm > o.gtol ? KS_ENOCONV : KS_OK;
  double oerr = 0;
  KS_TRY(launch_mass<double>(P, X_inout, blk<double>(P, B_G)));
  KS_TRY(ortho_error<double>(P, X_inout, blk<double>(P, B_G), &oerr));
  if (res) {
    res->E = fr.E;
    res->gradnorm = fr.dnorm;
    res->ortho_err = oerr;
    for (int i = 0; i < 5; ++i) res->E_parts[i] = P.last_parts[i];
    res->iters = iters;
    res->cg_iters_total = cg;
    res->backtracks = backtracks;
    res->status = status;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    res->mixed_iters = o.precision == KS_MIXED ? P.mixed_iters : 0;
    res->mixed_gradnorm = o.precision == KS_MIXED ? P.mixed_dnorm : 0.0;
    res->mixed_E = o.precision == KS_MIXED ? P.mixed_E : 0.0;
  }
  if (status != KS_OK) set_error(status, "gradient norm above gtol after %d iterations", iters);
  return status;
}

// Checkpoint layout: header, then the current X, MX, E_X, D, MD and the
// previous X, MX, D, MD blocks (elem bytes per entry), then vH (FP64).  A
// state of the FP32 phase in increment form (split = 1) instead holds all
// n x p blocks at full capacity in their own slots (the base quantities share
// them with the increments), then vH, rho_b, V_b and S_b.  Both end with the
// Hartree solver's last residual and right-hand side (cg_r, cg_rho_prev),
// so that a resumed run starts its next solve exactly like the original.
struct StateHeader {
  uint64_t magic;
  int32_t version, N, p, elem, retraction, first_k, k, have_prev, last_improve;
  double C, Q, E, dnorm2, ss, sy, yy, best, last_tau;
  int32_t split, since_rebase;
  double T_b;
  int32_t slots[13];
  int32_t cg_inc_ok, cg_inc_count;
};
constexpr uint64_t kStateMagic = 0x4b53535441544531ull;   // "KSSTATE1"

static size_t block_capacity(const Problem &P) { return ((size_t)P.n * P.p + 32) * sizeof(double); }

static size_t state_bytes(const Problem &P, int elem, int split) {
  const size_t cg = (size_t)2 * P.n * sizeof(double);
  if (split)
    return sizeof(StateHeader) + (size_t)Problem::kNBlocks * block_capacity(P) +
           (size_t)3 * P.n * sizeof(double) + (size_t)P.p * P.p * sizeof(double) + cg;
  return sizeof(StateHeader) + (size_t)9 * P.n * P.p * elem + (size_t)P.n * sizeof(double) + cg;
}

// The Hartree solver's residual and right-hand side, after the rest.
static ks_status save_cg(Problem &P, char *dst) {
  KS_CUDA_TRY(cudaMemcpyAsync(dst, P.cg_r, (size_t)P.n * sizeof(double), cudaMemcpyDeviceToHost,
                              P.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(dst + (size_t)P.n * sizeof(double), P.cg_rho_prev,
                              (size_t)P.n * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
  return KS_OK;
}

static ks_status load_cg(Problem &P, const char *src) {
  KS_CUDA_TRY(cudaMemcpyAsync(P.cg_r, src, (size_t)P.n * sizeof(double), cudaMemcpyHostToDevice,
                              P.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(P.cg_rho_prev, src + (size_t)P.n * sizeof(double),
                              (size_t)P.n * sizeof(double), cudaMemcpyHostToDevice, P.stream));
  return KS_OK;
}

}  // namespace ks

using namespace ks;

extern "C" {

void ks_opts_default(ks_opts *o) {
  if (!o) return;
  o->retraction = KS_QR;
  o->gtol = 1e-6;
  o->maxit = 300;
  o->tau0 = 1e-3;
  o->rho1 = 1e-4;
  o->delta = 0.1;
  o->eta = 0.85;
  o->tau_min = 1e-10;
  o->tau_max = 1e10;
  o->max_backtrack = 10;
  o->ortho_tol = 1e-12;
  o->ortho_every = 20;
  o->verbose = 0;
  o->precision = KS_FP64;
  o->polish_gtol = 1e-4;
  o->stall_iters = 1;
  o->stall_df = 1e-11;
  o->resume = 0;
  o->mixed_cg_tol = 1e-7;
  o->fp64_split = 0;
  o->fp32_increment = 1;
}

const char *ks_last_error_string(void) { return g_err; }

size_t ks_problem_bytes(const ks_problem_desc *d) {
  if (validate_desc(d) != KS_OK) return 0;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  return problem_bytes(d->N, d->p, sms);
}

ks_status ks_problem_create(const ks_problem_desc *d, ks_problem **out) {
  if (!out) return set_error(KS_EINVAL, "null output handle");
  *out = nullptr;
  KS_TRY(validate_desc(d));
  ks_problem *kp = new (std::nothrow) ks_problem();
  if (!kp) return set_error(KS_ENOMEM, "host allocation failed");
  Problem &P = kp->P;
  auto fail = [&](ks_status st) {
    free_problem(P);
    delete kp;
    return st;
  };
  P.N = d->N;
  P.n = d->N * d->N * d->N;
  P.p = d->p;
  P.natoms = d->natoms;
  P.xc = d->xc;
  P.L = d->L;
  P.h = d->L / (d->N + 1);
  P.rc = d->rc;
  P.occ = d->occ;
  P.kinetic = d->kinetic;
  P.mass = d->mass;
  if (d->kinetic == KS_KIN_TFW) {
    P.kin_w = d->mu;
    P.ctf = 0.3 * std::pow(3.0 * M_PI * M_PI, 2.0 / 3.0);   // Eq. TFW's C_TF
  }
  P.cg_tol = d->cg_tol;
  P.cg_maxit = d->cg_maxit;
  P.cg_precond = d->cg_precond ? 1 : 0;
  P.atoms_host.resize((size_t)4 * (d->natoms > 0 ? d->natoms : 1), 0.0);
  for (int a = 0; a < d->natoms; ++a) {
    P.atoms_host[4 * a + 0] = d->R[3 * a + 0];
    P.atoms_host[4 * a + 1] = d->R[3 * a + 1];
    P.atoms_host[4 * a + 2] = d->R[3 * a + 2];
    P.atoms_host[4 * a + 3] = d->Z[a];
  }
  cudaError_t e = cudaGetDevice(&P.device);
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&P.sms, cudaDevAttrMultiProcessorCount, P.device);
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaDeviceGetAttribute"));
  if (d->stream) {
    P.stream = (cudaStream_t)d->stream;
  } else {
    e = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaStreamCreate"));
    P.own_stream = true;
  }
  const size_t n = P.n, np = (size_t)P.n * P.p;
  ks_status st;
#define ALLOC(ptr, cnt) \
  if ((st = dalloc(&(ptr), (cnt), P)) != KS_OK) return fail(st);
  ALLOC(P.vext, n); ALLOC(P.rho, n); ALLOC(P.vH, n); ALLOC(P.veff, n);
  ALLOC(P.rho_b, n); ALLOC(P.veff_b, n); ALLOC(P.zero_n, n);
  ALLOC(P.cg_r, n); ALLOC(P.cg_pa, n); ALLOC(P.cg_pb, n); ALLOC(P.cg_q, n); ALLOC(P.cg_z, n);
  ALLOC(P.cg_rho_prev, n);
  ALLOC(P.cg_t1, n); ALLOC(P.cg_t2, n);
  ALLOC(P.dst_phi, (size_t)P.N * P.N); ALLOC(P.dst_kap, (size_t)P.N); ALLOC(P.dst_mu, (size_t)P.N);
  // FP64 capacity plus 256 bytes, so that an FP32 block fits in the upper
  // half at a 256-byte aligned offset
  P.half_off = (np * sizeof(float) + 255) / 256 * 256;
  for (auto &b : P.blk) { ALLOC(b, np + 32); }
  P.pp_len = (size_t)S_COUNT * P.p * P.p;
  ALLOC(P.pp, P.pp_len);
  ALLOC(P.cf, (size_t)3 * P.p * P.p);
  ALLOC(P.rt32, (size_t)2 * P.p * P.p);
  P.tc_img_len = tc_image_floats(P.p);
  ALLOC(P.tc_img, P.tc_img_len);
  P.oz_emax_len = 2 * P.p + 128;
  ALLOC(P.oz_emax, (size_t)P.oz_emax_len);
  ALLOC(P.oz_img, oz_image_bytes(P.p));
  ALLOC(P.oz_rowexp, n);
  P.cg_blocks = cg_grid_blocks(P.sms, P.n, P.N);
  if (P.cg_blocks < 1) return fail(set_error(KS_ECUDA, "CG kernel configuration failed"));
  size_t part = gram_partials_len(P.p, P.sms);
  if ((size_t)4 * 8 * P.sms > part) part = (size_t)4 * 8 * P.sms;
  if ((size_t)4 * P.cg_blocks > part) part = (size_t)4 * P.cg_blocks;
  P.partials_len = part;
  ALLOC(P.partials, part);
  ALLOC(P.scal, SC_COUNT);
  ALLOC(P.atoms_dev, P.atoms_host.size());
  ALLOC(P.thomas_w, (size_t)P.N);
  ALLOC(P.bar, 1);
  ALLOC(P.red_counter, 1);
  ALLOC(P.dstatus, 1);
#undef ALLOC
  P.scal_host = new (std::nothrow) double[SC_COUNT];
  P.dstatus_host = new (std::nothrow) int[1];
  if (!P.scal_host || !P.dstatus_host) return fail(set_error(KS_ENOMEM, "host allocation failed"));
  e = cudaMemcpyAsync(P.atoms_dev, P.atoms_host.data(), P.atoms_host.size() * sizeof(double),
                      cudaMemcpyHostToDevice, P.stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "copy atoms"));
  e = cudaMemsetAsync(P.scal, 0, SC_COUNT * sizeof(double), P.stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "memset"));
  e = cudaMemsetAsync(P.red_counter, 0, sizeof(unsigned int), P.stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "memset"));
  e = cudaMemsetAsync(P.dstatus, 0, sizeof(int), P.stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "memset"));
  e = cudaMemsetAsync(P.vH, 0, n * sizeof(double), P.stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "memset"));
  e = cudaMemsetAsync(P.zero_n, 0, n * sizeof(double), P.stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "memset"));
  if ((st = configure_small_kernels()) != KS_OK) return fail(st);
  if ((st = configure_tc_kernels()) != KS_OK) return fail(st);
  if ((st = configure_blas_kernels()) != KS_OK) return fail(st);
  if ((st = launch_setup(P)) != KS_OK) return fail(st);
  if ((st = launch_sine_setup(P)) != KS_OK) return fail(st);
  if ((st = sync_scalars(P)) != KS_OK) return fail(st);
  *out = kp;
  return KS_OK;
}

ks_status ks_problem_destroy(ks_problem *kp) {
  if (!kp) return KS_OK;
  if (kp->P.stream) cudaStreamSynchronize(kp->P.stream);
  free_problem(kp->P);
  delete kp;
  return KS_OK;
}

ks_status ks_energy_grad(ks_problem *kp, const double *X, double *E, double *EX, double *D,
                         double *gradnorm) {
  if (!kp || !X || !E) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  P.state.valid = false;   // the workspace below holds the saved state's blocks
  const size_t bytes = (size_t)P.n * P.p * sizeof(double);
  double e = 0;
  KS_TRY(evaluate<double>(P, X, P.blk[B_EX0], P.blk[B_MX0], &e));
  if (D || gradnorm) {
    Traces tr;
    KS_TRY(project<double>(P, KS_QR, X, P.blk[B_EX0], P.blk[B_MX0], P.blk[B_D0], P.blk[B_MD0],
                           nullptr, &tr));
    if (gradnorm) *gradnorm = std::sqrt(std::fmax(tr.dnorm2, 0.0));
    if (D) KS_CUDA_TRY(cudaMemcpyAsync(D, P.blk[B_D0], bytes, cudaMemcpyDeviceToDevice, P.stream));
  }
  if (EX) KS_CUDA_TRY(cudaMemcpyAsync(EX, P.blk[B_EX0], bytes, cudaMemcpyDeviceToDevice, P.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  *E = e;
  return KS_OK;
}

ks_status ks_energy_parts(ks_problem *kp, double parts[5]) {
  if (!kp || !parts) return set_error(KS_EINVAL, "null argument");
  for (int i = 0; i < 5; ++i) parts[i] = kp->P.last_parts[i];
  return KS_OK;
}

ks_status ks_retract(ks_problem *kp, int kind, const double *X, const double *EX, double tau,
                     double *Xout) {
  if (!kp || !X || !EX || !Xout) return set_error(KS_EINVAL, "null argument");
  if (kind != KS_QR && kind != KS_CAYLEY) return set_error(KS_EINVAL, "bad retraction kind");
  if (Xout == X || Xout == EX) return set_error(KS_EINVAL, "Xout aliases an input");
  Problem &P = kp->P;
  P.state.valid = false;
  KS_TRY(launch_mass<double>(P, X, P.blk[B_MX0]));
  Traces tr;
  KS_TRY(project<double>(P, kind, X, EX, P.blk[B_MX0], P.blk[B_D0], P.blk[B_MD0], nullptr, &tr));
  KS_TRY(retract<double>(P, kind, X, P.blk[B_D0], tau, P.blk[B_X2]));
  KS_TRY(sync_scalars(P));
  KS_CUDA_TRY(cudaMemcpyAsync(Xout, P.blk[B_X2], (size_t)P.n * P.p * sizeof(double),
                              cudaMemcpyDeviceToDevice, P.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return KS_OK;
}

ks_status ks_orthonormalize(ks_problem *kp, double *X) {
  if (!kp || !X) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  P.state.valid = false;
  // work on a copy, so that X is left unchanged when the factor fails
  const size_t bytes = (size_t)P.n * P.p * sizeof(double);
  double *W = P.blk[B_X1];
  KS_CUDA_TRY(cudaMemcpyAsync(W, X, bytes, cudaMemcpyDeviceToDevice, P.stream));
  KS_TRY(orthonormalize<double>(P, W, P.blk[B_X2], P.blk[B_MX2], 2));
  KS_CUDA_TRY(cudaMemcpyAsync(X, W, bytes, cudaMemcpyDeviceToDevice, P.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return KS_OK;
}

ks_status ks_minimize(ks_problem *kp, double *X_inout, const ks_opts *opts, ks_result *res) {
  if (!kp || !X_inout) return set_error(KS_EINVAL, "null argument");
  ks_opts o;
  if (opts) o = *opts;
  else ks_opts_default(&o);
  if (o.retraction != KS_QR && o.retraction != KS_CAYLEY)
    return set_error(KS_EINVAL, "bad retraction");
  if (o.precision != KS_FP64 && o.precision != KS_MIXED) return set_error(KS_EINVAL, "bad precision");
  if (!(o.delta > 0.0 && o.delta < 1.0) || !(o.eta >= 0.0 && o.eta < 1.0) || o.maxit < 0 ||
      !(o.tau0 > 0.0) || o.max_backtrack < 0)
    return set_error(KS_EINVAL, "bad line-search parameters");
  if (o.resume && !kp->P.state.valid) return set_error(KS_EINVAL, "no saved state to resume");
  if (o.fp64_split < 0 || o.fp64_split > 2) return set_error(KS_EINVAL, "bad fp64_split");
  if (!o.resume) kp->P.vH_valid = false;
  const int use_oz = kp->P.use_oz;
  if (o.fp64_split > 0) kp->P.use_oz = o.fp64_split;
  const ks_status st = minimize_device(kp->P, X_inout, o, res, o.resume != 0);
  kp->P.use_oz = use_oz;
  return st;
}

ks_status ks_minimize_host(ks_problem *kp, double *Xh, const ks_opts *opts, ks_result *res) {
  if (!kp || !Xh) return set_error(KS_EINVAL, "null argument");
  const auto t0 = std::chrono::steady_clock::now();
  Problem &P = kp->P;
  const size_t bytes = (size_t)P.n * P.p * sizeof(double);
  // The driver reads its input block only before the first iteration and
  // writes its output only after the last one, so the block B_D1 (a
  // previous-gradient slot during the iterations) can stage the host copy.
  if (opts && opts->resume)
    return set_error(KS_EINVAL, "resume needs the device entry point ks_minimize");
  double *dX = P.blk[B_D1];
  KS_CUDA_TRY(cudaMemcpyAsync(dX, Xh, bytes, cudaMemcpyHostToDevice, P.stream));
  ks_status st = ks_minimize(kp, dX, opts, res);
  // the staging block may be one of the saved state's slots
  P.state.valid = false;
  if (st != KS_OK && st != KS_ENOCONV) return st;
  KS_CUDA_TRY(cudaMemcpyAsync(Xh, dX, bytes, cudaMemcpyDeviceToHost, P.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  if (res)
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

size_t ks_state_bytes(ks_problem *kp) {
  if (!kp || !kp->P.state.valid) return 0;
  return state_bytes(kp->P, kp->P.state.elem, kp->P.state.split);
}

ks_status ks_state_save(ks_problem *kp, void *host_buf, size_t bytes) {
  if (!kp || !host_buf) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  const Problem::RunState &S = P.state;
  if (!S.valid) return set_error(KS_EINVAL, "no minimisation state to save");
  if (bytes < state_bytes(P, S.elem, S.split)) return set_error(KS_EINVAL, "buffer too small");
  StateHeader hd{};
  hd.magic = kStateMagic;
  hd.version = 4;
  hd.cg_inc_ok = P.cg_inc_ok ? 1 : 0;
  hd.cg_inc_count = P.cg_inc_count;
  hd.split = S.split; hd.since_rebase = S.since_rebase; hd.T_b = S.T_b;
  for (int i = 0; i < 3; ++i) { hd.slots[i] = S.ix[i]; hd.slots[3 + i] = S.imx[i]; }
  for (int i = 0; i < 2; ++i) {
    hd.slots[6 + i] = S.iex[i]; hd.slots[8 + i] = S.id[i]; hd.slots[10 + i] = S.imd[i];
  }
  hd.N = P.N; hd.p = P.p; hd.elem = S.elem; hd.retraction = S.retraction;
  hd.first_k = S.first_k; hd.k = S.k; hd.have_prev = S.have_prev; hd.last_improve = S.last_improve;
  hd.C = S.C; hd.Q = S.Q; hd.E = S.E; hd.dnorm2 = S.dnorm2;
  hd.ss = S.ss; hd.sy = S.sy; hd.yy = S.yy; hd.best = S.best; hd.last_tau = S.last_tau;
  char *dst = (char *)host_buf;
  std::memcpy(dst, &hd, sizeof(hd));
  dst += sizeof(hd);
  if (S.split) {
    for (int b = 0; b < Problem::kNBlocks; ++b) {
      KS_CUDA_TRY(cudaMemcpyAsync(dst, P.blk[b], block_capacity(P), cudaMemcpyDeviceToHost,
                                  P.stream));
      dst += block_capacity(P);
    }
    KS_CUDA_TRY(cudaMemcpyAsync(dst, P.vH, (size_t)P.n * sizeof(double), cudaMemcpyDeviceToHost,
                                P.stream));
    dst += (size_t)P.n * sizeof(double);
    KS_CUDA_TRY(cudaMemcpyAsync(dst, P.rho_b, (size_t)P.n * sizeof(double),
                                cudaMemcpyDeviceToHost, P.stream));
    dst += (size_t)P.n * sizeof(double);
    KS_CUDA_TRY(cudaMemcpyAsync(dst, P.veff_b, (size_t)P.n * sizeof(double),
                                cudaMemcpyDeviceToHost, P.stream));
    dst += (size_t)P.n * sizeof(double);
    KS_CUDA_TRY(cudaMemcpyAsync(dst, sm(P, S_SB), (size_t)P.p * P.p * sizeof(double),
                                cudaMemcpyDeviceToHost, P.stream));
    dst += (size_t)P.p * P.p * sizeof(double);
    KS_TRY(save_cg(P, dst));
    KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
    return KS_OK;
  }
  const int order[9] = {S.ix[0], S.imx[0], S.iex[0], S.id[0], S.imd[0],
                        S.ix[1], S.imx[1], S.id[1], S.imd[1]};
  const size_t blkb = (size_t)P.n * P.p * S.elem;
  for (int i = 0; i < 9; ++i) {
    KS_CUDA_TRY(cudaMemcpyAsync(dst, P.blk[order[i]], blkb, cudaMemcpyDeviceToHost, P.stream));
    dst += blkb;
  }
  KS_CUDA_TRY(cudaMemcpyAsync(dst, P.vH, (size_t)P.n * sizeof(double), cudaMemcpyDeviceToHost,
                              P.stream));
  dst += (size_t)P.n * sizeof(double);
  KS_TRY(save_cg(P, dst));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return KS_OK;
}

ks_status ks_state_load(ks_problem *kp, const void *host_buf, size_t bytes) {
  if (!kp || !host_buf) return set_error(KS_EINVAL, "null argument");
  Problem &P = kp->P;
  StateHeader hd;
  if (bytes < sizeof(hd)) return set_error(KS_EINVAL, "buffer too small");
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != 4) return set_error(KS_EINVAL, "not a saved state");
  if (hd.N != P.N || hd.p != P.p || (hd.elem != 4 && hd.elem != 8) ||
      (hd.split != 0 && (hd.split != 1 || hd.elem != 4)))
    return set_error(KS_EINVAL, "saved state does not match this problem");
  if (bytes < state_bytes(P, hd.elem, hd.split)) return set_error(KS_EINVAL, "buffer too small");
  if (hd.split) {
    // the slots must be a permutation of the blocks with X, MX, E_X, D, MD
    // in their own families
    int seen = 0;
    const int lo[5] = {B_X0, B_MX0, B_EX0, B_D0, B_MD0}, cnt[5] = {3, 3, 2, 2, 2};
    int at = 0;
    for (int f = 0; f < 5; ++f)
      for (int i = 0; i < cnt[f]; ++i, ++at) {
        const int b = hd.slots[at];
        if (b < lo[f] || b >= lo[f] + cnt[f] || (seen & (1 << b)))
          return set_error(KS_EINVAL, "saved state has invalid block slots");
        seen |= 1 << b;
      }
  }
  Problem::RunState S;
  S.valid = true;
  S.elem = hd.elem; S.retraction = hd.retraction; S.first_k = hd.first_k; S.k = hd.k;
  S.have_prev = hd.have_prev; S.last_improve = hd.last_improve;
  S.C = hd.C; S.Q = hd.Q; S.E = hd.E; S.dnorm2 = hd.dnorm2;
  S.ss = hd.ss; S.sy = hd.sy; S.yy = hd.yy; S.best = hd.best; S.last_tau = hd.last_tau;
  if (hd.retraction != KS_QR && hd.retraction != KS_CAYLEY)
    return set_error(KS_EINVAL, "saved state has an unknown retraction");
  S.split = hd.split;
  S.since_rebase = hd.since_rebase;
  S.T_b = hd.T_b;
  // the blocks are overwritten below: a copy that fails leaves no state
  P.state.valid = false;
  P.rho_block = -1;
  P.cg_inc_ok = false;
  if (hd.split) {
    for (int i = 0; i < 3; ++i) { S.ix[i] = hd.slots[i]; S.imx[i] = hd.slots[3 + i]; }
    for (int i = 0; i < 2; ++i) {
      S.iex[i] = hd.slots[6 + i]; S.id[i] = hd.slots[8 + i]; S.imd[i] = hd.slots[10 + i];
    }
    const char *src = (const char *)host_buf + sizeof(hd);
    for (int b = 0; b < Problem::kNBlocks; ++b) {
      KS_CUDA_TRY(cudaMemcpyAsync(P.blk[b], src, block_capacity(P), cudaMemcpyHostToDevice,
                                  P.stream));
      src += block_capacity(P);
    }
    KS_CUDA_TRY(cudaMemcpyAsync(P.vH, src, (size_t)P.n * sizeof(double), cudaMemcpyHostToDevice,
                                P.stream));
    src += (size_t)P.n * sizeof(double);
    KS_CUDA_TRY(cudaMemcpyAsync(P.rho_b, src, (size_t)P.n * sizeof(double),
                                cudaMemcpyHostToDevice, P.stream));
    src += (size_t)P.n * sizeof(double);
    KS_CUDA_TRY(cudaMemcpyAsync(P.veff_b, src, (size_t)P.n * sizeof(double),
                                cudaMemcpyHostToDevice, P.stream));
    src += (size_t)P.n * sizeof(double);
    KS_CUDA_TRY(cudaMemcpyAsync(sm(P, S_SB), src, (size_t)P.p * P.p * sizeof(double),
                                cudaMemcpyHostToDevice, P.stream));
    src += (size_t)P.p * P.p * sizeof(double);
    KS_TRY(load_cg(P, src));
    KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
    P.state = S;
    P.cg_inc_ok = hd.cg_inc_ok != 0;
    P.cg_inc_count = hd.cg_inc_count;
    return KS_OK;
  }
  // canonical slots: current in slot 0, previous in slot 1
  const int order[9] = {B_X0, B_MX0, B_EX0, B_D0, B_MD0, B_X1, B_MX1, B_D1, B_MD1};
  const char *src = (const char *)host_buf + sizeof(hd);
  const size_t blkb = (size_t)P.n * P.p * hd.elem;
  for (int i = 0; i < 9; ++i) {
    KS_CUDA_TRY(cudaMemcpyAsync(P.blk[order[i]], src, blkb, cudaMemcpyHostToDevice, P.stream));
    src += blkb;
  }
  KS_CUDA_TRY(cudaMemcpyAsync(P.vH, src, (size_t)P.n * sizeof(double), cudaMemcpyHostToDevice,
                              P.stream));
  src += (size_t)P.n * sizeof(double);
  KS_TRY(load_cg(P, src));
  KS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  P.state = S;
  P.cg_inc_ok = hd.cg_inc_ok != 0;
  P.cg_inc_count = hd.cg_inc_count;
  return KS_OK;
}

}  // extern "C"
