// Batched job table (ks_batch_*): Alg. ConOptM with the QR retraction of
// Prop. 3.1 for many independent systems in lockstep iterations.  Each step
// of an iteration is one launch over the jobs still iterating (the active
// mask); the host keeps every job's line-search state (step, nonmonotone
// reference C/Q of Eq. NMLS-Armijo, Barzilai-Borwein traces of Eq. bb-1) and
// reads all jobs' device scalars with one copy per synchronisation.
//
// The n x p blocks of every job rotate together: after an accepted step the
// trial block becomes the current one for all running jobs (a backtracking
// job repeats its trial while the others keep theirs).  A job that stops
// keeps its final block where it is and is masked out of later launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>

#include "ks_device.cuh"

using namespace ks;

struct ks_batch {
  Batch B;
};

namespace ks {

namespace {

ks_status sync_batch(Batch &B) {
  KS_CUDA_TRY(cudaMemcpyAsync(B.scal_host, B.scal_dev, sizeof(double) * SC_COUNT * B.J,
                              cudaMemcpyDeviceToHost, B.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(B.status_host, B.status_dev, sizeof(int) * B.J,
                              cudaMemcpyDeviceToHost, B.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
  B.ring_used = 0;
  prof_collect();
  return KS_OK;
}

// Host-to-device copies of the mask and the steps go through a ring of
// pinned slices, so a slice is never rewritten while its copy may still be
// pending (the ring is recycled at every synchronisation, and a full ring
// synchronises first).
ks_status upload(Batch &B, void *dst, const void *src, size_t bytes) {
  const size_t slice = ((bytes + 255) / 256) * 256;
  if (B.ring_used + slice > B.ring_bytes) {
    KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
    B.ring_used = 0;
  }
  char *h = B.ring_host + B.ring_used;
  B.ring_used += slice;
  std::memcpy(h, src, bytes);
  KS_CUDA_TRY(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, B.stream));
  return KS_OK;
}

// Device scalars, status words and the CG's remaining-job count to the
// pinned host mirrors (capturable: fixed addresses, no synchronisation).
ks_status copy_scalars(Batch &B) {
  KS_CUDA_TRY(cudaMemcpyAsync(B.scal_host, B.scal_dev, sizeof(double) * SC_COUNT * B.J,
                              cudaMemcpyDeviceToHost, B.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(B.status_host, B.status_dev, sizeof(int) * B.J,
                              cudaMemcpyDeviceToHost, B.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(B.cg_remaining_host, B.cg_remaining_dev, sizeof(int),
                              cudaMemcpyDeviceToHost, B.stream));
  return KS_OK;
}

ks_status wait_batch(Batch &B) {
  KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
  B.ring_used = 0;
  prof_collect();
  return KS_OK;
}

// Graph kinds of the captured step sequences.
enum GraphKind { G_TRIAL = 1, G_EVAL, G_PROJECT };
constexpr int kGraphCgIters = 3;   // CG iterations inside a captured evaluation

bool graphs_usable(const Batch &B) { return B.use_graphs && !prof_enabled(); }

// Run `issue` (launches on B.stream only) through the graph cached under
// `key`, capturing it on first use.
template <typename F>
ks_status replay(Batch &B, const std::array<int, 14> &key, F issue) {
  auto it = B.graphs.find(key);
  if (it == B.graphs.end()) {
    const unsigned long long l0 = ks_kernel_launches();
    KS_CUDA_TRY(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal));
    const ks_status st = issue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(B.stream, &g);
    const long long nl = (long long)(ks_kernel_launches() - l0);
    count_launches(-nl);
    if (st != KS_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return cuda_error(e2, "cudaGraphInstantiate");
    it = B.graphs.emplace(key, std::make_pair(exec, nl)).first;
  }
  KS_CUDA_TRY(cudaGraphLaunch(it->second.first, B.stream));
  count_launches(it->second.second);
  return KS_OK;
}

ks_status upload_mask(Batch &B, const std::vector<unsigned char> &m) {
  for (int j = 0; j < B.J; ++j) B.active_host[j] = m[j];
  return upload(B, B.active_dev, m.data(), (size_t)B.J);
}

ks_status upload_tau(Batch &B, const std::vector<double> &tau) {
  return upload(B, B.tau_dev, tau.data(), sizeof(double) * B.J);
}

double sc(const Batch &B, int j, int which) { return B.scal_host[(size_t)j * SC_COUNT + which]; }

// Per-job state of one phase.
struct JobState {
  bool running = false;            // iterating in this phase
  bool in_phase = false;           // took part in this phase
  int status = KS_OK;              // device or numerical failure
  double E = 0, C = 0, Q = 1, best = 0, Et = 0;
  double dnorm2 = 0, ss = 0, sy = 0, yy = 0;
  bool have_prev = false;
  int k = 0, cg = 0, backtracks = 0, h = 0;
  int maxk = 0;                    // iteration limit of the job in this phase
  int first_k = 0;                 // iterations before this phase (BB parity, ortho cadence)
  double tau = 0, last_tau = 0, tau_first = 0;
  double df[3] = {1, 1, 1}, Eprev = 0;
  int last_improve = 0;            // iteration of the last 0.1 % improvement of best
  bool forced = false;             // the last trial was accepted without meeting the test
  bool stalled = false, converged = false;
  int slot = B_X0;                 // block holding the job's final X when it stopped
};

struct Slots {
  int ix[3] = {B_X0, B_X1, B_X2};  // cur, prev, trial
  int imx[3] = {B_MX0, B_MX1, B_MX2};
  int iex[2] = {B_EX0, B_EX1};     // cur, trial
  int id[2] = {B_D0, B_D1};        // cur, prev
  int imd[2] = {B_MD0, B_MD1};
};

double bb_step(int k, const JobState &t, const ks_opts &o) {
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

// A failed job (device status or non-finite numbers) leaves the phase.
void fail_job(Batch &B, JobState &s, int j, int st) {
  s.running = false;
  if (s.status == KS_OK) s.status = st;
  B.status_host[j] = 0;
}

// Device status words of the jobs in `mask`: failures leave the phase and
// their words are cleared on the device.
ks_status check_status(Batch &B, std::vector<JobState> &S, const std::vector<unsigned char> &mask) {
  bool clear = false;
  for (int j = 0; j < B.J; ++j) {
    if (!mask[j] || B.status_host[j] == 0) continue;
    fail_job(B, S[j], j, B.status_host[j]);
    clear = true;
  }
  if (clear) KS_CUDA_TRY(cudaMemsetAsync(B.status_dev, 0, sizeof(int) * B.J, B.stream));
  return KS_OK;
}

// Energy of the jobs in the mask at slot sX: density, Hartree PCG,
// potential and energy sums, Hamiltonian stencil, scalars to the host.
template <typename T>
ks_status launch_evaluate(Batch &B, int sX, int sEX, int sMX, int cg_iters) {
  KS_TRY(batch_density<T>(B, sX));
  KS_TRY(batch_cg_launch(B, cg_iters));
  KS_TRY(batch_potential(B, sizeof(T) == 4));
  KS_TRY(batch_hamiltonian<T>(B, sX, sEX, sMX));
  return copy_scalars(B);
}

// QR retraction of the jobs in the mask (step B.tau_dev) into slot sOut.
template <typename T>
ks_status launch_retract(Batch &B, int sX, int sD, int sOut) {
  KS_TRY(batch_qr_factor(B, S_DMD, -1, true, S_C1, S_C2));
  return batch_combine<T>(B, sX, S_C1, sD, S_C2, 1.0, 0.0, -1, sOut);
}

// Runs the evaluation (after a retraction into sX when `trial_from` gives
// the current and direction slots), through a cached graph when possible.
// A graph holds kGraphCgIters CG iterations; jobs whose CG needs more
// continue outside it, after which the potential and stencil are redone.
template <typename T>
ks_status run_evaluate(Batch &B, double cg_tol, int sX, int sEX, int sMX, int rX, int rD) {
  KS_TRY(batch_cg_upload(B, cg_tol));
  if (graphs_usable(B)) {
    const std::array<int, 14> key = {rX >= 0 ? G_TRIAL : G_EVAL, (int)sizeof(T), sX, sEX, sMX,
                                     rX, rD, kGraphCgIters, 0, 0, 0, 0, 0, 0};
    KS_TRY(replay(B, key, [&]() -> ks_status {
      if (rX >= 0) KS_TRY(launch_retract<T>(B, rX, rD, sX));
      return launch_evaluate<T>(B, sX, sEX, sMX, kGraphCgIters);
    }));
    KS_TRY(wait_batch(B));
    if (*B.cg_remaining_host == 0) return KS_OK;
    KS_TRY(batch_cg_continue(B));
    KS_TRY(batch_potential(B, sizeof(T) == 4));
    KS_TRY(batch_hamiltonian<T>(B, sX, sEX, sMX));
    KS_TRY(copy_scalars(B));
    return wait_batch(B);
  }
  if (rX >= 0) KS_TRY(launch_retract<T>(B, rX, rD, sX));
  KS_TRY(batch_density<T>(B, sX));
  KS_TRY(batch_cg_launch(B, 0));
  KS_TRY(batch_cg_continue(B));
  KS_TRY(batch_potential(B, sizeof(T) == 4));
  KS_TRY(batch_hamiltonian<T>(B, sX, sEX, sMX));
  KS_TRY(copy_scalars(B));
  return wait_batch(B);
}

template <typename T>
ks_status evaluate(Batch &B, std::vector<JobState> &S, const std::vector<unsigned char> &mask,
                   double cg_tol, const std::vector<double> &eii, int sX, int sEX, int sMX,
                   bool trial, int rX = -1, int rD = -1) {
  KS_TRY(run_evaluate<T>(B, cg_tol, sX, sEX, sMX, rX, rD));
  KS_TRY(check_status(B, S, mask));
  for (int j = 0; j < B.J; ++j) {
    if (!mask[j] || !S[j].running) continue;
    B.warm[j] = 1;
    const double E = sc(B, j, SC_EKIN) + sc(B, j, SC_EEXT) + sc(B, j, SC_EH) + sc(B, j, SC_EXC) +
                     eii[j];
    S[j].cg += (int)sc(B, j, SC_CG_ITERS);
    if (!std::isfinite(E)) {
      fail_job(B, S[j], j, KS_ENAN);
      continue;
    }
    if (trial) S[j].Et = E;
    else S[j].E = E;
  }
  return KS_OK;
}

// G = M^{-1} E_X, S = E_X^T X, D = G - X S, MD = M D with ||D||_M^2 and the
// BB traces, D^T M D.
template <typename T>
ks_status launch_project(Batch &B, const Slots &sl, bool prev) {
  KS_TRY(batch_mass_inverse<T>(B, sl.iex[0], B_G));
  KS_TRY(batch_gram<T>(B, sl.iex[0], sl.ix[0], S_S));
  KS_TRY(batch_combine<T>(B, sl.ix[0], S_S, -1, -1, -1.0, 1.0, B_G, sl.id[0]));
  if (prev)
    KS_TRY(batch_mass_dots<T>(B, sl.id[0], sl.imd[0], sl.ix[0], sl.imx[0], sl.ix[1], sl.imx[1],
                              sl.id[1], sl.imd[1]));
  else
    KS_TRY(batch_mass_dots<T>(B, sl.id[0], sl.imd[0], -1, -1, -1, -1, -1, -1));
  KS_TRY(batch_gram<T>(B, sl.id[0], sl.imd[0], S_DMD));
  return copy_scalars(B);
}

template <typename T>
ks_status project(Batch &B, std::vector<JobState> &S, const std::vector<unsigned char> &mask,
                  const Slots &sl, bool prev) {
  if (graphs_usable(B)) {
    const std::array<int, 14> key = {G_PROJECT, (int)sizeof(T), sl.iex[0], sl.ix[0], sl.id[0],
                                     sl.imd[0], sl.imx[0], sl.ix[1], sl.imx[1], sl.id[1],
                                     sl.imd[1], prev ? 1 : 0, 0, 0};
    KS_TRY(replay(B, key, [&]() { return launch_project<T>(B, sl, prev); }));
  } else {
    KS_TRY(launch_project<T>(B, sl, prev));
  }
  KS_TRY(wait_batch(B));
  KS_TRY(check_status(B, S, mask));
  for (int j = 0; j < B.J; ++j) {
    if (!mask[j] || !S[j].running) continue;
    S[j].dnorm2 = sc(B, j, SC_DNORM2);
    if (prev) {
      S[j].ss = sc(B, j, SC_BB_SS);
      S[j].sy = sc(B, j, SC_BB_SY);
      S[j].yy = sc(B, j, SC_BB_YY);
    }
    if (!std::isfinite(S[j].dnorm2)) fail_job(B, S[j], j, KS_ENAN);
  }
  return KS_OK;
}

// Cholesky QR in the M inner product (`passes` times) of the jobs in mask,
// in place in slot sX, with sTmp as scratch; sMX receives M X.
template <typename T>
ks_status orthonormalize(Batch &B, std::vector<JobState> &S, const std::vector<unsigned char> &mask,
                         int sX, int sTmp, int sMX, int passes) {
  for (int k = 0; k < passes; ++k) {
    KS_TRY(batch_mass<T>(B, sX, sMX));
    KS_TRY(batch_gram<T>(B, sX, sMX, S_O));
    KS_TRY(batch_qr_factor(B, -1, S_O, false, S_C1, -1));
    KS_TRY(batch_combine<T>(B, sX, S_C1, -1, -1, 1.0, 0.0, -1, sTmp));
    KS_TRY((batch_convert<T, T>(B, sTmp, sX)));
  }
  KS_TRY(batch_mass<T>(B, sX, sMX));
  KS_TRY(sync_batch(B));
  return check_status(B, S, mask);
}

std::vector<unsigned char> running_mask(const std::vector<JobState> &S) {
  std::vector<unsigned char> m(S.size());
  for (size_t j = 0; j < S.size(); ++j) m[j] = S[j].running ? 1 : 0;
  return m;
}

bool any(const std::vector<unsigned char> &m) {
  for (unsigned char c : m)
    if (c) return true;
  return false;
}

// One lockstep phase in precision T for the jobs with S[j].running set; each
// starts from slot sStart (copied to the current block), stops at
// ||D||_M <= gtol, S[j].maxk iterations, or (stall) energy stagnation.
template <typename T>
ks_status run_phase(Batch &B, std::vector<JobState> &S, const ks_opts &o, double gtol, bool stall,
                    double cg_tol, double ortho_tol, int sStart, const std::vector<double> &eii) {
  Slots sl;
  std::vector<unsigned char> m = running_mask(S);
  for (int j = 0; j < B.J; ++j) {
    S[j].in_phase = m[j] != 0;
    S[j].k = 0;
    S[j].have_prev = false;
    S[j].converged = S[j].stalled = false;
  }
  if (!any(m)) return KS_OK;
  KS_TRY(upload_mask(B, m));
  KS_TRY((batch_convert<T, T>(B, sStart, sl.ix[0])));
  KS_TRY(orthonormalize<T>(B, S, m, sl.ix[0], sl.ix[2], sl.imx[0], 2));
  m = running_mask(S);
  KS_TRY(upload_mask(B, m));
  KS_TRY(evaluate<T>(B, S, m, cg_tol, eii, sl.ix[0], sl.iex[0], sl.imx[0], false));
  m = running_mask(S);
  KS_TRY(upload_mask(B, m));
  KS_TRY(project<T>(B, S, m, sl, false));
  for (int j = 0; j < B.J; ++j) {
    if (!S[j].running) continue;
    S[j].C = S[j].E;
    S[j].Q = 1.0;
    S[j].best = std::sqrt(std::fmax(S[j].dnorm2, 0.0));
    S[j].last_improve = 0;
    S[j].Eprev = S[j].E;
    for (double &d : S[j].df) d = 1.0;
  }
  auto stop_check = [&](int j) {
    JobState &s = S[j];
    const double dn = std::sqrt(std::fmax(s.dnorm2, 0.0));
    if (dn <= gtol) s.converged = true;
    if (s.converged || s.k >= s.maxk || s.stalled) s.running = false;
  };
  for (int j = 0; j < B.J; ++j)
    if (S[j].running) stop_check(j);
  const int every = sizeof(T) == 4 ? std::min(o.ortho_every, 5) : o.ortho_every;
  std::vector<double> tau(B.J, 0.0);
  for (;;) {
    m = running_mask(S);
    // jobs that stopped keep their current block
    for (int j = 0; j < B.J; ++j)
      if (S[j].in_phase && !S[j].running && S[j].slot == -1) S[j].slot = sl.ix[0];
    if (!any(m)) break;
    for (int j = 0; j < B.J; ++j) {
      if (!m[j]) continue;
      JobState &s = S[j];
      s.tau = s.have_prev ? bb_step(s.first_k + s.k, s, o)
                          : (s.tau_first > 0.0 ? s.tau_first : o.tau0);
      s.h = 0;
      s.forced = false;
      tau[j] = s.tau;
    }
    std::vector<unsigned char> search = m;
    while (any(search)) {
      KS_TRY(upload_mask(B, search));
      KS_TRY(upload_tau(B, tau));
      KS_TRY(evaluate<T>(B, S, search, cg_tol, eii, sl.ix[2], sl.iex[1], sl.imx[2], true,
                         sl.ix[0], sl.id[0]));
      for (int j = 0; j < B.J; ++j) {
        if (!search[j]) continue;
        JobState &s = S[j];
        if (!s.running) {
          search[j] = 0;
          continue;
        }
        const double parts[5] = {sc(B, j, SC_EKIN), sc(B, j, SC_EEXT), sc(B, j, SC_EH),
                                 sc(B, j, SC_EXC), eii[j]};
        const bool ok = s.Et <= s.C - o.rho1 * s.tau * s.dnorm2 + armijo_slack<T>(parts);
        if (ok || s.h == o.max_backtrack) {
          search[j] = 0;
          s.forced = !ok;
        } else {
          s.tau *= o.delta;
          tau[j] = s.tau;
          ++s.h;
        }
      }
    }
    // accept for every job still running
    m = running_mask(S);
    for (int j = 0; j < B.J; ++j) {
      if (!m[j]) continue;
      JobState &s = S[j];
      s.backtracks += s.h;
      s.last_tau = s.tau;
      const double Qn = o.eta * s.Q + 1.0;
      s.C = (o.eta * s.Q * s.C + s.Et) / Qn;
      s.Q = Qn;
      if (s.forced && sizeof(T) == 8) {   // FP64: restart the nonmonotone reference
        s.C = s.Et;
        s.Q = 1.0;
      }
      s.E = s.Et;
      ++s.k;
    }
    // jobs that failed during the search keep the current block as final
    for (int j = 0; j < B.J; ++j)
      if (S[j].in_phase && !S[j].running && S[j].slot == -1) S[j].slot = sl.ix[0];
    std::swap(sl.ix[1], sl.ix[0]);
    std::swap(sl.ix[0], sl.ix[2]);
    std::swap(sl.imx[1], sl.imx[0]);
    std::swap(sl.imx[0], sl.imx[2]);
    std::swap(sl.iex[0], sl.iex[1]);
    std::swap(sl.id[0], sl.id[1]);
    std::swap(sl.imd[0], sl.imd[1]);
    // the orthogonality check of the jobs due for it (every `every`
    // iterations of each job's count)
    std::vector<unsigned char> due(B.J, 0);
    for (int j = 0; j < B.J; ++j)
      if (m[j] && every > 0 && (S[j].first_k + S[j].k) % every == 0) due[j] = 1;
    if (any(due)) {
      KS_TRY(upload_mask(B, due));
      KS_TRY(batch_gram<T>(B, sl.ix[0], sl.imx[0], S_T));
      KS_TRY(batch_ortho_err(B, S_T));
      KS_TRY(sync_batch(B));
      KS_TRY(check_status(B, S, due));
      std::vector<unsigned char> re(B.J, 0);
      for (int j = 0; j < B.J; ++j)
        if (due[j] && S[j].running && std::sqrt(sc(B, j, SC_ORTHO)) > ortho_tol) re[j] = 1;
      if (any(re)) {
        KS_TRY(upload_mask(B, re));
        KS_TRY(orthonormalize<T>(B, S, re, sl.ix[0], sl.ix[2], sl.imx[0], 1));
        KS_TRY(evaluate<T>(B, S, re, cg_tol, eii, sl.ix[0], sl.iex[0], sl.imx[0], false));
      }
    }
    m = running_mask(S);
    KS_TRY(upload_mask(B, m));
    KS_TRY(project<T>(B, S, m, sl, true));
    for (int j = 0; j < B.J; ++j) {
      if (!m[j] || !S[j].running) continue;
      JobState &s = S[j];
      s.have_prev = true;
      s.df[s.k % 3] = std::fabs(s.Eprev - s.E) / (std::fabs(s.Eprev) + 1.0);
      s.Eprev = s.E;
      const double dn = std::sqrt(std::fmax(s.dnorm2, 0.0));
      if (dn < 0.999 * s.best) {
        s.best = dn;
        s.last_improve = s.k;
      }
      if (stall && s.k >= 3 &&
          ((s.df[0] + s.df[1] + s.df[2]) / 3.0 < o.stall_df || s.k - s.last_improve >= kStallWindow))
        s.stalled = true;
      if (o.verbose > 0 && s.k % o.verbose == 0)
        fprintf(stderr, "ks_batch[%s] job %d: k=%d E=%.12f |D|=%.3e tau=%.3e\n",
                sizeof(T) == 8 ? "fp64" : "fp32", j, s.k, s.E, dn, s.tau);
      stop_check(j);
      if (!s.running) s.slot = sl.ix[0];
    }
  }
  return KS_OK;
}

// Launch-family block counts of every job (host) and the prefix maps.
ks_status build_maps(Batch &B) {
  const int J = B.J;
  B.maps_host.assign((size_t)BM_COUNT * (J + 1), 0);
  auto put = [&](int m, int j, long long blocks) {
    B.maps_host[(size_t)m * (J + 1) + j + 1] = (int)blocks;
  };
  for (int j = 0; j < J; ++j) {
    BJob &b = B.jobs_host[j];
    const Problem &P = B.probs[j]->P;
    const long long n = b.n, p = b.p;
    put(BM_DENSITY, j, (n + 255) / 256);
    const long long per_pot = 256LL * B.tune.pot_per_thread;
    long long pot = (n + per_pot - 1) / per_pot;
    if (pot > 64) pot = 64;
    if (pot < 1) pot = 1;
    b.pot_nb = (int)pot;
    put(BM_POTENTIAL, j, pot);
    const int cls = p >= 32 ? BM_ST32 : p >= 16 ? BM_ST16 : p >= 8 ? BM_ST8 : BM_ST4;
    put(cls, j, b.st_nb);
    put(BM_THOMAS, j, ((long long)b.N * b.N * p + 255) / 256);
    long long chunks = (n + B.tune.gram_rows - 1) / B.tune.gram_rows;
    const long long cap = (long long)(P.partials_len / (size_t)(p * p));
    if (chunks > cap) chunks = cap;
    if (chunks < 1) chunks = 1;
    long long rows = (n + chunks - 1) / chunks;
    rows = (rows + kTileK - 1) / kTileK * kTileK;
    chunks = (n + rows - 1) / rows;
    b.gram_chunks = (int)chunks;
    b.gram_rows_per = rows;
    const long long tiles = ((p + kTile - 1) / kTile) * ((p + kTile - 1) / kTile);
    if (p <= 8) put(BM_GRAM_SMALL, j, chunks);
    else if (p <= 32) put(BM_GRAM_MID, j, chunks);
    else put(BM_GRAM_TILED, j, tiles * chunks);
    put(BM_GRAM_REDUCE, j, (8 * p * p + kThreads - 1) / kThreads);
    if (p <= 32) {
      // the narrow update's work items are groups of 4 columns of a row
      const long long per_comb = 256LL * B.tune.comb_per_thread;
      long long nb = (n * ((p + 3) / 4) * 4 + per_comb - 1) / per_comb;
      if (nb < 1) nb = 1;
      b.comb_nb = (int)nb;
      put(BM_COMB_NARROW, j, nb);
    } else {
      b.comb_nb = 0;
      put(BM_COMB_TILED, j, ((n + kTile - 1) / kTile) * ((p + kTile - 1) / kTile));
    }
    put(BM_COEF, j, (2 * p * p + kThreads - 1) / kThreads);
    put(BM_CG_NODES, j, (n + kCgThreads - 1) / kCgThreads);
    put(BM_CG_PLANES, j, b.N);
    put(BM_COPY, j, (n * p + 4 * kThreads - 1) / (4 * kThreads));
  }
  for (int m = 0; m < BM_COUNT; ++m) {
    long long acc = 0;
    for (int j = 0; j <= J; ++j) {
      acc += B.maps_host[(size_t)m * (J + 1) + j];
      if (acc > 0x7fffffffLL) return set_error(KS_EINVAL, "batch: launch too large");
      B.maps_host[(size_t)m * (J + 1) + j] = (int)acc;
    }
  }
  return KS_OK;
}

void free_batch(Batch &B) {
  if (B.stream) cudaStreamSynchronize(B.stream);
  for (auto &kv : B.graphs) cudaGraphExecDestroy(kv.second.first);
  B.graphs.clear();
  for (ks_problem *p : B.probs) ks_problem_destroy(p);
  B.probs.clear();
  if (B.jobs_dev) cudaFree(B.jobs_dev);
  if (B.maps_dev) cudaFree(B.maps_dev);
  if (B.active_dev) cudaFree(B.active_dev);
  if (B.tau_dev) cudaFree(B.tau_dev);
  if (B.scal_dev) cudaFree(B.scal_dev);
  if (B.status_dev) cudaFree(B.status_dev);
  if (B.cg_args_dev) cudaFree(B.cg_args_dev);
  if (B.active_host) cudaFreeHost(B.active_host);
  if (B.tau_host) cudaFreeHost(B.tau_host);
  if (B.scal_host) cudaFreeHost(B.scal_host);
  if (B.status_host) cudaFreeHost(B.status_host);
  if (B.cg_tolw_host) cudaFreeHost(B.cg_tolw_host);
  if (B.cg_remaining_host) cudaFreeHost(B.cg_remaining_host);
  if (B.cg_remaining_dev) cudaFree(B.cg_remaining_dev);
  if (B.ring_host) cudaFreeHost(B.ring_host);
  if (B.own_stream && B.stream) cudaStreamDestroy(B.stream);
  cudaGetLastError();
  B = Batch();
}

}  // namespace

}  // namespace ks

extern "C" {

ks_status ks_batch_create(const ks_problem_desc *descs, int njobs, void *stream, ks_batch **out) {
  if (!out || !descs || njobs < 1) return set_error(KS_EINVAL, "bad argument");
  *out = nullptr;
  // every description is checked before the first device call
  for (int j = 0; j < njobs; ++j) {
    KS_TRY(validate_desc(&descs[j]));
    if (descs[j].p > 104) return set_error(KS_EINVAL, "batch: job %d has p > 104", j);
    if (descs[j].kinetic != KS_KIN_ORBITALS || descs[j].mass != KS_MASS_CONSISTENT)
      return set_error(KS_EINVAL,
                       "batch: job %d is orbital-free or lumped (single-system path only)", j);
  }
  ks_batch *kb = new (std::nothrow) ks_batch();
  if (!kb) return set_error(KS_ENOMEM, "host allocation failed");
  Batch &B = kb->B;
  auto fail = [&](ks_status st) {
    free_batch(B);
    delete kb;
    return st;
  };
  B.J = njobs;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(cuda_error(e, "cudaDeviceGetAttribute"));
  if (stream) {
    B.stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaStreamCreate"));
    B.own_stream = true;
  }
  for (int j = 0; j < njobs; ++j) {
    ks_problem_desc d = descs[j];
    d.stream = B.stream;
    ks_problem *p = nullptr;
    const ks_status st = ks_problem_create(&d, &p);
    if (st != KS_OK) return fail(st);
    B.probs.push_back(p);
    B.bytes += p->P.bytes;
    if (d.N > B.maxN) B.maxN = d.N;
    if (d.p > B.maxp) B.maxp = d.p;
  }
#define BALLOC(ptr, nbytes)                                                               \
  if ((e = cudaMalloc((void **)&(ptr), (nbytes))) != cudaSuccess)                          \
    return fail(cuda_error(e, "cudaMalloc"));                                              \
  B.bytes += (nbytes);
#define HALLOC(ptr, nbytes)                                                               \
  if ((e = cudaMallocHost((void **)&(ptr), (nbytes))) != cudaSuccess)                      \
    return fail(cuda_error(e, "cudaMallocHost"));
  BALLOC(B.scal_dev, sizeof(double) * SC_COUNT * njobs);
  BALLOC(B.status_dev, sizeof(int) * njobs);
  BALLOC(B.active_dev, (size_t)njobs);
  BALLOC(B.tau_dev, sizeof(double) * njobs);
  BALLOC(B.cg_remaining_dev, sizeof(int));
  HALLOC(B.scal_host, sizeof(double) * SC_COUNT * njobs);
  HALLOC(B.status_host, sizeof(int) * njobs);
  HALLOC(B.active_host, (size_t)njobs);
  HALLOC(B.tau_host, sizeof(double) * njobs);
  HALLOC(B.cg_tolw_host, sizeof(double) * 2 * njobs);
  HALLOC(B.cg_remaining_host, sizeof(int));
  B.ring_bytes = (size_t)64 * (((size_t)njobs * sizeof(double) + 255) / 256 * 256);
  HALLOC(B.ring_host, B.ring_bytes);
  if ((e = cudaMemsetAsync(B.scal_dev, 0, sizeof(double) * SC_COUNT * njobs, B.stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(B.status_dev, 0, sizeof(int) * njobs, B.stream)) != cudaSuccess)
    return fail(cuda_error(e, "memset"));
  B.jobs_host.resize(njobs);
  for (int j = 0; j < njobs; ++j) {
    Problem &P = B.probs[j]->P;
    BJob &b = B.jobs_host[j];
    b = BJob{};
    b.N = P.N;
    b.p = P.p;
    b.n = P.n;
    b.h = P.h;
    b.occ = P.occ;
    b.h3 = P.h * P.h * P.h;
    b.cg_tol = P.cg_tol;
    b.xc = P.xc;
    b.cg_maxit = P.cg_maxit;
    b.cg_precond = P.cg_precond;
    for (int i = 0; i < Problem::kNBlocks; ++i) b.blk[i] = P.blk[i];
    b.vext = P.vext;
    b.rho = P.rho;
    b.vH = P.vH;
    b.veff = P.veff;
    b.cg_r = P.cg_r;
    P.cg_inc_ok = false;   // the batch's own solves write vH and r
    b.pp = P.pp;
    b.cf = P.cf;
    b.partials = P.partials;
    b.red_counter = P.red_counter;
    b.thomas_w = P.thomas_w;
    b.scal = B.scal_dev + (size_t)SC_COUNT * j;
    b.status = B.status_dev + j;
    const StencilCoef c = q1_coefficients(P.h);
    const double qc[8] = {c.k0, c.kf, c.ke, c.kc, c.m0, c.mf, c.me, c.mc};
    for (int i = 0; i < 8; ++i) b.qc[i] = qc[i];
    const double qcf[9] = {c.k0, c.ke, c.kc, c.m0, c.mf, c.me, c.mc, P.occ, 2.0 * P.occ * b.h3};
    for (int i = 0; i < 9; ++i) b.qcf[i] = (float)qcf[i];
  }
  ks_status st;
  if ((st = batch_stencil_geometry(B)) != KS_OK) return fail(st);
  if ((st = build_maps(B)) != KS_OK) return fail(st);
  BALLOC(B.jobs_dev, sizeof(BJob) * njobs);
  BALLOC(B.maps_dev, sizeof(int) * B.maps_host.size());
#undef BALLOC
#undef HALLOC
  if ((e = cudaMemcpyAsync(B.jobs_dev, B.jobs_host.data(), sizeof(BJob) * njobs,
                           cudaMemcpyHostToDevice, B.stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.maps_dev, B.maps_host.data(), sizeof(int) * B.maps_host.size(),
                           cudaMemcpyHostToDevice, B.stream)) != cudaSuccess)
    return fail(cuda_error(e, "copy job table"));
  if ((st = batch_cg_setup(B)) != KS_OK) return fail(st);
  B.warm.assign(njobs, 0);
  if ((e = cudaStreamSynchronize(B.stream)) != cudaSuccess) return fail(cuda_error(e, "sync"));
  *out = kb;
  return KS_OK;
}

size_t ks_batch_bytes(const ks_batch *kb) { return kb ? kb->B.bytes : 0; }

// Autotuner: each launch shape in turn, every candidate timed with CUDA
// events (one warm-up launch, then the mean of three) on the job table with
// zeroed FP32 blocks; the fastest is kept.
ks_status ks_batch_autotune(ks_batch *kb, int out[4]) {
  if (!kb) return set_error(KS_EINVAL, "null batch");
  Batch &B = kb->B;
  std::vector<unsigned char> all(B.J, 1);
  KS_TRY(upload_mask(B, all));
  for (int j = 0; j < B.J; ++j) {
    const Problem &P = B.probs[j]->P;
    for (int b : {B_X0, B_X1, B_X2, B_EX0, B_MX0})
      KS_CUDA_TRY(cudaMemsetAsync(P.blk[b], 0, sizeof(double) * P.n * P.p, B.stream));
    KS_CUDA_TRY(cudaMemsetAsync(P.pp, 0, sizeof(double) * P.pp_len, B.stream));
  }
  cudaEvent_t e0, e1;
  KS_CUDA_TRY(cudaEventCreate(&e0));
  KS_CUDA_TRY(cudaEventCreate(&e1));
  auto rebuild = [&]() -> ks_status {
    KS_TRY(batch_stencil_geometry(B));
    KS_TRY(build_maps(B));
    KS_CUDA_TRY(cudaMemcpyAsync(B.jobs_dev, B.jobs_host.data(), sizeof(BJob) * B.J,
                                cudaMemcpyHostToDevice, B.stream));
    KS_CUDA_TRY(cudaMemcpyAsync(B.maps_dev, B.maps_host.data(), sizeof(int) * B.maps_host.size(),
                                cudaMemcpyHostToDevice, B.stream));
    return KS_OK;
  };
  auto time_it = [&](auto launch, float *ms) -> ks_status {
    KS_TRY(launch());
    KS_CUDA_TRY(cudaEventRecord(e0, B.stream));
    for (int r = 0; r < 3; ++r) KS_TRY(launch());
    KS_CUDA_TRY(cudaEventRecord(e1, B.stream));
    KS_CUDA_TRY(cudaEventSynchronize(e1));
    KS_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return KS_OK;
  };
  auto tune = [&](int *field, std::initializer_list<int> cands, auto launch) -> ks_status {
    float best = 1e30f;
    int best_v = *field;
    for (int v : cands) {
      *field = v;
      const ks_status st = rebuild();
      if (st != KS_OK) continue;                 // a candidate the partials cannot hold
      float ms = 0.f;
      KS_TRY(time_it(launch, &ms));
      if (ms < best) {
        best = ms;
        best_v = v;
      }
    }
    *field = best_v;
    return rebuild();
  };
  ks_status st = KS_OK;
  if (st == KS_OK)
    st = tune(&B.tune.gram_rows, {1024, 2048, 4096, 8192, 16384},
              [&]() { return batch_gram<float>(B, B_X0, B_X1, S_T); });
  if (st == KS_OK)
    st = tune(&B.tune.comb_per_thread, {2, 4, 8, 16}, [&]() {
      return batch_combine<float>(B, B_X0, S_C1, B_X1, S_C2, 1.0, 0.0, -1, B_X2);
    });
  if (st == KS_OK)
    st = tune(&B.tune.pot_per_thread, {1, 2, 4, 8}, [&]() { return batch_potential(B, true); });
  if (st == KS_OK)
    st = tune(&B.tune.st_planes, {0, 8, 16, 32, 64},
              [&]() { return batch_hamiltonian<float>(B, B_X0, B_EX0, B_MX0); });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  KS_TRY(st);
  // the timings left the reduction counters re-armed; the graphs hold the
  // old launch shapes
  for (auto &kv : B.graphs) cudaGraphExecDestroy(kv.second.first);
  B.graphs.clear();
  KS_CUDA_TRY(cudaMemsetAsync(B.status_dev, 0, sizeof(int) * B.J, B.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
  if (out) {
    out[0] = B.tune.gram_rows;
    out[1] = B.tune.comb_per_thread;
    out[2] = B.tune.pot_per_thread;
    out[3] = B.tune.st_planes;
  }
  return KS_OK;
}

ks_status ks_batch_set_graphs(ks_batch *kb, int enable) {
  if (!kb || enable < 0 || enable > 1) return set_error(KS_EINVAL, "bad argument");
  kb->B.use_graphs = enable != 0;
  return KS_OK;
}

ks_status ks_batch_minimize(ks_batch *kb, double *const *X_inout, const ks_opts *opts_in,
                            ks_result *results) {
  if (!kb || !X_inout) return set_error(KS_EINVAL, "null argument");
  Batch &B = kb->B;
  ks_opts o;
  if (opts_in) o = *opts_in;
  else ks_opts_default(&o);
  if (o.retraction != KS_QR) return set_error(KS_EINVAL, "batch: only the QR retraction");
  if (o.resume) return set_error(KS_EINVAL, "batch: resume is not supported");
  const auto t0 = std::chrono::steady_clock::now();
  const int J = B.J;
  for (int j = 0; j < J; ++j)
    if (!X_inout[j]) return set_error(KS_EINVAL, "null X for job %d", j);
  std::vector<double> eii(J);
  for (int j = 0; j < J; ++j) eii[j] = B.probs[j]->P.scal_host[SC_EII];
  std::fill(B.warm.begin(), B.warm.end(), 0);
  std::vector<JobState> S(J);
  for (auto &s : S) {
    s.running = true;
    s.slot = -1;
  }
  // initial blocks: FP64 into B_MD1 of every job
  for (int j = 0; j < J; ++j) {
    const Problem &P = B.probs[j]->P;
    KS_CUDA_TRY(cudaMemcpyAsync(P.blk[B_MD1], X_inout[j], sizeof(double) * P.n * P.p,
                                cudaMemcpyHostToDevice, B.stream));
  }
  std::vector<int> mixed_iters(J, 0);
  std::vector<double> mixed_E(J, 0.0), mixed_dn(J, 0.0);
  std::vector<unsigned char> all(J, 1);
  if (o.precision == KS_MIXED) {
    // FP32 phase for every job, then the FP64 polish for the jobs that
    // reached polish_gtol or stagnated (a job that ran out of iterations in
    // the FP32 phase stops there, as in ks_minimize)
    KS_TRY(upload_mask(B, all));
    KS_TRY((batch_convert<double, float>(B, B_MD1, B_G)));
    for (auto &s : S) s.maxk = o.maxit;
    KS_TRY(run_phase<float>(B, S, o, std::fmax(o.polish_gtol, o.gtol), o.stall_iters > 0,
                            std::fmin(o.mixed_cg_tol, 1e-3), std::fmax(o.ortho_tol, 1e-5), B_G,
                            eii));
    for (int j = 0; j < J; ++j) {
      JobState &s = S[j];
      mixed_iters[j] = s.k;
      mixed_E[j] = s.E;
      mixed_dn[j] = std::sqrt(std::fmax(s.dnorm2, 0.0));
      s.tau_first = s.last_tau;
      if (s.status == KS_OK && s.slot >= 0 && s.slot != B_G) {
        const Problem &P = B.probs[j]->P;
        KS_CUDA_TRY(cudaMemcpyAsync(P.blk[B_G], P.blk[s.slot], sizeof(float) * P.n * P.p,
                                    cudaMemcpyDeviceToDevice, B.stream));
      }
      s.running = s.status == KS_OK && (s.converged || s.stalled);
      s.maxk = o.maxit - s.k;
      s.first_k = s.k;
      s.slot = -1;
    }
    KS_TRY(upload_mask(B, all));
    KS_TRY((batch_convert<float, double>(B, B_G, B_MD1)));
  } else {
    for (auto &s : S) s.maxk = o.maxit;
  }
  KS_TRY(run_phase<double>(B, S, o, o.gtol, false, 0.0, o.ortho_tol, B_MD1, eii));
  int overall = KS_OK;
  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int j = 0; j < J; ++j) {
    JobState &s = S[j];
    const Problem &P = B.probs[j]->P;
    const bool fp64_ran = s.in_phase;
    int slot = s.slot >= 0 ? s.slot : B_X0;
    if (!fp64_ran) slot = B_MD1;             // stopped in the FP32 phase: its FP64 copy
    KS_CUDA_TRY(cudaMemcpyAsync(X_inout[j], P.blk[slot], sizeof(double) * P.n * P.p,
                                cudaMemcpyDeviceToHost, B.stream));
    int status = s.status;
    const double dn = fp64_ran ? std::sqrt(std::fmax(s.dnorm2, 0.0)) : mixed_dn[j];
    if (status == KS_OK && dn > o.gtol) status = KS_ENOCONV;
    if (status != KS_OK && overall == KS_OK) overall = status == KS_ENOCONV ? KS_ENOCONV : status;
    if (status != KS_OK && status != KS_ENOCONV) overall = status;
    if (results) {
      ks_result &r = results[j];
      r = ks_result{};
      r.E = fp64_ran ? s.E : mixed_E[j];
      r.gradnorm = dn;
      r.ortho_err = -1.0;
      r.iters = (fp64_ran ? s.k : 0) + mixed_iters[j];
      r.cg_iters_total = s.cg;
      r.backtracks = s.backtracks;
      r.status = status;
      r.seconds = secs;
      r.mixed_iters = mixed_iters[j];
      r.mixed_gradnorm = mixed_dn[j];
      r.mixed_E = mixed_E[j];
      r.E_parts[0] = sc(B, j, SC_EKIN);
      r.E_parts[1] = sc(B, j, SC_EEXT);
      r.E_parts[2] = sc(B, j, SC_EH);
      r.E_parts[3] = sc(B, j, SC_EXC);
      r.E_parts[4] = eii[j];
    }
  }
  KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
  if (overall != KS_OK)
    return set_error((ks_status)overall, "batch: some jobs did not converge or failed");
  return KS_OK;
}

ks_status ks_batch_destroy(ks_batch *kb) {
  if (!kb) return KS_OK;
  free_batch(kb->B);
  delete kb;
  return KS_OK;
}

}  // extern "C"
