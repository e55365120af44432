// Serving loop with continuous batching (ks_server_* in include/ks.h).
//
// Jobs (one KS system each) are admitted in arrival order while their
// device memory fits the HBM budget and a slot is free.  Each slot is a host
// worker thread that owns one problem and one CUDA stream for the duration
// of a job and drives Alg. ConOptM on it, so admitted jobs overlap on the
// device; when a job finishes its slot and memory are released and the next
// queued job is admitted at once.  Jobs share no device state (each has its
// own problem, buffers and stream, and every reduction has a fixed order),
// so a job's result is bitwise the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ks_internal.cuh"

namespace ks {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  ks_problem_desc desc{};
  ks_opts opts{};
  std::vector<double> R, Z;       // copies of the geometry
  std::vector<double> X;          // initial block in, result out (host)
  size_t bytes = 0;               // device bytes while running
  int state = 0;                  // 0 queued, 1 running, 2 done
  ks_status status = KS_OK;
  ks_result result{};
  Clock::time_point t_submit, t_start, t_end;
};

struct Server {
  int device = 0;
  size_t budget = 0;
  int slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_id = 1;
  size_t in_use = 0, peak_in_use = 0;
  int running = 0, peak_running = 0;
  uint64_t completed = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

static size_t job_bytes(const ks_problem_desc &d) {
  const size_t pb = ks_problem_bytes(&d);
  if (pb == 0) return 0;
  return pb + (size_t)d.N * d.N * d.N * d.p * sizeof(double);
}

// Run one job on this thread: problem + stream + device X, minimise, copy
// the result back, release everything.
static void run_job(Server &S, Job &J) {
  cudaSetDevice(S.device);
  cudaStream_t stream = nullptr;
  ks_problem *prob = nullptr;
  double *dX = nullptr;
  const size_t xbytes = J.X.size() * sizeof(double);
  ks_status st = KS_OK;
  auto cu = [&](cudaError_t e, const char *w) {
    if (e != cudaSuccess && st == KS_OK) st = cuda_error(e, w);
    return st == KS_OK;
  };
  if (cu(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "cudaStreamCreate")) {
    ks_problem_desc d = J.desc;
    d.R = J.R.data();
    d.Z = J.Z.data();
    d.stream = stream;
    st = ks_problem_create(&d, &prob);
  }
  if (st == KS_OK && cu(cudaMallocAsync((void **)&dX, xbytes, stream), "cudaMallocAsync") &&
      cu(cudaMemcpyAsync(dX, J.X.data(), xbytes, cudaMemcpyHostToDevice, stream), "copy X0")) {
    st = ks_minimize(prob, dX, &J.opts, &J.result);
    if (st == KS_OK || st == KS_ENOCONV) {
      cu(cudaMemcpyAsync(J.X.data(), dX, xbytes, cudaMemcpyDeviceToHost, stream), "copy X");
      cu(cudaStreamSynchronize(stream), "sync");
    }
  }
  if (dX) cudaFreeAsync(dX, stream);
  if (prob) ks_problem_destroy(prob);
  if (stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
  cudaGetLastError();
  J.status = st;
  if (st != KS_OK && st != KS_ENOCONV) J.result.status = st;
}

static void worker_main(Server *S) {
  for (;;) {
    Job *J = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // admit the queue head when its memory fits (arrival order)
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        const Job &head = *S->jobs[S->queue.front()];
        return S->in_use + head.bytes <= S->budget;
      });
      if (S->stop) return;
      J = S->jobs[S->queue.front()].get();
      S->queue.pop_front();
      S->in_use += J->bytes;
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      ++S->running;
      S->peak_running = std::max(S->peak_running, S->running);
      J->state = 1;
      J->t_start = Clock::now();
    }
    run_job(*S, *J);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      J->t_end = Clock::now();
      J->state = 2;
      S->in_use -= J->bytes;
      --S->running;
      ++S->completed;
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
}

}  // namespace ks

using namespace ks;

struct ks_server {
  Server S;
};

extern "C" {

ks_status ks_server_create(size_t hbm_budget_bytes, int max_slots, ks_server **out) {
  if (!out) return set_error(KS_EINVAL, "null output handle");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 256) return set_error(KS_EINVAL, "max_slots out of [1, 256]");
  if (hbm_budget_bytes == 0) return set_error(KS_EINVAL, "zero HBM budget");
  ks_server *sv = new (std::nothrow) ks_server();
  if (!sv) return set_error(KS_ENOMEM, "host allocation failed");
  Server &S = sv->S;
  cudaError_t e = cudaGetDevice(&S.device);
  if (e != cudaSuccess) {
    delete sv;
    return cuda_error(e, "cudaGetDevice");
  }
  S.budget = hbm_budget_bytes;
  S.slots = max_slots;
  for (int i = 0; i < max_slots; ++i) S.workers.emplace_back(worker_main, &S);
  *out = sv;
  return KS_OK;
}

ks_status ks_server_submit(ks_server *sv, const ks_problem_desc *desc, const ks_opts *opts,
                           const double *X0_host, uint64_t *job_id) {
  if (!sv || !desc || !X0_host || !job_id) return set_error(KS_EINVAL, "null argument");
  Server &S = sv->S;
  const size_t bytes = job_bytes(*desc);
  if (bytes == 0) return KS_EINVAL;   // ks_problem_bytes recorded the reason
  if (bytes > S.budget)
    return set_error(KS_ENOMEM, "job needs %zu bytes, more than the whole budget %zu", bytes,
                     S.budget);
  auto J = std::make_unique<Job>();
  J->desc = *desc;
  J->R.assign(desc->R, desc->R + 3 * (size_t)desc->natoms);
  J->Z.assign(desc->Z, desc->Z + (size_t)desc->natoms);
  const size_t np = (size_t)desc->N * desc->N * desc->N * desc->p;
  J->X.assign(X0_host, X0_host + np);
  if (opts) J->opts = *opts;
  else ks_opts_default(&J->opts);
  J->opts.resume = 0;
  J->bytes = bytes;
  J->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    J->id = S.next_id++;
    *job_id = J->id;
    S.queue.push_back(J->id);
    S.jobs[J->id] = std::move(J);
  }
  S.cv_work.notify_all();
  return KS_OK;
}

ks_status ks_server_poll(ks_server *sv, uint64_t job_id, int wait, ks_result *res,
                         double *X_host, double *latency_s) {
  if (!sv) return set_error(KS_EINVAL, "null server");
  Server &S = sv->S;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.jobs.find(job_id);
  if (it == S.jobs.end()) return set_error(KS_EINVAL, "unknown job %llu", (unsigned long long)job_id);
  if (wait) {
    // look the job up again on every wake-up: another thread's poll of the
    // same id may have collected (and erased) it meanwhile
    S.cv_done.wait(lk, [&] {
      it = S.jobs.find(job_id);
      return it == S.jobs.end() || it->second->state == 2;
    });
    if (it == S.jobs.end())
      return set_error(KS_EINVAL, "job %llu was collected by another poll", (unsigned long long)job_id);
  }
  Job &J = *it->second;
  if (J.state != 2) return KS_EAGAIN;
  if (res) *res = J.result;
  if (X_host) std::memcpy(X_host, J.X.data(), J.X.size() * sizeof(double));
  if (latency_s) *latency_s = std::chrono::duration<double>(J.t_end - J.t_submit).count();
  const ks_status st = J.status;
  S.jobs.erase(it);
  if (st != KS_OK && st != KS_ENOCONV) return set_error(st, "job %llu failed", (unsigned long long)job_id);
  return KS_OK;
}

ks_status ks_server_stats(ks_server *sv, ks_server_counters *out) {
  if (!sv || !out) return set_error(KS_EINVAL, "null argument");
  Server &S = sv->S;
  std::lock_guard<std::mutex> lk(S.mu);
  out->queued = (int)S.queue.size();
  out->running = S.running;
  out->peak_running = S.peak_running;
  out->completed = S.completed;
  out->bytes_in_use = S.in_use;
  out->peak_bytes_in_use = S.peak_in_use;
  out->budget = S.budget;
  return KS_OK;
}

ks_status ks_server_destroy(ks_server *sv) {
  if (!sv) return KS_OK;
  Server &S = sv->S;
  {
    // wait for the running jobs; queued jobs are dropped
    std::unique_lock<std::mutex> lk(S.mu);
    S.queue.clear();
    S.cv_done.wait(lk, [&] { return S.running == 0; });
    S.stop = true;
  }
  S.cv_work.notify_all();
  for (auto &t : S.workers) t.join();
  delete sv;
  return KS_OK;
}

}  // extern "C"
