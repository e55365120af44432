// Launch counting and optional per-kernel-class CUDA-event timing.
//
// Every kernel launch of the library goes through count_launch(); when
// timing is switched on (ks_profile_start), launches are bracketed by CUDA
// events recorded on the launching stream, and the elapsed times are
// accumulated per class whenever the stream has been synchronised.
#include <atomic>
#include <mutex>
#include <vector>

#include "ks_internal.cuh"

namespace ks {

namespace {

std::atomic<unsigned long long> g_launches{0};

struct Pending {
  int cls;
  cudaEvent_t a, b;
};

struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  double ms[KS_PROF_CLASSES] = {};
  long long count[KS_PROF_CLASSES] = {};
  double flops[KS_PROF_CLASSES] = {};
  double bytes[KS_PROF_CLASSES] = {};
} g_prof;

cudaEvent_t take_event() {
  if (!g_prof.pool.empty()) {
    cudaEvent_t e = g_prof.pool.back();
    g_prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Resolve completed event pairs (all of them when `all`).
void resolve(bool all) {
  std::vector<Pending> keep;
  for (auto &p : g_prof.pending) {
    if (!all && cudaEventQuery(p.b) != cudaSuccess) {
      cudaGetLastError();
      keep.push_back(p);
      continue;
    }
    float t = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      g_prof.ms[p.cls] += t;
      g_prof.count[p.cls] += 1;
    }
    cudaGetLastError();
    g_prof.pool.push_back(p.a);
    g_prof.pool.push_back(p.b);
  }
  g_prof.pending.swap(keep);
}

const char *kNames[KS_PROF_CLASSES] = {
    "density", "hartree_cg", "potential", "hamiltonian", "mass", "mass_inverse",
    "gram", "combine", "small_factor", "reduce", "setup", "other"};

}  // namespace

ProfScope::ProfScope(cudaStream_t s, int cls, double flops, double bytes, int nlaunch)
    : stream(s), cls(cls), a(nullptr) {
  g_launches.fetch_add((unsigned long long)nlaunch, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.on) return;
  g_prof.flops[cls] += flops;
  g_prof.bytes[cls] += bytes;
  a = take_event();
  if (a) cudaEventRecord((cudaEvent_t)a, stream);
}

ProfScope::~ProfScope() {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t b = take_event();
  if (!b) {
    g_prof.pool.push_back((cudaEvent_t)a);
    return;
  }
  cudaEventRecord(b, stream);
  g_prof.pending.push_back({cls, (cudaEvent_t)a, b});
  if (g_prof.pending.size() > 4096) resolve(false);
}

bool prof_enabled() {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  return g_prof.on;
}

void count_launches(long long delta) {
  if (delta >= 0) g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed);
  else g_launches.fetch_sub((unsigned long long)(-delta), std::memory_order_relaxed);
}

void prof_collect() {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!g_prof.pending.empty()) resolve(false);
}

}  // namespace ks

extern "C" {

unsigned long long ks_kernel_launches(void) {
  return ks::g_launches.load(std::memory_order_relaxed);
}

ks_status ks_profile_start(void) {
  std::lock_guard<std::mutex> lk(ks::g_prof.mu);
  ks::resolve(true);
  for (int i = 0; i < KS_PROF_CLASSES; ++i) {
    ks::g_prof.ms[i] = 0.0;
    ks::g_prof.count[i] = 0;
    ks::g_prof.flops[i] = 0.0;
    ks::g_prof.bytes[i] = 0.0;
  }
  ks::g_prof.on = true;
  return KS_OK;
}

ks_status ks_profile_stop(double ms[KS_PROF_CLASSES], long long counts[KS_PROF_CLASSES]) {
  std::lock_guard<std::mutex> lk(ks::g_prof.mu);
  ks::resolve(true);
  ks::g_prof.on = false;
  for (int i = 0; i < KS_PROF_CLASSES; ++i) {
    if (ms) ms[i] = ks::g_prof.ms[i];
    if (counts) counts[i] = ks::g_prof.count[i];
  }
  return KS_OK;
}

ks_status ks_profile_work(double flops[KS_PROF_CLASSES], double bytes[KS_PROF_CLASSES]) {
  std::lock_guard<std::mutex> lk(ks::g_prof.mu);
  for (int i = 0; i < KS_PROF_CLASSES; ++i) {
    if (flops) flops[i] = ks::g_prof.flops[i];
    if (bytes) bytes[i] = ks::g_prof.bytes[i];
  }
  return KS_OK;
}

const char *ks_profile_class_name(int cls) {
  if (cls < 0 || cls >= KS_PROF_CLASSES) return "";
  return ks::kNames[cls];
}

}  // extern "C"

#ifdef KS_DEBUG_BOUNDS
namespace ks {
void oob_read_stencil(unsigned long long *, int *);
void oob_read_blas(unsigned long long *, int *);
void oob_read_density(unsigned long long *, int *);
void oob_read_minv(unsigned long long *, int *);
void oob_read_cg(unsigned long long *, int *);
void oob_read_split(unsigned long long *, int *);
void oob_read_tc(unsigned long long *, int *);
}  // namespace ks
#endif

extern "C" int ks_debug_bounds(unsigned long long *count, const char **file, int *line) {
  unsigned long long total = 0;
  const char *first_file = nullptr;
  int first_line = 0;
#ifdef KS_DEBUG_BOUNDS
  struct Reader {
    const char *file;
    void (*read)(unsigned long long *, int *);
  };
  const Reader readers[] = {{"ks_stencil.cu", ks::oob_read_stencil},
                            {"ks_blas.cu", ks::oob_read_blas},
                            {"ks_density.cu", ks::oob_read_density},
                            {"ks_minv.cu", ks::oob_read_minv},
                            {"ks_cg.cu", ks::oob_read_cg},
                            {"ks_split.cu", ks::oob_read_split},
                            {"ks_tc.cu", ks::oob_read_tc}};
  for (const Reader &r : readers) {
    unsigned long long c = 0;
    int l = 0;
    r.read(&c, &l);
    if (c && !first_file) {
      first_file = r.file;
      first_line = l;
    }
    total += c;
  }
#endif
  if (count) *count = total;
  if (file) *file = first_file;
  if (line) *line = first_line;
#ifdef KS_DEBUG_BOUNDS
  return 1;
#else
  return 0;
#endif
}
