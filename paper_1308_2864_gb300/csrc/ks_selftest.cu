// Self-test of the bounded device waits (ks_selftest_wait_timeout in
// include/ks_steps.h).  Every wait in the library -- the software grid
// barrier of the cooperative kernels and the mbarrier waits of the TMA and
// tensor-core pipelines -- polls a bounded number of times, then records
// KS_ETIMEOUT in the launch's status word and returns, so a wait that cannot
// complete leaves the context usable and reaches the host as an error.
//
// The probe runs the library's own grid barrier in a launch of one block
// while the barrier expects two: the second arrival never comes, the
// waiting thread gives up after kSpinLimit polls (about a second with the
// back-off), and the kernel returns with KS_ETIMEOUT recorded.
#include <chrono>

#include "ks_device.cuh"
#include "ks_steps.h"

namespace ks {
namespace {

__global__ void wait_timeout_probe_kernel(GridBarrier *bar, int *status) {
  grid_barrier_n(bar, status, 2u);
}

struct ProbeState {
  GridBarrier bar;
  int status;
};

}  // namespace
}  // namespace ks

using namespace ks;

extern "C" {

ks_status ks_selftest_wait_timeout(void *stream, int *status, double *seconds) {
  if (!status) return set_error(KS_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  ProbeState *d = nullptr;
  KS_CUDA_TRY(cudaMalloc((void **)&d, sizeof(ProbeState)));
  ProbeState h{};
  ks_status st = KS_OK;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(ProbeState), s);
  if (e == cudaSuccess) {
    {
      ProfScope ps_(s, KP_OTHER);
      wait_timeout_probe_kernel<<<1, 32, 0, s>>>(&d->bar, &d->status);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(ProbeState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) st = cuda_error(e, "wait-timeout probe");
  cudaFree(d);
  if (st != KS_OK) return st;
  *status = h.status;
  if (seconds)
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return KS_OK;
}

}  // extern "C"
