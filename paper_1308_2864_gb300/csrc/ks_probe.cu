// Peak-rate probe of the FP64 and FP32 FMA pipes (ks_probe_fma in
// include/ks_steps.h).  The roofline of every n p^2 contraction in FP64 and
// of the FP32 SIMT kernels is the FMA rate of the part as it runs now (clock,
// power cap), so the benchmark measures it in the same job instead of taking
// it from a data sheet.
//
// Each thread keeps a 4 x 4 block of accumulators and updates it with the
// outer product of two 4-vectors held in registers, acc[i][j] += x[i] y[j],
// `iters` times: sixteen independent FMA chains per thread with distinct
// register operands, the shape of the inner loop of the Gram and update
// kernels, and no memory traffic.  The sum is stored only under a condition
// the recurrence cannot meet, which the compiler cannot prove, so the FMAs
// are kept.
#include "ks_internal.cuh"
#include "ks_steps.h"

namespace ks {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeFmaPerIter = 16;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, T seed, double *sink) {
  T x[4], y[4], acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    x[i] = seed * (T)(1 + i) + (T)threadIdx.x * (T)1e-9;
    y[i] = seed * (T)(5 - i);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  // four rounds per trip keep the loop's own instructions to a few per 64 FMAs
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
  }
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[i][j];
  if (s == (T)-12345.0) sink[blockIdx.x] = (double)s;
}

}  // namespace
}  // namespace ks

using namespace ks;

extern "C" {

ks_status ks_probe_fma(int fp64, int blocks, int iters, void *stream, double *sink,
                       double *flops) {
  if (!sink || !flops) return set_error(KS_EINVAL, "null argument");
  if (blocks < 1 || iters < 1) return set_error(KS_EINVAL, "blocks and iters must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  // the accumulators grow by at most 20 seed^2 per round: no overflow and no
  // denormals for any iteration count the caller can time
  {
    ProfScope ps_(s, KP_OTHER);
    if (fp64)
      fma_probe_kernel<double><<<blocks, kProbeThreads, 0, s>>>(iters, 1e-3, sink);
    else
      fma_probe_kernel<float><<<blocks, kProbeThreads, 0, s>>>(iters, 1e-3f, sink);
  }
  KS_CUDA_TRY(cudaGetLastError());
  // rounds are done four at a time
  const double rounds = 4.0 * (double)((iters + 3) / 4);
  *flops = 2.0 * kProbeFmaPerIter * rounds * (double)blocks * kProbeThreads;
  return KS_OK;
}

}  // extern "C"
