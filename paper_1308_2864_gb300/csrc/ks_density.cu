// Density rho = f diag(X X^T) (Sec. 2.3, rho(X) = diag(X X^T), with the
// occupation f of each orbital).  X is FP64 or FP32 (mixed precision: the
// row sum of p squares is accumulated in the storage precision); rho is
// always FP64.
#include "ks_device.cuh"

namespace ks {

// p >= 32: one warp per node, lanes stride over the node's row (coalesced),
// fixed butterfly sum.
template <typename T>
__global__ void density_warp_kernel(int n, int p, double occ, const T *__restrict__ X,
                                    double *__restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k = warp; k < n; k += nwarps) {
    const T *row = X + k * p;
    T acc = 0;
    for (int i = lane; i < p; i += 32) {
      const T x = row[i];
      acc = fma(x, x, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rho[k] = occ * (double)acc;
  }
}

// p < 32: one thread per node.
template <typename T>
__global__ void density_thread_kernel(int n, int p, double occ, const T *__restrict__ X,
                                      double *__restrict__ rho) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const T *row = X + k * p;
  T acc = 0;
  for (int i = 0; i < p; ++i) acc = fma(row[i], row[i], acc);
  rho[k] = occ * (double)acc;
}

template <typename T>
ks_status launch_density(Problem &P, const T *X, double *rho) {
  if (P.p >= 32) {
    const long long warps = P.n;
    long long blocks = (warps * 32 + kThreads - 1) / kThreads;
    if (blocks > 64LL * P.sms) blocks = 64LL * P.sms;
    ProfScope ps_(P.stream, KP_DENSITY, 2.0 * P.n * P.p, (double)P.n * P.p * sizeof(T) + 8.0 * P.n);
    density_warp_kernel<T><<<(int)blocks, kThreads, 0, P.stream>>>(P.n, P.p, P.occ, X, rho);
  } else {
    ProfScope ps_(P.stream, KP_DENSITY, 2.0 * P.n * P.p, (double)P.n * P.p * sizeof(T) + 8.0 * P.n);
    density_thread_kernel<T><<<(P.n + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(
        P.n, P.p, P.occ, X, rho);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template ks_status launch_density<double>(Problem &, const double *, double *);
template ks_status launch_density<float>(Problem &, const float *, double *);

}  // namespace ks
