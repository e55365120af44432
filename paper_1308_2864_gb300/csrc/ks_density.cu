// Density rho = f diag(X X^T) (Sec. 2.3, rho(X) = diag(X X^T), with the
// occupation f of each orbital).  X is FP64 or FP32 (mixed precision: the
// row sum of p squares is accumulated in the storage precision); rho is
// always FP64.
#include "ks_device.cuh"

namespace ks {

// p >= 32: a warp takes 32 consecutive nodes, eight at a time; for each
// node the lanes stride over its row (coalesced) and a fixed butterfly sums
// the row.  The eight rows are loaded before any is used, so a lane has
// eight loads in flight.  Lane l keeps the sum of node l of the group and
// converts and stores it once: the FP64 tail is one warp instruction per 32
// nodes, not one per node (every FP64 warp instruction is a 16-cycle issue).
constexpr int kDenRows = 8;

template <typename T>
__global__ void density_warp_kernel(int n, int p, double occ, const T *__restrict__ X,
                                    double *__restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k0 = warp * 32; k0 < n; k0 += nwarps * 32) {
    T mine = 0;
    const int cnt = (int)min(32LL, (long long)n - k0);
    for (int j0 = 0; j0 < cnt; j0 += kDenRows) {
      T acc[kDenRows];
#pragma unroll
      for (int u = 0; u < kDenRows; ++u) acc[u] = 0;
      for (int i = lane; i < p; i += 32) {
        T v[kDenRows];
#pragma unroll
        for (int u = 0; u < kDenRows; ++u)
          v[u] = j0 + u < cnt ? X[(k0 + j0 + u) * p + i] : (T)0;
#pragma unroll
        for (int u = 0; u < kDenRows; ++u) acc[u] = fma(v[u], v[u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < kDenRows; ++u) {
        T a = acc[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == j0 + u) mine = a;
      }
    }
    if (lane < cnt) rho[k0 + lane] = occ * (double)mine;
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
    const long long warps = (P.n + 31) / 32;
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

// Increment form of the FP32 phase (X = X_b + delta, base hi part xb):
// rho = rho_b + f sum_i delta_i (2 xb_i + delta_i), with rho_b = f sum X_b^2
// in FP64.  The FP32 row sum carries rounding relative to the increment, not
// to rho, so the density of the iterate stays accurate to the FP64 level of
// rho_b plus eps_32 |delta| |X|.
__global__ void density_inc_warp_kernel(int n, int p, double occ, const float *__restrict__ d,
                                        const float *__restrict__ xb,
                                        const double *__restrict__ rho_b,
                                        double *__restrict__ rho) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long k0 = warp * 32; k0 < n; k0 += nwarps * 32) {
    float mine = 0;
    const int cnt = (int)min(32LL, (long long)n - k0);
    for (int j0 = 0; j0 < cnt; j0 += kDenRows) {
      float acc[kDenRows];
#pragma unroll
      for (int u = 0; u < kDenRows; ++u) acc[u] = 0;
      for (int i = lane; i < p; i += 32) {
        float vd[kDenRows], vx[kDenRows];
#pragma unroll
        for (int u = 0; u < kDenRows; ++u) {
          const long long idx = (k0 + j0 + u) * p + i;
          const bool ok = j0 + u < cnt && KS_IN(idx, (long long)n * p);
          vd[u] = ok ? d[idx] : 0.f;
          vx[u] = ok ? xb[idx] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kDenRows; ++u) acc[u] = fmaf(vd[u], fmaf(2.f, vx[u], vd[u]), acc[u]);
      }
#pragma unroll
      for (int u = 0; u < kDenRows; ++u) {
        float a = acc[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == j0 + u) mine = a;
      }
    }
    if (lane < cnt) rho[k0 + lane] = rho_b[k0 + lane] + occ * (double)mine;
  }
}

__global__ void density_inc_thread_kernel(int n, int p, double occ, const float *__restrict__ d,
                                          const float *__restrict__ xb,
                                          const double *__restrict__ rho_b,
                                          double *__restrict__ rho) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float *rd = d + k * p;
  const float *rx = xb + k * p;
  float acc = 0;
  for (int i = 0; i < p; ++i) acc = fmaf(rd[i], fmaf(2.f, rx[i], rd[i]), acc);
  rho[k] = rho_b[k] + occ * (double)acc;
}

ks_status launch_density_inc(Problem &P, const float *d, const float *xb, const double *rho_b,
                             double *rho) {
  const double bytes = 8.0 * P.n * P.p + 16.0 * P.n;
  if (P.p >= 32) {
    const long long warps = (P.n + 31) / 32;
    long long blocks = (warps * 32 + kThreads - 1) / kThreads;
    if (blocks > 64LL * P.sms) blocks = 64LL * P.sms;
    ProfScope ps_(P.stream, KP_DENSITY, 3.0 * P.n * P.p, bytes);
    density_inc_warp_kernel<<<(int)blocks, kThreads, 0, P.stream>>>(P.n, P.p, P.occ, d, xb,
                                                                     rho_b, rho);
  } else {
    ProfScope ps_(P.stream, KP_DENSITY, 3.0 * P.n * P.p, bytes);
    density_inc_thread_kernel<<<(P.n + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(
        P.n, P.p, P.occ, d, xb, rho_b, rho);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Batched: one thread per node of every active job.
template <typename T>
__global__ void density_batch_kernel(const BJob *__restrict__ jobs, const int *__restrict__ start,
                                     int J, const unsigned char *__restrict__ active, int sX) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const long long k = (long long)(blockIdx.x - start[j]) * blockDim.x + threadIdx.x;
  if (k >= b.n) return;
  const int p = b.p;
  const T *row = (const T *)b.blk[sX] + k * p;
  T acc = 0;
  for (int i = 0; i < p; ++i) acc = fma(row[i], row[i], acc);
  b.rho[k] = b.occ * (double)acc;
}

template <typename T>
ks_status batch_density(Batch &B, int sX) {
  const int nb = B.total(BM_DENSITY);
  if (nb == 0) return KS_OK;
  {
    ProfScope ps_(B.stream, KP_DENSITY);
    density_batch_kernel<T><<<nb, kThreads, 0, B.stream>>>(B.jobs_dev, B.map(BM_DENSITY), B.J,
                                                           B.active_dev, sX);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template ks_status batch_density<double>(Batch &, int);
template ks_status batch_density<float>(Batch &, int);

template ks_status launch_density<double>(Problem &, const double *, double *);
template ks_status launch_density<float>(Problem &, const float *, double *);

KS_OOB_READER(density)

}  // namespace ks
