// Elementwise kernels of the FP32 phase that carries its iterate as an FP64
// base plus an FP32 increment, X = X_b + delta (the "increment form" of the
// mixed-precision minimisation; the paper computes in FP64 throughout).
//
// The base X_b is held as two FP32 blocks, hi = fl32(X_b) and
// lo = fl32(X_b - hi), so X_b = hi + lo exactly to 48 bits; the FP64 value is
// formed only when the base is refreshed.  Rounding errors of the FP32 work
// then scale with |delta| instead of |X|: the energies that the line search
// of Eq. NMLS-Armijo compares stay accurate far below the FP32 rounding of
// the orbitals themselves.
#include "ks_device.cuh"

namespace ks {
namespace {

__global__ void split_join_kernel(long long len, const float *__restrict__ hi,
                                  const float *__restrict__ lo, const float *__restrict__ d,
                                  double *__restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = ((double)hi[i] + (double)lo[i]) + (double)d[i];
}

__global__ void split_hilo_kernel(long long len, const double *__restrict__ x,
                                  float *__restrict__ hi, float *__restrict__ lo) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

// out may be the same array as a (in-place update)
__global__ void axpy_f32_kernel(long long len, const float *a, float s, const float *b,
                                float *out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] + s * b[i];
}

__global__ void add_f64_f32_kernel(long long len, double *__restrict__ x,
                                   const float *__restrict__ d) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

// out may be the same array as A
__global__ void add_identity_kernel(int p, const double *A, double s, double *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * p; i += gridDim.x * blockDim.x)
    out[i] = A[i] + (i / p == i % p ? s : 0.0);
}

// C = alpha op(A) op(B) + beta C for p x p row-major FP64 matrices
// (op = transpose when the flag is set); 16 x 16 output tiles, K staged in
// shared memory in chunks of 16.  C must not alias A or B.
constexpr int kSg = 16;
__global__ void small_gemm_kernel(int p, int ta, const double *__restrict__ A, int tb,
                                  const double *__restrict__ B, double alpha, double beta,
                                  double *__restrict__ C) {
  __shared__ double As[kSg][kSg + 1], Bs[kSg][kSg + 1];
  const int tx = threadIdx.x % kSg, ty = threadIdx.x / kSg;
  const int row = blockIdx.y * kSg + ty, col = blockIdx.x * kSg + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < p; k0 += kSg) {
    // As[ty][tx] = op(A)[row][k0 + tx], Bs[ty][tx] = op(B)[k0 + ty][col]
    const int ka = k0 + tx, kb = k0 + ty;
    double a = 0.0, b = 0.0;
    if (row < p && ka < p) a = ta ? A[(size_t)ka * p + row] : A[(size_t)row * p + ka];
    if (col < p && kb < p) b = tb ? B[(size_t)col * p + kb] : B[(size_t)kb * p + col];
    As[ty][tx] = a;
    Bs[ty][tx] = b;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSg; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (row < p && col < p) {
    const size_t i = (size_t)row * p + col;
    C[i] = alpha * acc + (beta != 0.0 ? beta * C[i] : 0.0);
  }
}

// out = A + s B (p x p); out may be A or B
__global__ void add_pp_kernel(int p, const double *A, double s, const double *B, double *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * p; i += gridDim.x * blockDim.x)
    out[i] = A[i] + s * B[i];
}

// out = R - (T + T^T) / tau: with it, I + tau^2 out = I - tau (T + T^T) + tau^2 R
// is the exact Gram (X - tau D)^T M (X - tau D) when X^T M X = I, T = X^T M D
// and R = D^T M D.
__global__ void qr_exact_gram_kernel(int p, const double *__restrict__ R,
                                     const double *__restrict__ T, double tau,
                                     double *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * p; i += gridDim.x * blockDim.x) {
    const int r = i / p, c = i % p;
    out[i] = R[i] - (T[i] + T[(size_t)c * p + r]) / tau;
  }
}

// out = X + Y + Y^T (p x p)
__global__ void sym_add_kernel(int p, const double *__restrict__ X, const double *__restrict__ Y,
                               double *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p * p; i += gridDim.x * blockDim.x) {
    const int r = i / p, c = i % p;
    out[i] = X[i] + (Y[i] + Y[(size_t)c * p + r]);
  }
}

int stream_blocks(const Problem &P, long long len) {
  long long b = (len + kThreads - 1) / kThreads;
  const long long cap = 16LL * P.sms;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

ks_status launch_split_join(Problem &P, const float *hi, const float *lo, const float *d,
                            double *out) {
  const long long len = (long long)P.n * P.p;
  {
    ProfScope ps_(P.stream, KP_OTHER, (double)len * 2, (double)len * 20);
    split_join_kernel<<<stream_blocks(P, len), kThreads, 0, P.stream>>>(len, hi, lo, d, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_split_hilo(Problem &P, const double *x, float *hi, float *lo) {
  const long long len = (long long)P.n * P.p;
  {
    ProfScope ps_(P.stream, KP_OTHER, (double)len, (double)len * 16);
    split_hilo_kernel<<<stream_blocks(P, len), kThreads, 0, P.stream>>>(len, x, hi, lo);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_axpy_f32(Problem &P, const float *a, float s, const float *b, float *out) {
  const long long len = (long long)P.n * P.p;
  {
    ProfScope ps_(P.stream, KP_OTHER, (double)len * 2, (double)len * 12);
    axpy_f32_kernel<<<stream_blocks(P, len), kThreads, 0, P.stream>>>(len, a, s, b, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_add_f64_f32(Problem &P, double *x, const float *d) {
  const long long len = (long long)P.n * P.p;
  {
    ProfScope ps_(P.stream, KP_OTHER, (double)len, (double)len * 20);
    add_f64_f32_kernel<<<stream_blocks(P, len), kThreads, 0, P.stream>>>(len, x, d);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_small_gemm(Problem &P, int ta, const double *A, int tb, const double *B,
                            double alpha, double beta, double *C) {
  const int t = (P.p + kSg - 1) / kSg;
  {
    ProfScope ps_(P.stream, KP_SMALL, 2.0 * P.p * P.p * P.p);
    small_gemm_kernel<<<dim3(t, t), kSg * kSg, 0, P.stream>>>(P.p, ta, A, tb, B, alpha, beta, C);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_add_pp(Problem &P, const double *A, double s, const double *B, double *out) {
  const int len = P.p * P.p;
  {
    ProfScope ps_(P.stream, KP_SMALL);
    add_pp_kernel<<<(len + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(P.p, A, s, B, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_qr_exact_gram(Problem &P, const double *R, const double *T, double tau,
                               double *out) {
  const int len = P.p * P.p;
  {
    ProfScope ps_(P.stream, KP_SMALL);
    qr_exact_gram_kernel<<<(len + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(P.p, R, T,
                                                                                    tau, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_sym_add(Problem &P, const double *X, const double *Y, double *out) {
  const int len = P.p * P.p;
  {
    ProfScope ps_(P.stream, KP_SMALL);
    sym_add_kernel<<<(len + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(P.p, X, Y, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_add_identity(Problem &P, const double *A, double s, double *out) {
  const int len = P.p * P.p;
  {
    ProfScope ps_(P.stream, KP_SMALL);
    add_identity_kernel<<<(len + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(P.p, A, s,
                                                                                   out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

}  // namespace ks
