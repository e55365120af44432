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
// Increment form of the QR step (Alg. ChQR with the exact trial Gram
// W = Y^T M Y = I + E, E = tau^2 R - tau (T + T^T), R = D^T M D,
// T = X^T M D): the Cholesky factor and its inverse carried as deviations
// from the identity, L = I + G and L^{-1} = I + H, in FP32.  G and H are of
// the size of E, so every rounding error is relative to |E| -- the size of
// A - I = L^{-T} - I, which the three-term update applies in FP32 anyway --
// where a plain FP32 Cholesky of W would err by eps_32 relative to 1.  The
// recurrences are those of the right-looking Cholesky of W with the unit
// diagonal kept implicit (e' is the trailing part of E):
//   pivot   (1 + g_jj)^2 = 1 + e'_jj, g_jj = e'_jj / (1 + sqrt(1 + e'_jj))
//   column  g_ij = e'_ij / (1 + g_jj)                  (i > j)
//   update  e'_ic -= g_ij g_cj                         (j < c <= i)
// and of V = L^{-1} = I + H built alongside: row j of V divided by 1 + g_jj
// (h_jj = -g_jj / (1 + g_jj)), then V_ic -= g_ij V_jc for c <= j.  Output:
// the FP32 coefficients of the update X_b (A - I) + delta A + D B with
// A = L^{-T} = I + H^T and B = -tau A, as [H^T; I + H^T; -tau (I + H^T)].
// One block of 256 threads, a thread per column of four rows at a time in
// the trailing update; every thread forms the pivot itself, so a column
// costs two barriers.  G
// and H (row stride p + 1, so that column reads do not collide in a bank)
// and column j of G live in dynamic shared memory; a non-positive or
// non-finite pivot records KS_ENOTPD and leaves P.cf as it was.
constexpr int kDevThreads = 256;
constexpr int kDevMaxP = 64;

__global__ void __launch_bounds__(kDevThreads) qr_factor_dev_kernel(int p,
                                                                    const float *__restrict__ R,
                                                                    const float *__restrict__ T,
                                                                    float tau, float *__restrict__ cf,
                                                                    int *status) {
  extern __shared__ float dev_sh[];
  const int ld = p + 1;
  float *G = dev_sh, *H = dev_sh + p * ld, *colj = dev_sh + 2 * p * ld;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarps = kDevThreads / 32;
  // E (lower triangle) with all loads of a thread issued first
  {
    float r[kDevMaxP / kWarps][2], t1[kDevMaxP / kWarps][2], t2[kDevMaxP / kWarps][2];
#pragma unroll
    for (int a = 0; a < kDevMaxP / kWarps; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int i = w + kWarps * a, c = lane + 32 * b;
        const bool in = i < p && c < p && c <= i;
        r[a][b] = in ? R[i * p + c] : 0.f;
        t1[a][b] = in ? T[i * p + c] : 0.f;
        t2[a][b] = in ? T[c * p + i] : 0.f;
      }
#pragma unroll
    for (int a = 0; a < kDevMaxP / kWarps; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int i = w + kWarps * a, c = lane + 32 * b;
        if (i < p && c < p) {
          G[i * ld + c] = fmaf(tau * tau, r[a][b], -tau * (t1[a][b] + t2[a][b]));
          H[i * ld + c] = 0.f;
        }
      }
  }
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const float t = G[j * ld + j];
    const float wv = 1.f + t;
    if (!(wv > 0.f) || !isfinite(wv)) {
      if (threadIdx.x == 0) atomicCAS(status, 0, (int)KS_ENOTPD);
      return;
    }
    const float gjj = t / (1.f + sqrtf(wv));
    const float il = 1.f / (1.f + gjj);
    const float hjj = -gjj * il;
    for (int i = j + 1 + threadIdx.x; i < p; i += kDevThreads) {
      if (!KS_IN(i * ld + j, p * ld)) continue;
      const float g = G[i * ld + j] * il;
      G[i * ld + j] = g;
      colj[i] = g;
    }
    for (int c = threadIdx.x; c < j; c += kDevThreads) H[j * ld + c] *= il;
    if (threadIdx.x == 0) H[j * ld + j] = hjj;
    __syncthreads();
    // rows i > j, four at a time (row group tid / 64, column tid % 64): the
    // updates of different rows are independent, so a thread's loads of
    // four rows are in flight together
    {
      const int c = threadIdx.x & 63, r0 = j + 1 + (threadIdx.x >> 6);
      if (c < p) {
        const float hjc = c < j ? H[j * ld + c] : 0.f;
        const float gcj = c > j ? colj[c] : 0.f;
#pragma unroll 4
        for (int i = r0; i < p; i += 4) {
          if (c > i || !KS_IN(i * ld + c, p * ld)) continue;
          const float gij = colj[i];
          if (c > j) G[i * ld + c] = fmaf(-gij, gcj, G[i * ld + c]);
          else if (c < j) H[i * ld + c] = fmaf(-gij, hjc, H[i * ld + c]);
          else H[i * ld + j] = -fmaf(gij, hjj, gij);
        }
      }
    }
    __syncthreads();
  }
  const int pp = p * p;
  for (int i = w; i < p; i += kWarps)
    for (int c = lane; c < p; c += 32) {
      const float h = H[c * ld + i];                 // (L^{-T} - I)_{ic} = H_{ci}
      const float a = (i == c ? 1.f : 0.f) + h;
      cf[i * p + c] = h;
      cf[pp + i * p + c] = a;
      cf[2 * pp + i * p + c] = -tau * a;
    }
}

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

bool qr_factor_dev_applies(const Problem &P) { return P.p <= kDevMaxP; }

ks_status launch_qr_factor_dev(Problem &P, const float *rt32, double tau) {
  if (!qr_factor_dev_applies(P)) return set_error(KS_EINVAL, "qr_factor_dev: p above %d", kDevMaxP);
  const int p = P.p;
  const size_t smem = ((size_t)2 * p * (p + 1) + p) * sizeof(float);
  {
    ProfScope ps_(P.stream, KP_SMALL);
    qr_factor_dev_kernel<<<1, kDevThreads, smem, P.stream>>>(p, rt32, rt32 + (size_t)p * p,
                                                             (float)tau, P.cf, P.dstatus);
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

KS_OOB_READER(split)

}  // namespace ks
