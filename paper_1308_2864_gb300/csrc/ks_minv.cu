// G = M^{-1} E for the Q1 consistent mass M = M1 (x) M1 (x) M1,
// M1 = (h/6) tridiag(1, 4, 1): three sweeps of the Thomas algorithm, one
// along each grid axis.  This is the M^{-1} of the projected gradient
// D = M^{-1} E_X - X (E_X^T X), i.e. the B^{-1/2} change of variables of
// Eq. OFDFT-y applied to Eq. def-nablaE.  One thread owns one (grid line,
// orbital) pair; consecutive threads take consecutive orbitals, so every
// access of a warp is a contiguous row segment.
#include "ks_device.cuh"

namespace ks {

// Solve tridiag(1, 4, 1) y = scale * d along one axis, in place on `out`
// (reading `in` on the forward pass).  w holds the pivots 1/(4 - w_{j-1});
// they are copied to shared memory in the working precision once per block
// (a conversion per step would run on the FP64 pipe).  Each sweep reads
// kAhead entries of the line before it writes any of them, so a thread has
// kAhead loads in flight instead of one (in and out may be the same array,
// and the compiler cannot reorder loads across the stores by itself).
constexpr int kAhead = 8;

// One (line, orbital) pair t of a sweep; w: the pivots in shared memory.
// add (nullable, same layout as out): added to every final value written,
// while the recurrence runs on the solution itself.
template <typename T>
__device__ __forceinline__ void thomas_line(long long t, int N, int p, int axis, T scale,
                                            const T *w, const T *in, T *out,
                                            const T *add = nullptr) {
  const long long lines = (long long)N * N;
  if (t >= lines * p) return;
  const int i = (int)(t % p);
  const long long line = t / p;
  const int a = (int)(line % N), b = (int)(line / N);
  long long base, stride;
  if (axis == 0) {        // x lines, (a, b) = (iy, iz)
    base = ((long long)b * N + a) * N;
    stride = 1;
  } else if (axis == 1) { // y lines, (a, b) = (ix, iz)
    base = (long long)b * N * N + a;
    stride = N;
  } else {                // z lines, (a, b) = (ix, iy)
    base = (long long)b * N + a;
    stride = (long long)N * N;
  }
  const T *src = in + base * p + i;
  T *dst = out + base * p + i;
  const long long es = stride * p;
  // forward elimination
  T prev = 0;
  for (int j0 = 0; j0 < N; j0 += kAhead) {
    T v[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u)
      if (j0 + u < N) v[u] = src[(long long)(j0 + u) * es];
#pragma unroll
    for (int u = 0; u < kAhead; ++u)
      if (j0 + u < N) {
        prev = (scale * v[u] - prev) * w[j0 + u];
        dst[(long long)(j0 + u) * es] = prev;
      }
  }
  // back substitution (prev holds entry N-1, which is final)
  if (add) dst[(long long)(N - 1) * es] = prev + add[(base + (long long)(N - 1) * stride) * p + i];
  T next = prev;
  for (int j1 = N - 2; j1 >= 0; j1 -= kAhead) {
    T v[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u)
      if (j1 - u >= 0) v[u] = dst[(long long)(j1 - u) * es];
#pragma unroll
    for (int u = 0; u < kAhead; ++u)
      if (j1 - u >= 0) {
        next = v[u] - w[j1 - u] * next;
        dst[(long long)(j1 - u) * es] =
            add ? next + add[(base + (long long)(j1 - u) * stride) * p + i] : next;
      }
  }
}

// Lines of at most kRegN nodes: the whole line in registers (all its loads
// in flight at once, one read and one write of each entry in memory).
// Indices into the line array are compile-time constants throughout, and
// the recurrences run over all kRegN entries with the pivots w zero past N:
// the padding then stays 0 in both sweeps (the back substitution enters
// entry N - 1 with next = 0), so no data-dependent branch touches the array
// and it stays in registers.
constexpr int kRegN = 64;

template <typename T>
__device__ __forceinline__ void thomas_line_reg(long long t, int N, int p, int axis, T scale,
                                                const T *w, const T *in, T *out, const T *add) {
  const long long lines = (long long)N * N;
  if (t >= lines * p) return;
  const int i = (int)(t % p);
  const long long line = t / p;
  const int a = (int)(line % N), b = (int)(line / N);
  long long base, stride;
  if (axis == 0) {
    base = ((long long)b * N + a) * N;
    stride = 1;
  } else if (axis == 1) {
    base = (long long)b * N * N + a;
    stride = N;
  } else {
    base = (long long)b * N + a;
    stride = (long long)N * N;
  }
  const long long es = stride * p;
  // the line's last entry lies inside the block
  if (!KS_IN(base * p + i + (long long)(N - 1) * es, lines * N * p)) return;
  T v[kRegN];
  {
    const T *ps = in + base * p + i;
#pragma unroll
    for (int u = 0; u < kRegN; ++u) {
      v[u] = u < N ? *ps : (T)0;
      ps += es;
    }
  }
  // forward elimination, then back substitution (w[u] = 0 for u >= N)
  T prev = 0;
#pragma unroll
  for (int u = 0; u < kRegN; ++u) {
    prev = (scale * v[u] - prev) * w[u];
    v[u] = prev;
  }
  T next = 0;
#pragma unroll
  for (int u = kRegN - 1; u >= 0; --u) {
    next = v[u] - w[u] * next;
    v[u] = next;
  }
  if (add) {
    const T *pa = add + base * p + i;
#pragma unroll
    for (int u = 0; u < kRegN; ++u) {
      if (u < N) v[u] += *pa;
      pa += es;
    }
  }
  T *pd = out + base * p + i;
#pragma unroll
  for (int u = 0; u < kRegN; ++u) {
    if (u < N) *pd = v[u];
    pd += es;
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) thomas_reg_kernel(int N, int p, int axis, double scale_d,
                                                         const double *__restrict__ w_d,
                                                         const T *in, T *out, const T *add) {
  __shared__ T w[kRegN];
  for (int j = threadIdx.x; j < kRegN; j += blockDim.x) w[j] = j < N ? (T)w_d[j] : (T)0;
  __syncthreads();
  thomas_line_reg<T>((long long)blockIdx.x * blockDim.x + threadIdx.x, N, p, axis, (T)scale_d, w,
                     in, out, add);
}

template <typename T>
__global__ void __launch_bounds__(256) thomas_kernel(int N, int p, int axis, double scale_d,
                                                     const double *__restrict__ w_d, const T *in,
                                                     T *out, const T *add) {
  extern __shared__ unsigned char thomas_smem[];
  T *w = reinterpret_cast<T *>(thomas_smem);
  for (int j = threadIdx.x; j < N; j += blockDim.x) w[j] = (T)w_d[j];
  __syncthreads();
  thomas_line<T>((long long)blockIdx.x * blockDim.x + threadIdx.x, N, p, axis, (T)scale_d, w, in,
                 out, add);
}

// Batched: the blocks of job j cover its N^2 p (line, orbital) pairs.
template <typename T>
__global__ void __launch_bounds__(256) thomas_batch_kernel(const BJob *__restrict__ jobs,
                                                           const int *__restrict__ start, int J,
                                                           const unsigned char *__restrict__ active,
                                                           int axis, int sIn, int sOut) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  extern __shared__ unsigned char thomas_smem[];
  T *w = reinterpret_cast<T *>(thomas_smem);
  const int N = b.N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = (T)b.thomas_w[i];
  __syncthreads();
  double scale = 1.0;
  if (axis == 0) {
    const double s = 6.0 / b.h;
    scale = s * s * s;
  }
  const T *in = (const T *)b.blk[axis == 0 ? sIn : sOut];
  thomas_line<T>((long long)(blockIdx.x - start[j]) * blockDim.x + threadIdx.x, N, b.p, axis,
                 (T)scale, w, in, (T *)b.blk[sOut]);
}

template <typename T>
ks_status batch_mass_inverse(Batch &B, int sE, int sG) {
  const int nb = B.total(BM_THOMAS);
  if (nb == 0) return KS_OK;
  const size_t smem = (size_t)B.maxN * sizeof(T);
  for (int axis = 0; axis < 3; ++axis) {
    {
      ProfScope ps_(B.stream, KP_MASS_INV);
      thomas_batch_kernel<T><<<nb, kThreads, smem, B.stream>>>(B.jobs_dev, B.map(BM_THOMAS), B.J,
                                                               B.active_dev, axis, sE, sG);
    }
    KS_CUDA_TRY(cudaGetLastError());
  }
  return KS_OK;
}

template ks_status batch_mass_inverse<double>(Batch &, int, int);
template ks_status batch_mass_inverse<float>(Batch &, int, int);

// G = s E elementwise (the inverse of the lumped mass h^3 I), plus add when
// given; E and G may alias.
template <typename T>
__global__ void scale_kernel(long long len, T s, const T *E, T *G, const T *add) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    G[i] = add ? s * E[i] + add[i] : s * E[i];
}

template <typename T>
ks_status launch_mass_inverse(Problem &P, const T *E, T *G, const T *add) {
  if (P.mass == KS_MASS_LUMPED) {
    const long long len = (long long)P.n * P.p;
    long long nb = (len + 4LL * kThreads - 1) / (4LL * kThreads);
    if (nb > 64LL * P.sms) nb = 64LL * P.sms;
    const double h = P.h;
    ProfScope ps_(P.stream, KP_MASS_INV, (double)len, 2.0 * len * sizeof(T));
    scale_kernel<T><<<(int)nb, kThreads, 0, P.stream>>>(len, (T)(1.0 / (h * h * h)), E, G, add);
    KS_CUDA_TRY(cudaGetLastError());
    return KS_OK;
  }
  const long long work = (long long)P.N * P.N * P.p;
  const int nb = (int)((work + kThreads - 1) / kThreads);
  const double s = 6.0 / P.h;
  const size_t smem = (size_t)P.N * sizeof(T);
  // FP32 lines of at most kRegN nodes in registers (in FP64 the sweep is
  // bound by the FP64 pipe, and 64 doubles a thread would halve occupancy)
  const bool reg = sizeof(T) == 4 && P.N <= kRegN;
  for (int axis = 0; axis < 3; ++axis) {
    const T *src = axis == 0 ? E : G;
    const double sc = axis == 0 ? s * s * s : 1.0;
    const T *ad = axis == 2 ? add : nullptr;
    const double bytes = (2.0 + (ad ? 1.0 : 0.0)) * P.n * P.p * sizeof(T);
    ProfScope ps_(P.stream, KP_MASS_INV, 4.0 * P.n * P.p, bytes);
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (reg) {
        thomas_reg_kernel<T><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, axis, sc, P.thomas_w, src,
                                                               G, ad);
        done = true;
      }
    }
    if (!done)
      thomas_kernel<T><<<nb, kThreads, smem, P.stream>>>(P.N, P.p, axis, sc, P.thomas_w, src, G,
                                                         ad);
    KS_CUDA_TRY(cudaGetLastError());
  }
  return KS_OK;
}

template ks_status launch_mass_inverse<double>(Problem &, const double *, double *,
                                               const double *);
template ks_status launch_mass_inverse<float>(Problem &, const float *, float *, const float *);

KS_OOB_READER(minv)

}  // namespace ks
