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
// (reading `in` on the forward pass).  w holds the pivots 1/(4 - w_{j-1}).
template <typename T>
__global__ void thomas_kernel(int N, int p, int axis, double scale_d,
                              const double *__restrict__ w, const T *in, T *out) {
  const T scale = (T)scale_d;
  const long long lines = (long long)N * N;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
  const long long e0 = base * p + i;
  const long long es = stride * p;
  // forward elimination
  T prev = 0;
  for (int j = 0; j < N; ++j) {
    const long long e = e0 + j * es;
    const T d = (scale * in[e] - prev) * (T)w[j];
    out[e] = d;
    prev = d;
  }
  // back substitution
  T next = out[e0 + (long long)(N - 1) * es];
  for (int j = N - 2; j >= 0; --j) {
    const long long e = e0 + j * es;
    next = out[e] - (T)w[j] * next;
    out[e] = next;
  }
}

template <typename T>
ks_status launch_mass_inverse(Problem &P, const T *E, T *G) {
  const long long work = (long long)P.N * P.N * P.p;
  const int nb = (int)((work + kThreads - 1) / kThreads);
  const double s = 6.0 / P.h;
  {
    ProfScope ps_(P.stream, KP_MASS_INV, 4.0 * P.n * P.p, 2.0 * P.n * P.p * sizeof(T));
    thomas_kernel<T><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, 0, s * s * s, P.thomas_w, E, G);
  }
  KS_CUDA_TRY(cudaGetLastError());
  {
    ProfScope ps_(P.stream, KP_MASS_INV, 4.0 * P.n * P.p, 2.0 * P.n * P.p * sizeof(T));
    thomas_kernel<T><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, 1, 1.0, P.thomas_w, G, G);
  }
  KS_CUDA_TRY(cudaGetLastError());
  {
    ProfScope ps_(P.stream, KP_MASS_INV, 4.0 * P.n * P.p, 2.0 * P.n * P.p * sizeof(T));
    thomas_kernel<T><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, 2, 1.0, P.thomas_w, G, G);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template ks_status launch_mass_inverse<double>(Problem &, const double *, double *);
template ks_status launch_mass_inverse<float>(Problem &, const float *, float *);

}  // namespace ks
