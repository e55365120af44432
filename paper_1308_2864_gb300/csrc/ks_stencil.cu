// 27-point Q1 stencils over blocks of orbitals (row-major n x p, orbital
// index fastest, so a warp reading one neighbour of consecutive orbitals is
// a coalesced access).
//
//   hamiltonian:  E_X = f K X + 2 f h^3 Diag(V_eff) X   (the derivative of
//                 Eq. EKS discretised, Sec. 2.3's E_X = H(X) X), M X, and
//                 the kinetic energy (f/2) sum X . K X
//   mass:         M X
//   mass_dots:    M D, ||D||_M^2 = sum D . M D and the Barzilai-Borwein
//                 traces of Eq. bb-1 in the M inner product.
#include "ks_device.cuh"

namespace ks {

// Neighbour sums of one orbital column around node (ix, iy, iz) by class:
// centre, faces, edges, corners (Dirichlet: outside nodes are zero).
template <typename T>
struct ClassSums {
  T s0, sf, se, sc;
};

template <typename T>
__device__ __forceinline__ ClassSums<T> class_sums(const T *__restrict__ A, int p, int i,
                                                   int N, int ix, int iy, int iz) {
  ClassSums<T> s{0, 0, 0, 0};
  const long long NN = (long long)N * N;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = iz + dz;
    if (z < 0 || z >= N) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = iy + dy;
      if (y < 0 || y >= N) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = ix + dx;
        if (x < 0 || x >= N) continue;
        const int nzc = (dx != 0) + (dy != 0) + (dz != 0);
        const T v = __ldg(A + (z * NN + (long long)y * N + x) * p + i);
        if (nzc == 0) s.s0 = v;
        else if (nzc == 1) s.sf += v;
        else if (nzc == 2) s.se += v;
        else s.sc += v;
      }
    }
  }
  return s;
}

// T = double (FP64 path) or float (mixed path: stencil arithmetic in FP32,
// per-thread partial sums in FP32, block and grid sums in FP64).
template <typename T>
__global__ void hamiltonian_kernel(int N, int p, long long total, StencilCoef cd, double occ_d,
                                   double h3, const T *__restrict__ X,
                                   const double *__restrict__ veff, T *__restrict__ EX,
                                   T *__restrict__ MX, double *__restrict__ part) {
  __shared__ double smem[33];
  const T k0 = (T)cd.k0, ke = (T)cd.ke, kc = (T)cd.kc;
  const T m0 = (T)cd.m0, mf = (T)cd.mf, me = (T)cd.me, mc = (T)cd.mc;
  const T occ = (T)occ_d, vscale = (T)(2.0 * occ_d * h3);
  T kin = 0;
  const long long NN = (long long)N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / p;
    const int i = (int)(e - k * p);
    const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
    const ClassSums<T> s = class_sums<T>(X, p, i, N, ix, iy, iz);
    const T kx = k0 * s.s0 + ke * s.se + kc * s.sc;   // face coefficient is 0
    EX[e] = occ * kx + vscale * (T)veff[k] * s.s0;
    if (MX) MX[e] = m0 * s.s0 + mf * s.sf + me * s.se + mc * s.sc;
    kin = fma(s.s0, kx, kin);
  }
  const double sb = block_sum((double)kin, smem);
  if (threadIdx.x == 0) part[blockIdx.x] = sb;
}

// Mode 0: MX = M X only.  Mode 1: MD = M D and sum D.MD.  Mode 2: as 1 plus
// the three BB traces against the previous iterate.
template <typename T, int Mode>
__global__ void mass_kernel(int N, int p, long long total, StencilCoef cd,
                            const T *__restrict__ D, T *__restrict__ MD,
                            const T *__restrict__ X, const T *__restrict__ MX,
                            const T *__restrict__ Xp, const T *__restrict__ MXp,
                            const T *__restrict__ Dp, const T *__restrict__ MDp,
                            double *__restrict__ part) {
  __shared__ double smem[33];
  const T m0 = (T)cd.m0, mf = (T)cd.mf, me = (T)cd.me, mc = (T)cd.mc;
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const long long NN = (long long)N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / p;
    const int i = (int)(e - k * p);
    const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
    const ClassSums<T> s = class_sums<T>(D, p, i, N, ix, iy, iz);
    const T md = m0 * s.s0 + mf * s.sf + me * s.se + mc * s.sc;
    MD[e] = md;
    if (Mode >= 1) a0 = fma(s.s0, md, a0);
    if (Mode == 2) {
      const T dx = X[e] - Xp[e];
      const T dmx = MX[e] - MXp[e];
      const T dd = s.s0 - Dp[e];
      const T dmd = md - MDp[e];
      a1 = fma(dx, dmx, a1);
      a2 = fma(dx, dmd, a2);
      a3 = fma(dd, dmd, a3);
    }
  }
  if (Mode >= 1) {
    const int nb = gridDim.x;
    const double s0 = block_sum((double)a0, smem);
    if (threadIdx.x == 0) part[blockIdx.x] = s0;
    if (Mode == 2) {
      const double s1 = block_sum((double)a1, smem);
      const double s2 = block_sum((double)a2, smem);
      const double s3 = block_sum((double)a3, smem);
      if (threadIdx.x == 0) {
        part[nb + blockIdx.x] = s1;
        part[2 * nb + blockIdx.x] = s2;
        part[3 * nb + blockIdx.x] = s3;
      }
    }
  }
}

template <typename T>
ks_status launch_hamiltonian(Problem &P, const T *X, const double *veff, T *EX, T *MX,
                             double *ekin_out) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  const double h3 = P.h * P.h * P.h;
  {
    ProfScope ps_(P.stream, KP_HAMILTONIAN, 34.0 * total, (double)total * sizeof(T) * (MX ? 3 : 2) + 8.0 * P.n);
    hamiltonian_kernel<T><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, q1_coefficients(P.h),
                                                         P.occ, h3, X, veff, EX, MX, P.partials);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return launch_reduce(P, P.partials, 1, nb, ekin_out, 0.5 * P.occ);
}

template <typename T>
ks_status launch_mass(Problem &P, const T *X, T *MX) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  {
    ProfScope ps_(P.stream, KP_MASS, 30.0 * total, 2.0 * total * sizeof(T));
    mass_kernel<T, 0><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, q1_coefficients(P.h), X,
                                                     MX, nullptr, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr, nullptr);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template <typename T>
ks_status launch_mass_dots(Problem &P, const T *D, T *MD, const T *X, const T *MX,
                           const BBPrevT<T> *prev, double *out4) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  const StencilCoef c = q1_coefficients(P.h);
  if (prev) {
    {
      ProfScope ps_(P.stream, KP_MASS, 40.0 * total, 8.0 * total * sizeof(T));
      mass_kernel<T, 2><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, c, D, MD, X, MX,
                                                       prev->X, prev->MX, prev->D, prev->MD,
                                                       P.partials);
    }
    KS_CUDA_TRY(cudaGetLastError());
    return launch_reduce(P, P.partials, 4, nb, out4);
  }
  {
    ProfScope ps_(P.stream, KP_MASS, 32.0 * total, 2.0 * total * sizeof(T));
    mass_kernel<T, 1><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, c, D, MD, nullptr,
                                                     nullptr, nullptr, nullptr, nullptr, nullptr,
                                                     P.partials);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return launch_reduce(P, P.partials, 1, nb, out4);
}

#define KS_INST(T)                                                                        \
  template ks_status launch_hamiltonian<T>(Problem &, const T *, const double *, T *, T *, \
                                           double *);                                    \
  template ks_status launch_mass<T>(Problem &, const T *, T *);                          \
  template ks_status launch_mass_dots<T>(Problem &, const T *, T *, const T *, const T *, \
                                         const BBPrevT<T> *, double *);
KS_INST(double)
KS_INST(float)
#undef KS_INST

}  // namespace ks
