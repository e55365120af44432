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
struct ClassSums {
  double s0, sf, se, sc;
};

__device__ __forceinline__ ClassSums class_sums(const double *__restrict__ A, int p, int i,
                                                int N, int ix, int iy, int iz) {
  ClassSums s{0.0, 0.0, 0.0, 0.0};
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
        const double v = __ldg(A + (z * NN + (long long)y * N + x) * p + i);
        if (nzc == 0) s.s0 = v;
        else if (nzc == 1) s.sf += v;
        else if (nzc == 2) s.se += v;
        else s.sc += v;
      }
    }
  }
  return s;
}

__global__ void hamiltonian_kernel(int N, int p, long long total, StencilCoef c, double occ,
                                   double h3, const double *__restrict__ X,
                                   const double *__restrict__ veff, double *__restrict__ EX,
                                   double *__restrict__ MX, double *__restrict__ part) {
  __shared__ double smem[33];
  double kin = 0.0;
  const long long NN = (long long)N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / p;
    const int i = (int)(e - k * p);
    const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
    const ClassSums s = class_sums(X, p, i, N, ix, iy, iz);
    const double kx = c.k0 * s.s0 + c.ke * s.se + c.kc * s.sc;   // face coefficient is 0
    EX[e] = occ * kx + 2.0 * occ * h3 * veff[k] * s.s0;
    if (MX) MX[e] = c.m0 * s.s0 + c.mf * s.sf + c.me * s.se + c.mc * s.sc;
    kin = fma(s.s0, kx, kin);
  }
  const double sb = block_sum(kin, smem);
  if (threadIdx.x == 0) part[blockIdx.x] = sb;
}

// Mode 0: MX = M X only.  Mode 1: MD = M D and sum D.MD.  Mode 2: as 1 plus
// the three BB traces against the previous iterate.
template <int Mode>
__global__ void mass_kernel(int N, int p, long long total, StencilCoef c,
                            const double *__restrict__ D, double *__restrict__ MD,
                            const double *__restrict__ X, const double *__restrict__ MX,
                            const double *__restrict__ Xp, const double *__restrict__ MXp,
                            const double *__restrict__ Dp, const double *__restrict__ MDp,
                            double *__restrict__ part) {
  __shared__ double smem[33];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const long long NN = (long long)N * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / p;
    const int i = (int)(e - k * p);
    const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
    const ClassSums s = class_sums(D, p, i, N, ix, iy, iz);
    const double md = c.m0 * s.s0 + c.mf * s.sf + c.me * s.se + c.mc * s.sc;
    MD[e] = md;
    if (Mode >= 1) a0 = fma(s.s0, md, a0);
    if (Mode == 2) {
      const double dx = X[e] - Xp[e];
      const double dmx = MX[e] - MXp[e];
      const double dd = s.s0 - Dp[e];
      const double dmd = md - MDp[e];
      a1 = fma(dx, dmx, a1);
      a2 = fma(dx, dmd, a2);
      a3 = fma(dd, dmd, a3);
    }
  }
  if (Mode >= 1) {
    const int nb = gridDim.x;
    const double s0 = block_sum(a0, smem);
    if (threadIdx.x == 0) part[blockIdx.x] = s0;
    if (Mode == 2) {
      const double s1 = block_sum(a1, smem);
      const double s2 = block_sum(a2, smem);
      const double s3 = block_sum(a3, smem);
      if (threadIdx.x == 0) {
        part[nb + blockIdx.x] = s1;
        part[2 * nb + blockIdx.x] = s2;
        part[3 * nb + blockIdx.x] = s3;
      }
    }
  }
}

ks_status launch_hamiltonian(Problem &P, const double *X, const double *veff, double *EX,
                             double *MX, double *ekin_out) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  const double h3 = P.h * P.h * P.h;
  {
    ProfScope ps_(P.stream, KP_HAMILTONIAN);
    hamiltonian_kernel<<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, q1_coefficients(P.h), P.occ,
                                                      h3, X, veff, EX, MX, P.partials);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return launch_reduce(P, P.partials, 1, nb, ekin_out, 0.5 * P.occ);
}

ks_status launch_mass(Problem &P, const double *X, double *MX) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  {
    ProfScope ps_(P.stream, KP_MASS);
    mass_kernel<0><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, q1_coefficients(P.h), X, MX,
                                                  nullptr, nullptr, nullptr, nullptr, nullptr,
                                                  nullptr, nullptr);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_mass_dots(Problem &P, const double *D, double *MD, const double *X,
                           const double *MX, const BBPrev *prev, double *out4) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  const StencilCoef c = q1_coefficients(P.h);
  if (prev) {
    {
      ProfScope ps_(P.stream, KP_MASS);
      mass_kernel<2><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, c, D, MD, X, MX, prev->X,
                                                    prev->MX, prev->D, prev->MD, P.partials);
    }
    KS_CUDA_TRY(cudaGetLastError());
    return launch_reduce(P, P.partials, 4, nb, out4);
  }
  {
    ProfScope ps_(P.stream, KP_MASS);
    mass_kernel<1><<<nb, kThreads, 0, P.stream>>>(P.N, P.p, total, c, D, MD, nullptr, nullptr,
                                                  nullptr, nullptr, nullptr, nullptr, P.partials);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return launch_reduce(P, P.partials, 1, nb, out4);
}

}  // namespace ks
