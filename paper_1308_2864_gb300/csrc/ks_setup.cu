// One-time tabulation for a problem: external potential on the nodes, the
// ion-ion energy and the pivots of the 1-D mass solve.
#include "ks_device.cuh"

namespace ks {

// Vext(r_k) = sum_a -Z_a erf(|r_k - R_a| / rc) / |r_k - R_a|, with the
// small-r series -Z_a (2/(sqrt(pi) rc)) (1 - r^2/(3 rc^2)) below 1e-6 bohr
// (the local pseudo-atom of Eq. EKS's E_ext).
__global__ void vext_kernel(int N, double h, const double *__restrict__ atoms, int natoms,
                            double rc, double *__restrict__ vext) {
  const long long n = (long long)N * N * N;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / ((long long)N * N));
  const double x = (ix + 1) * h, y = (iy + 1) * h, z = (iz + 1) * h;
  const double c0 = 2.0 / (sqrt(M_PI) * rc);
  double v = 0.0;
  for (int a = 0; a < natoms; ++a) {
    const double dx = x - atoms[4 * a + 0], dy = y - atoms[4 * a + 1], dz = z - atoms[4 * a + 2];
    const double Za = atoms[4 * a + 3];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r < 1e-6)
      v += -Za * c0 * (1.0 - r * r / (3.0 * rc * rc));
    else
      v += -Za * erf(r / rc) / r;
  }
  vext[k] = v;
}

// E_II = 1/2 sum_{i != j} Z_i Z_j / |R_i - R_j| (Eq. EKS), one block,
// pairs summed in a fixed order.
__global__ void eii_kernel(const double *__restrict__ atoms, int natoms, double *out) {
  __shared__ double smem[33];
  double acc = 0.0;
  const long long npairs = (long long)natoms * natoms;
  for (long long t = threadIdx.x; t < npairs; t += blockDim.x) {
    const int i = (int)(t / natoms), j = (int)(t % natoms);
    if (i == j) continue;
    const double dx = atoms[4 * i] - atoms[4 * j], dy = atoms[4 * i + 1] - atoms[4 * j + 1],
                 dz = atoms[4 * i + 2] - atoms[4 * j + 2];
    acc += 0.5 * atoms[4 * i + 3] * atoms[4 * j + 3] / sqrt(dx * dx + dy * dy + dz * dz);
  }
  const double s = block_sum(acc, smem);
  if (threadIdx.x == 0) *out = s;
}

// Pivots of the Thomas elimination for tridiag(1, 4, 1) of order N:
// w_0 = 1/4, w_j = 1/(4 - w_{j-1}).  (M1 = (h/6) tridiag(1, 4, 1).)
__global__ void thomas_pivots_kernel(int N, double *w) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double c = 0.0;
  for (int j = 0; j < N; ++j) {
    c = 1.0 / (4.0 - c);
    w[j] = c;
  }
}

ks_status launch_setup(Problem &P) {
  const int nb = (P.n + kThreads - 1) / kThreads;
  {
    ProfScope ps_(P.stream, KP_SETUP);
    vext_kernel<<<nb, kThreads, 0, P.stream>>>(P.N, P.h, P.atoms_dev, P.natoms, P.rc, P.vext);
  }
  KS_CUDA_TRY(cudaGetLastError());
  {
    ProfScope ps_(P.stream, KP_SETUP);
    eii_kernel<<<1, kThreads, 0, P.stream>>>(P.atoms_dev, P.natoms, P.scal + SC_EII);
  }
  KS_CUDA_TRY(cudaGetLastError());
  {
    ProfScope ps_(P.stream, KP_SETUP);
    thomas_pivots_kernel<<<1, 32, 0, P.stream>>>(P.N, P.thomas_w);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

}  // namespace ks
