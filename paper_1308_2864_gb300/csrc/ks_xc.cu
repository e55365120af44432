// Effective potential and the density-dependent energy terms (Sec. 2.1 /
// Sec. 2.3): E_ext = h^3 sum Vext rho, E_H (variational form), E_xc =
// h^3 sum rho eps_xc(rho), and V_eff = Vext + vH + v_xc with
// v_xc = d(rho eps_xc)/d rho.  LDA = Slater exchange, optionally with the
// Perdew-Zunger (1981) correlation of the unpolarised electron gas.
#include "ks_device.cuh"

namespace ks {

// Perdew-Zunger parameters (hartree): gamma, beta1, beta2, A, B as
// published; C and D from continuity of eps_c and d eps_c / d r_s at r_s = 1
// (the published 0.0020 and -0.0116 are these rounded; rounded, they leave a
// 3.2e-5 Ha jump that makes the energy discontinuous).
constexpr double kPzGamma = -0.1423, kPzBeta1 = 1.0529, kPzBeta2 = 0.3334;
constexpr double kPzA = 0.0311, kPzB = -0.048;
constexpr double kPzDen1 = 1.0 + kPzBeta1 + kPzBeta2;
constexpr double kPzD = kPzGamma / kPzDen1 - kPzB;
constexpr double kPzC = -kPzGamma * (0.5 * kPzBeta1 + kPzBeta2) / (kPzDen1 * kPzDen1) - kPzA - kPzD;

__device__ __forceinline__ void lda_point(double rho, int xc, double &eps, double &v) {
  if (!(rho >= 1e-30)) {
    eps = 0.0;
    v = 0.0;
    return;
  }
  const double c = cbrt(3.0 / M_PI);
  const double r13 = cbrt(rho);
  eps = -0.75 * c * r13;
  v = -c * r13;
  if (xc == KS_XC_SLATER_PZ81) {
    const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
    double ec, dec;
    if (rs >= 1.0) {
      const double srs = sqrt(rs);
      const double den = 1.0 + kPzBeta1 * srs + kPzBeta2 * rs;
      ec = kPzGamma / den;
      dec = -kPzGamma * (0.5 * kPzBeta1 / srs + kPzBeta2) / (den * den);
    } else {
      const double lrs = log(rs);
      ec = kPzA * lrs + kPzB + kPzC * rs * lrs + kPzD * rs;
      dec = kPzA / rs + kPzC * (lrs + 1.0) + kPzD;
    }
    eps += ec;
    v += ec - (rs / 3.0) * dec;
  }
}

// Channels of the block partials: 0 = E_ext, 1 = E_H, 2 = E_xc.
__global__ void potential_kernel(long long n, double h3, int xc, int with_h,
                                 const double *__restrict__ rho, const double *__restrict__ vext,
                                 const double *__restrict__ vH, const double *__restrict__ r,
                                 double *__restrict__ veff, double *__restrict__ part,
                                 double *__restrict__ out, unsigned int *counter) {
  __shared__ double smem[33];
  const double inv8pi = 1.0 / (8.0 * M_PI);
  double e_ext = 0.0, e_h = 0.0, e_xc = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double rk = rho[k], ve = vext[k];
    double eps, vxc;
    lda_point(rk, xc, eps, vxc);
    double v = ve + vxc;
    e_ext = fma(h3 * ve, rk, e_ext);
    e_xc = fma(h3 * rk, eps, e_xc);
    if (with_h) {
      const double vh = vH[k];
      v += vh;
      e_h += 0.5 * h3 * vh * rk + vh * r[k] * inv8pi;
    }
    veff[k] = v;
  }
  const int nb = gridDim.x;
  const double s0 = block_sum(e_ext, smem);
  const double s1 = block_sum(e_h, smem);
  const double s2 = block_sum(e_xc, smem);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[nb + blockIdx.x] = s1;
    part[2 * nb + blockIdx.x] = s2;
  }
  grid_reduce_tail(part, nb, 3, out, 1.0, counter, smem);
}

// out[c] = scale * sum_{b < nb} part[c * nb + b], one block per channel, in
// a fixed order.
__global__ void reduce_kernel(const double *__restrict__ part, int nb, double scale,
                              double *__restrict__ out) {
  __shared__ double smem[33];
  const double s = block_sum_array(part + (long long)blockIdx.x * nb, nb, smem);
  if (threadIdx.x == 0) out[blockIdx.x] = scale * s;
}

int reduce_blocks(const Problem &P, long long work) {
  long long nb = (work + kThreads - 1) / kThreads;
  const long long cap = 8LL * P.sms;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  return (int)nb;
}

ks_status launch_reduce(Problem &P, const double *partials, int nchan, int nb, double *out,
                        double scale) {
  {
    ProfScope ps_(P.stream, KP_REDUCE);
    reduce_kernel<<<nchan, kThreads, 0, P.stream>>>(partials, nb, scale, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_potential(Problem &P, const double *rho, const double *vH, const double *r,
                           double *veff, bool with_hartree) {
  const int nb = reduce_blocks(P, P.n);
  const double h3 = P.h * P.h * P.h;
  {
    ProfScope ps_(P.stream, KP_POTENTIAL, 40.0 * P.n, 40.0 * P.n);
    potential_kernel<<<nb, kThreads, 0, P.stream>>>(P.n, h3, P.xc, with_hartree ? 1 : 0, rho,
                                                    P.vext, vH, r, veff, P.partials,
                                                    P.scal + SC_EEXT, P.red_counter);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

}  // namespace ks
