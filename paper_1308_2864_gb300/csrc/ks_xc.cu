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

// rho^(-1/3) for rho >= 1e-30: single-precision start, then two Newton steps
// on f(z) = z^-3 - rho, z <- z (4 - rho z^3) / 3 (no division; each step
// squares the relative error, 1e-7 -> 1e-14 -> below FP64 rounding).  On
// GB300 every FP64 instruction is a 16-cycle issue, so this replaces two
// library cube roots and three divisions per point.
__device__ __forceinline__ double inv_cbrt(double rho) {
  double z = (double)rcbrtf((float)rho);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double z3 = z * z * z;
    z = z * fma(-rho, z3, 4.0) * (1.0 / 3.0);
  }
  return z;
}

// eps_xc and v_xc = d(rho eps_xc)/d rho at one point, in precision R
// (FP64; FP32 for the mixed-precision phase, whose orbitals carry FP32
// rounding already; the energy sums stay FP64 in both).
//   Slater: eps_x = -(3/4) (3/pi)^(1/3) rho^(1/3), v_x = (4/3) eps_x;
//   PZ81 (r_s = (3 / (4 pi rho))^(1/3)): eps_c = gamma / (1 + beta1 sqrt(r_s)
//   + beta2 r_s) for r_s >= 1, A ln r_s + B + C r_s ln r_s + D r_s below;
//   v_c = eps_c - (r_s / 3) d eps_c / d r_s.
template <typename R>
__device__ __forceinline__ void lda_point(double rho_d, int xc, R &eps, R &v) {
  if (!(rho_d >= 1e-30)) {
    eps = 0;
    v = 0;
    return;
  }
  const R c = (R)0.98474502184269654;              // (3/pi)^(1/3)
  const R crs = (R)0.62035049089940001;            // (3/(4 pi))^(1/3)
  const R rho = (R)rho_d;
  R z;                                             // rho^(-1/3)
  if constexpr (sizeof(R) == 8) z = inv_cbrt(rho_d);
  else z = rcbrtf(rho);
  const R r13 = rho * z * z;                       // rho^(1/3)
  eps = (R)-0.75 * c * r13;
  v = -c * r13;
  if (xc == KS_XC_SLATER_PZ81) {
    const R rs = crs * z;
    R ec, dec;
    if (rs >= (R)1) {
      R irs;                                       // 1 / sqrt(r_s)
      if constexpr (sizeof(R) == 8) irs = rsqrt(rs);
      else irs = rsqrtf(rs);
      const R srs = rs * irs;
      const R iden = (R)1 / ((R)1 + (R)kPzBeta1 * srs + (R)kPzBeta2 * rs);
      ec = (R)kPzGamma * iden;
      dec = -(R)kPzGamma * ((R)(0.5 * kPzBeta1) * irs + (R)kPzBeta2) * (iden * iden);
    } else {
      R lrs;
      if constexpr (sizeof(R) == 8) lrs = log(rs);
      else lrs = logf(rs);
      ec = (R)kPzA * lrs + (R)kPzB + (R)kPzC * rs * lrs + (R)kPzD * rs;
      // A / r_s = A rho^(1/3) / crs
      dec = (R)kPzA * (r13 * (R)(1.0 / 0.62035049089940001)) + (R)kPzC * (lrs + (R)1) + (R)kPzD;
    }
    eps += ec;
    v += ec - (rs / (R)3) * dec;
  }
}

// Thomas-Fermi kinetic energy per unit volume C_TF rho^(5/3) and its
// derivative v_TF = (5/3) C_TF rho^(2/3) (the T_TF term of Eq. TFW), both 0
// below the density floor; ctf = C_TF and vtf = (5/3) C_TF in precision R.
template <typename R>
__device__ __forceinline__ void tf_point(double rho_d, R ctf, R vtf, R &e, R &v) {
  if (!(rho_d >= 1e-30)) {
    e = 0;
    v = 0;
    return;
  }
  const R rho = (R)rho_d;
  R z;                                             // rho^(-1/3)
  if constexpr (sizeof(R) == 8) z = inv_cbrt(rho_d);
  else z = rcbrtf(rho);
  const R r23 = rho * z;                           // rho^(2/3)
  v = vtf * r23;
  e = ctf * rho * r23;
}

// Channels of the block partials: 0 = E_ext, 1 = E_H, 2 = E_xc and, when
// ctf != 0 (orbital-free model), 3 = E_TF, with v_TF added to V_eff.  Block
// vb of vnb (grid-stride over the n nodes); the last block to finish sums
// the partials in block order.
template <typename R>
__device__ __forceinline__ void potential_body(long long n, double h3, int xc, int with_h,
                                               double ctf,
                                               const double *__restrict__ rho,
                                               const double *__restrict__ vext,
                                               const double *__restrict__ vH,
                                               const double *__restrict__ r,
                                               double *__restrict__ veff, double *__restrict__ part,
                                               double *__restrict__ out, unsigned int *counter,
                                               int vb, int vnb) {
  __shared__ double smem[33];
  const double inv8pi = 1.0 / (8.0 * M_PI);
  const R ctf_r = (R)ctf, vtf_r = (R)(ctf * (5.0 / 3.0));
  double e_ext = 0.0, e_h = 0.0, e_xc = 0.0, e_tf = 0.0;
  for (long long k = (long long)vb * blockDim.x + threadIdx.x; k < n;
       k += (long long)vnb * blockDim.x) {
    const double rk = rho[k], ve = vext[k];
    R eps_r, vxc_r;
    lda_point<R>(rk, xc, eps_r, vxc_r);
    const double eps = (double)eps_r;
    double v = ve + (double)vxc_r;
    e_ext = fma(h3 * ve, rk, e_ext);
    e_xc = fma(h3 * rk, eps, e_xc);
    if (with_h) {
      const double vh = vH[k];
      v += vh;
      e_h += 0.5 * h3 * vh * rk + vh * r[k] * inv8pi;
    }
    if (ctf != 0.0) {
      R etf_r, vtf_p;
      tf_point<R>(rk, ctf_r, vtf_r, etf_r, vtf_p);
      v += (double)vtf_p;
      e_tf = fma(h3, (double)etf_r, e_tf);
    }
    veff[k] = v;
  }
  const double s0 = block_sum(e_ext, smem);
  const double s1 = block_sum(e_h, smem);
  const double s2 = block_sum(e_xc, smem);
  const int nchan = ctf != 0.0 ? 4 : 3;
  const double s3 = nchan == 4 ? block_sum(e_tf, smem) : 0.0;
  if (threadIdx.x == 0) {
    part[vb] = s0;
    part[vnb + vb] = s1;
    part[2 * vnb + vb] = s2;
    if (nchan == 4) part[3 * vnb + vb] = s3;
  }
  grid_reduce_tail(part, vnb, nchan, out, 1.0, counter, smem);
}

template <typename R>
__global__ void potential_kernel(long long n, double h3, int xc, int with_h, double ctf,
                                 const double *__restrict__ rho, const double *__restrict__ vext,
                                 const double *__restrict__ vH, const double *__restrict__ r,
                                 double *__restrict__ veff, double *__restrict__ part,
                                 double *__restrict__ out, unsigned int *counter) {
  potential_body<R>(n, h3, xc, with_h, ctf, rho, vext, vH, r, veff, part, out, counter,
                    blockIdx.x, gridDim.x);
}

// Batched: job j takes pot_nb blocks.
template <typename R>
__global__ void potential_batch_kernel(const BJob *__restrict__ jobs, const int *__restrict__ start,
                                       int J, const unsigned char *__restrict__ active) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  potential_body<R>(b.n, b.h3, b.xc, 1, 0.0, b.rho, b.vext, b.vH, b.cg_r, b.veff, b.partials,
                    b.scal + SC_EEXT, b.red_counter, blockIdx.x - start[j], b.pot_nb);
}

ks_status batch_potential(Batch &B, bool fp32_xc) {
  const int nb = B.total(BM_POTENTIAL);
  if (nb == 0) return KS_OK;
  {
    ProfScope ps_(B.stream, KP_POTENTIAL);
    if (fp32_xc)
      potential_batch_kernel<float><<<nb, kThreads, 0, B.stream>>>(B.jobs_dev, B.map(BM_POTENTIAL),
                                                                   B.J, B.active_dev);
    else
      potential_batch_kernel<double><<<nb, kThreads, 0, B.stream>>>(
          B.jobs_dev, B.map(BM_POTENTIAL), B.J, B.active_dev);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
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
                           double *veff, bool with_hartree, bool fp32_xc) {
  const int nb = reduce_blocks(P, P.n);
  const double h3 = P.h * P.h * P.h;
  {
    ProfScope ps_(P.stream, KP_POTENTIAL, 40.0 * P.n, 40.0 * P.n);
    if (fp32_xc)
      potential_kernel<float><<<nb, kThreads, 0, P.stream>>>(
          P.n, h3, P.xc, with_hartree ? 1 : 0, P.ctf, rho, P.vext, vH, r, veff, P.partials,
          P.scal + SC_EEXT, P.red_counter);
    else
      potential_kernel<double><<<nb, kThreads, 0, P.stream>>>(
          P.n, h3, P.xc, with_hartree ? 1 : 0, P.ctf, rho, P.vext, vH, r, veff, P.partials,
          P.scal + SC_EEXT, P.red_counter);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

}  // namespace ks
