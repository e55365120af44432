// Hartree potential: conjugate gradients for K vH = 4 pi h^3 rho with zero
// Dirichlet values (the discrete L^+ rho of Sec. 2.3 for the Q1 stiffness),
// as one persistent cooperative kernel.
//
// Each iteration needs two grid-wide reductions (p.q and r.r).  The search
// direction update p_j = r_j + beta p_{j-1} is folded into the stencil of the
// next iteration (p is double-buffered and recomputed on the fly for the
// neighbours), so one iteration costs exactly two grid barriers.  Partial
// sums are written per block and summed by every block in the same order,
// so all blocks take identical branch decisions and the result is
// deterministic.
#include "ks_device.cuh"

namespace ks {

struct CgArgs {
  int N;
  long long n;
  StencilCoef c;
  double bscale;              // 4 pi h^3
  const double *rho;
  double *x, *r, *pa, *pb, *q;
  double *part;               // 3 * gridDim.x
  GridBarrier *bar;
  int *status;
  double *iters_out;
  double tol;
  int maxit;
  int warm;
};

// (K v)_k for v = a + beta * b (b ignored when UseB is false), Dirichlet.
// The Q1 stiffness has zero face coefficients, so only the centre, the 12
// edge and the 8 corner neighbours contribute.
template <bool UseB>
__device__ __forceinline__ double stiff_apply(const double *a, const double *b, double beta,
                                              int N, int ix, int iy, int iz,
                                              const StencilCoef &c, double *centre) {
  double se = 0.0, sc = 0.0, s0 = 0.0;
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
        if (nzc == 1) continue;
        const long long kk = z * NN + (long long)y * N + x;
        double v = ldcg(a + kk);
        if (UseB) v = fma(beta, ldcg(b + kk), v);
        if (nzc == 0) s0 = v;
        else if (nzc == 2) se += v;
        else sc += v;
      }
    }
  }
  *centre = s0;
  return c.k0 * s0 + c.ke * se + c.kc * sc;
}

__global__ void __launch_bounds__(kCgThreads) cg_kernel(CgArgs a) {
  __shared__ double smem[33];
  const int nb = gridDim.x;
  double *partA = a.part, *partB = a.part + nb, *partC = a.part + 2 * nb;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int N = a.N;
  const long long NN = (long long)N * N;

  // r = b - K x0 (x0 = 0 for a cold start)
  double rr_l = 0.0, bb_l = 0.0;
  for (long long k = tid; k < a.n; k += stride) {
    const double b = a.bscale * a.rho[k];
    double kx = 0.0, dummy;
    if (a.warm) {
      const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
      kx = stiff_apply<false>(a.x, nullptr, 0.0, N, ix, iy, iz, a.c, &dummy);
    }
    const double rk = b - kx;
    a.r[k] = rk;
    rr_l = fma(rk, rk, rr_l);
    bb_l = fma(b, b, bb_l);
  }
  {
    const double s1 = block_sum(rr_l, smem);
    const double s2 = block_sum(bb_l, smem);
    if (threadIdx.x == 0) { partB[blockIdx.x] = s1; partC[blockIdx.x] = s2; }
  }
  if (!grid_barrier(a.bar, a.status)) return;
  if (!a.warm) {
    for (long long k = tid; k < a.n; k += stride) a.x[k] = 0.0;
  }
  double rr = block_sum_array(partB, nb, smem);
  const double bb = block_sum_array(partC, nb, smem);
  const double thr = a.tol * a.tol * bb;

  int it = 0;
  double beta = 0.0;
  double *pold = a.pa, *pnew = a.pb;
  bool bad = false;
  while (rr > thr && it < a.maxit) {
    // phase 1: p = r + beta p_old (own nodes), q = K p, p.q
    double pq_l = 0.0;
    for (long long k = tid; k < a.n; k += stride) {
      const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
      double pk;
      const double qk = (it == 0)
          ? stiff_apply<false>(a.r, nullptr, 0.0, N, ix, iy, iz, a.c, &pk)
          : stiff_apply<true>(a.r, pold, beta, N, ix, iy, iz, a.c, &pk);
      pnew[k] = pk;
      a.q[k] = qk;
      pq_l = fma(pk, qk, pq_l);
    }
    {
      const double s = block_sum(pq_l, smem);
      if (threadIdx.x == 0) partA[blockIdx.x] = s;
    }
    if (!grid_barrier(a.bar, a.status)) return;
    const double pq = block_sum_array(partA, nb, smem);
    if (!(pq > 0.0) || !isfinite(pq)) { bad = true; break; }
    const double alpha = rr / pq;
    // phase 2: x += alpha p, r -= alpha q, r.r
    double rl = 0.0;
    for (long long k = tid; k < a.n; k += stride) {
      a.x[k] = fma(alpha, pnew[k], a.x[k]);
      const double rk = fma(-alpha, a.q[k], a.r[k]);
      a.r[k] = rk;
      rl = fma(rk, rk, rl);
    }
    {
      const double s = block_sum(rl, smem);
      if (threadIdx.x == 0) partB[blockIdx.x] = s;
    }
    if (!grid_barrier(a.bar, a.status)) return;
    const double rr_new = block_sum_array(partB, nb, smem);
    if (!isfinite(rr_new)) { bad = true; break; }
    beta = rr_new / rr;
    rr = rr_new;
    double *t = pold; pold = pnew; pnew = t;
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.iters_out = (double)it;
    if (bad) atomicCAS(a.status, 0, (int)KS_ENAN);
    else if (rr > thr) atomicCAS(a.status, 0, (int)KS_ENOCONV);
  }
}

ks_status launch_cg(Problem &P, const double *rho, double *v, double *r, bool warm) {
  CgArgs a;
  a.N = P.N;
  a.n = P.n;
  a.c = q1_coefficients(P.h);
  a.bscale = 4.0 * M_PI * P.h * P.h * P.h;
  a.rho = rho;
  a.x = v;
  a.r = r;
  a.pa = P.cg_pa;
  a.pb = P.cg_pb;
  a.q = P.cg_q;
  a.part = P.partials;
  a.bar = P.bar;
  a.status = P.dstatus;
  a.iters_out = P.scal + SC_CG_ITERS;
  a.tol = P.cg_tol;
  a.maxit = P.cg_maxit;
  a.warm = warm ? 1 : 0;
  KS_CUDA_TRY(cudaMemsetAsync(P.bar, 0, sizeof(GridBarrier), P.stream));
  void *args[] = {&a};
  {
    ProfScope ps_(P.stream, KP_CG);
    KS_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)cg_kernel, dim3(P.cg_blocks),
                                            dim3(kCgThreads), args, 0, P.stream));
  }
  return KS_OK;
}

int cg_grid_blocks(int sms, int n) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel, kCgThreads, 0) !=
      cudaSuccess || per_sm < 1)
    per_sm = 1;
  long long want = (n + kCgThreads - 1) / kCgThreads;
  long long cap = (long long)sms * (per_sm < 2 ? per_sm : 2);
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace ks
