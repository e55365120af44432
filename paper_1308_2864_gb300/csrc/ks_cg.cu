// Hartree potential: conjugate gradients for K vH = 4 pi h^3 rho with zero
// Dirichlet values (the discrete L^+ rho of Sec. 2.3 for the Q1 stiffness),
// as one persistent cooperative kernel.
//
// Preconditioner (optional, on by default): the exact inverse of K applied
// in FP32 through the orthonormal sine basis that diagonalises the 1-D
// factors K1 and M1, K^{-1} = (Phi x Phi x Phi) Lambda^{-1} (Phi x Phi x Phi)
// with Lambda_abc = k_a m_b m_c + m_a k_b m_c + m_a m_b k_c.  Applied in
// single precision it is an SPD approximation of K^{-1} to about 1e-6, so
// the FP64 CG reaches 1e-10 in two or three iterations.  Each sine transform
// is a dense N x N product along one grid axis: fused in shared memory for
// N <= 128 (three grid barriers per application), tiled through shared
// memory above (six axis passes, one grid barrier after each).
//
// Each CG iteration needs two grid-wide reductions (p.q and r.r, plus r.z
// when preconditioned).  The search direction p_j = s_j + beta p_{j-1}
// (s = z or r) is folded into the stencil of the next iteration (p is
// double-buffered and recomputed on the fly for the neighbours).  Partial
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
  double *x, *r, *pa, *pb, *q, *z;
  float *t1, *t2;             // sine-transform work vectors
  const float *phi;           // N x N sine basis
  const float *kap, *mu;      // 1-D eigenvalues of K1 and M1
  double *part;               // 4 * vnb
  GridBarrier *bar;
  int *status;
  double *iters_out;
  double tol;
  int maxit;
  int warm;
  int precond;
  int fused;                  // fused shared-memory preconditioner (N <= kFusedMaxN)
  int vb, vnb;                // this block's index among the vnb blocks that solve this system
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

// Tiled form for N > kFusedMaxN: each axis pass is the product C = Phi X,
// where the columns of X are the grid lines along the axis (element (s, k, c)
// of slab s, axis index k and column c at s*ss + k*sa + c*sc).  A work item
// is a tile of kTJ frequencies x kTC columns; the K dimension is staged in
// chunks of kTK axis points (X chunk and Phi chunk in shared memory), and a
// thread keeps a 4 x 8 block of outputs (rows tj + 16 a, columns tc + 16 b)
// whose FMA chains run over k in ascending order.  Phi is symmetric and
// orthogonal, so the same matrix serves the forward and the inverse passes.
// Mode 1 (after the forward z pass) divides by Lambda of the frequency
// triple; Mode 2 (the last inverse pass) writes FP64 z and accumulates r.z.
constexpr int kTJ = 64, kTC = 128, kTK = 32, kTCPad = kTC + 1;
static_assert(kCgThreads == 256, "the 16 x 16 thread grid of the tiled sine pass");

template <typename Tin, int Mode>
__device__ double tiled_pass(const CgArgs &a, const Tin *in, float *out32, double *out64, int axis,
                             float *sh) {
  const int N = a.N;
  const long long NN = (long long)N * N;
  long long sa, sc, ss, C;
  int S;
  if (axis == 0) { sa = 1; sc = N; ss = 0; S = 1; C = NN; }
  else if (axis == 1) { sa = N; sc = 1; ss = NN; S = N; C = N; }
  else { sa = NN; sc = 1; ss = 0; S = 1; C = NN; }
  const long long ctiles = (C + kTC - 1) / kTC;
  const int jblocks = (N + kTJ - 1) / kTJ;
  const long long total = (long long)S * ctiles * jblocks;
  float *Xs = sh, *Ps = sh + kTK * kTCPad;
  const int tid = threadIdx.x, tj = tid >> 4, tc = tid & 15;
  double rz = 0.0;
  for (long long w = a.vb; w < total; w += a.vnb) {
    const int jb = (int)(w % jblocks) * kTJ;
    const long long w2 = w / jblocks;
    const long long c0 = (w2 % ctiles) * kTC;
    const long long base = (w2 / ctiles) * ss;
    float acc[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
    for (int k0 = 0; k0 < N; k0 += kTK) {
      __syncthreads();
      // X chunk (kTK x kTC): consecutive threads take consecutive addresses
      // (along the axis for the x pass, along the columns otherwise)
      for (int t = tid; t < kTK * kTC; t += kCgThreads) {
        const int kk = axis == 0 ? t % kTK : t / kTC;
        const int cc = axis == 0 ? t / kTK : t % kTC;
        const int k = k0 + kk;
        const long long c = c0 + cc;
        float v = 0.f;
        if (k < N && c < C) {
          const long long idx = base + k * sa + c * sc;
          if constexpr (sizeof(Tin) == 8) v = (float)__ldcg((const double *)in + idx);
          else v = __ldcg((const float *)in + idx);
        }
        Xs[kk * kTCPad + cc] = v;
      }
      // Phi chunk (kTK x kTJ): Ps[kk][jj] = Phi[k0 + kk][jb + jj]
      for (int t = tid; t < kTK * kTJ; t += kCgThreads) {
        const int jj = t % kTJ, kk = t / kTJ;
        const int k = k0 + kk, j = jb + jj;
        Ps[t] = (k < N && j < N) ? __ldg(a.phi + (long long)k * N + j) : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kTK; ++kk) {
        float pv[4], xv[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) pv[u] = Ps[kk * kTJ + tj + 16 * u];
#pragma unroll
        for (int v = 0; v < 8; ++v) xv[v] = Xs[kk * kTCPad + tc + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(pv[u], xv[v], acc[u][v]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jb + tj + 16 * u;
      if (j >= N) continue;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const long long c = c0 + tc + 16 * v;
        if (c >= C) continue;
        const long long idx = base + j * sa + c * sc;
        float val = acc[u][v];
        if (Mode == 1) {
          const int ix = (int)(idx % N), iy = (int)((idx / N) % N), iz = (int)(idx / NN);
          const float lam = a.kap[ix] * a.mu[iy] * a.mu[iz] + a.mu[ix] * a.kap[iy] * a.mu[iz] +
                            a.mu[ix] * a.mu[iy] * a.kap[iz];
          val = val / lam;
        }
        if (Mode == 2) {
          const double zv = (double)val;
          out64[idx] = zv;
          rz = fma(a.r[idx], zv, rz);
        } else {
          out32[idx] = val;
        }
      }
    }
  }
  return rz;
}

constexpr size_t kTiledSmem = (size_t)(kTK * kTCPad + kTK * kTJ) * sizeof(float);

// z = P^{-1} r (six tiled passes, each followed by a grid barrier); returns
// this thread's share of r.z, or false when a barrier failed.
__device__ bool apply_precond(const CgArgs &a, double *rz_l) {
  extern __shared__ float dyn[];
  tiled_pass<double, 0>(a, a.r, a.t1, nullptr, 0, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  tiled_pass<float, 0>(a, a.t1, a.t2, nullptr, 1, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  tiled_pass<float, 1>(a, a.t2, a.t1, nullptr, 2, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  tiled_pass<float, 0>(a, a.t1, a.t2, nullptr, 2, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  tiled_pass<float, 0>(a, a.t2, a.t1, nullptr, 1, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  *rz_l = tiled_pass<float, 2>(a, a.t1, nullptr, a.z, 0, dyn);
  return true;
}

// Fused form for N <= kFusedMaxN, with the planes in shared memory (3 N^2
// floats of dynamic shared memory: a plane, Phi and a work matrix):
//   A: each z-plane P (N x N, rows y, columns x) -> Phi P Phi   (x and y)
//   B: each y-slab S (rows z, columns x)          -> Phi (Lambda^{-1} o (Phi S))
//   C: each z-plane                               -> Phi P Phi, written as z
// (Phi is symmetric, so Phi P Phi transforms both in-plane axes), three grid
// barriers per application instead of six.
constexpr int kFusedMaxN = 128;

// out = A B for N x N row-major matrices in shared memory (kCgThreads
// threads, W = kCgThreads / 32 warps).  Each thread keeps a (64/W) x 2
// block of outputs in registers (rows ty + W a, columns tx + 32 b of a 64 x 64
// tile), so a k step costs 64/W broadcast loads of A and 2 conflict-free
// loads of B for 128/W FMAs.  Every output is the same k-ascending FMA chain
// as the one-output-per-thread form.
constexpr int kCgWarps = kCgThreads / 32;
constexpr int kRowsPerThread = 64 / kCgWarps;
static_assert(64 % kCgWarps == 0, "warps must divide the 64-row tile");

__device__ __forceinline__ void smem_matmul(const float *A, const float *B, float *out, int N) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int ib = 0; ib < N; ib += 64)
    for (int jb = 0; jb < N; jb += 64) {
      float acc[kRowsPerThread][2];
#pragma unroll
      for (int a = 0; a < kRowsPerThread; ++a) acc[a][0] = acc[a][1] = 0.f;
      const int j0 = jb + tx, j1 = jb + tx + 32;
      for (int k = 0; k < N; ++k) {
        const float b0 = j0 < N ? B[k * N + j0] : 0.f;
        const float b1 = j1 < N ? B[k * N + j1] : 0.f;
#pragma unroll
        for (int a = 0; a < kRowsPerThread; ++a) {
          const int i = ib + ty + kCgWarps * a;
          const float av = i < N ? A[i * N + k] : 0.f;
          acc[a][0] = fmaf(av, b0, acc[a][0]);
          acc[a][1] = fmaf(av, b1, acc[a][1]);
        }
      }
#pragma unroll
      for (int a = 0; a < kRowsPerThread; ++a) {
        const int i = ib + ty + kCgWarps * a;
        if (i >= N) continue;
        if (j0 < N) out[i * N + j0] = acc[a][0];
        if (j1 < N) out[i * N + j1] = acc[a][1];
      }
    }
}

// Phi P Phi for the plane z of `in` (FP64 r or FP32 work), into out32 or,
// for the last step, out64 with the r.z accumulation.
template <bool InD, bool OutD>
__device__ double fused_plane_pass(const CgArgs &a, const void *in, float *out32, double *out64,
                                   float *sh) {
  const int N = a.N;
  const long long NN = (long long)N * N;
  float *Pm = sh, *Ph = sh + NN, *W = sh + 2 * NN;
  double rz = 0.0;
  for (int z = a.vb; z < N; z += a.vnb) {
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
      Pm[e] = InD ? (float)__ldcg((const double *)in + z * NN + e)
                  : __ldcg((const float *)in + z * NN + e);
    }
    __syncthreads();
    smem_matmul(Pm, Ph, W, N);      // x: P Phi
    __syncthreads();
    smem_matmul(Ph, W, Pm, N);      // y: Phi (P Phi)
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
      if (OutD) {
        const double zv = (double)Pm[e];
        out64[z * NN + e] = zv;
        rz = fma(a.r[z * NN + e], zv, rz);
      } else {
        out32[z * NN + e] = Pm[e];
      }
    }
  }
  return rz;
}

// For each y: S[z][x] -> Phi (Lambda^{-1} o (Phi S)) along z.
__device__ void fused_slab_pass(const CgArgs &a, const float *in, float *out, float *sh) {
  const int N = a.N;
  const long long NN = (long long)N * N;
  float *Sm = sh, *Ph = sh + NN, *W = sh + 2 * NN;
  for (int y = a.vb; y < N; y += a.vnb) {
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
      const int zz = e / N, x = e % N;
      Sm[e] = __ldcg(in + (long long)zz * NN + (long long)y * N + x);
    }
    __syncthreads();
    smem_matmul(Ph, Sm, W, N);      // forward along z
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
      const int c = e / N, x = e % N;
      const float lam = a.kap[x] * a.mu[y] * a.mu[c] + a.mu[x] * a.kap[y] * a.mu[c] +
                        a.mu[x] * a.mu[y] * a.kap[c];
      W[e] = W[e] / lam;
    }
    __syncthreads();
    smem_matmul(Ph, W, Sm, N);      // inverse along z
    __syncthreads();
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
      const int zz = e / N, x = e % N;
      out[(long long)zz * NN + (long long)y * N + x] = Sm[e];
    }
  }
}

__device__ bool apply_precond_fused(const CgArgs &a, double *rz_l) {
  extern __shared__ float dyn[];
  const int N = a.N;
  const int NN = N * N;
  // Phi into shared memory once per application
  for (int e = threadIdx.x; e < NN; e += blockDim.x) dyn[NN + e] = __ldg(a.phi + e);
  fused_plane_pass<true, false>(a, a.r, a.t1, nullptr, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  fused_slab_pass(a, a.t1, a.t2, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  *rz_l = fused_plane_pass<false, true>(a, a.t2, nullptr, a.z, dyn);
  return true;
}

// The whole PCG of one system on the blocks a.vb = 0 .. a.vnb - 1 (which must
// be co-resident: a cooperative launch).
__device__ void cg_body(const CgArgs &a) {
  __shared__ double smem[33];
  const int nb = a.vnb;
  double *partA = a.part, *partB = a.part + nb, *partC = a.part + 2 * nb, *partD = a.part + 3 * nb;
  const long long tid = (long long)a.vb * blockDim.x + threadIdx.x;
  const long long stride = (long long)a.vnb * blockDim.x;
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
    if (threadIdx.x == 0) { partB[a.vb] = s1; partD[a.vb] = s2; }
  }
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return;
  if (!a.warm) {
    for (long long k = tid; k < a.n; k += stride) a.x[k] = 0.0;
  }
  double rr = block_sum_array(partB, nb, smem);
  const double bb = block_sum_array(partD, nb, smem);
  const double thr = a.tol * a.tol * bb;
  double rho_cg = rr;                       // r.z (preconditioned) or r.r
  const double *s_vec = a.precond ? a.z : a.r;
  if (a.precond && rr > thr) {
    double rz_l = 0.0;
    if (a.fused ? !apply_precond_fused(a, &rz_l) : !apply_precond(a, &rz_l)) return;
    const double s = block_sum(rz_l, smem);
    if (threadIdx.x == 0) partC[a.vb] = s;
    if (!grid_barrier_n(a.bar, a.status, a.vnb)) return;
    rho_cg = block_sum_array(partC, nb, smem);
  }

  int it = 0;
  double beta = 0.0;
  double *pold = a.pa, *pnew = a.pb;
  // a non-finite right-hand side or start makes every comparison below false
  bool bad = !isfinite(rr) || !isfinite(bb);
  while (rr > thr && it < a.maxit) {
    // phase 1: p = s + beta p_old (own nodes), q = K p, p.q
    double pq_l = 0.0;
    for (long long k = tid; k < a.n; k += stride) {
      const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
      double pk;
      const double qk = (it == 0)
          ? stiff_apply<false>(s_vec, nullptr, 0.0, N, ix, iy, iz, a.c, &pk)
          : stiff_apply<true>(s_vec, pold, beta, N, ix, iy, iz, a.c, &pk);
      pnew[k] = pk;
      a.q[k] = qk;
      pq_l = fma(pk, qk, pq_l);
    }
    {
      const double s = block_sum(pq_l, smem);
      if (threadIdx.x == 0) partA[a.vb] = s;
    }
    if (!grid_barrier_n(a.bar, a.status, a.vnb)) return;
    const double pq = block_sum_array(partA, nb, smem);
    if (!(pq > 0.0) || !isfinite(pq)) { bad = true; break; }
    const double alpha = rho_cg / pq;
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
      if (threadIdx.x == 0) partB[a.vb] = s;
    }
    if (!grid_barrier_n(a.bar, a.status, a.vnb)) return;
    const double rr_new = block_sum_array(partB, nb, smem);
    if (!isfinite(rr_new)) { bad = true; break; }
    double rho_new = rr_new;
    if (a.precond && rr_new > thr) {
      double rz_l = 0.0;
      if (a.fused ? !apply_precond_fused(a, &rz_l) : !apply_precond(a, &rz_l)) return;
      const double s = block_sum(rz_l, smem);
      if (threadIdx.x == 0) partC[a.vb] = s;
      if (!grid_barrier_n(a.bar, a.status, a.vnb)) return;
      rho_new = block_sum_array(partC, nb, smem);
      if (!isfinite(rho_new)) { bad = true; break; }
    }
    beta = rho_new / rho_cg;
    rho_cg = rho_new;
    rr = rr_new;
    double *t = pold; pold = pnew; pnew = t;
    ++it;
  }
  if (a.vb == 0 && threadIdx.x == 0) {
    *a.iters_out = (double)it;
    if (bad) atomicCAS(a.status, 0, (int)KS_ENAN);
    else if (rr > thr) atomicCAS(a.status, 0, (int)KS_ENOCONV);
  }
}

__global__ void __launch_bounds__(kCgThreads) cg_kernel(CgArgs a) {
  a.vb = blockIdx.x;
  a.vnb = gridDim.x;
  cg_body(a);
}

// Sine basis Phi_{jk} = sqrt(2/(N+1)) sin(j k pi/(N+1)) (j, k = 1..N) and
// the 1-D eigenvalues kappa_j = (2/h)(1 - cos t_j), mu_j = (h/3)(2 + cos t_j),
// t_j = j pi/(N+1), in single precision for the preconditioner.
__global__ void sine_setup_kernel(int N, double h, float *phi, float *kap, float *mu) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N * N) {
    const int j = e / N + 1, k = e % N + 1;
    const long long jk = (long long)j * k % (2 * (N + 1));
    phi[e] = (float)(sqrt(2.0 / (N + 1)) * sinpi((double)jk / (N + 1)));
  }
  if (e < N) {
    const double c = cospi((double)(e + 1) / (N + 1));
    kap[e] = (float)((2.0 / h) * (1.0 - c));
    mu[e] = (float)((h / 3.0) * (2.0 + c));
  }
}

ks_status launch_sine_setup(Problem &P) {
  const int total = P.N * P.N;
  {
    ProfScope ps_(P.stream, KP_SETUP);
    sine_setup_kernel<<<(total + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(
        P.N, P.h, P.dst_phi, P.dst_kap, P.dst_mu);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
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
  a.z = P.cg_z;
  a.t1 = P.cg_t1;
  a.t2 = P.cg_t2;
  a.phi = P.dst_phi;
  a.kap = P.dst_kap;
  a.mu = P.dst_mu;
  a.part = P.partials;
  a.bar = P.bar;
  a.status = P.dstatus;
  a.iters_out = P.scal + SC_CG_ITERS;
  a.tol = P.cg_tol_phase > 0.0 ? P.cg_tol_phase : P.cg_tol;
  a.maxit = P.cg_maxit;
  a.warm = warm ? 1 : 0;
  a.precond = P.cg_precond;
  a.fused = P.N <= kFusedMaxN ? 1 : 0;
  const size_t dyn = cg_dynamic_smem(P.N);
  KS_CUDA_TRY(cudaMemsetAsync(P.bar, 0, sizeof(GridBarrier), P.stream));
  void *args[] = {&a};
  {
    ProfScope ps_(P.stream, KP_CG);
    KS_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)cg_kernel, dim3(P.cg_blocks),
                                            dim3(kCgThreads), args, dyn, P.stream));
  }
  return KS_OK;
}

// ---------------------------------------------------------------- batched
// The PCG of every job of a batch, one launch per CG phase over all jobs
// (no grid barrier: a phase's last block of each job finishes that job's
// reductions and scalar updates in device memory).  Phases:
//   init   r = b - K x (x = 0 when cold), r.r, b.b, tolerance
//   A/B/C  the fused sine-basis preconditioner, one block per (job, plane)
//          resp. (job, y-slab); C writes z and r.z and updates rho, beta
//   it1    p = s + beta p_old, q = K p, p.q -> alpha
//   it2    x += alpha p, r -= alpha q, r.r -> convergence
// A job that has converged (or failed) skips every later phase.  The host
// reads the number of jobs still iterating once per CG iteration.
struct CgState {
  double rr, bb, thr, rho, beta, alpha;
  int it, done, maxit, precond;
};

// Last block of one job's nb blocks: sums of the nchan partial channels
// part[c * nb + vb] (in block order) into s[]; true in that block only.
__device__ bool job_tail(double *part, int nb, int nchan, unsigned int *counter, double *smem,
                         double *s) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned int)nb - 1u);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int c = 0; c < nchan; ++c) s[c] = block_sum_array(part + (long long)c * nb, nb, smem);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

struct CgBatchView {
  const CgArgs *args;
  CgState *st;
  const int *start;                // block map of the phase
  int J;
  const unsigned char *active;
  const double *tolw;              // per job: tolerance, warm flag
  unsigned int *counters;          // one per job
};

__device__ __forceinline__ bool cg_job(const CgBatchView &v, int &j, int &vb, int &nb) {
  j = batch_job_of(v.start, v.J, blockIdx.x);
  if (!v.active[j] || v.st[j].done) return false;
  vb = blockIdx.x - v.start[j];
  nb = v.start[j + 1] - v.start[j];
  return true;
}

__global__ void __launch_bounds__(kCgThreads) cg_b_init(CgBatchView v) {
  __shared__ double smem[33];
  const int j = batch_job_of(v.start, v.J, blockIdx.x);
  if (!v.active[j]) return;
  const int vb = blockIdx.x - v.start[j], nb = v.start[j + 1] - v.start[j];
  const CgArgs &a = v.args[j];
  const int warm = v.tolw[2 * j + 1] != 0.0;
  const int N = a.N;
  const long long NN = (long long)N * N;
  double rr_l = 0.0, bb_l = 0.0;
  for (long long k = (long long)vb * blockDim.x + threadIdx.x; k < a.n;
       k += (long long)nb * blockDim.x) {
    const double b = a.bscale * a.rho[k];
    double kx = 0.0, dummy;
    if (warm) {
      const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
      kx = stiff_apply<false>(a.x, nullptr, 0.0, N, ix, iy, iz, a.c, &dummy);
    } else {
      a.x[k] = 0.0;
    }
    const double rk = b - kx;
    a.r[k] = rk;
    rr_l = fma(rk, rk, rr_l);
    bb_l = fma(b, b, bb_l);
  }
  const double s1 = block_sum(rr_l, smem), s2 = block_sum(bb_l, smem);
  if (threadIdx.x == 0) {
    a.part[vb] = s1;
    a.part[nb + vb] = s2;
  }
  double s[2];
  if (!job_tail(a.part, nb, 2, v.counters + j, smem, s)) return;
  if (threadIdx.x == 0) {
    CgState &t = v.st[j];
    const double tol = v.tolw[2 * j];
    t.rr = s[0];
    t.bb = s[1];
    t.thr = tol * tol * s[1];
    t.rho = s[0];
    t.beta = 0.0;
    t.it = 0;
    t.maxit = a.maxit;
    t.precond = a.precond;
    t.done = t.rr <= t.thr ? 1 : 0;
    *a.iters_out = 0.0;
  }
}

// Preconditioner passes (fused form; jobs with N > kFusedMaxN are refused at
// batch creation).  Stage 0: planes of r -> t1; 1: slabs t1 -> t2; 2: planes
// t2 -> z with r.z, then rho and beta.
template <int Stage>
__global__ void __launch_bounds__(kCgThreads) cg_b_precond(CgBatchView v) {
  __shared__ double smem[33];
  extern __shared__ float dyn[];
  int j, vb, nb;
  if (!cg_job(v, j, vb, nb)) return;
  CgArgs a = v.args[j];
  if (!v.st[j].precond) return;
  const int N = a.N, NN = N * N;
  a.vb = vb;
  a.vnb = nb;
  for (int e = threadIdx.x; e < NN; e += blockDim.x) dyn[NN + e] = __ldg(a.phi + e);
  if (Stage == 0) {
    fused_plane_pass<true, false>(a, a.r, a.t1, nullptr, dyn);
  } else if (Stage == 1) {
    fused_slab_pass(a, a.t1, a.t2, dyn);
  } else {
    const double rz_l = fused_plane_pass<false, true>(a, a.t2, nullptr, a.z, dyn);
    const double sum = block_sum(rz_l, smem);
    if (threadIdx.x == 0) a.part[vb] = sum;
    double s[1];
    if (!job_tail(a.part, nb, 1, v.counters + j, smem, s)) return;
    if (threadIdx.x == 0) {
      CgState &t = v.st[j];
      if (!isfinite(s[0])) {
        t.done = 1;
        atomicCAS(a.status, 0, (int)KS_ENAN);
      } else {
        t.beta = t.it == 0 ? 0.0 : s[0] / t.rho;
        t.rho = s[0];
      }
    }
  }
}

__global__ void __launch_bounds__(kCgThreads) cg_b_it1(CgBatchView v) {
  __shared__ double smem[33];
  int j, vb, nb;
  if (!cg_job(v, j, vb, nb)) return;
  const CgArgs &a = v.args[j];
  const CgState t = v.st[j];
  const int N = a.N;
  const long long NN = (long long)N * N;
  const double *s_vec = t.precond ? a.z : a.r;
  double *pold = (t.it % 2 == 0) ? a.pb : a.pa, *pnew = (t.it % 2 == 0) ? a.pa : a.pb;
  double pq_l = 0.0;
  for (long long k = (long long)vb * blockDim.x + threadIdx.x; k < a.n;
       k += (long long)nb * blockDim.x) {
    const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
    double pk;
    const double qk = t.it == 0 ? stiff_apply<false>(s_vec, nullptr, 0.0, N, ix, iy, iz, a.c, &pk)
                                : stiff_apply<true>(s_vec, pold, t.beta, N, ix, iy, iz, a.c, &pk);
    pnew[k] = pk;
    a.q[k] = qk;
    pq_l = fma(pk, qk, pq_l);
  }
  const double sum = block_sum(pq_l, smem);
  if (threadIdx.x == 0) a.part[vb] = sum;
  double s[1];
  if (!job_tail(a.part, nb, 1, v.counters + j, smem, s)) return;
  if (threadIdx.x == 0) {
    CgState &u = v.st[j];
    if (!(s[0] > 0.0) || !isfinite(s[0])) {
      u.done = 1;
      atomicCAS(a.status, 0, (int)KS_ENAN);
    } else {
      u.alpha = u.rho / s[0];
    }
  }
}

__global__ void __launch_bounds__(kCgThreads) cg_b_it2(CgBatchView v) {
  __shared__ double smem[33];
  int j, vb, nb;
  if (!cg_job(v, j, vb, nb)) return;
  const CgArgs &a = v.args[j];
  const CgState t = v.st[j];
  const double *p = (t.it % 2 == 0) ? a.pa : a.pb;
  double rl = 0.0;
  for (long long k = (long long)vb * blockDim.x + threadIdx.x; k < a.n;
       k += (long long)nb * blockDim.x) {
    a.x[k] = fma(t.alpha, p[k], a.x[k]);
    const double rk = fma(-t.alpha, a.q[k], a.r[k]);
    a.r[k] = rk;
    rl = fma(rk, rk, rl);
  }
  const double sum = block_sum(rl, smem);
  if (threadIdx.x == 0) a.part[vb] = sum;
  double s[1];
  if (!job_tail(a.part, nb, 1, v.counters + j, smem, s)) return;
  if (threadIdx.x == 0) {
    CgState &u = v.st[j];
    ++u.it;
    u.rr = s[0];
    *a.iters_out = (double)u.it;
    if (!isfinite(s[0])) {
      u.done = 1;
      atomicCAS(a.status, 0, (int)KS_ENAN);
    } else if (s[0] <= u.thr) {
      u.done = 1;
    } else if (u.it >= u.maxit) {
      u.done = 1;
      atomicCAS(a.status, 0, (int)KS_ENOCONV);
    } else if (!u.precond) {
      u.beta = s[0] / u.rho;
      u.rho = s[0];
    }
  }
}

// Number of active jobs still iterating.
__global__ void cg_b_count(const CgState *st, const unsigned char *active, int J, int *out) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) c += active[j] && !st[j].done;
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) *out = cnt;
}

ks_status batch_cg_setup(Batch &B) {
  if (B.maxN > kFusedMaxN)
    return set_error(KS_EINVAL, "batch: N above %d (the fused Hartree preconditioner)", kFusedMaxN);
  KS_CUDA_TRY(cudaFuncSetAttribute(cg_b_precond<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)cg_dynamic_smem(kFusedMaxN)));
  KS_CUDA_TRY(cudaFuncSetAttribute(cg_b_precond<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)cg_dynamic_smem(kFusedMaxN)));
  KS_CUDA_TRY(cudaFuncSetAttribute(cg_b_precond<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)cg_dynamic_smem(kFusedMaxN)));
  std::vector<CgArgs> args(B.J);
  for (int j = 0; j < B.J; ++j) {
    Problem &P = B.probs[j]->P;
    const BJob &b = B.jobs_host[j];
    CgArgs &a = args[j];
    a = CgArgs{};
    a.N = P.N;
    a.n = P.n;
    a.c = q1_coefficients(P.h);
    a.bscale = 4.0 * M_PI * P.h * P.h * P.h;
    a.rho = P.rho;
    a.x = P.vH;
    a.r = P.cg_r;
    a.pa = P.cg_pa;
    a.pb = P.cg_pb;
    a.q = P.cg_q;
    a.z = P.cg_z;
    a.t1 = P.cg_t1;
    a.t2 = P.cg_t2;
    a.phi = P.dst_phi;
    a.kap = P.dst_kap;
    a.mu = P.dst_mu;
    a.part = P.partials;
    a.bar = P.bar;
    a.status = b.status;
    a.iters_out = b.scal + SC_CG_ITERS;
    a.tol = P.cg_tol;
    a.maxit = P.cg_maxit;
    a.precond = P.cg_precond;
    a.fused = 1;
  }
  void *mem = nullptr;
  const size_t abytes = ((sizeof(CgArgs) * B.J + 255) / 256) * 256;
  const size_t sbytes = ((sizeof(CgState) * B.J + 255) / 256) * 256;
  const size_t tbytes = sizeof(double) * 2 * B.J, cbytes = sizeof(unsigned int) * (B.J + 1);
  KS_CUDA_TRY(cudaMalloc(&mem, abytes + sbytes + tbytes + cbytes));
  char *m = static_cast<char *>(mem);
  B.cg_args_dev = mem;
  B.cg_state_dev = m + abytes;
  B.cg_tolw_dev = reinterpret_cast<double *>(m + abytes + sbytes);
  B.cg_counters = reinterpret_cast<unsigned int *>(m + abytes + sbytes + tbytes);
  KS_CUDA_TRY(cudaMemsetAsync(B.cg_state_dev, 0, sbytes, B.stream));
  KS_CUDA_TRY(cudaMemsetAsync(B.cg_counters, 0, cbytes, B.stream));
  KS_CUDA_TRY(cudaMemcpyAsync(B.cg_args_dev, args.data(), sizeof(CgArgs) * B.J,
                              cudaMemcpyHostToDevice, B.stream));
  KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
  B.bytes += abytes + sbytes + tbytes + cbytes;
  return KS_OK;
}

// Hartree solve of every active job (warm-started where B.warm says so) to
// relative residual max(tol, the job's cg_tol), in three pieces so that the
// launches can be captured in a CUDA graph:
//   batch_cg_upload   per-job tolerance and warm flag (host -> device)
//   batch_cg_launch   init + preconditioner + `iters` CG iterations and the
//                     count of jobs still iterating (no host synchronisation)
//   batch_cg_continue more iterations, one host check each, until no job is
//                     left (after a synchronisation that read the count)
static CgBatchView cg_view(Batch &B, int map) {
  return CgBatchView{static_cast<const CgArgs *>(B.cg_args_dev),
                     static_cast<CgState *>(B.cg_state_dev), B.map(map), B.J, B.active_dev,
                     B.cg_tolw_dev, B.cg_counters};
}

static ks_status cg_precond_launch(Batch &B) {
  const CgBatchView planes = cg_view(B, BM_CG_PLANES);
  const int np = B.total(BM_CG_PLANES);
  const size_t dyn = cg_dynamic_smem(B.maxN);
  cg_b_precond<0><<<np, kCgThreads, dyn, B.stream>>>(planes);
  cg_b_precond<1><<<np, kCgThreads, dyn, B.stream>>>(planes);
  cg_b_precond<2><<<np, kCgThreads, dyn, B.stream>>>(planes);
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

static ks_status cg_iteration_launch(Batch &B) {
  const CgBatchView nodes = cg_view(B, BM_CG_NODES);
  const int nn = B.total(BM_CG_NODES);
  ProfScope ps_(B.stream, KP_CG, 0.0, 0.0, 6);
  cg_b_it1<<<nn, kCgThreads, 0, B.stream>>>(nodes);
  cg_b_it2<<<nn, kCgThreads, 0, B.stream>>>(nodes);
  KS_CUDA_TRY(cudaGetLastError());
  KS_TRY(cg_precond_launch(B));
  cg_b_count<<<1, 256, 0, B.stream>>>(static_cast<const CgState *>(B.cg_state_dev), B.active_dev,
                                      B.J, B.cg_remaining_dev);
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status batch_cg_upload(Batch &B, double tol) {
  for (int j = 0; j < B.J; ++j) {
    const double t = tol > B.probs[j]->P.cg_tol ? tol : B.probs[j]->P.cg_tol;
    B.cg_tolw_host[2 * j] = t;
    B.cg_tolw_host[2 * j + 1] = B.warm[j] ? 1.0 : 0.0;
  }
  KS_CUDA_TRY(cudaMemcpyAsync(B.cg_tolw_dev, B.cg_tolw_host, sizeof(double) * 2 * B.J,
                              cudaMemcpyHostToDevice, B.stream));
  return KS_OK;
}

ks_status batch_cg_launch(Batch &B, int iters) {
  const CgBatchView nodes = cg_view(B, BM_CG_NODES);
  {
    ProfScope ps_(B.stream, KP_CG, 0.0, 0.0, 5);
    cg_b_init<<<B.total(BM_CG_NODES), kCgThreads, 0, B.stream>>>(nodes);
    KS_CUDA_TRY(cudaGetLastError());
    KS_TRY(cg_precond_launch(B));
    cg_b_count<<<1, 256, 0, B.stream>>>(static_cast<const CgState *>(B.cg_state_dev),
                                        B.active_dev, B.J, B.cg_remaining_dev);
    KS_CUDA_TRY(cudaGetLastError());
  }
  for (int it = 0; it < iters; ++it) KS_TRY(cg_iteration_launch(B));
  return KS_OK;
}

ks_status batch_cg_continue(Batch &B) {
  int maxit = 0;
  for (int j = 0; j < B.J; ++j)
    if (B.active_host[j] && B.probs[j]->P.cg_maxit > maxit) maxit = B.probs[j]->P.cg_maxit;
  for (int it = 0; it < maxit; ++it) {
    KS_CUDA_TRY(cudaMemcpyAsync(B.cg_remaining_host, B.cg_remaining_dev, sizeof(int),
                                cudaMemcpyDeviceToHost, B.stream));
    KS_CUDA_TRY(cudaStreamSynchronize(B.stream));
    if (*B.cg_remaining_host == 0) break;
    KS_TRY(cg_iteration_launch(B));
  }
  return KS_OK;
}

ks_status batch_cg(Batch &B, double tol) {
  KS_TRY(batch_cg_upload(B, tol));
  KS_TRY(batch_cg_launch(B, 0));
  return batch_cg_continue(B);
}

size_t cg_dynamic_smem(int N) {
  return N <= kFusedMaxN ? (size_t)3 * N * N * sizeof(float) : kTiledSmem;
}

int cg_grid_blocks(int sms, int n, int N) {
  const size_t dyn = cg_dynamic_smem(N);
  // always opt in to the largest fused size, so that problems of different
  // N (e.g. concurrent server jobs) never lower the limit under each other
  if (cudaFuncSetAttribute(cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cg_dynamic_smem(kFusedMaxN)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel, kCgThreads, dyn) !=
      cudaSuccess || per_sm < 1)
    per_sm = 1;
  long long want = (n + kCgThreads - 1) / kCgThreads;
  long long cap = (long long)sms * (per_sm < 2 ? per_sm : 2);
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace ks
