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
  int incr;                   // warm start with r = b_old - K x still in r
  double *rho_prev;           // density of the last solve (its b / bscale)
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

// Fused form for N <= kFusedMaxN, with the planes in shared memory (three
// N x ld matrices of dynamic shared memory: a plane, Phi and a work matrix;
// ld = 68 for N <= 64, 132 above, so that every 16-byte row access of a
// 64-wide output tile stays inside its row):
//   A: each z-plane P (N x N, rows y, columns x) -> Phi P Phi   (y, then x)
//   B: each y-slab S (rows z, columns x)          -> Phi (Lambda^{-1} o (Phi S))
//   C: each z-plane                               -> Phi P Phi, written as z
// (Phi is symmetric, so Phi P Phi transforms both in-plane axes), three grid
// barriers per application instead of six.
constexpr int kFusedMaxN = 128;

__host__ __device__ constexpr int fused_ld(int N) { return N <= 64 ? 68 : 132; }

// out = A B for N x N matrices in shared memory (row stride ld), A given by
// its transpose At (At[k][i] = A[i][k]; Phi is its own transpose).  Each
// thread keeps a 4 x 4 block of a 64 x 64 output tile (rows 4 ty .. + 3,
// columns 4 tx .. + 3 with ty = tid / 16, tx = tid % 16): per k one 16-byte
// load of At (two addresses per warp, broadcast) and one of B (16
// consecutive ones) for 16 FMAs.  Each output is one k-ascending FMA chain.
// Trans: out is stored transposed (out[j][i]), ready to be the At of the
// next product.
template <bool Trans>
__device__ __forceinline__ void smem_matmul(const float *At, const float *B, float *out, int N,
                                            int ld) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int ib = 0; ib < N; ib += 64)
    for (int jb = 0; jb < N; jb += 64) {
      const int i0 = ib + 4 * ty, j0 = jb + 4 * tx;
      if (i0 >= N || j0 >= N) continue;
      // every 16-byte row access of the tile stays inside its row
      if (!KS_IN(i0 + 3, ld) || !KS_IN(j0 + 3, ld)) continue;
      float acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 4
      for (int k = 0; k < N; ++k) {
        const float4 av = *reinterpret_cast<const float4 *>(At + k * ld + i0);
        const float4 bv = *reinterpret_cast<const float4 *>(B + k * ld + j0);
        const float a4[4] = {av.x, av.y, av.z, av.w};
        const float b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a4[u], b4[v], acc[u][v]);
      }
      // rows / columns past N land in the padding of the row (never read as
      // data: every product sums k < N only)
      if (Trans) {
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (j0 + v < N)
            *reinterpret_cast<float4 *>(out + (j0 + v) * ld + i0) =
                make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i0 + u < N)
            *reinterpret_cast<float4 *>(out + (i0 + u) * ld + j0) =
                make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
      }
    }
}

// Element (r, c) of an N x N plane for every r, c < N: warp w takes rows
// w, w + 8, ..., its lanes the columns (coalesced, no index division), in
// 64 x 64 patches of 16 values per thread whose loads are all issued before
// the first is used, so a patch costs about one memory latency.
template <typename V, typename L, typename U>
__device__ __forceinline__ void plane_batched(int N, L load, U use) {
  static_assert(kCgThreads == 256, "8 warps x 8 rows make a 64-row patch");
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int r0 = 0; r0 < N; r0 += 64)
    for (int c0 = 0; c0 < N; c0 += 64) {
      V v[8][2];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r = r0 + w + 8 * i, c = c0 + l + 32 * j;
          v[i][j] = (r < N && c < N) ? load(r, c) : V(0);
        }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r = r0 + w + 8 * i, c = c0 + l + 32 * j;
          if (r < N && c < N) use(r, c, v[i][j]);
        }
    }
}

// Shared memory of the fused preconditioner: plane, Phi and work matrices
// (N x ld each), then the 1-D eigenvalues kappa and mu (N each).
__host__ __device__ constexpr size_t fused_smem_floats(int N) {
  return (size_t)3 * N * fused_ld(N) + 2 * (size_t)N;
}

// Phi, kappa and mu into shared memory (once per kernel).
__device__ __forceinline__ void load_phi(const CgArgs &a, float *sh) {
  const int N = a.N, ld = fused_ld(N);
  float *Ph = sh + N * ld, *kap = sh + 3 * N * ld, *mu = kap + N;
  plane_batched<float>(
      N, [&](int r, int c) { return __ldg(a.phi + r * N + c); },
      [&](int r, int c, float v) { Ph[r * ld + c] = v; });
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    kap[i] = __ldg(a.kap + i);
    mu[i] = __ldg(a.mu + i);
  }
}

// Phi P Phi of the plane in Pm (already staged), y then x; the result is
// left in Pm.
__device__ __forceinline__ void plane_transform(int N, int ld, float *sh) {
  float *Pm = sh, *Ph = sh + N * ld, *W = sh + 2 * N * ld;
  __syncthreads();
  smem_matmul<true>(Ph, Pm, W, N, ld);     // W^T, W = Phi P (along y)
  __syncthreads();
  smem_matmul<false>(W, Ph, Pm, N, ld);    // (Phi P) Phi (along x)
  __syncthreads();
}

// Phi P Phi for the plane z of `in` (FP64 r or FP32 work), into out32 or,
// for the last step, out64 with the r.z accumulation.
template <bool InD, bool OutD>
__device__ double fused_plane_pass(const CgArgs &a, const void *in, float *out32, double *out64,
                                   float *sh) {
  const int N = a.N, ld = fused_ld(N);
  const long long NN = (long long)N * N;
  float *Pm = sh;
  double rz = 0.0;
  for (int z = a.vb; z < N; z += a.vnb) {
    const long long zo = z * NN;
    __syncthreads();
    if (InD)
      plane_batched<double>(
          N,
          [&](int y, int x) {
            return KS_IN(zo + y * N + x, a.n) ? __ldcg((const double *)in + zo + y * N + x) : 0.0;
          },
          [&](int y, int x, double v) { Pm[y * ld + x] = (float)v; });
    else
      plane_batched<float>(
          N,
          [&](int y, int x) {
            return KS_IN(zo + y * N + x, a.n) ? __ldcg((const float *)in + zo + y * N + x) : 0.f;
          },
          [&](int y, int x, float v) { Pm[y * ld + x] = v; });
    plane_transform(N, ld, sh);
    if (OutD)
      plane_batched<double>(
          N, [&](int y, int x) { return __ldcg(a.r + zo + y * N + x); },
          [&](int y, int x, double rv) {
            const double zv = (double)Pm[y * ld + x];
            if (KS_IN(zo + y * N + x, a.n)) out64[zo + y * N + x] = zv;
            rz = fma(rv, zv, rz);
          });
    else
      plane_batched<float>(
          N, [&](int y, int x) { return Pm[y * ld + x]; },
          [&](int y, int x, float v) {
            if (KS_IN(zo + y * N + x, a.n)) out32[zo + y * N + x] = v;
          });
  }
  return rz;
}

// For each y: S[z][x] -> Phi (Lambda^{-1} o (Phi S)) along z.
__device__ void fused_slab_pass(const CgArgs &a, const float *in, float *out, float *sh) {
  const int N = a.N, ld = fused_ld(N);
  const long long NN = (long long)N * N;
  float *Sm = sh, *Ph = sh + N * ld, *W = sh + 2 * N * ld;
  const float *kap = sh + 3 * N * ld, *mu = kap + N;
  for (int y = a.vb; y < N; y += a.vnb) {
    __syncthreads();
    plane_batched<float>(
        N,
        [&](int zz, int x) {
          const long long k = zz * NN + (long long)y * N + x;
          return KS_IN(k, a.n) ? __ldcg(in + k) : 0.f;
        },
        [&](int zz, int x, float v) { Sm[zz * ld + x] = v; });
    __syncthreads();
    smem_matmul<false>(Ph, Sm, W, N, ld);   // forward along z
    __syncthreads();
    const float ky = kap[y], my = mu[y];
    for (int c = threadIdx.x >> 5; c < N; c += kCgThreads / 32)
      for (int x = threadIdx.x & 31; x < N; x += 32) {
        const float lam = kap[x] * my * mu[c] + mu[x] * ky * mu[c] + mu[x] * my * kap[c];
        W[c * ld + x] = W[c * ld + x] / lam;
      }
    __syncthreads();
    smem_matmul<false>(Ph, W, Sm, N, ld);   // inverse along z
    __syncthreads();
    plane_batched<float>(
        N, [&](int zz, int x) { return Sm[zz * ld + x]; },
        [&](int zz, int x, float v) {
          const long long k = zz * NN + (long long)y * N + x;
          if (KS_IN(k, a.n)) out[k] = v;
        });
  }
}

__device__ bool apply_precond_fused(const CgArgs &a, double *rz_l) {
  extern __shared__ float dyn[];
  fused_plane_pass<true, false>(a, a.r, a.t1, nullptr, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  fused_slab_pass(a, a.t1, a.t2, dyn);
  if (!grid_barrier_n(a.bar, a.status, a.vnb)) return false;
  *rz_l = fused_plane_pass<false, true>(a, a.t2, nullptr, a.z, dyn);
  return true;
}

// The whole PCG of one system on the blocks a.vb = 0 .. a.vnb - 1 (which must
// be co-resident: a cooperative launch).
//
// On GB300 every FP64 FMA is scarce (two lanes per SM and clock), so each
// iteration applies the 27-point stiffness once: q = K p is carried as
// q = K s + beta q_old (K p by linearity, p = s + beta p_old), and a warm
// start whose residual is still in r (a.incr) forms the new one without a
// stencil, r = r_old + (b - b_old), from the right-hand side of the last
// solve (rho_prev).
__device__ void cg_body(const CgArgs &a) {
  __shared__ double smem[33];
  const int nb = a.vnb;
  double *partA = a.part, *partB = a.part + nb, *partC = a.part + 2 * nb, *partD = a.part + 3 * nb;
  const long long tid = (long long)a.vb * blockDim.x + threadIdx.x;
  const long long stride = (long long)a.vnb * blockDim.x;
  const int N = a.N;
  const long long NN = (long long)N * N;
  if (a.fused && a.precond) {
    extern __shared__ float dyn[];
    load_phi(a, dyn);
  }

  // r = b - K x0 (x0 = 0 for a cold start; r_old + b - b_old when
  // incremental), b.b, and rho_prev = rho for the next solve
  double rr_l = 0.0, bb_l = 0.0;
  for (long long k = tid; k < a.n; k += stride) {
    const double rk_rho = a.rho[k];
    const double b = a.bscale * rk_rho;
    double rk;
    if (a.incr) {
      rk = a.r[k] + a.bscale * (rk_rho - a.rho_prev[k]);
    } else {
      double kx = 0.0, dummy;
      if (a.warm) {
        const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
        kx = stiff_apply<false>(a.x, nullptr, 0.0, N, ix, iy, iz, a.c, &dummy);
      }
      rk = b - kx;
    }
    a.r[k] = rk;
    a.rho_prev[k] = rk_rho;
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
    // phase 1: p = s + beta p_old and q = K s + beta q_old (own nodes), p.q
    double pq_l = 0.0;
    for (long long k = tid; k < a.n; k += stride) {
      const int ix = (int)(k % N), iy = (int)((k / N) % N), iz = (int)(k / NN);
      double sk;
      const double ks = stiff_apply<false>(s_vec, nullptr, 0.0, N, ix, iy, iz, a.c, &sk);
      const double pk = it == 0 ? sk : fma(beta, pold[k], sk);
      const double qk = it == 0 ? ks : fma(beta, a.q[k], ks);
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

constexpr int kCgIncrMax = 64;

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
  // the residual of the last solve is reused while the problem's own vH and
  // r carry it; every kCgIncrMax-th warm start recomputes it from x, so
  // that the rounding of the recurrences cannot build up
  const bool own = v == P.vH && r == P.cg_r;
  a.incr = (warm && own && P.cg_inc_ok && P.cg_inc_count < kCgIncrMax) ? 1 : 0;
  a.rho_prev = P.cg_rho_prev;
  P.cg_inc_count = a.incr ? P.cg_inc_count + 1 : 0;
  P.cg_inc_ok = own;
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
  a.vb = vb;
  a.vnb = nb;
  load_phi(a, dyn);
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
  return N <= kFusedMaxN ? fused_smem_floats(N) * sizeof(float) : kTiledSmem;
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

KS_OOB_READER(cg)

}  // namespace ks
