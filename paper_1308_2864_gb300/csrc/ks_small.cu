// Small dense FP64 algebra of the retractions, one thread block each (the
// p x p and 2p x 2p systems are serial in the paper too; here they stay on
// the device so the iteration needs no host round trip for them):
//   qr_factor:     Cholesky of Y^T M Y = I + tau^2 D^T M D (Prop. 3.1 in the
//                  M metric; Alg. ChQR), then C = L^{-T}, giving
//                  X+ = (X - tau D) L^{-T} = X C + D (-tau C)   (Eq. QR)
//   cayley_factor: LU with partial pivoting of I + tau/2 V^T U (2p x 2p) and
//                  the solve against V^T Y (Eq. WY3); for p = 1 the closed
//                  form of Lemma 3.1 (3) (Eq. WY-1d), no solve.
#include "ks_device.cuh"

namespace ks {

constexpr int kSmallThreads = 1024;

// The factor keeps W, L^{-1} and the pivots (2 p^2 + p doubles) in shared
// memory up to p = kSmemMaxP, in global scratch (L2-resident) above.
constexpr int kSmemMaxP = 104;

// 1/sqrt(d) for d > 0 in FP64: FP32 seed, then two Newton steps
// y <- y (3 - d y^2) / 2 (each doubles the correct bits: 24 -> 48 -> 53).
__device__ __forceinline__ double rsqrt_newton(double d) {
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}

// Flat index t of the lower triangle (diagonal included, rows in order, row
// i starting at i (i + 1) / 2) -> (i, c), c <= i.  FP32 square root plus an
// integer correction: no FP64 instruction.
__device__ __forceinline__ void tri_decode(int t, int &i, int &c) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r > 0 && r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  i = r;
  c = t - r * (r + 1) / 2;
}

// Pivot j: L_jj = sqrt(w) and its reciprocal; false on a non-positive or
// non-finite w (records KS_ENOTPD).
__device__ __forceinline__ bool chol_pivot(double w, int j, double *W, int p, double *rdiag,
                                           int *s_fail, int *status) {
  if (!(w > 0.0) || !isfinite(w)) {
    *s_fail = 1;
    atomicCAS(status, 0, (int)KS_ENOTPD);
    return false;
  }
  const double y = rsqrt_newton(w);
  W[j * p + j] = w * y;
  rdiag[j] = y;
  return true;
}

// Right-looking Cholesky W = L L^T merged with the inversion of L: with
// R = I at the start, step j (i) scales column j of L by 1/L_jj and row j of
// R by the same, which makes it row j of L^{-1}; (ii) for every row i > j
// updates W[i][k] -= L_ij L_kj (j < k <= i) and R[i][c] -= L_ij V[j][c]
// (c <= j).  Step (ii) is one flat loop over the lower triangle below row
// j, so all warps stay busy; the thread that updates W[j+1][j+1] also takes
// the next pivot, leaving two barriers per column.  On GB300 one SM retires
// two FP64 lanes per clock, so dense warps and no divisions matter more
// than anything else here.
// The loop of the merged factor on W (p x p, W -> L) and V (= I at the
// start, -> L^{-1}); false (block-uniform) on a failed pivot.
__device__ __forceinline__ bool chol_inv_core(double *W, double *V, double *rdiag, int p,
                                              int *status) {
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  if (threadIdx.x == 0) chol_pivot(W[0], 0, W, p, rdiag, &s_fail, status);
  __syncthreads();
  const int tend = p * (p + 1) / 2;
  for (int j = 0; j < p; ++j) {
    if (s_fail) return false;
    const double inv = rdiag[j];
    const int below = p - j - 1;
    for (int t = threadIdx.x; t < below + j + 1; t += blockDim.x) {
      if (t < below) W[(j + 1 + t) * p + j] *= inv;
      else V[j * p + (t - below)] *= inv;
    }
    __syncthreads();
    for (int t = (j + 1) * (j + 2) / 2 + threadIdx.x; t < tend; t += blockDim.x) {
      int i, c;
      tri_decode(t, i, c);
      const double lij = W[i * p + j];
      if (c <= j) {
        V[i * p + c] = fma(-lij, V[j * p + c], V[i * p + c]);
      } else {
        const double w = fma(-lij, W[c * p + j], W[i * p + c]);
        W[i * p + c] = w;
        if (i == j + 1 && c == j + 1) chol_pivot(w, j + 1, W, p, rdiag, &s_fail, status);
      }
    }
    __syncthreads();
  }
  return true;
}

// W (p*p: W -> L), V (p*p: R -> L^{-1}, row-major) and rdiag (p) live in
// shared memory (p <= kSmemMaxP).
__device__ __forceinline__ void qr_factor_body(int p, const double *DMD, const double *O,
                                               double tau, double *C1, double *C2, int *status,
                                               double *W, double *V, double *rdiag) {
  const double t2 = tau * tau;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    double r = O ? O[e] : (i == j ? 1.0 : 0.0);
    if (DMD) r = fma(t2, DMD[e], r);
    W[e] = r;
    V[e] = i == j ? 1.0 : 0.0;
  }
  if (!chol_inv_core(W, V, rdiag, p, status)) return;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    const double cval = V[j * p + i];     // (L^{-T})_{ij} = (L^{-1})_{ji}
    C1[e] = cval;
    if (C2) C2[e] = -tau * cval;
  }
}

__device__ __forceinline__ void qr_factor_smem_body(int p, const double *DMD, const double *O,
                                                    double tau, double *C1, double *C2,
                                                    int *status) {
  extern __shared__ double sh_w[];
  qr_factor_body(p, DMD, O, tau, C1, C2, status, sh_w, sh_w + p * p, sh_w + 2 * p * p);
}

__global__ void __launch_bounds__(kSmallThreads) qr_factor_smem_kernel(
    int p, const double *DMD, const double *O, double tau, double *C1, double *C2, int *status) {
  qr_factor_smem_body(p, DMD, O, tau, C1, C2, status);
}

// ---------------------------------------------------------------- large p
// p > kSmemMaxP: the same factorisation blocked by panels of kBlk columns,
// so that the O(p^3) work spreads over the SMs (one SM retires only two
// FP64 lanes per clock).  W (p x p, ld p) becomes L and V (= I at the
// start) becomes L^{-1}; for each panel k:
//   diag:   L_kk L_kk^T = W_kk and L_kk^{-1} (the merged kernel, one block)
//   row/pn: V_km = L_kk^{-1} R_km (m <= k)  and  L_ik = W_ik L_kk^{-T} (i > k)
//   update: W_ij -= L_ik L_jk^T (k < j <= i)  and  R_im -= L_ik V_km (i > k, m <= k)
// (R is V before its rows are final; block rows below the panel are updated
// by every panel above them, exactly the scalar algorithm by blocks).
constexpr int kBlk = 32;
constexpr int kBlkThreads = 256;

__global__ void blk_init_kernel(int p, const double *DMD, const double *O, double tau, double *W,
                                double *V) {
  const double t2 = tau * tau;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)p * p;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / p), j = (int)(e % p);
    double r = O ? O[e] : (i == j ? 1.0 : 0.0);
    if (DMD) r = fma(t2, DMD[e], r);
    W[e] = r;
    V[e] = i == j ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(kBlkThreads) blk_diag_kernel(double *W, int p, int k0,
                                                               double *Dinv, int *status) {
  __shared__ double Ws[kBlk * kBlk], Vs[kBlk * kBlk], rd[kBlk];
  const int nb = min(kBlk, p - k0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    Ws[e] = W[(long long)(k0 + i) * p + k0 + j];
    Vs[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  if (!chol_inv_core(Ws, Vs, rd, nb, status)) return;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    W[(long long)(k0 + i) * p + k0 + j] = j <= i ? Ws[e] : 0.0;
    Dinv[i * kBlk + j] = Vs[e];
  }
}

// out (mr x mc, ld ldo) = (acc ? out : 0) + sgn * A (mr x kk, ld lda) op(B),
// op(B) = B (kk x mc, ld ldb) or B^T (B mc x kk); both operands are staged
// in shared memory before out is written, so out may alias either.
__device__ void blk_gemm(double *out, int ldo, const double *A, int lda, const double *B, int ldb,
                         bool transB, int mr, int mc, int kk, double sgn, bool acc) {
  __shared__ double As[kBlk][kBlk + 1], Bs[kBlk][kBlk + 1];
  for (int e = threadIdx.x; e < kBlk * kBlk; e += blockDim.x) {
    const int r = e / kBlk, c = e % kBlk;
    As[r][c] = (r < mr && c < kk) ? A[(long long)r * lda + c] : 0.0;
    // Bs[k][c] = op(B)[k][c]
    if (transB) Bs[r][c] = (c < mc && r < kk) ? B[(long long)c * ldb + r] : 0.0;
    else Bs[r][c] = (r < kk && c < mc) ? B[(long long)r * ldb + c] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  double a4[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < kk; ++k) {
    const double a = As[r][k];
#pragma unroll
    for (int u = 0; u < 4; ++u) a4[u] = fma(a, Bs[k][c0 + u], a4[u]);
  }
  if (r < mr)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      if (c < mc) {
        double *o = out + (long long)r * ldo + c;
        *o = acc ? fma(sgn, a4[u], *o) : sgn * a4[u];
      }
    }
}

__device__ __forceinline__ int blk_size(int p, int b) { return min(kBlk, p - b * kBlk); }

// rows of V (block row k) and the panel below the diagonal block
__global__ void __launch_bounds__(kBlkThreads) blk_rowpanel_kernel(double *W, double *V, int p,
                                                                   int k, const double *Dinv) {
  const int K = (p + kBlk - 1) / kBlk;
  const int nk = blk_size(p, k);
  const int b = blockIdx.x;
  if (b <= k) {                      // V_kb = L_kk^{-1} R_kb
    const int m = b;
    double *vb = V + (long long)k * kBlk * p + m * kBlk;
    blk_gemm(vb, p, Dinv, kBlk, vb, p, false, nk, blk_size(p, m), nk, 1.0, false);
  } else {                           // L_ik = W_ik L_kk^{-T}
    const int i = k + (b - k);
    if (i >= K) return;
    double *wb = W + (long long)i * kBlk * p + k * kBlk;
    blk_gemm(wb, p, wb, p, Dinv, kBlk, true, blk_size(p, i), nk, nk, 1.0, false);
  }
}

__global__ void __launch_bounds__(kBlkThreads) blk_update_kernel(double *W, double *V, int p,
                                                                 int k) {
  const int K = (p + kBlk - 1) / kBlk;
  const int nk = blk_size(p, k);
  const int below = K - k - 1;
  const int ntri = below * (below + 1) / 2;
  int b = blockIdx.x;
  if (b < ntri) {                    // W_ij -= L_ik L_jk^T, k < j <= i
    int ii = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while (ii > 0 && ii * (ii + 1) / 2 > b) --ii;
    while ((ii + 1) * (ii + 2) / 2 <= b) ++ii;
    const int jj = b - ii * (ii + 1) / 2;
    const int i = k + 1 + ii, j = k + 1 + jj;
    blk_gemm(W + (long long)i * kBlk * p + j * kBlk, p, W + (long long)i * kBlk * p + k * kBlk, p,
             W + (long long)j * kBlk * p + k * kBlk, p, true, blk_size(p, i), blk_size(p, j), nk,
             -1.0, true);
  } else {                           // R_im -= L_ik V_km, i > k, m <= k
    b -= ntri;
    const int i = k + 1 + b / (k + 1), m = b % (k + 1);
    if (i >= K) return;
    blk_gemm(V + (long long)i * kBlk * p + m * kBlk, p, W + (long long)i * kBlk * p + k * kBlk, p,
             V + (long long)k * kBlk * p + m * kBlk, p, false, blk_size(p, i), blk_size(p, m), nk,
             -1.0, true);
  }
}

__global__ void blk_out_kernel(int p, const double *V, double tau, double *C1, double *C2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)p * p;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / p), j = (int)(e % p);
    const double c = V[(long long)j * p + i];
    C1[e] = c;
    if (C2) C2[e] = -tau * c;
  }
}

static ks_status launch_qr_factor_blocked(Problem &P, const double *DMD, const double *O,
                                          double tau, double *C1, double *C2) {
  const int p = P.p, K = (p + kBlk - 1) / kBlk;
  double *W = P.pp + (size_t)S_WORK * p * p, *V = W + (size_t)p * p, *Dinv = V + (size_t)p * p;
  const int ng = (int)(((long long)p * p + 255) / 256);
  blk_init_kernel<<<ng, 256, 0, P.stream>>>(p, DMD, O, tau, W, V);
  for (int k = 0; k < K; ++k) {
    blk_diag_kernel<<<1, kBlkThreads, 0, P.stream>>>(W, p, k * kBlk, Dinv, P.dstatus);
    blk_rowpanel_kernel<<<K, kBlkThreads, 0, P.stream>>>(W, V, p, k, Dinv);
    const int below = K - k - 1;
    const int nupd = below * (below + 1) / 2 + below * (k + 1);
    if (nupd > 0) blk_update_kernel<<<nupd, kBlkThreads, 0, P.stream>>>(W, V, p, k);
  }
  blk_out_kernel<<<ng, 256, 0, P.stream>>>(p, V, tau, C1, C2);
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Batched: block j factors job j (p <= kSmemMaxP): R = I + tau_j^2 DMD
// (with_tau) or R = O, written to C1 (and C2 = -tau_j C1 when smC2 >= 0).
__global__ void __launch_bounds__(kSmallThreads) qr_factor_batch_kernel(
    const BJob *__restrict__ jobs, const unsigned char *__restrict__ active,
    const double *__restrict__ tau, int smDMD, int smO, int with_tau, int smC1, int smC2) {
  const int j = blockIdx.x;
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const size_t len = (size_t)b.p * b.p;
  qr_factor_smem_body(b.p, with_tau ? b.pp + smDMD * len : nullptr,
                      smO >= 0 ? b.pp + smO * len : nullptr, with_tau ? tau[j] : 0.0,
                      b.pp + smC1 * len, smC2 >= 0 ? b.pp + smC2 * len : nullptr, b.status);
}

ks_status batch_qr_factor(Batch &B, int smDMD, int smO, bool with_tau, int smC1, int smC2) {
  if (B.maxp > kSmemMaxP) return set_error(KS_EINVAL, "batch: p above %d", kSmemMaxP);
  const size_t smem = ((size_t)2 * B.maxp * B.maxp + B.maxp) * sizeof(double);
  {
    ProfScope ps_(B.stream, KP_SMALL);
    qr_factor_batch_kernel<<<B.J, kSmallThreads, smem, B.stream>>>(
        B.jobs_dev, B.active_dev, B.tau_dev, smDMD, smO, with_tau ? 1 : 0, smC1, smC2);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Opt the shared-memory factor kernel into its dynamic shared memory (on the
// current device; called when a problem is created).
ks_status configure_small_kernels() {
  const int smem = (int)(((size_t)2 * kSmemMaxP * kSmemMaxP + kSmemMaxP) * sizeof(double));
  KS_CUDA_TRY(cudaFuncSetAttribute(qr_factor_smem_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  KS_CUDA_TRY(cudaFuncSetAttribute(qr_factor_batch_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return KS_OK;
}

ks_status launch_qr_factor(Problem &P, const double *DMD, const double *O, double tau,
                           double *C1, double *C2) {
  const int p = P.p;
  const double pf = (double)p;
  if (p <= kSmemMaxP) {
    const size_t smem = ((size_t)2 * p * p + p) * sizeof(double);
    {
      ProfScope ps_(P.stream, KP_SMALL, 2.0 * pf * pf * pf / 3.0, 0.0);
      qr_factor_smem_kernel<<<1, kSmallThreads, smem, P.stream>>>(p, DMD, O, tau, C1, C2,
                                                                  P.dstatus);
    }
    KS_CUDA_TRY(cudaGetLastError());
    return KS_OK;
  }
  {
    const int K = (p + kBlk - 1) / kBlk;
    ProfScope ps_(P.stream, KP_SMALL, 2.0 * pf * pf * pf / 3.0, 0.0, 3 * K + 1);
    KS_TRY(launch_qr_factor_blocked(P, DMD, O, tau, C1, C2));
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Solve (I + tau/2 N) P = R with N = [[A, O], [-B, -S]] and R = [O; -S]
// (all p x p blocks, O = I when null), by Gaussian elimination with partial
// pivoting on the augmented 2p x 3p matrix W.
__global__ void __launch_bounds__(kSmallThreads) cayley_factor_kernel(
    int p, const double *A, const double *S, const double *B, const double *O, double tau,
    double *W, double *C1, double *C2, int *status) {
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  __shared__ int s_fail;
  const int n2 = 2 * p, w = 3 * p;
  const double ht = 0.5 * tau;
  if (p == 1) {
    // x+ = x - beta1 a - beta2 x in the Y = M^{1/2} X coordinates, where
    // a^T x = E_X^T X (S), a^T a = E_X^T M^{-1} E_X (B), x^T x = X^T M X (O);
    // the denominator is 1 + (tau/2)^2 (a^T a x^T x - (a^T x)^2) >= 1
    // (Cauchy-Schwarz), so the step always exists.
    if (threadIdx.x == 0) {
      const double ax = S[0], aa = B[0], xx = O ? O[0] : 1.0;
      const double den = 1.0 + ht * ht * (aa * xx - ax * ax);
      const double beta1 = tau * xx / den;
      const double beta2 = -tau * (ax + ht * (ax * ax - aa * xx)) / den;
      if (!isfinite(beta1) || !isfinite(beta2) || !(den > 0.0)) {
        atomicCAS(status, 0, (int)KS_ESINGULAR);
        return;
      }
      C1[0] = 1.0 - beta2;               // X+ = X C1 + G C2, G = M^{-1} E_X
      C2[0] = -beta1;
    }
    return;
  }
  for (int e = threadIdx.x; e < n2 * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    double v;
    if (j < n2) {
      const int bi = i / p, bj = j / p, ii = i % p, jj = j % p;
      double nv;
      if (bi == 0 && bj == 0) nv = A[ii * p + jj];
      else if (bi == 0 && bj == 1) nv = O ? O[ii * p + jj] : (ii == jj ? 1.0 : 0.0);
      else if (bi == 1 && bj == 0) nv = -B[ii * p + jj];
      else nv = -S[ii * p + jj];
      v = (i == j ? 1.0 : 0.0) + ht * nv;
    } else {
      const int jj = j - n2, ii = i % p;
      if (i < p) v = O ? O[ii * p + jj] : (ii == jj ? 1.0 : 0.0);
      else v = -S[ii * p + jj];
    }
    W[e] = v;
  }
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < n2; ++j) {
    // pivot search over rows j..n2-1 (largest |W[i][j]|, lowest index on ties)
    double best = -1.0;
    int bi = n2;
    for (int i = j + threadIdx.x; i < n2; i += blockDim.x) {
      const double a = fabs(W[i * w + j]);
      if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = -1.0;
      int ib = n2;
      for (int t = 0; t < (int)(blockDim.x >> 5); ++t)
        if (s_val[t] > bb || (s_val[t] == bb && s_idx[t] < ib)) { bb = s_val[t]; ib = s_idx[t]; }
      if (!(bb > 1e-300) || !isfinite(bb)) {
        s_fail = 1;
        atomicCAS(status, 0, (int)KS_ESINGULAR);
      }
      s_piv = ib;
    }
    __syncthreads();
    if (s_fail) return;
    const int pv = s_piv;
    if (pv != j) {
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        const double t = W[j * w + c];
        W[j * w + c] = W[pv * w + c];
        W[pv * w + c] = t;
      }
      __syncthreads();
    }
    const double d = W[j * w + j];
    const int rows = n2 - j - 1, cols = w - j - 1;
    for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) {
      const int i = j + 1 + t / cols, c = j + 1 + t % cols;
      W[i * w + c] = fma(-W[i * w + j] / d, W[j * w + c], W[i * w + c]);
    }
    __syncthreads();
  }
  // back substitution, one right-hand side column per thread
  for (int c = threadIdx.x; c < p; c += blockDim.x) {
    const int col = n2 + c;
    for (int i = n2 - 1; i >= 0; --i) {
      double s = W[i * w + col];
      for (int k = i + 1; k < n2; ++k) s = fma(-W[i * w + k], W[k * w + col], s);
      W[i * w + col] = s / W[i * w + i];
    }
  }
  __syncthreads();
  // X+ = X (I - tau P2) + G (-tau P1)
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    const double p1 = W[i * w + n2 + j], p2 = W[(p + i) * w + n2 + j];
    C1[e] = (i == j ? 1.0 : 0.0) - tau * p2;
    C2[e] = -tau * p1;
  }
}

ks_status launch_cayley_factor(Problem &P, const double *A, const double *S, const double *B,
                               const double *O, double tau, double *C1, double *C2) {
  {
    ProfScope ps_(P.stream, KP_SMALL);
    cayley_factor_kernel<<<1, kSmallThreads, 0, P.stream>>>(P.p, A, S, B, O, tau, P.pp, C1, C2,
                                                            P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

__global__ void transpose_kernel(int p, const double *A, double *out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * p; e += gridDim.x * blockDim.x) {
    const int i = e / p, j = e % p;
    out[j * p + i] = A[e];
  }
}

ks_status launch_transpose(Problem &P, const double *A, double *out) {
  {
    ProfScope ps_(P.stream, KP_OTHER);
    transpose_kernel<<<(P.p * P.p + kThreads - 1) / kThreads, kThreads, 0, P.stream>>>(P.p, A, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

}  // namespace ks
