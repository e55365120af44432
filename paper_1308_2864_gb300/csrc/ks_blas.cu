// FP64 tall-skinny products of the iteration (Sec. 3's O(np^2) part):
//   gram:     out = A^T B (p x q Grams such as E_X^T X, D^T M D, X^T M X),
//             split over row chunks; partial tiles are summed in chunk
//             order, so the result is deterministic;
//   combine:  out = A1 C1 + A2 C2 + beta B (the retraction updates
//             X+ = X C1 + D C2 of Eq. QR / Eq. WY3 and D = G - X S).
// FP64 arithmetic is the bound of both on GB300 (n p^2 FMAs against n p
// words of traffic); tiles are 64 x 64 with a 4 x 4 register block per
// thread, strided so that shared-memory reads are conflict-free.
#include <mutex>

#include "ks_async.cuh"
#include "ks_device.cuh"
#include "ks_steps.h"

namespace ks {

// 16-byte global -> shared copy (cp.async, L2 only); src_bytes = 0 copies
// nothing and zero-fills the 16 bytes.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Tensor cores for the FP32 phase when the products are wide enough for the
// SIMT FP32 pipes to be the bound (use_tc = 1: from 256 columns; 2: always;
// 0: never).  At p = 64 the SIMT kernels are as fast as the register-staged
// tensor-core kernels, which do not yet overlap their loads deeply enough.
static bool use_tensor_cores(const Problem &P, int a, int b) {
  if (P.use_tc == 0 || a <= 8 || b <= 8) return false;
  return P.use_tc == 2 || (a >= 256 && b >= 256);
}

static int gram_chunks(const Problem &P, int pa, int qb) {
  const int tiles = ((pa + kTile - 1) / kTile) * ((qb + kTile - 1) / kTile);
  // (the small and mid kernels run one block per chunk: tiles = 1 there too)
  int chunks = (4 * P.sms + tiles - 1) / tiles;
  // at least 256 rows per chunk, so small problems do not pay for many
  // partial tiles
  const int maxc = (P.n + 255) / 256;
  if (chunks > maxc) chunks = maxc;
  if (chunks < 1) chunks = 1;
  return chunks;
}

// T = double, or float for the mixed path (FP32 products and per-chunk
// FP32 sums, chunk partials summed in FP64).
// K-values per stage of the 64-tile update: 32 in FP32 (more bytes in
// flight per thread), 16 in FP64 (FP64-pipe-bound; keeps the two stage
// buffers within the 48 KiB of static shared memory).  The Gram stages
// kTileK rows (measured faster than 32 at p = 64).
template <typename T>
__host__ __device__ constexpr int stage_k() { return sizeof(T) == 4 ? 32 : 16; }

// Vector of 4 consecutive T in shared memory (16- or 32-byte aligned).
template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 q0 = reinterpret_cast<const double2 *>(p)[0];
    const double2 q1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
}

// One 64 x 64 output tile (index `tile`, row-major over the tile grid) of
// one row chunk.  Thread (ty, tx) of 16 x 16 owns the contiguous 4 x 4 block
// a0 + 4ty + i, b0 + 4tx + j, so a row step costs two vector shared-memory
// loads for 16 FMAs; the next stage of rows is loaded into registers while
// the current one is consumed, and two shared buffers alternate (one
// barrier per stage).  Each entry is the same row-ascending FMA chain as a
// one-output-per-thread loop.
template <typename T>
__device__ __forceinline__ void gram_tile_body(long long n, int pa, int qb, long long rows_per,
                                               const T *__restrict__ A, const T *__restrict__ B,
                                               double *__restrict__ part, int tile, int chunk) {
  constexpr int SK = kTileK;
  __shared__ __align__(16) T As[2][SK][kTile];
  __shared__ __align__(16) T Bs[2][SK][kTile];
  const int tq = (qb + kTile - 1) / kTile;
  const int ta = tile / tq, tb = tile % tq;
  const long long r0 = chunk * rows_per;
  long long r1 = r0 + rows_per;
  if (r1 > n) r1 = n;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int a0 = ta * kTile, b0 = tb * kTile;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  constexpr int kPer = SK * kTile / 256;         // staged values per thread and operand
  T ra[kPer], rb[kPer];
  auto fetch = [&](long long r) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int idx = tid + t * 256;
      const int rr = idx >> 6, cc = idx & 63;
      const long long row = r + rr;
      const bool rowok = row < r1;
      ra[t] = (rowok && a0 + cc < pa) ? A[row * pa + a0 + cc] : (T)0;
      rb[t] = (rowok && b0 + cc < qb) ? B[row * qb + b0 + cc] : (T)0;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int idx = tid + t * 256;
      As[buf][idx >> 6][idx & 63] = ra[t];
      Bs[buf][idx >> 6][idx & 63] = rb[t];
    }
  };
  if (r0 < r1) {
    fetch(r0);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (long long r = r0; r < r1; r += SK, buf ^= 1) {
    const bool more = r + SK < r1;
    if (more) fetch(r + SK);
#pragma unroll
    for (int rr = 0; rr < SK; ++rr) {
      T av[4], bv[4];
      ld4(&As[buf][rr][4 * ty], av);
      ld4(&Bs[buf][rr][4 * tx], bv);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
  }
  double *dst = part + (long long)chunk * pa * qb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + 4 * ty + i;
    if (a >= pa) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + 4 * tx + j;
      if (b < qb) dst[(long long)a * qb + b] = (double)acc[i][j];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(long long n, int pa, int qb, long long rows_per,
                                                   const T *__restrict__ A,
                                                   const T *__restrict__ B,
                                                   double *__restrict__ part) {
  gram_tile_body<T>(n, pa, qb, rows_per, A, B, part, blockIdx.x, blockIdx.y);
}

// out[e] = sum over chunks of part[c * len + e]: 8 threads per output, each
// summing a strided eighth of the chunks, then a fixed butterfly (the order
// is the same on every run).
__global__ void gram_reduce_kernel(int chunks, long long len, const double *__restrict__ part,
                                   double *__restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long e = t >> 3;
  const int sub = (int)(t & 7);
  double acc = 0.0;
  if (e < len)
    for (int c = sub; c < chunks; c += 8) acc += part[(long long)c * len + e];
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  if (sub == 0 && e < len) out[e] = acc;
}

// Small Grams (pa, qb <= kSmallPQ): each thread accumulates the whole pa x qb
// outer-product sum of its rows in registers, so no arithmetic is spent on
// padding (on GB300 every wasted FP64 FMA costs as much as a useful one);
// warp butterflies then a fixed-order sum over the warps give the chunk
// partial.
constexpr int kSmallPQ = 8;

template <typename T>
__device__ __forceinline__ void gram_small_body(long long n, int pa, int qb, long long rows_per,
                                                const T *__restrict__ A, const T *__restrict__ B,
                                                double *__restrict__ part, int chunk) {
  __shared__ double red[8][kSmallPQ * kSmallPQ];
  const long long r0 = chunk * rows_per;
  long long r1 = r0 + rows_per;
  if (r1 > n) r1 = n;
  T acc[kSmallPQ][kSmallPQ];
#pragma unroll
  for (int a = 0; a < kSmallPQ; ++a)
#pragma unroll
    for (int b = 0; b < kSmallPQ; ++b) acc[a][b] = 0;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    T av[kSmallPQ], bv[kSmallPQ];
#pragma unroll
    for (int a = 0; a < kSmallPQ; ++a) av[a] = a < pa ? A[r * pa + a] : (T)0;
#pragma unroll
    for (int b = 0; b < kSmallPQ; ++b) bv[b] = b < qb ? B[r * qb + b] : (T)0;
#pragma unroll
    for (int a = 0; a < kSmallPQ; ++a) {
      if (a >= pa) break;
#pragma unroll
      for (int b = 0; b < kSmallPQ; ++b) {
        if (b >= qb) break;
        acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < kSmallPQ; ++a) {
    if (a >= pa) break;
#pragma unroll
    for (int b = 0; b < kSmallPQ; ++b) {
      if (b >= qb) break;
      double v = (double)acc[a][b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][a * kSmallPQ + b] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < pa * qb; e += blockDim.x) {
    const int a = e / qb, b = e % qb;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][a * kSmallPQ + b];
    part[(long long)chunk * pa * qb + e] = v;
  }
}

// Mid-size Grams (kSmallPQ < pa, qb <= kMidPQ): the block keeps the whole
// pa x qb result of its row chunk, one thread per output (up to four per
// thread), staging kMidRows rows of A and B in shared memory at a time.
// Threads map onto the pa qb outputs with no padding, so no FMA is spent on
// entries outside the Gram (the 64-wide tile would spend (64/p)^2 times the
// work at p = 16).
constexpr int kMidPQ = 32, kMidRows = 32;
static_assert(kMidRows * kMidPQ <= 4 * 256, "a stage is 4 values per thread of a 256-thread block");

template <typename T>
__device__ __forceinline__ void gram_mid_body(long long n, int pa, int qb, long long rows_per,
                                              const T *__restrict__ A, const T *__restrict__ B,
                                              double *__restrict__ part, int chunk) {
  __shared__ T As[kMidRows * kMidPQ];
  __shared__ T Bs[kMidRows * kMidPQ];
  const long long r0 = chunk * rows_per;
  long long r1 = r0 + rows_per;
  if (r1 > n) r1 = n;
  const int outs = pa * qb;
  int oa[4], ob[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + u * blockDim.x;
    oa[u] = e < outs ? e / qb : 0;
    ob[u] = e < outs ? e % qb : 0;
  }
  T acc[4] = {0, 0, 0, 0};
  // the next stage's values travel in registers while this stage computes
  // (256 threads x 4 cover a stage of kMidRows x kMidPQ)
  T ra[4], rb[4];
  auto fetch = [&](long long r) {
    const int rows = (int)min((long long)kMidRows, r1 - r);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      ra[u] = t < rows * pa ? A[r * pa + t] : (T)0;
      rb[u] = t < rows * qb ? B[r * qb + t] : (T)0;
    }
  };
  if (r0 < r1) fetch(r0);
  for (long long r = r0; r < r1; r += kMidRows) {
    const int rows = (int)min((long long)kMidRows, r1 - r);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = threadIdx.x + u * blockDim.x;
      if (t < rows * pa) As[t] = ra[u];
      if (t < rows * qb) Bs[t] = rb[u];
    }
    __syncthreads();
    if (r + kMidRows < r1) fetch(r + kMidRows);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (threadIdx.x + u * blockDim.x >= outs) break;
      T a = acc[u];
      for (int k = 0; k < rows; ++k) a = fma(As[k * pa + oa[u]], Bs[k * qb + ob[u]], a);
      acc[u] = a;
    }
  }
  double *dst = part + (long long)chunk * outs;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + u * blockDim.x;
    if (e < outs) dst[e] = (double)acc[u];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) gram_mid_kernel(long long n, int pa, int qb,
                                                       long long rows_per,
                                                       const T *__restrict__ A,
                                                       const T *__restrict__ B,
                                                       double *__restrict__ part) {
  gram_mid_body<T>(n, pa, qb, rows_per, A, B, part, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(256) gram_small_kernel(long long n, int pa, int qb,
                                                         long long rows_per,
                                                         const T *__restrict__ A,
                                                         const T *__restrict__ B,
                                                         double *__restrict__ part) {
  gram_small_body<T>(n, pa, qb, rows_per, A, B, part, blockIdx.x);
}

// Pipelined FP32 Grams for 32 < max(pa, qb) <= 64 and 16-byte-aligned
// operands (widths multiples of 4): persistent blocks take stages of 32 rows
// in turn (block b: stages b, b + G, ...), copied global -> shared by
// cp.async three stages ahead (columns beyond pa, qb zero-filled), and keep
// 64 x 64 FP32 tiles (4 x 4 per thread) over all their rows; each block
// writes its FP32 partial tiles, summed afterwards in FP64 in block order.
// Two forms:
//   pair   (Dual = false): out = A1^T B1 + A2^T B2 -- the rows of the second
//          pair follow those of the first (A2 null: one Gram);
//   shared (Dual = true):  out1 = A1^T B, out2 = A2^T B with B read once.
constexpr int kGaStages = 3, kGaRows = 32;

template <bool Dual>
constexpr size_t gram_ta_smem() {
  return (size_t)kGaStages * (Dual ? 3 : 2) * kGaRows * kTile * sizeof(float);
}

template <bool Dual>
__global__ void __launch_bounds__(256, Dual ? 3 : 4) gram2_ta_kernel(
    long long n, int pa, int qb, const float *__restrict__ A1, const float *__restrict__ B1,
    const float *__restrict__ A2, const float *__restrict__ B2, float *__restrict__ part) {
  extern __shared__ __align__(16) float ga_smem[];
  constexpr int kOps = Dual ? 3 : 2;                 // staged operands: A1, B (, A2)
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long nv = (!Dual && A2) ? 2 * n : n;    // rows streamed (both pairs)
  const long long nst = (nv + kGaRows - 1) / kGaRows;
  const long long W = nst > blockIdx.x ? (nst - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  auto issue = [&](long long w) {
    const long long r0 = (blockIdx.x + w * gridDim.x) * kGaRows;
    float *dst = ga_smem + (size_t)(w % kGaStages) * kOps * kGaRows * kTile;
#pragma unroll
    for (int t = 0; t < kOps * 2; ++t) {
      const int idx = tid + t * 256;               // operand, row, 4-column chunk
      const int op = idx >> 9, rr = (idx >> 4) & 31, c4 = (idx & 15) * 4;
      long long row = r0 + rr;
      const int w_ = op == 1 ? qb : pa;
      const float *M;
      if (Dual) {
        M = op == 0 ? A1 : op == 1 ? B1 : A2;
      } else if (row < n) {
        M = op == 0 ? A1 : B1;
      } else {
        M = op == 0 ? A2 : B2;
        row -= n;
      }
      const float *src = A1;
      uint32_t bytes = 0;
      if (row < n && r0 + rr < nv && c4 < w_ && KS_IN(row * w_ + c4 + 3, n * w_)) {
        src = M + row * w_ + c4;
        bytes = 16;
      }
      const int di = op * kGaRows * kTile + rr * kTile + c4;
      if (KS_IN(di + 3, kOps * kGaRows * kTile)) cp_async16(smem_addr(dst + di), src, bytes);
    }
  };
  float acc[4][4], acc2[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = acc2[i][j] = 0.f;
  for (int st = 0; st < kGaStages - 1; ++st) {
    if (st < W) issue(st);
    cp_async_commit();
  }
  for (long long w = 0; w < W; ++w) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kGaStages - 2) : "memory");
    __syncthreads();
    if (w + kGaStages - 1 < W) issue(w + kGaStages - 1);
    cp_async_commit();
    const float *As = ga_smem + (size_t)(w % kGaStages) * kOps * kGaRows * kTile;
    const float *Bs = As + kGaRows * kTile;
    const float *A2s = Bs + kGaRows * kTile;
#pragma unroll 8
    for (int r = 0; r < kGaRows; ++r) {
      const float4 av = *reinterpret_cast<const float4 *>(As + r * kTile + 4 * ty);
      const float4 bv = *reinterpret_cast<const float4 *>(Bs + r * kTile + 4 * tx);
      const float a4[4] = {av.x, av.y, av.z, av.w};
      const float b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a4[i], b4[j], acc[i][j]);
      if (Dual) {
        const float4 cv = *reinterpret_cast<const float4 *>(A2s + r * kTile + 4 * ty);
        const float c4[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc2[i][j] = fmaf(c4[i], b4[j], acc2[i][j]);
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  const long long len = (long long)pa * qb;
  float *dst = part + (long long)blockIdx.x * (Dual ? 2 : 1) * len;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = 4 * ty + i;
    if (a >= pa) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = 4 * tx + j;
      if (b >= qb) continue;
      if (!KS_IN((long long)blockIdx.x * (Dual ? 2 : 1) * len + (Dual ? len : 0) + a * qb + b,
                 (long long)gridDim.x * (Dual ? 2 : 1) * len))
        continue;
      dst[(long long)a * qb + b] = acc[i][j];
      if (Dual) dst[len + (long long)a * qb + b] = acc2[i][j];
    }
  }
}

// FP64 sums of FP32 chunk partials in chunk order: element e < len1 of each
// chunk goes to out1[e], the rest to out2[e - len1]; out32 (optional) gets
// every sum rounded to FP32 at index e.
__global__ void gram_reduce_f32_kernel(int chunks, long long len, long long len1,
                                       const float *__restrict__ part, double *__restrict__ out1,
                                       double *__restrict__ out2, float *__restrict__ out32) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long e = t >> 3;
  const int sub = (int)(t & 7);
  double acc = 0.0;
  if (e < len)
    for (int c = sub; c < chunks; c += 8) acc += (double)part[(long long)c * len + e];
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  if (sub == 0 && e < len) {
    if (e < len1) out1[e] = acc;
    else out2[e - len1] = acc;
    if (out32) out32[e] = (float)acc;
  }
}

// The pipelined Gram kernels apply: FP32, 32 < max(pa, qb) <= 64, widths
// multiples of 4 and 16-byte-aligned operands.
static bool gram_ta_applies(int pa, int qb, std::initializer_list<const float *> ops) {
  if (pa > kTile || qb > kTile || (pa <= kMidPQ && qb <= kMidPQ) || pa % 4 || qb % 4) return false;
  for (const float *A : ops)
    if (reinterpret_cast<uintptr_t>(A) % 16) return false;
  return true;
}

template <bool Dual>
static ks_status launch_gram2_ta(Problem &P, int pa, int qb, const float *A1, const float *B1,
                                 const float *A2, const float *B2, double *out1, double *out2,
                                 float *out32 = nullptr) {
  const long long nv = (!Dual && A2) ? 2 * P.n : P.n;
  const long long nst = (nv + kGaRows - 1) / kGaRows;
  long long blocks = (Dual ? 3LL : 4LL) * P.sms;
  if (blocks > nst) blocks = nst;
  const long long len = (long long)pa * qb * (Dual ? 2 : 1);
  // FP32 partials in the FP64 partial buffer
  if ((size_t)blocks * len > 2 * P.partials_len)
    return set_error(KS_EINVAL, "gram: partial buffer too small");
  float *part = reinterpret_cast<float *>(P.partials);
  {
    ProfScope ps_(P.stream, KP_GRAM, 2.0 * nv * pa * qb * (Dual ? 2 : 1),
                  (double)nv * (pa + qb + (Dual ? pa : 0)) * sizeof(float));
    gram2_ta_kernel<Dual><<<(int)blocks, 256, gram_ta_smem<Dual>(), P.stream>>>(
        P.n, pa, qb, A1, B1, A2, B2, part);
  }
  KS_CUDA_TRY(cudaGetLastError());
  {
    ProfScope ps_(P.stream, KP_REDUCE);
    gram_reduce_f32_kernel<<<(int)((8 * len + kThreads - 1) / kThreads), kThreads, 0, P.stream>>>(
        (int)blocks, len, (long long)pa * qb, part, out1, out2, out32);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template <typename T>
ks_status launch_gram(Problem &P, const T *A, int pa, const T *B, int qb, double *out) {
  if (sizeof(T) == 8 && P.use_oz > 0 && pa + qb <= P.oz_emax_len &&
      (P.use_oz == 2 || (pa >= 48 && qb >= 48))) {
    // FP64: digit-split products on the tensor cores, FP64 chunk partials
    const int chunks = gram_oz_chunks(P, pa, qb);
    if ((size_t)chunks * pa * qb > P.partials_len)
      return set_error(KS_EINVAL, "gram: partial buffer too small");
    KS_TRY(launch_gram_oz(P, (const double *)A, pa, (const double *)B, qb, P.oz_emax, P.partials,
                          chunks));
    const long long len = (long long)pa * qb;
    {
      ProfScope ps_(P.stream, KP_REDUCE);
      gram_reduce_kernel<<<(int)((8 * len + kThreads - 1) / kThreads), kThreads, 0, P.stream>>>(
          chunks, len, P.partials, out);
    }
    KS_CUDA_TRY(cudaGetLastError());
    return KS_OK;
  }
  if (sizeof(T) == 4 && use_tensor_cores(P, pa, qb)) {
    // FP32 phase: tensor cores (3 x TF32), FP64 chunk partials
    const int chunks = gram_tc_chunks(P, pa, qb);
    if ((size_t)chunks * pa * qb > P.partials_len)
      return set_error(KS_EINVAL, "gram: partial buffer too small");
    KS_TRY(launch_gram_tc(P, (const float *)A, pa, (const float *)B, qb, P.partials, chunks));
    const long long len = (long long)pa * qb;
    {
      ProfScope ps_(P.stream, KP_REDUCE);
      gram_reduce_kernel<<<(int)((8 * len + kThreads - 1) / kThreads), kThreads, 0, P.stream>>>(
          chunks, len, P.partials, out);
    }
    KS_CUDA_TRY(cudaGetLastError());
    return KS_OK;
  }
  if (sizeof(T) == 4 && gram_ta_applies(pa, qb, {(const float *)A, (const float *)B}))
    return launch_gram2_ta<false>(P, pa, qb, (const float *)A, (const float *)B, nullptr, nullptr,
                                  out, nullptr);
  const int chunks = gram_chunks(P, pa, qb);
  long long rows_per = (P.n + chunks - 1) / chunks;
  rows_per = (rows_per + kTileK - 1) / kTileK * kTileK;
  const int tiles = ((pa + kTile - 1) / kTile) * ((qb + kTile - 1) / kTile);
  const size_t need = (size_t)chunks * pa * qb;
  if (need > P.partials_len)
    return set_error(KS_EINVAL, "gram: partial buffer too small (%zu > %zu)", need, P.partials_len);
  {
    ProfScope ps_(P.stream, KP_GRAM, 2.0 * P.n * pa * qb, (double)P.n * (pa + qb) * sizeof(T));
    if (pa <= kSmallPQ && qb <= kSmallPQ)
      gram_small_kernel<T><<<chunks, 256, 0, P.stream>>>(P.n, pa, qb, rows_per, A, B, P.partials);
    else if (pa <= kMidPQ && qb <= kMidPQ)
      gram_mid_kernel<T><<<chunks, 256, 0, P.stream>>>(P.n, pa, qb, rows_per, A, B, P.partials);
    else
      gram_kernel<T><<<dim3(tiles, chunks), 256, 0, P.stream>>>(P.n, pa, qb, rows_per, A, B,
                                                                P.partials);
  }
  KS_CUDA_TRY(cudaGetLastError());
  const long long len = (long long)pa * qb;
  {
    ProfScope ps_(P.stream, KP_REDUCE);
    gram_reduce_kernel<<<(int)((8 * len + kThreads - 1) / kThreads), kThreads, 0, P.stream>>>(
        chunks, len, P.partials, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_gram_pair(Problem &P, const float *A1, const float *B1, const float *A2,
                           const float *B2, int pa, int qb, double *out, double *tmp) {
  if (gram_ta_applies(pa, qb, {A1, B1, A2, B2}))
    return launch_gram2_ta<false>(P, pa, qb, A1, B1, A2, B2, out, nullptr, nullptr);
  KS_TRY(launch_gram<float>(P, A1, pa, B1, qb, out));
  KS_TRY(launch_gram<float>(P, A2, pa, B2, qb, tmp));
  return launch_add_pp(P, out, 1.0, tmp, out);
}

// FP32 copies of two p x p FP64 matrices, one after the other.
__global__ void pair_to_f32_kernel(long long len, const double *__restrict__ a,
                                   const double *__restrict__ b, float *__restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) out[e] = (float)a[e];
  else if (e < 2 * len) out[e] = (float)b[e - len];
}

ks_status launch_gram_dual(Problem &P, const float *A1, const float *A2, const float *B, int pa,
                           int qb, double *out1, double *out2, float *out32) {
  if (gram_ta_applies(pa, qb, {A1, A2, B}))
    return launch_gram2_ta<true>(P, pa, qb, A1, B, A2, nullptr, out1, out2, out32);
  KS_TRY(launch_gram<float>(P, A1, pa, B, qb, out1));
  KS_TRY(launch_gram<float>(P, A2, pa, B, qb, out2));
  if (out32) {
    const long long len = (long long)pa * qb;
    {
      ProfScope ps_(P.stream, KP_REDUCE);
      pair_to_f32_kernel<<<(int)((2 * len + kThreads - 1) / kThreads), kThreads, 0, P.stream>>>(
          len, out1, out2, out32);
    }
    KS_CUDA_TRY(cudaGetLastError());
  }
  return KS_OK;
}

// TC is the type of the coefficients C1, C2: double, or float copies made
// once per update for the FP32 phase (converting in every block would put
// a conversion per staged element on the FP64 pipe).
// One 64 x 64 output tile: thread (ty, tx) owns rows r0 + 4ty + i and
// columns c0 + 4tx + j.  The A slice is stored transposed (K-rows of 64
// rows, padded to keep the vector loads aligned) and the C slice as is, so a
// K-step costs two vector loads for 16 FMAs; stages of K-values run over
// A1 C1 then A2 C2, the next one loaded into registers while the current
// one is consumed (two shared buffers, one barrier per stage).  Each entry
// is the same K-ascending FMA chain as before.
constexpr int kAtLd = kTile + 4;

template <typename T, typename TC>
__device__ __forceinline__ void combine_tile_body(long long n, int q, const T *__restrict__ A1,
                                                  int k1, const TC *__restrict__ C1,
                                                  const T *__restrict__ A2, int k2,
                                                  const TC *__restrict__ C2, double alpha_d,
                                                  double beta_d, const T *__restrict__ Bm,
                                                  T *__restrict__ out, int bx, int by) {
  constexpr int SK = stage_k<T>();
  __shared__ __align__(16) T At[2][SK][kAtLd];
  __shared__ __align__(16) T Cs[2][SK][kTile];
  const T alpha = (T)alpha_d, beta = (T)beta_d;
  const long long r0 = (long long)bx * kTile;
  const int c0 = by * kTile;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  const int s1 = (k1 + SK - 1) / SK;
  const int s2 = A2 ? (k2 + SK - 1) / SK : 0;
  const int stages = s1 + s2;
  constexpr int kPer = SK * kTile / 256;         // staged values per thread and operand
  T ra[kPer], rc[kPer];
  auto fetch = [&](int s) {
    const bool first = s < s1;
    const T *A = first ? A1 : A2;
    const TC *C = first ? C1 : C2;
    const int kk = first ? k1 : k2;
    const int k0 = (first ? s : s - s1) * SK;
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int idx = tid + t * 256;
      const int rr = idx / SK, cc = idx % SK;              // A slice: 64 rows x SK
      const long long row = r0 + rr;
      ra[t] = (row < n && k0 + cc < kk) ? A[row * kk + k0 + cc] : (T)0;
      const int cr = idx >> 6, ccol = idx & 63;            // C slice: SK x 64
      rc[t] = (k0 + cr < kk && c0 + ccol < q) ? (T)C[(long long)(k0 + cr) * q + c0 + ccol] : (T)0;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int idx = tid + t * 256;
      At[buf][idx % SK][idx / SK] = ra[t];
      Cs[buf][idx >> 6][idx & 63] = rc[t];
    }
  };
  if (stages > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  for (int s = 0; s < stages; ++s) {
    const int buf = s & 1;
    const bool more = s + 1 < stages;
    if (more) fetch(s + 1);
#pragma unroll
    for (int t = 0; t < SK; ++t) {
      T av[4], cv[4];
      ld4(&At[buf][t][4 * ty], av);
      ld4(&Cs[buf][t][4 * tx], cv);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], cv[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long row = r0 + 4 * ty + i;
    if (row >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + 4 * tx + j;
      if (col >= q) continue;
      T v = alpha * acc[i][j];
      if (Bm) v = fma(beta, Bm[row * q + col], v);
      out[row * q + col] = v;
    }
  }
}

template <typename T, typename TC>
__global__ void __launch_bounds__(256) combine_kernel(long long n, int q, const T *__restrict__ A1,
                                                      int k1, const TC *__restrict__ C1,
                                                      const T *__restrict__ A2, int k2,
                                                      const TC *__restrict__ C2, double alpha_d,
                                                      double beta_d,
                                                      const T *__restrict__ Bm,
                                                      T *__restrict__ out) {
  combine_tile_body<T, TC>(n, q, A1, k1, C1, A2, k2, C2, alpha_d, beta_d, Bm, out, blockIdx.x,
                           blockIdx.y);
}

// Narrow updates (q <= kNarrowQ): one thread per output entry, the small
// C matrices in shared memory, no padded arithmetic.
constexpr int kNarrowQ = 32;
constexpr int kNarrowK = 2 * kNarrowQ;
constexpr int kNarrowCols = 4;                     // output columns per thread

template <typename T>
__device__ __forceinline__ void combine_narrow_body(
    long long n, int q, const T *__restrict__ A1, int k1, const double *__restrict__ C1,
    const T *__restrict__ A2, int k2, const double *__restrict__ C2, double alpha_d,
    double beta_d, const T *__restrict__ Bm, T *__restrict__ out, int vb, int vnb) {
  __shared__ T Cs[2][kNarrowK * kNarrowQ];
  for (int e = threadIdx.x; e < k1 * q; e += blockDim.x) Cs[0][e] = (T)C1[e];
  if (A2)
    for (int e = threadIdx.x; e < k2 * q; e += blockDim.x) Cs[1][e] = (T)C2[e];
  __syncthreads();
  const T alpha = (T)alpha_d, beta = (T)beta_d;
  // a thread takes kNarrowCols consecutive columns of one row, so each value
  // of the row of A is loaded once for kNarrowCols FMAs (each output's FMA
  // chain runs over k in ascending order, as with one output per thread)
  const int ncg = (q + kNarrowCols - 1) / kNarrowCols;
  const long long total = n * ncg;
  for (long long e = (long long)vb * blockDim.x + threadIdx.x; e < total;
       e += (long long)vnb * blockDim.x) {
    const long long row = e / ncg;
    const int col0 = (int)(e - row * ncg) * kNarrowCols;
    const int nc = q - col0 < kNarrowCols ? q - col0 : kNarrowCols;
    T acc[kNarrowCols];
#pragma unroll
    for (int u = 0; u < kNarrowCols; ++u) acc[u] = 0;
    const T *a1 = A1 + row * k1;
    for (int k = 0; k < k1; ++k) {
      const T a = a1[k];
#pragma unroll
      for (int u = 0; u < kNarrowCols; ++u)
        if (u < nc) acc[u] = fma(a, Cs[0][k * q + col0 + u], acc[u]);
    }
    if (A2) {
      const T *a2 = A2 + row * k2;
      for (int k = 0; k < k2; ++k) {
        const T a = a2[k];
#pragma unroll
        for (int u = 0; u < kNarrowCols; ++u)
          if (u < nc) acc[u] = fma(a, Cs[1][k * q + col0 + u], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kNarrowCols; ++u) {
      if (u >= nc) break;
      const long long o = row * q + col0 + u;
      T v = alpha * acc[u];
      if (Bm) v = fma(beta, Bm[o], v);
      out[o] = v;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) combine_narrow_kernel(
    long long n, int q, const T *__restrict__ A1, int k1, const double *__restrict__ C1,
    const T *__restrict__ A2, int k2, const double *__restrict__ C2, double alpha_d,
    double beta_d, const T *__restrict__ Bm, T *__restrict__ out) {
  combine_narrow_body<T>(n, q, A1, k1, C1, A2, k2, C2, alpha_d, beta_d, Bm, out, blockIdx.x,
                         gridDim.x);
}

// Tall-skinny FP32 update, q <= 64 output columns and K = k1 + k2 + k3 <= 192
// (the retraction and projection updates of the FP32 phase at p <= 64):
// persistent blocks keep the whole coefficient matrix [C1; C2] (K x 64, zero
// padded) in shared memory for the life of the block and stream row tiles
// of 128 rows of [A1, A2] through a double-buffered stage of 32 K-values,
// the next stage (of this tile or of the block's next tile) loaded into
// registers while the current one is consumed.  Thread (ty, tx) of 16 x 16
// owns rows 8 ty .. 8 ty + 7 and columns 4 tx .. 4 tx + 3 of a tile: 32 FMAs
// per three vector shared-memory loads.  Each output is the same K-ascending
// FMA chain (A1 C1, then A2 C2) and the same final alpha/beta step as
// combine_tile_body, so the two kernels give bitwise-equal results for two
// blocks.  A third block (A3 C3) and a second output out2 = add2 + out
// serve the increment form's retraction in one pass.
constexpr int kTsRows = 128, kTsK = 32, kTsMaxK = 192, kTsLd = kTsRows + 4;

size_t combine_ts_smem(int K) {
  const int nst = (K + kTsK - 1) / kTsK;
  return ((size_t)nst * kTsK * kTile + (size_t)2 * kTsK * kTsLd) * sizeof(float);
}

// Optional outputs of the tall-skinny update's epilogue: the density of the
// new iterate (rho set) and whether every array allows 16-byte accesses.
struct TsDensity {
  const double *rho_b = nullptr;
  double *rho = nullptr;
  double occ = 0.0;
  int vec = 0;
};

// Epilogue of the tall-skinny update for one thread's 8 rows (row0 ..
// row0 + 7) x 4 columns (4 tx .. 4 tx + 3): out = alpha acc + beta Bm and
// out2 = add2 + out, 16-byte accesses when the four columns are in range and
// every array is 16-byte aligned.  With dn.rho set (out2 the FP32 copy of
// X_b + delta, add2 = X_b, out = delta) it also forms the density of the
// new iterate in the increment form, rho = rho_b + f sum delta (2 X_b +
// delta) (Sec. 2.3, rho = diag(X X^T) per occupied orbital): the 16 threads
// of a row (the lanes tx of one half-warp) sum their columns by a butterfly.
// The accumulators are cleared for the next tile.
__device__ __forceinline__ void ts_epilogue(long long n, int q, long long row0, int tx,
                                            float (&acc)[8][4], float alpha, float beta,
                                            const float *__restrict__ Bm, float *__restrict__ out,
                                            const float *__restrict__ add2,
                                            float *__restrict__ out2, const TsDensity &dn) {
  const int col0 = 4 * tx;
  const bool vec = dn.vec && col0 + 3 < q;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long row = row0 + i;
    float dsum = 0.f;
    if (row < n) {
      const long long o = row * q + col0;
      if (vec && KS_IN(o + 3, n * q)) {
        float4 v = make_float4(alpha * acc[i][0], alpha * acc[i][1], alpha * acc[i][2],
                               alpha * acc[i][3]);
        if (Bm) {
          const float4 b = *reinterpret_cast<const float4 *>(Bm + o);
          v.x = fmaf(beta, b.x, v.x); v.y = fmaf(beta, b.y, v.y);
          v.z = fmaf(beta, b.z, v.z); v.w = fmaf(beta, b.w, v.w);
        }
        *reinterpret_cast<float4 *>(out + o) = v;
        if (out2) {
          const float4 h = *reinterpret_cast<const float4 *>(add2 + o);
          *reinterpret_cast<float4 *>(out2 + o) =
              make_float4(h.x + v.x, h.y + v.y, h.z + v.z, h.w + v.w);
          if (dn.rho) {
            dsum = fmaf(v.x, fmaf(2.f, h.x, v.x), dsum);
            dsum = fmaf(v.y, fmaf(2.f, h.y, v.y), dsum);
            dsum = fmaf(v.z, fmaf(2.f, h.z, v.z), dsum);
            dsum = fmaf(v.w, fmaf(2.f, h.w, v.w), dsum);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (col0 + j < q && KS_IN(o + j, n * q)) {
            float v = alpha * acc[i][j];
            if (Bm) v = fmaf(beta, Bm[o + j], v);
            out[o + j] = v;
            if (out2) {
              const float h = add2[o + j];
              out2[o + j] = h + v;
              if (dn.rho) dsum = fmaf(v, fmaf(2.f, h, v), dsum);
            }
          }
        }
      }
    }
    if (dn.rho) {
#pragma unroll
      for (int s = 8; s > 0; s >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, s);
      if (tx == 0 && row < n) dn.rho[row] = dn.rho_b[row] + dn.occ * (double)dsum;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  }
}

__global__ void __launch_bounds__(256, 2) combine_ts_kernel(
    long long n, int q, const float *__restrict__ A1, int k1, const float *__restrict__ c1,
    const float *__restrict__ A2, int k2, const float *__restrict__ c2,
    const float *__restrict__ A3, int k3, const float *__restrict__ c3, float alpha, float beta,
    const float *__restrict__ Bm, float *__restrict__ out, const float *__restrict__ add2,
    float *__restrict__ out2, long long ntiles, TsDensity dn) {
  extern __shared__ __align__(16) float ts_smem[];
  const int k12 = k1 + (A2 ? k2 : 0);
  const int K = k12 + (A3 ? k3 : 0);
  const int nst = (K + kTsK - 1) / kTsK;
  float *Cs = ts_smem;                              // [nst * kTsK][64]
  float *As = ts_smem + (size_t)nst * kTsK * kTile;  // [2][kTsK][kTsLd]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int e = tid; e < nst * kTsK * kTile; e += 256) {
    const int r = e / kTile, c = e % kTile;
    float v = 0.f;
    if (c < q) {
      if (r < k1) v = c1[(long long)r * q + c];
      else if (r < k12) v = c2[(long long)(r - k1) * q + c];
      else if (r < K) v = c3[(long long)(r - k12) * q + c];
    }
    Cs[e] = v;
  }
  const long long mine = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long W = mine * nst;                   // (tile, stage) steps of this block
  constexpr int kPer = kTsRows * kTsK / 256;       // staged A values per thread
  float ra[kPer];
  auto fetch = [&](long long w) {
    const long long tile = blockIdx.x + (w / nst) * gridDim.x;
    const int k0 = (int)(w % nst) * kTsK;
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int idx = tid + t * 256;
      const int rr = idx / kTsK, kk = idx % kTsK;
      const long long row = tile * kTsRows + rr;
      const int k = k0 + kk;
      float v = 0.f;
      if (row < n) {
        if (k < k1) v = A1[row * k1 + k];
        else if (k < k12) v = A2[row * k2 + (k - k1)];
        else if (k < K) v = A3[row * k3 + (k - k12)];
      }
      ra[t] = v;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int idx = tid + t * 256;
      As[((size_t)buf * kTsK + idx % kTsK) * kTsLd + idx / kTsK] = ra[t];
    }
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  if (W > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  for (long long w = 0; w < W; ++w) {
    const int buf = (int)(w & 1);
    const bool more = w + 1 < W;
    if (more) fetch(w + 1);
    const int k0 = (int)(w % nst) * kTsK;
    const float *Ab = As + (size_t)buf * kTsK * kTsLd;
#pragma unroll 8
    for (int k = 0; k < kTsK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(Ab + k * kTsLd + 8 * ty);
      const float4 a1 = *reinterpret_cast<const float4 *>(Ab + k * kTsLd + 8 * ty + 4);
      const float4 cv = *reinterpret_cast<const float4 *>(Cs + (size_t)(k0 + k) * kTile + 4 * tx);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], cc[j], acc[i][j]);
    }
    if (w % nst == nst - 1) {
      const long long tile = blockIdx.x + (w / nst) * gridDim.x;
      ts_epilogue(n, q, tile * kTsRows + 8 * ty, tx, acc, alpha, beta, Bm, out, add2, out2, dn);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
  }
}

static void launch_ts(Problem &P, int q, const float *A1, int k1, const float *c1,
                      const float *A2, int k2, const float *c2, const float *A3, int k3,
                      const float *c3, float alpha, float beta, const float *Bm, float *out,
                      const float *add2, float *out2, TsDensity dn = TsDensity());

// FP32 copies of the update coefficients (one launch for both matrices).
__global__ void coef_convert_kernel(long long len1, const double *__restrict__ C1,
                                    float *__restrict__ c1, long long len2,
                                    const double *__restrict__ C2, float *__restrict__ c2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len1) c1[e] = (float)C1[e];
  else if (e < len1 + len2) c2[e - len1] = (float)C2[e - len1];
}

template <typename T>
ks_status launch_combine(Problem &P, const T *A1, int k1, const double *C1, const T *A2, int k2,
                         const double *C2, double alpha, double beta, const T *Bm, T *out, int q) {
  if (sizeof(T) == 8 && combine_oz_applies(P, k1, A2 ? k2 : 0, q))
    return launch_combine_oz(P, (const double *)A1, k1, C1, (const double *)A2, k2, C2, alpha,
                             beta, (const double *)Bm, (double *)out, q);
  if (sizeof(T) == 4 && q > kNarrowQ && use_tensor_cores(P, k1, q))
    return launch_combine_tc(P, (const float *)A1, k1, C1, (const float *)A2, k2, C2, alpha, beta,
                             (const float *)Bm, (float *)out, q);
  if (q <= kNarrowQ && k1 <= kNarrowK && (!A2 || k2 <= kNarrowK)) {
    const long long total = (long long)P.n * ((q + kNarrowCols - 1) / kNarrowCols);
    long long nb = (total + 255) / 256;
    if (nb > 32LL * P.sms) nb = 32LL * P.sms;
    {
      ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * (k1 + (A2 ? k2 : 0)),
                    (double)P.n * ((k1 + (A2 ? k2 : 0)) + q * (Bm ? 2 : 1)) * sizeof(T));
      combine_narrow_kernel<T><<<(int)nb, 256, 0, P.stream>>>(P.n, q, A1, k1, C1, A2, k2, C2,
                                                              alpha, beta, Bm, out);
    }
    KS_CUDA_TRY(cudaGetLastError());
    return KS_OK;
  }
  dim3 grid((unsigned)((P.n + kTile - 1) / kTile), (unsigned)((q + kTile - 1) / kTile));
  if (sizeof(T) == 4) {
    float *c1 = P.cf, *c2 = P.cf + (size_t)P.p * P.p;
    const long long len1 = (long long)k1 * q, len2 = A2 ? (long long)k2 * q : 0;
    {
      ProfScope ps_(P.stream, KP_REDUCE);
      coef_convert_kernel<<<(int)((len1 + len2 + 255) / 256), 256, 0, P.stream>>>(
          len1, C1, c1, len2, C2, c2);
    }
    KS_CUDA_TRY(cudaGetLastError());
    const int K = k1 + (A2 ? k2 : 0);
    // tensor cores: beta Bm enters as a third operand with the coefficient
    // beta I, alpha scales the other coefficients
    if (combine_tc64_applies(P, q, {k1, A2 ? k2 : 0, Bm ? q : 0}, {A1, A2, Bm, out}))
      return launch_combine_tc64(P, q, (const float *)A1, k1, c1, (float)alpha,
                                 (const float *)A2, k2, A2 ? c2 : nullptr, (float)alpha,
                                 (const float *)Bm, q, nullptr, (float)beta, (float *)out,
                                 nullptr, nullptr, nullptr);
    if (q <= kTile && K <= kTsMaxK) {
      ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * K,
                    (double)P.n * (K + q * (Bm ? 2 : 1)) * sizeof(T));
      launch_ts(P, q, (const float *)A1, k1, c1, (const float *)A2, k2, A2 ? c2 : nullptr, nullptr,
                0, nullptr, (float)alpha, (float)beta, (const float *)Bm, (float *)out, nullptr,
                nullptr);
      KS_CUDA_TRY(cudaGetLastError());
      return KS_OK;
    }
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * (k1 + (A2 ? k2 : 0)),
                  (double)P.n * ((k1 + (A2 ? k2 : 0)) + q * (Bm ? 2 : 1)) * sizeof(T));
    combine_kernel<T, float><<<grid, 256, 0, P.stream>>>(P.n, q, A1, k1, c1, A2, k2,
                                                         A2 ? c2 : nullptr, alpha, beta, Bm, out);
  } else {
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * (k1 + (A2 ? k2 : 0)),
                  (double)P.n * ((k1 + (A2 ? k2 : 0)) + q * (Bm ? 2 : 1)) * sizeof(T));
    combine_kernel<T, double><<<grid, 256, 0, P.stream>>>(P.n, q, A1, k1, C1, A2, k2, C2, alpha,
                                                          beta, Bm, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// ---------------------------------------------------------------- batched
// Grams of every active job: tiles x chunks blocks per job (64-tile kernel)
// or chunks blocks (p <= kSmallPQ), then the chunk sums into pp + smOut p^2.
template <typename T>
__global__ void __launch_bounds__(256) gram_batch_kernel(const BJob *__restrict__ jobs,
                                                         const int *__restrict__ start, int J,
                                                         const unsigned char *__restrict__ active,
                                                         int sA, int sB, int small) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const int vb = blockIdx.x - start[j];
  const T *A = (const T *)b.blk[sA], *Bp = (const T *)b.blk[sB];
  if (small == 1) {
    gram_small_body<T>(b.n, b.p, b.p, b.gram_rows_per, A, Bp, b.partials, vb);
  } else if (small == 2) {
    gram_mid_body<T>(b.n, b.p, b.p, b.gram_rows_per, A, Bp, b.partials, vb);
  } else {
    const int tiles = ((b.p + kTile - 1) / kTile) * ((b.p + kTile - 1) / kTile);
    gram_tile_body<T>(b.n, b.p, b.p, b.gram_rows_per, A, Bp, b.partials, vb % tiles, vb / tiles);
  }
}

__global__ void gram_reduce_batch_kernel(const BJob *__restrict__ jobs,
                                         const int *__restrict__ start, int J,
                                         const unsigned char *__restrict__ active, int smOut) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const long long t = (long long)(blockIdx.x - start[j]) * blockDim.x + threadIdx.x;
  const long long len = (long long)b.p * b.p;
  const long long e = t >> 3;
  const int sub = (int)(t & 7);
  double acc = 0.0;
  if (e < len)
    for (int c = sub; c < b.gram_chunks; c += 8) acc += b.partials[(long long)c * len + e];
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  if (sub == 0 && e < len) b.pp[(size_t)smOut * len + e] = acc;
}

template <typename T>
ks_status batch_gram(Batch &B, int sA, int sB, int smOut) {
  for (int small = 2; small >= 0; --small) {
    const int m = small == 2 ? BM_GRAM_MID : small == 1 ? BM_GRAM_SMALL : BM_GRAM_TILED;
    const int nb = B.total(m);
    if (nb == 0) continue;
    {
      ProfScope ps_(B.stream, KP_GRAM);
      gram_batch_kernel<T><<<nb, 256, 0, B.stream>>>(B.jobs_dev, B.map(m), B.J, B.active_dev, sA,
                                                     sB, small);
    }
    KS_CUDA_TRY(cudaGetLastError());
  }
  const int nr = B.total(BM_GRAM_REDUCE);
  {
    ProfScope ps_(B.stream, KP_REDUCE);
    gram_reduce_batch_kernel<<<nr, kThreads, 0, B.stream>>>(B.jobs_dev, B.map(BM_GRAM_REDUCE), B.J,
                                                            B.active_dev, smOut);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// out = alpha (A1 C1 + A2 C2) + beta Bm with q = k1 = k2 = p per job; C from
// pp (FP64; the 64-tile form of the FP32 phase reads the FP32 copies that
// coef_batch_kernel leaves in cf).
struct CombSlots {
  int a1, c1, a2, c2, bm, out;
  double alpha, beta;
};

__global__ void coef_batch_kernel(const BJob *__restrict__ jobs, const int *__restrict__ start,
                                  int J, const unsigned char *__restrict__ active, int smC1,
                                  int smC2) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const long long len = (long long)b.p * b.p;
  const long long e = (long long)(blockIdx.x - start[j]) * blockDim.x + threadIdx.x;
  if (e < len) b.cf[e] = (float)b.pp[(size_t)smC1 * len + e];
  else if (smC2 >= 0 && e < 2 * len) b.cf[e] = (float)b.pp[(size_t)smC2 * len + e - len];
}

template <typename T>
__global__ void __launch_bounds__(256) combine_batch_kernel(const BJob *__restrict__ jobs,
                                                            const int *__restrict__ start, int J,
                                                            const unsigned char *__restrict__ active,
                                                            CombSlots sl, int narrow) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const int p = b.p;
  const long long len = (long long)p * p;
  const int vb = blockIdx.x - start[j];
  const T *A1 = (const T *)b.blk[sl.a1];
  const T *A2 = sl.a2 >= 0 ? (const T *)b.blk[sl.a2] : nullptr;
  const T *Bm = sl.bm >= 0 ? (const T *)b.blk[sl.bm] : nullptr;
  T *out = (T *)b.blk[sl.out];
  const double *C1 = b.pp + (size_t)sl.c1 * len;
  const double *C2 = sl.c2 >= 0 ? b.pp + (size_t)sl.c2 * len : nullptr;
  if (narrow) {
    combine_narrow_body<T>(b.n, p, A1, p, C1, A2, p, C2, sl.alpha, sl.beta, Bm, out, vb,
                           b.comb_nb);
  } else {
    const int ct = (p + kTile - 1) / kTile;
    if (sizeof(T) == 4)
      combine_tile_body<T, float>(b.n, p, A1, p, b.cf, A2, p, C2 ? b.cf + len : nullptr,
                                  sl.alpha, sl.beta, Bm, out, vb / ct, vb % ct);
    else
      combine_tile_body<T, double>(b.n, p, A1, p, C1, A2, p, C2, sl.alpha, sl.beta, Bm, out,
                                   vb / ct, vb % ct);
  }
}

template <typename T>
ks_status batch_combine(Batch &B, int sA1, int smC1, int sA2, int smC2, double alpha, double beta,
                        int sBm, int sOut) {
  const CombSlots sl{sA1, smC1, sA2, smC2, sBm, sOut, alpha, beta};
  const int nt = B.total(BM_COMB_TILED);
  if (sizeof(T) == 4 && nt > 0) {
    {
      ProfScope ps_(B.stream, KP_REDUCE);
      coef_batch_kernel<<<B.total(BM_COEF), kThreads, 0, B.stream>>>(
          B.jobs_dev, B.map(BM_COEF), B.J, B.active_dev, smC1, sA2 >= 0 ? smC2 : -1);
    }
    KS_CUDA_TRY(cudaGetLastError());
  }
  for (int narrow = 1; narrow >= 0; --narrow) {
    const int m = narrow ? BM_COMB_NARROW : BM_COMB_TILED;
    const int nb = B.total(m);
    if (nb == 0) continue;
    {
      ProfScope ps_(B.stream, KP_COMBINE);
      combine_batch_kernel<T><<<nb, 256, 0, B.stream>>>(B.jobs_dev, B.map(m), B.J, B.active_dev,
                                                        sl, narrow);
    }
    KS_CUDA_TRY(cudaGetLastError());
  }
  return KS_OK;
}

// Precision conversion / copy of a block of every active job.
template <typename A, typename Bt>
__global__ void convert_batch_kernel(const BJob *__restrict__ jobs, const int *__restrict__ start,
                                     int J, const unsigned char *__restrict__ active, int sIn,
                                     int sOut) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  const long long total = b.n * b.p;
  const A *in = (const A *)b.blk[sIn];
  Bt *out = (Bt *)b.blk[sOut];
  const long long base = (long long)(blockIdx.x - start[j]) * blockDim.x * 4 + threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long e = base + (long long)u * blockDim.x;
    if (e < total) out[e] = (Bt)in[e];
  }
}

template <typename Tin, typename Tout>
ks_status batch_convert(Batch &B, int sIn, int sOut) {
  {
    ProfScope ps_(B.stream, KP_OTHER);
    convert_batch_kernel<Tin, Tout><<<B.total(BM_COPY), kThreads, 0, B.stream>>>(
        B.jobs_dev, B.map(BM_COPY), B.J, B.active_dev, sIn, sOut);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// ||O - I||_F^2 of every active job into its scalar row.
__global__ void ortho_err_batch_kernel(const BJob *__restrict__ jobs,
                                       const unsigned char *__restrict__ active, int smO) {
  const int j = blockIdx.x;
  if (!active[j]) return;
  const BJob &b = jobs[j];
  __shared__ double smem[33];
  const int p = b.p;
  const double *O = b.pp + (size_t)smO * p * p;
  double acc = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, k = e % p;
    const double d = O[e] - (i == k ? 1.0 : 0.0);
    acc = fma(d, d, acc);
  }
  const double s = block_sum(acc, smem);
  if (threadIdx.x == 0) b.scal[SC_ORTHO] = s;
}

ks_status batch_ortho_err(Batch &B, int smO) {
  {
    ProfScope ps_(B.stream, KP_REDUCE);
    ortho_err_batch_kernel<<<B.J, kThreads, 0, B.stream>>>(B.jobs_dev, B.active_dev, smO);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template ks_status batch_gram<double>(Batch &, int, int, int);
template ks_status batch_gram<float>(Batch &, int, int, int);
template ks_status batch_combine<double>(Batch &, int, int, int, int, double, double, int, int);
template ks_status batch_combine<float>(Batch &, int, int, int, int, double, double, int, int);
template ks_status batch_convert<double, float>(Batch &, int, int);
template ks_status batch_convert<float, double>(Batch &, int, int);
template ks_status batch_convert<double, double>(Batch &, int, int);
template ks_status batch_convert<float, float>(Batch &, int, int);

template ks_status launch_gram<double>(Problem &, const double *, int, const double *, int,
                                       double *);
template ks_status launch_gram<float>(Problem &, const float *, int, const float *, int, double *);
// Pipelined form of combine_ts_kernel for 16-byte-aligned operands (every k
// a multiple of 4 and every A base 16-byte aligned): the A stages are copied
// global -> shared by cp.async (16 bytes per copy, zero-filled past the last
// row and past K) three stages ahead, row-major with a 4-float pad, so no
// registers hold staged data and three stages of loads are in flight per
// block.  A thread reads, per 4 K-values, one float4 of each of its 8 rows
// and one float4 of C per K-value: 128 FMAs per 12 vector loads.  The FMA
// chains and the final step are those of combine_ts_kernel (K ascending).
constexpr int kTaStages = 3, kTaLd = kTsK + 4;

size_t combine_ta_smem(int K) {
  const int nst = (K + kTsK - 1) / kTsK;
  return ((size_t)nst * kTsK * kTile + (size_t)kTaStages * kTsRows * kTaLd) * sizeof(float);
}


__global__ void __launch_bounds__(256, 2) combine_ta_kernel(
    long long n, int q, const float *__restrict__ A1, int k1, const float *__restrict__ c1,
    const float *__restrict__ A2, int k2, const float *__restrict__ c2,
    const float *__restrict__ A3, int k3, const float *__restrict__ c3, float alpha, float beta,
    const float *__restrict__ Bm, float *__restrict__ out, const float *__restrict__ add2,
    float *__restrict__ out2, long long ntiles, TsDensity dn) {
  extern __shared__ __align__(16) float ta_smem[];
  const int k12 = k1 + (A2 ? k2 : 0);
  const int K = k12 + (A3 ? k3 : 0);
  const int nst = (K + kTsK - 1) / kTsK;
  float *Cs = ta_smem;                                  // [nst * kTsK][64]
  float *As = ta_smem + (size_t)nst * kTsK * kTile;     // [kTaStages][kTsRows][kTaLd]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int e = tid; e < nst * kTsK * kTile; e += 256) {
    const int r = e / kTile, c = e % kTile;
    float v = 0.f;
    if (c < q) {
      if (r < k1) v = c1[(long long)r * q + c];
      else if (r < k12) v = c2[(long long)(r - k1) * q + c];
      else if (r < K) v = c3[(long long)(r - k12) * q + c];
    }
    Cs[e] = v;
  }
  const long long mine = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long W = mine * nst;
  // stage w: 128 rows x 32 K-values = 1024 16-byte copies, 4 per thread
  auto issue = [&](long long w) {
    const long long tile = blockIdx.x + (w / nst) * gridDim.x;
    const int k0 = (int)(w % nst) * kTsK;
    float *dst = As + (size_t)(w % kTaStages) * kTsRows * kTaLd;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int idx = tid + t * 256;
      const int rr = idx >> 3, kq = (idx & 7) * 4;
      const long long row = tile * kTsRows + rr;
      const int k = k0 + kq;
      const float *src = A1;
      uint32_t bytes = 0;
      if (row < n) {
        if (k < k1) {
          if (KS_IN(row * k1 + k + 3, n * k1)) { src = A1 + row * k1 + k; bytes = 16; }
        } else if (k < k12) {
          if (KS_IN(row * k2 + (k - k1) + 3, n * k2)) { src = A2 + row * k2 + (k - k1); bytes = 16; }
        } else if (k < K) {
          if (KS_IN(row * k3 + (k - k12) + 3, n * k3)) { src = A3 + row * k3 + (k - k12); bytes = 16; }
        }
      }
      const long long di = (long long)(w % kTaStages) * kTsRows * kTaLd + rr * kTaLd + kq;
      if (KS_IN(di + 3, (long long)kTaStages * kTsRows * kTaLd))
        cp_async16(smem_addr(dst + rr * kTaLd + kq), src, bytes);
    }
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int st = 0; st < kTaStages - 1; ++st) {
    if (st < W) issue(st);
    cp_async_commit();
  }
  __syncthreads();                                      // C staged
  for (long long w = 0; w < W; ++w) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kTaStages - 2) : "memory");  // stage w landed
    __syncthreads();                                    // ... everyone's; stage w-1 consumed
    if (w + kTaStages - 1 < W) issue(w + kTaStages - 1);
    cp_async_commit();
    const int k0 = (int)(w % nst) * kTsK;
    const float *Ab = As + (size_t)(w % kTaStages) * kTsRows * kTaLd + (size_t)8 * ty * kTaLd;
#pragma unroll 2
    for (int kq = 0; kq < kTsK; kq += 4) {
      float4 a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = *reinterpret_cast<const float4 *>(Ab + i * kTaLd + kq);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 cv = *reinterpret_cast<const float4 *>(Cs + (size_t)(k0 + kq + kk) * kTile +
                                                            4 * tx);
        const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float av = kk == 0 ? a[i].x : kk == 1 ? a[i].y : kk == 2 ? a[i].z : a[i].w;
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av, cc[j], acc[i][j]);
        }
      }
    }
    if (w % nst == nst - 1) {
      const long long tile = blockIdx.x + (w / nst) * gridDim.x;
      ts_epilogue(n, q, tile * kTsRows + 8 * ty, tx, acc, alpha, beta, Bm, out, add2, out2, dn);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// The pipelined kernel applies when every 16-byte copy of A stays inside one
// row of one operand: each width a multiple of 4 and each base 16-byte aligned.
static bool ta_aligned(const float *A1, int k1, const float *A2, int k2, const float *A3, int k3) {
  auto ok = [](const float *A, int k) {
    return !A || (k % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0);
  };
  return ok(A1, k1) && ok(A2, k2) && ok(A3, k3);
}

// Launch of the tall-skinny update (pipelined when aligned).
static void launch_ts(Problem &P, int q, const float *A1, int k1, const float *c1,
                      const float *A2, int k2, const float *c2, const float *A3, int k3,
                      const float *c3, float alpha, float beta, const float *Bm, float *out,
                      const float *add2, float *out2, TsDensity dn) {
  auto al16 = [](const void *ptr) { return reinterpret_cast<uintptr_t>(ptr) % 16 == 0; };
  dn.vec = q % 4 == 0 && al16(out) && al16(Bm) && al16(add2) && al16(out2) ? 1 : 0;
  const int K = k1 + (A2 ? k2 : 0) + (A3 ? k3 : 0);
  const long long ntiles = (P.n + kTsRows - 1) / kTsRows;
  long long nb = 2LL * P.sms;
  if (nb > ntiles) nb = ntiles;
  if (ta_aligned(A1, k1, A2, k2, A3, k3))
    combine_ta_kernel<<<(int)nb, 256, combine_ta_smem(K), P.stream>>>(
        P.n, q, A1, k1, c1, A2, k2, c2, A3, k3, c3, alpha, beta, Bm, out, add2, out2, ntiles, dn);
  else
    combine_ts_kernel<<<(int)nb, 256, combine_ts_smem(K), P.stream>>>(
        P.n, q, A1, k1, c1, A2, k2, c2, A3, k3, c3, alpha, beta, Bm, out, add2, out2, ntiles, dn);
}

// out = A1 C1 + A2 C2 + A3 C3 and out2 = add2 + out in one pass of the
// tall-skinny FP32 kernel (n x q blocks, q <= 64, k1 + k2 + k3 <= 192); false
// (nothing launched) for other shapes or when the tensor cores take the
// products.
bool combine3_f32_applies(const Problem &P, int k1, int k2, int k3, int q) {
  return q <= kTile && k1 + k2 + k3 <= kTsMaxK && !use_tensor_cores(P, k1, q);
}

ks_status launch_combine3_f32(Problem &P, const float *A1, int k1, const double *C1,
                              const float *A2, int k2, const double *C2, const float *A3, int k3,
                              const double *C3, float *out, const float *add2, float *out2, int q,
                              const double *rho_b, double *rho, bool images_ready) {
  if (!combine3_f32_applies(P, k1, k2, k3, q))
    return set_error(KS_EINVAL, "combine3: shape outside the tall-skinny kernel");
  // FP32 images of C1, C2, C3 one after the other in P.cf (3 p^2 floats)
  float *c1 = P.cf, *c2 = P.cf + (size_t)k1 * q, *c3 = c2 + (size_t)k2 * q;
  if ((size_t)(k1 + k2 + k3) * q > (size_t)3 * P.p * P.p)
    return set_error(KS_EINVAL, "combine3: coefficient image too small");
  const long long len1 = (long long)k1 * q, len2 = (long long)k2 * q, len3 = (long long)k3 * q;
  if (!images_ready) {
    ProfScope ps_(P.stream, KP_REDUCE);
    coef_convert_kernel<<<(int)((len1 + len2 + 255) / 256), 256, 0, P.stream>>>(len1, C1, c1,
                                                                                len2, C2, c2);
    coef_convert_kernel<<<(int)((len3 + 255) / 256), 256, 0, P.stream>>>(len3, C3, c3, 0,
                                                                         nullptr, nullptr);
  }
  KS_CUDA_TRY(cudaGetLastError());
  const int K = k1 + k2 + k3;
  // tensor cores when out2 adds A1 (the retraction: A1 = X_b): A1 goes last,
  // where the epilogue reads it back from the ring
  if (combine_tc64_applies(P, q, {k1, k2, k3}, {A1, A2, A3, out, out2}) &&
      (!out2 || (add2 == A1 && k1 == q))) {
    const bool dens = rho && out2 && q == P.p;
    return launch_combine_tc64(P, q, A2, k2, c2, 1.0f, A3, k3, c3, 1.0f, A1, k1, c1, 1.0f, out,
                               out2, dens ? rho_b : nullptr, dens ? rho : nullptr);
  }
  {
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * K,
                  (double)P.n * (K + q * (out2 ? 3 : 1)) * sizeof(float));
    TsDensity dn;
    if (rho && add2 && out2 && q == P.p) {
      dn.rho_b = rho_b;
      dn.rho = rho;
      dn.occ = P.occ;
    }
    launch_ts(P, q, A1, k1, c1, A2, k2, c2, A3, k3, c3, 1.0f, 0.0f, nullptr, out, add2, out2, dn);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Dynamic shared memory of the tall-skinny update beyond the default 48 KiB
// (on the current device; called when a problem is created).
ks_status configure_blas_kernels() {
  KS_CUDA_TRY(cudaFuncSetAttribute(gram2_ta_kernel<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)gram_ta_smem<true>()));
  KS_CUDA_TRY(cudaFuncSetAttribute(gram2_ta_kernel<false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)gram_ta_smem<false>()));
  KS_CUDA_TRY(cudaFuncSetAttribute(combine_ts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)combine_ts_smem(kTsMaxK)));
  KS_CUDA_TRY(cudaFuncSetAttribute(combine_ta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)combine_ta_smem(kTsMaxK)));
  return KS_OK;
}

template ks_status launch_combine<double>(Problem &, const double *, int, const double *,
                                          const double *, int, const double *, double, double,
                                          const double *, double *, int);
template ks_status launch_combine<float>(Problem &, const float *, int, const double *,
                                         const float *, int, const double *, double, double,
                                         const float *, float *, int);

template <typename A, typename B>
__global__ void convert_kernel(long long total, const A *__restrict__ in, B *__restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (B)in[e];
}

template <typename A, typename B>
static ks_status convert_impl(Problem &P, const A *in, B *out) {
  const long long total = (long long)P.n * P.p;
  const int nb = reduce_blocks(P, total);
  {
    ProfScope ps_(P.stream, KP_OTHER);
    convert_kernel<A, B><<<nb, kThreads, 0, P.stream>>>(total, in, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_convert(Problem &P, const double *in, float *out) { return convert_impl(P, in, out); }
ks_status launch_convert(Problem &P, const float *in, double *out) { return convert_impl(P, in, out); }

__global__ void ortho_err_kernel(int p, const double *__restrict__ O, double *out) {
  __shared__ double smem[33];
  double acc = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    const double d = O[e] - (i == j ? 1.0 : 0.0);
    acc = fma(d, d, acc);
  }
  const double s = block_sum(acc, smem);
  if (threadIdx.x == 0) *out = s;
}

ks_status launch_ortho_err(Problem &P, const double *O, double *out) {
  {
    ProfScope ps_(P.stream, KP_REDUCE);
    ortho_err_kernel<<<1, kThreads, 0, P.stream>>>(P.p, O, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// ---------------------------------------------------------------- no-alloc
// Scratch of ks_gram_noalloc: the per-chunk partial Grams live in this
// file-scope device array instead of memory from cudaMalloc.  Every GPU that
// loads the library holds it (16 MiB) until the process exits.
constexpr size_t kNoAllocDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
double *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

KS_OOB_READER(blas)

}  // namespace ks

extern "C" ks_status ks_gram_noalloc(const double *A, int pa, const double *B, int qb,
                                     long long n, double *out, void *stream) {
  using namespace ks;
  if (!A || !B || !out) return set_error(KS_EINVAL, "null argument");
  if (pa < 1 || qb < 1 || n < 1) return set_error(KS_EINVAL, "bad sizes");
  if ((size_t)pa * (size_t)qb > kNoAllocDoubles)
    return set_error(KS_EINVAL, "ks_gram_noalloc: pa * qb = %zu exceeds the scratch capacity %zu",
                     (size_t)pa * qb, kNoAllocDoubles);
  int dev = 0;
  KS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(KS_EINVAL, "device index out of range");
  double *scratch = nullptr;
  {
    // first call on this device: translate the array's host-side name into
    // its device address (with this device current)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *ptr = nullptr;
      KS_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
      g_noalloc_ptr[dev] = (double *)ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  int sms = 0;
  KS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int tiles = ((pa + kTile - 1) / kTile) * ((qb + kTile - 1) / kTile);
  long long chunks = (4LL * sms + tiles - 1) / tiles;
  const long long maxc = (n + kTileK - 1) / kTileK;
  const long long capc = (long long)(kNoAllocDoubles / ((size_t)pa * qb));
  if (chunks > maxc) chunks = maxc;
  if (chunks > capc) chunks = capc;
  if (chunks < 1) chunks = 1;
  long long rows_per = (n + chunks - 1) / chunks;
  rows_per = (rows_per + kTileK - 1) / kTileK * kTileK;
  cudaStream_t s = (cudaStream_t)stream;
  {
    // every partial tile is written in full (zeros for empty row ranges)
    // before the reduction reads it, so nothing needs clearing
    ProfScope ps_(s, KP_GRAM, 2.0 * n * pa * qb, (double)n * (pa + qb) * sizeof(double));
    gram_kernel<double><<<dim3(tiles, (unsigned)chunks), 256, 0, s>>>(n, pa, qb, rows_per, A, B,
                                                                       scratch);
  }
  KS_CUDA_TRY(cudaGetLastError());
  const long long len = (long long)pa * qb;
  {
    ProfScope ps_(s, KP_REDUCE);
    gram_reduce_kernel<<<(int)((8 * len + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        (int)chunks, len, scratch, out);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}
