// FP64 products on the tensor cores by error-free splitting (the Ozaki
// scheme).  GB300's FP64 pipe does 2 FMA per clock per SM; its BF16 tensor
// cores do three orders of magnitude more.
//
// Split.  An FP64 entry x is written below an exponent E that bounds a whole
// line of entries (a Gram column; a row of the update's A, a column of its C)
// as |x| ~= sum_{s=1..8} d_s 2^(E - 1022 - b s), with digits d_s in
// [0, 2^b) taken from the integer mantissa by shifts on the integer pipes
// (b = 6 for the Gram, 48 bits; b = 7 for the update, 56 bits).  A signed
// digit is exact in BF16, a product of two digits is an exact integer, and
// the pairs (s, t) with the same g = s + t share one scale.  Each group g
// accumulates in its own FP32 TMEM region and stays an exact integer as long
// as (g - 1) x K x (2^b - 1)^2 < 2^24 (Gram: K = 512 rows per chunk with
// b = 6; update: K <= 128 with b = 7).  Pairs with s + t > 9 are not formed
// (weight below 2^(-8 b) of the leading one).  The groups are folded exactly
// into an int64 before one FP64 rounding, so the result carries the rounding
// of a 48- or 56-bit split of its operands plus one FP64 rounding.
//
// MMAs.  The 8 slice tiles of an operand are stored back to back with one
// row-group stride, so B slices t0 .. t0 + k - 1 form one operand of 64 k
// rows; one MMA of N = 64 k then puts the products of A slice s with them
// into the consecutive group regions s + t0 .. s + t0 + k - 1: 12 MMAs of
// M = 128 per K-step of 16 cover the 36 digit pairs.
//
// Gram A^T B (A: n x pa, B: n x qb, row-major): a block owns a 64 x 64 output
// tile and a range of rows, in chunks of 512 rows.  A stage holds 32 rows:
// the 8 A-slice tiles (64 x 32) back to back and a zero tile after them, so an
// M = 128 MMA at slice s reads slice s in its first 64 rows (the other 64 TMEM
// lanes see slice s + 1 and are ignored), and the 8 B-slice tiles (64 x 32).
// The column exponents come from a pre-pass (oz_colexp_kernel).
//
// Update out = alpha (A1 C1 + A2 C2) + beta Bm (K = k1 + k2 <= 128): the split
// C (8 slice tiles of 64 columns x Kp) is built per call and held in shared
// memory; row tiles of 128 rows are staged 16 K-values at a time; the row
// exponents come from a pre-pass (oz_rowexp_kernel).
//
// Stage buffers alternate; one thread issues a stage's MMAs and commits them
// to the stage's mbarrier, and a buffer is refilled only after those MMAs
// completed.  Every wait is bounded: a block that waits too long records
// KS_ETIMEOUT and stops.
#include <cstdint>

#include "ks_device.cuh"

namespace ks {

namespace {

constexpr int kOzS = 8;                       // digits per value
constexpr int kOzT = 64;                      // output tile edge / B slice rows
constexpr int kOzThreads = 256;
constexpr int kOzCols = 512;                  // TMEM columns: 8 groups x 64

// Gram
constexpr int kGzB = 6;
constexpr int kGzK = 32;                      // rows of n per stage
constexpr int kGzChunk = 512;                 // rows per exact FP32 accumulation
constexpr int kGzSlice = kOzT * kGzK * 2;     // 64 x 32 BF16: 4 KiB
constexpr int kGzABytes = (kOzS + 1) * kGzSlice;   // 8 slices + a zero tile
constexpr int kGzBBytes = kOzS * kGzSlice;
constexpr int kGzStage = kGzABytes + kGzBBytes;    // 68 KiB
constexpr int kGzSmem = 2 * kGzStage + 1024;
static_assert(8 * kGzChunk * 63 * 63 < (1 << 24), "Gram group sums must stay exact in FP32");

// update
constexpr int kCzB = 7;
constexpr int kCzM = 128, kCzKs = 16, kCzKmax = 128;
constexpr int kCzASlice = kCzM * kCzKs * 2;                // 128 x 16 BF16: 4 KiB
constexpr int kCzAStage = kOzS * kCzASlice;                 // 32 KiB
constexpr int kCzCTile = kOzT * kCzKmax * 2;                // 16 KiB per slice at Kp = 128
constexpr int kCzSmem = kOzS * kCzCTile + 2 * kCzAStage + 1024;
static_assert(8 * kCzKmax * 127 * 127 < (1 << 24), "update group sums must stay exact in FP32");

__device__ __forceinline__ uint32_t oz_smem(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a tile of kw K-values per row: core
// matrices of 8 rows x 8 K (16 bytes), K-adjacent ones 128 bytes apart
// (LBO), row groups of 8 rows 16 kw bytes apart (SBO)
__device__ __forceinline__ int oz_offset(int r, int k, int kw) {
  return (r >> 3) * (16 * kw) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr, int sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = 64 nt
__device__ __forceinline__ uint32_t oz_idesc(int nt) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nt * kOzT >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// The 36 digit pairs of one K-step of 16 as 12 MMAs: A slice s (a_base +
// (s - 1) a_step) against B slices t0 .. t0 + nt - 1 (b_base + (t0 - 1) b_step)
// into the group regions s + t0 .. (TMEM columns 64 (g - 2)).  `first`: the
// regions start afresh (the s = 1 MMAs cover every region once).
__device__ __forceinline__ void oz_issue_kstep(uint32_t tmem, uint32_t a_base, uint32_t a_step,
                                               int a_sbo, uint32_t b_base, uint32_t b_step,
                                               int b_sbo, bool first) {
#pragma unroll
  for (int s = 1; s <= kOzS; ++s) {
    const int tmax = kOzS + 1 - s;
#pragma unroll
    for (int t0 = 1; t0 <= tmax; t0 += 4) {
      const int nt = tmax - t0 + 1 < 4 ? tmax - t0 + 1 : 4;
      oz_mma(tmem + (uint32_t)(kOzT * (s + t0 - 2)), oz_desc(a_base + (s - 1) * a_step, a_sbo),
             oz_desc(b_base + (t0 - 1) * b_step, b_sbo), oz_idesc(nt),
             (first && s == 1) ? 0u : 1u);
    }
  }
}

__device__ __forceinline__ bool oz_wait(uint32_t mbar, uint32_t parity) {
  for (long long spins = 0; spins < kSpinLimit; ++spins) {
    uint32_t done;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, q;\n}\n" : "=r"(done) : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void oz_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(oz_smem(bar)));
}

// 32 FP32 accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void oz_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__device__ __forceinline__ uint32_t oz_tmem_alloc(uint32_t *slot, uint64_t *mbar) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(oz_smem(slot)), "r"(kOzCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(oz_smem(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(oz_smem(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  return *slot;
}

__device__ __forceinline__ void oz_tmem_free(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kOzCols));
}

// Wait for the commits of the last one or two stages of a pipeline run of
// `issued` stages and consume both barriers' phases; block-uniform result.
__device__ __forceinline__ bool oz_drain(uint64_t *mbar, uint32_t *phase, int issued,
                                         int *status) {
  int ok = 1;
  if (issued > 0) {
    const int last = (issued - 1) & 1;
    if (issued >= 2 && !oz_wait(oz_smem(&mbar[last ^ 1]), phase[last ^ 1])) ok = 0;
    if (!oz_wait(oz_smem(&mbar[last]), phase[last])) ok = 0;
    if (issued >= 2) phase[last ^ 1] ^= 1u;
    phase[last] ^= 1u;
  }
  ok = __syncthreads_and(ok);
  if (!ok && threadIdx.x == 0) atomicCAS(status, 0, (int)KS_ETIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok != 0;
}

// Before refilling stage buffer `buf` (stage number `issued` of the run):
// wait for the MMAs of two stages ago.
__device__ __forceinline__ bool oz_reuse(uint64_t *mbar, uint32_t *phase, int buf, int issued,
                                         int *status) {
  if (issued < 2) return true;
  int ok = oz_wait(oz_smem(&mbar[buf]), phase[buf]) ? 1 : 0;
  phase[buf] ^= 1u;
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) atomicCAS(status, 0, (int)KS_ETIMEOUT);
    return false;
  }
  return true;
}

// Effective biased exponent (subnormals and zero as 1, so that the mantissa
// integer m of a value is m 2^(e - 1075) with the implicit bit for normals).
__device__ __forceinline__ int oz_exp(uint64_t bits) {
  const int e = (int)((bits >> 52) & 0x7FF);
  return e > 0 ? e : 1;
}

// BF16 bit pattern of the signed integer digit d (0 <= d < 256): the FP32
// value 2^23 + d (d in the mantissa of 2^23) minus 2^23 is d exactly, on the
// logic and FMA pipes; d has at most 8 significant bits, so its top 16 bits
// are its BF16 pattern.  A zero digit with the sign set is -0, harmless in
// the sums.
__device__ __forceinline__ uint32_t oz_bf16(uint32_t d, uint32_t sign) {
  const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
  return (__float_as_uint(f) >> 16) | sign;
}

// The 8 digits of Bits bits each of x below exponent ecol (so that
// |x| ~= sum_s d_s 2^(ecol - 1022 - Bits s)), as BF16 patterns in the low
// 16 bits of dig[s]; truncation, error below 2^(ecol - 1022 - 8 Bits).
template <int Bits>
__device__ __forceinline__ void oz_split(double x, int ecol, uint32_t (&dig)[kOzS]) {
  constexpr int W = Bits * kOzS;                            // 48 or 56
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  uint64_t m = bits & 0xFFFFFFFFFFFFFull;
  if ((bits >> 52) & 0x7FF) m |= 1ull << 52;
  const int sh = ecol - oz_exp(bits) + 53 - W;              // >= 53 - W
  const uint64_t M = sh >= 64 ? 0ull : (sh >= 0 ? (m >> sh) : (m << -sh));   // < 2^W
  const uint32_t sign = (uint32_t)(bits >> 48) & 0x8000u;
#pragma unroll
  for (int s = 0; s < kOzS; ++s)
    dig[s] = oz_bf16((uint32_t)(M >> (W - Bits * (s + 1))) & ((1u << Bits) - 1u), sign);
}

// Split a pair of K-adjacent values (k even, k + 1) and store the 8 slices
// (slice tiles `step` bytes apart) as 32-bit words at byte offset off.
template <int Bits>
__device__ __forceinline__ void oz_store_pair(unsigned char *base, int step, int off, double x0,
                                              double x1, int e) {
  uint32_t d0[kOzS], d1[kOzS];
  oz_split<Bits>(x0, e, d0);
  oz_split<Bits>(x1, e, d1);
#pragma unroll
  for (int s = 0; s < kOzS; ++s) *(uint32_t *)(base + s * step + off) = d0[s] | (d1[s] << 16);
}

// x 2^e: a multiplication by an exact power of two in the normal range, else ldexp
__device__ __forceinline__ double oz_pow2(double x, int e) {
  return (e >= -1022 && e <= 1023) ? x * __longlong_as_double((long long)(e + 1023) << 52)
                                   : ldexp(x, e);
}

}  // namespace

// Largest biased exponent of every column of the n x p row-major block X
// into emax[p] (zero-initialised by the caller); deterministic (a maximum).
// Thread t of a block takes column c = t % p (p <= blockDim, rows t / p in
// steps of blockDim / p) or columns t, t + blockDim, ... (p > blockDim) and
// keeps its maximum in a register: one atomic per thread and column.
__global__ void oz_colexp_kernel(long long n, int p, const double *__restrict__ X,
                                 int *__restrict__ emax) {
  const int t = threadIdx.x, nt = blockDim.x;
  if (p <= nt) {
    const int rpi = nt / p;
    if (t >= rpi * p) return;
    const int c = t % p;
    int m = 0;
    for (long long k = (long long)blockIdx.x * rpi + t / p; k < n; k += (long long)gridDim.x * rpi) {
      const int ex = (int)(((uint64_t)__double_as_longlong(__ldg(X + k * p + c)) >> 52) & 0x7FF);
      m = max(m, ex);
    }
    if (m > 0) atomicMax(&emax[c], m);
    return;
  }
  for (int c = t; c < p; c += nt) {
    int m = 0;
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
      const int ex = (int)(((uint64_t)__double_as_longlong(__ldg(X + k * p + c)) >> 52) & 0x7FF);
      m = max(m, ex);
    }
    if (m > 0) atomicMax(&emax[c], m);
  }
}

// Largest effective exponent of every row of [A1 A2] (k1 + k2 entries) into
// erow[n]: one warp per row.
__global__ void oz_rowexp_kernel(long long n, const double *__restrict__ A1, int k1,
                                 const double *__restrict__ A2, int k2, int *__restrict__ erow) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = w; r < n; r += nw) {
    int e = 0;
    for (int k = lane; k < k1; k += 32)
      e = max(e, (int)(((uint64_t)__double_as_longlong(__ldg(A1 + r * k1 + k)) >> 52) & 0x7FF));
    for (int k = lane; k < k2; k += 32)
      e = max(e, (int)(((uint64_t)__double_as_longlong(__ldg(A2 + r * k2 + k)) >> 52) & 0x7FF));
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) erow[r] = max(e, 1);
  }
}

__global__ void __launch_bounds__(kOzThreads, 1) gram_oz_kernel(
    long long n, int pa, int qb, long long rows_per, int tiles_b, const double *__restrict__ A,
    const double *__restrict__ B, const int *__restrict__ ea, const int *__restrict__ eb,
    double *__restrict__ part, int *status) {
  extern __shared__ __align__(1024) unsigned char oz_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int sea[kOzT], seb[kOzT];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a0 = (blockIdx.x / tiles_b) * kOzT, b0 = (blockIdx.x % tiles_b) * kOzT;
  const long long r0 = (long long)blockIdx.y * rows_per;
  long long r1 = r0 + rows_per;
  if (r1 > n) r1 = n;

  // the zero tile after the last A slice of both stages
  for (int i = tid; i < kGzSlice / 16; i += kOzThreads) {
    ((uint4 *)(smem + kOzS * kGzSlice))[i] = make_uint4(0, 0, 0, 0);
    ((uint4 *)(smem + kGzStage + kOzS * kGzSlice))[i] = make_uint4(0, 0, 0, 0);
  }
  for (int c = tid; c < kOzT; c += kOzThreads) {
    sea[c] = a0 + c < pa ? max(ea[a0 + c], 1) : 1;
    seb[c] = b0 + c < qb ? max(eb[b0 + c], 1) : 1;
  }
  const uint32_t tmem = oz_tmem_alloc(&tmem_slot, mbar);

  // staging map: combination w + 8 i (i < 4) of column group (8 columns) and
  // K group (8 rows), lane -> column 8 cg + (lane & 7), rows 8 kg + 2 (lane >> 3)
  // and + 1: each warp store covers 32 banks
  int scol[4], sk[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int combo = warp + 8 * i;
    scol[i] = (combo & 7) * 8 + (lane & 7);
    sk[i] = (combo >> 3) * 8 + 2 * (lane >> 3);
  }
  double va[8], vb[8];
  auto fetch = [&](long long r) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long long row = r + sk[i] + h;
        const bool ok = row < r1;
        va[2 * i + h] = (ok && a0 + scol[i] < pa) ? __ldg(A + row * pa + a0 + scol[i]) : 0.0;
        vb[2 * i + h] = (ok && b0 + scol[i] < qb) ? __ldg(B + row * qb + b0 + scol[i]) : 0.0;
      }
    }
  };

  // epilogue lanes: warps 0, 1, 4, 5 read TMEM lanes 0..63 (tile rows); warps
  // w and w + 4 split the 64 columns
  const bool reader = (warp & 3) < 2;
  const int orow = (warp & 3) * 32 + lane;
  const int ocol0 = (warp >> 2) * 32;
  double sum[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) sum[j] = 0.0;

  uint32_t phase[2] = {0u, 0u};
  bool failed = false;
  if (r0 < r1) fetch(r0);
  for (long long c0 = r0; c0 < r1 && !failed; c0 += kGzChunk) {
    const long long c1 = c0 + kGzChunk < r1 ? c0 + kGzChunk : r1;
    int issued = 0;
    for (long long r = c0; r < c1; r += kGzK, ++issued) {
      const int buf = issued & 1;
      unsigned char *st = smem + buf * kGzStage;
      if (!oz_reuse(mbar, phase, buf, issued, status)) {
        failed = true;
        break;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int off = oz_offset(scol[i], sk[i], kGzK);
        oz_store_pair<kGzB>(st, kGzSlice, off, va[2 * i], va[2 * i + 1], sea[scol[i]]);
        oz_store_pair<kGzB>(st + kGzABytes, kGzSlice, off, vb[2 * i], vb[2 * i + 1], seb[scol[i]]);
      }
      if (r + kGzK < r1) fetch(r + kGzK);          // in flight during this stage's MMAs
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sa = oz_smem(st), sb = sa + kGzABytes;
#pragma unroll 1
        for (int ks = 0; ks < kGzK / 16; ++ks)
          oz_issue_kstep(tmem, sa + ks * 256, kGzSlice, 16 * kGzK, sb + ks * 256, kGzSlice,
                         16 * kGzK, issued == 0 && ks == 0);
        oz_commit(&mbar[buf]);
      }
    }
    if (failed) break;
    if (!oz_drain(mbar, phase, issued, status)) {
      failed = true;
      break;
    }
    if (reader) {
      // fold the groups exactly: groups 2..7 into an int64 (group g shifted
      // left by 6 (7 - g) bits; below 2^54 at 512 rows), 8 and 9 in FP32
      // (their weight keeps the FP32 rounding below 2^-60 of the total)
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      long long tot[32];
      float tail[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        tot[j] = 0;
        tail[j] = 0.f;
      }
#pragma unroll 1
      for (int g = 2; g <= kOzS + 1; ++g) {
        uint32_t v[32];
        oz_ld32(tmem + lane_base + (uint32_t)(kOzT * (g - 2) + ocol0), v);
        if (g <= 7) {
          const long long mul = 1LL << (kGzB * (7 - g));
#pragma unroll
          for (int j = 0; j < 32; ++j)
            tot[j] += (long long)__float2int_rn(__uint_as_float(v[j])) * mul;
        } else {
          const float w = g == 8 ? 1.f / 64.f : 1.f / 4096.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) tail[j] = fmaf(__uint_as_float(v[j]), w, tail[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) sum[j] += (double)tot[j] + (double)tail[j];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  // the groups' sum is in units of 2^-42 (group 7) of 2^(E_a + E_b - 2044)
  if (!failed && reader && a0 + orow < pa) {
    const int er = sea[orow];
    double *dst = part + (long long)blockIdx.y * pa * qb + (long long)(a0 + orow) * qb;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int cj = b0 + ocol0 + j;
      if (cj < qb) dst[cj] = oz_pow2(sum[j], er + seb[ocol0 + j] - 2086);
    }
  }
  oz_tmem_free(tmem);
}

// Split C = [C1; C2] (K x q) into img: for column tile ct, 8 slice tiles of
// 64 columns x kp (BF16, K-major), and ec[q] the column exponents.  One block
// per column tile, thread j < 64 owns column ct*64 + j.
__global__ void oz_cimage_kernel(int q, int k1, const double *__restrict__ C1, int k2,
                                 const double *__restrict__ C2, int kp, unsigned char *img,
                                 int *ec) {
  const int ct = blockIdx.x, j = threadIdx.x;
  if (j >= kOzT) return;
  const int col = ct * kOzT + j;
  const int K = k1 + k2;
  auto val = [&](int k) -> double {
    if (col >= q || k >= K) return 0.0;
    return k < k1 ? C1[(long long)k * q + col] : C2[(long long)(k - k1) * q + col];
  };
  int e = 0;
  for (int k = 0; k < K; ++k)
    e = max(e, (int)(((uint64_t)__double_as_longlong(val(k)) >> 52) & 0x7FF));
  e = max(e, 1);
  if (col < q) ec[col] = e;
  const int step = kOzT * kp * 2;
  unsigned char *base = img + (size_t)ct * kOzS * step;
  for (int k = 0; k < kp; k += 2)
    oz_store_pair<kCzB>(base, step, oz_offset(j, k, kp), val(k), val(k + 1), e);
}

__global__ void __launch_bounds__(kOzThreads, 1) combine_oz_kernel(
    long long n, int q, const double *__restrict__ A1, int k1, const double *__restrict__ A2,
    int k2, const unsigned char *__restrict__ img, const int *__restrict__ ec,
    const int *__restrict__ erow_g, int kp, double alpha, double beta, const double *Bm,
    double *out, int *status) {
  extern __shared__ __align__(1024) unsigned char cz_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)cz_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *cimg = smem;                                // 8 slices x 64 x kp
  unsigned char *astage = smem + kOzS * kCzCTile;            // 2 stages x 8 slices x 128 x 16
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int erow[kCzM];
  __shared__ int ecol[kOzT];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ct = blockIdx.y, c0 = ct * kOzT;
  const int K = k1 + k2;
  const int ctile = kOzT * kp * 2;
  {
    const uint4 *src = (const uint4 *)(img + (size_t)ct * kOzS * ctile);
    for (int i = tid; i < kOzS * ctile / 16; i += kOzThreads) ((uint4 *)cimg)[i] = src[i];
    for (int j = tid; j < kOzT; j += kOzThreads) ecol[j] = c0 + j < q ? ec[c0 + j] : 1;
  }
  const uint32_t tmem = oz_tmem_alloc(&tmem_slot, mbar);
  auto aval = [&](long long r, int k) -> double {
    if (r >= n || k >= K) return 0.0;
    return k < k1 ? __ldg(A1 + r * k1 + k) : __ldg(A2 + r * k2 + (k - k1));
  };
  // staging map of a 128 x 16 stage: combination w + 8 i (i < 4) of row group
  // (8 rows) and K half, lane -> row 8 rg + (lane & 7), K 8 kh + 2 (lane >> 3)
  int srow[4], sk[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int combo = warp + 8 * i;
    srow[i] = (combo >> 1) * 8 + (lane & 7);
    sk[i] = (combo & 1) * 8 + 2 * (lane >> 3);
  }
  const int orow = (warp & 3) * 32 + lane, ocol0 = (warp >> 2) * 32;
  const long long tiles = (n + kCzM - 1) / kCzM;
  const int nst = kp / kCzKs;
  double va[8];
  auto fetch = [&](long long rb, int st) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      va[2 * i] = aval(rb + srow[i], st * kCzKs + sk[i]);
      va[2 * i + 1] = aval(rb + srow[i], st * kCzKs + sk[i] + 1);
    }
  };
  uint32_t phase[2] = {0u, 0u};
  bool failed = false;
  if ((long long)blockIdx.x < tiles) fetch((long long)blockIdx.x * kCzM, 0);
  for (long long tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const long long r0 = tile * kCzM;
    for (int r = tid; r < kCzM; r += kOzThreads) erow[r] = r0 + r < n ? erow_g[r0 + r] : 1;
    __syncthreads();
    int issued = 0;
    for (int st = 0; st < nst; ++st, ++issued) {
      const int buf = issued & 1;
      unsigned char *sa = astage + buf * kCzAStage;
      if (!oz_reuse(mbar, phase, buf, issued, status)) {
        failed = true;
        break;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        oz_store_pair<kCzB>(sa, kCzASlice, oz_offset(srow[i], sk[i], kCzKs), va[2 * i],
                            va[2 * i + 1], erow[srow[i]]);
      // the next stage's values (or the next tile's first) in flight
      if (st + 1 < nst) fetch(r0, st + 1);
      else if (tile + gridDim.x < tiles) fetch((tile + gridDim.x) * kCzM, 0);
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        oz_issue_kstep(tmem, oz_smem(sa), kCzASlice, 16 * kCzKs, oz_smem(cimg) + st * 256, ctile,
                       16 * kp, st == 0);
        oz_commit(&mbar[buf]);
      }
    }
    if (failed) break;
    if (!oz_drain(mbar, phase, issued, status)) {
      failed = true;
      break;
    }
    {
      // groups 2..7 exactly into an int64 (group g shifted left by 7 (7 - g)
      // bits, below 2^57), 8 and 9 in FP32 (weight below 2^-42 of the leading
      // group: the FP32 rounding stays below 2^-66 of the result); units
      // 2^-49 of 2^(E_r + E_c - 2044)
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
      long long tot[32];
      float tail[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        tot[j] = 0;
        tail[j] = 0.f;
      }
#pragma unroll 1
      for (int g = 2; g <= kOzS + 1; ++g) {
        uint32_t v[32];
        oz_ld32(tmem + lane_base + (uint32_t)(kOzT * (g - 2) + ocol0), v);
        if (g <= 7) {
          const long long mul = 1LL << (kCzB * (7 - g));
#pragma unroll
          for (int j = 0; j < 32; ++j)
            tot[j] += (long long)__float2int_rn(__uint_as_float(v[j])) * mul;
        } else {
          const float w = g == 8 ? 1.f : 1.f / 128.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) tail[j] = fmaf(__uint_as_float(v[j]), w, tail[j]);
        }
      }
      const long long r = r0 + orow;
      if (r < n) {
        const int er = erow[orow];
        const bool unit = alpha == 1.0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int cj = c0 + ocol0 + j;
          if (cj >= q) continue;
          const double x = fma((double)tail[j], 1.0 / 128.0, (double)tot[j]);
          // x 2^e by adding e to the exponent field (integer pipe) when the
          // result stays normal, else ldexp
          const int e = er + ecol[ocol0 + j] - 2093;
          const long long xb = __double_as_longlong(x);
          const int ex = (int)((xb >> 52) & 0x7FF);
          const double v = (ex >= 1 && ex + e >= 1 && ex + e <= 2046)
                               ? __longlong_as_double(xb + ((long long)e << 52))
                               : ldexp(x, e);
          double o = unit ? v : alpha * v;
          if (Bm) o = fma(beta, Bm[r * q + cj], o);
          out[r * q + cj] = o;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  oz_tmem_free(tmem);
}

static bool gz_configured = false, cz_configured = false;

size_t oz_image_bytes(int p) { return (size_t)((p + kOzT - 1) / kOzT) * kOzS * kCzCTile; }

bool combine_oz_applies(const Problem &P, int k1, int k2, int q) {
  return P.use_oz > 0 && k1 + k2 <= kCzKmax && q <= P.p && P.oz_img && P.oz_rowexp &&
         (P.use_oz == 2 || q >= 48);
}

ks_status launch_combine_oz(Problem &P, const double *A1, int k1, const double *C1,
                            const double *A2, int k2, const double *C2, double alpha, double beta,
                            const double *Bm, double *out, int q) {
  if (!cz_configured) {
    KS_CUDA_TRY(cudaFuncSetAttribute(combine_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kCzSmem));
    cz_configured = true;
  }
  if (!A2) k2 = 0;
  const int K = k1 + k2;
  const int kp = (K + kCzKs - 1) / kCzKs * kCzKs;
  const int ctiles = (q + kOzT - 1) / kOzT;
  {
    ProfScope ps_(P.stream, KP_COMBINE, 0.0, (double)P.n * K * sizeof(double), 2);
    oz_cimage_kernel<<<ctiles, kOzT, 0, P.stream>>>(q, k1, C1, k2, C2, kp, P.oz_img, P.oz_emax);
    oz_rowexp_kernel<<<4 * P.sms, kThreads, 0, P.stream>>>(P.n, A1, k1, A2, k2, P.oz_rowexp);
  }
  KS_CUDA_TRY(cudaGetLastError());
  const long long tiles = (P.n + kCzM - 1) / kCzM;
  long long rb = (P.sms + ctiles - 1) / ctiles;
  if (rb > tiles) rb = tiles;
  {
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * K,
                  (double)P.n * (K + q * (Bm ? 2 : 1)) * sizeof(double));
    combine_oz_kernel<<<dim3((unsigned)rb, (unsigned)ctiles), kOzThreads, kCzSmem, P.stream>>>(
        P.n, q, A1, k1, A2, k2, P.oz_img, P.oz_emax, P.oz_rowexp, kp, alpha, beta, Bm, out,
        P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

ks_status launch_gram_oz(Problem &P, const double *A, int pa, const double *B, int qb,
                         int *emax, double *part, int chunks) {
  if (!gz_configured) {
    KS_CUDA_TRY(cudaFuncSetAttribute(gram_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kGzSmem));
    gz_configured = true;
  }
  KS_CUDA_TRY(cudaMemsetAsync(emax, 0, sizeof(int) * (size_t)(pa + qb), P.stream));
  {
    ProfScope ps_(P.stream, KP_GRAM, 0.0, (double)P.n * (pa + qb) * sizeof(double), 2);
    oz_colexp_kernel<<<4 * P.sms, kThreads, 0, P.stream>>>(P.n, pa, A, emax);
    oz_colexp_kernel<<<4 * P.sms, kThreads, 0, P.stream>>>(P.n, qb, B, emax + pa);
  }
  KS_CUDA_TRY(cudaGetLastError());
  const int tiles_a = (pa + kOzT - 1) / kOzT, tiles_b = (qb + kOzT - 1) / kOzT;
  long long rows_per = (P.n + chunks - 1) / chunks;
  rows_per = (rows_per + kGzK - 1) / kGzK * kGzK;
  {
    ProfScope ps_(P.stream, KP_GRAM, 2.0 * P.n * pa * qb, (double)P.n * (pa + qb) * sizeof(double));
    gram_oz_kernel<<<dim3(tiles_a * tiles_b, chunks), kOzThreads, kGzSmem, P.stream>>>(
        P.n, pa, qb, rows_per, tiles_b, A, B, emax, emax + pa, part, P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

int gram_oz_chunks(const Problem &P, int pa, int qb) {
  const long long tiles = (long long)((pa + kOzT - 1) / kOzT) * ((qb + kOzT - 1) / kOzT);
  long long chunks = (P.sms + tiles - 1) / tiles;
  const long long by_rows = (P.n + kGzK - 1) / kGzK;
  if (chunks > by_rows) chunks = by_rows;
  const long long cap = (long long)(P.partials_len / ((size_t)pa * qb));
  if (chunks > cap) chunks = cap;
  if (chunks < 1) chunks = 1;
  return (int)chunks;
}

}  // namespace ks
