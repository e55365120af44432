// Tall-skinny products of the FP32 phase on the 5th-generation tensor cores
// (tcgen05, kind::tf32), accumulators in tensor memory:
//   gram:    A^T B with A (n x pa), B (n x qb) row-major FP32;
//   combine: alpha (A1 C1 + A2 C2) + beta Bm with FP32 blocks and FP64 C.
// Each block owns a 128 x 256 output tile (256 TMEM columns).  Operands are
// staged 32 K-values at a time in the K-major core-matrix layout (8 rows x
// 16 bytes per core matrix, no swizzle) and split into TF32 high and low
// parts (x = hi + lo, hi = x with the low 13 mantissa bits cleared); one
// thread issues hi.hi + hi.lo + lo.hi (3 x 4 MMAs of 128 x 256 x 8 per stage,
// about 2^-21 relative error per product) into one FP32 accumulator.  Two
// stage buffers alternate; a buffer is refilled only after the MMAs that
// read it have committed to its mbarrier, and the next stage's global loads
// are in flight (registers for the streamed blocks, cp.async for the
// coefficient image of the update) while the current stage's MMAs run.
// A warp stages an 8-row x 4-K patch per step, so its 32 shared-memory
// stores hit 32 different banks.  All waits are bounded: a block that waits
// too long records KS_ETIMEOUT and stops.
#include <cstdint>
#include <initializer_list>

#include "ks_async.cuh"
#include "ks_device.cuh"

namespace ks {

namespace {

constexpr int kTcM = 128, kTcN = 256, kTcK = 32;  // tile rows, cols, K per stage
constexpr int kTcThreads = 256;
constexpr int kTcCols = 256;                      // TMEM columns allocated
constexpr int kTileABytes = kTcM * kTcK * 4;      // 16 KiB
constexpr int kTileBBytes = kTcN * kTcK * 4;      // 32 KiB
constexpr int kStageBytes = 2 * kTileABytes + 2 * kTileBBytes;   // hi + lo of A and B: 96 KiB
constexpr int kTcSmem = 2 * kStageBytes + 1024;   // two stages + alignment slack
constexpr int kRegA = kTcM * kTcK / kTcThreads;   // 16 staged values per thread
constexpr int kRegB = kTcN * kTcK / kTcThreads;   // 32
constexpr int kOutLd = kTcM + 1;                  // transposed output tile row stride (floats)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of an R x 32 K-major tile: core matrices of
// 8 rows x 16 bytes, K-adjacent ones 128 bytes apart (LBO), row groups of 8
// 1024 bytes apart (SBO)
__device__ __forceinline__ int kmajor_offset(int r, int k) {
  return (r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start address, LBO = 128 B, SBO = 1024 B,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(tmem), "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}

// bounded wait for phase `parity` of the mbarrier; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long spins = 0; spins < kSpinLimit; ++spins) {
    uint32_t done;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, q;\n}\n" : "=r"(done) : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// Staging map of an R x 32 K-major tile: step i of warp w handles patch
// g = w + 8 i, rows 8 (g % (R/8)) .. + 7 (lane & 7) and K-values
// 4 (g / (R/8)) .. + 3 (lane >> 3).
template <int R>
__device__ __forceinline__ void patch(int warp, int lane, int i, int &r, int &k) {
  const int g = warp + 8 * i;
  r = (g % (R / 8)) * 8 + (lane & 7);
  k = (g / (R / 8)) * 4 + (lane >> 3);
}

__device__ __forceinline__ void store_split(unsigned char *hi_base, unsigned char *lo_base, int r,
                                            int k, float x) {
  float hi, lo;
  split_tf32(x, hi, lo);
  const int off = kmajor_offset(r, k);
  *(float *)(hi_base + off) = hi;
  *(float *)(lo_base + off) = lo;
}

// 3 x 4 MMAs of one stage (K = 32) into the accumulator.
__device__ __forceinline__ void issue_stage(uint32_t tmem, const unsigned char *st, bool first) {
  const uint32_t sah = smem_u32(st), sal = sah + kTileABytes;
  const uint32_t sbh = sah + 2 * kTileABytes, sbl = sbh + kTileBBytes;
#pragma unroll
  for (int ks = 0; ks < kTcK / 8; ++ks) {
    const uint32_t o = ks * 256;
    mma_tf32(tmem, smem_desc(sah + o), smem_desc(sbh + o), (!first || ks > 0) ? 1u : 0u);
    mma_tf32(tmem, smem_desc(sah + o), smem_desc(sbl + o), 1u);
    mma_tf32(tmem, smem_desc(sal + o), smem_desc(sbh + o), 1u);
  }
}

__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(bar)));
}

// 64 FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]),
        "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]),
        "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]),
        "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]),
        "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]),
        "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// TMEM allocation (warp 0) and the two stage mbarriers (thread 0).
__device__ __forceinline__ uint32_t tc_setup(uint32_t *tmem_slot, uint64_t *mbar) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tmem_slot)), "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  return *tmem_slot;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

// Wait for the commits of the last one or two stages; block-uniform result.
__device__ __forceinline__ bool drain(uint64_t *mbar, uint32_t *phase, int issued, bool failed,
                                      int *status) {
  int ok = failed ? 0 : 1;
  if (ok && issued > 0) {
    const int last = (issued - 1) & 1;
    if (issued >= 2 && !mbar_wait(smem_u32(&mbar[last ^ 1]), phase[last ^ 1])) ok = 0;
    if (!mbar_wait(smem_u32(&mbar[last]), phase[last])) ok = 0;
  }
  ok = __syncthreads_and(ok);
  if (!ok && threadIdx.x == 0 && !failed) atomicCAS(status, 0, (int)KS_ETIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok != 0;
}

// Before refilling stage buffer `buf`: wait for the MMAs of two stages ago.
__device__ __forceinline__ bool reuse_wait(uint64_t *mbar, uint32_t *phase, int buf, int issued,
                                           int *status) {
  if (issued < 2) return true;
  int ok = mbar_wait(smem_u32(&mbar[buf]), phase[buf]) ? 1 : 0;
  phase[buf] ^= 1u;
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) atomicCAS(status, 0, (int)KS_ETIMEOUT);
    return false;
  }
  return true;
}

__global__ void __launch_bounds__(kTcThreads, 1) gram_tc_kernel(long long n, int pa, int qb,
                                                               long long rows_per, int tiles_b,
                                                               const float *__restrict__ A,
                                                               const float *__restrict__ B,
                                                               double *__restrict__ part,
                                                               int *status) {
  extern __shared__ __align__(1024) unsigned char dyn_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ta = blockIdx.x / tiles_b, tb = blockIdx.x % tiles_b;
  const int a0 = ta * kTcM, b0 = tb * kTcN;
  const int chunk = blockIdx.y;
  const long long r0 = chunk * rows_per;
  long long r1 = r0 + rows_per;
  if (r1 > n) r1 = n;
  const uint32_t tmem = tc_setup(&tmem_slot, mbar);

  // next stage's values in registers: A (row k, column a0 + m), B (row k, column b0 + c)
  float ra[kRegA], rb[kRegB];
  auto fetch = [&](long long r) {
#pragma unroll
    for (int i = 0; i < kRegA; ++i) {
      int m, k;
      patch<kTcM>(warp, lane, i, m, k);
      const long long row = r + k;
      ra[i] = (row < r1 && a0 + m < pa) ? A[row * pa + a0 + m] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < kRegB; ++i) {
      int c, k;
      patch<kTcN>(warp, lane, i, c, k);
      const long long row = r + k;
      rb[i] = (row < r1 && b0 + c < qb) ? B[row * qb + b0 + c] : 0.f;
    }
  };
  uint32_t phase[2] = {0u, 0u};
  int issued = 0;
  bool failed = false;
  if (r0 < r1) fetch(r0);
  for (long long r = r0; r < r1; r += kTcK, ++issued) {
    const int buf = issued & 1;
    unsigned char *st = smem + buf * kStageBytes;
    if (!reuse_wait(mbar, phase, buf, issued, status)) {
      failed = true;
      break;
    }
#pragma unroll
    for (int i = 0; i < kRegA; ++i) {
      int m, k;
      patch<kTcM>(warp, lane, i, m, k);
      store_split(st, st + kTileABytes, m, k, ra[i]);
    }
#pragma unroll
    for (int i = 0; i < kRegB; ++i) {
      int c, k;
      patch<kTcN>(warp, lane, i, c, k);
      store_split(st + 2 * kTileABytes, st + 2 * kTileABytes + kTileBBytes, c, k, rb[i]);
    }
    if (r + kTcK < r1) fetch(r + kTcK);          // in flight during this stage's MMAs
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_stage(tmem, st, issued == 0);
      commit(&mbar[buf]);
    }
  }
  const bool ok = drain(mbar, phase, issued, failed, status);
  if (ok) {
    // warps w and w + 4 read the same 32 lanes (rows), each half of the columns
    const int arow = a0 + (warp & 3) * 32 + lane;
    const int half = warp >> 2;
    double *dst = part + (long long)chunk * pa * qb + (long long)arow * qb;
#pragma unroll 1
    for (int blk = 0; blk < 2; ++blk) {
      const int cb = half * 128 + blk * 64;
      uint32_t v[64];
      tmem_ld64(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
      if (arow < pa)
        for (int j = 0; j < 64; ++j)
          if (b0 + cb + j < qb) dst[b0 + cb + j] = issued > 0 ? (double)__uint_as_float(v[j]) : 0.0;
    }
  }
  tc_teardown(tmem);
}

// Coefficient image of the update: for column tile ct (256 columns of
// q) and stage s (K-values 32 s .. 32 s + 31 of [C1; C2]), the hi and lo
// K-major tiles exactly as a stage buffer holds them, so a block copies
// each stage's 64 KiB with cp.async.
__global__ void combine_image_kernel(int q, int k1, const double *__restrict__ C1, int k2,
                                     const double *__restrict__ C2, int stages, float *img) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_stage = (long long)kTcN * kTcK;
  const long long total = (long long)((q + kTcN - 1) / kTcN) * stages * per_stage;
  if (e >= total) return;
  const int within = (int)(e % per_stage);
  const long long ts = e / per_stage;             // ct * stages + s
  const int s = (int)(ts % stages), ct = (int)(ts / stages);
  const int c = within / kTcK, k = within % kTcK;
  const int kk = s * kTcK + k, col = ct * kTcN + c;
  double x = 0.0;
  if (col < q) {
    if (kk < k1) x = C1[(long long)kk * q + col];
    else if (kk < k1 + k2) x = C2[(long long)(kk - k1) * q + col];
  }
  float hi, lo;
  split_tf32((float)x, hi, lo);
  unsigned char *base = (unsigned char *)(img + ts * 2 * per_stage);
  const int off = kmajor_offset(c, k);
  *(float *)(base + off) = hi;
  *(float *)(base + kTileBBytes + off) = lo;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src)
               : "memory");
}

// out = alpha (A1 C1 + A2 C2) + beta Bm: a block owns 128 rows x 256
// columns; K runs over the columns of A1 then A2 in stages of 32.
__global__ void __launch_bounds__(kTcThreads, 1) combine_tc_kernel(
    long long n, int q, const float *__restrict__ A1, int k1, const float *__restrict__ A2, int k2,
    const float *__restrict__ img, int stages, float alpha, float beta,
    const float *__restrict__ Bm, float *__restrict__ out, int *status) {
  extern __shared__ __align__(1024) unsigned char dyn_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long row0 = (long long)blockIdx.x * kTcM;
  const int ct = blockIdx.y, c0 = ct * kTcN;
  const int K = k1 + (A2 ? k2 : 0);
  const int nw = min(kTcN, q - c0);
  const uint32_t tmem = tc_setup(&tmem_slot, mbar);

  float ra[kRegA];
  auto fetch = [&](int kb) {
#pragma unroll
    for (int i = 0; i < kRegA; ++i) {
      int m, k;
      patch<kTcM>(warp, lane, i, m, k);
      const long long row = row0 + m;
      const int kk = kb + k;
      float x = 0.f;
      if (row < n && kk < K) x = kk < k1 ? A1[row * k1 + kk] : A2[row * k2 + (kk - k1)];
      ra[i] = x;
    }
  };
  // the stage's hi and lo coefficient tiles: 64 KiB, 16 x 16 bytes per thread
  auto copy_image = [&](int s, unsigned char *st) {
    const unsigned char *src = (const unsigned char *)(img + ((long long)ct * stages + s) * 2 *
                                                             kTcN * kTcK);
    unsigned char *dst = st + 2 * kTileABytes;
#pragma unroll
    for (int i = 0; i < 2 * kTileBBytes / 16 / kTcThreads; ++i) {
      const int o = (tid + i * kTcThreads) * 16;
      cp_async16(dst + o, src + o);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  uint32_t phase[2] = {0u, 0u};
  int issued = 0;
  bool failed = false;
  fetch(0);
  for (int s = 0; s < stages; ++s, ++issued) {
    const int buf = issued & 1;
    unsigned char *st = smem + buf * kStageBytes;
    if (!reuse_wait(mbar, phase, buf, issued, status)) {
      failed = true;
      break;
    }
    copy_image(s, st);
#pragma unroll
    for (int i = 0; i < kRegA; ++i) {
      int m, k;
      patch<kTcM>(warp, lane, i, m, k);
      store_split(st, st + kTileABytes, m, k, ra[i]);
    }
    if (s + 1 < stages) fetch((s + 1) * kTcK);   // in flight during this stage's MMAs
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_stage(tmem, st, issued == 0);
      commit(&mbar[buf]);
    }
  }
  const bool ok = drain(mbar, phase, issued, failed, status);
  if (ok) {
    // accumulator -> transposed tile T[c][m] in the (now idle) stage buffers,
    // then row-contiguous, coalesced stores with the alpha / beta epilogue
    float *T = reinterpret_cast<float *>(smem);
    const int m = (warp & 3) * 32 + lane;
    const int half = warp >> 2;
#pragma unroll 1
    for (int blk = 0; blk < 2; ++blk) {
      const int cb = half * 128 + blk * 64;
      uint32_t v[64];
      tmem_ld64(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
      for (int j = 0; j < 64; ++j) T[(cb + j) * kOutLd + m] = __uint_as_float(v[j]);
    }
    __syncthreads();
    for (int rr = warp; rr < kTcM; rr += kTcThreads / 32) {
      const long long row = row0 + rr;
      if (row >= n) break;
      float *dst = out + row * q + c0;
      const float *bm = Bm ? Bm + row * q + c0 : nullptr;
      for (int c = lane; c < nw; c += 32) {
        float y = alpha * T[c * kOutLd + rr];
        if (bm) y = fmaf(beta, bm[c], y);
        dst[c] = y;
      }
    }
  }
  tc_teardown(tmem);
}

// ---------------------------------------------------------------- narrow updates
// out (n x q, q <= 64) = s1 A1 C1 + s2 A2 C2 + s3 A3 C3 and optionally
// out2 = A3 + out (k3 = q) with the increment form's density rho = rho_b +
// f sum out (2 A3 + out): the updates of the retraction and of the
// projected gradient at p <= 64 on the tensor cores.  One persistent block
// per SM walks its 128-row tiles.  Each operand's columns are cut into
// stages of 32 (the last one zero-filled past k_i); a stage (128 rows x 128
// bytes) arrives by one TMA tile load in the 128-byte-swizzled K-major
// layout the MMA reads.  The block's warps take one role each and hand
// stages on through mbarriers, never a block barrier: one thread issues the
// copies into a ring of kNRaw slots; four warps split each landed stage
// elementwise into TF32 high and low parts (x = hi + lo, hi rounded to
// nearest; hi in place, lo into one of kNLo buffers, same layout); one
// thread issues hi.hi + hi.lo + lo.hi (3 x 4 MMAs of 128 x 64 x 8, about
// 2^-21 relative error per product) into one of two 64-column FP32
// accumulators in tensor memory, and its commits release the slot and the
// lo buffer; four warps read a finished tile's accumulator (one row per
// thread) and write it out while the MMAs of the next tile run into the
// other.  The coefficients' image (hi and lo of every stage, scaled, a null
// C_i standing for the identity so that a whole matrix can be added) stays
// in shared memory for the launch; A3 for out2 is read back from global
// memory (the tile's copy is still in L2).  Every wait is bounded; a role
// that gives up sets the block's abort flag, the others stop at their next
// wait, the block waits for its copies and MMAs in flight and records
// KS_ETIMEOUT.
constexpr int kNM = 128, kNN = 64, kNK = 32;     // tile rows, columns, K per stage
constexpr int kNEpiWarps = 4, kNSplitWarps = 4;  // warps 0-3 epilogue, 4-7 split
constexpr int kNProdWarp = 8, kNMmaWarp = 9;     // copies, MMAs (one thread each)
constexpr int kNThreads = 320;
constexpr int kNEpiThreads = 32 * kNEpiWarps, kNSplitThreads = 32 * kNSplitWarps;
constexpr int kNRaw = 6;                         // ring of A stages (raw, then hi in place)
constexpr int kNLo = 2;                          // lo buffers
constexpr int kNTileBytes = kNM * kNK * 4;       // 16 KiB: one A stage (raw, hi or lo)
constexpr int kNImgBytes = 2 * kNN * kNK * 4;    // 16 KiB: hi + lo of one coefficient stage
constexpr int kNMaxStages = 6;                   // K (padded per operand) <= 192
constexpr int kNCols = 2 * kNN;                  // tensor-memory columns: two accumulators
constexpr size_t kNSmem = (size_t)kNMaxStages * kNImgBytes +
                          (size_t)(kNRaw + kNLo) * kNTileBytes + 1024;
static_assert(kNTileBytes % (16 * kNSplitThreads) == 0, "split share");
constexpr uint32_t kIdescN64 = (1u << 4) | (2u << 7) | (2u << 10) |
                               ((uint32_t)(kNN >> 3) << 17) | ((uint32_t)(kNM >> 4) << 24);

struct Tc64Args {
  CUtensorMap map[3];          // A_i as (k_i, n) FP32, box (32, 128), 128-byte swizzle
  long long n, ntiles;
  int q, stages;
  int st_end[3];               // cumulative stage counts of the operands
  const float *img;
  const float *a3;             // A3 (n x q) for out2
  float *out, *out2;
  const double *rho_b;
  double *rho;
  double occ;
  int *status;
};

__device__ __forceinline__ void mma_tf32_n64(uint32_t tmem, uint64_t da, uint64_t db,
                                             uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(tmem), "l"(da), "l"(db), "r"(kIdescN64), "r"(acc));
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO),
// descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// byte offset of element (r, k) of a rows x 32 FP32 tile in the 128-byte
// swizzle (16-byte chunk k / 4 of row r at chunk (k / 4) ^ (r % 8))
__device__ __forceinline__ int sw128_offset(int r, int k) {
  return r * 128 + ((((k >> 2) ^ (r & 7))) << 4) + (k & 3) * 4;
}

// x = hi + lo with hi the TF32 value nearest to x (ties away from zero) and
// lo = x - hi exactly; |lo| <= 2^-11 |x|.
__device__ __forceinline__ void split_rn(float x, float &hi, float &lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

// 32 FP32 accumulator columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
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

__device__ __forceinline__ void cp_async16_zf(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(smem_u32(dst)), "l"(src),
               "r"(bytes) : "memory");
}

// Coefficient image of a narrow update: stage st belongs to operand i
// (st_end cumulative) and holds rows 32 j .. 32 j + 31 of s_i C_i (k_i x q
// FP32, a null C_i the identity; zero past k_i and q), as hi and lo 64 x 32
// tiles in the 128-byte swizzle, exactly as the kernel's shared memory
// holds them.
struct Img64 {
  const float *C[3];
  int k[3];
  float s[3];
  int st_end[3];
};

__global__ void combine_image64_kernel(int q, Img64 im, int stages, float *__restrict__ img) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int per_stage = kNN * kNK;
  if (e >= stages * per_stage) return;
  const int st = e / per_stage, within = e % per_stage;
  const int c = within / kNK, k = within % kNK;
  const int i = st < im.st_end[0] ? 0 : st < im.st_end[1] ? 1 : 2;
  const int r = (st - (i > 0 ? im.st_end[i - 1] : 0)) * kNK + k;
  float x = 0.f;
  if (c < q && r < im.k[i])
    x = im.s[i] * (im.C[i] ? im.C[i][(long long)r * q + c] : (r == c ? 1.f : 0.f));
  float hi, lo;
  split_rn(x, hi, lo);
  unsigned char *base = (unsigned char *)(img + (long long)st * 2 * per_stage);
  const int off = sw128_offset(c, k);
  *(float *)(base + off) = hi;
  *(float *)(base + kNImgBytes / 2 + off) = lo;
}

// Bounded wait on a phase of an mbarrier that also gives up once another
// role of the block has set *abort; a wait that runs out sets it.
__device__ __forceinline__ bool role_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  const uint32_t a = smem_u32(bar);
  for (long long spins = 0; spins < kSpinLimit; ++spins) {
    uint32_t done;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (*abort) return false;
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// Epilogue of 32 accumulator columns c0 .. c0 + 31 of one row: out, and with
// out2 the sum A3 + out and the row's share of the density, returned.
__device__ __forceinline__ float narrow_epilogue(const Tc64Args &ga, const uint32_t (&v)[32],
                                                 long long row, int c0) {
  const int q = ga.q;
  float dsum = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = c0 + 4 * j;
    if (c >= q || !KS_IN(row * q + c + 3, ga.n * q)) continue;
    const float4 y = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
    *reinterpret_cast<float4 *>(ga.out + row * q + c) = y;
    if (ga.out2) {
      const float4 a = *reinterpret_cast<const float4 *>(ga.a3 + row * q + c);
      *reinterpret_cast<float4 *>(ga.out2 + row * q + c) =
          make_float4(a.x + y.x, a.y + y.y, a.z + y.z, a.w + y.w);
      if (ga.rho) {
        dsum = fmaf(y.x, fmaf(2.f, a.x, y.x), dsum);
        dsum = fmaf(y.y, fmaf(2.f, a.y, y.y), dsum);
        dsum = fmaf(y.z, fmaf(2.f, a.z, y.z), dsum);
        dsum = fmaf(y.w, fmaf(2.f, a.w, y.w), dsum);
      }
    }
  }
  return dsum;
}

__global__ void __launch_bounds__(kNThreads, 1) combine_tc64_kernel(
    const __grid_constant__ Tc64Args ga) {
  extern __shared__ __align__(1024) unsigned char dyn_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)dyn_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *Bs = smem;                                       // coefficient image
  unsigned char *Ring = Bs + (size_t)kNMaxStages * kNImgBytes;    // A stages, hi in place
  unsigned char *Lo = Ring + (size_t)kNRaw * kNTileBytes;         // lo parts
  __shared__ __align__(8) uint64_t full[kNRaw];        // stage landed
  __shared__ __align__(8) uint64_t ready[kNRaw];       // stage split (kNSplitThreads arrivals)
  __shared__ __align__(8) uint64_t slot_free[kNRaw];   // stage's MMAs done: ring slot free
  __shared__ __align__(8) uint64_t lo_free[kNLo];      // stage's MMAs done: lo buffer free
  __shared__ __align__(8) uint64_t acc_full[2];        // tile's MMAs done
  __shared__ __align__(8) uint64_t acc_empty[2];       // tile's accumulator read
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int stages = ga.stages;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kNCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i)
      if (ga.st_end[i] > (i > 0 ? ga.st_end[i - 1] : 0)) prefetch_tensor_map(&ga.map[i]);
    for (int b = 0; b < kNRaw; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&ready[b], kNSplitThreads);
      mbar_init(&slot_free[b], 1);
    }
    for (int b = 0; b < kNLo; ++b) mbar_init(&lo_free[b], 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kNEpiThreads);
    }
    abort_flag = 0;
    fence_barrier_init();
  }
  // the coefficient image, once, made visible to the MMAs' reads
  for (int o = tid * 16; o < stages * kNImgBytes; o += kNThreads * 16)
    cp_async16_zf(Bs + o, (const unsigned char *)ga.img + o, 16u);
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  volatile int *abort = &abort_flag;
  const long long mine =
      ga.ntiles > blockIdx.x ? (ga.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long W = mine * stages;
  long long issued = 0;                      // producer: stages whose copy was issued

  if (warp < kNEpiWarps) {
    // epilogue: thread = one row of the tile (its warp's quarter of the
    // accumulator lanes), all q columns
    const int rl = 32 * warp + lane;
    for (long long t = 0; t < mine; ++t) {
      const int b = (int)(t & 1);
      const bool ok = role_wait(&acc_full[b], (uint32_t)((t >> 1) & 1), abort);
      if (!__all_sync(0xffffffffu, ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t v0[32], v1[32];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * kNN);
      tmem_ld32(ta, v0);
      tmem_ld32(ta + 32, v1);
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(&acc_empty[b]);            // the MMAs of tile t + 2 may overwrite it
      const long long row = (blockIdx.x + t * gridDim.x) * kNM + rl;
      if (row < ga.n) {
        const float d0 = narrow_epilogue(ga, v0, row, 0);
        const float d1 = narrow_epilogue(ga, v1, row, 32);
        if (ga.rho) ga.rho[row] = ga.rho_b[row] + ga.occ * (double)(d0 + d1);
      }
    }
  } else if (warp < kNEpiWarps + kNSplitWarps) {
    // split: x = hi + lo of each landed stage, hi in place in its ring
    // slot, lo into the stage's lo buffer once the MMAs that read it before
    // are done
    const int st = tid - kNEpiThreads;
    for (long long v = 0; v < W; ++v) {
      const int slot = (int)(v % kNRaw), lb = (int)(v % kNLo);
      if (v >= kNLo && !role_wait(&lo_free[lb], (uint32_t)((v / kNLo - 1) & 1), abort)) break;
      if (!role_wait(&full[slot], (uint32_t)((v / kNRaw) & 1), abort)) break;
      unsigned char *H = Ring + (size_t)slot * kNTileBytes, *L = Lo + (size_t)lb * kNTileBytes;
#pragma unroll
      for (int t = 0; t < kNTileBytes / 16 / kNSplitThreads; ++t) {
        const int o = (st + t * kNSplitThreads) * 16;
        if (!KS_IN(o + 15, kNTileBytes)) continue;
        const float4 x = *reinterpret_cast<const float4 *>(H + o);
        float4 h, l;
        split_rn(x.x, h.x, l.x); split_rn(x.y, h.y, l.y);
        split_rn(x.z, h.z, l.z); split_rn(x.w, h.w, l.w);
        *reinterpret_cast<float4 *>(H + o) = h;
        *reinterpret_cast<float4 *>(L + o) = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&ready[slot]);
    }
  } else if (warp == kNProdWarp) {
    // copies: stage v = one TMA tile of operand i at column 32 j, rows of
    // the tile, into ring slot v % kNRaw once the MMAs of stage v - kNRaw
    // have released it
    if (lane == 0) {
      for (long long v = 0; v < W; ++v) {
        const int slot = (int)(v % kNRaw);
        if (v >= kNRaw &&
            !role_wait(&slot_free[slot], (uint32_t)((v / kNRaw - 1) & 1), abort))
          break;
        const long long tile = blockIdx.x + (v / stages) * gridDim.x;
        const int s = (int)(v % stages);
        const int i = s < ga.st_end[0] ? 0 : s < ga.st_end[1] ? 1 : 2;
        const int j = s - (i > 0 ? ga.st_end[i - 1] : 0);
        mbar_arrive_expect_tx(&full[slot], (uint32_t)kNTileBytes);
        tma_load_2d(Ring + (size_t)slot * kNTileBytes, &ga.map[i], &full[slot], j * kNK,
                    (int)(tile * kNM));
        issued = v + 1;
      }
    }
    __syncwarp();
  } else if (warp == kNMmaWarp) {
    // MMAs: hi.hi + hi.lo + lo.hi of each split stage into the tile's
    // accumulator (two alternate, so the epilogue of tile t overlaps the
    // MMAs of tile t + 1)
    if (lane == 0) {
      long long v = 0;
      for (; v < W; ++v) {
        const long long t = v / stages;
        const int s = (int)(v % stages), b = (int)(t & 1);
        const int slot = (int)(v % kNRaw), lb = (int)(v % kNLo);
        if (s == 0 && t >= 2 &&
            !role_wait(&acc_empty[b], (uint32_t)((t / 2 - 1) & 1), abort))
          break;
        if (!role_wait(&ready[slot], (uint32_t)((v / kNRaw) & 1), abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ah = smem_u32(Ring + (size_t)slot * kNTileBytes);
        const uint32_t al = smem_u32(Lo + (size_t)lb * kNTileBytes);
        const uint32_t bh = smem_u32(Bs + (size_t)s * kNImgBytes), bl = bh + kNImgBytes / 2;
        const uint32_t d = tmem + (uint32_t)(b * kNN);
#pragma unroll
        for (int ks = 0; ks < kNK / 8; ++ks) {
          const uint32_t o = ks * 32;
          mma_tf32_n64(d, smem_desc_sw128(ah + o), smem_desc_sw128(bh + o),
                       (s > 0 || ks > 0) ? 1u : 0u);
          mma_tf32_n64(d, smem_desc_sw128(ah + o), smem_desc_sw128(bl + o), 1u);
          mma_tf32_n64(d, smem_desc_sw128(al + o), smem_desc_sw128(bh + o), 1u);
        }
        // slot_free last: its arrival means the others have arrived
        if (s == stages - 1) commit(&acc_full[b]);
        commit(&lo_free[lb]);
        commit(&slot_free[slot]);
      }
      // this thread's MMAs still running read the ring: wait for the last
      // (bounded, whatever the flag says)
      if (v > 0) mbar_wait_parity(&slot_free[(v - 1) % kNRaw], (uint32_t)(((v - 1) / kNRaw) & 1));
    }
    __syncwarp();
  }
  __syncthreads();
  if (*abort) {
    if (tid == 0) atomicCAS(ga.status, 0, (int)KS_ETIMEOUT);
    // copies still in flight write the ring: wait for the last use of each
    // slot (bounded)
    if (warp == kNProdWarp && lane == 0)
      for (long long u = issued > kNRaw ? issued - kNRaw : 0; u < issued; ++u)
        mbar_wait_parity(&full[u % kNRaw], (uint32_t)((u / kNRaw) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kNCols));
}

}  // namespace

ks_status configure_tc_kernels() {
  KS_CUDA_TRY(cudaFuncSetAttribute(combine_tc64_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNSmem));
  KS_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kTcSmem));
  KS_CUDA_TRY(cudaFuncSetAttribute(combine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kTcSmem));
  return KS_OK;
}

size_t tc_image_floats(int p) {
  return (size_t)((p + kTcN - 1) / kTcN) * ((2 * p + kTcK - 1) / kTcK) * 2 * kTcN * kTcK;
}

ks_status launch_combine_tc(Problem &P, const float *A1, int k1, const double *C1,
                            const float *A2, int k2, const double *C2, double alpha, double beta,
                            const float *Bm, float *out, int q) {
  const int K = k1 + (A2 ? k2 : 0);
  const int stages = (K + kTcK - 1) / kTcK;
  const long long img_len = (long long)((q + kTcN - 1) / kTcN) * stages * 2 * kTcN * kTcK;
  if ((size_t)img_len > P.tc_img_len) return set_error(KS_EINVAL, "combine_tc: image too large");
  {
    ProfScope ps_(P.stream, KP_REDUCE);
    const long long elems = img_len / 2;
    combine_image_kernel<<<(int)((elems + 255) / 256), 256, 0, P.stream>>>(
        q, k1, C1, A2 ? k2 : 0, C2, stages, P.tc_img);
  }
  KS_CUDA_TRY(cudaGetLastError());
  dim3 grid((unsigned)((P.n + kTcM - 1) / kTcM), (unsigned)((q + kTcN - 1) / kTcN));
  {
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * K,
                  (double)P.n * (K + q * (Bm ? 2 : 1)) * sizeof(float));
    combine_tc_kernel<<<grid, kTcThreads, kTcSmem, P.stream>>>(
        P.n, q, A1, k1, A2, A2 ? k2 : 0, P.tc_img, stages, (float)alpha, (float)beta, Bm, out,
        P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

// Chunks of the tensor-core Gram: one block per SM over all tiles (each
// block needs most of an SM's shared memory), at least 512 rows per chunk,
// and no more chunks than the partial buffer holds.
int gram_tc_chunks(const Problem &P, int pa, int qb) {
  const int tiles = ((pa + kTcM - 1) / kTcM) * ((qb + kTcN - 1) / kTcN);
  int chunks = (P.sms + tiles - 1) / tiles;
  const int maxc = (P.n + 511) / 512;
  if (chunks > maxc) chunks = maxc;
  const long long room = (long long)(P.partials_len / ((size_t)pa * qb));
  if (chunks > room) chunks = (int)room;
  if (chunks < 1) chunks = 1;
  return chunks;
}

ks_status launch_gram_tc(Problem &P, const float *A, int pa, const float *B, int qb,
                         double *part, int chunks) {
  const int tiles_a = (pa + kTcM - 1) / kTcM, tiles_b = (qb + kTcN - 1) / kTcN;
  long long rows_per = (P.n + chunks - 1) / chunks;
  rows_per = (rows_per + kTcK - 1) / kTcK * kTcK;
  {
    ProfScope ps_(P.stream, KP_GRAM, 2.0 * P.n * pa * qb, (double)P.n * (pa + qb) * sizeof(float));
    gram_tc_kernel<<<dim3(tiles_a * tiles_b, chunks), kTcThreads, kTcSmem, P.stream>>>(
        P.n, pa, qb, rows_per, tiles_b, A, B, part, P.dstatus);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

bool combine_tc64_applies(const Problem &P, int q, std::initializer_list<int> ks,
                          std::initializer_list<const void *> ptrs) {
  if (P.use_tc != 3 || q < 1 || q > kNN || q % 4) return false;
  int stages = 0;
  for (int k : ks) {
    if (k % 4) return false;
    stages += (k + kNK - 1) / kNK;
  }
  if (stages < 1 || stages > kNMaxStages) return false;
  for (const void *ptr : ptrs)
    if (reinterpret_cast<uintptr_t>(ptr) % 16) return false;
  return true;
}

ks_status launch_combine_tc64(Problem &P, int q, const float *A1, int k1, const float *C1,
                              float s1, const float *A2, int k2, const float *C2, float s2,
                              const float *A3, int k3, const float *C3, float s3, float *out,
                              float *out2, const double *rho_b, double *rho) {
  const float *A[3] = {A1, A2, A3};
  int k[3] = {k1, A2 ? k2 : 0, A3 ? k3 : 0};
  Img64 im{{C1, C2, C3}, {k[0], k[1], k[2]}, {s1, s2, s3}, {0, 0, 0}};
  Tc64Args ga{};
  int stages = 0;
  for (int i = 0; i < 3; ++i) {
    if (k[i] % 4) return set_error(KS_EINVAL, "combine_tc64: operand width not a multiple of 4");
    stages += (k[i] + kNK - 1) / kNK;
    im.st_end[i] = ga.st_end[i] = stages;
    if (k[i] > 0)
      KS_TRY(encode_tensor_map_2d_sw128(&ga.map[i], A[i], (uint64_t)P.n, (uint64_t)k[i],
                                        (uint32_t)kNM));
  }
  if (stages < 1 || stages > kNMaxStages ||
      (size_t)stages * kNImgBytes / sizeof(float) > P.tc_img_len)
    return set_error(KS_EINVAL, "combine_tc64: K above the image");
  // out2 = A3 + out reads A3 back row by row
  if (out2 && (k[2] != q || k[2] == 0))
    return set_error(KS_EINVAL, "combine_tc64: out2 needs A3 with q columns");
  if (out2 && (const void *)out == (const void *)A3)
    return set_error(KS_EINVAL, "combine_tc64: out must not alias A3 when out2 is formed");
  {
    ProfScope ps_(P.stream, KP_REDUCE);
    const int elems = stages * kNN * kNK;
    combine_image64_kernel<<<(elems + 255) / 256, 256, 0, P.stream>>>(q, im, stages, P.tc_img);
  }
  KS_CUDA_TRY(cudaGetLastError());
  ga.n = P.n;
  ga.ntiles = (P.n + kNM - 1) / kNM;
  ga.q = q;
  ga.stages = stages;
  ga.img = P.tc_img;
  ga.a3 = A3;
  ga.out = out;
  ga.out2 = out2;
  ga.rho_b = rho_b;
  ga.rho = rho;
  ga.occ = P.occ;
  ga.status = P.dstatus;
  long long grid = P.sms;
  if (grid > ga.ntiles) grid = ga.ntiles;
  const int K = k[0] + k[1] + k[2];
  {
    ProfScope ps_(P.stream, KP_COMBINE, 2.0 * P.n * q * K,
                  (double)P.n * (K + q * (out2 ? 2 : 1)) * sizeof(float));
    combine_tc64_kernel<<<(int)grid, kNThreads, kNSmem, P.stream>>>(ga);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

KS_OOB_READER(tc)

}  // namespace ks
