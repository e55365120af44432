// 27-point Q1 stencils over blocks of orbitals (row-major n x p, orbital
// index fastest):
//
//   hamiltonian:  E_X = f K X + 2 f h^3 Diag(V_eff) X   (the derivative of
//                 Eq. EKS discretised, Sec. 2.3's E_X = H(X) X), M X, and
//                 the kinetic energy (f/2) sum X . K X
//   mass:         M X
//   mass_dots:    M D, ||D||_M^2 = sum D . M D and the Barzilai-Borwein
//                 traces of Eq. bb-1 in the M inner product.
//   hamiltonian, increment form (FP32 phase with X = X_b + delta): the
//                 stencil runs on delta and, with the base X_b, its gradient
//                 E_b = f K X_b + 2 f h^3 Diag(V_b) X_b and potential V_b,
//                 gives the change of the gradient from the base,
//                 e = E_X - E_b = f K delta + 2 f h^3 (Diag(V - V_b) X_b
//                 + Diag(V) delta), M delta, and the change of the kinetic
//                 energy, sum delta . (f K X_b + (f/2) K delta) with
//                 f K X_b = E_b - 2 f h^3 V_b X_b, accumulated with
//                 compensation; every rounding scales with delta or V - V_b.
//
// Plane-marching form.  For a plane z' and a node (x, y) let
//   c(z') = X(x, y, z'),  f(z') = sum of the 4 in-plane face neighbours,
//   e(z') = sum of the 4 in-plane corner neighbours.
// The 27-point neighbourhood of (x, y, z) splits into classes
//   centre = c(z), faces = f(z) + c(z-1) + c(z+1),
//   edges = e(z) + f(z-1) + f(z+1), corners = e(z-1) + e(z+1),
// and the Q1 coefficients depend only on the class (the stiffness face
// coefficient is zero).  A block owns a TX x TY tile of nodes and a chunk of
// PC orbitals, marches along z over a segment of planes, stages one plane
// (with a one-node halo) in shared memory per step, and keeps (c, f, e) of
// the last three planes in registers, so each plane sum is formed once and
// used by three output planes.  Consecutive threads take consecutive
// orbitals of one node, so every global access is a contiguous row segment.
//
// Two ways of staging a plane:
//   TMA (default when the row pitch p * sizeof(T) and the base address are
//     multiples of 16 bytes): the (TX+2) x (TY+2) x PC halo box of a plane is
//     one cp.async.bulk.tensor load into a ring of kStStages shared-memory
//     stages, issued kStStages planes ahead by one thread and completed on
//     an mbarrier; the zero Dirichlet halo comes from the copy's
//     out-of-bounds fill.  V_eff of the output plane is staged in the
//     working precision once per node.
//   plain loads (any p): all threads copy the halo box element by element.
#include <mutex>

#include "ks_async.cuh"
#include "ks_device.cuh"

namespace ks {

enum StencilKind : int { SK_HAM = 0, SK_MASS = 1, SK_MASS_DOT = 2, SK_MASS_BB = 3, SK_HAM_INC = 4 };

constexpr int kStThreads = 256;
constexpr int kStNodesPerThread = 4;

template <int PC>
struct StTile {
  static constexpr int G = kStThreads / PC;                // node groups
  static constexpr int NODES = G * kStNodesPerThread;      // nodes per tile
  static constexpr int TX = PC >= 16 ? 8 : 16;
  static constexpr int TY = NODES / TX;
  static constexpr int HX = TX + 2, HY = TY + 2;
};

struct StArgs {
  int N, p, zseg, tiles_x, tiles_y, chunks;
  StencilCoef c;
  double occ, h3;
  double kfac;                // factor of K X in E_X: occ, or mu occ (TFW kinetic)
  const void *A;              // input block (X or D)
  void *out1;                 // E_X (SK_HAM) or M A
  void *out2;                 // M X (SK_HAM, optional)
  const double *veff;
  const void *X, *MX, *Xp, *MXp, *Dp, *MDp;   // SK_MASS_BB; SK_HAM_INC: X = X_b, MX = E_b
  const double *veff_b;       // SK_HAM_INC: V_b
  double *part;               // block partials, channel-major
  int nb;                     // number of blocks (partials stride)
  double *red_out;            // reduced channels (scaled by red_scale)
  double red_scale;
  unsigned int *counter;
  int *status;                // device status word (TMA waits that give up)
  float cf[9];                // k0, ke, kc, m0, mf, me, mc, kfac, 2 occ h^3 rounded to FP32 (host)
};

// Coefficients in the working precision (FP32 ones rounded on the host: a
// per-thread conversion would be nine FP64-pipe instructions per thread).
template <typename T>
struct StCoefT {
  T k0, ke, kc, m0, mf, me, mc, kin, vscale;
  __device__ explicit StCoefT(const StArgs &a) {
    if constexpr (sizeof(T) == 4) {
      k0 = a.cf[0]; ke = a.cf[1]; kc = a.cf[2]; m0 = a.cf[3]; mf = a.cf[4];
      me = a.cf[5]; mc = a.cf[6]; kin = a.cf[7]; vscale = a.cf[8];
    } else {
      k0 = a.c.k0; ke = a.c.ke; kc = a.c.kc; m0 = a.c.m0; mf = a.c.mf;
      me = a.c.me; mc = a.c.mc; kin = a.kfac; vscale = 2.0 * a.occ * a.h3;
    }
  }
};

// Plain-load form of one block (vb = the block's index in the system's
// launch geometry); the single-system kernel and the batched kernel of a
// job table both run it.
template <typename T, int PC, int Kind>
__device__ __forceinline__ void stencil_plain_body(const StArgs &a, int vb) {
  using Tl = StTile<PC>;
  __shared__ T tile[Tl::HY * Tl::HX * PC];
  __shared__ double smem[33];
  const int N = a.N, p = a.p;
  // block -> (tile x, tile y, orbital chunk, z segment)
  int b = vb;
  const int txi = b % a.tiles_x; b /= a.tiles_x;
  const int tyi = b % a.tiles_y; b /= a.tiles_y;
  const int oc = b % a.chunks; b /= a.chunks;
  const int zs = b;
  const int x0 = txi * Tl::TX, y0 = tyi * Tl::TY;
  const int z0 = zs * a.zseg;
  const int z1 = min(z0 + a.zseg, N);
  const int lane = threadIdx.x % PC, grp = threadIdx.x / PC;
  const int o = oc * PC + lane;
  const bool ovalid = o < p;
  const T *A = (const T *)a.A;

  int lx[kStNodesPerThread], ly[kStNodesPerThread];
#pragma unroll
  for (int r = 0; r < kStNodesPerThread; ++r) {
    const int node = grp + r * Tl::G;
    lx[r] = node % Tl::TX;
    ly[r] = node / Tl::TX;
  }
  T c_old[kStNodesPerThread], f_old[kStNodesPerThread], e_old[kStNodesPerThread];
  T c_mid[kStNodesPerThread], f_mid[kStNodesPerThread], e_mid[kStNodesPerThread];

  // the halo box of the next plane travels in registers (pf) while the
  // current plane's outputs are formed; plane() stores it to the shared tile
  // and forms (c, f, e) of this thread's nodes
  constexpr int kBox = Tl::HY * Tl::HX * PC;
  constexpr int kPf = (kBox + kStThreads - 1) / kStThreads;
  T pf[kPf];
  auto fetch = [&](int zp) {
    const bool zok = zp >= 0 && zp < N;
#pragma unroll
    for (int i = 0; i < kPf; ++i) {
      const int t = threadIdx.x + i * kStThreads;
      const int l = t % PC, hn = t / PC;
      const int hx = hn % Tl::HX, hy = hn / Tl::HX;
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, go = oc * PC + l;
      T v = 0;
      if (t < kBox && zok && gx >= 0 && gx < N && gy >= 0 && gy < N && go < p)
        v = __ldg(A + (((long long)zp * N + gy) * N + gx) * p + go);
      pf[i] = v;
    }
  };
  auto plane = [&](T *c, T *f, T *e) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPf; ++i) {
      const int t = threadIdx.x + i * kStThreads;
      if (t < kBox) tile[t] = pf[i];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kStNodesPerThread; ++r) {
      const int hx = lx[r] + 1, hy = ly[r] + 1;
      auto at = [&](int dx, int dy) {
        const int ti = ((hy + dy) * Tl::HX + hx + dx) * PC + lane;
        return KS_IN(ti, kBox) ? tile[ti] : (T)0;
      };
      c[r] = at(0, 0);
      f[r] = (at(-1, 0) + at(1, 0)) + (at(0, -1) + at(0, 1));
      e[r] = (at(-1, -1) + at(1, -1)) + (at(-1, 1) + at(1, 1));
    }
  };

  fetch(z0 - 1);
  plane(c_old, f_old, e_old);
  fetch(z0);
  plane(c_mid, f_mid, e_mid);
  if (z0 < z1) fetch(z0 + 1);

  const StCoefT<T> cf(a);
  const T k0 = cf.k0, ke = cf.ke, kc = cf.kc;
  const T m0 = cf.m0, mf = cf.mf, me = cf.me, mc = cf.mc;
  const T kin = cf.kin, vscale = cf.vscale;
  T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;

  for (int z = z0; z < z1; ++z) {
    T c_new[kStNodesPerThread], f_new[kStNodesPerThread], e_new[kStNodesPerThread];
    plane(c_new, f_new, e_new);                    // plane z + 1
    if (z + 1 < z1) fetch(z + 2);                  // in flight during the outputs of plane z
#pragma unroll
    for (int r = 0; r < kStNodesPerThread; ++r) {
      const int gx = x0 + lx[r], gy = y0 + ly[r];
      const T centre = c_mid[r];
      const T faces = f_mid[r] + (c_old[r] + c_new[r]);
      const T edges = e_mid[r] + (f_old[r] + f_new[r]);
      const T corners = e_old[r] + e_new[r];
      const long long nodes = (long long)N * N * N;
      if (ovalid && gx < N && gy < N && KS_IN(((long long)z * N + gy) * N + gx, nodes) &&
          KS_IN((((long long)z * N + gy) * N + gx) * p + o, nodes * p)) {
        const long long k = ((long long)z * N + gy) * N + gx;
        const long long idx = k * p + o;
        const T m = m0 * centre + mf * faces + me * edges + mc * corners;
        if (Kind == SK_HAM) {
          const T kx = k0 * centre + ke * edges + kc * corners;
          ((T *)a.out1)[idx] = kin * kx + vscale * (T)a.veff[k] * centre;
          if (a.out2) ((T *)a.out2)[idx] = m;
          acc0 = fma(centre, kx, acc0);
        } else if (Kind == SK_HAM_INC) {
          const T kx = k0 * centre + ke * edges + kc * corners;
          const T xb = ((const T *)a.X)[idx], eb = ((const T *)a.MX)[idx];
          const T v = (T)a.veff[k], vb = (T)a.veff_b[k], dv = (T)(a.veff[k] - a.veff_b[k]);
          ((T *)a.out1)[idx] = kin * kx + vscale * (dv * xb + v * centre);
          if (a.out2) ((T *)a.out2)[idx] = m;
          // compensated sum of delta . (2 f K X_b + f K delta); acc1 holds the
          // running rounding error
          const T fkxb = eb - vscale * vb * xb;
          const T t = centre * ((T)2 * fkxb + kin * kx);
          const T y = t - acc1;
          const T sum = acc0 + y;
          acc1 = (sum - acc0) - y;
          acc0 = sum;
        } else {
          ((T *)a.out1)[idx] = m;
          if (Kind >= SK_MASS_DOT) acc0 = fma(centre, m, acc0);
          if (Kind == SK_MASS_BB) {
            const T dx = ((const T *)a.X)[idx] - ((const T *)a.Xp)[idx];
            const T dmx = ((const T *)a.MX)[idx] - ((const T *)a.MXp)[idx];
            const T dd = centre - ((const T *)a.Dp)[idx];
            const T dmd = m - ((const T *)a.MDp)[idx];
            acc1 = fma(dx, dmx, acc1);
            acc2 = fma(dx, dmd, acc2);
            acc3 = fma(dd, dmd, acc3);
          }
        }
      }
      c_old[r] = c_mid[r]; f_old[r] = f_mid[r]; e_old[r] = e_mid[r];
      c_mid[r] = c_new[r]; f_mid[r] = f_new[r]; e_mid[r] = e_new[r];
    }
  }
  if (Kind == SK_MASS) return;
  const double s0 =
      block_sum(Kind == SK_HAM_INC ? (double)acc0 - (double)acc1 : (double)acc0, smem);
  if (threadIdx.x == 0) a.part[vb] = s0;
  if (Kind == SK_MASS_BB) {
    const double s1 = block_sum((double)acc1, smem);
    const double s2 = block_sum((double)acc2, smem);
    const double s3 = block_sum((double)acc3, smem);
    if (threadIdx.x == 0) {
      a.part[a.nb + vb] = s1;
      a.part[2 * a.nb + vb] = s2;
      a.part[3 * a.nb + vb] = s3;
    }
  }
  grid_reduce_tail(a.part, a.nb, Kind == SK_MASS_BB ? 4 : 1, a.red_out, a.red_scale, a.counter,
                   smem);
}

template <typename T, int PC, int Kind>
__global__ void __launch_bounds__(kStThreads) stencil_kernel(StArgs a) {
  stencil_plain_body<T, PC, Kind>(a, blockIdx.x);
}

constexpr int kStStages = 3;

// Blocks read at the output node only (no halo), staged by TMA with the
// plane: SK_HAM_INC X_b and E_b; SK_MASS_BB X, MX, Xp, MXp, Dp, MDp in FP32
// (in FP64 the six boxes would not leave room for two blocks per SM: the
// kernel loads them from global memory at the output step instead).
template <typename T, int Kind>
constexpr int st_naux() {
  return Kind == SK_HAM_INC ? 2 : (Kind == SK_MASS_BB && sizeof(T) == 4) ? 6 : 0;
}

template <typename T, int PC, int Kind>
struct StRing {
  using Tl = StTile<PC>;
  static constexpr int NAUX = st_naux<T, Kind>();
  static constexpr int BOX = Tl::HY * Tl::HX * PC;                 // elements of one halo box
  static constexpr uint32_t BOX_BYTES = BOX * sizeof(T);
  static constexpr int HALO = ((BOX_BYTES + 127) / 128) * 128 / sizeof(T);   // 128-byte aligned
  static constexpr int AUXB = Tl::TY * Tl::TX * PC;                // elements of one node box
  static constexpr uint32_t AUX_BYTES = AUXB * sizeof(T);
  static constexpr int AUX = ((AUX_BYTES + 127) / 128) * 128 / sizeof(T);
  static constexpr int STAGE = HALO + NAUX * AUX;
  // the stages plus slack to align the ring to 128 bytes at run time
  static constexpr size_t SMEM = (size_t)kStStages * STAGE * sizeof(T) + 128;
};

struct StTmaArgs {
  CUtensorMap map;            // (orbital, x, y, z) view of the input block
  CUtensorMap aux[6];         // the same views of the node-local inputs (st_naux of them)
  StArgs a;
};

template <typename T, int PC, int Kind>
__global__ void __launch_bounds__(kStThreads, 2) stencil_tma_kernel(const __grid_constant__ StTmaArgs ta) {
  using Tl = StTile<PC>;
  using Rg = StRing<T, PC, Kind>;
  constexpr int TXY = Tl::TX * Tl::TY;
  constexpr int NAUX = Rg::NAUX;
  static_assert(TXY <= kStThreads, "one V_eff loader per node");
  extern __shared__ __align__(128) unsigned char st_ring_raw[];
  T *ring = reinterpret_cast<T *>(st_ring_raw + ((128u - (smem_addr(st_ring_raw) & 127u)) & 127u));
  __shared__ __align__(8) uint64_t full[kStStages];
  __shared__ T vs[3][TXY];
  // SK_HAM_INC: V_b and V - V_b (formed in FP64) of the same planes
  __shared__ T vbs[Kind == SK_HAM_INC ? 3 : 1][Kind == SK_HAM_INC ? TXY : 1];
  __shared__ T dvs[Kind == SK_HAM_INC ? 3 : 1][Kind == SK_HAM_INC ? TXY : 1];
  __shared__ double smem[33];
  const StArgs &a = ta.a;
  const int N = a.N, p = a.p;
  int b = blockIdx.x;
  const int txi = b % a.tiles_x; b /= a.tiles_x;
  const int tyi = b % a.tiles_y; b /= a.tiles_y;
  const int oc = b % a.chunks; b /= a.chunks;
  const int zs = b;
  const int x0 = txi * Tl::TX, y0 = tyi * Tl::TY;
  const int z0 = zs * a.zseg;
  const int z1 = min(z0 + a.zseg, N);
  const int nplanes = z1 - z0 + 2;          // planes z0 - 1 .. z1
  const int lane = threadIdx.x % PC, grp = threadIdx.x / PC;
  const int o = oc * PC + lane;
  const bool ovalid = o < p;

  // stage q holds the halo box of plane z0 - 1 + q and, from q = 2 on, the
  // node boxes of the output plane of step q (z0 - 2 + q)
  auto load_stage = [&](int q) {
    T *dst = ring + (q % kStStages) * Rg::STAGE;
    uint64_t *bar = &full[q % kStStages];
    const bool with_aux = NAUX > 0 && q >= 2;
    mbar_arrive_expect_tx(bar, Rg::BOX_BYTES + (with_aux ? NAUX * Rg::AUX_BYTES : 0u));
    tma_load_4d(dst, &ta.map, bar, oc * PC, x0 - 1, y0 - 1, z0 - 1 + q);
    if (with_aux)
#pragma unroll
      for (int i = 0; i < NAUX; ++i)
        tma_load_4d(dst + Rg::HALO + i * Rg::AUX, &ta.aux[i], bar, oc * PC, x0, y0, z0 - 2 + q);
  };
  if (threadIdx.x == 0) {
    prefetch_tensor_map(&ta.map);
#pragma unroll
    for (int i = 0; i < NAUX; ++i) prefetch_tensor_map(&ta.aux[i]);
#pragma unroll
    for (int st = 0; st < kStStages; ++st) mbar_init(&full[st], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < kStStages && q < nplanes; ++q) load_stage(q);

  int lx[kStNodesPerThread], ly[kStNodesPerThread];
#pragma unroll
  for (int r = 0; r < kStNodesPerThread; ++r) {
    const int node = grp + r * Tl::G;
    lx[r] = node % Tl::TX;
    ly[r] = node / Tl::TX;
  }
  // V_eff of plane z0 - 1 + q is read one iteration ahead by the thread that
  // owns the node, converted once and kept in vs[q % 3]
  const int vx = x0 + (int)threadIdx.x % Tl::TX, vy = y0 + (int)threadIdx.x / Tl::TX;
  constexpr bool kHam = Kind == SK_HAM || Kind == SK_HAM_INC;
  const bool vown = kHam && (int)threadIdx.x < TXY && vx < N && vy < N;
  double vreg = 0.0, vbreg = 0.0;
  const long long nodes = (long long)N * N * N;
  if (vown && z0 >= 1 && KS_IN(((long long)(z0 - 1) * N + vy) * N + vx, nodes)) {
    vreg = a.veff[((long long)(z0 - 1) * N + vy) * N + vx];
    if (Kind == SK_HAM_INC) vbreg = a.veff_b[((long long)(z0 - 1) * N + vy) * N + vx];
  }

  const StCoefT<T> cf(a);
  T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
  T c_old[kStNodesPerThread], f_old[kStNodesPerThread], e_old[kStNodesPerThread];
  T c_mid[kStNodesPerThread], f_mid[kStNodesPerThread], e_mid[kStNodesPerThread];
  int failed_at = -1;
  for (int q = 0; q < nplanes; ++q) {
    const int zp = z0 - 1 + q;
    const int st = q % kStStages;
    if (kHam && (int)threadIdx.x < TXY) {
      vs[q % 3][threadIdx.x] = (T)vreg;
      if (Kind == SK_HAM_INC) {
        vbs[q % 3][threadIdx.x] = (T)vbreg;
        dvs[q % 3][threadIdx.x] = (T)(vreg - vbreg);
      }
      vreg = 0.0;
      vbreg = 0.0;
      if (vown && zp + 1 < N && KS_IN(((long long)(zp + 1) * N + vy) * N + vx, nodes)) {
        vreg = a.veff[((long long)(zp + 1) * N + vy) * N + vx];
        if (Kind == SK_HAM_INC) vbreg = a.veff_b[((long long)(zp + 1) * N + vy) * N + vx];
      }
    }
    const bool got = mbar_wait_parity(&full[st], (uint32_t)((q / kStStages) & 1));
    const T *tile = ring + st * Rg::STAGE;
    T c_new[kStNodesPerThread], f_new[kStNodesPerThread], e_new[kStNodesPerThread];
#pragma unroll
    for (int r = 0; r < kStNodesPerThread; ++r) {
      const int hx = lx[r] + 1, hy = ly[r] + 1;
      auto at = [&](int dx, int dy) {
        const int ti = ((hy + dy) * Tl::HX + hx + dx) * PC + lane;
        return KS_IN(ti, Rg::BOX) ? tile[ti] : (T)0;
      };
      c_new[r] = at(0, 0);
      f_new[r] = (at(-1, 0) + at(1, 0)) + (at(0, -1) + at(0, 1));
      e_new[r] = (at(-1, -1) + at(1, -1)) + (at(-1, 1) + at(1, 1));
    }
    if (q >= 2) {
      const int z = zp - 1;
      const T *vz = vs[(q + 2) % 3];
      T bb[6][kStNodesPerThread];
      if constexpr (NAUX > 0) {
        // the node-local inputs of this output plane, staged with it
#pragma unroll
        for (int i = 0; i < NAUX; ++i)
#pragma unroll
          for (int r = 0; r < kStNodesPerThread; ++r)
          {
            const int ti = (ly[r] * Tl::TX + lx[r]) * PC + lane;
            bb[i][r] = KS_IN(ti, Rg::AUXB) ? tile[Rg::HALO + i * Rg::AUX + ti] : (T)0;
          }
      } else if (Kind == SK_MASS_BB) {
        // all loads of the plane first, so they are in flight together
#pragma unroll
        for (int r = 0; r < kStNodesPerThread; ++r) {
          const int gx = x0 + lx[r], gy = y0 + ly[r];
          if (ovalid && gx < N && gy < N &&
              KS_IN((((long long)z * N + gy) * N + gx) * p + o, nodes * p)) {
            const long long idx = (((long long)z * N + gy) * N + gx) * p + o;
            bb[0][r] = ((const T *)a.X)[idx];
            bb[1][r] = ((const T *)a.MX)[idx];
            bb[2][r] = ((const T *)a.Xp)[idx];
            bb[3][r] = ((const T *)a.MXp)[idx];
            bb[4][r] = ((const T *)a.Dp)[idx];
            bb[5][r] = ((const T *)a.MDp)[idx];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kStNodesPerThread; ++r) {
        const int gx = x0 + lx[r], gy = y0 + ly[r];
        const T centre = c_mid[r];
        const T faces = f_mid[r] + (c_old[r] + c_new[r]);
        const T edges = e_mid[r] + (f_old[r] + f_new[r]);
        const T corners = e_old[r] + e_new[r];
        if (ovalid && gx < N && gy < N && KS_IN(((long long)z * N + gy) * N + gx, nodes) &&
            KS_IN((((long long)z * N + gy) * N + gx) * p + o, nodes * p)) {
          const long long k = ((long long)z * N + gy) * N + gx;
          const long long idx = k * p + o;
          const T m = cf.m0 * centre + cf.mf * faces + cf.me * edges + cf.mc * corners;
          if (Kind == SK_HAM) {
            const T kx = cf.k0 * centre + cf.ke * edges + cf.kc * corners;
            ((T *)a.out1)[idx] = cf.kin * kx + cf.vscale * vz[ly[r] * Tl::TX + lx[r]] * centre;
            if (a.out2) ((T *)a.out2)[idx] = m;
            acc0 = fma(centre, kx, acc0);
          } else if (Kind == SK_HAM_INC) {
            const T kx = cf.k0 * centre + cf.ke * edges + cf.kc * corners;
            const T xb = bb[0][r], eb = bb[1][r];
            const int nd = ly[r] * Tl::TX + lx[r];
            const int pl = (q + 2) % 3;
            const T v = vz[nd], vb = vbs[pl][nd], dv = dvs[pl][nd];
            ((T *)a.out1)[idx] = cf.kin * kx + cf.vscale * (dv * xb + v * centre);
            if (a.out2) ((T *)a.out2)[idx] = m;
            const T fkxb = eb - cf.vscale * vb * xb;
            const T t = centre * ((T)2 * fkxb + cf.kin * kx);
            const T y = t - acc1;
            const T sum = acc0 + y;
            acc1 = (sum - acc0) - y;
            acc0 = sum;
          } else {
            ((T *)a.out1)[idx] = m;
            if (Kind >= SK_MASS_DOT) acc0 = fma(centre, m, acc0);
            if (Kind == SK_MASS_BB) {
              const T dx = bb[0][r] - bb[2][r];
              const T dmx = bb[1][r] - bb[3][r];
              const T dd = centre - bb[4][r];
              const T dmd = m - bb[5][r];
              acc1 = fma(dx, dmx, acc1);
              acc2 = fma(dx, dmd, acc2);
              acc3 = fma(dd, dmd, acc3);
            }
          }
        }
      }
    }
    // every thread is done with this stage: refill it kStStages planes ahead
    if (__syncthreads_or(!got)) {
      failed_at = q;
      break;
    }
    if (threadIdx.x == 0 && q + kStStages < nplanes) load_stage(q + kStStages);
#pragma unroll
    for (int r = 0; r < kStNodesPerThread; ++r) {
      c_old[r] = c_mid[r]; f_old[r] = f_mid[r]; e_old[r] = e_mid[r];
      c_mid[r] = c_new[r]; f_mid[r] = f_new[r]; e_mid[r] = e_new[r];
    }
  }
  if (failed_at >= 0) {
    // record the timeout, give the copies still in flight a bounded wait,
    // and still take part in the reduction so that its counter re-arms
    if (threadIdx.x == 0) {
      atomicCAS(a.status, 0, (int)KS_ETIMEOUT);
      for (int q = failed_at; q < failed_at + kStStages && q < nplanes; ++q)
        mbar_wait_parity(&full[q % kStStages], (uint32_t)((q / kStStages) & 1));
    }
    acc0 = acc1 = acc2 = acc3 = 0;
  }
  if (Kind == SK_MASS) return;
  const double s0 =
      block_sum(Kind == SK_HAM_INC ? (double)acc0 - (double)acc1 : (double)acc0, smem);
  if (threadIdx.x == 0) a.part[blockIdx.x] = s0;
  if (Kind == SK_MASS_BB) {
    const double s1 = block_sum((double)acc1, smem);
    const double s2 = block_sum((double)acc2, smem);
    const double s3 = block_sum((double)acc3, smem);
    if (threadIdx.x == 0) {
      a.part[a.nb + blockIdx.x] = s1;
      a.part[2 * a.nb + blockIdx.x] = s2;
      a.part[3 * a.nb + blockIdx.x] = s3;
    }
  }
  grid_reduce_tail(a.part, a.nb, Kind == SK_MASS_BB ? 4 : 1, a.red_out, a.red_scale, a.counter,
                   smem);
}

// Geometry of a launch: tiles, orbital chunks and z segments; the number of
// segments is lowered until the block partials (nchan per block) fit.
template <int PC>
static ks_status stencil_geometry(const Problem &P, int nchan, StArgs &a, int planes = 0) {
  using Tl = StTile<PC>;
  a.N = P.N;
  a.p = P.p;
  a.tiles_x = (P.N + Tl::TX - 1) / Tl::TX;
  a.tiles_y = (P.N + Tl::TY - 1) / Tl::TY;
  a.chunks = (P.p + PC - 1) / PC;
  const long long base = (long long)a.tiles_x * a.tiles_y * a.chunks;
  // aim for about 8 blocks per SM, with segments of at least 8 planes (or
  // segments of `planes` planes when given)
  long long segs = (8LL * P.sms + base - 1) / base;
  const long long maxsegs = (P.N + 7) / 8;
  if (segs > maxsegs) segs = maxsegs;
  if (planes > 0) segs = (P.N + planes - 1) / planes;
  if (segs < 1) segs = 1;
  for (;;) {
    a.zseg = (int)((P.N + segs - 1) / segs);
    const long long used = (P.N + a.zseg - 1) / a.zseg;
    const long long nb = base * used;
    if (nchan == 0 || (size_t)(nb * nchan) <= P.partials_len) {
      if (nb > 0x7fffffffLL) return set_error(KS_EINVAL, "stencil: grid too large");
      a.nb = (int)nb;
      return KS_OK;
    }
    if (used == 1) return set_error(KS_EINVAL, "stencil: partial buffer too small");
    segs = used / 2;
  }
}

// TMA form of one launch; false (and nothing launched) when the input
// cannot be described by a tensor map (row pitch or base address not a
// multiple of 16 bytes).
template <typename T, int PC, int Kind>
static bool stencil_launch_tma(Problem &P, const StArgs &a, int cls, double flops, double bytes,
                               ks_status *st) {
  using Tl = StTile<PC>;
  using Rg = StRing<T, PC, Kind>;
  *st = KS_OK;
  const void *aux[6] = {a.X, a.MX, a.Xp, a.MXp, a.Dp, a.MDp};
  if (!P.use_tma || ((size_t)P.p * sizeof(T)) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(a.A) % 16 != 0)
    return false;
  for (int i = 0; i < Rg::NAUX; ++i)
    if (!aux[i] || reinterpret_cast<uintptr_t>(aux[i]) % 16 != 0) return false;
  StTmaArgs ta;
  ta.a = a;
  const uint64_t dims[4] = {(uint64_t)P.p, (uint64_t)P.N, (uint64_t)P.N, (uint64_t)P.N};
  const uint32_t box[4] = {(uint32_t)PC, (uint32_t)Tl::HX, (uint32_t)Tl::HY, 1u};
  const uint32_t nbox[4] = {(uint32_t)PC, (uint32_t)Tl::TX, (uint32_t)Tl::TY, 1u};
  if (encode_tensor_map_4d(&ta.map, a.A, (int)sizeof(T), dims, box) != KS_OK) return false;
  for (int i = 0; i < Rg::NAUX; ++i)
    if (encode_tensor_map_4d(&ta.aux[i], aux[i], (int)sizeof(T), dims, nbox) != KS_OK)
      return false;
  // the ring plus the static shared memory (mbarriers, V_eff planes,
  // reduction scratch: up to ~10 KiB) for two blocks per SM; the kernel
  // opts in to the ring's size once
  static_assert(Rg::SMEM + 10 * 1024 <= 113 * 1024, "two blocks of the ring fit an SM");
  {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
      attr = cudaFuncSetAttribute(stencil_tma_kernel<T, PC, Kind>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Rg::SMEM);
    });
    if (attr != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  }
  {
    ProfScope ps_(P.stream, cls, flops, bytes);
    stencil_tma_kernel<T, PC, Kind><<<a.nb, kStThreads, Rg::SMEM, P.stream>>>(ta);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) *st = cuda_error(e, "stencil_tma_kernel");
  return true;
}

template <typename T, int PC, int Kind>
static ks_status stencil_launch_pc(Problem &P, StArgs &a, int nchan, double flops, double bytes) {
  KS_TRY(stencil_geometry<PC>(P, nchan, a));
  a.c = q1_coefficients(P.h);
  if (P.mass == KS_MASS_LUMPED) {      // row sums of M: h^3 on the centre
    a.c.m0 = P.h * P.h * P.h;
    a.c.mf = a.c.me = a.c.mc = 0.0;
  }
  const double cd[9] = {a.c.k0, a.c.ke, a.c.kc, a.c.m0, a.c.mf, a.c.me, a.c.mc, a.kfac,
                        2.0 * a.occ * a.h3};
  for (int i = 0; i < 9; ++i) a.cf[i] = (float)cd[i];
  a.part = P.partials;
  a.counter = P.red_counter;
  a.status = P.dstatus;
  const int cls = (Kind == SK_HAM || Kind == SK_HAM_INC) ? KP_HAMILTONIAN : KP_MASS;
  ks_status st;
  // one amplitude (PC = 1, p = 1) has an 8-byte row pitch, which no tensor
  // map can describe: plain staging only
  if constexpr (PC >= 4)
    if (stencil_launch_tma<T, PC, Kind>(P, a, cls, flops, bytes, &st)) return st;
  {
    ProfScope ps_(P.stream, cls, flops, bytes);
    stencil_kernel<T, PC, Kind><<<a.nb, kStThreads, 0, P.stream>>>(a);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template <typename T, int Kind>
static ks_status stencil_launch(Problem &P, StArgs &a, int nchan, double flops, double bytes) {
  if (P.p >= 32) return stencil_launch_pc<T, 32, Kind>(P, a, nchan, flops, bytes);
  if (P.p >= 16) return stencil_launch_pc<T, 16, Kind>(P, a, nchan, flops, bytes);
  if (P.p >= 8) return stencil_launch_pc<T, 8, Kind>(P, a, nchan, flops, bytes);
  if (P.p == 1) return stencil_launch_pc<T, 1, Kind>(P, a, nchan, flops, bytes);
  return stencil_launch_pc<T, 4, Kind>(P, a, nchan, flops, bytes);
}

template <typename T>
ks_status launch_hamiltonian(Problem &P, const T *X, const double *veff, T *EX, T *MX,
                             double *ekin_out) {
  StArgs a{};
  a.occ = P.occ;
  a.kfac = P.occ * P.kin_w;
  a.h3 = P.h * P.h * P.h;
  a.A = X;
  a.out1 = EX;
  a.out2 = MX;
  a.veff = veff;
  a.red_out = ekin_out;
  a.red_scale = 0.5 * a.kfac;
  const double total = (double)P.n * P.p;
  return stencil_launch<T, SK_HAM>(P, a, 1, 27.0 * total,
                                   total * sizeof(T) * (MX ? 3 : 2) + 8.0 * P.n);
}

ks_status launch_hamiltonian_inc(Problem &P, const float *d, const double *veff,
                                 const double *veff_b, const float *xb, const float *eb,
                                 float *e, float *Md, double *dkin_out) {
  StArgs a{};
  a.occ = P.occ;
  a.kfac = P.occ * P.kin_w;
  a.h3 = P.h * P.h * P.h;
  a.A = d;
  a.out1 = e;
  a.out2 = Md;
  a.veff = veff;
  a.veff_b = veff_b;
  a.X = xb;
  a.MX = eb;
  a.red_out = dkin_out;
  a.red_scale = 0.5;
  const double total = (double)P.n * P.p;
  return stencil_launch<float, SK_HAM_INC>(P, a, 1, 33.0 * total,
                                           total * sizeof(float) * (Md ? 5 : 4) + 8.0 * P.n);
}

template <typename T>
ks_status launch_mass(Problem &P, const T *X, T *MX) {
  StArgs a{};
  a.A = X;
  a.out1 = MX;
  const double total = (double)P.n * P.p;
  return stencil_launch<T, SK_MASS>(P, a, 0, 21.0 * total, 2.0 * total * sizeof(T));
}

template <typename T>
ks_status launch_mass_dots(Problem &P, const T *D, T *MD, const T *X, const T *MX,
                           const BBPrevT<T> *prev, double *out4) {
  StArgs a{};
  a.A = D;
  a.out1 = MD;
  a.red_out = out4;
  a.red_scale = 1.0;
  const double total = (double)P.n * P.p;
  if (prev) {
    a.X = X;
    a.MX = MX;
    a.Xp = prev->X;
    a.MXp = prev->MX;
    a.Dp = prev->D;
    a.MDp = prev->MD;
    return stencil_launch<T, SK_MASS_BB>(P, a, 4, 31.0 * total, 8.0 * total * sizeof(T));
  }
  return stencil_launch<T, SK_MASS_DOT>(P, a, 1, 23.0 * total, 2.0 * total * sizeof(T));
}

// ---------------------------------------------------------------- batched
// Slots of one batched stencil launch (BJob::blk indices, -1 = none).
struct StSlots {
  int a, o1, o2, x, mx, xp, mxp, dp, mdp;
};

template <typename T, int PC, int Kind>
__global__ void __launch_bounds__(kStThreads) stencil_batch_kernel(
    const BJob *__restrict__ jobs, const int *__restrict__ start, int J,
    const unsigned char *__restrict__ active, StSlots sl) {
  const int j = batch_job_of(start, J, blockIdx.x);
  if (!active[j]) return;
  const BJob &b = jobs[j];
  StArgs a;
  a.N = b.N;
  a.p = b.p;
  a.zseg = b.st_zseg;
  a.tiles_x = b.st_tiles_x;
  a.tiles_y = b.st_tiles_y;
  a.chunks = b.st_chunks;
  a.c.k0 = b.qc[0]; a.c.kf = b.qc[1]; a.c.ke = b.qc[2]; a.c.kc = b.qc[3];
  a.c.m0 = b.qc[4]; a.c.mf = b.qc[5]; a.c.me = b.qc[6]; a.c.mc = b.qc[7];
#pragma unroll
  for (int i = 0; i < 9; ++i) a.cf[i] = b.qcf[i];
  a.occ = b.occ;
  a.kfac = b.occ;
  a.h3 = b.h3;
  a.A = b.blk[sl.a];
  a.out1 = b.blk[sl.o1];
  a.out2 = sl.o2 >= 0 ? b.blk[sl.o2] : nullptr;
  a.veff = b.veff;
  if (Kind == SK_MASS_BB) {
    a.X = b.blk[sl.x];
    a.MX = b.blk[sl.mx];
    a.Xp = b.blk[sl.xp];
    a.MXp = b.blk[sl.mxp];
    a.Dp = b.blk[sl.dp];
    a.MDp = b.blk[sl.mdp];
  }
  a.part = b.partials;
  a.nb = b.st_nb;
  a.red_out = b.scal + (Kind == SK_HAM ? SC_EKIN : SC_DNORM2);
  a.red_scale = Kind == SK_HAM ? 0.5 * b.occ : 1.0;
  a.counter = b.red_counter;
  a.status = b.status;
  stencil_plain_body<T, PC, Kind>(a, blockIdx.x - start[j]);
}

template <typename T, int Kind>
static ks_status stencil_batch_launch(Batch &B, const StSlots &sl) {
  const int maps[4] = {BM_ST4, BM_ST8, BM_ST16, BM_ST32};
  const int cls = Kind == SK_HAM ? KP_HAMILTONIAN : KP_MASS;
  for (int c = 0; c < 4; ++c) {
    const int nb = B.total(maps[c]);
    if (nb == 0) continue;
    {
      ProfScope ps_(B.stream, cls);
      const int *st = B.map(maps[c]);
      if (c == 0) stencil_batch_kernel<T, 4, Kind><<<nb, kStThreads, 0, B.stream>>>(B.jobs_dev, st, B.J, B.active_dev, sl);
      else if (c == 1) stencil_batch_kernel<T, 8, Kind><<<nb, kStThreads, 0, B.stream>>>(B.jobs_dev, st, B.J, B.active_dev, sl);
      else if (c == 2) stencil_batch_kernel<T, 16, Kind><<<nb, kStThreads, 0, B.stream>>>(B.jobs_dev, st, B.J, B.active_dev, sl);
      else stencil_batch_kernel<T, 32, Kind><<<nb, kStThreads, 0, B.stream>>>(B.jobs_dev, st, B.J, B.active_dev, sl);
    }
    KS_CUDA_TRY(cudaGetLastError());
  }
  return KS_OK;
}

template <typename T>
ks_status batch_hamiltonian(Batch &B, int sX, int sEX, int sMX) {
  const StSlots sl{sX, sEX, sMX, -1, -1, -1, -1, -1, -1};
  return stencil_batch_launch<T, SK_HAM>(B, sl);
}

template <typename T>
ks_status batch_mass(Batch &B, int sX, int sMX) {
  const StSlots sl{sX, sMX, -1, -1, -1, -1, -1, -1, -1};
  return stencil_batch_launch<T, SK_MASS>(B, sl);
}

template <typename T>
ks_status batch_mass_dots(Batch &B, int sD, int sMD, int sX, int sMX, int sXp, int sMXp, int sDp,
                          int sMDp) {
  const StSlots sl{sD, sMD, -1, sX, sMX, sXp, sMXp, sDp, sMDp};
  if (sXp >= 0) return stencil_batch_launch<T, SK_MASS_BB>(B, sl);
  return stencil_batch_launch<T, SK_MASS_DOT>(B, sl);
}

// Per job: PC class of its p and the block geometry of that class (room for
// four reduction channels in its partials).
ks_status batch_stencil_geometry(Batch &B) {
  const int planes = B.tune.st_planes;
  for (int j = 0; j < B.J; ++j) {
    Problem &P = B.probs[j]->P;
    BJob &b = B.jobs_host[j];
    StArgs a{};
    if (P.p >= 32) KS_TRY(stencil_geometry<32>(P, 4, a, planes));
    else if (P.p >= 16) KS_TRY(stencil_geometry<16>(P, 4, a, planes));
    else if (P.p >= 8) KS_TRY(stencil_geometry<8>(P, 4, a, planes));
    else KS_TRY(stencil_geometry<4>(P, 4, a, planes));
    b.st_zseg = a.zseg;
    b.st_tiles_x = a.tiles_x;
    b.st_tiles_y = a.tiles_y;
    b.st_chunks = a.chunks;
    b.st_nb = a.nb;
  }
  return KS_OK;
}

#define KS_BINST(T)                                                                        \
  template ks_status batch_hamiltonian<T>(Batch &, int, int, int);                         \
  template ks_status batch_mass<T>(Batch &, int, int);                                     \
  template ks_status batch_mass_dots<T>(Batch &, int, int, int, int, int, int, int, int);
KS_BINST(double)
KS_BINST(float)
#undef KS_BINST

#define KS_INST(T)                                                                        \
  template ks_status launch_hamiltonian<T>(Problem &, const T *, const double *, T *, T *, \
                                           double *);                                    \
  template ks_status launch_mass<T>(Problem &, const T *, T *);                          \
  template ks_status launch_mass_dots<T>(Problem &, const T *, T *, const T *, const T *, \
                                         const BBPrevT<T> *, double *);
KS_INST(double)
KS_INST(float)
#undef KS_INST

KS_OOB_READER(stencil)

}  // namespace ks
