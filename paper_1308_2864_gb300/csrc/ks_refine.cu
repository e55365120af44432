// Uniform refinement (Alg. AdpConOptM, Sec. 4.3, with every element refined
// and a fixed number of levels): Alg. ConOptM on the grids
// N_l = (N + 1) / 2^(levels-1-l) - 1, each level started from the Q1
// interpolant of the previous level's solution.
//
// Nested grids: the grid with N' = 2N + 1 interior nodes has spacing h/2 and
// fine node 2i + 1 is coarse node i, so a coarse trilinear field is exactly a
// fine one.  Its fine nodal values are (P1 x P1 x P1) X with the 1-D
// interpolation P1: weight 1 at coinciding nodes, 1/2 to each neighbour at
// midpoints, zero Dirichlet values beyond the ends.
#include <cstring>
#include <vector>

#include "ks_device.cuh"

namespace ks {

// Coarse nodes and weights behind fine index f along one axis: f odd is
// coarse node (f - 1) / 2 (weight 1); f even lies halfway between coarse
// nodes f/2 - 1 and f/2 (weight 1/2 each, a node outside the grid dropped).
__device__ __forceinline__ int prolong_axis(int f, int Nc, int c[2]) {
  if (f & 1) {
    c[0] = (f - 1) >> 1;
    return 1;
  }
  int m = 0;
  if (f / 2 - 1 >= 0) c[m++] = f / 2 - 1;
  if (f / 2 < Nc) c[m++] = f / 2;
  return m;
}

// One thread per fine entry (node, orbital; orbital fastest, so a warp
// reads and writes contiguous row segments).  The sums nest z innermost,
// then y, then x; every weight is 1 or 1/2, so the products are exact and
// each level rounds once.
template <typename T>
__global__ void prolong_kernel(int Nc, int p, const T *__restrict__ Xc, T *__restrict__ Xf) {
  const int Nf = 2 * Nc + 1;
  const long long total = (long long)Nf * Nf * Nf * p;
  const long long NNc = (long long)Nc * Nc;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(e % p);
    long long k = e / p;
    const int fx = (int)(k % Nf);
    k /= Nf;
    const int fy = (int)(k % Nf);
    const int fz = (int)(k / Nf);
    int cx[2], cy[2], cz[2];
    const int nx = prolong_axis(fx, Nc, cx), ny = prolong_axis(fy, Nc, cy),
              nz = prolong_axis(fz, Nc, cz);
    const T wx = (fx & 1) ? (T)1 : (T)0.5, wy = (fy & 1) ? (T)1 : (T)0.5,
            wz = (fz & 1) ? (T)1 : (T)0.5;
    T sx = 0;
    for (int a = 0; a < nx; ++a) {
      T sy = 0;
      for (int b = 0; b < ny; ++b) {
        T sz = 0;
        for (int c = 0; c < nz; ++c)
          sz += wz * Xc[((cz[c] * NNc) + (long long)cy[b] * Nc + cx[a]) * p + o];
        sy += wy * sz;
      }
      sx += wx * sy;
    }
    Xf[e] = sx;
  }
}

template <typename T>
static ks_status launch_prolong(int Nc, int p, const T *Xc, T *Xf, cudaStream_t s) {
  const int Nf = 2 * Nc + 1;
  const long long total = (long long)Nf * Nf * Nf * p;
  int dev = 0, sms = 0;
  KS_CUDA_TRY(cudaGetDevice(&dev));
  KS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  long long nb = (total + kThreads - 1) / kThreads;
  if (nb > 32LL * sms) nb = 32LL * sms;
  {
    ProfScope ps_(s, KP_OTHER, 0.0, (double)total * sizeof(T) * 9.0 / 8.0);
    prolong_kernel<T><<<(int)nb, kThreads, 0, s>>>(Nc, p, Xc, Xf);
  }
  KS_CUDA_TRY(cudaGetLastError());
  return KS_OK;
}

template <typename T>
static ks_status prolong_checked(int Nc, int p, const T *Xc, T *Xf, void *stream) {
  if (Nc < 1 || p < 1 || Nc > 1023) return set_error(KS_EINVAL, "prolong: Nc = %d, p = %d", Nc, p);
  if (!Xc || !Xf) return set_error(KS_EINVAL, "prolong: null pointer");
  const long long nf = (long long)(2 * Nc + 1) * (2 * Nc + 1) * (2 * Nc + 1) * p;
  const long long nc = (long long)Nc * Nc * Nc * p;
  const char *a = (const char *)Xc, *b = (const char *)Xf;
  if (a < b + nf * (long long)sizeof(T) && b < a + nc * (long long)sizeof(T))
    return set_error(KS_EINVAL, "prolong: input and output overlap");
  return launch_prolong<T>(Nc, p, Xc, Xf, (cudaStream_t)stream);
}

}  // namespace ks

using namespace ks;

extern "C" {

ks_status ks_prolong(int Nc, int p, const double *Xc, double *Xf, void *stream) {
  return prolong_checked<double>(Nc, p, Xc, Xf, stream);
}

ks_status ks_prolong_f32(int Nc, int p, const float *Xc, float *Xf, void *stream) {
  return prolong_checked<float>(Nc, p, Xc, Xf, stream);
}

ks_status ks_minimize_refine(const ks_problem_desc *desc, int levels, const double *X0_host,
                             const ks_opts *opts, double coarse_gtol, double *X_host_out,
                             ks_result *level_results) {
  if (!desc || !X0_host || !opts || !level_results) return set_error(KS_EINVAL, "null argument");
  KS_TRY(validate_desc(desc));
  if (levels < 1 || levels > 10) return set_error(KS_EINVAL, "levels = %d out of range", levels);
  if ((desc->N + 1) % (1 << (levels - 1)) != 0)
    return set_error(KS_EINVAL, "N + 1 = %d is not divisible by 2^(levels - 1)", desc->N + 1);
  std::vector<int> grid(levels);
  for (int l = 0; l < levels; ++l) grid[l] = (desc->N + 1) / (1 << (levels - 1 - l)) - 1;
  if (grid[0] < 2) return set_error(KS_EINVAL, "coarsest grid below 2 nodes per edge");
  if (!(coarse_gtol > 0.0)) return set_error(KS_EINVAL, "coarse_gtol must be positive");

  cudaStream_t s = (cudaStream_t)desc->stream;
  bool own = false;
  if (!s) {
    KS_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    own = true;
  }
  const int p = desc->p;
  double *X = nullptr;
  ks_problem *prob = nullptr;
  ks_status st = KS_OK;
  auto bytes_of = [&](int N) { return (size_t)N * N * N * p * sizeof(double); };
  for (int l = 0; l < levels && st == KS_OK; ++l) {
    ks_problem_desc d = *desc;
    d.N = grid[l];
    d.stream = s;
    ks_problem *next = nullptr;
    st = ks_problem_create(&d, &next);
    if (st != KS_OK) break;
    double *Xn = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&Xn, bytes_of(grid[l]), s);
    if (e != cudaSuccess) {
      ks_problem_destroy(next);
      st = cuda_error(e, "cudaMallocAsync");
      break;
    }
    if (l == 0) {
      e = cudaMemcpyAsync(Xn, X0_host, bytes_of(grid[0]), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync");
    } else {
      st = launch_prolong<double>(grid[l - 1], p, X, Xn, s);
      ks_problem_destroy(prob);
      prob = nullptr;
      cudaFreeAsync(X, s);
      X = nullptr;
    }
    X = Xn;
    prob = next;
    if (st != KS_OK) break;
    ks_opts o = *opts;
    o.resume = 0;
    if (l < levels - 1) o.gtol = coarse_gtol;
    st = ks_minimize(prob, X, &o, &level_results[l]);
    // a coarse level that stops at its iteration limit still seeds the next
    if (st == KS_ENOCONV && l < levels - 1) st = KS_OK;
  }
  if (X && X_host_out && (st == KS_OK || st == KS_ENOCONV)) {
    const cudaError_t e =
        cudaMemcpyAsync(X_host_out, X, bytes_of(grid[levels - 1]), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync");
  }
  if (X) cudaFreeAsync(X, s);
  if (prob) ks_problem_destroy(prob);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (st == KS_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamSynchronize");
  if (own) cudaStreamDestroy(s);
  return st;
}

}  // extern "C"
