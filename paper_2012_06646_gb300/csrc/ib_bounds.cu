// ib_bounds.cu -- non-periodic ("bounded") dimensions.  Section 3.1 extends
// the grid so that every de facto cell holds a grid point and lets the grid
// indexing function # return the empty marker for the points outside the
// domain: they take no part in spreading or interpolation.  A bounded
// dimension of n nodes is handled on a periodic grid of n + 8 nodes with the
// same spacing: positions lie in [0, L], so a point's support reaches at most
// 4 nodes above the domain and 3 below it (wrapped to the top), and the two
// ghost ranges never meet.  Spreading runs on the extended grid and
// k_bounds_crop copies the domain's nodes out (the ghost nodes' sums are the
// dropped contributions); interpolation first fills the extended grid with
// the field and zero ghosts (k_bounds_pad).
#include "ib_internal.h"

namespace ibgb {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// One thread per domain node (all components): f = fx (or f + fx).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bounds_crop(const __grid_constant__ Job jb, int ncomp,
                                                          const T* __restrict__ fx, T* __restrict__ f,
                                                          int accumulate) {
  const long long nd = (long long)jb.nin[0] * jb.nin[1] * jb.nin[2];
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= nd * ncomp) return;
  const int a = (int)(i / nd);
  const long long r = i - a * nd;
  const int x = (int)(r % jb.nin[0]);
  const long long q = r / jb.nin[0];
  const int y = (int)(q % jb.nin[1]);
  const int z = (int)(q / jb.nin[1]);
  const T v = fx[a * jb.ncell + x + (long long)jb.n[0] * (y + (long long)jb.n[1] * z)];
  f[i] = accumulate ? f[i] + v : v;
}

// One thread per extended node (all components): ux = u inside the domain, 0 on ghosts.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bounds_pad(const __grid_constant__ Job jb, int ncomp,
                                                         const T* __restrict__ u, T* __restrict__ ux) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= jb.ncell * ncomp) return;
  const int a = (int)(i / jb.ncell);
  const long long r = i - a * jb.ncell;
  const int x = (int)(r % jb.n[0]);
  const long long q = r / jb.n[0];
  const int y = (int)(q % jb.n[1]);
  const int z = (int)(q / jb.n[1]);
  const bool in = x < jb.nin[0] && y < jb.nin[1] && z < jb.nin[2];
  const long long nd = (long long)jb.nin[0] * jb.nin[1] * jb.nin[2];
  ux[i] = in ? u[a * nd + x + (long long)jb.nin[0] * (y + (long long)jb.nin[1] * z)] : (T)0;
}

}  // namespace

cudaError_t launch_bounds_crop(const Job& jb, int ncomp, int dtype, const void* fx, void* f, bool accumulate,
                               cudaStream_t s) {
  const long long n = (long long)jb.nin[0] * jb.nin[1] * jb.nin[2] * ncomp;
  if (n == 0) return cudaSuccess;
  if (dtype == 0)
    k_bounds_crop<float><<<grid_for(n, kThreads), kThreads, 0, s>>>(jb, ncomp, (const float*)fx, (float*)f,
                                                                     accumulate ? 1 : 0);
  else
    k_bounds_crop<double><<<grid_for(n, kThreads), kThreads, 0, s>>>(jb, ncomp, (const double*)fx, (double*)f,
                                                                      accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_bounds_pad(const Job& jb, int ncomp, int dtype, const void* u, void* ux, cudaStream_t s) {
  const long long n = jb.ncell * ncomp;
  if (n == 0) return cudaSuccess;
  if (dtype == 0)
    k_bounds_pad<float><<<grid_for(n, kThreads), kThreads, 0, s>>>(jb, ncomp, (const float*)u, (float*)ux);
  else
    k_bounds_pad<double><<<grid_for(n, kThreads), kThreads, 0, s>>>(jb, ncomp, (const double*)u, (double*)ux);
  return cudaGetLastError();
}

}  // namespace ibgb
