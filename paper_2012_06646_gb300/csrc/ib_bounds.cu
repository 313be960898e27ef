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

constexpr int kThreads = 128;

constexpr unsigned kMaxGridYZ = 65535;

// Blocks over x-rows of the domain (y in grid y, (component a, z) in grid z,
// both strided), threads along x: f = fx (or f + fx).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bounds_crop(const __grid_constant__ Job jb, int ncomp,
                                                          const T* __restrict__ fx, T* __restrict__ f,
                                                          int accumulate) {
  const int x = blockIdx.x * kThreads + threadIdx.x;
  if (x >= jb.nin[0]) return;
  for (int az = blockIdx.z; az < jb.nin[2] * ncomp; az += gridDim.z) {
    const int a = az / jb.nin[2], z = az - a * jb.nin[2];
    for (int y = blockIdx.y; y < jb.nin[1]; y += gridDim.y) {
      const long long o = (((long long)a * jb.nin[2] + z) * jb.nin[1] + y) * jb.nin[0] + x;
      const T v = fx[a * jb.ncell + ((long long)z * jb.n[1] + y) * jb.n[0] + x];
      f[o] = accumulate ? f[o] + v : v;
    }
  }
}

// Blocks over x-rows of the extended grid (as k_bounds_crop): ux = u inside the
// domain, 0 on the ghost nodes.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bounds_pad(const __grid_constant__ Job jb, int ncomp,
                                                         const T* __restrict__ u, T* __restrict__ ux) {
  const int x = blockIdx.x * kThreads + threadIdx.x;
  if (x >= jb.n[0]) return;
  for (int az = blockIdx.z; az < jb.n[2] * ncomp; az += gridDim.z) {
    const int a = az / jb.n[2], z = az - a * jb.n[2];
    for (int y = blockIdx.y; y < jb.n[1]; y += gridDim.y) {
      const bool in = x < jb.nin[0] && y < jb.nin[1] && z < jb.nin[2];
      T v = (T)0;
      if (in) v = u[(((long long)a * jb.nin[2] + z) * jb.nin[1] + y) * jb.nin[0] + x];
      ux[a * jb.ncell + ((long long)z * jb.n[1] + y) * jb.n[0] + x] = v;
    }
  }
}

dim3 rows_grid(int nx, int ny, long long nzc) {
  return dim3((unsigned)((nx + kThreads - 1) / kThreads), (unsigned)(ny < (int)kMaxGridYZ ? ny : (int)kMaxGridYZ),
              (unsigned)(nzc < (long long)kMaxGridYZ ? nzc : (long long)kMaxGridYZ));
}

}  // namespace

cudaError_t launch_bounds_crop(const Job& jb, int ncomp, int dtype, const void* fx, void* f, bool accumulate,
                               cudaStream_t s) {
  const dim3 grid = rows_grid(jb.nin[0], jb.nin[1], (long long)jb.nin[2] * ncomp);
  if (dtype == 0)
    k_bounds_crop<float><<<grid, kThreads, 0, s>>>(jb, ncomp, (const float*)fx, (float*)f, accumulate ? 1 : 0);
  else
    k_bounds_crop<double><<<grid, kThreads, 0, s>>>(jb, ncomp, (const double*)fx, (double*)f, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_bounds_pad(const Job& jb, int ncomp, int dtype, const void* u, void* ux, cudaStream_t s) {
  const dim3 grid = rows_grid(jb.n[0], jb.n[1], (long long)jb.n[2] * ncomp);
  if (dtype == 0) k_bounds_pad<float><<<grid, kThreads, 0, s>>>(jb, ncomp, (const float*)u, (float*)ux);
  else k_bounds_pad<double><<<grid, kThreads, 0, s>>>(jb, ncomp, (const double*)u, (double*)ux);
  return cudaGetLastError();
}

}  // namespace ibgb
