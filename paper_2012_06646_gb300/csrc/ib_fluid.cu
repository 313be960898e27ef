// ib_fluid.cu -- the Eulerian step (e) of the IB timestep of Section 2 on the
// periodic MAC grid: an unsteady Stokes solve with a backward-Euler viscous
// term and an exact discrete projection,
//
//   (rho/k) u + G p - mu L u = g,   D u = 0,   g = (rho/k) u_old + f,
//
// where D is the face-to-centre divergence, G the centre-to-face gradient and
// L the face Laplacian of the staggered grid (component a on the faces normal
// to e_a, Section 2).  Every operator is a circulant stencil, so the Fourier
// modes diagonalise it: with theta_b = 2 pi k_b / n_b,
//   D_b = (e^{i theta_b} - 1) / h_b = (2i / h_b) sin(theta_b / 2) e^{i theta_b / 2},
//   G_b = -conj(D_b),  L = -|d|^2 = -sum_b |D_b|^2,
// and per mode  p^ = -(D . g^) / |d|^2,
//   u^_a = (g^_a - conj(D_a) (D . g^) / |d|^2) / (rho/k + mu |d|^2).
// The mean mode keeps u^ = g^ / (rho/k) (zero when rho/k = 0).  The transforms
// are cuFFT (real-to-complex over x, then y, z), the per-mode arithmetic one
// kernel; sin^2 is used instead of 1 - cos so small wavenumbers keep their
// relative accuracy.
#include <cufft.h>
#include <math.h>
#include <string.h>

#include <new>

#include "../../include/ib.h"
#include "ib_internal.h"

namespace ibgb {
namespace {

constexpr int kThreads = 256;

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = cufftComplex; };
template <> struct Cplx<double> { using type = cufftDoubleComplex; };

struct FluidGeo {
  int dim, n[3];          // n[0] fastest (x); n[2] = 1 in 2-D
  int nh;                 // n[0] / 2 + 1 complex entries along x
  double h[3];            // spacing per dimension
  long long modes;        // modes per component
};

template <typename T>
__device__ __forceinline__ void sincospi_t(T x, T* s, T* c);
template <>
__device__ __forceinline__ void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }

// One thread per Fourier mode, all components of the mode at once.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_stokes_modes(typename Cplx<T>::type* __restrict__ c, FluidGeo g,
                                                           T rho_k, T mu, T inv_n) {
  const long long m = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (m >= g.modes) return;
  int k[3];
  k[0] = (int)(m % g.nh);
  const long long r = m / g.nh;
  k[1] = (int)(r % g.n[1]);
  k[2] = (D == 3) ? (int)(r / g.n[1]) : 0;
  // With (s_b, c_b) = (sin, cos)(pi k_b / n_b):  D_b = (2 s_b / h_b) (-s_b + i c_b).
  T dre[3], dim_[3], d2 = 0;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    T s, co;
    sincospi_t<T>((T)k[b] / (T)g.n[b], &s, &co);
    const T a = (T)2 * s / (T)g.h[b];
    dre[b] = -a * s;
    dim_[b] = a * co;
    d2 += a * a;                            // |D_b|^2 = (2 s_b / h_b)^2
  }
  typename Cplx<T>::type v[3];
#pragma unroll
  for (int a = 0; a < D; ++a) v[a] = c[a * g.modes + m];
  if (d2 == (T)0) {                                   // mean mode
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const T f = rho_k > (T)0 ? inv_n / rho_k : (T)0;
      v[a].x *= f;
      v[a].y *= f;
      c[a * g.modes + m] = v[a];
    }
    return;
  }
  // s = D . g^
  T sre = 0, sim = 0;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    sre += dre[b] * v[b].x - dim_[b] * v[b].y;
    sim += dre[b] * v[b].y + dim_[b] * v[b].x;
  }
  const T inv_d2 = (T)1 / d2;
  const T scale = inv_n / (rho_k + mu * d2);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    // conj(D_a) s = (dre - i dim)(sre + i sim)
    const T pre = dre[a] * sre + dim_[a] * sim;
    const T pim = dre[a] * sim - dim_[a] * sre;
    v[a].x = (v[a].x - pre * inv_d2) * scale;
    v[a].y = (v[a].y - pim * inv_d2) * scale;
    c[a * g.modes + m] = v[a];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_stokes_rhs(const T* __restrict__ f, const T* __restrict__ u_old,
                                                         T rho_k, T* __restrict__ g, long long n) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  g[i] = (u_old ? rho_k * u_old[i] : (T)0) + f[i];
}

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace
}  // namespace ibgb

using namespace ibgb;

struct ib_stokes_s {
  ib_plan_desc desc;
  FluidGeo geo;
  long long ncell;        // real entries per component
  cufftHandle fwd, inv;
  void* cbuf;             // complex modes of every component
  void* rbuf;             // real right-hand side g (every component)
};

extern "C" {

ib_status ib_stokes_create(const ib_plan_desc* desc, ib_stokes* out) {
  if (!out) return IB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || (desc->dim != 2 && desc->dim != 3) || desc->grid != IB_GRID_MAC || desc->ncomp != desc->dim ||
      (desc->dtype != IB_F32 && desc->dtype != IB_F64))
    return IB_ERR_INVALID_ARG;
  ib_stokes s = new (std::nothrow) ib_stokes_s;
  if (!s) return IB_ERR_OOM;
  memset(s, 0, sizeof(*s));
  s->desc = *desc;
  FluidGeo& g = s->geo;
  g.dim = desc->dim;
  long long ncell = 1;
  for (int b = 0; b < 3; ++b) {
    const bool live = b < desc->dim;
    g.n[b] = live ? desc->n[b] : 1;
    g.h[b] = live ? desc->L[b] / desc->n[b] : 1.0;
    if (live && (desc->n[b] < 2 || !(desc->L[b] > 0.0) || !isfinite(desc->L[b]))) {
      delete s;
      return IB_ERR_INVALID_ARG;
    }
    ncell *= g.n[b];
  }
  if (ncell > (1ll << 31)) {
    delete s;
    return IB_ERR_INVALID_ARG;
  }
  g.nh = g.n[0] / 2 + 1;
  g.modes = (long long)g.nh * g.n[1] * g.n[2];
  s->ncell = ncell;
  // Real layout [comp][n2][n1][n0]; the FFT dimensions slowest first.
  int dims[3], rank = desc->dim;
  if (rank == 3) { dims[0] = g.n[2]; dims[1] = g.n[1]; dims[2] = g.n[0]; }
  else { dims[0] = g.n[1]; dims[1] = g.n[0]; }
  const bool dbl = desc->dtype == IB_F64;
  const size_t eb = dbl ? 8 : 4;
  const cufftType tf = dbl ? CUFFT_D2Z : CUFFT_R2C, ti = dbl ? CUFFT_Z2D : CUFFT_C2R;
  if (cufftPlanMany(&s->fwd, rank, dims, nullptr, 1, (int)ncell, nullptr, 1, (int)g.modes, tf, desc->dim) !=
          CUFFT_SUCCESS ||
      cufftPlanMany(&s->inv, rank, dims, nullptr, 1, (int)g.modes, nullptr, 1, (int)ncell, ti, desc->dim) !=
          CUFFT_SUCCESS) {
    if (s->fwd) cufftDestroy(s->fwd);
    delete s;
    return IB_ERR_CUDA;
  }
  if (cudaMalloc(&s->cbuf, 2 * eb * (size_t)g.modes * desc->dim) != cudaSuccess ||
      cudaMalloc(&s->rbuf, eb * (size_t)ncell * desc->dim) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->cbuf);
    cufftDestroy(s->fwd);
    cufftDestroy(s->inv);
    delete s;
    return IB_ERR_OOM;
  }
  *out = s;
  return IB_OK;
}

ib_status ib_stokes_solve(ib_stokes s, const void* f, const void* u_old, void* u, double rho_over_k, double mu,
                          void* stream) {
  if (!s || !f || !u) return IB_ERR_INVALID_ARG;
  if (!(rho_over_k >= 0.0) || !(mu >= 0.0) || !isfinite(rho_over_k) || !isfinite(mu) ||
      (rho_over_k == 0.0 && mu == 0.0))
    return IB_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cufftSetStream(s->fwd, st) != CUFFT_SUCCESS || cufftSetStream(s->inv, st) != CUFFT_SUCCESS) return IB_ERR_CUDA;
  const FluidGeo& g = s->geo;
  const long long nreal = s->ncell * s->desc.dim;
  const double inv_n = 1.0 / (double)s->ncell;
  const unsigned gr = grid_for(nreal, kThreads), gm = grid_for(g.modes, kThreads);
  if (s->desc.dtype == IB_F32) {
    k_stokes_rhs<float><<<gr, kThreads, 0, st>>>((const float*)f, (const float*)u_old, (float)rho_over_k,
                                                 (float*)s->rbuf, nreal);
    if (cufftExecR2C(s->fwd, (cufftReal*)s->rbuf, (cufftComplex*)s->cbuf) != CUFFT_SUCCESS) return IB_ERR_CUDA;
    if (g.dim == 3)
      k_stokes_modes<float, 3><<<gm, kThreads, 0, st>>>((cufftComplex*)s->cbuf, g, (float)rho_over_k, (float)mu,
                                                         (float)inv_n);
    else
      k_stokes_modes<float, 2><<<gm, kThreads, 0, st>>>((cufftComplex*)s->cbuf, g, (float)rho_over_k, (float)mu,
                                                         (float)inv_n);
    if (cufftExecC2R(s->inv, (cufftComplex*)s->cbuf, (cufftReal*)u) != CUFFT_SUCCESS) return IB_ERR_CUDA;
  } else {
    k_stokes_rhs<double><<<gr, kThreads, 0, st>>>((const double*)f, (const double*)u_old, rho_over_k,
                                                  (double*)s->rbuf, nreal);
    if (cufftExecD2Z(s->fwd, (cufftDoubleReal*)s->rbuf, (cufftDoubleComplex*)s->cbuf) != CUFFT_SUCCESS)
      return IB_ERR_CUDA;
    if (g.dim == 3)
      k_stokes_modes<double, 3><<<gm, kThreads, 0, st>>>((cufftDoubleComplex*)s->cbuf, g, rho_over_k, mu, inv_n);
    else
      k_stokes_modes<double, 2><<<gm, kThreads, 0, st>>>((cufftDoubleComplex*)s->cbuf, g, rho_over_k, mu, inv_n);
    if (cufftExecZ2D(s->inv, (cufftDoubleComplex*)s->cbuf, (cufftDoubleReal*)u) != CUFFT_SUCCESS) return IB_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status ib_stokes_destroy(ib_stokes s) {
  if (!s) return IB_OK;
  cudaDeviceSynchronize();
  cufftDestroy(s->fwd);
  cufftDestroy(s->inv);
  cudaFree(s->cbuf);
  cudaFree(s->rbuf);
  delete s;
  return IB_OK;
}

}  // extern "C"
