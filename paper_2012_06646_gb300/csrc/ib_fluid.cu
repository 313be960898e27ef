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
// kernel reading D_b from per-axis tables evaluated in FP64 at creation
// (sin^2 rather than 1 - cos, so small wavenumbers keep their relative
// accuracy).
#include <cufft.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
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

// D_b(k) per axis, made once in FP64 on the host: with (s, c) = (sin, cos)(pi
// k / n_b), D_b = (2 s / h_b) (-s + i c) and |D_b|^2 = (2 s / h_b)^2.
template <typename T>
struct AxisD {
  T re, im, d2;
};

constexpr unsigned kMaxGridYZ = 65535;

// The solve of one mode m: u^ = (g^ - conj(D) (D . g^) / |d|^2) / (rho/k + mu |d|^2),
// the 1/N of the inverse transform folded in; the mean mode keeps g^ / (rho/k).
template <typename T, int D>
__device__ __forceinline__ void stokes_mode(typename Cplx<T>::type* __restrict__ c, long long modes, long long m,
                                            const T dre[3], const T dim_[3], T d2, T rho_k, T mu, T inv_n) {
  typename Cplx<T>::type v[3];
#pragma unroll
  for (int a = 0; a < D; ++a) v[a] = c[a * modes + m];
  if (d2 == (T)0) {                                   // mean mode
    const T f = rho_k > (T)0 ? inv_n / rho_k : (T)0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      v[a].x *= f;
      v[a].y *= f;
      c[a * modes + m] = v[a];
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
    c[a * modes + m] = v[a];
  }
}

// One thread per Fourier mode (kx along threads, ky and kz over blocks,
// strided), all components of the mode at once.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_stokes_modes(typename Cplx<T>::type* __restrict__ c, FluidGeo g,
                                                           const AxisD<T>* __restrict__ tab, T rho_k, T mu,
                                                           T inv_n) {
  const int kx = blockIdx.x * kThreads + threadIdx.x;
  if (kx >= g.nh) return;
  const AxisD<T>* ty = tab + g.nh;
  const AxisD<T>* tz = ty + g.n[1];
  for (int kz = blockIdx.z; kz < ((D == 3) ? g.n[2] : 1); kz += gridDim.z)
    for (int ky = blockIdx.y; ky < g.n[1]; ky += gridDim.y) {
      const long long m = ((long long)kz * g.n[1] + ky) * g.nh + kx;
      const AxisD<T> ax[3] = {tab[kx], ty[ky], (D == 3) ? tz[kz] : AxisD<T>{(T)0, (T)0, (T)0}};
      T dre[3], dim_[3], d2 = 0;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        dre[b] = ax[b].re;
        dim_[b] = ax[b].im;
        d2 += ax[b].d2;
      }
      stokes_mode<T, D>(c, g.modes, m, dre, dim_, d2, rho_k, mu, inv_n);
    }
}

// g = (rho/k) u_old + f (u_old may be null), 16 bytes per thread when the three
// arrays are 16-byte aligned and n a multiple of the vector width.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_stokes_rhs(const T* __restrict__ f, const T* __restrict__ u_old,
                                                         T rho_k, T* __restrict__ g, long long n, int vec) {
  constexpr int P = 16 / (int)sizeof(T);
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (vec) {
    if (t * P >= n) return;
    const uint4 fv = reinterpret_cast<const uint4*>(f)[t];
    const T* fe = reinterpret_cast<const T*>(&fv);
    T out[P];
    if (u_old) {
      const uint4 uv = reinterpret_cast<const uint4*>(u_old)[t];
      const T* ue = reinterpret_cast<const T*>(&uv);
#pragma unroll
      for (int k = 0; k < P; ++k) out[k] = rho_k * ue[k] + fe[k];
    } else {
#pragma unroll
      for (int k = 0; k < P; ++k) out[k] = fe[k];
    }
    reinterpret_cast<uint4*>(g)[t] = *reinterpret_cast<const uint4*>(out);
    return;
  }
  if (t >= n) return;
  g[t] = (u_old ? rho_k * u_old[t] : (T)0) + f[t];
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
  void* tabs;             // AxisD tables of x (n0/2 + 1 wavenumbers), y (n1), z (n2)
};

// D_b per axis for x (n0/2 + 1 wavenumbers), y (n1) and z (n2), in FP64 then T.
template <typename T>
static ib_status make_axis_tables(ib_stokes s) {
  const FluidGeo& g = s->geo;
  const int counts[3] = {g.nh, g.n[1], g.n[2]};
  const int nax = counts[0] + counts[1] + counts[2];
  AxisD<T>* host = (AxisD<T>*)malloc(sizeof(AxisD<T>) * (size_t)nax);
  if (!host) return IB_ERR_OOM;
  int o = 0;
  for (int b = 0; b < 3; ++b)
    for (int k = 0; k < counts[b]; ++k, ++o) {
      const bool live = b < g.dim;
      const double th = M_PI * (double)k / (double)g.n[b];
      const double sn = live ? sin(th) : 0.0, cs = live ? cos(th) : 0.0, a = 2.0 * sn / g.h[b];
      host[o].re = (T)(-a * sn);
      host[o].im = (T)(a * cs);
      host[o].d2 = (T)(a * a);
    }
  const size_t bytes = sizeof(AxisD<T>) * (size_t)nax;
  if (cudaMalloc(&s->tabs, bytes) != cudaSuccess) {
    cudaGetLastError();
    free(host);
    return IB_ERR_OOM;
  }
  const bool ok = cudaMemcpy(s->tabs, host, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  free(host);
  if (!ok) {
    cudaFree(s->tabs);
    s->tabs = nullptr;
    return IB_ERR_CUDA;
  }
  return IB_OK;
}

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
  const ib_status st = dbl ? make_axis_tables<double>(s) : make_axis_tables<float>(s);
  if (st != IB_OK) {
    cudaFree(s->cbuf);
    cudaFree(s->rbuf);
    cufftDestroy(s->fwd);
    cufftDestroy(s->inv);
    delete s;
    return st;
  }
  *out = s;
  return IB_OK;
}

ib_status ib_stokes_solve(ib_stokes s, const void* f, const void* u_old, void* u, double rho_over_k, double mu,
                          void* stream) {
  const ibgb::NvtxRange nvtx_range("ib_stokes_solve");
  if (!s || !f || !u) return IB_ERR_INVALID_ARG;
  if (!(rho_over_k >= 0.0) || !(mu >= 0.0) || !isfinite(rho_over_k) || !isfinite(mu) ||
      (rho_over_k == 0.0 && mu == 0.0))
    return IB_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cufftSetStream(s->fwd, st) != CUFFT_SUCCESS || cufftSetStream(s->inv, st) != CUFFT_SUCCESS) return IB_ERR_CUDA;
  const FluidGeo& g = s->geo;
  const long long nreal = s->ncell * s->desc.dim;
  const double inv_n = 1.0 / (double)s->ncell;
  const size_t eb = s->desc.dtype == IB_F64 ? 8 : 4;
  const int vec = (nreal % (long long)(16 / eb) == 0 && ((uintptr_t)f | (uintptr_t)u_old | (uintptr_t)s->rbuf) % 16 == 0)
                      ? 1 : 0;
  const unsigned gr = grid_for(vec ? nreal / (long long)(16 / eb) : nreal, kThreads);
  const dim3 gm((unsigned)((g.nh + kThreads - 1) / kThreads), (unsigned)(g.n[1] < (int)kMaxGridYZ ? g.n[1] : (int)kMaxGridYZ),
                (unsigned)(g.n[2] < (int)kMaxGridYZ ? g.n[2] : (int)kMaxGridYZ));
  if (s->desc.dtype == IB_F32) {
    k_stokes_rhs<float><<<gr, kThreads, 0, st>>>((const float*)f, (const float*)u_old, (float)rho_over_k,
                                                 (float*)s->rbuf, nreal, vec);
    if (cufftExecR2C(s->fwd, (cufftReal*)s->rbuf, (cufftComplex*)s->cbuf) != CUFFT_SUCCESS) return IB_ERR_CUDA;
    if (g.dim == 3)
      k_stokes_modes<float, 3><<<gm, kThreads, 0, st>>>((cufftComplex*)s->cbuf, g, (const AxisD<float>*)s->tabs,
                                                         (float)rho_over_k, (float)mu,
                                                         (float)inv_n);
    else
      k_stokes_modes<float, 2><<<gm, kThreads, 0, st>>>((cufftComplex*)s->cbuf, g, (const AxisD<float>*)s->tabs,
                                                         (float)rho_over_k, (float)mu,
                                                         (float)inv_n);
    if (cufftExecC2R(s->inv, (cufftComplex*)s->cbuf, (cufftReal*)u) != CUFFT_SUCCESS) return IB_ERR_CUDA;
  } else {
    k_stokes_rhs<double><<<gr, kThreads, 0, st>>>((const double*)f, (const double*)u_old, rho_over_k,
                                                  (double*)s->rbuf, nreal, vec);
    if (cufftExecD2Z(s->fwd, (cufftDoubleReal*)s->rbuf, (cufftDoubleComplex*)s->cbuf) != CUFFT_SUCCESS)
      return IB_ERR_CUDA;
    if (g.dim == 3)
      k_stokes_modes<double, 3><<<gm, kThreads, 0, st>>>((cufftDoubleComplex*)s->cbuf, g,
                                                          (const AxisD<double>*)s->tabs, rho_over_k, mu, inv_n);
    else
      k_stokes_modes<double, 2><<<gm, kThreads, 0, st>>>((cufftDoubleComplex*)s->cbuf, g,
                                                          (const AxisD<double>*)s->tabs, rho_over_k, mu, inv_n);
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
  cudaFree(s->tabs);
  delete s;
  return IB_OK;
}

}  // extern "C"
