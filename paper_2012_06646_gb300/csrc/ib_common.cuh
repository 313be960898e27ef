// ib_common.cuh -- device-side types and helpers shared by the kernels of the
// GB300 immersed-boundary coupling library (arXiv 2012.06646).
//
// A "job" is one independent problem: a periodic grid, a point set and its
// fields.  A single-job call passes its job by value in the kernel parameter
// block; a batched wave passes a device table of jobs.  Every global array of
// the scratch arena is indexed by a global point index (job.pt_base + local),
// a global cell id (job.cell_base + local key) or a global tile id
// (job.tile_base + local tile), so one launch covers every job of a wave.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ibgb {

constexpr uint32_t ERR_NONFINITE = 1u;
constexpr uint32_t ERR_RANGE = 2u;
constexpr uint32_t ERR_STALE = 4u;   // a point's cell no longer matches its bin (X changed after binning)
constexpr uint32_t ERR_BOUNDS = 8u;  // an index check of the IB_DEBUG_BOUNDS build failed (access skipped)
constexpr uint32_t ERR_TIMEOUT = 16u; // a bounded device-side wait ran out (the kernel ended without it)

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched by launch_pdl may begin
// while the kernel before it on the stream is still running, as soon as every
// block of that kernel has called pdl_launch_dependents() (or exited); its
// pdl_wait() returns once the kernel before has completed and its writes are
// visible.  Kernels launched the ordinary way start after the kernel before
// has completed, and for them both calls do nothing.
// The rules the kernels here keep: every block of a programmatically launched
// kernel calls pdl_wait() before it reads anything another kernel wrote (the
// one exception, the spreading tile kernel under IB_OVERLAP_PREVIOUS, still
// waits in one block, so that its completion implies its predecessor's); a
// kernel signals its dependents only after its own pdl_wait(), and early only
// when what it writes is scratch of the library (the binning kernels) or when
// the one dependent that reads its output early is the tile kernel under
// IB_OVERLAP_PREVIOUS, whose caller vouches that it reads none of it
// (interpolation).  Launched here: the scan, scatter and fix-up of binning,
// interpolation, the spreading tile kernel and the box combination.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Index checks of the debug build.  Compiled with IB_DEBUG_BOUNDS, IB_IN(err,
// i, n) is true when 0 <= i < n; otherwise it sets ERR_BOUNDS in the error
// word and the access it guards is skipped, so a wrong index is reported
// through ib_plan_check / ib_batch_check instead of touching memory.  In the
// release build it is the constant true and the checks compile away.
#ifdef IB_DEBUG_BOUNDS
__device__ __forceinline__ bool ib_in(uint32_t* err, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(err, ERR_BOUNDS);
  return false;
}
#define IB_IN(err, i, n) ::ibgb::ib_in((err), (long long)(i), (long long)(n))
#else
#define IB_IN(err, i, n) true
#endif

// Positions are accepted while |X_b N_b / L_b| < 2^30 (cell indices fit in int).
constexpr double kMaxCells = 1073741824.0;

struct Job {
  int n[3];              // grid points per dimension (n[2] = 1 in 2-D)
  int ntile[3];          // spreading tiles per dimension (ntile[2] = 1 in 2-D)
  int sS[3], sE[3];      // scale_b = sS_b * 2^sE_b exactly when sS_b > 0 ("short" scale)
  float sSf[3], p2E[3];  // sS_b and 2^sE_b as floats (two-product cell path)
  int fastc[3];          // 1: the two-product cell path applies to dimension b
  unsigned long long mg[3];  // floor(2^64 / n_b) + 1 (exact division of 32-bit values by n_b >= 2)
  int itile[3];          // interpolation tiles per dimension
  long long itile_base;  // first global interpolation tile of this job
  long long nitiles;
  double scale[3];       // N_b / L_b, computed on the host as (double)N_b / L_b
  double hmd;            // h^-d = prod_b scale_b
  float Lf[3];           // box side per dimension (FP32, for the position update)
  double Ld[3];          // box side per dimension (FP64)
  int bnd[3];            // 1: bounded dimension (no wrap; n[b] = nin[b] + ghost nodes)
  int nin[3];            // nodes of the domain per dimension (n[b] when periodic)
  long long cell_base;   // first global cell id of this job
  long long ncell;       // n0 n1 n2
  long long pt_base;     // first global point index of this job
  long long npts;
  long long tile_base;   // first global tile id of this job
  long long ntiles;
  const void* X;         // (npts, dim)
  const void* G;         // (npts, ncomp) spread input
  void* f;               // [ncomp][grid] spread output
  const void* u;         // [ncomp][grid] interpolation input
  void* U;               // (npts, ncomp) interpolation output
};

struct Jobs {
  const Job* table;      // device table of njobs jobs, or nullptr for a single job
  Job one;               // the job when table == nullptr
  int njobs;
};

// Static description shared by all jobs of a launch.
struct Shape {
  int dim;               // 2 or 3
  int ncomp;             // components per field
  int mac;               // 1: MAC staggering, 0: cell-centred
  int kernel;            // 0: standard 4-point, 1: cosine 4-point, 2: 3-point, 3: 6-point B-spline
};

// Scratch arena views (global arrays over all jobs of a wave).
struct Bins {
  uint32_t* count;       // [ncell_total + 2]: per-cell counts, then exclusive prefix (cell_start)
  uint32_t* key;         // [npts_total]: global cell id of each point (ncell_total = invalid point)
  uint32_t* rank;        // [npts_total]: arrival rank of the point inside its cell
  uint2* perm_tmp;       // [npts_total]: (point, cell) in cell order, arbitrary order inside a cell
  uint32_t* perm;        // [npts_total]: points in cell order, index order inside a cell (stable)
  unsigned long long* scan;  // scan state right after count: ticket, then one state word per chunk
  const uint32_t* order; // processing order of the points (a permutation, e.g. the previous perm), or null
  uint32_t* err;         // device error word
  uint32_t* tflags;      // [tiles]: 1 if the spreading tile holds points (its boxes were written), or null
  long long ncell_total;
  long long npts_total;
};

__device__ __forceinline__ const Job& job_at(const Jobs& J, int j) {
  return J.table ? J.table[j] : J.one;
}

// Largest job index j with field(j) <= v, for a field that is non-decreasing in j.
#define IBGB_JOB_SEARCH(NAME, FIELD)                                        \
  __device__ __forceinline__ int NAME(const Jobs& J, long long v) {         \
    if (!J.table) return 0;                                                 \
    int lo = 0, hi = J.njobs - 1;                                           \
    while (lo < hi) {                                                       \
      int mid = (lo + hi + 1) >> 1;                                         \
      if (J.table[mid].FIELD <= v) lo = mid; else hi = mid - 1;             \
    }                                                                       \
    return lo;                                                              \
  }
IBGB_JOB_SEARCH(job_of_point, pt_base)
IBGB_JOB_SEARCH(job_of_cell, cell_base)
IBGB_JOB_SEARCH(job_of_tile, tile_base)
IBGB_JOB_SEARCH(job_of_itile, itile_base)
#undef IBGB_JOB_SEARCH

// ---------------------------------------------------------------------------
// Cell map (Section 3.1, Fig. 1a): for staggering xi, i = floor(X (N/L) - xi)
// and r = X (N/L) - xi - i.  The integer i must equal the FP64 evaluation of
// that formula (two rounded operations, no fused multiply-add).  Only the
// staggerings xi = 0 and xi = 1/2 occur (MAC and cell-centred grids).
// ---------------------------------------------------------------------------

template <typename R>
struct Cell1 {
  int i0, i1;   // cells for xi = 0 and xi = 1/2 (unwrapped)
  R r0, r1;     // offsets in [0, 1] (1 only through rounding of r -> 1-)
  R c0, c1;     // 1 - r0, 1 - r1, each rounded from its exact value (the small
                // weight (1 - r)^2 / ... keeps its relative accuracy as r -> 1)
};

// FP32 position with a short scale (scale = S 2^E, 0 < S < 2^24).  X (N/L) is
// then exact in FP64, so floor(X (N/L)) and floor(X (N/L) - 1/2) are plain
// integer questions; this evaluates them exactly with 64-bit integers, giving
// the FP64 result without the GPU's FP64 pipe.  |u| = P 2^e with P < 2^48.
__device__ __forceinline__ float pow2_neg(int k) {  // 2^-k, 1 <= k <= 126
  return __int_as_float((127 - k) << 23);
}

__device__ __forceinline__ uint32_t cell_short(float X, int S, int E, Cell1<float>& c) {
  const uint32_t bits = __float_as_uint(X);
  const uint32_t ex = (bits >> 23) & 0xffu;
  if (ex == 0xffu) return ERR_NONFINITE;
  uint64_t M = bits & 0x7fffffu;
  int e;
  if (ex == 0u) {
    e = -149 + E;
  } else {
    M |= 0x800000u;
    e = (int)ex - 150 + E;
  }
  const uint64_t P = M * (uint64_t)S;
  const bool neg = (bits >> 31) != 0u;
  if (P == 0) {  // X = +-0
    c.i0 = 0; c.r0 = 0.f; c.c0 = 1.f; c.i1 = -1; c.r1 = 0.5f; c.c1 = 0.5f;
    return 0;
  }
  if (e >= 0) {  // u is an integer
    if (e >= 30 || (P >> (30 - e)) != 0) return ERR_RANGE;
    const int ip = (int)(P << e);
    c.i0 = neg ? -ip : ip; c.r0 = 0.f; c.c0 = 1.f; c.i1 = c.i0 - 1; c.r1 = 0.5f; c.c1 = 0.5f;
    return 0;
  }
  const int k = -e;
  if (k >= 64) {  // |u| < 2^-16
    const float t = ldexpf(__ull2float_rn(P), -k);
    if (!neg) { c.i0 = 0; c.r0 = t; c.c0 = 1.f - t; c.i1 = -1; c.r1 = 0.5f + t; c.c1 = 0.5f - t; }
    else      { c.i0 = -1; c.r0 = 1.f - t; c.c0 = t; c.i1 = -1; c.r1 = 0.5f - t; c.c1 = 0.5f + t; }
    return 0;
  }
  const uint64_t ip = P >> k;
  if (ip >= (1ull << 30)) return ERR_RANGE;
  uint64_t F = P & ((1ull << k) - 1ull);   // fractional part numerator over 2^k
  long long i0;
  if (!neg) {
    i0 = (long long)ip;
  } else if (F == 0) {
    i0 = -(long long)ip;
  } else {
    i0 = -(long long)ip - 1;
    F = (1ull << k) - F;
  }
  const uint64_t half = 1ull << (k - 1);
  long long i1;
  uint64_t F1;
  if (F >= half) { i1 = i0; F1 = F - half; } else { i1 = i0 - 1; F1 = F + half; }
  const uint64_t one = 1ull << k;
  c.i0 = (int)i0;
  c.i1 = (int)i1;
  c.r0 = __ull2float_rn(F) * pow2_neg(k);
  c.c0 = __ull2float_rn(one - F) * pow2_neg(k);
  c.r1 = __ull2float_rn(F1) * pow2_neg(k);
  c.c1 = __ull2float_rn(one - F1) * pow2_neg(k);
  return 0;
}

// FP32 position with a short scale, the common case: X S = p + e exactly
// (TwoProduct with one FMA), so u = X scale = (p + e) 2^E exactly.  floor(u)
// is floor(p), lowered by one when p is an integer and e < 0 (|e| is below
// half an ulp of p, so it cannot cross any other integer).  The fraction
// u - floor(u) is D + e = 1 - (C - e) with D = p - floor and C = (floor + 1) - p:
// D is exact for p >= 0 (the fraction of a float) and C for p < 0 (Sterbenz,
// or 0 - p), and the exact one is a multiple of ulp(p) > 2|e|.  So the cell of
// xi = 1/2 (floor(u - 1/2) = floor(u) - [fraction < 1/2]) is decided exactly
// from the exact part, and every offset is formed from it with e added last:
// r and 1 - r for both staggerings keep their relative accuracy whenever they
// are small (a value p - 1/2 formed in FP32 would not: it rounds for p < 1/4).
// Outside |p| in [2^-100, 2^22) (or for a non-finite X) the integer path decides.
__device__ __forceinline__ uint32_t cell_twoprod(float X, const Job& jb, int b, Cell1<float>& c) {
  const float p0 = X * jb.sSf[b];
  const float e0 = fmaf(X, jb.sSf[b], -p0);
  const float p = p0 * jb.p2E[b];
  const float e = e0 * jb.p2E[b];
  const float ap = fabsf(p);
  if (!(ap < 4194304.f) || !(ap >= 7.8886e-31f)) return cell_short(X, jb.sS[b], jb.sE[b], c);
  float f0 = floorf(p);
  if (p == f0 && e < 0.f) f0 -= 1.f;
  const float D = p - f0;
  const float C = (f0 + 1.f) - p;
  const bool pos = p >= 0.f;
  // fraction below 1/2: the xi = 1/2 cell is one lower
  const bool lower = pos ? (D < 0.5f || (D == 0.5f && e < 0.f)) : (C > 0.5f || (C == 0.5f && e < 0.f));
  c.i0 = (int)f0;
  c.i1 = (int)f0 - (lower ? 1 : 0);
  c.r0 = D + e;
  c.c0 = C - e;
  const float rA = pos ? (lower ? D + 0.5f : D - 0.5f) : (lower ? 1.5f - C : 0.5f - C);
  const float cA = pos ? (lower ? 0.5f - D : 1.5f - D) : (lower ? C - 0.5f : C + 0.5f);
  c.r1 = rA + e;
  c.c1 = cA - e;
  return 0;
}

// FP64 evaluation, the oracle's formula literally (u = X * scale; u - xi).
template <typename R>
__device__ __forceinline__ uint32_t cell_fp64(double X, double scale, Cell1<R>& c) {
  if (!isfinite(X)) return ERR_NONFINITE;
  const double u = __dmul_rn(X, scale);
  if (!(fabs(u) < kMaxCells)) return ERR_RANGE;
  const double f0 = floor(u);
  const double v = __dsub_rn(u, 0.5);
  const double f1 = floor(v);
  c.i0 = (int)f0;
  c.i1 = (int)f1;
  const double r0 = __dsub_rn(u, f0), r1 = __dsub_rn(v, f1);
  c.r0 = (R)r0;
  c.r1 = (R)r1;
  c.c0 = (R)__dsub_rn(1.0, r0);
  c.c1 = (R)__dsub_rn(1.0, r1);
  return 0;
}

template <typename T>
__device__ __forceinline__ uint32_t point_cell(T X, const Job& jb, int b, Cell1<T>& c);

template <>
__device__ __forceinline__ uint32_t point_cell<float>(float X, const Job& jb, int b, Cell1<float>& c) {
  if (jb.fastc[b]) return cell_twoprod(X, jb, b, c);
  if (jb.sS[b] > 0) return cell_short(X, jb.sS[b], jb.sE[b], c);
  return cell_fp64<float>((double)X, jb.scale[b], c);
}

template <>
__device__ __forceinline__ uint32_t point_cell<double>(double X, const Job& jb, int b, Cell1<double>& c) {
  return cell_fp64<double>(X, jb.scale[b], c);
}

// Bounded (non-periodic) dimension b: the position must lie in [0, L_b], i.e.
// its xi = 0 cell is 0 .. nin - 1, or nin exactly on the far face.  Always true
// for periodic dimensions.
template <typename T>
__device__ __forceinline__ bool in_bounds(const Job& jb, int b, const Cell1<T>& c) {
  return !jb.bnd[b] || (c.i0 >= 0 && (c.i0 < jb.nin[b] || (c.i0 == jb.nin[b] && c.r0 == (T)0)));
}

// x / d for 0 <= x < 2^32 and d >= 1, with M = floor(2^64 / d) + 1 (M unused for
// d = 1): floor(x M / 2^64) = floor(x / d) because x d < 2^64.
__device__ __forceinline__ int udiv(int x, int d, unsigned long long M) {
  return d == 1 ? x : (int)__umul64hi((unsigned long long)(unsigned)x, M);
}

// Periodic wrap of v into [0, n) for v in [-2n, 3n).
__device__ __forceinline__ int wrapn(int v, int n) {
  if (v < 0) v += n;
  if (v < 0) v += n;
  if (v >= n) v -= n;
  if (v >= n) v -= n;
  return v;
}

// Positive modulo for arbitrary v (|v| < 2^30).
__device__ __forceinline__ int modn(int v, int n) {
  int m = v % n;
  return m < 0 ? m + n : m;
}

// ---------------------------------------------------------------------------
// Weights w[t+1] = phi(t - r), t in {-1, 0, 1, 2}, r in [0, 1], rc = 1 - r
// (Eq. delta-defs).  Standard 4-point kernel, with q = sqrt(1 + 4 r rc):
//   phi(-1-r) = (3-2r-q)/8, phi(-r) = (3-2r+q)/8, phi(1-r) = (1+2r+q)/8,
//   phi(2-r) = (1+2r-q)/8,
// written with a = 1 + 2 rc + q (= 3 - 2r + q), b = 1 + 2r + q and the two
// small ones without cancellation: (3-2r-q)/8 = rc^2/a, (1+2r-q)/8 = r^2/b.
// Cosine kernel phi(x) = cos(pi x/4)^2 / 2: with (s1,c1) = sincospi(r/4) and
// (s2,c2) = sincospi(rc/4) the weights are s2^2/2, c1^2/2, c2^2/2, s1^2/2.
// dw[t+1] = d phi(t - r) / d r, used by the position gradients.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float msqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double msqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float mfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ void msincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void msincospi(double x, double* s, double* c) { sincospi(x, s, c); }

// FP32: q from x rsqrt(x) (x in [1, 2]) and one approximate reciprocal
// 1/(a b) (a b in [4, 16]) for the two small weights, rc^2/a = rc^2 b/(a b) and
// r^2/b = r^2 a/(a b); relative error of a few ulp, far inside the 1e-5
// accuracy target.
__device__ __forceinline__ void weights(int kernel, float r, float rc, float w[4]) {
  if (kernel == 0) {
    const float x = fmaf(4.f * r, rc, 1.f);
    const float q = x * rsqrtf(x);
    const float a = 1.f + 2.f * rc + q;
    const float b = 1.f + 2.f * r + q;
    const float inv = __fdividef(1.f, a * b);
    w[0] = rc * rc * b * inv;
    w[1] = 0.125f * a;
    w[2] = 0.125f * b;
    w[3] = r * r * a * inv;
  } else {
    float s1, c1, s2, c2;
    sincospif(0.25f * r, &s1, &c1);
    sincospif(0.25f * rc, &s2, &c2);
    w[0] = 0.5f * s2 * s2;
    w[1] = 0.5f * c1 * c1;
    w[2] = 0.5f * c2 * c2;
    w[3] = 0.5f * s1 * s1;
  }
}

template <typename R>
__device__ __forceinline__ void weights(int kernel, R r, R rc, R w[4]) {
  if (kernel == 0) {
    const R q = msqrt(mfma((R)4 * r, rc, (R)1));
    const R a = (R)1 + (R)2 * rc + q;
    const R b = (R)1 + (R)2 * r + q;
    w[0] = rc * rc / a;
    w[1] = (R)0.125 * a;
    w[2] = (R)0.125 * b;
    w[3] = r * r / b;
  } else {
    R s1, c1, s2, c2;
    msincospi((R)0.25 * r, &s1, &c1);
    msincospi((R)0.25 * rc, &s2, &c2);
    w[0] = (R)0.5 * s2 * s2;
    w[1] = (R)0.5 * c1 * c1;
    w[2] = (R)0.5 * c2 * c2;
    w[3] = (R)0.5 * s1 * s1;
  }
}

template <typename R>
__device__ __forceinline__ void weights_and_derivs(int kernel, R r, R rc, R w[4], R dw[4]) {
  weights(kernel, r, rc, w);
  if (kernel == 0) {
    const R q = msqrt(mfma((R)4 * r, rc, (R)1));
    const R qp = (R)2 * (rc - r) / q;             // dq/dr
    dw[0] = (R)0.125 * (-(R)2 - qp);
    dw[1] = (R)0.125 * (-(R)2 + qp);
    dw[2] = (R)0.125 * ((R)2 + qp);
    dw[3] = (R)0.125 * ((R)2 - qp);
  } else {
    R s1, c1, s2, c2;
    msincospi((R)0.25 * r, &s1, &c1);
    msincospi((R)0.25 * rc, &s2, &c2);
    const R k = (R)0.78539816339744830962;  // pi / 4
    dw[0] = -k * s2 * c2;
    dw[1] = -k * s1 * c1;
    dw[2] = k * s2 * c2;
    dw[3] = k * s1 * c1;
  }
}

// Staggering of component a in dimension b: 1 means xi = 1/2, 0 means xi = 0.
__device__ __forceinline__ int half_stag(const Shape& s, int a, int b) {
  return s.mac ? (a != b) : 1;
}

template <typename T> struct Acc;            // accumulation type for node sums
template <> struct Acc<float> { using type = float; };
template <> struct Acc<double> { using type = double; };

}  // namespace ibgb
