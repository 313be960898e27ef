// ib_paper.cu -- the paper's own parallel spreading algorithms, written for
// sm_103a as in-repo comparators of the tile-box spreading of ib_ops.cu
// (arXiv 2012.06646, Section 3.4 and the buffered variants that follow it).
//
// Algorithm 4 sorts the points once by key (the cell a point inhabits, in the
// staggering of the component being spread) and then, for every shift of the
// s^d support in turn, computes each point's value for that shift, reduces the
// values of each run of equal keys (segmented reduce) and adds the reduced
// value of every inhabited cell to the node "cell + shift".  Within one shift
// distinct cells reach distinct nodes, so the additions need no atomics; the
// shifts are separated by a synchronisation, here the boundary between two
// launches on the stream (s^d = 64 launches per component in 3-D, the cost
// the paper names).  Algorithms 5 and 6 take beta shifts per pass and add the
// reduced value of shift k of the pass into buffer k (beta grid-sized
// buffers, no contention within a launch), then sum the buffers; Algorithm 6
// allocates the buffers itself.
//
// The GPU form: the key-value sort is the binning of ib_bin.cu keyed by the
// component's cells, the unique count a compaction of the inhabited cells, and
// one thread per inhabited cell walks the cell's points in sorted order (the
// segmented reduce, with a fixed order) and writes its node.  Results are
// therefore run-to-run reproducible.
#include "ib_internal.h"

namespace ibgb {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPass = 16;   // shifts handled by one launch (a pass of beta > 16 takes several launches)

// "Count unique": the inhabited cells of the bins, appended to `cells` (any
// order: every cell reaches its own node for a given shift, so the order of
// the list does not change any sum), their number in *q.
__global__ void __launch_bounds__(kThreads) k_paper_cells(const Bins B, uint32_t* __restrict__ cells,
                                                          uint32_t* __restrict__ q) {
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  const bool inhabited = c < B.ncell_total && B.count[c + 1] > B.count[c];
  const unsigned m = __ballot_sync(0xffffffffu, inhabited);
  if (m == 0) return;
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(q, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);   // every lane is here (no divergence above)
  if (inhabited) cells[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)c;
}

// One thread per inhabited cell (q of them, at most npts).
template <typename T, int D, int NS>
__global__ void __launch_bounds__(kThreads) k_paper_shifts(const __grid_constant__ Jobs J, const Shape sh,
                                                           const Bins B, int a, int j0, int nshift, T* __restrict__ out,
                                                           long long out_stride, const uint32_t* __restrict__ cells,
                                                           const uint32_t* __restrict__ q) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= *q) return;
  const long long c = cells[i];
  const uint32_t s = B.count[c], e = B.count[c + 1];
  const Job& jb = J.one;
  const T* X = (const T*)jb.X;
  const T* G = (const T*)jb.G;
  const int nc = sh.ncomp;
  const T hmd = (T)jb.hmd;
  T V[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) V[k] = (T)0;
  // Segmented reduce: the cell's points in sorted order.
  for (uint32_t q = s; q < e; ++q) {
    const long long p = B.perm[q];
    T w[D][4];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      Cell1<T> cl;
      point_cell<T>(X[p * D + b], jb, b, cl);
      if (half_stag(sh, a, b)) weights(sh.kernel, cl.r1, cl.c1, w[b]);
      else weights(sh.kernel, cl.r0, cl.c0, w[b]);
    }
    const T g = hmd * G[p * nc + a];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (k >= nshift) break;
      const int j = j0 + k;                             // shift digits, x fastest (Algorithm 1)
      T wt = w[0][j & 3] * w[1][(j >> 2) & 3];
      if (D == 3) wt *= w[2][(j >> 4) & 3];
      V[k] += wt * g;
    }
  }
  // Node of cell c for each shift (t - 1 per dimension, wrapped).
  const int n0 = jb.n[0], n1 = jb.n[1];
  const int cx = (int)(c % n0);
  const int cy = (int)((c / n0) % n1);
  const int cz = (D == 3) ? (int)(c / ((long long)n0 * n1)) : 0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (k >= nshift) break;
    const int j = j0 + k;
    long long node = wrapn(cx + (j & 3) - 1, n0) + (long long)n0 * wrapn(cy + ((j >> 2) & 3) - 1, n1);
    if (D == 3) node += (long long)n0 * n1 * wrapn(cz + ((j >> 4) & 3) - 1, jb.n[2]);
    T* o = out + k * out_stride + node;
    *o = *o + V[k];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_paper_sum(const __grid_constant__ Jobs J, int a, int beta,
                                                        const T* __restrict__ buf) {
  const long long m = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long ncell = J.one.ncell;
  if (m >= ncell) return;
  T s = buf[m];
  for (int k = 1; k < beta; ++k) s += buf[k * ncell + m];
  ((T*)J.one.f)[a * ncell + m] = s;
}

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_paper_cells(const Bins& B, uint32_t* cells, uint32_t* q, cudaStream_t s) {
  if (cudaMemsetAsync(q, 0, sizeof(uint32_t), s) != cudaSuccess) return cudaErrorUnknown;
  const unsigned g = grid_for(B.ncell_total, kThreads);
  if (g > 0) k_paper_cells<<<g, kThreads, 0, s>>>(B, cells, q);
  return cudaGetLastError();
}

cudaError_t launch_paper_shifts(const Jobs& J, const Shape& sh, const Bins& B, int dtype, int a, int j0, int nshift,
                                void* out, long long out_stride, const uint32_t* cells, const uint32_t* q,
                                cudaStream_t s) {
  // q <= min(ncell, npts) threads do work; the grid covers the bound.
  const long long bound = B.npts_total < B.ncell_total ? B.npts_total : B.ncell_total;
  const unsigned g = grid_for(bound, kThreads);
  if (g == 0) return cudaSuccess;
  for (int k0 = 0; k0 < nshift; k0 += kMaxPass) {
    const int ns = nshift - k0 < kMaxPass ? nshift - k0 : kMaxPass;
    if (dtype == 0) {
      float* o = (float*)out + (long long)k0 * out_stride;
      if (ns == 1) {
        if (sh.dim == 3) k_paper_shifts<float, 3, 1><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, 1, o, out_stride, cells, q);
        else k_paper_shifts<float, 2, 1><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, 1, o, out_stride, cells, q);
      } else {
        if (sh.dim == 3) k_paper_shifts<float, 3, kMaxPass><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, ns, o, out_stride, cells, q);
        else k_paper_shifts<float, 2, kMaxPass><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, ns, o, out_stride, cells, q);
      }
    } else {
      double* o = (double*)out + (long long)k0 * out_stride;
      if (ns == 1) {
        if (sh.dim == 3) k_paper_shifts<double, 3, 1><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, 1, o, out_stride, cells, q);
        else k_paper_shifts<double, 2, 1><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, 1, o, out_stride, cells, q);
      } else {
        if (sh.dim == 3) k_paper_shifts<double, 3, kMaxPass><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, ns, o, out_stride, cells, q);
        else k_paper_shifts<double, 2, kMaxPass><<<g, kThreads, 0, s>>>(J, sh, B, a, j0 + k0, ns, o, out_stride, cells, q);
      }
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_paper_sum(const Jobs& J, int dtype, int a, int beta, const void* buf, cudaStream_t s) {
  const unsigned g = grid_for(J.one.ncell, kThreads);
  if (g == 0) return cudaSuccess;
  if (dtype == 0) k_paper_sum<float><<<g, kThreads, 0, s>>>(J, a, beta, (const float*)buf);
  else k_paper_sum<double><<<g, kThreads, 0, s>>>(J, a, beta, (const double*)buf);
  return cudaGetLastError();
}

}  // namespace ibgb
