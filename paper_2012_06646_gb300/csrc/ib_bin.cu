// ib_bin.cu -- binning of Lagrangian points by Eulerian cell: the key
// computation, key-value sort and unique-key offsets of Algorithm 4 (Section
// 3.4, Fig. 2), as a stable counting sort over cells.
//
//   1. k_bin_count   per point: exact cell of xi = 0, key = c_x + n0 (c_y + n1 c_z)
//                    (plus the job's cell base), atomic per-cell count; the
//                    value returned by the atomic is the point's arrival rank.
//   2. scan          exclusive prefix of the counts -> cell_start (chunk
//                    totals, then each chunk adds the totals before it).
//   3. k_bin_scatter perm_tmp[cell_start[key] + rank] = (point, key) (any order
//                    in a cell).
//   4. k_bin_stable  per sorted position: perm[cell_start[key] + #(same-cell
//                    points with a smaller index)] = point: ties keep index
//                    order, as in Fig. 2 where X3 precedes X5 in cell 5.  Walking
//                    sorted positions keeps every access but one coalesced.
// Invalid points (non-finite or out of range) get the sentinel cell
// ncell_total and end up after every valid point.
#include "ib_internal.h"

namespace ibgb {

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;
static_assert(kScanChunk == kScanChunkCells, "scan chunk size shared with the scratch layout");

// Key of one point (ncell_total for an invalid position, reported in B.err):
// its cell of xi = 0, or with key_comp >= 0 its cell in the staggering of
// component key_comp.
template <typename T, int D>
__device__ __forceinline__ uint32_t point_key(const Job& jb, const Bins& B, const T* X, const Shape& sh,
                                              int key_comp) {
  uint32_t err = 0;
  long long key = 0, stride = 1;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    Cell1<T> c;
    err |= point_cell<T>(X[b], jb, b, c);
    if (!in_bounds(jb, b, c)) err |= ERR_RANGE;   // bounded dimension: outside [0, L]
    const int n = jb.n[b];
    const int ib = (key_comp >= 0 && half_stag(sh, key_comp, b)) ? c.i1 : c.i0;
    const int cb = ((unsigned)ib < (unsigned)n) ? ib : modn(ib, n);
    key += (long long)cb * stride;
    stride *= n;
  }
  if (err) {
    atomicOr(B.err, err);
    return (uint32_t)B.ncell_total;
  }
  return (uint32_t)(jb.cell_base + key);
}

// Four consecutive points per thread (single job, 16-byte aligned X, FP32):
// three vector loads of positions, four independent counting atomics in
// flight, vector stores of keys and ranks.
template <int D>
__global__ void __launch_bounds__(kThreads) k_bin_count4(const __grid_constant__ Jobs J, const Bins B, const Shape sh,
                                                         int key_comp) {
  const long long g0 = ((long long)blockIdx.x * kThreads + threadIdx.x) * 4;
  const long long n = B.npts_total;
  if (g0 >= n) return;
  const Job& jb = J.one;
  const float* X = (const float*)jb.X + g0 * D;
  float x[4 * D];
  const bool full = g0 + 4 <= n;
  if (full) {
#pragma unroll
    for (int k = 0; k < D; ++k) reinterpret_cast<float4*>(x)[k] = reinterpret_cast<const float4*>(X)[k];
  } else {
#pragma unroll
    for (int k = 0; k < 4 * D; ++k)
      if (g0 * D + k < n * D) x[k] = X[k];
  }
  uint32_t key[4], rank[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (full || g0 + i < n) key[i] = point_key<float, D>(jb, B, x + i * D, sh, key_comp);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (full || g0 + i < n) rank[i] = IB_IN(B.err, key[i], B.ncell_total + 1) ? atomicAdd(&B.count[key[i]], 1u) : 0u;
  if (full) {
    *reinterpret_cast<uint4*>(B.key + g0) = make_uint4(key[0], key[1], key[2], key[3]);
    *reinterpret_cast<uint4*>(B.rank + g0) = make_uint4(rank[0], rank[1], rank[2], rank[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (g0 + i < n) {
        B.key[g0 + i] = key[i];
        B.rank[g0 + i] = rank[i];
      }
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_bin_count(const __grid_constant__ Jobs J, const Bins B, const Shape sh,
                                                        int key_comp) {
  const long long g = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (g >= B.npts_total) return;
  const Job& jb = job_at(J, job_of_point(J, g));
  const uint32_t k = point_key<T, D>(jb, B, (const T*)jb.X + (g - jb.pt_base) * D, sh, key_comp);
  B.key[g] = k;
  B.rank[g] = IB_IN(B.err, k, B.ncell_total + 1) ? atomicAdd(&B.count[k], 1u) : 0u;
}

// Block-level exclusive scan of per-thread totals; returns this thread's
// exclusive offset and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = (warp > 0) ? warp_tot[warp - 1] : 0u;
  *total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Eight consecutive entries from index base on (two 16-byte loads when they
// are all in range; base is a multiple of 8, so the vectors are aligned).
__device__ __forceinline__ void load8(const uint32_t* __restrict__ a, long long base, long long m, uint32_t v[8]) {
  if (base + kScanItems <= m) {
    const uint4 x = *reinterpret_cast<const uint4*>(a + base);
    const uint4 y = *reinterpret_cast<const uint4*>(a + base + 4);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = (base + i < m) ? a[base + i] : 0u;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ a, long long m,
                                                               uint32_t* __restrict__ sums) {
  const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
  load8(a, base, m, v);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += v[i];
  uint32_t tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the block sums in place; sums[nb] = grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* __restrict__ sums, long long nb) {
  uint32_t carry = 0;
  for (long long base = 0; base < nb; base += kScanChunk) {
    const long long i0 = base + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      v[i] = (i0 + i < nb) ? sums[i0 + i] : 0u;
      s += v[i];
    }
    uint32_t tot;
    uint32_t off = carry + block_exclusive(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      if (i0 + i < nb) sums[i0 + i] = off;
      off += v[i];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

// Exclusive offsets of the chunks.  With `direct` the block sums are still raw
// chunk totals (k_scan_sums skipped, nb <= kDirectBlocks): each block adds up
// the totals of the chunks before it itself.
constexpr long long kDirectBlocks = 4 * kScanThreads;

__device__ __forceinline__ uint32_t block_sum(uint32_t v) {
  __shared__ uint32_t part[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) part[warp] = v;
  __syncthreads();
  uint32_t t = (lane < kScanThreads / 32) ? part[lane] : 0u;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t* __restrict__ a, long long m,
                                                              const uint32_t* __restrict__ sums, long long nb,
                                                              int direct) {
  const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
  load8(a, base, m, v);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += v[i];
  uint32_t before;
  if (direct) {
    uint32_t p = 0;
    for (long long j = threadIdx.x; j < blockIdx.x; j += kScanThreads) p += sums[j];
    before = block_sum(p);
    if (blockIdx.x == gridDim.x - 1) {
      uint32_t q = 0;
      for (long long j = threadIdx.x; j < nb; j += kScanThreads) q += sums[j];
      q = block_sum(q);
      if (threadIdx.x == 0) a[m] = q;
    }
  } else {
    before = sums[blockIdx.x];
  }
  uint32_t tot;
  uint32_t off = before + block_exclusive(s, &tot);
  uint32_t o[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    o[i] = off;
    off += v[i];
  }
  if (base + kScanItems <= m) {
    *reinterpret_cast<uint4*>(a + base) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4*>(a + base + 4) = make_uint4(o[4], o[5], o[6], o[7]);
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
      if (base + i < m) a[base + i] = o[i];
  }
  if (!direct && blockIdx.x == 0 && threadIdx.x == 0) a[m] = sums[nb];
}

__global__ void __launch_bounds__(kThreads) k_bin_scatter(const Bins B) {
  const long long g = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (g >= B.npts_total) return;
  const uint32_t k = B.key[g];
  if (!IB_IN(B.err, k, B.ncell_total + 1)) return;
  const long long dst = (long long)B.count[k] + B.rank[g];
  if (IB_IN(B.err, dst, B.npts_total)) B.perm_tmp[dst] = make_uint2((uint32_t)g, k);
}

// Stable order inside a cell, one thread per sorted position q: the point at
// q ranks, among the points of its cell, by the number of them with a smaller
// index.  O(cell size) per point; cells hold a handful of points in every
// workload of interest, and the cost stays bounded (quadratic in the largest
// cell) for adversarial input.
__global__ void __launch_bounds__(kThreads) k_bin_stable(const Bins B) {
  const long long q = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (q >= B.npts_total) return;
  const uint2 e = B.perm_tmp[q];
  if (!IB_IN(B.err, e.y, B.ncell_total + 1)) return;
  const uint32_t s = B.count[e.y];
  const uint32_t t = B.count[e.y + 1];
  if (t - s == 1) {
    B.perm[q] = e.x;
    return;
  }
  if (!IB_IN(B.err, t, B.npts_total + 1) || !IB_IN(B.err, s, (long long)t)) return;
  uint32_t r = 0;
  for (uint32_t j = s; j < t; ++j) r += (B.perm_tmp[j].x < e.x) ? 1u : 0u;
  B.perm[s + r] = e.x;
}

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

long long scan_blocks(long long m) { return (m + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_bin(const Jobs& J, const Shape& sh, const Bins& B, int dtype, cudaStream_t s, int key_comp) {
  const long long n = B.npts_total;
  if (n > 0) {
    // key and rank are 256-byte aligned sections of the arena
    const bool vec = !J.table && ((uintptr_t)J.one.X % 16) == 0;
    if (dtype == 0 && vec) {
      if (sh.dim == 3) k_bin_count4<3><<<grid_for((n + 3) / 4, kThreads), kThreads, 0, s>>>(J, B, sh, key_comp);
      else k_bin_count4<2><<<grid_for((n + 3) / 4, kThreads), kThreads, 0, s>>>(J, B, sh, key_comp);
    } else if (dtype == 0) {
      if (sh.dim == 3) k_bin_count<float, 3><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, B, sh, key_comp);
      else k_bin_count<float, 2><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, B, sh, key_comp);
    } else {
      if (sh.dim == 3) k_bin_count<double, 3><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, B, sh, key_comp);
      else k_bin_count<double, 2><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, B, sh, key_comp);
    }
  }
  const long long m = B.ncell_total + 1;  // cells plus the sentinel; count[m] receives the total
  const long long nb = scan_blocks(m);
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(B.count, m, B.block_sums);
  const int direct = nb <= kDirectBlocks ? 1 : 0;
  if (!direct) k_scan_sums<<<1, kScanThreads, 0, s>>>(B.block_sums, nb);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(B.count, m, B.block_sums, nb, direct);
  if (n > 0) {
    k_bin_scatter<<<grid_for(n, kThreads), kThreads, 0, s>>>(B);
    k_bin_stable<<<grid_for(n, kThreads), kThreads, 0, s>>>(B);
  }
  return cudaGetLastError();
}

}  // namespace ibgb
