// ib_bin.cu -- binning of Lagrangian points by Eulerian cell: the key
// computation, key-value sort and unique-key offsets of Algorithm 4 (Section
// 3.4, Fig. 2), as a stable counting sort over cells.
//
//   1. k_bin_count   per point: exact cell of xi = 0, key = c_x + n0 (c_y + n1 c_z)
//                    (plus the job's cell base), atomic per-cell count; the
//                    value returned by the atomic is the point's arrival rank.
//                    Points are taken in the order of the previous binning of
//                    the plan when it had as many points (k_bin_count_ord).
//   2. scan          exclusive prefix of the counts -> cell_start, one pass
//                    with decoupled look-back (bounded waits).
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

// Four consecutive points per thread (single job, 16-byte aligned X, FP32,
// identity order): three vector loads of positions, four independent
// counting atomics in flight, vector stores of keys and ranks.
template <int D>
__global__ void __launch_bounds__(kThreads) k_bin_count4(const __grid_constant__ Jobs J, const Bins B, const Shape sh,
                                                         int key_comp) {
  pdl_launch_dependents();   // writes keys, ranks and counts (scratch) only
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

// Four points per thread taken in the order of the previous binning of the
// same number of points (single job): positions t .. t + 3 of that order.
// Between the timesteps of the method a point moves by a fraction of a cell,
// so consecutive threads count into neighbouring cells (the atomics of a warp
// fall on a few cache lines) and the scatter that follows writes nearly in
// sequence.  Keys and ranks are stored by position t.  The result does not
// depend on the order: the stable fix-up orders each cell by point index.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_bin_count_ord(const __grid_constant__ Jobs J, const Bins B,
                                                            const Shape sh, int key_comp) {
  pdl_launch_dependents();
  const long long t0 = ((long long)blockIdx.x * kThreads + threadIdx.x) * 4;
  const long long n = B.npts_total;
  if (t0 >= n) return;
  const Job& jb = J.one;
  const T* X = (const T*)jb.X;
  const bool full = t0 + 4 <= n;
  uint32_t g[4] = {0u, 0u, 0u, 0u};
  if (full) {
    const uint4 o = *reinterpret_cast<const uint4*>(B.order + t0);
    g[0] = o.x; g[1] = o.y; g[2] = o.z; g[3] = o.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (t0 + i < n) g[i] = B.order[t0 + i];
  }
  T x[4 * D];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long gi = IB_IN(B.err, g[i], n) ? (long long)g[i] : 0;
#pragma unroll
    for (int b = 0; b < D; ++b) x[i * D + b] = (full || t0 + i < n) ? X[gi * D + b] : (T)0;
  }
  uint32_t key[4], rank[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (full || t0 + i < n) key[i] = point_key<T, D>(jb, B, x + i * D, sh, key_comp);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (full || t0 + i < n) rank[i] = IB_IN(B.err, key[i], B.ncell_total + 1) ? atomicAdd(&B.count[key[i]], 1u) : 0u;
  if (full) {
    *reinterpret_cast<uint4*>(B.key + t0) = make_uint4(key[0], key[1], key[2], key[3]);
    *reinterpret_cast<uint4*>(B.rank + t0) = make_uint4(rank[0], rank[1], rank[2], rank[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (t0 + i < n) {
        B.key[t0 + i] = key[i];
        B.rank[t0 + i] = rank[i];
      }
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_bin_count(const __grid_constant__ Jobs J, const Bins B, const Shape sh,
                                                        int key_comp) {
  pdl_launch_dependents();
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

// ---------------------------------------------------------------------------
// Exclusive prefix of the counts in one pass (decoupled look-back): a block
// takes the next chunk of kScanChunk counts from a ticket counter, so chunks
// are started in increasing order and a block only ever waits on chunks
// whose blocks are already running.  It publishes its chunk total
// (aggregate), then reads the states of the chunks before it, 32 at a time,
// adding aggregates until it meets a published inclusive prefix; it publishes
// its own inclusive prefix and writes the chunk's exclusive offsets.  A state
// is one 64-bit word (flag << 32 | value), written and read whole.  The ticket
// and the states are cleared with the counts before each binning.  Every
// wait polls a bounded number of times (kScanSpinLimit, about a second with
// the pauses between polls); a wait that runs out sets ERR_TIMEOUT in the
// error word (reported as IB_ERR_TIMEOUT) and the block goes on with the sum
// it has, so the launch always ends.
// ---------------------------------------------------------------------------
constexpr unsigned long long kStAgg = 1ull << 32;
constexpr unsigned long long kStInc = 2ull << 32;
constexpr int kScanSpinLimit = 1 << 23;

__device__ __forceinline__ unsigned long long load_state(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void store_state(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// Warp 0: the exclusive prefix of chunk `id` from the states of chunks
// id - 1, id - 2, ... (state[1 + c] for chunk c).  Returns the sum; on a
// wait that runs out, the sum of what was read.
__device__ __forceinline__ uint32_t look_back(const unsigned long long* state, long long id, uint32_t* err,
                                              int spin_limit) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0;
  long long pos = id;   // chunks [0, pos) not yet summed
  while (pos > 0) {
    const long long c = pos - 1 - lane;
    unsigned long long v = c >= 0 ? load_state(state + 1 + c) : kStInc;
    int spins = 0;
    while (__any_sync(0xffffffffu, (v >> 32) == 0ull)) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        return prefix;
      }
      __nanosleep(100);
      if ((v >> 32) == 0ull) v = load_state(state + 1 + c);
    }
    const unsigned inc = __ballot_sync(0xffffffffu, (v >> 32) == 2ull);
    // lanes up to the first inclusive prefix (nearest chunk first) contribute
    const int stop = inc ? __ffs(inc) - 1 : 31;
    uint32_t x = lane <= stop ? (uint32_t)v : 0u;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    prefix += x;
    if (inc) break;
    pos -= 32;
  }
  return prefix;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_lookback(uint32_t* __restrict__ a, long long m,
                                                                 unsigned long long* __restrict__ state, long long nb,
                                                                 uint32_t* err, int spin_limit, long long fixed_id) {
  __shared__ long long s_id;
  __shared__ uint32_t s_prefix;
  pdl_wait();                 // the counts of the kernel before
  pdl_launch_dependents();
  if (threadIdx.x == 0) s_id = fixed_id >= 0 ? fixed_id : (long long)atomicAdd(state, 1ull);
  __syncthreads();
  const long long id = s_id;
  if (id >= nb) return;
  const long long base = id * kScanChunk + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
  load8(a, base, m, v);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += v[i];
  uint32_t tot;
  uint32_t off = block_exclusive(s, &tot);
  if (threadIdx.x < 32) {
    uint32_t prefix = 0;
    if (id == 0) {
      if (threadIdx.x == 0) store_state(state + 1, kStInc | tot);
    } else {
      if (threadIdx.x == 0) store_state(state + 1 + id, kStAgg | tot);
      prefix = look_back(state, id, err, spin_limit);
      if (threadIdx.x == 0) store_state(state + 1 + id, kStInc | (uint32_t)(prefix + tot));
    }
    if (threadIdx.x == 0) s_prefix = prefix;
  }
  __syncthreads();
  off += s_prefix;
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
  if (id == nb - 1 && threadIdx.x == 0) a[m] = s_prefix + tot;   // the grand total
}

// perm_tmp[cell_start[key] + rank] = (point, key), position t of the
// processing order (the point is order[t], or t without an order).
__global__ void __launch_bounds__(kThreads) k_bin_scatter(const Bins B) {
  pdl_wait();
  pdl_launch_dependents();
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (t >= B.npts_total) return;
  const uint32_t k = B.key[t];
  const uint32_t g = B.order ? B.order[t] : (uint32_t)t;
  if (!IB_IN(B.err, k, B.ncell_total + 1)) return;
  const long long dst = (long long)B.count[k] + B.rank[t];
  if (IB_IN(B.err, dst, B.npts_total)) B.perm_tmp[dst] = make_uint2(g, k);
}

// Stable order inside a cell, one thread per sorted position q: the point at
// q ranks, among the points of its cell, by the number of them with a smaller
// index.  O(cell size) per point; cells hold a handful of points in every
// workload of interest, and the cost stays bounded (quadratic in the largest
// cell) for adversarial input.
__global__ void __launch_bounds__(kThreads) k_bin_stable(const Bins B) {
  pdl_wait();
  pdl_launch_dependents();   // the bins are scratch; readers wait for this kernel
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

// Owner slab of each point: its cell of xi = 0 along z (the exact cell map,
// wrapped periodically) lies in tile layer L = cell / 8, and slab k owns the
// layers [bounds[k], bounds[k + 1]).  Invalid positions get -1.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_slab_owner(const __grid_constant__ Jobs J, const SlabBounds sb,
                                                         long long n, int* __restrict__ owner) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const Job& jb = J.one;
  Cell1<T> c;
  const uint32_t e = point_cell<T>(((const T*)jb.X)[i * 3 + 2], jb, 2, c);
  int o = -1;
  if (e == 0) {
    const int nz = jb.n[2];
    const int cz = ((unsigned)c.i0 < (unsigned)nz) ? c.i0 : modn(c.i0, nz);
    const int layer = cz / sb.tile;
    for (int k = 0; k < sb.nslab; ++k)
      if (layer >= sb.bound[k] && layer < sb.bound[k + 1]) o = k;
  }
  owner[i] = o;
}

}  // namespace

long long scan_blocks(long long m) { return (m + kScanChunk - 1) / kScanChunk; }

size_t bin_clear_bytes(const Bins& B) {
  return (size_t)((const char*)(B.scan + 1 + scan_blocks(B.ncell_total + 1)) - (const char*)B.count);
}

cudaError_t clear_bins(const Bins& B, cudaStream_t s) { return cudaMemsetAsync(B.count, 0, bin_clear_bytes(B), s); }

cudaError_t launch_bin(const Jobs& J, const Shape& sh, const Bins& B, int dtype, cudaStream_t s, int key_comp) {
  const long long n = B.npts_total;
  if (n > 0) {
    // key and rank are 256-byte aligned sections of the arena
    const bool vec = !J.table && ((uintptr_t)J.one.X % 16) == 0;
    const unsigned g4 = grid_for((n + 3) / 4, kThreads);
    if (B.order && !J.table) {
      if (dtype == 0) {
        if (sh.dim == 3) k_bin_count_ord<float, 3><<<g4, kThreads, 0, s>>>(J, B, sh, key_comp);
        else k_bin_count_ord<float, 2><<<g4, kThreads, 0, s>>>(J, B, sh, key_comp);
      } else {
        if (sh.dim == 3) k_bin_count_ord<double, 3><<<g4, kThreads, 0, s>>>(J, B, sh, key_comp);
        else k_bin_count_ord<double, 2><<<g4, kThreads, 0, s>>>(J, B, sh, key_comp);
      }
    } else if (dtype == 0 && vec) {
      if (sh.dim == 3) k_bin_count4<3><<<g4, kThreads, 0, s>>>(J, B, sh, key_comp);
      else k_bin_count4<2><<<g4, kThreads, 0, s>>>(J, B, sh, key_comp);
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
  // The scan, scatter and fix-up start while the kernel before finishes (each
  // waits for it before reading its results).
  cudaError_t e = launch_pdl(k_scan_lookback, dim3((unsigned)nb), dim3(kScanThreads), 0, s, B.count, m, B.scan, nb,
                             B.err, kScanSpinLimit, -1ll);
  if (e == cudaSuccess && n > 0) {
    e = launch_pdl(k_bin_scatter, dim3(grid_for(n, kThreads)), dim3(kThreads), 0, s, B);
    if (e == cudaSuccess) e = launch_pdl(k_bin_stable, dim3(grid_for(n, kThreads)), dim3(kThreads), 0, s, B);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_scan_wait_selftest(uint32_t* a, unsigned long long* state, uint32_t* err, int spin_limit,
                                      cudaStream_t s) {
  // Chunk 1 of two, with chunk 0 never published: its look-back waits on a
  // state that nothing sets and must give up after spin_limit polls.
  k_scan_lookback<<<1, kScanThreads, 0, s>>>(a, 2 * kScanChunk, state, 2, err, spin_limit, 1);
  return cudaGetLastError();
}

cudaError_t launch_slab_owner(const Jobs& J, const SlabBounds& sb, long long n, int dtype, int* owner, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (dtype == 0) k_slab_owner<float><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, sb, n, owner);
  else k_slab_owner<double><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, sb, n, owner);
  return cudaGetLastError();
}

}  // namespace ibgb
