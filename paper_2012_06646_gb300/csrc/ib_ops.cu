// ib_ops.cu -- spreading, interpolation, position gradient and position
// update kernels of the GB300 immersed-boundary coupling library
// (arXiv 2012.06646).
//
// Spreading (Eq. disc-spread) is the paper's parallel spread re-designed for
// one GPU with shared memory instead of a per-shift sort and segmented
// reduce (Algorithm 4): the grid is cut into tiles; the CTA of a tile takes
// the points binned into the tile's cells (no duplication) and adds their
// s^d support contributions into a shared-memory box covering the tile plus
// a 2-node apron on every side, then writes the box to scratch.  A second
// kernel forms every grid node as the sum of the (at most 2^d) boxes that
// cover it, in a fixed tile order.  Inside a box, warps work on cell layers
// that are 5 layers apart at any moment (the support of a cell layer spans 5
// node layers), so no two warps touch the same node concurrently, and each
// warp issues its additions in program order.  Every node sum therefore has
// a fixed order and the result is bit-reproducible run to run.
//
// Interpolation (Eq. disc-interp, Algorithm 3) keeps one thread per point,
// visiting points in cell order (the bins) so neighbouring threads gather
// neighbouring grid values.
#include <math.h>

#include "ib_internal.h"

namespace ibgb {

namespace {

constexpr int kBoxThreads = 128;   // 4 warps: one per group of 5 cell layers
constexpr int kThreads = 256;

template <int D, int TS>
struct Geo {
  static constexpr int TX = TS, TY = TS, TZ = (D == 3) ? TS : 1;
  static constexpr int BX = TS + 4, BY = TS + 4, BZ = (D == 3) ? TS + 4 : 1;
  static constexpr int BV = BX * BY * BZ;
  static constexpr int NT = (D == 3) ? 4 : 1;  // support size along z
};

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Tile coordinates of local tile lt of job jb.
template <int D, int TS>
__device__ __forceinline__ void tile_coords(const Job& jb, long long lt, int T0[3], int TE[3]) {
  const int c0 = (int)(lt % jb.ntile[0]);
  const long long r = lt / jb.ntile[0];
  const int c1 = (int)(r % jb.ntile[1]);
  const int c2 = (int)(r / jb.ntile[1]);
  T0[0] = c0 * TS;
  T0[1] = c1 * TS;
  T0[2] = (D == 3) ? c2 * TS : 0;
  TE[0] = min(TS, jb.n[0] - T0[0]);
  TE[1] = min(TS, jb.n[1] - T0[1]);
  TE[2] = (D == 3) ? min(TS, jb.n[2] - T0[2]) : 1;
}

// Rows of one cell layer of a tile, flattened for a warp: lane r < rows
// holds the sorted start and count of row r; returns the layer's point count.
template <int D>
__device__ __forceinline__ uint32_t layer_rows(const Job& jb, const Bins& B, const int T0[3], const int TE[3],
                                               int l, int lane, uint32_t* rstart, uint32_t* rpre) {
  const int rows = (D == 3) ? TE[1] : 1;
  uint32_t st = 0, cnt = 0;
  if (lane < rows) {
    long long cell;
    if (D == 3) cell = T0[0] + (long long)jb.n[0] * ((T0[1] + lane) + (long long)jb.n[1] * (T0[2] + l));
    else cell = T0[0] + (long long)jb.n[0] * (T0[1] + l);
    cell += jb.cell_base;
    st = B.count[cell];
    cnt = B.count[cell + TE[0]] - st;
  }
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  rstart[lane] = st;
  rpre[lane] = inc - cnt;
  __syncwarp();
  return __shfl_sync(0xffffffffu, inc, 31);
}

// Sorted position of flattened index q of a layer.
__device__ __forceinline__ uint32_t layer_pos(uint32_t q, int rows, const uint32_t* rstart, const uint32_t* rpre) {
  int lo = 0, hi = rows - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rpre[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return rstart[lo] + (q - rpre[lo]);
}

// Per-point cell data relative to a tile box: offsets of the t = -1 node for
// xi = 0 and xi = 1/2, and the four weights of each.
template <typename T, int D>
struct PointBox {
  int o0[D], o1[D];
  T w0[D][4], w1[D][4];
};

template <typename T, int D>
__device__ __forceinline__ void point_box(const Job& jb, const Shape& sh, const T* Xp, const int T0[3],
                                          PointBox<T, D>& P) {
#pragma unroll
  for (int b = 0; b < D; ++b) {
    Cell1<T> c;
    point_cell<T>(Xp[b], jb, b, c);
    const int n = jb.n[b];
    const int cphys = ((unsigned)c.i0 < (unsigned)n) ? c.i0 : modn(c.i0, n);
    const int cc = cphys - T0[b];
    P.o0[b] = cc + 1;
    P.o1[b] = cc + (c.i1 - c.i0) + 1;
    if (sh.mac) weights(sh.kernel, c.r0, P.w0[b]);
    weights(sh.kernel, c.r1, P.w1[b]);
  }
}

// ---------------------------------------------------------------------------
// Spreading, plain accumulation: shared-memory atomics (red.shared.add),
// ordered as described at the top of the file.
// ---------------------------------------------------------------------------
template <typename T, int D, int TS>
__global__ void __launch_bounds__(kBoxThreads) k_spread_box(const __grid_constant__ Jobs J, const Shape sh,
                                                            const Bins B, T* __restrict__ boxes) {
  using Gm = Geo<D, TS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* box = reinterpret_cast<T*>(smem_raw);
  __shared__ uint32_t rstart_s[4][32];
  __shared__ uint32_t rpre_s[4][32];
  const int nc = sh.ncomp;
  const long long gt = blockIdx.x;
  const Job& jb = job_at(J, job_of_tile(J, gt));
  if (jb.G == nullptr) return;
  int T0[3], TE[3];
  tile_coords<D, TS>(jb, gt - jb.tile_base, T0, TE);
  for (int i = threadIdx.x; i < nc * Gm::BV; i += kBoxThreads) box[i] = (T)0;
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nlayers = TE[D - 1];
  const int rows = (D == 3) ? TE[1] : 1;
  const T* Gp = (const T*)jb.G;
  const T hmd = (T)jb.hmd;
  for (int phase = 0; phase < 5; ++phase) {
    for (int l = 5 * warp + phase; l < nlayers; l += 20) {
      const uint32_t M = layer_rows<D>(jb, B, T0, TE, l, lane, rstart_s[warp], rpre_s[warp]);
      const uint32_t K = (M + 31) / 32;
      for (uint32_t k = 0; k < K; ++k) {
        const uint32_t q = lane * K + k;
        const bool act = q < M;
        PointBox<T, D> P;
        T gv[4] = {0, 0, 0, 0};
        if (act) {
          const uint32_t g = B.perm[layer_pos(q, rows, rstart_s[warp], rpre_s[warp])];
          const long long li = (long long)g - jb.pt_base;
          point_box<T, D>(jb, sh, (const T*)jb.X + li * D, T0, P);
#pragma unroll
          for (int a = 0; a < 4; ++a)
            if (a < nc) gv[a] = hmd * Gp[li * nc + a];
        } else {
#pragma unroll
          for (int b = 0; b < D; ++b) {
            P.o0[b] = P.o1[b] = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) P.w0[b][t] = P.w1[b][t] = (T)0;
          }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (a >= nc) break;
          int o[3] = {0, 0, 0};
          T wx[4], wy[4], wz[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            wx[t] = half_stag(sh, a, 0) ? P.w1[0][t] : P.w0[0][t];
            wy[t] = half_stag(sh, a, 1) ? P.w1[1][t] : P.w0[1][t];
            wz[t] = (D == 3) ? (half_stag(sh, a, 2) ? P.w1[D - 1][t] : P.w0[D - 1][t]) : (T)1;
          }
#pragma unroll
          for (int b = 0; b < D; ++b) o[b] = half_stag(sh, a, b) ? P.o1[b] : P.o0[b];
          const uint32_t key = act ? (uint32_t)(o[0] | (o[1] << 8) | (o[2] << 16)) : (0x80000000u | lane);
          const uint32_t peers = __match_any_sync(0xffffffffu, key);
          const int rank = __popc(peers & ((1u << lane) - 1u));
          const int nround = __reduce_max_sync(0xffffffffu, (unsigned)__popc(peers));
          T* bp = box + a * Gm::BV + (o[2] * Gm::BY + o[1]) * Gm::BX + o[0];
          T wzg[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) wzg[t] = wz[t] * gv[a];
          for (int rd = 0; rd < nround; ++rd) {
            if (act && rank == rd) {
#pragma unroll
              for (int tz = 0; tz < Gm::NT; ++tz)
#pragma unroll
                for (int ty = 0; ty < 4; ++ty) {
                  const T wyz = wy[ty] * wzg[tz];
#pragma unroll
                  for (int tx = 0; tx < 4; ++tx)
                    atomicAdd(bp + (tz * Gm::BY + ty) * Gm::BX + tx, wx[tx] * wyz);
                }
            }
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // Box -> scratch, 16-byte vectors (nc * BV * sizeof(T) is a multiple of 16).
  const int nvec = (int)(nc * Gm::BV * sizeof(T) / 16);
  const uint4* src = reinterpret_cast<const uint4*>(box);
  uint4* dst = reinterpret_cast<uint4*>(boxes + gt * (long long)(nc * Gm::BV));
  for (int i = threadIdx.x; i < nvec; i += kBoxThreads) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Spreading, compensated: every node carries a (sum, error) pair updated by
// TwoSum (Knuth); one warp processes one point at a time with its lanes on
// distinct support nodes, so plain read-modify-write is race-free.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void two_sum_into(T* s, T* e, T v) {
  const T a = *s;
  const T sum = a + v;
  const T bb = sum - a;
  const T err = (a - (sum - bb)) + (v - bb);
  *s = sum;
  *e = *e + err;
}

template <typename T>
__device__ __forceinline__ T pick4(const T w[4], int t) {
  return (t == 0) ? w[0] : (t == 1) ? w[1] : (t == 2) ? w[2] : w[3];
}

template <typename T, int D, int TS>
__global__ void __launch_bounds__(kBoxThreads) k_spread_box_comp(const __grid_constant__ Jobs J, const Shape sh,
                                                                 const Bins B, T* __restrict__ boxes) {
  using Gm = Geo<D, TS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = sh.ncomp;
  T* boxS = reinterpret_cast<T*>(smem_raw);
  T* boxE = boxS + nc * Gm::BV;
  __shared__ uint32_t rstart_s[4][32];
  __shared__ uint32_t rpre_s[4][32];
  const long long gt = blockIdx.x;
  const Job& jb = job_at(J, job_of_tile(J, gt));
  if (jb.G == nullptr) return;
  int T0[3], TE[3];
  tile_coords<D, TS>(jb, gt - jb.tile_base, T0, TE);
  for (int i = threadIdx.x; i < 2 * nc * Gm::BV; i += kBoxThreads) boxS[i] = (T)0;
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nlayers = TE[D - 1];
  const int rows = (D == 3) ? TE[1] : 1;
  const T* Gp = (const T*)jb.G;
  const T hmd = (T)jb.hmd;
  // Lane -> support node: x = lane & 3, y = (lane >> 2) & 3, z = (lane >> 4) and +2 (3-D).
  const int tx = lane & 3, ty = (lane >> 2) & 3, tzb = lane >> 4;
  const bool lane_on = (D == 3) || lane < 16;
  for (int phase = 0; phase < 5; ++phase) {
    for (int l = 5 * warp + phase; l < nlayers; l += 20) {
      const uint32_t M = layer_rows<D>(jb, B, T0, TE, l, lane, rstart_s[warp], rpre_s[warp]);
      for (uint32_t base = 0; base < M; base += 32) {
        // Lane i fetches point base + i; the warp then walks the 32 points in order.
        const uint32_t q = base + lane;
        T xs[3] = {0, 0, 0}, gs[4] = {0, 0, 0, 0};
        if (q < M) {
          const uint32_t g = B.perm[layer_pos(q, rows, rstart_s[warp], rpre_s[warp])];
          const long long li = (long long)g - jb.pt_base;
#pragma unroll
          for (int b = 0; b < D; ++b) xs[b] = ((const T*)jb.X)[li * D + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
            if (a < nc) gs[a] = hmd * Gp[li * nc + a];
        }
        const int cnt = (int)min(32u, M - base);
        for (int i = 0; i < cnt; ++i) {
          T xp[D];
#pragma unroll
          for (int b = 0; b < D; ++b) xp[b] = __shfl_sync(0xffffffffu, xs[b], i);
          T gp[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) gp[a] = __shfl_sync(0xffffffffu, gs[a], i);
          PointBox<T, D> P;
          point_box<T, D>(jb, sh, xp, T0, P);
          if (lane_on) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              if (a >= nc) break;
              const bool hx = half_stag(sh, a, 0), hy = half_stag(sh, a, 1);
              const int ox = hx ? P.o1[0] : P.o0[0];
              const int oy = hy ? P.o1[1] : P.o0[1];
              const T wxv = hx ? pick4(P.w1[0], tx) : pick4(P.w0[0], tx);
              const T wyv = hy ? pick4(P.w1[1], ty) : pick4(P.w0[1], ty);
              const T wxy = wxv * wyv * gp[a];
              if (D == 3) {
                const bool hz = half_stag(sh, a, 2);
                const int oz = hz ? P.o1[D - 1] : P.o0[D - 1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int tz = tzb + 2 * h;
                  const T wzv = hz ? pick4(P.w1[D - 1], tz) : pick4(P.w0[D - 1], tz);
                  const int idx = a * Gm::BV + ((oz + tz) * Gm::BY + oy + ty) * Gm::BX + ox + tx;
                  two_sum_into(boxS + idx, boxE + idx, wxy * wzv);
                }
              } else {
                const int idx = a * Gm::BV + (oy + ty) * Gm::BX + ox + tx;
                two_sum_into(boxS + idx, boxE + idx, wxy);
              }
            }
          }
          __syncwarp();
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
  const int nvec = (int)(2 * nc * Gm::BV * sizeof(T) / 16);
  const uint4* src = reinterpret_cast<const uint4*>(boxS);
  uint4* dst = reinterpret_cast<uint4*>(boxes + gt * (long long)(2 * nc * Gm::BV));
  for (int i = threadIdx.x; i < nvec; i += kBoxThreads) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Combination of boxes into the grid.  Node x_b is covered by the boxes of the
// tiles t whose unwrapped box range [t TS - 2, t TS + TS + 2) contains some
// periodic copy v = x_b + k n_b; the sum runs over v then t, increasing.
// ---------------------------------------------------------------------------
constexpr int kMaxCover = 8;

__device__ __forceinline__ int floor_div(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

template <int TS>
__device__ __forceinline__ int cover_list(int x, int n, int ntile, int* tl, int* of) {
  int cnt = 0;
  int v = x;
  while (v - n >= -2) v -= n;
  const int vend = ntile * TS + 2;
  for (; v < vend; v += n) {
    const int t_lo = max(0, floor_div(v - TS - 1, TS));
    const int t_hi = min(ntile - 1, floor_div(v + 2, TS));
    for (int t = t_lo; t <= t_hi; ++t) {
      const int o = v - t * TS + 2;
      if (o >= 0 && o < TS + 4 && cnt < kMaxCover) {
        tl[cnt] = t;
        of[cnt] = o;
        ++cnt;
      }
    }
  }
  return cnt;
}

template <typename T, int D, int TS, bool CP>
__global__ void __launch_bounds__(kThreads) k_spread_combine(const __grid_constant__ Jobs J, const Shape sh,
                                                             const T* __restrict__ boxes, long long ncell_total,
                                                             int accumulate) {
  using Gm = Geo<D, TS>;
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (c >= ncell_total) return;
  const Job& jb = job_at(J, job_of_cell(J, c));
  if (jb.G == nullptr) return;
  const long long lc = c - jb.cell_base;
  int x[3];
  x[0] = (int)(lc % jb.n[0]);
  x[1] = (int)((lc / jb.n[0]) % jb.n[1]);
  x[2] = (D == 3) ? (int)(lc / ((long long)jb.n[0] * jb.n[1])) : 0;
  int tl[3][kMaxCover], of[3][kMaxCover], nco[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b < D) {
      nco[b] = cover_list<TS>(x[b], jb.n[b], jb.ntile[b], tl[b], of[b]);
    } else {
      nco[b] = 1;
      tl[b][0] = 0;
      of[b][0] = 0;
    }
  }
  const int nc = sh.ncomp;
  const long long box_elems = (long long)(CP ? 2 : 1) * nc * Gm::BV;
  T* f = (T*)jb.f;
  for (int a = 0; a < nc; ++a) {
    T S = 0, E = 0;
    for (int iz = 0; iz < nco[2]; ++iz)
      for (int iy = 0; iy < nco[1]; ++iy)
        for (int ix = 0; ix < nco[0]; ++ix) {
          const long long tile = jb.tile_base + tl[0][ix] + (long long)jb.ntile[0] * (tl[1][iy] + (long long)jb.ntile[1] * tl[2][iz]);
          const long long idx = tile * box_elems + a * Gm::BV + (of[2][iz] * Gm::BY + of[1][iy]) * Gm::BX + of[0][ix];
          if (CP) {
            const T s = boxes[idx];
            const T e = boxes[idx + nc * Gm::BV];
            const T sum = S + s;
            const T bb = sum - S;
            E += ((S - (sum - bb)) + (s - bb)) + e;
            S = sum;
          } else {
            S += boxes[idx];
          }
        }
    const T val = CP ? S + E : S;
    const long long o = a * jb.ncell + lc;
    f[o] = accumulate ? f[o] + val : val;
  }
}

// ---------------------------------------------------------------------------
// Interpolation (Algorithm 3): one thread per point in cell order.
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void node_offsets(const Job& jb, int b, int i, long long stride, long long off[4]) {
  const int n = jb.n[b];
  const int base = ((unsigned)i < (unsigned)n) ? i : modn(i, n);
#pragma unroll
  for (int t = 0; t < 4; ++t) off[t] = (long long)wrapn(base + t - 1, n) * stride;
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_interp(const __grid_constant__ Jobs J, const Shape sh, const Bins B,
                                                     const T scale) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= B.npts_total) return;
  const uint32_t g = B.perm[p];
  const Job& jb = job_at(J, job_of_point(J, (long long)g));
  if (jb.u == nullptr) return;
  const long long li = (long long)g - jb.pt_base;
  const int nc = sh.ncomp;
  T* U = (T*)jb.U + li * nc;
  const T* Xp = (const T*)jb.X + li * D;
  Cell1<T> c[D];
  uint32_t err = 0;
#pragma unroll
  for (int b = 0; b < D; ++b) err |= point_cell<T>(Xp[b], jb, b, c[b]);
  if (err) {
    for (int a = 0; a < nc; ++a) U[a] = (T)NAN;
    return;
  }
  T w0[D][4], w1[D][4];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    if (sh.mac) weights(sh.kernel, c[b].r0, w0[b]);
    weights(sh.kernel, c[b].r1, w1[b]);
  }
  const T* u = (const T*)jb.u;
  const long long s1 = jb.n[0], s2 = (long long)jb.n[0] * jb.n[1];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (a >= nc) break;
    long long ox[4], oy[4], oz[4] = {0, 0, 0, 0};
    T wx[4], wy[4], wz[4] = {1, 0, 0, 0};
    const bool hx = half_stag(sh, a, 0), hy = half_stag(sh, a, 1);
    node_offsets<T, D>(jb, 0, hx ? c[0].i1 : c[0].i0, 1, ox);
    node_offsets<T, D>(jb, 1, hy ? c[1].i1 : c[1].i0, s1, oy);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      wx[t] = hx ? w1[0][t] : w0[0][t];
      wy[t] = hy ? w1[1][t] : w0[1][t];
    }
    if (D == 3) {
      const bool hz = half_stag(sh, a, 2);
      node_offsets<T, D>(jb, D - 1, hz ? c[D - 1].i1 : c[D - 1].i0, s2, oz);
#pragma unroll
      for (int t = 0; t < 4; ++t) wz[t] = hz ? w1[D - 1][t] : w0[D - 1][t];
    }
    const T* ua = u + a * jb.ncell;
    T acc = 0;
#pragma unroll
    for (int tz = 0; tz < Geo<D, 8>::NT; ++tz) {
      T accy = 0;
#pragma unroll
      for (int ty = 0; ty < 4; ++ty) {
        const T* row = ua + oz[tz] + oy[ty];
        T accx = wx[0] * __ldg(row + ox[0]);
#pragma unroll
        for (int tx = 1; tx < 4; ++tx) accx += wx[tx] * __ldg(row + ox[tx]);
        accy += wy[ty] * accx;
      }
      acc += wz[tz] * accy;
    }
    U[a] = acc * scale;
  }
}

// ---------------------------------------------------------------------------
// Position gradient: D_{j,b} = scale sum_a v_{j,a} sum_t field_a[i+t] dW_b(t),
// dW_b(t) = (N_b/L_b) (d/dr_b) phi(t_b - r_b) prod_{c != b} phi(t_c - r_c).
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_pos_grad(const __grid_constant__ Jobs J, const Shape sh, const Bins B,
                                                       const T* __restrict__ field, const T* __restrict__ v,
                                                       T scale, T* __restrict__ Dout) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= B.npts_total) return;
  const uint32_t g = B.perm[p];
  const Job& jb = job_at(J, job_of_point(J, (long long)g));
  const long long li = (long long)g - jb.pt_base;
  const int nc = sh.ncomp;
  const T* Xp = (const T*)jb.X + li * D;
  T* Dp = Dout + li * D;
  Cell1<T> c[D];
  uint32_t err = 0;
#pragma unroll
  for (int b = 0; b < D; ++b) err |= point_cell<T>(Xp[b], jb, b, c[b]);
  if (err) {
#pragma unroll
    for (int b = 0; b < D; ++b) Dp[b] = (T)NAN;
    return;
  }
  T w0[D][4], w1[D][4], d0[D][4], d1[D][4];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    if (sh.mac) weights_and_derivs<T>(sh.kernel, c[b].r0, w0[b], d0[b]);
    weights_and_derivs<T>(sh.kernel, c[b].r1, w1[b], d1[b]);
  }
  const long long s1 = jb.n[0], s2 = (long long)jb.n[0] * jb.n[1];
  T out[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (a >= nc) break;
    long long ox[4], oy[4], oz[4] = {0, 0, 0, 0};
    T wx[4], wy[4], wz[4] = {1, 0, 0, 0}, dx[4], dy[4], dz[4] = {0, 0, 0, 0};
    const bool hx = half_stag(sh, a, 0), hy = half_stag(sh, a, 1);
    node_offsets<T, D>(jb, 0, hx ? c[0].i1 : c[0].i0, 1, ox);
    node_offsets<T, D>(jb, 1, hy ? c[1].i1 : c[1].i0, s1, oy);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      wx[t] = hx ? w1[0][t] : w0[0][t];
      dx[t] = hx ? d1[0][t] : d0[0][t];
      wy[t] = hy ? w1[1][t] : w0[1][t];
      dy[t] = hy ? d1[1][t] : d0[1][t];
    }
    if (D == 3) {
      const bool hz = half_stag(sh, a, 2);
      node_offsets<T, D>(jb, D - 1, hz ? c[D - 1].i1 : c[D - 1].i0, s2, oz);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        wz[t] = hz ? w1[D - 1][t] : w0[D - 1][t];
        dz[t] = hz ? d1[D - 1][t] : d0[D - 1][t];
      }
    }
    const T* fa = field + a * jb.ncell;
    T gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int tz = 0; tz < Geo<D, 8>::NT; ++tz) {
#pragma unroll
      for (int ty = 0; ty < 4; ++ty) {
        const T* row = fa + oz[tz] + oy[ty];
        T rx = 0, rdx = 0;
#pragma unroll
        for (int tx = 0; tx < 4; ++tx) {
          const T val = __ldg(row + ox[tx]);
          rx += wx[tx] * val;
          rdx += dx[tx] * val;
        }
        gx += wy[ty] * wz[tz] * rdx;
        gy += dy[ty] * wz[tz] * rx;
        gz += wy[ty] * dz[tz] * rx;
      }
    }
    const T va = v[li * nc + a];
    out[0] += va * gx;
    out[1] += va * gy;
    out[2] += va * gz;
  }
  // d r_b / d X_b = N_b / L_b.
#pragma unroll
  for (int b = 0; b < D; ++b) Dp[b] = scale * (T)jb.scale[b] * out[b];
}

// ---------------------------------------------------------------------------
// Position update X <- X + dt U, wrapped into [0, L) (steps b and g of Section 2).
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_advect(const __grid_constant__ Jobs J, const T* __restrict__ U, T dt,
                                                     T* __restrict__ Xout) {
  const long long e = (long long)blockIdx.x * kThreads + threadIdx.x;
  const Job& jb = J.one;
  if (e >= jb.npts * D) return;
  const int b = (int)(e % D);
  const T L = (T)jb.Ld[b];
  T x = ((const T*)jb.X)[e] + dt * U[e];
  if (x >= L || x < (T)0) {
    x -= L * floor(x / L);
    if (x >= L) x -= L;
    if (x < (T)0) x += L;
  }
  Xout[e] = x;
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int D, int TS>
cudaError_t spread_impl(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, bool comp,
                        bool accumulate, cudaStream_t s) {
  using Gm = Geo<D, TS>;
  if (ntiles > 0) {
    if (comp) {
      const size_t bytes = 2 * (size_t)sh.ncomp * Gm::BV * sizeof(T);
      allow_smem(k_spread_box_comp<T, D, TS>, bytes);
      k_spread_box_comp<T, D, TS><<<(unsigned)ntiles, kBoxThreads, bytes, s>>>(J, sh, B, (T*)boxes);
    } else {
      const size_t bytes = (size_t)sh.ncomp * Gm::BV * sizeof(T);
      allow_smem(k_spread_box<T, D, TS>, bytes);
      k_spread_box<T, D, TS><<<(unsigned)ntiles, kBoxThreads, bytes, s>>>(J, sh, B, (T*)boxes);
    }
  }
  if (B.ncell_total > 0) {
    if (comp)
      k_spread_combine<T, D, TS, true><<<grid_for(B.ncell_total, kThreads), kThreads, 0, s>>>(
          J, sh, (const T*)boxes, B.ncell_total, accumulate ? 1 : 0);
    else
      k_spread_combine<T, D, TS, false><<<grid_for(B.ncell_total, kThreads), kThreads, 0, s>>>(
          J, sh, (const T*)boxes, B.ncell_total, accumulate ? 1 : 0);
  }
  return cudaGetLastError();
}

}  // namespace

int spread_tile_side(int dim, int entry_bytes, int ncomp) {
  if (dim == 2) return 32;
  return (20 * 20 * 20 * (size_t)entry_bytes * ncomp <= 200 * 1024) ? 16 : 8;
}

size_t box_bytes(int dim, int tile, int entry_bytes, int ncomp) {
  const size_t side = (size_t)tile + 4;
  return (dim == 3 ? side * side * side : side * side) * (size_t)entry_bytes * ncomp;
}

cudaError_t launch_spread(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, int tile,
                          int dtype, bool comp, bool accumulate, cudaStream_t s) {
  if (dtype == 0) {
    if (sh.dim == 2) return spread_impl<float, 2, 32>(J, sh, B, boxes, ntiles, comp, accumulate, s);
    if (tile == 16) return spread_impl<float, 3, 16>(J, sh, B, boxes, ntiles, comp, accumulate, s);
    return spread_impl<float, 3, 8>(J, sh, B, boxes, ntiles, comp, accumulate, s);
  }
  if (sh.dim == 2) return spread_impl<double, 2, 32>(J, sh, B, boxes, ntiles, comp, accumulate, s);
  if (tile == 16) return spread_impl<double, 3, 16>(J, sh, B, boxes, ntiles, comp, accumulate, s);
  return spread_impl<double, 3, 8>(J, sh, B, boxes, ntiles, comp, accumulate, s);
}

cudaError_t launch_interp(const Jobs& J, const Shape& sh, const Bins& B, int dtype, double scale, cudaStream_t s) {
  const long long n = B.npts_total;
  if (n == 0) return cudaSuccess;
  if (dtype == 0) {
    if (sh.dim == 3) k_interp<float, 3><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, sh, B, (float)scale);
    else k_interp<float, 2><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, sh, B, (float)scale);
  } else {
    if (sh.dim == 3) k_interp<double, 3><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, sh, B, scale);
    else k_interp<double, 2><<<grid_for(n, kThreads), kThreads, 0, s>>>(J, sh, B, scale);
  }
  return cudaGetLastError();
}

cudaError_t launch_pos_grad(const Jobs& J, const Shape& sh, const Bins& B, int dtype, const void* field,
                            const void* v, double scale, void* D, cudaStream_t s) {
  const long long n = B.npts_total;
  if (n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, kThreads);
  if (dtype == 0) {
    if (sh.dim == 3)
      k_pos_grad<float, 3><<<grid, kThreads, 0, s>>>(J, sh, B, (const float*)field, (const float*)v, (float)scale, (float*)D);
    else
      k_pos_grad<float, 2><<<grid, kThreads, 0, s>>>(J, sh, B, (const float*)field, (const float*)v, (float)scale, (float*)D);
  } else {
    if (sh.dim == 3)
      k_pos_grad<double, 3><<<grid, kThreads, 0, s>>>(J, sh, B, (const double*)field, (const double*)v, scale, (double*)D);
    else
      k_pos_grad<double, 2><<<grid, kThreads, 0, s>>>(J, sh, B, (const double*)field, (const double*)v, scale, (double*)D);
  }
  return cudaGetLastError();
}

cudaError_t launch_advect(const Jobs& J, const Shape& sh, int dtype, const void* U, double dt, void* Xout,
                          cudaStream_t s) {
  const long long n = J.one.npts * sh.dim;
  if (n == 0) return cudaSuccess;
  const unsigned grid = grid_for(n, kThreads);
  if (dtype == 0) {
    if (sh.dim == 3) k_advect<float, 3><<<grid, kThreads, 0, s>>>(J, (const float*)U, (float)dt, (float*)Xout);
    else k_advect<float, 2><<<grid, kThreads, 0, s>>>(J, (const float*)U, (float)dt, (float*)Xout);
  } else {
    if (sh.dim == 3) k_advect<double, 3><<<grid, kThreads, 0, s>>>(J, (const double*)U, dt, (double*)Xout);
    else k_advect<double, 2><<<grid, kThreads, 0, s>>>(J, (const double*)U, dt, (double*)Xout);
  }
  return cudaGetLastError();
}

}  // namespace ibgb
