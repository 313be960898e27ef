// ib_ops.cu -- spreading, interpolation, position gradient and position
// update kernels of the GB300 immersed-boundary coupling library
// (arXiv 2012.06646).
//
// Spreading (Eq. disc-spread) is the paper's parallel spread re-designed for
// one GPU with shared memory instead of a per-shift sort and segmented
// reduce (Algorithm 4): the grid is cut into 8^3 tiles; one warp takes the
// points binned into a tile's cells (each point exactly once, in cell order)
// and adds their s^d support contributions into shared-memory boxes covering
// the tile plus a 2-node apron on every side, then writes the boxes to
// scratch.  A second kernel forms every grid node as the sum of the (at most
// 2^d) boxes that cover it, in a fixed tile order.  A box has a single writer
// (its warp), which adds the points in a fixed order, so every node sum has a
// fixed order and the result is bit-reproducible run to run.
//
// Interpolation (Eq. disc-interp, Algorithm 3) keeps one thread per point
// (each point's sum has one writer), grouped by tile: the tile's grid values
// plus a 2-node apron are staged in shared memory once, and every point of
// the tile gathers its support from there.
#include <math.h>

#include "ib_internal.h"

namespace ibgb {

namespace {

constexpr int kThreads = 256;

template <int D, int TS>
struct Geo {   // box of a TS^D tile plus a 2-node apron on every side
  static constexpr int BX = TS + 4, BY = TS + 4, BZ = (D == 3) ? TS + 4 : 1;
  static constexpr int BV = BX * BY * BZ;
  static constexpr int NT = (D == 3) ? 4 : 1;  // support size along z
};

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Tile coordinates of local tile lt of a job with ntile tiles per dimension.
template <int D, int TS>
__device__ __forceinline__ void tile_coords(const int* ntile, const int* n, long long lt, int T0[3], int TE[3]) {
  const int l = (int)lt;
  const int c0 = l % ntile[0];
  const int r = l / ntile[0];
  const int c1 = r % ntile[1];
  const int c2 = r / ntile[1];
  T0[0] = c0 * TS;
  T0[1] = c1 * TS;
  T0[2] = (D == 3) ? c2 * TS : 0;
  TE[0] = min(TS, n[0] - T0[0]);
  TE[1] = min(TS, n[1] - T0[1]);
  TE[2] = (D == 3) ? min(TS, n[2] - T0[2]) : 1;
}

// Per-point cell data relative to a tile box: offsets of the t = -1 node for
// xi = 0 and xi = 1/2, and the four weights of each.
template <typename T, int D>
struct PointBox {
  int o0[D], o1[D];
  T w0[D][4], w1[D][4];
};

// Returns false when the point's cell (xi = 0) is not inside the tile (X
// changed after binning).
template <typename T, int D>
__device__ __forceinline__ bool point_box(const Job& jb, const Shape& sh, const T* Xp, const int T0[3],
                                          const int TE[3], PointBox<T, D>& P) {
  bool inside = true;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    Cell1<T> c;
    const uint32_t e = point_cell<T>(Xp[b], jb, b, c);
    const int n = jb.n[b];
    const int cphys = ((unsigned)c.i0 < (unsigned)n) ? c.i0 : modn(c.i0, n);
    const int cc = cphys - T0[b];
    inside = inside && e == 0 && (unsigned)cc < (unsigned)TE[b] && (c.i1 - c.i0) >= -1 && (c.i1 - c.i0) <= 0;
    P.o0[b] = cc + 1;
    P.o1[b] = cc + (c.i1 - c.i0) + 1;
    if (sh.mac) weights(sh.kernel, c.r0, c.c0, P.w0[b]);
    weights(sh.kernel, c.r1, c.c1, P.w1[b]);
  }
  return inside;
}

// ---------------------------------------------------------------------------
// Spreading into tile boxes, one warp per (tile, component).  The warp owns a
// shared-memory box holding one component of the tile plus a 2-node apron on
// every side (two planes in compensated mode), so no other warp touches it
// and no block-wide barrier is needed.  The warp walks the points binned in
// the tile's cells (each point exactly once, cell order, index order inside a
// cell) in batches of kSpreadBatch, two stages per batch:
//   1. lanes = points: each lane computes its point's cell in each dimension,
//      the component's four weights per dimension and, with g = h^-d G, the
//      16 products wx[tx] wy[ty] g, the four z weights and the box offset of
//      the t = -1 corner; it stores them as one staging record;
//   2. warp = point: the warp walks the batch's records in order; lane
//      (tx, ty, tzb) owns the support nodes (tx, ty, tzb) and (tx, ty, tzb+2)
//      of the point's 4x4x4 box (4x4 in 2-D, lanes 16-31 idle), so the 32
//      lanes touch 64 distinct nodes and a plain read-modify-write is
//      race-free; __syncwarp orders consecutive points.  Each node's additions
//      therefore happen in the fixed point order.  The next record is read
//      before the current point's additions, and the next batch's point data
//      is fetched from global memory before this batch's additions.
// With 8^3 tiles the 32 lanes of one addition hit 32 distinct banks (rows 12
// entries apart, the two z planes 144 = 16 mod 32 apart).
// Compensated mode keeps (sum, error) per node and adds by TwoSum.
// ---------------------------------------------------------------------------
constexpr int kSpreadWarps = 2;   // independent (tile, component) units per CTA (W below)
constexpr int kSpreadBatch = 32;  // points per staging batch (one per lane in stage 1)

// Record of one point-component: the 16 products, then in 3-D two groups
// (w0, w2, off, 0) and (w1, w3, off, 0) -- lane half tzb reads group tzb
// with one vector load -- and in 2-D (off, 0, 0, 0).  7 (5) 16-byte chunks,
// an odd number, so the stage-1 vector stores of 8 lanes hit distinct banks.
template <int D>
struct WRec {
  static constexpr int words = D == 3 ? 28 : 20;
};

__device__ __forceinline__ float off_bits(int o, float) { return __int_as_float(o); }
__device__ __forceinline__ double off_bits(int o, double) { return __longlong_as_double((long long)o); }
__device__ __forceinline__ int bits_off(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_off(double v) { return (int)__double_as_longlong(v); }

template <typename T>
__device__ __forceinline__ void two_sum_into(T* s, T* e, T v) {
  const T a = *s;
  const T sum = a + v;
  const T bb = sum - a;
  const T err = (a - (sum - bb)) + (v - bb);
  *s = sum;
  *e = *e + err;
}

__device__ __forceinline__ void store4(float* d, float a, float b, float c, float e) {
  *reinterpret_cast<float4*>(d) = make_float4(a, b, c, e);
}
__device__ __forceinline__ void store4(double* d, double a, double b, double c, double e) {
  reinterpret_cast<double2*>(d)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(d)[1] = make_double2(c, e);
}
__device__ __forceinline__ void load3(const float* s, float& a, float& b, float& c) {
  const float4 q = *reinterpret_cast<const float4*>(s);
  a = q.x; b = q.y; c = q.z;
}
__device__ __forceinline__ void load3(const double* s, double& a, double& b, double& c) {
  const double2 q = reinterpret_cast<const double2*>(s)[0];
  a = q.x; b = q.y;
  c = s[2];
}

// Cell offset (box coordinates of the t = -1 node) and weights of one
// component of a point, in every dimension.
// Returns false when the point's cell (xi = 0) is not inside the tile, which
// happens only if X changed after binning; the caller then drops the point.
template <typename T, int D>
__device__ __forceinline__ bool point_comp(const Job& jb, const Shape& sh, const T* xp, const int T0[3],
                                           const int TE[3], int a, int o[3], T w[3][4]) {
  bool inside = true;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    Cell1<T> c;
    const uint32_t e = point_cell<T>(xp[b], jb, b, c);
    const int n = jb.n[b];
    const int cphys = ((unsigned)c.i0 < (unsigned)n) ? c.i0 : modn(c.i0, n);
    inside = inside && e == 0 && (unsigned)(cphys - T0[b]) < (unsigned)TE[b] && (c.i1 - c.i0) >= -1 &&
             (c.i1 - c.i0) <= 0;
    const bool h = half_stag(sh, a, b);
    o[b] = cphys - T0[b] + 1 + (h ? (c.i1 - c.i0) : 0);
    if (h) weights(sh.kernel, c.r1, c.c1, w[b]);
    else weights(sh.kernel, c.r0, c.c0, w[b]);
  }
  return inside;
}

template <typename T, int D, int TS, bool COMP, int W = kSpreadWarps>
__global__ void __launch_bounds__(32 * W) k_spread_warp(const __grid_constant__ Jobs J, const Shape sh, const Bins B,
                                                         T* __restrict__ boxes, long long nunits, int skip_empty) {
  using Gm = Geo<D, TS>;
  constexpr int REC = WRec<D>::words;
  constexpr int PLANES = COMP ? 2 : 1;
  constexpr int NROWS = (D == 3) ? TS * TS : TS;     // cell rows (x runs) of a full tile
  static_assert(NROWS % 32 == 0 && (NROWS & (NROWS - 1)) == 0, "rows: a power of two, at least 32");
  constexpr int WARP_T = PLANES * Gm::BV + kSpreadBatch * REC;
  static_assert((PLANES * Gm::BV * sizeof(T)) % 16 == 0 && (WARP_T * sizeof(T)) % 16 == 0, "16-byte sections");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t rstart_s[W][NROWS];
  __shared__ uint32_t rpre_s[W][NROWS + 1];
  __shared__ Job sjob[W];                          // one copy of the job per warp (broadcast reads)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long unit = (long long)blockIdx.x * W + warp;
  if (unit >= nunits) return;                      // the whole warp leaves; no block barrier follows
  T* boxS = reinterpret_cast<T*>(smem_raw) + warp * WARP_T;
  T* boxE = boxS + Gm::BV;                         // compensated mode only
  T* rec_s = boxS + PLANES * Gm::BV;
  uint32_t* rstart = rstart_s[warp];
  uint32_t* rpre = rpre_s[warp];
  const int nc = sh.ncomp;
  const long long gt = unit / nc;
  const int a = (int)(unit - gt * nc);
  {
    const int j = __shfl_sync(0xffffffffu, lane == 0 ? job_of_tile(J, gt) : 0, 0);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&job_at(J, j));
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sjob[warp]);
    for (int w = lane; w < (int)(sizeof(Job) / 4); w += 32) dst[w] = src[w];
    __syncwarp();
  }
  const Job& jb = sjob[warp];
  if (jb.G == nullptr) return;
  int T0[3], TE[3];
  tile_coords<D, TS>(jb.ntile, jb.n, gt - jb.tile_base, T0, TE);
  {
    constexpr int NV = (int)(PLANES * Gm::BV * sizeof(T) / 16);
    uint4* z = reinterpret_cast<uint4*>(boxS);
    for (int i = lane; i < NV; i += 32) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  // Rows of the tile's cells (x fastest inside a row): sorted start and exclusive prefix of the counts.
  const int rows = (D == 3) ? TE[1] * TE[2] : TE[1];
  uint32_t M = 0;
#pragma unroll
  for (int k = 0; k < NROWS / 32; ++k) {
    const int r = lane + 32 * k;
    uint32_t st = 0, cnt = 0;
    if (r < rows) {
      const int y = T0[1] + ((D == 3) ? r % TE[1] : r);
      const int z = (D == 3) ? T0[2] + r / TE[1] : 0;
      const long long cell = jb.cell_base + T0[0] + (long long)jb.n[0] * (y + (long long)jb.n[1] * z);
      if (IB_IN(B.err, cell + TE[0], B.ncell_total + 1)) {
        st = B.count[cell];
        cnt = B.count[cell + TE[0]] - st;
      }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    rstart[r] = st;
    rpre[r] = M + inc - cnt;
    M += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  if (skip_empty) {                                // sparse call: an empty tile writes no boxes
    if (lane == 0) B.tflags[gt] = M > 0 ? 1u : 0u;
    if (M == 0) return;
  }

  const T* Xg = (const T*)jb.X;
  const T* Gp = (const T*)jb.G;
  const T hmd = (T)jb.hmd;
  // Sorted point q of the tile -> its coordinates and component-a value.
  auto load_point = [&](uint32_t q, T xs[D], T& gs) {
    int lo = 0;
#pragma unroll
    for (int step = NROWS / 2; step >= 1; step >>= 1)
      if (lo + step < rows && rpre[lo + step] <= q) lo += step;
    const long long pi = (long long)rstart[lo] + (q - rpre[lo]);
    long long li = IB_IN(B.err, pi, B.npts_total) ? (long long)B.perm[pi] - jb.pt_base : 0;
    if (!IB_IN(B.err, li, jb.npts)) li = 0;
#pragma unroll
    for (int b = 0; b < D; ++b) xs[b] = Xg[li * D + b];
    gs = Gp[li * nc + a];
  };

  const int tx = lane & 3, ty = (lane >> 2) & 3, tzb = lane >> 4;
  const int lane_off = (D == 3) ? ((tzb * Gm::BY + ty) * Gm::BX + tx) : (ty * Gm::BX + tx);
  const bool lane_on = (D == 3) || lane < 16;
  constexpr int ZSTEP = 2 * Gm::BY * Gm::BX;
  const int zsel = (D == 3) ? 16 + 4 * tzb : 16;   // this lane's (z0, z1, off) group of a record
  T xs[D], gs = (T)0;
  if (lane < M) load_point(lane, xs, gs);
  for (uint32_t base = 0; base < M; base += kSpreadBatch) {
    // Stage 1: lane q prepares the record of point base + q.
    if (base + lane < M) {
      int o[3] = {0, 0, 0};
      T w[3][4];
      bool inside = point_comp<T, D>(jb, sh, xs, T0, TE, a, o, w);
#pragma unroll
      for (int b = 0; b < D; ++b) inside = inside && IB_IN(B.err, o[b], Gm::BX - 3);
      T ga = hmd * gs;
      if (!inside) {                 // X changed after binning: contribute nothing, report
        atomicOr(B.err, ERR_STALE);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          o[b] = 1;
#pragma unroll
          for (int t = 0; t < 4; ++t) w[b][t] = (T)0;
        }
        ga = (T)0;
      }
      T* rec = rec_s + lane * REC;
      T wxg[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) wxg[t] = w[0][t] * ga;
#pragma unroll
      for (int yy = 0; yy < 4; ++yy)
        store4(rec + yy * 4, wxg[0] * w[1][yy], wxg[1] * w[1][yy], wxg[2] * w[1][yy], wxg[3] * w[1][yy]);
      int off = o[1] * Gm::BX + o[0];
      if (D == 3) {
        off += o[D - 1] * Gm::BY * Gm::BX;
        const T ob = off_bits(off, (T)0);
        store4(rec + 16, w[D - 1][0], w[D - 1][2], ob, (T)0);
        store4(rec + 20, w[D - 1][1], w[D - 1][3], ob, (T)0);
      } else {
        store4(rec + 16, off_bits(off, (T)0), (T)0, (T)0, (T)0);
      }
    }
    // fetch the next batch's point data while this batch is added
    const uint32_t nq = base + kSpreadBatch + lane;
    if (nq < M) load_point(nq, xs, gs);
    __syncwarp();
    // Stage 2: the warp adds the points of the batch one by one.
    const int cnt = (int)min((uint32_t)kSpreadBatch, M - base);
    T npv = rec_s[lane & 15];
    T nz0, nz1, nob;
    if (D == 3) {
      load3(rec_s + zsel, nz0, nz1, nob);
    } else {
      nz0 = (T)1;
      nz1 = (T)0;
      nob = rec_s[16];
    }
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
      const int idx = bits_off(nob) + lane_off;
      const T pv = npv, z0 = nz0, z1 = nz1;
      if (i + 1 < cnt) {
        const T* rn = rec_s + (i + 1) * REC;
        npv = rn[lane & 15];
        if (D == 3) load3(rn + zsel, nz0, nz1, nob);
        else nob = rn[16];
      }
      if (lane_on && IB_IN(B.err, idx, (D == 3) ? Gm::BV - ZSTEP : Gm::BV)) {
        if (D == 3) {
          if (COMP) {
            two_sum_into(boxS + idx, boxE + idx, pv * z0);
            two_sum_into(boxS + idx + ZSTEP, boxE + idx + ZSTEP, pv * z1);
          } else {
            const T v0 = boxS[idx], v1 = boxS[idx + ZSTEP];
            boxS[idx] = v0 + pv * z0;
            boxS[idx + ZSTEP] = v1 + pv * z1;
          }
        } else {
          if (COMP) two_sum_into(boxS + idx, boxE + idx, pv);
          else boxS[idx] += pv;
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();
  // Box -> scratch [tile][comp][plane][BV], 16-byte vectors.
  constexpr int NV = (int)(PLANES * Gm::BV * sizeof(T) / 16);
  const uint4* src = reinterpret_cast<const uint4*>(boxS);
  uint4* dst = reinterpret_cast<uint4*>(boxes + unit * (long long)(PLANES * Gm::BV));
  for (int i = lane; i < NV; i += 32) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Spreading of three-component fields in 3-D (the MAC velocity grid, or three
// cell-centred components): one warp per 8^3 tile owns the three component
// boxes of the tile, so each point's cell map and weights are computed once
// for all components, and the three components' read-modify-writes of a point
// are independent of one another (loads first, then stores).  The same two
// stages and per-node order of additions as k_spread_warp.
// Record of a point (76 words, 19 16-byte chunks, an odd number so the
// stage-1 vector stores of 8 lanes hit distinct banks):
//   chunk j = ty*4 + tx (j < 16): (p0, p1, p2, pk), p_a = wx_a[tx] wy_a[ty] g_a
//     and pk the three box offsets (o_0 in bits 0-11, o_1 - o_0 + 512 in bits
//     12-21, o_2 - o_0 + 512 in bits 22-31);
//   chunk 16 + tzb: (wz[tzb], wz[tzb+2]) for xi_z = 1/2 (components 0 and 1),
//     then the same for component 2 (xi_z = 0 on the MAC grid);
// so stage 2 reads two vectors per point and lane.  Point data is fetched two
// batches ahead (sorted position and point index for batch b + 2, coordinates
// and forces for batch b + 1), so stage 1 never waits on a dependent gather.
// ---------------------------------------------------------------------------
constexpr int kRec3 = 76;

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
struct Dbl4 { double x, y, z, w; };   // four doubles read as two 16-byte halves
template <> struct Vec4<double> { using type = Dbl4; };
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
__device__ __forceinline__ float4 load4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ Dbl4 load4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return Dbl4{a.x, a.y, b.x, b.y};
}

// Stage 1 for one point: the record at rec, with multipliers g[a] (h^-d G_a
// for spreading, 1 for interpolation).  Returns false when X changed after
// binning (the record then carries zero weights at a corner inside the box).
template <typename T, bool MAC>
__device__ __forceinline__ bool tile3_record(const Job& jb, const Shape& sh, const Bins& B, const T xs[3],
                                             const T g[3], const int T0[3], const int TE[3], T* rec) {
  using Gm = Geo<3, 8>;
  int o0[3], dl[3];
  T w0[3][4], w1[3][4];
  bool inside = true;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    Cell1<T> c;
    const uint32_t e = point_cell<T>(xs[b], jb, b, c);
    const int n = jb.n[b];
    const int cphys = ((unsigned)c.i0 < (unsigned)n) ? c.i0 : modn(c.i0, n);
    dl[b] = c.i1 - c.i0;
    inside = inside && e == 0 && (unsigned)(cphys - T0[b]) < (unsigned)TE[b] && dl[b] >= -1 && dl[b] <= 0;
    o0[b] = cphys - T0[b] + 1;
    if (MAC) weights(sh.kernel, c.r0, c.c0, w0[b]);
    weights(sh.kernel, c.r1, c.c1, w1[b]);
  }
#pragma unroll
  for (int b = 0; b < 3; ++b)   // both staggerings' corners inside the box (debug build)
    inside = inside && IB_IN(B.err, o0[b], Gm::BX - 3) && IB_IN(B.err, o0[b] + dl[b], Gm::BX - 3);
  if (!inside) {                 // X changed after binning: contribute nothing, report
    atomicOr(B.err, ERR_STALE);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      o0[b] = 1;
      dl[b] = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) w0[b][t] = w1[b][t] = (T)0;
    }
  }
  // component a: xi = 0 in dimension a on the MAC grid, 1/2 elsewhere
  int oa[3];
  T wxg[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool hx = !MAC || a != 0, hy = !MAC || a != 1, hz = !MAC || a != 2;
#pragma unroll
    for (int t = 0; t < 4; ++t) wxg[a][t] = (hx ? w1[0][t] : w0[0][t]) * g[a];
    oa[a] = (o0[0] + (hx ? dl[0] : 0)) + (o0[1] + (hy ? dl[1] : 0)) * Gm::BX +
            (o0[2] + (hz ? dl[2] : 0)) * (Gm::BY * Gm::BX);
  }
  const T pkb = off_bits(oa[0] | ((oa[1] - oa[0] + 512) << 12) | ((oa[2] - oa[0] + 512) << 22), (T)0);
  const T* wy1 = MAC ? w0[1] : w1[1];   // component 1's y weights
#pragma unroll
  for (int yy = 0; yy < 4; ++yy)
#pragma unroll
    for (int xx = 0; xx < 4; ++xx)
      store4(rec + 4 * (yy * 4 + xx), wxg[0][xx] * w1[1][yy], wxg[1][xx] * wy1[yy], wxg[2][xx] * w1[1][yy], pkb);
  const T* wz2 = MAC ? w0[2] : w1[2];   // component 2's z weights
  store4(rec + 64, w1[2][0], w1[2][2], wz2[0], wz2[2]);
  store4(rec + 68, w1[2][1], w1[2][3], wz2[1], wz2[3]);
  return inside;
}

// Stage 2 for one batch of cnt records starting at rb (one record past the
// batch is allocated, so the look-ahead read of record cnt stays in bounds).
template <typename T, bool COMP>
__device__ __forceinline__ void tile3_add(T* box, const T* rb, int cnt, int lane, uint32_t* err) {
  using Gm = Geo<3, 8>;
  constexpr int PLANES = COMP ? 2 : 1;
  constexpr int ZSTEP = 2 * Gm::BY * Gm::BX;
  const int tx = lane & 3, ty = (lane >> 2) & 3, tzb = lane >> 4;
  const int lane_off = (tzb * Gm::BY + ty) * Gm::BX + tx;
  const int ch = 4 * (lane & 15);
  const int zc = 64 + 4 * tzb;
  typename Vec4<T>::type q = load4(rb + ch);
  typename Vec4<T>::type z = load4(rb + zc);
#pragma unroll 2
  for (int i = 0; i < cnt; ++i) {
    const T c0 = q.x, c1 = q.y, c2 = q.z;
    const int pk = bits_off(q.w);
    const T z0 = z.x, z1 = z.y, z20 = z.z, z21 = z.w;
    const T* rn = rb + (i + 1) * kRec3;
    q = load4(rn + ch);
    z = load4(rn + zc);
    const int q0 = (pk & 4095) + lane_off;
    const int q1 = q0 + ((pk >> 12) & 1023) - 512 + PLANES * Gm::BV;
    const int q2 = q0 + (int)((unsigned)pk >> 22) - 512 + 2 * PLANES * Gm::BV;
    if (!(IB_IN(err, q0, Gm::BV - ZSTEP) && IB_IN(err, q1 - PLANES * Gm::BV, Gm::BV - ZSTEP) &&
          IB_IN(err, q2 - 2 * PLANES * Gm::BV, Gm::BV - ZSTEP))) {
      __syncwarp();
      continue;
    }
    if (COMP) {
      two_sum_into(box + q0, box + q0 + Gm::BV, c0 * z0);
      two_sum_into(box + q0 + ZSTEP, box + q0 + ZSTEP + Gm::BV, c0 * z1);
      two_sum_into(box + q1, box + q1 + Gm::BV, c1 * z0);
      two_sum_into(box + q1 + ZSTEP, box + q1 + ZSTEP + Gm::BV, c1 * z1);
      two_sum_into(box + q2, box + q2 + Gm::BV, c2 * z20);
      two_sum_into(box + q2 + ZSTEP, box + q2 + ZSTEP + Gm::BV, c2 * z21);
    } else {
      const T v00 = box[q0], v01 = box[q0 + ZSTEP];
      const T v10 = box[q1], v11 = box[q1 + ZSTEP];
      const T v20 = box[q2], v21 = box[q2 + ZSTEP];
      box[q0] = v00 + c0 * z0;
      box[q0 + ZSTEP] = v01 + c0 * z1;
      box[q1] = v10 + c1 * z0;
      box[q1 + ZSTEP] = v11 + c1 * z1;
      box[q2] = v20 + c2 * z20;
      box[q2 + ZSTEP] = v21 + c2 * z21;
    }
    __syncwarp();
  }
}

// The job of a tile kernel's block (spreading, interpolation): a single-job
// launch reads it straight from the kernel parameters (constant-bank operands;
// filling a shared-memory copy costs each tile 0.2-0.7 us), a batched wave from
// the block's shared-memory copy.  Two specialisations, so that neither reads
// through a generic pointer that may point to either space (which was slower
// than both).
template <bool ONE> __device__ __forceinline__ const Job& pick_job(const Jobs& J, const Job& s);
template <> __device__ __forceinline__ const Job& pick_job<true>(const Jobs& J, const Job&) { return J.one; }
template <> __device__ __forceinline__ const Job& pick_job<false>(const Jobs&, const Job& s) { return s; }

template <typename T, bool COMP, bool MAC, bool ONE>
__global__ void __launch_bounds__(32) k_spread_tile3(const __grid_constant__ Jobs J, const Shape sh, const Bins B,
                                                     T* __restrict__ boxes, int skip_empty, long long tile_begin,
                                                     int overlap) {
  constexpr int TS = 8;
  // Under IB_OVERLAP_PREVIOUS the caller guarantees that the kernel before
  // wrote nothing this one reads: only block 0 waits for it (so that this
  // kernel's completion still implies the previous one's).
  if (!overlap || blockIdx.x == 0) pdl_wait();
  using Gm = Geo<3, TS>;
  constexpr int PLANES = COMP ? 2 : 1;
  constexpr int NROWS = TS * TS;
  static_assert((3 * PLANES * Gm::BV * sizeof(T)) % 16 == 0, "16-byte sections");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t rstart[NROWS];
  __shared__ uint32_t rpre[NROWS + 1];
  __shared__ Job sjob;
  const int lane = threadIdx.x;
  const long long gt = tile_begin + blockIdx.x;   // tile_begin > 0: a z-slab's tiles only
  // boxes of component a: sums at a * PLANES * BV, errors (compensated) at + BV;
  // then kSpreadBatch + 1 records
  T* box = reinterpret_cast<T*>(smem_raw);
  T* rec_s = box + 3 * PLANES * Gm::BV;
  if constexpr (!ONE) {
    const int j = __shfl_sync(0xffffffffu, lane == 0 ? job_of_tile(J, gt) : 0, 0);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&job_at(J, j));
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sjob);
    for (int w = lane; w < (int)(sizeof(Job) / 4); w += 32) dst[w] = src[w];
    __syncwarp();
  }
  const Job& jb = pick_job<ONE>(J, sjob);
  if (jb.G == nullptr) return;
  int T0[3], TE[3];
  tile_coords<3, TS>(jb.ntile, jb.n, gt - jb.tile_base, T0, TE);
  // Cell rows of the tile: counts requested first, boxes zeroed while they arrive.
  const int rows = TE[1] * TE[2];
  uint32_t st[NROWS / 32], cn[NROWS / 32];
#pragma unroll
  for (int k = 0; k < NROWS / 32; ++k) {
    const int r = lane + 32 * k;
    st[k] = cn[k] = 0;
    if (r < rows) {
      const int y = T0[1] + r % TE[1];
      const int z = T0[2] + r / TE[1];
      const long long cell = jb.cell_base + T0[0] + (long long)jb.n[0] * (y + (long long)jb.n[1] * z);
      if (IB_IN(B.err, cell + TE[0], B.ncell_total + 1)) {
        st[k] = B.count[cell];
        cn[k] = B.count[cell + TE[0]];
      }
    }
  }
  {
    constexpr int NV = (int)(3 * PLANES * Gm::BV * sizeof(T) / 16);
    uint4* zz = reinterpret_cast<uint4*>(box);
    for (int i = lane; i < NV; i += 32) zz[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  uint32_t M = 0;
#pragma unroll
  for (int k = 0; k < NROWS / 32; ++k) {
    const uint32_t cnt = cn[k] - st[k];
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    rstart[lane + 32 * k] = st[k];
    rpre[lane + 32 * k] = M + inc - cnt;
    M += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  if (skip_empty) {                                // sparse call: an empty tile writes no boxes
    if (lane == 0) B.tflags[gt] = M > 0 ? 1u : 0u;
    if (M == 0) return;
  }

  const T* Xg = (const T*)jb.X;
  const T* Gp = (const T*)jb.G;
  // sorted point q of the tile -> its global point index
  auto point_of = [&](uint32_t q) -> uint32_t {
    int lo = 0;
#pragma unroll
    for (int step = NROWS / 2; step >= 1; step >>= 1)
      if (lo + step < rows && rpre[lo + step] <= q) lo += step;
    const long long pi = (long long)rstart[lo] + (q - rpre[lo]);
    return IB_IN(B.err, pi, B.npts_total) ? B.perm[pi] : (uint32_t)jb.pt_base;
  };
  auto fetch = [&](uint32_t g, T xs[3], T gs[3]) {
    long long li = (long long)g - jb.pt_base;
    if (!IB_IN(B.err, li, jb.npts)) li = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) xs[b] = Xg[li * 3 + b];
#pragma unroll
    for (int b = 0; b < 3; ++b) gs[b] = Gp[li * 3 + b];
  };
  T xs[3], gs[3] = {(T)0, (T)0, (T)0};
  uint32_t pn = 0;                                 // point index of batch b + 1 (this lane)
  if (lane < M) fetch(point_of(lane), xs, gs);
  if (kSpreadBatch + lane < M) pn = point_of(kSpreadBatch + lane);
  for (uint32_t base = 0; base < M; base += kSpreadBatch) {
    if (base + lane < M) {
      const T hmd = (T)jb.hmd;
      const T g[3] = {hmd * gs[0], hmd * gs[1], hmd * gs[2]};
      tile3_record<T, MAC>(jb, sh, B, xs, g, T0, TE, rec_s + lane * kRec3);
    }
    if (base + kSpreadBatch + lane < M) fetch(pn, xs, gs);
    if (base + 2 * kSpreadBatch + lane < M) pn = point_of(base + 2 * kSpreadBatch + lane);
    __syncwarp();
    tile3_add<T, COMP>(box, rec_s, (int)min((uint32_t)kSpreadBatch, M - base), lane, B.err);
    __syncwarp();
  }
  // Boxes -> scratch [tile][comp][plane][BV]: the shared layout, one contiguous copy.
  constexpr int NV = (int)(3 * PLANES * Gm::BV * sizeof(T) / 16);
  const uint4* src = reinterpret_cast<const uint4*>(box);
  uint4* dst = reinterpret_cast<uint4*>(boxes + gt * (long long)(3 * PLANES * Gm::BV));
  for (int i = lane; i < NV; i += 32) dst[i] = src[i];
  // The combination may launch once every tile is done (it waits for this
  // kernel before reading a box).  Signalled at the end: combination blocks
  // launched at the start of the last wave only sat waiting on the SMs and
  // slowed the spread call (177 us against 165 us).
  pdl_launch_dependents();
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

// Fast cover list for n >= TS + 4 (a box never wraps onto its own tile):
// entries in increasing unwrapped position, then tile -- the periodic copy
// x - n in tile 0, the previous tile, the node's own tile, the next tile,
// and the periodic copy x + n in the last tile -- at most 3 of them at once.
// Kept in three scalar slots so the list stays in registers.
struct Cover3 {
  int t0, o0, t1, o1, t2, o2, n;
  __device__ __forceinline__ void push(int t, int o) {
    if (n == 0) { t0 = t; o0 = o; } else if (n == 1) { t1 = t; o1 = o; } else { t2 = t; o2 = o; }
    ++n;
  }
  __device__ __forceinline__ int t(int i) const { return i == 0 ? t0 : (i == 1 ? t1 : t2); }
  __device__ __forceinline__ int o(int i) const { return i == 0 ? o0 : (i == 1 ? o1 : o2); }
};

template <int TS>
__device__ __forceinline__ Cover3 cover_fast(int x, int n, int ntile) {
  Cover3 c;
  c.n = 0;
  c.t0 = c.o0 = c.t1 = c.o1 = c.t2 = c.o2 = 0;
  const int t = x / TS, xl = x - t * TS;
  if (x >= n - 2) c.push(0, x - n + 2);
  if (xl < 2 && t >= 1) c.push(t - 1, xl + TS + 2);
  c.push(t, xl + 2);
  if (xl >= TS - 2 && t + 1 < ntile) c.push(t + 1, xl - TS + 2);
  // The copy x + n: the last tile's box, and the one before it when the last
  // tile holds a single cell (its box then ends exactly at node n).
  const int vp = x + n - (ntile - 2) * TS + 2;
  if (vp < TS + 4) c.push(ntile - 2, vp);
  const int vo = x + n - (ntile - 1) * TS + 2;
  if (vo < TS + 4) c.push(ntile - 1, vo);
  return c;
}

// Debug build: every entry of a cover list names a tile of the job's row of
// tiles and an offset inside its box (room for `width` consecutive nodes).
template <int TS>
__device__ __forceinline__ bool cover_ok(uint32_t* err, const Cover3& c, int ntile, int width) {
#ifdef IB_DEBUG_BOUNDS
  bool ok = IB_IN(err, c.n, 4);
  for (int i = 0; i < 3; ++i)
    if (i < c.n) ok = ok && IB_IN(err, c.t(i), ntile) && IB_IN(err, c.o(i), TS + 4 - (width - 1));
  return ok;
#else
  (void)err; (void)c; (void)ntile; (void)width;
  return true;
#endif
}

template <typename T, int D, int TS, bool CP, bool CHECK>
__device__ __noinline__ void combine_general(const Jobs& J, int j, const Shape& sh, const T* __restrict__ boxes,
                                             const uint32_t* __restrict__ tflags, const int* x, long long lc,
                                             int accumulate, uint32_t* err) {
  using Gm = Geo<D, TS>;
  const Job& jb = job_at(J, j);
  int tl[3][kMaxCover], of[3][kMaxCover], nco[3];
  for (int b = 0; b < D; ++b) {
    nco[b] = cover_list<TS>(x[b], jb.n[b], jb.ntile[b], tl[b], of[b]);
    for (int i = 0; i < nco[b]; ++i)
      if (!(IB_IN(err, tl[b][i], jb.ntile[b]) && IB_IN(err, of[b][i], TS + 4))) return;
  }
  if (D == 2) {
    nco[2] = 1;
    tl[2][0] = 0;
    of[2][0] = 0;
  }
  const int nc = sh.ncomp;
  const long long plane = (long long)(CP ? 2 : 1) * Gm::BV;
  T* f = (T*)jb.f;
  for (int a = 0; a < nc; ++a) {
    T S = 0, E = 0;
    for (int iz = 0; iz < nco[2]; ++iz)
      for (int iy = 0; iy < nco[1]; ++iy)
        for (int ix = 0; ix < nco[0]; ++ix) {
          const long long tile = jb.tile_base + tl[0][ix] + (long long)jb.ntile[0] * (tl[1][iy] + (long long)jb.ntile[1] * tl[2][iz]);
          if (CHECK && !tflags[tile]) continue;  // empty tile: its boxes are zero and were not written
          const long long idx = (tile * nc + a) * plane + (of[2][iz] * Gm::BY + of[1][iy]) * Gm::BX + of[0][ix];
          if (CP) {
            const T sv = boxes[idx];
            const T ev = boxes[idx + Gm::BV];
            const T sum = S + sv;
            const T bb = sum - S;
            E += ((S - (sum - bb)) + (sv - bb)) + ev;
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

// V consecutive x nodes per thread (V = 2 needs every job's n0 even: then the
// two nodes of an even-aligned pair have the same covering boxes at
// consecutive, 2-element-aligned offsets, and each box is read with one
// vector load).
template <typename T, int V>
struct Vec;
template <> struct Vec<float, 1> { using type = float; };
template <> struct Vec<double, 1> { using type = double; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<double, 2> { using type = double2; };

template <typename T, int V>
__device__ __forceinline__ void load_v(const T* p, T* out) {
  if constexpr (V == 1) {
    out[0] = *p;
  } else {
    const typename Vec<T, 2>::type q = *reinterpret_cast<const typename Vec<T, 2>::type*>(p);
    out[0] = q.x;
    out[1] = q.y;
  }
}

template <typename T, int V>
__device__ __forceinline__ void store_v(T* p, const T* v) {
  if constexpr (V == 1) {
    *p = v[0];
  } else {
    typename Vec<T, 2>::type q;
    q.x = v[0];
    q.y = v[1];
    *reinterpret_cast<typename Vec<T, 2>::type*>(p) = q;
  }
}

// CHECK: some tiles may be empty (a sparse call); their boxes were not written
// and count as zero.
template <typename T, int D, int TS, bool CP, int V, bool CHECK>
__global__ void __launch_bounds__(kThreads) k_spread_combine(const __grid_constant__ Jobs J, const Shape sh,
                                                             const T* __restrict__ boxes,
                                                             const uint32_t* __restrict__ tflags, long long ncell_total,
                                                             int accumulate, uint32_t* err, long long cell_begin) {
  using Gm = Geo<D, TS>;
  pdl_wait();   // the tile boxes
  pdl_launch_dependents();   // only a call under IB_OVERLAP_PREVIOUS reads before waiting, and not f
  // Blocks walk the grid from its end: the tile kernel writes the boxes in
  // tile order, so the last-written boxes (the ones still in L2) are read first.
  // Cells [cell_begin, ncell_total): every cell, or a z-slab's planes.
  const int c = (int)cell_begin + ((gridDim.x - 1 - blockIdx.x) * kThreads + threadIdx.x) * V;   // ids below 2^31
  if (c >= ncell_total) return;
  const int jj = job_of_cell(J, c);
  const Job jb = job_at(J, jj);
  if (jb.G == nullptr) return;
  const int lc = c - (int)jb.cell_base;
  int x[3];
  const int q = udiv(lc, jb.n[0], jb.mg[0]);
  x[0] = lc - q * jb.n[0];
  if (D == 3) {
    x[2] = udiv(q, jb.n[1], jb.mg[1]);
    x[1] = q - x[2] * jb.n[1];
  } else {
    x[1] = q;
    x[2] = 0;
  }
  bool fast = true;
#pragma unroll
  for (int b = 0; b < D; ++b) fast = fast && jb.n[b] >= TS + 4;
  if (!fast) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      int xv[3] = {x[0] + v, x[1], x[2]};
      combine_general<T, D, TS, CP, CHECK>(J, jj, sh, boxes, tflags, xv, lc + v, accumulate, err);
    }
    return;
  }
  const Cover3 cx = cover_fast<TS>(x[0], jb.n[0], jb.ntile[0]);
  const Cover3 cy = cover_fast<TS>(x[1], jb.n[1], jb.ntile[1]);
  Cover3 cz;
  if (D == 3) {
    cz = cover_fast<TS>(x[2], jb.n[2], jb.ntile[2]);
  } else {
    cz.n = 1;
    cz.t0 = cz.o0 = cz.t1 = cz.o1 = cz.t2 = cz.o2 = 0;
  }
  if (!(cover_ok<TS>(err, cx, jb.ntile[0], V) && cover_ok<TS>(err, cy, jb.ntile[1], 1) &&
        (D == 2 || cover_ok<TS>(err, cz, jb.ntile[2], 1))))
    return;
  const int nc = sh.ncomp;
  const long long plane = (long long)(CP ? 2 : 1) * Gm::BV;
  T S[4][V], E[4][V];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int v = 0; v < V; ++v) S[a][v] = E[a][v] = (T)0;
  // Covering boxes in increasing (z, y, x) unwrapped order; every component
  // sums them in that same order.
  if constexpr (!CP && sizeof(T) == 4) {
    if (cx.n <= 2 && cy.n <= 2 && cz.n <= 2 && nc <= 3) {
      // At most 2 boxes per dimension (every node but a few at the periodic
      // seam): the up to 8 entries of every component are loaded before any
      // addition, so the loads are in flight together; the sums keep the order.
      const T* bp[8];
      bool ok[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int iz = k >> 2, iy = (k >> 1) & 1, ix = k & 1;
        ok[k] = iz < cz.n && iy < cy.n && ix < cx.n;
        const int trow = (int)jb.tile_base + jb.ntile[0] * (cy.t(iy) + jb.ntile[1] * cz.t(iz));
        const int orow = (cz.o(iz) * Gm::BY + cy.o(iy)) * Gm::BX;
        if (CHECK) ok[k] = ok[k] && tflags[trow + cx.t(ix)] != 0u;   // empty tile: zero boxes, not written
        bp[k] = ok[k] ? boxes + (long long)(trow + cx.t(ix)) * nc * plane + (orow + cx.o(ix)) : boxes;
      }
      T val[3][8][V];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (a < nc && ok[k]) load_v<T, V>(bp[k] + a * plane, val[a][k]);
          else {
#pragma unroll
            for (int v = 0; v < V; ++v) val[a][k][v] = (T)0;
          }
        }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (ok[k]) {
#pragma unroll
            for (int v = 0; v < V; ++v) S[a][v] += val[a][k][v];
          }
      T* f = (T*)jb.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= nc) break;
        T* o = f + a * jb.ncell + lc;
        T out[V];
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = S[a][v];
        if (accumulate) {
          T old[V];
          load_v<T, V>(o, old);
#pragma unroll
          for (int v = 0; v < V; ++v) out[v] = old[v] + out[v];
        }
        store_v<T, V>(o, out);
      }
      return;
    }
  }
#pragma unroll
  for (int iz = 0; iz < 3; ++iz) {
    if (iz >= cz.n) break;
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) {
      if (iy >= cy.n) break;
      const int trow = (int)jb.tile_base + jb.ntile[0] * (cy.t(iy) + jb.ntile[1] * cz.t(iz));
      const int orow = (cz.o(iz) * Gm::BY + cy.o(iy)) * Gm::BX;
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        if (ix >= cx.n) break;
        if (CHECK && !tflags[trow + cx.t(ix)]) continue;   // empty tile: zero boxes, not written
        const T* bp = boxes + (long long)(trow + cx.t(ix)) * nc * plane + (orow + cx.o(ix));
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (a >= nc) break;
          T sv[V];
          load_v<T, V>(bp + a * plane, sv);
          if (CP) {
            T ev[V];
            load_v<T, V>(bp + a * plane + Gm::BV, ev);
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const T sum = S[a][v] + sv[v];
              const T bb = sum - S[a][v];
              E[a][v] += ((S[a][v] - (sum - bb)) + (sv[v] - bb)) + ev[v];
              S[a][v] = sum;
            }
          } else {
#pragma unroll
            for (int v = 0; v < V; ++v) S[a][v] += sv[v];
          }
        }
      }
    }
  }
  T* f = (T*)jb.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (a >= nc) break;
    T val[V];
#pragma unroll
    for (int v = 0; v < V; ++v) val[v] = CP ? S[a][v] + E[a][v] : S[a][v];
    T* o = f + a * jb.ncell + lc;
    if (accumulate) {
      T old[V];
      load_v<T, V>(o, old);
#pragma unroll
      for (int v = 0; v < V; ++v) val[v] = old[v] + val[v];
    }
    store_v<T, V>(o, val);
  }
}

// ---------------------------------------------------------------------------
// Node offsets of a point's 4 support nodes in one dimension (wrapped).
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void node_offsets(const Job& jb, int b, int i, long long stride, long long off[4]) {
  const int n = jb.n[b];
  const int base = ((unsigned)i < (unsigned)n) ? i : modn(i, n);
#pragma unroll
  for (int t = 0; t < 4; ++t) off[t] = (long long)wrapn(base + t - 1, n) * stride;
}

// ---------------------------------------------------------------------------
// Grid values of a tile's box -- nodes T0 - 2 .. T0 + TS + 1 (unwrapped) of
// every component -- copied into shared memory through registers: each thread
// loads stage_k entries (pairs when n0 is even and the field 2-entry
// aligned: an x pair starting at an even node then never straddles the
// periodic seam, T0 - 2 being even) before storing them, so the loads of a
// thread are in flight together, and the 32 lanes of a store write
// consecutive shared addresses (a row of the box after another).  An
// asynchronous 8-byte copy (cp.async) costs about 22 shared wavefronts per
// warp instruction here against 2 for the plain stores.  Wrapped column, row
// and plane offsets come from small tables built with a true modulo, so any
// grid size n >= 1 (several periodic images inside one box) is read in range.
// Ends with the stores issued; the caller synchronises the block.
// ---------------------------------------------------------------------------
// Entries a thread has in flight while staging: 12 FP32 pairs (a thread's
// share of a 3-D box, 20-21 pairs, in two rounds at 72 registers; 24 in one
// round cost 80 registers and spills), half as many FP64 pairs.
template <typename T> __host__ __device__ constexpr int stage_k() { return sizeof(T) == 4 ? 12 : 6; }

template <typename T, int D, int TS, int NTH>
__device__ __forceinline__ void stage_box(const Job& jb, int nc, const int T0[3], T* box, uint32_t* err) {
  using Gm = Geo<D, TS>;
  static_assert(NTH >= Gm::BX && NTH >= Gm::BY, "one thread per table entry");
  __shared__ int xoff_s[Gm::BX];
  __shared__ int yoff_s[Gm::BY];
  __shared__ int zoff_s[Gm::BZ];
  const int tid = threadIdx.x;
  const int n0 = jb.n[0], n1 = jb.n[1];
  if (tid < Gm::BX) xoff_s[tid] = modn(T0[0] - 2 + tid, n0);
  if (tid < Gm::BY) yoff_s[tid] = modn(T0[1] - 2 + tid, n1) * n0;
  if (tid < Gm::BZ) zoff_s[tid] = (D == 3) ? modn(T0[2] - 2 + tid, jb.n[2]) * n0 * n1 : 0;
  __syncthreads();
  const T* u = (const T*)jb.u;
  const int nrows_box = nc * Gm::BZ * Gm::BY;
  constexpr int K = stage_k<T>();
  if ((n0 % 2) == 0 && ((uintptr_t)u % (2 * sizeof(T))) == 0) {
    using P2 = typename Vec2<T>::type;
    constexpr int NP = Gm::BX / 2;
    const int total = nrows_box * NP;
    for (int i0 = tid; i0 < total; i0 += NTH * K) {
      P2 v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = i0 + k * NTH;
        if (i < total) {
          const int row = i / NP;
          const int c = i - row * NP;
          const int a = row / (Gm::BZ * Gm::BY);
          const int rem = row - a * (Gm::BZ * Gm::BY);
          const int bz = rem / Gm::BY;
          const int by = rem - bz * Gm::BY;
          const long long si = (long long)a * jb.ncell + (zoff_s[bz] + yoff_s[by] + xoff_s[2 * c]);
          v[k] = IB_IN(err, si, nc * jb.ncell - 1) ? *reinterpret_cast<const P2*>(u + si) : P2{};
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = i0 + k * NTH;
        if (i < total) *reinterpret_cast<P2*>(box + 2 * i) = v[k];   // row * BX + 2 c = 2 i
      }
    }
  } else {
    const int total = nrows_box * Gm::BX;
    for (int i0 = tid; i0 < total; i0 += NTH * K) {
      T v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = i0 + k * NTH;
        if (i < total) {
          const int row = i / Gm::BX;
          const int bx = i - row * Gm::BX;
          const int a = row / (Gm::BZ * Gm::BY);
          const int rem = row - a * (Gm::BZ * Gm::BY);
          const int bz = rem / Gm::BY;
          const int by = rem - bz * Gm::BY;
          const long long si = (long long)a * jb.ncell + (zoff_s[bz] + yoff_s[by] + xoff_s[bx]);
          v[k] = IB_IN(err, si, nc * jb.ncell) ? u[si] : (T)0;
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = i0 + k * NTH;
        if (i < total) box[i] = v[k];                                 // row * BX + bx = i
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Interpolation by tiles: the CTA of a tile copies the grid values of the
// tile plus a 2-node apron (every component) into shared memory with
// asynchronous copies, then each thread takes one of the tile's points (cell
// order) and sums its 4^d support from shared memory.  Points outside every
// tile (invalid positions) are handled by one extra block of the same launch.
// ---------------------------------------------------------------------------
constexpr int kInterpThreads = 128;   // 64 registers per thread: 8 tiles per SM
constexpr int kInterpWarps = kInterpThreads / 32;
static_assert(kInterpThreads >= 64, "a tile has up to 64 cell rows (3-D) or 32 (2-D), one per thread");

template <typename T, int D, int TS, bool ONE>
__global__ void __launch_bounds__(kInterpThreads) k_interp_tile(const __grid_constant__ Jobs J, const Shape sh,
                                                                 const Bins B, const T scale) {
  using Gm = Geo<D, TS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* box = reinterpret_cast<T*>(smem_raw);
  __shared__ uint32_t rstart[kInterpThreads];
  __shared__ uint32_t rpre[kInterpThreads + 1];
  __shared__ uint32_t wsum[kInterpWarps];
  __shared__ Job sjob;                  // one copy of the job per CTA (broadcast reads)
  pdl_wait();                           // the bins (and u) of the kernels before
  pdl_launch_dependents();              // a spreading call under IB_OVERLAP_PREVIOUS may start
  const long long gt = blockIdx.x;
  if (gt == gridDim.x - 1) {
    // The last block: points with an invalid position, which sit after every
    // valid point in the bins, get U = NaN (no point of a valid input).
    for (long long p = B.count[B.ncell_total] + threadIdx.x; p < B.npts_total; p += kInterpThreads) {
      const uint32_t g = B.perm[p];
      const Job& jp = job_at(J, job_of_point(J, (long long)g));
      if (jp.u == nullptr) continue;
      T* U = (T*)jp.U + ((long long)g - jp.pt_base) * sh.ncomp;
      for (int a = 0; a < sh.ncomp; ++a) U[a] = (T)NAN;
    }
    return;
  }
  if constexpr (!ONE) {
    // a batched wave: the tile's job into shared memory, one word per thread
    const int j = job_of_itile(J, gt);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&job_at(J, j));
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sjob);
    for (int w = threadIdx.x; w < (int)(sizeof(Job) / 4); w += kInterpThreads) dst[w] = src[w];
    __syncthreads();
  }
  const Job& jb = pick_job<ONE>(J, sjob);
  if (jb.u == nullptr) return;
  int T0[3], TE[3];
  tile_coords<D, TS>(jb.itile, jb.n, gt - jb.itile_base, T0, TE);
  const int nc = sh.ncomp;
  const int tid = threadIdx.x;

  // Rows of the tile's own cells (x fastest inside a row): start and count in the
  // bins, requested before the box is staged.
  const int nrows = (D == 3) ? TE[1] * TE[2] : TE[1];
  uint32_t cnt = 0, st = 0;
  if (tid < nrows) {
    const int y = T0[1] + ((D == 3) ? tid % TE[1] : tid);
    const int z = (D == 3) ? T0[2] + tid / TE[1] : 0;
    const long long cell = jb.cell_base + T0[0] + (long long)jb.n[0] * (y + (long long)jb.n[1] * z);
    st = B.count[cell];
    cnt = B.count[cell + TE[0]] - st;
  }
  stage_box<T, D, TS, kInterpThreads>(jb, nc, T0, box, B.err);
  {
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t yv = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += yv;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = (lane < kInterpWarps) ? wsum[lane] : 0u;
#pragma unroll
      for (int o = 1; o < kInterpWarps; o <<= 1) {
        const uint32_t yv = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += yv;
      }
      if (lane < kInterpWarps) wsum[lane] = t;
    }
    __syncthreads();
    const uint32_t before = (warp > 0) ? wsum[warp - 1] : 0u;
    rstart[tid] = st;
    rpre[tid] = before + inc - cnt;
    if (tid == 0) rpre[kInterpThreads] = wsum[kInterpWarps - 1];
  }
  __syncthreads();

  const uint32_t P = rpre[kInterpThreads];
  // Sorted point q of the tile -> global point index.
  auto point_of = [&](uint32_t q) -> uint32_t {
    int lo = 0, hi = nrows - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rpre[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const long long pi = (long long)rstart[lo] + (q - rpre[lo]);
    const uint32_t gp = IB_IN(B.err, pi, B.npts_total) ? B.perm[pi] : (uint32_t)jb.pt_base;
    return IB_IN(B.err, (long long)gp - jb.pt_base, jb.npts) ? gp : (uint32_t)jb.pt_base;
  };
  const T* Xg = (const T*)jb.X;
  // Software pipeline over this thread's points: the next point's index is
  // requested at the top of an iteration and its coordinates after this
  // point's weights, so neither load is waited for on the critical path.
  uint32_t g = 0;
  T xs[D];
  if (tid < P) {
    g = point_of(tid);
#pragma unroll
    for (int b = 0; b < D; ++b) xs[b] = Xg[((long long)g - jb.pt_base) * D + b];
  }
  for (uint32_t q = tid; q < P; q += kInterpThreads) {
    const bool more = q + kInterpThreads < P;
    const uint32_t gn = more ? point_of(q + kInterpThreads) : 0u;
    const long long li = (long long)g - jb.pt_base;
    PointBox<T, D> Pb;
    T* U = (T*)jb.U + li * nc;
    bool ok = point_box<T, D>(jb, sh, xs, T0, TE, Pb);
#pragma unroll
    for (int b = 0; b < D; ++b)   // both staggerings' corners inside the box (debug build)
      ok = ok && IB_IN(B.err, Pb.o0[b], Gm::BX - 3) && IB_IN(B.err, Pb.o1[b], Gm::BX - 3);
    if (more) {
#pragma unroll
      for (int b = 0; b < D; ++b) xs[b] = Xg[((long long)gn - jb.pt_base) * D + b];
    }
    g = gn;
    if (!ok) {
      atomicOr(B.err, ERR_STALE);        // X changed after binning: no gather outside the box
      for (int a = 0; a < nc; ++a) U[a] = (T)NAN;
      continue;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (a >= nc) break;
      const bool hx = half_stag(sh, a, 0), hy = half_stag(sh, a, 1);
      T wx[4], wy[4], wz[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        wx[t] = hx ? Pb.w1[0][t] : Pb.w0[0][t];
        wy[t] = hy ? Pb.w1[1][t] : Pb.w0[1][t];
        wz[t] = (D == 3) ? (half_stag(sh, a, 2) ? Pb.w1[D - 1][t] : Pb.w0[D - 1][t]) : (T)1;
      }
      const int ox = hx ? Pb.o1[0] : Pb.o0[0];
      const int oy = hy ? Pb.o1[1] : Pb.o0[1];
      const int oz = (D == 3) ? (half_stag(sh, a, 2) ? Pb.o1[D - 1] : Pb.o0[D - 1]) : 0;
      const T* bp = box + a * Gm::BV + (oz * Gm::BY + oy) * Gm::BX + ox;
      T acc = 0;
#pragma unroll
      for (int tz = 0; tz < Gm::NT; ++tz) {
        T accy = 0;
#pragma unroll
        for (int ty = 0; ty < 4; ++ty) {
          const T* row = bp + (tz * Gm::BY + ty) * Gm::BX;
          T accx = wx[0] * row[0];
#pragma unroll
          for (int tx = 1; tx < 4; ++tx) accx += wx[tx] * row[tx];
          accy += wy[ty] * accx;
        }
        acc += wz[tz] * accy;
      }
      U[a] = acc * scale;
    }
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
  const Job jb = job_at(J, job_of_point(J, (long long)g));
  const long long li = (long long)g - jb.pt_base;
  if (!IB_IN(B.err, li, jb.npts)) return;
  const int nc = sh.ncomp;
  const T* Xp = (const T*)jb.X + li * D;
  T* Dp = Dout + li * D;
  Cell1<T> c[D];
  uint32_t err = 0;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    err |= point_cell<T>(Xp[b], jb, b, c[b]);
    if (!in_bounds(jb, b, c[b])) err |= ERR_RANGE;
  }
  if (err) {
#pragma unroll
    for (int b = 0; b < D; ++b) Dp[b] = (T)NAN;
    return;
  }
  T w0[D][4], w1[D][4], d0[D][4], d1[D][4];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    if (sh.mac) weights_and_derivs<T>(sh.kernel, c[b].r0, c[b].c0, w0[b], d0[b]);
    weights_and_derivs<T>(sh.kernel, c[b].r1, c[b].c1, w1[b], d1[b]);
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
          const T val = IB_IN(B.err, oz[tz] + oy[ty] + ox[tx], jb.ncell) ? __ldg(row + ox[tx]) : (T)0;
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
// Each thread moves P = 16 / sizeof(T) consecutive points (D P elements, a
// whole number of 16-byte vectors) with vector loads and stores when X, U and
// Xout are 16-byte aligned; the last partial group and unaligned arrays take
// the scalar path.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_advect(const __grid_constant__ Jobs J, const T* __restrict__ U, T dt,
                                                     T* __restrict__ Xout, int vec, int overlap) {
  constexpr int P = 16 / (int)sizeof(T);
  constexpr int NE = P * D;
  constexpr int NV = NE * (int)sizeof(T) / 16;
  // IB_OVERLAP_PREVIOUS: the kernel before wrote neither X nor U; block 0 still
  // waits for it, so that this kernel's completion implies the previous one's.
  if (!overlap || blockIdx.x == 0) pdl_wait();
  const long long n = J.one.npts;
  const long long p0 = ((long long)blockIdx.x * kThreads + threadIdx.x) * P;
  if (p0 >= n) return;
  const T* X = (const T*)J.one.X;
  T L[D];
  bool wrap[D];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    L[b] = (T)J.one.Ld[b];
    wrap[b] = J.one.bnd[b] == 0;    // bounded dimensions keep the position as it is
  }
  const long long e0 = p0 * D;
  const bool full = vec && p0 + P <= n;
  const int ne = full ? NE : (int)((n - p0) * D);
  T xv[NE], uv[NE];
  if (full) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      reinterpret_cast<uint4*>(xv)[k] = reinterpret_cast<const uint4*>(X + e0)[k];
      reinterpret_cast<uint4*>(uv)[k] = reinterpret_cast<const uint4*>(U + e0)[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < NE; ++k)
      if (k < ne) {
        xv[k] = X[e0 + k];
        uv[k] = U[e0 + k];
      }
  }
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    const T Lb = L[k % D];
    T x = xv[k] + dt * uv[k];
    if (wrap[k % D] && (x >= Lb || x < (T)0)) {
      x -= Lb * floor(x / Lb);
      if (x >= Lb) x -= Lb;
      if (x < (T)0) x += Lb;
    }
    xv[k] = x;
  }
  if (full) {
#pragma unroll
    for (int k = 0; k < NV; ++k) reinterpret_cast<uint4*>(Xout + e0)[k] = reinterpret_cast<const uint4*>(xv)[k];
  } else {
#pragma unroll
    for (int k = 0; k < NE; ++k)
      if (k < ne) Xout[e0 + k] = xv[k];
  }
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  // Always set: dynamic plus static shared memory may pass 48 KB while the dynamic part alone does not.
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int D, int TS>
size_t spread_smem(bool comp) {
  using Gm = Geo<D, TS>;
  return (size_t)kSpreadWarps * ((comp ? 2 : 1) * (size_t)Gm::BV + (size_t)kSpreadBatch * WRec<D>::words) * sizeof(T);
}

template <typename T, int D, int TS, bool COMP>
void launch_spread_warp(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long nunits, int skip_empty,
                        cudaStream_t s) {
  const size_t bytes = spread_smem<T, D, TS>(COMP);
  cudaFuncSetAttribute(k_spread_warp<T, D, TS, COMP>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  allow_smem(k_spread_warp<T, D, TS, COMP>, bytes);
  const unsigned grid = (unsigned)((nunits + kSpreadWarps - 1) / kSpreadWarps);
  k_spread_warp<T, D, TS, COMP><<<grid, 32 * kSpreadWarps, bytes, s>>>(J, sh, B, (T*)boxes, nunits, skip_empty);
}

template <typename T, bool COMP, bool MAC>
void launch_spread_tile3(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, int skip_empty,
                         cudaStream_t s, long long tile_begin = 0, int overlap = 0) {
  using Gm = Geo<3, 8>;
  const size_t bytes = ((size_t)3 * (COMP ? 2 : 1) * Gm::BV + (size_t)(kSpreadBatch + 1) * kRec3) * sizeof(T);
  if (J.table) {
    cudaFuncSetAttribute(k_spread_tile3<T, COMP, MAC, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    allow_smem(k_spread_tile3<T, COMP, MAC, false>, bytes);
    launch_pdl(k_spread_tile3<T, COMP, MAC, false>, dim3((unsigned)ntiles), dim3(32), bytes, s, J, sh, B, (T*)boxes,
               skip_empty, tile_begin, overlap);
  } else {
    cudaFuncSetAttribute(k_spread_tile3<T, COMP, MAC, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    allow_smem(k_spread_tile3<T, COMP, MAC, true>, bytes);
    launch_pdl(k_spread_tile3<T, COMP, MAC, true>, dim3((unsigned)ntiles), dim3(32), bytes, s, J, sh, B, (T*)boxes,
               skip_empty, tile_begin, overlap);
  }
}

template <typename T, int D, int TS, bool CP, int V>
void launch_combine(const Jobs& J, const Shape& sh, const Bins& B, const void* boxes, int acc, bool sparse,
                    cudaStream_t s, long long cell_begin = 0, long long cell_end = -1) {
  if (cell_end < 0) cell_end = B.ncell_total;
  const unsigned g = grid_for((cell_end - cell_begin + V - 1) / V, kThreads);
  if (g == 0) return;
  if (sparse)
    launch_pdl(k_spread_combine<T, D, TS, CP, V, true>, dim3(g), dim3(kThreads), 0, s, J, sh, (const T*)boxes,
               (const uint32_t*)B.tflags, cell_end, acc, B.err, cell_begin);
  else
    launch_pdl(k_spread_combine<T, D, TS, CP, V, false>, dim3(g), dim3(kThreads), 0, s, J, sh, (const T*)boxes,
               (const uint32_t*)B.tflags, cell_end, acc, B.err, cell_begin);
}

template <typename T, int D, int TS>
cudaError_t spread_impl(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, bool comp,
                        bool accumulate, bool pairs, cudaStream_t s, int overlap) {
  // A sparse call (fewer than 8 points per tile on average, e.g. a few membranes
  // in a large box) skips the boxes of empty tiles; a dense one writes every box
  // and combines without looking at tile flags.
  const bool sparse = B.tflags != nullptr && B.npts_total < 8 * ntiles;
  const int skip = sparse ? 1 : 0;
  if (ntiles > 0) {
    bool done = false;
    if constexpr (D == 3 && TS == 8) {
      if (sh.ncomp == 3) {   // three components: one warp per tile for all of them
        if (sh.mac) {
          if (comp) launch_spread_tile3<T, true, true>(J, sh, B, boxes, ntiles, skip, s, 0, overlap);
          else launch_spread_tile3<T, false, true>(J, sh, B, boxes, ntiles, skip, s, 0, overlap);
        } else {
          if (comp) launch_spread_tile3<T, true, false>(J, sh, B, boxes, ntiles, skip, s, 0, overlap);
          else launch_spread_tile3<T, false, false>(J, sh, B, boxes, ntiles, skip, s, 0, overlap);
        }
        done = true;
      }
    }
    if (!done) {
      const long long nunits = ntiles * sh.ncomp;
      if (comp) launch_spread_warp<T, D, TS, true>(J, sh, B, boxes, nunits, skip, s);
      else launch_spread_warp<T, D, TS, false>(J, sh, B, boxes, nunits, skip, s);
    }
  }
  if (B.ncell_total > 0) {
    const int acc = accumulate ? 1 : 0;
    if (pairs) {
      if (comp) launch_combine<T, D, TS, true, 2>(J, sh, B, boxes, acc, sparse, s);
      else launch_combine<T, D, TS, false, 2>(J, sh, B, boxes, acc, sparse, s);
    } else {
      if (comp) launch_combine<T, D, TS, true, 1>(J, sh, B, boxes, acc, sparse, s);
      else launch_combine<T, D, TS, false, 1>(J, sh, B, boxes, acc, sparse, s);
    }
  }
  return cudaGetLastError();
}

}  // namespace

int spread_tile_side(int dim, int elem_bytes, bool comp, int ncomp) {
  (void)elem_bytes;
  (void)comp;
  (void)ncomp;
  // One warp per tile: 12^3 boxes in 3-D, 36^2 in 2-D (two planes when
  // compensated), plus the staging records.
  return dim == 2 ? 32 : 8;
}

size_t box_bytes(int dim, int tile, int entry_bytes, int ncomp, int width) {
  const size_t side = (size_t)tile + (size_t)width;
  return (dim == 3 ? side * side * side : side * side) * (size_t)entry_bytes * ncomp;
}

cudaError_t launch_spread(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, int tile,
                          int dtype, bool comp, bool accumulate, bool even_n0, cudaStream_t s, bool overlap) {
  const bool p = even_n0;
  const int ov = overlap ? 1 : 0;
  if (dtype == 0) {
    if (sh.dim == 2) return spread_impl<float, 2, 32>(J, sh, B, boxes, ntiles, comp, accumulate, p, s, ov);
    return spread_impl<float, 3, 8>(J, sh, B, boxes, ntiles, comp, accumulate, p, s, ov);
  }
  if (sh.dim == 2) return spread_impl<double, 2, 32>(J, sh, B, boxes, ntiles, comp, accumulate, p, s, ov);
  (void)tile;
  return spread_impl<double, 3, 8>(J, sh, B, boxes, ntiles, comp, accumulate, p, s, ov);
}

template <typename T>
cudaError_t slab_boxes_impl(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long tile_begin,
                            long long ntiles, bool comp, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (sh.mac) {
    if (comp) launch_spread_tile3<T, true, true>(J, sh, B, boxes, ntiles, 0, s, tile_begin);
    else launch_spread_tile3<T, false, true>(J, sh, B, boxes, ntiles, 0, s, tile_begin);
  } else {
    if (comp) launch_spread_tile3<T, true, false>(J, sh, B, boxes, ntiles, 0, s, tile_begin);
    else launch_spread_tile3<T, false, false>(J, sh, B, boxes, ntiles, 0, s, tile_begin);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t slab_combine_impl(const Jobs& J, const Shape& sh, const Bins& B, const void* boxes, long long cell_begin,
                              long long cell_end, bool comp, bool accumulate, bool even_n0, cudaStream_t s) {
  const int acc = accumulate ? 1 : 0;
  if (even_n0) {
    if (comp) launch_combine<T, 3, 8, true, 2>(J, sh, B, boxes, acc, false, s, cell_begin, cell_end);
    else launch_combine<T, 3, 8, false, 2>(J, sh, B, boxes, acc, false, s, cell_begin, cell_end);
  } else {
    if (comp) launch_combine<T, 3, 8, true, 1>(J, sh, B, boxes, acc, false, s, cell_begin, cell_end);
    else launch_combine<T, 3, 8, false, 1>(J, sh, B, boxes, acc, false, s, cell_begin, cell_end);
  }
  return cudaGetLastError();
}

template <typename T, int D, int TS>
cudaError_t interp_impl(const Jobs& J, const Shape& sh, const Bins& B, long long ntiles, double scale,
                        cudaStream_t s) {
  using Gm = Geo<D, TS>;
  // One block per tile, plus one for the points with invalid positions.
  if (ntiles > 0 || B.npts_total > 0) {
    const size_t bytes = (size_t)sh.ncomp * Gm::BV * sizeof(T);
    if (J.table) {
      allow_smem(k_interp_tile<T, D, TS, false>, bytes);
      launch_pdl(k_interp_tile<T, D, TS, false>, dim3((unsigned)(ntiles + 1)), dim3(kInterpThreads), bytes, s, J, sh,
                 B, (T)scale);
    } else {
      allow_smem(k_interp_tile<T, D, TS, true>, bytes);
      launch_pdl(k_interp_tile<T, D, TS, true>, dim3((unsigned)(ntiles + 1)), dim3(kInterpThreads), bytes, s, J, sh,
                 B, (T)scale);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_interp(const Jobs& J, const Shape& sh, const Bins& B, long long nitiles, int dtype, double scale,
                          cudaStream_t s) {
  if (dtype == 0) {
    if (sh.dim == 2) return interp_impl<float, 2, 32>(J, sh, B, nitiles, scale, s);
    return interp_impl<float, 3, 8>(J, sh, B, nitiles, scale, s);
  }
  if (sh.dim == 2) return interp_impl<double, 2, 32>(J, sh, B, nitiles, scale, s);
  return interp_impl<double, 3, 8>(J, sh, B, nitiles, scale, s);
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
                          cudaStream_t s, bool overlap) {
  const int ov = overlap ? 1 : 0;
  const long long n = J.one.npts;
  if (n == 0) return cudaSuccess;
  const int vec = ((((uintptr_t)J.one.X) | ((uintptr_t)U) | ((uintptr_t)Xout)) % 16 == 0) ? 1 : 0;
  if (dtype == 0) {
    const unsigned grid = grid_for((n + 3) / 4, kThreads);
    if (sh.dim == 3) launch_pdl(k_advect<float, 3>, dim3(grid), dim3(kThreads), 0, s, J, (const float*)U, (float)dt,
                                (float*)Xout, vec, ov);
    else launch_pdl(k_advect<float, 2>, dim3(grid), dim3(kThreads), 0, s, J, (const float*)U, (float)dt,
                    (float*)Xout, vec, ov);
  } else {
    const unsigned grid = grid_for((n + 1) / 2, kThreads);
    if (sh.dim == 3) launch_pdl(k_advect<double, 3>, dim3(grid), dim3(kThreads), 0, s, J, (const double*)U, dt,
                                (double*)Xout, vec, ov);
    else launch_pdl(k_advect<double, 2>, dim3(grid), dim3(kThreads), 0, s, J, (const double*)U, dt, (double*)Xout,
                    vec, ov);
  }
  return cudaGetLastError();
}

cudaError_t launch_slab_boxes(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long tile_begin,
                              long long ntiles, int dtype, bool comp, cudaStream_t s) {
  if (dtype == 0) return slab_boxes_impl<float>(J, sh, B, boxes, tile_begin, ntiles, comp, s);
  return slab_boxes_impl<double>(J, sh, B, boxes, tile_begin, ntiles, comp, s);
}

cudaError_t launch_slab_combine(const Jobs& J, const Shape& sh, const Bins& B, const void* boxes, long long cell_begin,
                                long long cell_end, int dtype, bool comp, bool accumulate, bool even_n0,
                                cudaStream_t s) {
  if (dtype == 0) return slab_combine_impl<float>(J, sh, B, boxes, cell_begin, cell_end, comp, accumulate, even_n0, s);
  return slab_combine_impl<double>(J, sh, B, boxes, cell_begin, cell_end, comp, accumulate, even_n0, s);
}

}  // namespace ibgb
