// ib_width.cu -- spreading and interpolation for kernels whose support width
// s (Section 3.1) is not 4: the 3-point kernel of Roma, Peskin and Berger
// (s = 3) and the 6-point quintic B-spline (s = 6).  The methods of the paper
// do not depend on phi (Section 2); only the cell map and the box sizes do.
//
// Cell map for width s (Section 3.1, Fig. 1): the cell of a point is the
// region of points with the same s^d support nodes.  With u = X N/L - xi it is
// bounded by grid nodes for even s (node index i = floor(u), offset
// rho = u - i in [0, 1)) and centred on the nearest node for odd s
// (i = floor(u + 1/2), rho = u - i in [-1/2, 1/2)).  The support nodes are
// i + t for t in [tlo, tlo + s) with tlo = 1 - s/2 (even) or (1 - s)/2 (odd),
// weight phi(t - rho) per dimension.  For odd s, u + 1/2 = X N/L - (xi - 1/2)
// is the even map with the staggerings 0 and 1/2 exchanged (cell one higher
// for xi = 0), so the exact two-product offsets of the 4-point path serve
// both: the fraction of u + 1/2 is r and 1 - r of the other staggering.
//
// The points are binned exactly as for the 4-point kernels (by the xi = 0
// cell), and a tile of cells T0 .. T0 + TS - 1 owns a box of side TS + s
// starting at node T0 + lo, lo = tlo - 1 (even s) or tlo (odd s): the nodes
// its points can reach in any staggering.  One warp per (tile, component)
// adds its points' s^d contributions in a fixed order (the order of the
// bins), a second kernel sums the boxes covering each node in a fixed order,
// so results are bit-reproducible as on the 4-point path.  Interpolation
// stages a tile's box of grid values in shared memory and gives each point
// one thread.
#include <math.h>

#include "ib_internal.h"

namespace ibgb {
namespace {

constexpr int kWWarps = 2;     // (tile, component) units per CTA, one warp each
constexpr int kWBatch = 32;    // points per staging batch
constexpr int kWCover = 8;     // covering boxes per node and dimension (at most 1 + ceil(s / n) <= 7)
constexpr int kWInterpThreads = 128;
constexpr int kThreads = 256;

template <int D, int S, int TS>
struct WGeo {
  static constexpr bool odd = (S & 1) != 0;
  static constexpr int tlo = odd ? -(S - 1) / 2 : 1 - S / 2;
  static constexpr int lo = odd ? tlo : tlo - 1;            // box origin relative to the tile's first cell
  static constexpr int BS = TS + S;                         // box side
  static constexpr int BV = (D == 3) ? BS * BS * BS : BS * BS;
  static constexpr int NODES = (D == 3) ? S * S * S : S * S;
  static constexpr int PER = (NODES + 31) / 32;             // support nodes per lane
  static constexpr int REC = S * S + ((D == 3) ? S : 0);    // wx wy h^-d G products, then wz
  static constexpr int NROWS = (D == 3) ? TS * TS : TS;     // cell rows (x runs) of a full tile
};

inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Rounds of k_spread_w's read-modify-writes: lane L takes the support nodes
// whose box offset is L mod 32, so the lanes of a round hit distinct banks
// whatever the box corner; the rounds needed are the largest number of
// support nodes sharing one residue.
template <int D, int S, int BS>
__host__ __device__ constexpr int residue_rounds() {
  int cnt[32] = {};
  int m = 0;
  for (int q = 0; q < ((D == 3) ? S * S * S : S * S); ++q) {
    const int tx = q % S, ty = (q / S) % S, tz = q / (S * S);
    const int o = tx + BS * (ty + BS * tz);
    ++cnt[o & 31];
    if (cnt[o & 31] > m) m = cnt[o & 31];
  }
  return m;
}

template <int D, int TS>
__device__ __forceinline__ void wtile_coords(const int* ntile, const int* n, long long lt, int T0[3], int TE[3]) {
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

__device__ __forceinline__ int wfloor_div(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// Weights w[k] = phi(tlo + k - rho) from the fraction r (of u for even s, of
// u + 1/2 for odd s) and c = 1 - r, each without cancellation:
//   3-point (rho = r - 1/2, q = sqrt(1 - 3 rho^2) = sqrt(1/4 + 3 r c)):
//     2 c^2 / (1/2 + 3c + q),  (1 + q) / 3,  2 r^2 / (1/2 + 3r + q);
//   6-point B-spline (rho = r): c^5/120, m(c), p(r), p(c), m(r), r^5/120 with
//     p(x) = (66 - 60 x^2 + 30 x^4 - 10 x^5) / 120 (the piece on [0, 1)) and
//     m(x) = (1 + 5x + 10x^2 + 10x^3 + 5x^4 - 5x^5) / 120 (the piece on [1, 2)
//     in the distance x = 2 - |arg| to its far end).
template <typename T, int S>
__device__ __forceinline__ void wweights(T r, T c, T w[S]) {
  if constexpr (S == 3) {
    const T q = sqrt(fma((T)3 * r, c, (T)0.25));
    w[0] = (T)2 * c * c / ((T)0.5 + (T)3 * c + q);
    w[1] = ((T)1 + q) * (T)(1.0 / 3.0);
    w[2] = (T)2 * r * r / ((T)0.5 + (T)3 * r + q);
  } else {
    constexpr T k = (T)(1.0 / 120.0);
    const T r2 = r * r, c2 = c * c;
    w[0] = c2 * c2 * c * k;
    w[1] = ((T)1 + c * ((T)5 + c * ((T)10 + c * ((T)10 + c * ((T)5 - (T)5 * c))))) * k;
    w[2] = ((T)66 + r2 * ((T)-60 + r2 * ((T)30 - (T)10 * r))) * k;
    w[3] = ((T)66 + c2 * ((T)-60 + c2 * ((T)30 - (T)10 * c))) * k;
    w[4] = ((T)1 + r * ((T)5 + r * ((T)10 + r * ((T)10 + r * ((T)5 - (T)5 * r))))) * k;
    w[5] = r2 * r2 * r * k;
  }
}

// Weights and their derivatives with respect to the fraction r (dw[k] =
// d w[k] / dr; c = 1 - r), from the same pieces as wweights:
//   3-point: with e = (c - r) / (2q), dw = (-(1 + e) / 2, e, (1 - e) / 2);
//   6-point: -c^4/24, -m'(c), p'(r), -p'(c), m'(r), r^4/24 with
//     p'(x) = x (-120 + x^2 (120 - 50 x)) / 120,
//     m'(x) = (5 + x (20 + x (30 + x (20 - 25 x)))) / 120.
template <typename T>
__device__ __forceinline__ T bspline_pd(T x) {
  return x * ((T)-120 + x * x * ((T)120 - (T)50 * x)) * (T)(1.0 / 120.0);
}
template <typename T>
__device__ __forceinline__ T bspline_md(T x) {
  return ((T)5 + x * ((T)20 + x * ((T)30 + x * ((T)20 - (T)25 * x)))) * (T)(1.0 / 120.0);
}

template <typename T, int S>
__device__ __forceinline__ void wweights_d(T r, T c, T w[S], T dw[S]) {
  wweights<T, S>(r, c, w);
  if constexpr (S == 3) {
    const T q = sqrt(fma((T)3 * r, c, (T)0.25));
    const T e = (c - r) / ((T)2 * q);
    dw[0] = -((T)1 + e) * (T)0.5;
    dw[1] = e;
    dw[2] = ((T)1 - e) * (T)0.5;
  } else {
    dw[0] = -c * c * c * c * (T)(1.0 / 24.0);
    dw[1] = -bspline_md(c);
    dw[2] = bspline_pd(r);
    dw[3] = -bspline_pd(c);
    dw[4] = bspline_md(r);
    dw[5] = r * r * r * r * (T)(1.0 / 24.0);
  }
}

// Cell of a point in one dimension, relative to the tile: the physical xi = 0
// cell minus the tile origin, and the exact offsets of both staggerings.
// Returns false when that cell is not in the tile (X changed after binning).
template <typename T>
__device__ __forceinline__ bool wcell_dim(const Job& jb, T x, int b, const int T0[3], const int TE[3], Cell1<T>& cl,
                                          int& cc) {
  const uint32_t e = point_cell<T>(x, jb, b, cl);
  const int n = jb.n[b];
  const int cphys = ((unsigned)cl.i0 < (unsigned)n) ? cl.i0 : modn(cl.i0, n);
  cc = cphys - T0[b];
  return e == 0 && (unsigned)cc < (unsigned)TE[b] && (cl.i1 - cl.i0) >= -1 && (cl.i1 - cl.i0) <= 0;
}

// Box offset of the first support node and the s weights of one dimension,
// for the staggering h (xi = 1/2) or not (xi = 0).
template <typename T, int D, int S, int TS>
__device__ __forceinline__ void wselect(const Cell1<T>& cl, int cc, bool h, int& o, T w[S]) {
  using W = WGeo<D, S, TS>;
  int di;
  T r, c;
  if (W::odd == h) {          // even s with xi = 0, or odd s with xi = 1/2: floor(X N/L)
    di = 0;
    r = cl.r0;
    c = cl.c0;
  } else if (!W::odd) {       // even s, xi = 1/2: floor(X N/L - 1/2)
    di = cl.i1 - cl.i0;
    r = cl.r1;
    c = cl.c1;
  } else {                    // odd s, xi = 0: floor(X N/L + 1/2) = floor(X N/L - 1/2) + 1
    di = cl.i1 + 1 - cl.i0;
    r = cl.r1;
    c = cl.c1;
  }
  o = cc + di + (W::tlo - W::lo);
  wweights<T, S>(r, c, w);
}

// One dimension of a point for component a (wcell_dim, then wselect).
template <typename T, int D, int S, int TS>
__device__ __forceinline__ bool wpoint_dim(const Job& jb, const Shape& sh, T x, int b, int a, const int T0[3],
                                           const int TE[3], int& o, T w[S]) {
  Cell1<T> cl;
  int cc;
  const bool inside = wcell_dim<T>(jb, x, b, T0, TE, cl, cc);
  wselect<T, D, S, TS>(cl, cc, half_stag(sh, a, b), o, w);
  return inside;
}

// ---------------------------------------------------------------------------
// Spreading into tile boxes: one warp per (tile, component), the two stages
// of the 4-point path.  Stage 1 (lanes = points): a point's record holds the
// s^2 products wx[tx] wy[ty] h^-d G and the s weights wz, plus its box offset.
// Stage 2 (warp = point): lane l owns the support nodes whose box offset is
// l mod 32 (distinct nodes, so plain read-modify-writes are race-free, and the
// lanes of each round hit distinct banks); the lane's loads come before its
// stores, and __syncwarp orders consecutive points.
// ---------------------------------------------------------------------------
template <typename T, int D, int S, int TS>
__global__ void __launch_bounds__(32 * kWWarps) k_spread_w(const __grid_constant__ Jobs J, const Shape sh,
                                                            const Bins B, T* __restrict__ boxes, long long nunits) {
  using W = WGeo<D, S, TS>;
  static_assert(W::NROWS % 32 == 0, "rows: a multiple of 32");
  constexpr int R = residue_rounds<D, S, W::BS>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t rstart_s[kWWarps][W::NROWS];
  __shared__ uint32_t rpre_s[kWWarps][W::NROWS];
  __shared__ int roff_s[kWWarps][kWBatch];
  __shared__ uint32_t ltab_s[kWWarps][R][32];      // per round and lane: box offset | xy product << 16 | z << 24
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long unit = (long long)blockIdx.x * kWWarps + warp;
  if (unit >= nunits) return;                      // the whole warp leaves; no block barrier follows
  T* box = reinterpret_cast<T*>(smem_raw) + warp * (W::BV + kWBatch * W::REC);
  T* rec_s = box + W::BV;
  uint32_t* rstart = rstart_s[warp];
  uint32_t* rpre = rpre_s[warp];
  int* roff = roff_s[warp];
  const Job& jb = J.one;
  const int nc = sh.ncomp;
  const long long gt = unit / nc;
  const int a = (int)(unit - gt * nc);
  int T0[3], TE[3];
  wtile_coords<D, TS>(jb.ntile, jb.n, gt, T0, TE);
  for (int i = lane; i < W::BV; i += 32) box[i] = (T)0;

  const int rows = (D == 3) ? TE[1] * TE[2] : TE[1];
  uint32_t M = 0;
#pragma unroll
  for (int k = 0; k < W::NROWS / 32; ++k) {
    const int r = lane + 32 * k;
    uint32_t st = 0, cnt = 0;
    if (r < rows) {
      const int y = T0[1] + ((D == 3) ? r % TE[1] : r);
      const int z = (D == 3) ? T0[2] + r / TE[1] : 0;
      const long long cell = T0[0] + (long long)jb.n[0] * (y + (long long)jb.n[1] * z);
      if (IB_IN(B.err, cell + TE[0], B.ncell_total + 1)) {
        st = B.count[cell];
        cnt = B.count[cell + TE[0]] - st;
      }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    rstart[r] = st;
    rpre[r] = M + inc - cnt;
    M += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();

  const T* Xg = (const T*)jb.X;
  const T* Gp = (const T*)jb.G;
  const T hmd = (T)jb.hmd;
  auto load_point = [&](uint32_t q, T xs[D], T& gs) {
    int lo = 0;
#pragma unroll
    for (int step = W::NROWS / 2; step >= 1; step >>= 1)
      if (lo + step < rows && rpre[lo + step] <= q) lo += step;
    const long long pi = (long long)rstart[lo] + (q - rpre[lo]);
    long long li = IB_IN(B.err, pi, B.npts_total) ? (long long)B.perm[pi] : 0;
    if (!IB_IN(B.err, li, jb.npts)) li = 0;
#pragma unroll
    for (int b = 0; b < D; ++b) xs[b] = Xg[li * D + b];
    gs = Gp[li * nc + a];
  };

  // This lane's support nodes: those whose box offset is lane mod 32.
  {
    uint32_t(*ltab)[32] = ltab_s[warp];
    int cnt = 0;
    for (int q = 0; q < W::NODES; ++q) {
      const int tx = q % S, ty = (q / S) % S, tz = (D == 3) ? q / (S * S) : 0;
      const int o = tx + W::BS * (ty + W::BS * tz);
      if ((o & 31) == lane) {
        ltab[cnt][lane] = (uint32_t)o | ((uint32_t)(tx + S * ty) << 16) | ((uint32_t)(S * S + tz) << 24);
        ++cnt;
      }
    }
    for (int k = cnt; k < R; ++k) ltab[k][lane] = 0xFFFFFFFFu;
    __syncwarp();
  }
  int loff[R], lxy[R], lz[R];
  bool lon[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const uint32_t e = ltab_s[warp][k][lane];
    lon[k] = e != 0xFFFFFFFFu;
    loff[k] = (int)(e & 0xFFFFu);
    lxy[k] = (int)((e >> 16) & 0xFFu);
    lz[k] = (int)(e >> 24);
  }

  T xs[D], gs = (T)0;
  if (lane < M) load_point(lane, xs, gs);
  for (uint32_t base = 0; base < M; base += kWBatch) {
    if (base + lane < M) {
      int o[3] = {0, 0, 0};
      T w[3][S];
      bool inside = true;
#pragma unroll
      for (int b = 0; b < D; ++b) inside = wpoint_dim<T, D, S, TS>(jb, sh, xs[b], b, a, T0, TE, o[b], w[b]) && inside;
#pragma unroll
      for (int b = 0; b < D; ++b) inside = inside && IB_IN(B.err, o[b], W::BS - S + 1);
      T ga = hmd * gs;
      if (!inside) {                 // X changed after binning: contribute nothing, report
        atomicOr(B.err, ERR_STALE);
        ga = (T)0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          o[b] = 0;
#pragma unroll
          for (int t = 0; t < S; ++t) w[b][t] = (T)0;
        }
      }
      T* rec = rec_s + lane * W::REC;
#pragma unroll
      for (int ty = 0; ty < S; ++ty)
#pragma unroll
        for (int tx = 0; tx < S; ++tx) rec[tx + S * ty] = (w[0][tx] * ga) * w[1][ty];
      if (D == 3) {
#pragma unroll
        for (int tz = 0; tz < S; ++tz) rec[S * S + tz] = w[D - 1][tz];
      }
      roff[lane] = o[0] + W::BS * (o[1] + W::BS * o[2]);
    }
    const uint32_t nq = base + kWBatch + lane;     // next batch's point data, fetched during the additions
    if (nq < M) load_point(nq, xs, gs);
    __syncwarp();
    const int cnt = (int)min((uint32_t)kWBatch, M - base);
    for (int i = 0; i < cnt; ++i) {
      const T* rp = rec_s + i * W::REC;
      const int off = roff[i];
      T v[R], add[R];
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (lon[k]) {
          add[k] = (D == 3) ? rp[lxy[k]] * rp[lz[k]] : rp[lxy[k]];
          v[k] = box[off + loff[k]];
        }
      }
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (lon[k]) box[off + loff[k]] = v[k] + add[k];
      __syncwarp();
    }
  }
  __syncwarp();
  T* dst = boxes + unit * (long long)W::BV;        // scratch [tile][comp][BV]
  for (int i = lane; i < W::BV; i += 32) dst[i] = box[i];
}

// ---------------------------------------------------------------------------
// Three-component fields in 3-D (the MAC velocity grid, or three cell-centred
// components): one warp per tile owns the three component boxes, so a point's
// cell map is computed once and each lane's read-modify-writes of the three
// components are independent (loads first).  Record of a point per component:
// the s^2 products wx wy h^-d G_a, then the s weights wz; box offsets apart.
// The boxes are written in the [tile][component][BV] layout of k_spread_w.
// ---------------------------------------------------------------------------
template <typename T, int S>
__global__ void __launch_bounds__(32) k_spread_w3(const __grid_constant__ Jobs J, const Shape sh, const Bins B,
                                                  T* __restrict__ boxes) {
  constexpr int TS = 8;
  using W = WGeo<3, S, TS>;
  constexpr int RC = S * S + S;                    // record words per component
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t rstart[W::NROWS];
  __shared__ uint32_t rpre[W::NROWS];
  __shared__ int roff[kWBatch][3];
  const int lane = threadIdx.x;
  T* box = reinterpret_cast<T*>(smem_raw);         // [3][BV]
  T* rec_s = box + 3 * W::BV;                      // [kWBatch][3 RC]
  const Job& jb = J.one;
  const long long gt = blockIdx.x;
  int T0[3], TE[3];
  wtile_coords<3, TS>(jb.ntile, jb.n, gt, T0, TE);
  for (int i = lane; i < 3 * W::BV; i += 32) box[i] = (T)0;
  const int rows = TE[1] * TE[2];
  uint32_t M = 0;
#pragma unroll
  for (int k = 0; k < W::NROWS / 32; ++k) {
    const int r = lane + 32 * k;
    uint32_t st = 0, cnt = 0;
    if (r < rows) {
      const int y = T0[1] + r % TE[1];
      const int z = T0[2] + r / TE[1];
      const long long cell = T0[0] + (long long)jb.n[0] * (y + (long long)jb.n[1] * z);
      if (IB_IN(B.err, cell + TE[0], B.ncell_total + 1)) {
        st = B.count[cell];
        cnt = B.count[cell + TE[0]] - st;
      }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    rstart[r] = st;
    rpre[r] = M + inc - cnt;
    M += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  const T* Xg = (const T*)jb.X;
  const T* Gp = (const T*)jb.G;
  const T hmd = (T)jb.hmd;
  auto load_point = [&](uint32_t q, T xs[3], T gs[3]) {
    int lo = 0;
#pragma unroll
    for (int step = W::NROWS / 2; step >= 1; step >>= 1)
      if (lo + step < rows && rpre[lo + step] <= q) lo += step;
    const long long pi = (long long)rstart[lo] + (q - rpre[lo]);
    long long li = IB_IN(B.err, pi, B.npts_total) ? (long long)B.perm[pi] : 0;
    if (!IB_IN(B.err, li, jb.npts)) li = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) xs[b] = Xg[li * 3 + b];
#pragma unroll
    for (int b = 0; b < 3; ++b) gs[b] = Gp[li * 3 + b];
  };
  int loff[W::PER], lxy[W::PER], lz[W::PER];
  bool lon[W::PER];
#pragma unroll
  for (int k = 0; k < W::PER; ++k) {
    const int q = lane + 32 * k;
    lon[k] = q < W::NODES;
    const int tx = q % S, ty = (q / S) % S, tz = q / (S * S);
    loff[k] = tx + W::BS * (ty + W::BS * tz);
    lxy[k] = tx + S * ty;
    lz[k] = S * S + tz;
  }
  T xs[3], gs[3] = {(T)0, (T)0, (T)0};
  if (lane < M) load_point(lane, xs, gs);
  for (uint32_t base = 0; base < M; base += kWBatch) {
    if (base + lane < M) {
      Cell1<T> cl[3];
      int cc[3];
      bool inside = true;
#pragma unroll
      for (int b = 0; b < 3; ++b) inside = wcell_dim<T>(jb, xs[b], b, T0, TE, cl[b], cc[b]) && inside;
      if (!inside) atomicOr(B.err, ERR_STALE);     // X changed after binning: contribute nothing, report
      T* rec = rec_s + lane * 3 * RC;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int o[3];
        T w[3][S];
#pragma unroll
        for (int b = 0; b < 3; ++b) wselect<T, 3, S, TS>(cl[b], cc[b], half_stag(sh, a, b), o[b], w[b]);
        bool in_a = inside;
#pragma unroll
        for (int b = 0; b < 3; ++b) in_a = in_a && IB_IN(B.err, o[b], W::BS - S + 1);
        if (!in_a) o[0] = o[1] = o[2] = 0;
        const T ga = in_a ? hmd * gs[a] : (T)0;
        T* ra = rec + a * RC;
#pragma unroll
        for (int ty = 0; ty < S; ++ty)
#pragma unroll
          for (int tx = 0; tx < S; ++tx) ra[tx + S * ty] = inside ? (w[0][tx] * ga) * w[1][ty] : (T)0;
#pragma unroll
        for (int tz = 0; tz < S; ++tz) ra[S * S + tz] = inside ? w[2][tz] : (T)0;
        roff[lane][a] = inside ? o[0] + W::BS * (o[1] + W::BS * o[2]) : 0;
      }
    }
    const uint32_t nq = base + kWBatch + lane;     // next batch's point data, fetched during the additions
    if (nq < M) load_point(nq, xs, gs);
    __syncwarp();
    const int cnt = (int)min((uint32_t)kWBatch, M - base);
    for (int i = 0; i < cnt; ++i) {
      const T* rp = rec_s + i * 3 * RC;
      T v[3][W::PER], add[3][W::PER];
      int idx[3][W::PER];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int off = roff[i][a] + a * W::BV;
#pragma unroll
        for (int k = 0; k < W::PER; ++k) {
          if (lon[k]) {
            idx[a][k] = off + loff[k];
            add[a][k] = rp[a * RC + lxy[k]] * rp[a * RC + lz[k]];
            v[a][k] = box[idx[a][k]];
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < W::PER; ++k)
          if (lon[k]) box[idx[a][k]] = v[a][k] + add[a][k];
      __syncwarp();
    }
  }
  __syncwarp();
  T* dst = boxes + gt * (long long)(3 * W::BV);    // [tile][comp][BV]: the three boxes, contiguous
  for (int i = lane; i < 3 * W::BV; i += 32) dst[i] = box[i];
}

// Boxes covering node x of a dimension with n nodes and ntile tiles: every
// unwrapped copy v = x + k n inside some tile's used box range (offsets
// 0 .. TE + s - 1 from the box origin), in increasing v, then tile.
template <int S, int TS>
__device__ __forceinline__ int wcover(int x, int n, int ntile, int* tl, int* of) {
  using W = WGeo<3, S, TS>;
  int cnt = 0;
  int v = x;
  while (v - n >= W::lo) v -= n;
  const int last = (ntile - 1) * TS;
  const int vend = last + W::lo + (n - last) + S;
  for (; v < vend; v += n) {
    const int t0 = max(0, wfloor_div(v - W::lo - W::BS + 1, TS));
    const int t1 = min(ntile - 1, wfloor_div(v - W::lo, TS));
    for (int t = t0; t <= t1; ++t) {
      const int o = v - t * TS - W::lo;
      const int te = min(TS, n - t * TS);
      if (o >= 0 && o < te + S && cnt < kWCover) {
        tl[cnt] = t;
        of[cnt] = o;
        ++cnt;
      }
    }
  }
  return cnt;
}

// Fast cover list for n >= TS + s (a box never wraps onto its own tile): in
// increasing unwrapped position, then tile -- the periodic copy x - n in tile
// 0, the previous tile, the node's own tile, the next tile, and the copy
// x + n in the last two tiles -- at most 3 at once, the same entries in the
// same order as wcover.
struct WCover3 {        // three scalar slots (no dynamically indexed array: the list stays in registers)
  int t0, o0, t1, o1, t2, o2, n;
  __device__ __forceinline__ void push(int tt, int oo) {
    if (n == 0) { t0 = tt; o0 = oo; } else if (n == 1) { t1 = tt; o1 = oo; } else { t2 = tt; o2 = oo; }
    ++n;
  }
  __device__ __forceinline__ int t(int i) const { return i == 0 ? t0 : (i == 1 ? t1 : t2); }
  __device__ __forceinline__ int o(int i) const { return i == 0 ? o0 : (i == 1 ? o1 : o2); }
};

template <int S, int TS>
__device__ __forceinline__ WCover3 wcover_fast(int x, int n, int ntile) {
  using W = WGeo<3, S, TS>;
  WCover3 c;
  c.n = 0;
  c.t0 = c.o0 = c.t1 = c.o1 = c.t2 = c.o2 = 0;
  const int t = x / TS, xl = x - t * TS;
  const int last = ntile - 1, te_last = n - last * TS;
  if (x - n >= W::lo) c.push(0, x - n - W::lo);                       // copy x - n in tile 0
  if (t >= 1 && xl + TS - W::lo < TS + S) c.push(t - 1, xl + TS - W::lo);
  c.push(t, xl - W::lo);
  if (t + 1 <= last && xl - TS - W::lo >= 0) {
    const int te = min(TS, n - (t + 1) * TS);
    if (xl - TS - W::lo < te + S) c.push(t + 1, xl - TS - W::lo);
  }
  // copy x + n: the last tile, and the one before it when the last tile is short
  if (ntile >= 2) {
    const int o2 = x + n - (last - 1) * TS - W::lo;
    if (o2 < TS + S) c.push(last - 1, o2);
  }
  const int o1 = x + n - last * TS - W::lo;
  if (o1 < te_last + S) c.push(last, o1);
  return c;
}

template <typename T, int D, int S, int TS>
__global__ void __launch_bounds__(kThreads) k_combine_w(const __grid_constant__ Jobs J, const Shape sh,
                                                         const T* __restrict__ boxes, int accumulate, uint32_t* err) {
  using W = WGeo<D, S, TS>;
  const Job& jb = J.one;
  const long long lc = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (lc >= jb.ncell) return;
  int x[3];
  x[0] = (int)(lc % jb.n[0]);
  const long long q = lc / jb.n[0];
  x[1] = (int)(q % jb.n[1]);
  x[2] = (D == 3) ? (int)(q / jb.n[1]) : 0;
  const int nc = sh.ncomp;
  T* f = (T*)jb.f;
  bool fast = nc <= 4;
#pragma unroll
  for (int b = 0; b < D; ++b) fast = fast && jb.n[b] >= TS + S;
  if (fast) {
    const WCover3 cx = wcover_fast<S, TS>(x[0], jb.n[0], jb.ntile[0]);
    const WCover3 cy = wcover_fast<S, TS>(x[1], jb.n[1], jb.ntile[1]);
    WCover3 cz;
    if (D == 3) {
      cz = wcover_fast<S, TS>(x[2], jb.n[2], jb.ntile[2]);
    } else {
      cz.n = 1;
      cz.t0 = cz.o0 = cz.t1 = cz.o1 = cz.t2 = cz.o2 = 0;
    }
#ifdef IB_DEBUG_BOUNDS
    {
      const WCover3* cv[3] = {&cx, &cy, &cz};
      for (int b = 0; b < D; ++b) {
        if (!IB_IN(err, cv[b]->n, 4)) return;
        for (int i = 0; i < cv[b]->n; ++i)
          if (!(IB_IN(err, cv[b]->t(i), jb.ntile[b]) && IB_IN(err, cv[b]->o(i), W::BS))) return;
      }
    }
#endif
    // up to 27 boxes, all entries loaded before the sums (in the fixed order)
    T S4[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
    for (int iz = 0; iz < 3; ++iz) {
      if (iz >= cz.n) break;
#pragma unroll
      for (int iy = 0; iy < 3; ++iy) {
        if (iy >= cy.n) break;
        const long long trow = cy.t(iy) + (long long)jb.ntile[1] * cz.t(iz);
        const int orow = (cz.o(iz) * W::BS + cy.o(iy)) * W::BS;
        T v[3][4];
#pragma unroll
        for (int ix = 0; ix < 3; ++ix) {
          const long long tile = cx.t(ix) + (long long)jb.ntile[0] * trow;
          const T* bp = boxes + tile * nc * W::BV + orow + cx.o(ix);
#pragma unroll
          for (int a = 0; a < 4; ++a) v[ix][a] = (ix < cx.n && a < nc) ? bp[a * W::BV] : (T)0;
        }
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int a = 0; a < 4; ++a)
            if (ix < cx.n) S4[a] += v[ix][a];
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (a >= nc) break;
      const long long o = a * jb.ncell + lc;
      f[o] = accumulate ? f[o] + S4[a] : S4[a];
    }
    return;
  }
  int tl[3][kWCover], of[3][kWCover], nco[3];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    nco[b] = wcover<S, TS>(x[b], jb.n[b], jb.ntile[b], tl[b], of[b]);
    for (int i = 0; i < nco[b]; ++i)
      if (!(IB_IN(err, tl[b][i], jb.ntile[b]) && IB_IN(err, of[b][i], W::BS))) return;
  }
  if (D == 2) {
    nco[2] = 1;
    tl[2][0] = 0;
    of[2][0] = 0;
  }
  for (int a = 0; a < nc; ++a) {
    T s = 0;
    for (int iz = 0; iz < nco[2]; ++iz)
      for (int iy = 0; iy < nco[1]; ++iy) {
        const long long trow = tl[1][iy] + (long long)jb.ntile[1] * tl[2][iz];
        const int orow = (of[2][iz] * W::BS + of[1][iy]) * W::BS;
        for (int ix = 0; ix < nco[0]; ++ix) {
          const long long tile = tl[0][ix] + (long long)jb.ntile[0] * trow;
          s += boxes[(tile * nc + a) * W::BV + orow + of[0][ix]];
        }
      }
    const long long o = a * jb.ncell + lc;
    f[o] = accumulate ? f[o] + s : s;
  }
}

// ---------------------------------------------------------------------------
// Interpolation: one CTA per tile (plus a last block for the points with
// invalid positions, which get NaN); the tile's box of grid values (all
// components) is staged in shared memory, then each thread takes points of
// the tile (cell order) and sums their s^d support per component.
// ---------------------------------------------------------------------------
template <typename T, int D, int S, int TS>
__global__ void __launch_bounds__(kWInterpThreads, sizeof(T) == 4 ? 6 : 4) k_interp_w(const __grid_constant__ Jobs J, const Shape sh,
                                                                  const Bins B, const T scale) {
  using W = WGeo<D, S, TS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* box = reinterpret_cast<T*>(smem_raw);
  __shared__ uint32_t rstart[W::NROWS];
  __shared__ uint32_t rpre[W::NROWS + 1];
  const Job& jb = J.one;
  const int nc = sh.ncomp;
  const int tid = threadIdx.x;
  if (blockIdx.x == gridDim.x - 1) {
    for (long long p = B.count[B.ncell_total] + tid; p < B.npts_total; p += kWInterpThreads) {
      T* U = (T*)jb.U + (long long)B.perm[p] * nc;
      for (int a = 0; a < nc; ++a) U[a] = (T)NAN;
    }
    return;
  }
  int T0[3], TE[3];
  wtile_coords<D, TS>(jb.itile, jb.n, blockIdx.x, T0, TE);
  const T* u = (const T*)jb.u;
  for (int i = tid; i < nc * W::BV; i += kWInterpThreads) {
    const int a = i / W::BV;
    const int rem = i - a * W::BV;
    const int bx = rem % W::BS;
    const int by = (rem / W::BS) % W::BS;
    const int bz = (D == 3) ? rem / (W::BS * W::BS) : 0;
    long long node = modn(T0[0] + W::lo + bx, jb.n[0]) +
                     (long long)jb.n[0] * modn(T0[1] + W::lo + by, jb.n[1]);
    if (D == 3) node += (long long)jb.n[0] * jb.n[1] * modn(T0[2] + W::lo + bz, jb.n[2]);
    box[i] = u[a * jb.ncell + node];
  }
  const int rows = (D == 3) ? TE[1] * TE[2] : TE[1];
  if (tid < rows) {
    const int y = T0[1] + ((D == 3) ? tid % TE[1] : tid);
    const int z = (D == 3) ? T0[2] + tid / TE[1] : 0;
    const long long cell = T0[0] + (long long)jb.n[0] * (y + (long long)jb.n[1] * z);
    rstart[tid] = B.count[cell];
    rpre[tid] = B.count[cell + TE[0]] - rstart[tid];     // count, made a prefix below
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0;
    for (int r = 0; r < rows; ++r) {
      const uint32_t c = rpre[r];
      rpre[r] = run;
      run += c;
    }
    rpre[rows] = run;
  }
  __syncthreads();
  const uint32_t P = rpre[rows];
  const T* Xg = (const T*)jb.X;
  for (uint32_t q = tid; q < P; q += kWInterpThreads) {
    int lo = 0, hi = rows - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rpre[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const long long pi = (long long)rstart[lo] + (q - rpre[lo]);
    const long long li = IB_IN(B.err, pi, B.npts_total) ? (long long)B.perm[pi] : -1;
    if (!IB_IN(B.err, li, jb.npts)) continue;
    T xs[D];
#pragma unroll
    for (int b = 0; b < D; ++b) xs[b] = Xg[li * D + b];
    T* U = (T*)jb.U + li * nc;
    Cell1<T> cl[D];
    int cc[D];
    bool inside = true;
#pragma unroll
    for (int b = 0; b < D; ++b) inside = wcell_dim<T>(jb, xs[b], b, T0, TE, cl[b], cc[b]) && inside;
    if (!inside) {
      atomicOr(B.err, ERR_STALE);        // X changed after binning: no gather outside the box
      for (int a = 0; a < nc; ++a) U[a] = (T)NAN;
      continue;
    }
    for (int a = 0; a < nc; ++a) {
      int o[3] = {0, 0, 0};
      T w[3][S];
#pragma unroll
      for (int b = 0; b < D; ++b) wselect<T, D, S, TS>(cl[b], cc[b], half_stag(sh, a, b), o[b], w[b]);
      bool in_a = true;
#pragma unroll
      for (int b = 0; b < D; ++b) in_a = in_a && IB_IN(B.err, o[b], W::BS - S + 1);
      if (!in_a) continue;
      const T* bp = box + a * W::BV + (o[2] * W::BS + o[1]) * W::BS + o[0];
      T acc = 0;
#pragma unroll
      for (int tz = 0; tz < ((D == 3) ? S : 1); ++tz) {
        T accy = 0;
#pragma unroll
        for (int ty = 0; ty < S; ++ty) {
          const T* row = bp + (tz * W::BS + ty) * W::BS;
          T accx = w[0][0] * row[0];
#pragma unroll
          for (int tx = 1; tx < S; ++tx) accx += w[0][tx] * row[tx];
          accy += w[1][ty] * accx;
        }
        acc += ((D == 3) ? w[D - 1][tz] : (T)1) * accy;
      }
      U[a] = acc * scale;
    }
  }
}

// ---------------------------------------------------------------------------
// Position gradient for width s: thread per point (cell order), the field
// gathered from global memory over the s^d support of each component:
// D_b = scale (N_b / L_b) sum_a v_a sum_nodes field_a[node] dW / dr_b.
// ---------------------------------------------------------------------------
template <typename T, int D, int S>
__global__ void __launch_bounds__(kThreads) k_pos_grad_w(const __grid_constant__ Jobs J, const Shape sh,
                                                         const Bins B, const T* __restrict__ field,
                                                         const T* __restrict__ v, T scale, T* __restrict__ Dout) {
  using W = WGeo<D, S, 8>;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= B.npts_total) return;
  const Job& jb = J.one;
  const long long li = (long long)B.perm[p];
  if (!IB_IN(B.err, li, jb.npts)) return;
  const int nc = sh.ncomp;
  const T* Xp = (const T*)jb.X + li * D;
  T* Dp = Dout + li * D;
  Cell1<T> cl[D];
  uint32_t err = 0;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    err |= point_cell<T>(Xp[b], jb, b, cl[b]);
    if (!in_bounds(jb, b, cl[b])) err |= ERR_RANGE;
  }
  if (err) {
#pragma unroll
    for (int b = 0; b < D; ++b) Dp[b] = (T)NAN;
    return;
  }
  const long long stride[3] = {1, (long long)jb.n[0], (long long)jb.n[0] * jb.n[1]};
  T out[3] = {0, 0, 0};
  for (int a = 0; a < nc; ++a) {
    long long off[3][S];
    T w[3][S], dw[3][S];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const bool h = half_stag(sh, a, b);
      int i;
      T r, c;
      if (W::odd == h) {
        i = cl[b].i0;
        r = cl[b].r0;
        c = cl[b].c0;
      } else if (!W::odd) {
        i = cl[b].i1;
        r = cl[b].r1;
        c = cl[b].c1;
      } else {
        i = cl[b].i1 + 1;
        r = cl[b].r1;
        c = cl[b].c1;
      }
      wweights_d<T, S>(r, c, w[b], dw[b]);
#pragma unroll
      for (int k = 0; k < S; ++k) off[b][k] = (long long)modn(i + W::tlo + k, jb.n[b]) * stride[b];
    }
    const T* fa = field + a * jb.ncell;
    T g[3] = {0, 0, 0};
#pragma unroll
    for (int tz = 0; tz < ((D == 3) ? S : 1); ++tz) {
      const T wz = (D == 3) ? w[D - 1][tz] : (T)1;
      const T dzv = (D == 3) ? dw[D - 1][tz] : (T)0;
      const long long oz = (D == 3) ? off[D - 1][tz] : 0;
#pragma unroll
      for (int ty = 0; ty < S; ++ty) {
        const T* row = fa + oz + off[1][ty];
        T rx = 0, rdx = 0;
#pragma unroll
        for (int tx = 0; tx < S; ++tx) {
          const T val = IB_IN(B.err, oz + off[1][ty] + off[0][tx], jb.ncell) ? __ldg(row + off[0][tx]) : (T)0;
          rx += w[0][tx] * val;
          rdx += dw[0][tx] * val;
        }
        g[0] += w[1][ty] * wz * rdx;
        g[1] += dw[1][ty] * wz * rx;
        if (D == 3) g[2] += w[1][ty] * dzv * rx;
      }
    }
    const T va = v[li * nc + a];
#pragma unroll
    for (int b = 0; b < D; ++b) out[b] += va * g[b];
  }
#pragma unroll
  for (int b = 0; b < D; ++b) Dp[b] = scale * (T)jb.scale[b] * out[b];
}

template <typename K>
void allow_smem_w(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int D, int S, int TS>
cudaError_t spread_w(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, bool accumulate,
                     cudaStream_t s) {
  using W = WGeo<D, S, TS>;
  const long long nunits = ntiles * sh.ncomp;
  if constexpr (D == 3 && TS == 8 && S == 3) {
    if (sh.ncomp == 3 && ntiles > 0) {             // three components: one warp per tile for all of them
      const size_t bytes = (size_t)(3 * W::BV + kWBatch * 3 * (S * S + S)) * sizeof(T);
      allow_smem_w(k_spread_w3<T, S>, bytes);
      k_spread_w3<T, S><<<(unsigned)ntiles, 32, bytes, s>>>(J, sh, B, (T*)boxes);
      if (J.one.ncell > 0)
        k_combine_w<T, D, S, TS><<<grid_for(J.one.ncell, kThreads), kThreads, 0, s>>>(J, sh, (const T*)boxes,
                                                                                       accumulate ? 1 : 0, B.err);
      return cudaGetLastError();
    }
  }
  if (nunits > 0) {
    const size_t bytes = (size_t)kWWarps * (W::BV + kWBatch * W::REC) * sizeof(T);
    allow_smem_w(k_spread_w<T, D, S, TS>, bytes);
    k_spread_w<T, D, S, TS><<<grid_for(nunits, kWWarps), 32 * kWWarps, bytes, s>>>(J, sh, B, (T*)boxes, nunits);
  }
  if (J.one.ncell > 0)
    k_combine_w<T, D, S, TS><<<grid_for(J.one.ncell, kThreads), kThreads, 0, s>>>(J, sh, (const T*)boxes,
                                                                                   accumulate ? 1 : 0, B.err);
  return cudaGetLastError();
}

template <typename T, int D, int S, int TS>
cudaError_t interp_w(const Jobs& J, const Shape& sh, const Bins& B, long long nitiles, double scale, cudaStream_t s) {
  using W = WGeo<D, S, TS>;
  const size_t bytes = (size_t)sh.ncomp * W::BV * sizeof(T);
  allow_smem_w(k_interp_w<T, D, S, TS>, bytes);
  k_interp_w<T, D, S, TS><<<(unsigned)(nitiles + 1), kWInterpThreads, bytes, s>>>(J, sh, B, (T)scale);
  return cudaGetLastError();
}

template <typename T, int S>
cudaError_t spread_w_dim(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles, bool acc,
                         cudaStream_t s) {
  if (sh.dim == 3) return spread_w<T, 3, S, 8>(J, sh, B, boxes, ntiles, acc, s);
  return spread_w<T, 2, S, 32>(J, sh, B, boxes, ntiles, acc, s);
}

template <typename T, int S>
cudaError_t interp_w_dim(const Jobs& J, const Shape& sh, const Bins& B, long long nitiles, double scale,
                         cudaStream_t s) {
  if (sh.dim == 3) return interp_w<T, 3, S, 8>(J, sh, B, nitiles, scale, s);
  return interp_w<T, 2, S, 32>(J, sh, B, nitiles, scale, s);
}

}  // namespace

int kernel_width(int kernel) { return kernel == 2 ? 3 : (kernel == 3 ? 6 : 4); }

cudaError_t launch_spread_width(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles,
                                int dtype, bool accumulate, cudaStream_t s) {
  const int S = kernel_width(sh.kernel);
  if (dtype == 0) return S == 3 ? spread_w_dim<float, 3>(J, sh, B, boxes, ntiles, accumulate, s)
                                : spread_w_dim<float, 6>(J, sh, B, boxes, ntiles, accumulate, s);
  return S == 3 ? spread_w_dim<double, 3>(J, sh, B, boxes, ntiles, accumulate, s)
                : spread_w_dim<double, 6>(J, sh, B, boxes, ntiles, accumulate, s);
}

cudaError_t launch_pos_grad_width(const Jobs& J, const Shape& sh, const Bins& B, int dtype, const void* field,
                                  const void* v, double scale, void* D, cudaStream_t s) {
  const long long n = B.npts_total;
  if (n == 0) return cudaSuccess;
  const int S = kernel_width(sh.kernel);
  const unsigned g = grid_for(n, kThreads);
  if (dtype == 0) {
    const float *fl = (const float*)field, *vv = (const float*)v;
    float* Dd = (float*)D;
    if (sh.dim == 3 && S == 3) k_pos_grad_w<float, 3, 3><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, (float)scale, Dd);
    else if (sh.dim == 3) k_pos_grad_w<float, 3, 6><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, (float)scale, Dd);
    else if (S == 3) k_pos_grad_w<float, 2, 3><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, (float)scale, Dd);
    else k_pos_grad_w<float, 2, 6><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, (float)scale, Dd);
  } else {
    const double *fl = (const double*)field, *vv = (const double*)v;
    double* Dd = (double*)D;
    if (sh.dim == 3 && S == 3) k_pos_grad_w<double, 3, 3><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, scale, Dd);
    else if (sh.dim == 3) k_pos_grad_w<double, 3, 6><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, scale, Dd);
    else if (S == 3) k_pos_grad_w<double, 2, 3><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, scale, Dd);
    else k_pos_grad_w<double, 2, 6><<<g, kThreads, 0, s>>>(J, sh, B, fl, vv, scale, Dd);
  }
  return cudaGetLastError();
}

cudaError_t launch_interp_width(const Jobs& J, const Shape& sh, const Bins& B, long long nitiles, int dtype,
                                double scale, cudaStream_t s) {
  const int S = kernel_width(sh.kernel);
  if (dtype == 0) return S == 3 ? interp_w_dim<float, 3>(J, sh, B, nitiles, scale, s)
                                : interp_w_dim<float, 6>(J, sh, B, nitiles, scale, s);
  return S == 3 ? interp_w_dim<double, 3>(J, sh, B, nitiles, scale, s)
                : interp_w_dim<double, 6>(J, sh, B, nitiles, scale, s);
}

}  // namespace ibgb
