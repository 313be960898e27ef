/*
 * ib_oracle.h -- FP64 reference ("oracle") for immersed-boundary spreading and
 * interpolation, arXiv 2012.06646.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
 * CPU evaluation of the sums the CUDA library computes.  Only the tests, the
 * smoke check in __graft_entry__.py and the cpu_baseline / reference leg of
 * bench.py may load it.  It shares no code, header, table or helper with the
 * CUDA library (paper_2012_06646_gb300/), and neither includes the other.
 *
 * Every function evaluates a definition from the paper directly in double
 * precision (compiled with -ffp-contract=off), looping over points in index
 * order and over shifts in colexicographic order (x fastest), which is the
 * loop structure of the serial spread (Algorithm 2) and of the per-point
 * interpolation (Algorithm 3) run on one core.
 *
 * Conventions (the readings of the paper this oracle follows):
 *   - Grid point of integer index i with staggering xi: x = h (i + xi)  (Section 3.1).
 *   - Cell of a point X for staggering xi: i = floor(X/h - xi), offset
 *     r = X/h - xi - i in [0, 1), with X/h evaluated as X * (N/L) in FP64.
 *   - Support nodes are i + t for t in {-1, 0, 1, 2} per dimension, weight
 *     prod_b phi(t_b - r_b) (Eq. delta-defs with the lower-corner cell of Fig. 1a),
 *     for the 4-point kernels.  For a kernel of support width s the nodes
 *     examined are every i + t with |t - r| < s/2 possible (the definition of
 *     delta_h: phi vanishes outside), t in [1 - s/2, s/2] for even s and
 *     [(1 - s)/2, (1 + s)/2] for odd s.
 *   - Periodic box: node indices wrap modulo N in every dimension, except the
 *     bounded dimensions (Section 3.1: # returns the empty marker outside the
 *     domain): there a node index outside 0 .. N - 1 has no grid point and
 *     takes no part, and a point must lie in [0, L] (u = X N/L in [0, N]);
 *     a point outside spreads nothing and interpolates to NaN.
 *   - MAC grid (Section 2): component a has xi_a = 0 and xi_b = 1/2 for b != a.
 *     Cell-centred grid: xi_b = 1/2 for every component.
 *   - Spreading (Eq. disc-spread):  f_a[k] = sum_j h^-d prod_b phi(.) G_{j,a}
 *     with G = F dtheta supplied by the caller (Eq. matrix-spread).
 *   - Interpolation (Eq. disc-interp): U_{j,a} = sum_k prod_b phi(.) u_a[k]
 *     (the h^d of the quadrature cancels the h^-d of delta_h).
 *   - Grid arrays are component-major [a][z][y][x], x fastest; point arrays
 *     are row-major (n, d) and (n, ncomp).
 *
 * parity pins: see tests/test_oracle_pins.py (every function here is pinned).
 */
#ifndef IB_ORACLE_H
#define IB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;       /* 2 or 3 */
  int n[3];      /* grid points per dimension (n[2] ignored when dim == 2) */
  double L[3];   /* box side per dimension */
  int grid;      /* 0 = cell-centred, 1 = MAC (requires ncomp == dim) */
  int kernel;    /* 0 = standard 4-point (Peskin 2002), 1 = cosine 4-point,
                    2 = 3-point (Roma, Peskin, Berger 1999), 3 = 6-point quintic B-spline */
  int ncomp;     /* components of the spread / interpolated field */
  int bounded;   /* bit b set: dimension b is non-periodic (nodes outside 0 .. n_b - 1 do not exist) */
} or_grid;

/* 1-D kernel phi(r) and its derivative (Section 2; kernels of Peskin 2002 and
 * the 3- and 6-point kernels above). */
double or_phi(int kernel, double r);
double or_dphi(int kernel, double r);

/* Support width s[phi] of Section 3.1: 4, 4, 3, 6 for kernels 0 .. 3. */
int or_width(int kernel);

/* Cell map of Fig. 1 / Section 3.1: u = X*scale - xi, i = floor(u), r = u - i. */
void or_cell(double X, double scale, double xi, long long* i, double* r);

/* Staggering xi of component `comp` in dimension `b`. */
double or_stagger(const or_grid* g, int comp, int b);

/* Sort key of Algorithm 4 for each point: the cell of xi = 0 (the cell
 * bounded by the grid lines of Fig. 2), key = c_x + N_x (c_y + N_y c_z). */
int or_cell_keys(const or_grid* g, long long n, const double* X, unsigned long long* key);

/* Stable key-value sort of point indices by key (Algorithm 4, sort and count
 * unique): perm[p] = index of the p-th point in key order, ties in index
 * order; start[k] = first sorted position with key >= k (start[nkeys] = n).
 * Returns the number q of distinct keys present. */
long long or_bin_stable(long long n, const unsigned long long* key, unsigned long long nkeys,
                        long long* perm, long long* start);

/* Spreading, Eq. disc-spread.  f (ncomp * ncell) is overwritten; fabs, if not
 * NULL, receives sum_j |contribution| per node (the tolerance scale). */
int or_spread(const or_grid* g, long long n, const double* X, const double* G, double* f, double* fabs_out);

/* Interpolation, Eq. disc-interp.  U (n * ncomp) is overwritten; Uabs, if not
 * NULL, receives sum_k |weight * u| per point and component. */
int or_interp(const or_grid* g, long long n, const double* X, const double* u, double* U, double* Uabs);

/* Position derivative of the interpolation sum contracted with v (NaN for a
 * point outside a bounded dimension):
 *   D_{j,b} = sum_a v_{j,a} sum_k (d/dX_b) [prod_c phi(t_c - r_c)] field_a[k],
 * (d/dX_b) r_b = N_b / L_b.  For interpolation, dLoss/dX = D(field = u, v = dLoss/dU);
 * for spreading, dLoss/dX = h^-d D(field = dLoss/df, v = G).  D is (n, dim). */
int or_pos_grad(const or_grid* g, long long n, const double* X, const double* field, const double* v,
                double* D, double* Dabs);

/* Test hook: plant a deliberate mistake (0 = none) so that tests can show the
 * pins catch it.  1: drop h^-d in spreading; 2: flip the sign of the displacement (phi(t + r));
 * 3: use the offset of the wrong dimension; 4: drop the minus sign of dr/dX. */
void or_set_mutation(int m);

#ifdef __cplusplus
}
#endif
#endif
