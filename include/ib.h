/*
 * ib.h -- C ABI of the GB300 (sm_103a) immersed-boundary coupling library.
 *
 * The library evaluates the Eulerian-Lagrangian coupling steps of the
 * immersed boundary method of arXiv 2012.06646 ("A fine-grained
 * parallelization of the immersed boundary method"):
 *
 *   spreading      f_a[k]  = sum_j delta_h(x_k - X_j) G_{j,a}          (Eq. disc-spread, Eq. matrix-spread)
 *   interpolation  U_{j,a} = sum_k delta_h(x_k - X_j) u_a[k] h^d       (Eq. disc-interp, Eq. matrix-interp)
 *
 * with delta_h(x) = prod_b h_b^-1 phi(x_b / h_b) (Section 2) on a periodic
 * box (or one with non-periodic dimensions, IB_PLAN_BOUNDED_*), G = F dtheta
 * premultiplied by the caller.  It also solves the Eulerian step of the
 * timestep on the periodic MAC grid (ib_stokes_*).  The operator statements
 * par-spread(Gamma_h, Omega_h, L) and par-interpolate(Gamma_h, Omega_h, e)
 * of Algorithms 3 and 4 map onto ib_spread and ib_interpolate: a point set,
 * a grid description (the plan) and one field per component.
 *
 * Conventions, shared with the paper's Section 3.1:
 *   - Grid point of index i and staggering xi sits at h (i + xi).  MAC grid
 *     (IB_GRID_MAC, Section 2): component a has xi_a = 0, xi_b = 1/2 (b != a).
 *     Cell-centred grid: xi = (1/2, ..., 1/2) for every component.
 *   - Cell of a point: i_b = floor(X_b * (N_b/L_b) - xi_b), evaluated so that
 *     the integer agrees exactly with the FP64 evaluation of that formula;
 *     support nodes i + t, t in {-1, 0, 1, 2}, weight prod_b phi(t_b - r_b)
 *     with r = X (N/L) - xi - i (Eq. delta-defs, Fig. 1a), for the 4-point
 *     kernels; kernels of other support widths s take the s nodes around the
 *     cell of Section 3.1 (see the kernel list below).
 *   - Node indices wrap modulo N_b (triply periodic box, Section 4), except
 *     along a bounded dimension (see IB_PLAN_BOUNDED_X).
 *   - Points may lie outside [0, L) along periodic dimensions; they are
 *     wrapped.  A position with |X_b N_b / L_b| >= 2^30, one outside [0, L_b]
 *     along a bounded dimension, or a non-finite one is reported through
 *     ib_plan_check (IB_ERR_RANGE / IB_ERR_NONFINITE); such a point spreads
 *     nothing and interpolates to NaN.
 *   - Layouts: X is row-major (npts, dim); G and U are row-major
 *     (npts, ncomp); grid fields are component-major [ncomp][n2][n1][n0]
 *     (x fastest), n2 absent in 2-D.  All arrays are contiguous.
 *   - Every data pointer passed to a compute call is a DEVICE pointer owned
 *     by the caller; the library never frees or retains it past the call.
 *     The plan owns only its scratch.  Calls are asynchronous on `stream`
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).
 *   - Argument errors are detected on the host before any launch and return
 *     an error status with nothing enqueued.  Errors found on the device
 *     (non-finite or out-of-range positions) are latched in the plan and
 *     returned by ib_plan_check.
 *   - A plan is not thread-safe: use it from one host thread and one stream
 *     at a time.
 *   - Results are run-to-run bit-reproducible: every node sum is formed in
 *     a fixed order that does not depend on scheduling.
 *   - The shared library exports exactly the functions declared here.  Each
 *     compute call (ib_bin, ib_spread, ib_interpolate, ib_pos_grad,
 *     ib_advect, ib_spread_paper, ib_batch_run, ib_batch_run_host,
 *     ib_stokes_solve) pushes an NVTX range named after itself while it
 *     enqueues its work, for profilers; it costs nothing without one.
 */
#ifndef IB_H
#define IB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IB_OK = 0,
  IB_ERR_INVALID_ARG = 1,     /* bad descriptor, null pointer, unsupported combination */
  IB_ERR_OOM = 2,             /* device or pinned host allocation failed */
  IB_ERR_CUDA = 3,            /* a CUDA runtime call failed (launch or copy) */
  IB_ERR_TIMEOUT = 4,         /* a bounded device-side wait ran out (the binning scan's look-back, see
                                 ib_selftest_bounded_wait): that call's bins are wrong; reported by
                                 ib_plan_check / ib_batch_check */
  IB_ERR_CAPACITY = 5,        /* npts (or a batch wave) exceeds the capacity given at creation */
  IB_ERR_NOT_IMPLEMENTED = 6,
  IB_ERR_NONFINITE = 7,       /* a position was NaN or infinite (reported by ib_plan_check) */
  IB_ERR_RANGE = 8,           /* a position was 2^30 or more cells away from the box, or outside
                                 [0, L] along a bounded dimension */
  IB_ERR_NO_BINS = 9,         /* IB_REUSE_BINS without a matching ib_bin call */
  IB_ERR_BINS_STALE = 10,     /* positions changed after binning (or X aliased an output):
                                 the points concerned spread nothing and interpolate to NaN */
  IB_ERR_BOUNDS = 11          /* a library built with IB_DEBUG_BOUNDS found an index outside its
                                 array and skipped the access (a library defect; never returned
                                 by the release build, whose checks compile away) */
} ib_status;

/* One-dimensional kernel phi of delta_h (Section 2; the methods do not depend
 * on phi).  Support width s (Section 3.1): 4, 4, 3, 6.
 *   IB_KERNEL_PESKIN4   standard 4-point kernel (Peskin 2002)
 *   IB_KERNEL_COSINE4   cosine 4-point kernel (Peskin 2002), the paper's choice
 *   IB_KERNEL_ROMA3     3-point kernel (Roma, Peskin, Berger 1999), odd s: the
 *                       cell of a point is centred on its nearest node (Fig. 1b)
 *   IB_KERNEL_BSPLINE6  6-point kernel: the centred quintic B-spline
 * The 3- and 6-point kernels are available to ib_bin, ib_spread (not
 * IB_COMPENSATED), ib_interpolate, ib_pos_grad and ib_advect;
 * ib_spread_paper returns IB_ERR_NOT_IMPLEMENTED for them, and batches, the
 * no-alloc interpolation and IB_PLAN_COMPENSATED plans reject them
 * (IB_ERR_INVALID_ARG). */
enum { IB_KERNEL_PESKIN4 = 0, IB_KERNEL_COSINE4 = 1, IB_KERNEL_ROMA3 = 2, IB_KERNEL_BSPLINE6 = 3 };
enum { IB_GRID_CELL_CENTERED = 0, IB_GRID_MAC = 1 };
enum { IB_F32 = 0, IB_F64 = 1 };

/* Plan creation flags (ib_plan_desc.flags). */
#define IB_PLAN_COMPENSATED 0x1u   /* size the scratch for IB_COMPENSATED spreading (twice the box scratch) */
/* Non-periodic ("bounded") dimensions (Section 3.1: the grid indexing
 * function # returns the empty marker for grid points outside the domain).
 * In a bounded dimension b every component keeps its n_b nodes
 * x = h (i + xi), i = 0 .. n_b - 1; spreading drops the contributions to
 * nodes outside that range and interpolation takes nothing from them.
 * Positions must lie in [0, L_b] (else IB_ERR_RANGE: the point spreads
 * nothing and interpolates to NaN), and ib_advect does not wrap them.  The
 * plan works on the grid extended by 8 ghost nodes per bounded dimension (the
 * de facto cells of the extended grid of Section 3.1, with the same spacing)
 * and copies the domain's nodes out of it (spreading) or into it with zero
 * ghosts (interpolation, position gradients).  ib_spread_paper returns
 * IB_ERR_NOT_IMPLEMENTED on such plans; ib_plan_bins describes the cells of
 * the extended grid. */
#define IB_PLAN_BOUNDED_X 0x2u
#define IB_PLAN_BOUNDED_Y 0x4u
#define IB_PLAN_BOUNDED_Z 0x8u   /* 3-D plans only */

/* Per-call flags. */
#define IB_ACCUMULATE   0x1u   /* spread: f += S G (the paper's l_k <- l_k + w L_i), instead of f = S G */
#define IB_COMPENSATED  0x2u   /* spread: node sums carried as TwoSum (value, error) pairs */
#define IB_REUSE_BINS   0x4u   /* skip binning: reuse the bins of the last ib_bin call (same X, same npts) */
#define IB_ADJOINT      0x8u   /* the transpose of the other operator in the plain (unweighted) inner product:
                                  ib_spread computes sum_j W_kj G_j (no h^-d), the adjoint of interpolation;
                                  ib_interpolate computes h^-d sum_k W_kj u_k, the adjoint of spreading
                                  (W_kj = prod_b phi(t_b - r_b); Eqs. matrix-interp, matrix-spread: S* = S^T) */
#define IB_SPREAD_GRAD  0x10u  /* ib_pos_grad: differentiate the weights of spreading, which carry h^-d
                                  (Eq. disc-spread): the library multiplies `scale` by h^-d = prod_b N_b/L_b */
#define IB_OVERLAP_PREVIOUS 0x20u
                               /* ib_spread (with IB_REUSE_BINS) and ib_advect: the caller guarantees that
                                  the library call issued just before this one on the same stream wrote
                                  nothing this call reads (X, G and the plan's bins for spreading, X and U
                                  for the update) -- e.g. an ib_interpolate of the same points into a
                                  separate U before a spread, an ib_spread before the update.  The call's
                                  kernel may then start while that call's last kernel finishes
                                  (programmatic dependent launch), filling its tail.  Ignored by ib_spread
                                  without IB_REUSE_BINS.  Wrong if the previous call was ib_bin or wrote
                                  what this one reads: the result is then undefined. */

typedef struct ib_plan_s* ib_plan;

typedef struct {
  int dim;                /* 2 or 3 */
  int n[3];               /* grid points per dimension, each >= 1 (n[2] ignored in 2-D) */
  double L[3];            /* box side per dimension, > 0 */
  int grid;               /* IB_GRID_MAC (requires ncomp == dim) or IB_GRID_CELL_CENTERED */
  int kernel;             /* IB_KERNEL_PESKIN4, _COSINE4, _ROMA3 or _BSPLINE6 */
  int dtype;              /* IB_F32 or IB_F64: element type of X, G, f, u, U */
  int ncomp;              /* components per field, 1..4 */
  long long max_points;   /* largest npts any call on this plan will pass, 0 <= max_points < 2^31 */
  unsigned flags;         /* IB_PLAN_COMPENSATED | IB_PLAN_BOUNDED_X | _Y | _Z, or 0 */
} ib_plan_desc;

/* Device scratch bytes ib_plan_create would allocate for `desc`.  Host-only:
 * no CUDA call.  Returns IB_ERR_INVALID_ARG for an invalid descriptor. */
ib_status ib_plan_footprint(const ib_plan_desc* desc, size_t* bytes);

/* Device memory of the scratch arenas of plans and batches.  By default each
 * ib_plan_create / ib_batch_create takes its arena from cudaMalloc and the
 * matching destroy returns it with cudaFree.  ib_set_allocator installs a
 * caller pair instead (a framework's caching allocator, or an allocator that
 * fails on purpose to exercise out-of-memory handling):
 *   - alloc(bytes, ctx): device memory of at least `bytes` bytes on the
 *     current device, 256-byte aligned, or NULL when none is available;
 *   - free_fn(ptr, ctx): releases a pointer alloc returned.
 * Every object records the pair in force when it is created and frees its
 * arena through that pair (after synchronising the device), so the pair may
 * change while objects exist; the caller keeps the functions and ctx valid
 * until those objects are destroyed.  alloc = free_fn = NULL restores
 * cudaMalloc / cudaFree; exactly one NULL is IB_ERR_INVALID_ARG.  A create
 * call whose alloc returns NULL returns IB_ERR_OOM with nothing held; an
 * arena that is not 256-byte aligned is handed back to free_fn and the create
 * call returns IB_ERR_INVALID_ARG.  The Stokes solver's buffers, cuFFT's
 * work area and a batch's pinned host staging do not go through the pair.
 * Host-only; may be called from any thread.  Paper counterpart: none. */
typedef void* (*ib_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ib_free_fn)(void* ptr, void* ctx);
ib_status ib_set_allocator(ib_alloc_fn alloc, ib_free_fn free_fn, void* ctx);

/* Validate `desc`, allocate the plan's device scratch (one arena, from
 * cudaMalloc or the ib_set_allocator pair) on the current device, and return
 * the plan in *out.  Errors: IB_ERR_INVALID_ARG (descriptor, or a misaligned
 * arena from the allocator pair), IB_ERR_OOM (allocation). */
ib_status ib_plan_create(const ib_plan_desc* desc, ib_plan* out);

/* Synchronise the device, free the plan's scratch and the plan.  NULL is a no-op. */
ib_status ib_plan_destroy(ib_plan plan);

/* Bin the npts points X by Eulerian cell: the key computation, stable key
 * sort and unique-key offsets of Algorithm 4 (Fig. 2), keyed by the cell of
 * xi = 0, key = c_x + n0 (c_y + n1 c_z).  The bins stay in the plan and are
 * reused by later calls that pass IB_REUSE_BINS with the same X. */
ib_status ib_bin(ib_plan plan, long long npts, const void* X, void* stream);

/* Spreading (Eq. disc-spread): f = S G, or f += S G with IB_ACCUMULATE.
 * X (npts, dim), G (npts, ncomp) read; f [ncomp][grid] written.  Bins X
 * first unless IB_REUSE_BINS.  Flags: IB_ACCUMULATE, IB_COMPENSATED,
 * IB_REUSE_BINS, IB_ADJOINT, IB_OVERLAP_PREVIOUS (others: IB_ERR_INVALID_ARG).
 * IB_COMPENSATED carries every node sum as a
 * TwoSum (value, error) pair and rounds once at the end; it needs a plan
 * created with IB_PLAN_COMPENSATED (else IB_ERR_INVALID_ARG).  npts = 0
 * writes zeros (or leaves f unchanged with IB_ACCUMULATE). */
ib_status ib_spread(ib_plan plan, long long npts, const void* X, const void* G, void* f,
                    unsigned flags, void* stream);

/* Interpolation (Eq. disc-interp, Algorithm 3): U = S* u.
 * X (npts, dim), u [ncomp][grid] read; U (npts, ncomp) written.  Bins X first
 * unless IB_REUSE_BINS (binning orders the per-point work by cell). */
ib_status ib_interpolate(ib_plan plan, long long npts, const void* X, const void* u, void* U,
                         unsigned flags, void* stream);

/* Position derivative of the interpolation weights, contracted with a field
 * and a per-point vector (derived from Eqs. disc-interp and disc-spread):
 *   D_{j,b} = s * sum_a v_{j,a} sum_t field_a[i+t] d/dX_b[prod_c phi(t_c - r_c)],
 * s = scale, or scale * h^-d with IB_SPREAD_GRAD.  With field = u, v = dLoss/dU,
 * scale = 1 and no flag this is dLoss/dX of interpolation; with field =
 * dLoss/df, v = G, scale = 1 and IB_SPREAD_GRAD it is dLoss/dX of spreading
 * (the library applies h^-d).  X (npts, dim), field [ncomp][grid], v (npts,
 * ncomp) read; D (npts, dim) written.  Flags: IB_REUSE_BINS, IB_SPREAD_GRAD;
 * any other bit is IB_ERR_INVALID_ARG.  Bins X first unless IB_REUSE_BINS. */
ib_status ib_pos_grad(ib_plan plan, long long npts, const void* X, const void* field, const void* v,
                      double scale, void* D, unsigned flags, void* stream);

/* Lagrangian position update of the timestep (steps b and g of Section 2):
 * Xout = X + dt U, wrapped into [0, L) per dimension.  X, U (npts, dim);
 * Xout may alias X.  Requires ncomp == dim.  Flags: IB_OVERLAP_PREVIOUS (the
 * library call just before on the stream wrote neither X nor U -- e.g. an
 * ib_spread -- so the update may run during that call's last kernel); any
 * other bit is IB_ERR_INVALID_ARG. */
ib_status ib_advect(ib_plan plan, long long npts, const void* X, const void* U, double dt, void* Xout,
                    unsigned flags, void* stream);

/* Read and clear the plan's device error word with copies ordered on
 * `stream`, waiting for that stream only (work on other streams keeps
 * running): IB_OK, IB_ERR_NONFINITE, IB_ERR_RANGE, IB_ERR_BINS_STALE or
 * IB_ERR_BOUNDS (debug build only; it takes precedence over the others) (or
 * IB_ERR_CUDA if the stream reports an error). */
ib_status ib_plan_check(ib_plan plan, void* stream);

/* The paper's own parallel spreading algorithms, kept as comparators of
 * ib_spread on the same data (f = S G, overwrite; the same result up to the
 * order of the FP sums):
 *   IB_PAPER_ALG4  Algorithm 4 ("par-spread"): per component, key each point
 *                  by the cell it inhabits in that component's staggering,
 *                  sort once, then for each of the s^d shifts in turn reduce
 *                  the values of each inhabited cell (segmented reduce) and
 *                  add them to the nodes cell + shift, one launch per shift;
 *   IB_PAPER_ALG5  Algorithm 5 ("pa-par-spread"): beta shifts per pass, the
 *                  reduced value of shift k of a pass added into buffer k of
 *                  `buffer` (caller-owned device memory of beta * n0 n1 n2
 *                  entries of the plan's dtype, overwritten), then f = sum of
 *                  the beta buffers;
 *   IB_PAPER_ALG6  Algorithm 6 ("otf-par-spread"): Algorithm 5 with the
 *                  buffer allocated and freed by the call, stream-ordered
 *                  (cudaMallocAsync / cudaFreeAsync on `stream`).
 * beta: 1 <= beta <= s^d (16 in 2-D, 64 in 3-D) for Algorithms 5 and 6,
 * ignored by Algorithm 4; `buffer` is read only by Algorithm 5.  X (npts,
 * dim), G (npts, ncomp) read; f [ncomp][grid] written.  The call re-bins X
 * once per component staggering, so a later call needs fresh bins (it cannot
 * pass IB_REUSE_BINS).  Errors: IB_ERR_INVALID_ARG (unknown algorithm, beta
 * out of range, missing buffer), IB_ERR_CAPACITY, IB_ERR_OOM (Algorithm 6
 * allocation), IB_ERR_CUDA. */
#define IB_PAPER_ALG4 4
#define IB_PAPER_ALG5 5
#define IB_PAPER_ALG6 6
ib_status ib_spread_paper(ib_plan plan, long long npts, const void* X, const void* G, void* f, int algorithm,
                          int beta, void* buffer, void* stream);

/* Device pointers to the bins of the last ib_bin on this plan (for
 * inspection and tests): perm[p] = index of the p-th point in cell order
 * (uint32, npts entries), cell_start[c] = first sorted position of cell c
 * (uint32, ncell + 2 entries; entry ncell starts the invalid points). */
ib_status ib_plan_bins(ib_plan plan, const void** perm, const void** cell_start, long long* ncell,
                       long long* npts);

/* ---------------------------------------------------------------------------
 * z-slab decomposition: a prototype of splitting one problem over GPUs (the
 * paper's Section 5 names a different kappa or # on each node as the way to
 * distribute the method).  The grid is cut along z into slabs of whole
 * 8-node tile layers; slab k owns layers [b_k, b_{k+1}) and the points whose
 * cell (xi = 0) lies in them.  Each slab's plan is a plan of the whole grid
 * that only ever works on its own layers:
 *   spreading: ib_slab_spread bins the slab's points and forms the tile
 *     boxes of its layers, then packs the box planes that reach the
 *     neighbouring slabs (the two node planes below the slab, from its bottom
 *     layer, into send_lo; the two above it, from its top layer, into
 *     send_hi).  The caller moves send_lo to the lower neighbour's recv_hi and
 *     send_hi to the upper neighbour's recv_lo (periodically: slab 0's lower
 *     neighbour is the last slab) by any device copy -- a peer copy or a
 *     collective between GPUs, a plain copy on one GPU; then ib_slab_combine
 *     places the received planes and forms f on the slab's own node planes
 *     [8 b_k, 8 b_{k+1}) only.  Every node sum runs over the same boxes in the
 *     same order as ib_spread's, so the slabs' planes together equal ib_spread's
 *     f bit for bit.
 *   interpolation: a slab needs the field on its own planes and two planes on
 *     each side (the support of its points' cells); after that halo copy (plain
 *     copies of node planes, by the caller), ib_interpolate on the slab's
 *     points gives their values, equal to ib_interpolate's on the whole point
 *     set bit for bit.
 * Requirements (else IB_ERR_INVALID_ARG): dim 3, ncomp 3, a 4-point kernel, no
 * bounded dimension, n2 a multiple of 8 and at least 16.  The plan's scratch
 * is that of the whole grid (a production split would hold its layers and one
 * neighbouring layer each side).  Paper counterpart: the distribution the
 * paper's summary proposes; not in its algorithms.
 * ------------------------------------------------------------------------- */

/* Bytes of one side's packed planes (send_lo, send_hi, recv_lo, recv_hi each):
 * n0/8 x n1/8 tiles x 3 components x (2 with IB_COMPENSATED in flags, else 1)
 * box planes x 2 z planes x 12 x 12 entries of the dtype.  Host-only. */
ib_status ib_slab_halo_bytes(ib_plan plan, unsigned flags, size_t* bytes);

/* owner[j] = the slab k with layer_bounds[k] <= (cell of X_j along z) / 8 <
 * layer_bounds[k + 1], or -1 for an invalid position (the exact cell map of
 * ib_bin).  layer_bounds: host array of nslab + 1 increasing tile layers, from
 * 0 to n2 / 8; 1 <= nslab <= 64.  X (npts, 3) device, owner (npts) int32
 * device. */
ib_status ib_slab_owner(ib_plan plan, long long npts, const void* X, int nslab, const int* layer_bounds, int* owner,
                        void* stream);

/* Bin the slab's npts points X (all of them with their cell in layers
 * [zb, ze), as ib_slab_owner assigns them; a point outside contributes
 * nothing), form the tile boxes of layers [zb, ze) with forces G, and pack
 * the planes for the neighbours into send_lo and send_hi (device buffers of
 * ib_slab_halo_bytes each, caller-owned).  Flags: IB_COMPENSATED (a plan
 * created with IB_PLAN_COMPENSATED), IB_REUSE_BINS. */
ib_status ib_slab_spread(ib_plan plan, long long npts, const void* X, const void* G, int zb, int ze, void* send_lo,
                         void* send_hi, unsigned flags, void* stream);

/* Place the planes received from the lower (recv_lo: that slab's send_hi) and
 * upper (recv_hi: its send_lo) neighbours and form f on node planes
 * [8 zb, 8 ze) of the whole-grid array f [3][n2][n1][n0] (other planes are not
 * touched).  Follows ib_slab_spread on the same plan and layers.  Flags:
 * IB_COMPENSATED (as given to ib_slab_spread), IB_ACCUMULATE. */
ib_status ib_slab_combine(ib_plan plan, void* f, int zb, int ze, const void* recv_lo, const void* recv_hi,
                          unsigned flags, void* stream);

/* ---------------------------------------------------------------------------
 * Batched, served form: one wave of independent spread + interpolate jobs of
 * uneven grid and point counts runs as a fixed number of launches, whatever
 * the number of jobs.  Jobs in a wave share dim, grid kind, kernel, dtype and
 * ncomp (the batch descriptor); each has its own grid size, box, points and
 * fields.  Paper counterpart: none (the paper runs one problem at a time);
 * each job's result equals what ib_spread / ib_interpolate give for it alone.
 * ------------------------------------------------------------------------- */

typedef struct ib_batch_s* ib_batch;

typedef struct {
  int dim, grid, kernel, dtype, ncomp;   /* as in ib_plan_desc, shared by every job */
  int max_jobs;                          /* jobs per wave */
  long long max_points;                  /* total points per wave */
  long long max_cells;                   /* total grid cells per wave (sum of n0 n1 n2), < 2^31 */
  long long max_tiles;                   /* total spreading tiles per wave (see ib_batch_job_footprint) */
  unsigned flags;                        /* 0 or IB_BATCH_HOST_IO */
} ib_batch_desc;

/* ib_batch_desc.flags: the batch also owns device buffers for every job's
 * points, forces, velocities and grid (max_points x (dim + 2 ncomp) plus
 * max_cells x ncomp entries), used by ib_batch_run_host. */
#define IB_BATCH_HOST_IO 0x1u

typedef struct {
  int n[3];              /* grid points per dimension */
  double L[3];           /* box side per dimension */
  long long npts;        /* points of this job, >= 0 */
  const void* X;         /* (npts, dim), device */
  const void* G;         /* (npts, ncomp), device; spread input (NULL: skip spreading) */
  void* f;               /* [ncomp][grid], device; spread output */
  const void* u;         /* [ncomp][grid], device; interpolation input (may equal f; NULL: skip) */
  void* U;               /* (npts, ncomp), device; interpolation output */
} ib_job;

/* Device scratch bytes ib_batch_create would allocate.  Host-only. */
ib_status ib_batch_footprint(const ib_batch_desc* desc, size_t* bytes);

/* Scratch one job occupies inside a wave, for admission by HBM footprint:
 * bytes of points, cells and spreading boxes, and its number of spreading
 * tiles (counted against max_tiles).  Host-only; either output may be NULL. */
ib_status ib_batch_job_footprint(const ib_batch_desc* desc, const ib_job* job, size_t* bytes,
                                 long long* tiles);

ib_status ib_batch_create(const ib_batch_desc* desc, ib_batch* out);
ib_status ib_batch_destroy(ib_batch batch);

/* Run one wave of njobs jobs on `stream`: bin every job's points, spread
 * G -> f for every job with G != NULL, then interpolate u -> U for every job
 * with u != NULL.  The job array is copied before the call returns.  Waits
 * (host side) for the previous wave's job-table upload on this batch object
 * before reusing its staging buffer.  A wave of one job runs the single-job
 * launches of a plan (no table upload), with the same result.
 * IB_ERR_CAPACITY if the wave exceeds the batch capacity. */
ib_status ib_batch_run(ib_batch batch, int njobs, const ib_job* jobs, unsigned flags, void* stream);

/* A served job with host-resident data (see ib_batch_run_host). */
typedef struct {
  int n[3];              /* grid points per dimension */
  double L[3];           /* box side per dimension */
  long long npts;        /* points of this job, >= 0 */
  const void* X;         /* (npts, dim), host (pinned for asynchronous copies) */
  const void* G;         /* (npts, ncomp), host: the forces to spread */
  void* U;               /* (npts, ncomp), host: receives the interpolated velocities */
} ib_host_job;

/* One served wave with host-resident inputs and outputs, in one call: on
 * `stream`, copy each job's X and G into the batch's own device buffers,
 * run the wave (bin, spread G -> f onto the job's grid, interpolate f -> U;
 * the grid stays on the device), and copy each job's U back to the host.
 * Requires a batch created with IB_BATCH_HOST_IO.  Host buffers must stay
 * valid and unchanged until the stream has passed this wave (an event or a
 * stream synchronisation); with pageable host memory the copies are not
 * asynchronous.  IB_ERR_CAPACITY as for ib_batch_run.  Paper counterpart:
 * none (serving form). */
ib_status ib_batch_run_host(ib_batch batch, int njobs, const ib_host_job* jobs, void* stream);

/* As ib_plan_check, for the batch object's device error word. */
ib_status ib_batch_check(ib_batch batch, void* stream);

/* Status of the device error word as the last ib_batch_run_host wave on this
 * batch left it: that call ends by copying the word (not clearing it) into
 * pinned host memory on its stream, so once the caller knows the stream has
 * passed the wave (an event recorded after the call has completed) this
 * decodes the copy without any CUDA call or synchronisation.  The word keeps
 * accumulating until ib_batch_check reads and clears it: a server calls
 * ib_batch_check only when this reports an error, to learn and clear that
 * wave's outcome.  IB_ERR_INVALID_ARG for a batch without IB_BATCH_HOST_IO.
 * Host-only.  Paper counterpart: none (serving form). */
ib_status ib_batch_wave_status(ib_batch batch);

/* ---------------------------------------------------------------------------
 * Interpolation for callers that cannot allocate device memory.  The paper
 * has no counterpart.  Some callers must not call cudaMalloc: code whose
 * device memory belongs to another allocator under a fixed budget (a
 * framework's pool, a process sharing the GPU under a memory cap), where a
 * new allocation can fail or fragment that budget, and latency-critical
 * loops, where cudaMalloc and cudaFree can synchronise the whole device.
 * This entry point gives the same result as ib_plan_create + ib_interpolate
 * + ib_plan_destroy for the grid `desc`, but its binning scratch is a fixed
 * device array compiled into the library (about 28 MB, held on every GPU that
 * loads the library until the process exits), so nothing is allocated or
 * freed: no cudaMalloc, cudaFree or allocating library routine runs.
 *   - desc: grid description as for ib_plan_create; max_points is ignored,
 *     and flags must be 0 (else IB_ERR_INVALID_ARG).  X (npts, dim),
 *     u [ncomp][grid] read, U (npts, ncomp) written; device pointers owned by
 *     the caller.
 *   - Limits: n0 n1 n2 (n0 n1 in 2-D) <= IB_NOALLOC_MAX_CELLS and
 *     npts <= IB_NOALLOC_MAX_POINTS, else IB_ERR_CAPACITY with nothing
 *     enqueued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call on each
 *     device before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; each call clears what must start at zero.  Calls whose work
 *     overlaps on the GPU (different streams, or host threads) race on the
 *     array: order them on one stream.
 *   - No error word is read back: non-finite or out-of-range positions
 *     interpolate to NaN, and in a library built with IB_DEBUG_BOUNDS a
 *     failed index check skips its access without being reported.
 * ------------------------------------------------------------------------- */
#define IB_NOALLOC_MAX_CELLS (1ll << 21)
#define IB_NOALLOC_MAX_POINTS (1ll << 20)
ib_status ib_interpolate_noalloc(const ib_plan_desc* desc, long long npts, const void* X, const void* u, void* U,
                                 void* stream);

/* ---------------------------------------------------------------------------
 * The Eulerian step (e) of the IB timestep (Section 2, the step list (a)-(g))
 * on the periodic MAC grid, in its Stokes limit: the convective term of the
 * Navier-Stokes momentum equation is dropped, the viscous term is taken
 * backward Euler and incompressibility is enforced by an exact discrete
 * projection (on a periodic grid the projection of the paper's fluid solver
 * is exact).  Solves, for u and a cell-centred pressure p,
 *     (rho/k) u + G p - mu L u = (rho/k) u_old + f,     D u = 0,
 * with D the face-to-cell-centre divergence (forward differences), G = -D^T
 * the cell-centre-to-face gradient and L = sum_b of the 3-point second
 * difference along b, every component on its own staggered grid (component a
 * at x - h e_a / 2 for the cell centres x, as the spreading of a MAC plan).
 * The mean of u is (rho/k) mean(u_old) + mean(f), divided by rho/k (0 when
 * rho/k = 0: the steady Stokes problem, whose mean is undetermined).  The
 * solve is cuFFT real-to-complex transforms and one kernel of per-mode
 * arithmetic.  Paper counterpart: the fluid solver the paper uses (a
 * first-order IMEX Runge-Kutta step with projection) is outside the paper's
 * parallel algorithms; this is the periodic Stokes form of it.
 * ------------------------------------------------------------------------- */
typedef struct ib_stokes_s* ib_stokes;

/* Plans the transforms for the grid `desc` (dim, n, L, dtype; grid must be
 * IB_GRID_MAC with ncomp == dim, every n_b >= 2 and n0 n1 n2 <= 2^31;
 * kernel, max_points and flags are not used)
 * and allocates the scratch: the right-hand side and the complex modes, about
 * 2 ncomp n0 n1 n2 entries of the dtype.  Errors: IB_ERR_INVALID_ARG,
 * IB_ERR_OOM, IB_ERR_CUDA (a cuFFT plan failed). */
ib_status ib_stokes_create(const ib_plan_desc* desc, ib_stokes* out);

/* Enqueues one solve on `stream`.  f, u_old (may be NULL: zero) read and u
 * written, each [ncomp][n2][n1][n0] device arrays of the dtype owned by the
 * caller; u may alias u_old but not f.  rho_over_k >= 0 (density over time
 * step), mu >= 0 (viscosity), not both 0, finite, else IB_ERR_INVALID_ARG.
 * Solves on one stream at a time per object (they share its scratch). */
ib_status ib_stokes_solve(ib_stokes solver, const void* f, const void* u_old, void* u, double rho_over_k,
                          double mu, void* stream);

/* Synchronises the device, releases the plans and scratch; NULL is a no-op. */
ib_status ib_stokes_destroy(ib_stokes solver);

/* Self-test of the bounded device-side waits.  The binning scan (an exclusive
 * prefix of the per-cell counts in one pass with decoupled look-back: each
 * block waits for the chunk totals before its own) polls every wait a
 * bounded number of times; a wait that runs out records IB_ERR_TIMEOUT in
 * the error word and the kernel goes on to its end, so the device stays
 * usable.  This call runs that wait once against a chunk state that nothing
 * publishes, with a short limit (about 100 microseconds of polling), on
 * `stream`, and returns what the error word reports: IB_ERR_TIMEOUT when the
 * wait ran out and the kernel ended, as designed; IB_OK if it did not run
 * out; IB_ERR_OOM or IB_ERR_CUDA if the test could not run.  Uses its own
 * small stream-ordered scratch (cudaMallocAsync / cudaFreeAsync) and
 * synchronises `stream`.  Paper counterpart: none. */
ib_status ib_selftest_bounded_wait(void* stream);

/* Human-readable name of a status code (static storage). */
const char* ib_status_string(ib_status status);

/* Library version string (static storage). */
const char* ib_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IB_H */
