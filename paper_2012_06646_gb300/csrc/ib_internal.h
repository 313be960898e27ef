// ib_internal.h -- host-side launch interface between the C ABI (ib_api.cu)
// and the kernel translation units (ib_bin.cu, ib_ops.cu).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ib_common.cuh"

namespace ibgb {

// NVTX range over one C-ABI call: profilers attribute the kernels the call
// enqueues to a range named after the entry point (ncu --nvtx-include
// "ib_spread/").  Without a profiler attached the push and pop do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Tile side of the spreading boxes: 16 in 3-D when the box (side + 4)^3 of
// every component and the staging records fit in shared memory, else 8; 32 in 2-D.
int spread_tile_side(int dim, int elem_bytes, bool comp, int ncomp);

// Bytes of one spreading box (all components) for a tile side and a kernel
// support width s (box side tile + s).
size_t box_bytes(int dim, int tile, int entry_bytes, int ncomp, int width = 4);

// Support width s of a kernel (Section 3.1): 4 for the 4-point kernels, 3 for
// the 3-point kernel, 6 for the 6-point B-spline.
int kernel_width(int kernel);

// Spreading and interpolation for kernels of width s != 4 (ib_width.cu), a
// single job: tile boxes of side TS + s, then the fixed-order combination;
// interpolation by tiles with the box of grid values in shared memory.
cudaError_t launch_spread_width(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles,
                                int dtype, bool accumulate, cudaStream_t s);
cudaError_t launch_interp_width(const Jobs& J, const Shape& sh, const Bins& B, long long nitiles, int dtype,
                                double scale, cudaStream_t s);
cudaError_t launch_pos_grad_width(const Jobs& J, const Shape& sh, const Bins& B, int dtype, const void* field,
                                  const void* v, double scale, void* D, cudaStream_t s);

// Bounded (non-periodic) dimensions (ib_bounds.cu): f [ncomp][domain nodes] =
// (f +) the domain's nodes of fx [ncomp][extended nodes]; ux = u on the domain's
// nodes and 0 on the ghost nodes.
cudaError_t launch_bounds_crop(const Job& jb, int ncomp, int dtype, const void* fx, void* f, bool accumulate,
                               cudaStream_t s);
cudaError_t launch_bounds_pad(const Job& jb, int ncomp, int dtype, const void* u, void* ux, cudaStream_t s);

// Cells per block of the cell-count scan, and the number of blocks for m entries.
constexpr long long kScanChunkCells = 8192;
long long scan_blocks(long long m);

// Zero the per-cell counts and the scan state that follows them (one memset;
// B.scan must sit right after B.count), before every binning.
size_t bin_clear_bytes(const Bins& B);
cudaError_t clear_bins(const Bins& B, cudaStream_t s);

// The binning scan's look-back wait run against a chunk state that nothing
// publishes (a self-test of the bounded wait): `state` holds 3 zeroed words,
// `a` 2 kScanChunkCells + 1 entries; must set ERR_TIMEOUT after spin_limit polls.
cudaError_t launch_scan_wait_selftest(uint32_t* a, unsigned long long* state, uint32_t* err, int spin_limit,
                                      cudaStream_t s);

// Binning (Algorithm 4 keys, sort and unique-key offsets): count, scan,
// scatter and stable fix-up.  B.count must be zeroed by the caller.  Keys are
// cells of xi = 0, or with key_comp >= 0 cells in the staggering of that
// component (the per-component keys of the paper's spreading algorithms).
cudaError_t launch_bin(const Jobs& J, const Shape& sh, const Bins& B, int dtype, cudaStream_t s, int key_comp = -1);

// The paper's parallel spreading (Algorithm 4: one segmented reduce per
// shift; Algorithms 5 and 6: beta shifts per pass into beta grid buffers) for
// component a of a single job, on bins keyed by that component's cells and
// its list of inhabited cells:
// shifts j0 .. j0 + nshift - 1 (colexicographic digits, x fastest); the
// reduced value of shift j0 + k is added to out[k * out_stride + node] (out is
// the component's grid, or a buffer of grids).  Distinct shifts of one launch
// must go to distinct grids (out_stride >= ncell) or nshift must be 1.
cudaError_t launch_paper_shifts(const Jobs& J, const Shape& sh, const Bins& B, int dtype, int a, int j0, int nshift,
                                void* out, long long out_stride, const uint32_t* cells, const uint32_t* q,
                                cudaStream_t s);

// The inhabited cells of the bins ("count unique" of Algorithm 4): cells[0 .. *q).
cudaError_t launch_paper_cells(const Bins& B, uint32_t* cells, uint32_t* q, cudaStream_t s);

// f_a[node] = sum_{k < beta} buf[k * ncell + node], k increasing (Algorithm 5's final sum).
cudaError_t launch_paper_sum(const Jobs& J, int dtype, int a, int beta, const void* buf, cudaStream_t s);

// Spreading in two launches: per-tile boxes in shared memory written to
// `boxes`, then the fixed-order combination of overlapping boxes into f.
// even_n0: every job of the launch has an even n0 (the combination then
// handles two x-adjacent nodes per thread).
// overlap: the tile kernel may start before the kernel before it on the stream
// completes (IB_OVERLAP_PREVIOUS; the caller guarantees that kernel wrote
// nothing the spreading reads).
cudaError_t launch_spread(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long ntiles_total,
                          int tile, int dtype, bool compensated, bool accumulate, bool even_n0, cudaStream_t s,
                          bool overlap = false);

// z-slab pieces of three-component 3-D spreading (8^3 tiles): the tile boxes
// of tiles [tile_begin, tile_begin + ntiles) only (dense: every box written),
// and the combination of cells [cell_begin, cell_end) only.
cudaError_t launch_slab_boxes(const Jobs& J, const Shape& sh, const Bins& B, void* boxes, long long tile_begin,
                              long long ntiles, int dtype, bool comp, cudaStream_t s);
cudaError_t launch_slab_combine(const Jobs& J, const Shape& sh, const Bins& B, const void* boxes, long long cell_begin,
                                long long cell_end, int dtype, bool comp, bool accumulate, bool even_n0,
                                cudaStream_t s);

// Slab of each point (its xi = 0 cell's tile layer along z within the bounds),
// -1 for an invalid position.
constexpr int kMaxSlabs = 64;
struct SlabBounds {
  int nslab;
  int tile;                    // tile side along z
  int bound[kMaxSlabs + 1];    // tile layers: slab k owns [bound[k], bound[k + 1])
};
cudaError_t launch_slab_owner(const Jobs& J, const SlabBounds& sb, long long n, int dtype, int* owner, cudaStream_t s);

// Tile side of the interpolation tiles: 8 in 3-D, 32 in 2-D.
inline int interp_tile_side(int dim) { return dim == 3 ? 8 : 32; }

// Interpolation by tiles (Job::itile geometry); every value is multiplied by
// `scale` (1 for plain interpolation).
cudaError_t launch_interp(const Jobs& J, const Shape& sh, const Bins& B, long long nitiles, int dtype, double scale,
                          cudaStream_t s);

cudaError_t launch_pos_grad(const Jobs& J, const Shape& sh, const Bins& B, int dtype, const void* field,
                            const void* v, double scale, void* D, cudaStream_t s);

// overlap: IB_OVERLAP_PREVIOUS (the kernel before wrote neither X nor U).
cudaError_t launch_advect(const Jobs& J, const Shape& sh, int dtype, const void* U, double dt, void* Xout,
                          cudaStream_t s, bool overlap = false);

}  // namespace ibgb
