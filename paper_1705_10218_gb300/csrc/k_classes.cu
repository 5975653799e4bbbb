// k_classes.cu -- grouping of the C blocks by shape class (row size, column
// size), the "stacks" of the numeric phase: the paper's local multiply
// organises its small block products in batches (Sec. 2); here a batch is
// the set of C blocks of one (m, n) class, each C block carrying its own
// k-ordered product list. The grouping is a counting sort: a histogram over
// classes, an exclusive scan, and a scatter. The order inside a class is not
// fixed (it only decides which warp takes which block, never a result).
#include "bsm_internal.h"

namespace bsm {

__global__ void k_class_count(DevOut C, const int32_t *__restrict__ row_cls,
                              const int32_t *__restrict__ col_cls, int ncc, int ncls,
                              const DevStatus *st, int32_t *__restrict__ counts) {
  if (st->overflow) return;
  __shared__ int32_t hist[kMaxClasses];
  for (int c = threadIdx.x; c < ncls; c += blockDim.x) hist[c] = 0;
  __syncthreads();
  const int64_t n = st->nblk_c;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int c = row_cls[C.blk_row[g]] * ncc + col_cls[C.col_idx[g]];
    atomicAdd(&hist[c], 1);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncls; c += blockDim.x)
    if (hist[c]) atomicAdd(&counts[c], hist[c]);
}

__global__ void k_class_scan(int ncls, const DevStatus *st, const int32_t *__restrict__ counts,
                             int32_t *__restrict__ cursor, int64_t *__restrict__ segs) {
  if (st->overflow) return;
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int c = 0; c < ncls; c++) {
      segs[2 * c] = run;
      run += counts[c];
      segs[2 * c + 1] = run;
      cursor[c] = 0;
    }
  }
}

__global__ void k_class_scatter(DevOut C, const int32_t *__restrict__ row_cls,
                                const int32_t *__restrict__ col_cls, int ncc,
                                const DevStatus *st, const int64_t *__restrict__ segs,
                                int32_t *__restrict__ cursor, int32_t *__restrict__ items) {
  if (st->overflow) return;
  const int64_t n = st->nblk_c;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int c = row_cls[C.blk_row[g]] * ncc + col_cls[C.col_idx[g]];
    const int pos = atomicAdd(&cursor[c], 1);
    items[segs[2 * c] + pos] = (int32_t)g;
  }
}

cudaError_t launch_class_sort(DevOut C, const int32_t *row_cls, const int32_t *col_cls, int ncc,
                              int ncls, const DevStatus *st, int32_t *counts, int32_t *cursor,
                              int64_t *segs, int32_t *items, int nsm, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)ncls * sizeof(int32_t), stream);
  if (e != cudaSuccess) return e;
  k_class_count<<<nsm * 2, 256, 0, stream>>>(C, row_cls, col_cls, ncc, ncls, st, counts);
  k_class_scan<<<1, 32, 0, stream>>>(ncls, st, counts, cursor, segs);
  k_class_scatter<<<nsm * 2, 256, 0, stream>>>(C, row_cls, col_cls, ncc, st, segs, cursor, items);
  return cudaGetLastError();
}

// segs[2s], segs[2s + 1]: the s-th of n consecutive, nearly equal ranges of
// the multiply's C blocks (the count is known on the device only).
__global__ void k_slice_segs(const DevStatus *st, int n, int64_t *__restrict__ segs) {
  if (st->overflow) return;
  const int64_t total = st->nblk_c;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    segs[2 * s] = total * s / n;
    segs[2 * s + 1] = total * (s + 1) / n;
  }
}

cudaError_t launch_slice_segs(const DevStatus *st, int n, int64_t *segs, cudaStream_t stream) {
  k_slice_segs<<<1, 64, 0, stream>>>(st, n, segs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Work in a row order. row_order[p] is the C block row at position p of a
// permutation of the rows, row_pos[r] the position of row r. items receives
// the C blocks of row row_order[0] (in column order), then those of row
// row_order[1], and so on. The numeric kernels hand out C blocks in item
// order, so with a breadth-first order of A's pattern, C block rows whose
// neighbourhoods overlap run close together in time and find the B rows they
// read still in L2 (in the natural order of a system with random atom order,
// consecutive rows share almost nothing). The order decides only which warp
// takes which block when, never a result.

// start[p]: the first item of position p (exclusive scan of the rows' block
// counts in position order), one thread block in tiles of blockDim.x rows.
__global__ void k_order_scan(DevOut C, const int32_t *__restrict__ row_order, int32_t nbr,
                             const DevStatus *st, int32_t *__restrict__ start) {
  if (st->overflow) return;
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t base = 0; base < nbr; base += blockDim.x) {
    const int32_t p = base + threadIdx.x;
    int32_t v = 0;
    if (p < nbr) {
      const int32_t r = row_order[p];
      v = C.row_ptr[r + 1] - C.row_ptr[r];
    }
    int32_t x = v;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {  // inclusive scan of the warp totals
      int32_t t = lane < nwarps ? warp_tot[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nwarps) warp_tot[lane] = t;
    }
    __syncthreads();
    const int32_t excl = (warp ? warp_tot[warp - 1] : 0) + x - v;
    if (p < nbr) start[p] = carry + excl;
    __syncthreads();  // every thread has read carry
    if (threadIdx.x == blockDim.x - 1) carry += excl + v;
    __syncthreads();
  }
}

__global__ void k_order_fill(DevOut C, const int32_t *__restrict__ row_pos, const DevStatus *st,
                             const int32_t *__restrict__ start, int32_t *__restrict__ items) {
  if (st->overflow) return;
  const int64_t n = st->nblk_c;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = C.blk_row[g];
    items[start[row_pos[r]] + (int32_t)(g - C.row_ptr[r])] = (int32_t)g;
  }
}

cudaError_t launch_order_items(DevOut C, const int32_t *row_order, const int32_t *row_pos,
                               int32_t nbr, const DevStatus *st, int32_t *start, int32_t *items,
                               int nsm, cudaStream_t stream) {
  k_order_scan<<<1, 1024, 0, stream>>>(C, row_order, nbr, st, start);
  k_order_fill<<<nsm * 2, 256, 0, stream>>>(C, row_pos, st, start, items);
  return cudaGetLastError();
}

}  // namespace bsm
