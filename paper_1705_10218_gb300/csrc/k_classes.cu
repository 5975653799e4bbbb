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

}  // namespace bsm
