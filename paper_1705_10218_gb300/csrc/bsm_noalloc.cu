// bsm_noalloc.cu -- bsm_multiply_noalloc: the FP64 multiply for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not safe --
// inside a memory-pool-managed framework that owns all device memory, in a
// real-time or interrupt-like callback that must not block on the allocator,
// or in a process whose allocator is already at its limit. Such a caller can
// still hand over the device buffers it owns (inputs and outputs); the
// temporary memory the multiply needs (norms, per-row counters, the grouped
// product records, a status word) then comes from one fixed array that is part
// of the library image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds BSM_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so every call looks the address up with
// cudaGetSymbolAddress for the current device (no allocation; a device reset
// between calls is therefore harmless). The first call on a device also sets
// the numeric kernel's shared-memory attribute; it should come before any
// stream capture. All calls share the array and it keeps the contents of the
// previous call: whatever must start at zero is cleared here, and calls that
// overlap on the GPU (two streams, two threads) race on it.
//
// The caller's arrays are device memory the host cannot read cheaply, so a
// first kernel checks them (row pointers, column indices, block sizes, block
// offsets) and the call reads the outcome back before any other kernel uses
// them as indices: a malformed matrix is an error code, not a stray access.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bsm_internal.h"

using namespace bsm;

static __device__ __align__(256) unsigned char g_noalloc_scratch[BSM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
bool g_noalloc_init[kMaxDevices] = {};

// Outcome bits of the input check.
enum : int32_t {
  kBadRowPtr = 1,   // row_ptr[0] != 0, decreasing, or row_ptr[nbr] != nblk
  kBadColIdx = 2,   // a column index outside [0, nbc)
  kBadOrder = 4,    // columns of a row not strictly increasing (unsorted or duplicate)
  kBadSize = 8,     // a block size below 1
  kBadDims = 16,    // A's column sizes differ from B's row sizes
  kBadOffset = 32   // a negative block offset
};

struct CsrView {
  int32_t nbr, nbc;
  const int32_t *row_sizes, *col_sizes, *row_ptr, *col_idx;
  const int64_t *blk_off;
  int64_t nblk;
};

// One operand's blocked CSR: every read stays inside the sizes the caller
// declared (row_ptr[0..nbr], col_idx / blk_off[0..nblk), the size arrays);
// the column indices of a row are visited only when its row pointers are
// inside [0, nblk] and in order.
__device__ void check_csr(const CsrView &m, int64_t tid, int64_t nth, int32_t *flags) {
  int32_t bad = 0;
  if (tid == 0 && (m.row_ptr[0] != 0 || (int64_t)m.row_ptr[m.nbr] != m.nblk)) bad |= kBadRowPtr;
  for (int64_t i = tid; i < m.nbr; i += nth) {
    const int64_t a = m.row_ptr[i], b = m.row_ptr[i + 1];
    if (a < 0 || b < a || b > m.nblk) {
      bad |= kBadRowPtr;
      continue;
    }
    int32_t prev = -1;
    for (int64_t x = a; x < b; x++) {
      const int32_t c = m.col_idx[x];
      if (c < 0 || c >= m.nbc) bad |= kBadColIdx;
      else if (c <= prev) bad |= kBadOrder;
      if (c > prev) prev = c;
      if (m.blk_off[x] < 0) bad |= kBadOffset;
    }
  }
  for (int64_t i = tid; i < m.nbr; i += nth)
    if (m.row_sizes[i] < 1) bad |= kBadSize;
  for (int64_t i = tid; i < m.nbc; i += nth)
    if (m.col_sizes[i] < 1) bad |= kBadSize;
  if (bad) atomicOr(flags, bad);
}

__global__ void k_noalloc_check(CsrView A, CsrView B, int same, int32_t *flags) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  check_csr(A, tid, nth, flags);
  if (!same) check_csr(B, tid, nth, flags);
  // A's column block sizes against B's row block sizes (A.nbc == B.nbr here)
  int32_t bad = 0;
  for (int64_t k = tid; k < A.nbc; k += nth)
    if (A.col_sizes[k] != B.row_sizes[k]) bad |= kBadDims;
  if (bad) atomicOr(flags, bad);
}

// Expands CSR row pointers into per-block row indices, fills the two-word
// headers {nblk, nnz} of the operands and clears the status word.
__global__ void k_noalloc_setup(int32_t nbr_a, const int32_t *__restrict__ row_ptr_a,
                                int32_t *__restrict__ blk_row_a, int64_t *hdr_a, int64_t nblk_a,
                                int32_t nbr_b, const int32_t *__restrict__ row_ptr_b,
                                int32_t *__restrict__ blk_row_b, int64_t *hdr_b, int64_t nblk_b,
                                DevStatus *st) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0) {
    hdr_a[0] = nblk_a;
    hdr_a[1] = 0;
    if (hdr_b != hdr_a) {
      hdr_b[0] = nblk_b;
      hdr_b[1] = 0;
    }
    st->nblk_c = st->nnz_c = st->nprod = st->candidates = st->kept = st->flops = 0;
    st->overflow = 0;
    st->error = 0;
  }
  for (int64_t i = tid; i < nbr_a; i += nth)
    for (int32_t b = row_ptr_a[i]; b < row_ptr_a[i + 1]; b++) blk_row_a[b] = (int32_t)i;
  if (blk_row_b != blk_row_a)
    for (int64_t i = tid; i < nbr_b; i += nth)
      for (int32_t b = row_ptr_b[i]; b < row_ptr_b[i + 1]; b++) blk_row_b[b] = (int32_t)i;
}

// Bump allocation inside the static array, 256-byte aligned.
struct Carve {
  unsigned char *base;
  size_t used = 0;
  bool ok = true;
  template <class T>
  T *take(int64_t n) {
    const size_t bytes = ((size_t)(n > 0 ? n : 1) * sizeof(T) + 255) & ~(size_t)255;
    if (used + bytes > (size_t)BSM_NOALLOC_SCRATCH_BYTES) {
      ok = false;
      return nullptr;
    }
    T *p = reinterpret_cast<T *>(base + used);
    used += bytes;
    return p;
  }
};

int noalloc_cuda_fail(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? BSM_ERR_NOMEM : BSM_ERR_CUDA;
}

bool csr_ok(const bsm_dev_csr *m) {
  return m && m->nbr >= 0 && m->nbc >= 0 && m->nblk >= 0 && m->nblk < (int64_t)INT32_MAX &&
         (m->nbr == 0 || m->row_sizes) && (m->nbc == 0 || m->col_sizes) && m->row_ptr &&
         (m->nblk == 0 || (m->col_idx && m->blk_off && m->values));
}

}  // namespace

extern "C" int bsm_multiply_noalloc(double alpha, const bsm_dev_csr *A, const bsm_dev_csr *B,
                                    double eps, bsm_dev_csr_out *C, int64_t *sizes,
                                    void *stream) {
  if (!csr_ok(A) || !csr_ok(B) || !C || !sizes || !C->row_ptr || C->cap_blk < 0 ||
      C->cap_nnz < 0 || (C->cap_blk > 0 && (!C->col_idx || !C->blk_off)) ||
      (C->cap_nnz > 0 && !C->values))
    return BSM_ERR_INVALID_ARG;
  if (A->nbc != B->nbr) return BSM_ERR_DIM_MISMATCH;
  cudaStream_t s = (cudaStream_t)stream;

  // every call: the device address of the static array on the current device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return BSM_ERR_UNSUPPORTED;
  unsigned char *scratch;
  {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return noalloc_cuda_fail(e);
    scratch = static_cast<unsigned char *>(p);
    // the numeric kernel's shared-memory size attribute, once per device
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_init[dev]) {
      e = numeric_fp64_init();
      if (e != cudaSuccess) return noalloc_cuda_fail(e);
      g_noalloc_init[dev] = true;
    }
  }

  // A and B are one matrix (its norms and row indices computed once) only when
  // the descriptors agree field by field
  const bool same = (A == B) || memcmp(A, B, sizeof(bsm_dev_csr)) == 0;
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_cuda_fail(e);

  // the input check, read back before any kernel indexes with the caller's arrays
  {
    int32_t *flags = reinterpret_cast<int32_t *>(scratch);
    auto cv_of = [](const bsm_dev_csr *m) {
      return CsrView{m->nbr, m->nbc, m->row_sizes, m->col_sizes, m->row_ptr, m->col_idx,
                     m->blk_off, m->nblk};
    };
    int32_t h_flags = 0;
    if ((e = cudaMemsetAsync(flags, 0, sizeof(int32_t), s)) != cudaSuccess)
      return noalloc_cuda_fail(e);
    k_noalloc_check<<<nsm * 2, 256, 0, s>>>(cv_of(A), cv_of(B), same ? 1 : 0, flags);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_flags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return noalloc_cuda_fail(e);
    if (h_flags & kBadColIdx) return BSM_ERR_OUT_OF_RANGE;
    if (h_flags & ~kBadDims) return BSM_ERR_INVALID_ARG;
    if (h_flags) return BSM_ERR_DIM_MISMATCH;
  }

  // layout of the scratch for this problem
  Carve cv{scratch};
  DevStatus *st = cv.take<DevStatus>(1);
  double *norms_a = cv.take<double>(A->nblk);
  float *normsf_a = cv.take<float>(A->nblk);
  int32_t *brow_a = cv.take<int32_t>(A->nblk);
  int64_t *hdr_a = cv.take<int64_t>(2);
  double *norms_b = same ? norms_a : cv.take<double>(B->nblk);
  float *normsf_b = same ? normsf_a : cv.take<float>(B->nblk);
  int32_t *brow_b = same ? brow_a : cv.take<int32_t>(B->nblk);
  int64_t *hdr_b = same ? hdr_a : cv.take<int64_t>(2);
  const int64_t rows = (int64_t)A->nbr + 1;
  DevWs ws{};
  ws.row_cblk = cv.take<int32_t>(rows);
  ws.row_prod = cv.take<int64_t>(rows);
  ws.row_nnz = cv.take<int64_t>(rows);
  ws.row_cand = cv.take<int64_t>(rows);
  ws.row_flops = cv.take<int64_t>(rows);
  ws.prod_off = cv.take<int64_t>(rows);
  ws.nnz_off = cv.take<int64_t>(rows);
  ws.cap_rows = rows;
  const int64_t cap_blk = C->cap_blk;
  int32_t *c_brow = cv.take<int32_t>(cap_blk);
  int64_t *c_hdr = cv.take<int64_t>(2);
  ws.cnt = cv.take<int32_t>(cap_blk + 1);
  ws.c_cin = cv.take<int32_t>(cap_blk + 1);
  ws.prod_ptr = cv.take<int64_t>(cap_blk + 2);
  if (!cv.ok) return BSM_ERR_UNSUPPORTED;  // exceeds the static scratch
  // the rest holds the product records
  const size_t left = (size_t)BSM_NOALLOC_SCRATCH_BYTES - cv.used;
  ws.cap_prod = (int64_t)(left / sizeof(int2));
  ws.prods = reinterpret_cast<int2 *>(scratch + cv.used);

  k_noalloc_setup<<<nsm * 2, 256, 0, s>>>(A->nbr, A->row_ptr, brow_a, hdr_a, A->nblk, B->nbr,
                                          B->row_ptr, brow_b, hdr_b, B->nblk, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_cuda_fail(e);

  auto view = [](const bsm_dev_csr *m, const int32_t *brow, const double *norms,
                 const float *normsf, const int64_t *hdr) {
    DevMat v{};
    v.nbr = m->nbr;
    v.nbc = m->nbc;
    v.row_sizes = m->row_sizes;
    v.col_sizes = m->col_sizes;
    v.row_ptr = m->row_ptr;
    v.col_idx = m->col_idx;
    v.blk_row = brow;
    v.blk_off = m->blk_off;
    v.vals = m->values;
    v.norms = norms;
    v.normsf = normsf;
    v.hdr = hdr;
    return v;
  };
  DevMat dA = view(A, brow_a, norms_a, normsf_a, hdr_a);
  DevMat dB = view(B, brow_b, norms_b, normsf_b, hdr_b);
  DevMat none{};
  DevOut out{};
  out.nbr = A->nbr;
  out.nbc = B->nbc;
  out.row_sizes = A->row_sizes;
  out.col_sizes = B->col_sizes;
  out.row_ptr = C->row_ptr;
  out.col_idx = C->col_idx;
  out.blk_row = c_brow;
  out.blk_off = C->blk_off;
  out.vals = C->values;
  out.hdr = c_hdr;
  out.cap_blk = cap_blk;
  out.cap_nnz = C->cap_nnz;

  if ((e = launch_block_norms(A->row_sizes, A->col_sizes, brow_a, A->col_idx, A->blk_off,
                              A->values, hdr_a, norms_a, normsf_a, nsm * 8, s)) != cudaSuccess)
    return noalloc_cuda_fail(e);
  if (!same && (e = launch_block_norms(B->row_sizes, B->col_sizes, brow_b, B->col_idx,
                                       B->blk_off, B->values, hdr_b, norms_b, normsf_b, nsm * 8,
                                       s)) !=
                   cudaSuccess)
    return noalloc_cuda_fail(e);
  if ((e = launch_symbolic_count(dA, dB, none, 0, eps, ws, nsm * 6, s)) != cudaSuccess)
    return noalloc_cuda_fail(e);
  if ((e = launch_symbolic_scan(A->nbr, ws, out, st, s)) != cudaSuccess)
    return noalloc_cuda_fail(e);
  if ((e = launch_symbolic_fill(dA, dB, none, 0, eps, ws, out, st, nsm, 0, s)) != cudaSuccess)
    return noalloc_cuda_fail(e);
  // block sizes live on the device only: the 32 x 32 tile variant handles any size
  if ((e = launch_numeric_fp64(kFp64T32, dA, dB, out, none, alpha, 0.0, ws, st, nullptr, nullptr,
                                nsm * 3, nullptr, 32, 32, s)) != cudaSuccess)
    return noalloc_cuda_fail(e);

  DevStatus h{};
  if ((e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return noalloc_cuda_fail(e);
  sizes[0] = h.nblk_c;
  sizes[1] = h.nnz_c;
  sizes[2] = h.nprod;
  if (h.overflow) {
    // C's buffers too small (sizes[] says how much is needed), or the product
    // records do not fit in what is left of the static scratch
    if (h.nblk_c > cap_blk || h.nnz_c > C->cap_nnz) return BSM_ERR_INVALID_ARG;
    return BSM_ERR_UNSUPPORTED;
  }
  return BSM_OK;
}
