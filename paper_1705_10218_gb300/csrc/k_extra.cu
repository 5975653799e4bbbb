// k_extra.cu -- two operations on block-sparse matrices beside the multiply:
//
//  * the post-multiplication filter (Sec. 1: filtering also after each
//    multiplication; Sec. 2: blocks below the threshold are removed after the
//    multiplication): a block is dropped iff its canonical norm is below eps;
//  * block-sparse accumulation C = beta*C + alpha*A on the union of the
//    patterns (Algorithm 2: the partial C panels of the last ticks are summed
//    into the final panel; the paper does this on the CPU).
//
// Both write a new pattern into the matrix's back buffers (the caller swaps),
// through the same per-row count / scan / fill structure as the multiply.
#include "bsm_internal.h"

namespace bsm {

// ---------------------------------------------------------------------------
// Post filter. keep[b] = !(norm[b] < eps). One warp per block row.
// ---------------------------------------------------------------------------
__global__ void k_filter_count(DevMat M, double eps, DevWs ws) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < M.nbr; i += nw) {
    int64_t kb = 0, kv = 0;
    for (int p = M.row_ptr[i] + lane; p < M.row_ptr[i + 1]; p += 32) {
      if (!(M.norms[p] < eps)) {
        kb++;
        kv += (int64_t)M.row_sizes[i] * M.col_sizes[M.col_idx[p]];
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      kb += __shfl_xor_sync(0xffffffffu, kb, d);
      kv += __shfl_xor_sync(0xffffffffu, kv, d);
    }
    if (lane == 0) {
      ws.row_cblk[i] = (int32_t)kb;
      ws.row_nnz[i] = kv;
      ws.row_prod[i] = 0;
      ws.row_cand[i] = 0;
      ws.row_flops[i] = 0;
    }
  }
}

// Kept blocks to their new places (same order), values copied. One warp per row.
__global__ void k_filter_fill(DevMat M, double eps, DevWs ws, DevOut O, const DevStatus *st) {
  if (st->overflow) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < M.nbr; i += nw) {
    int g = O.row_ptr[i];
    int64_t off = ws.nnz_off[i];
    const int m = M.row_sizes[i];
    for (int base = M.row_ptr[i]; base < M.row_ptr[i + 1]; base += 32) {
      const int p = base + lane;
      const bool in = p < M.row_ptr[i + 1];
      const bool keep = in && !(M.norms[p] < eps);
      const int len = keep ? m * M.col_sizes[M.col_idx[p]] : 0;
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      // exclusive prefix of the kept lengths
      int pre = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, pre, d);
        if (lane >= d) pre += y;
      }
      const int total = __shfl_sync(0xffffffffu, pre, 31);
      pre -= len;
      if (keep) {
        const int q = g + __popc(ball & ((1u << lane) - 1u));
        O.col_idx[q] = M.col_idx[p];
        O.blk_row[q] = (int32_t)i;
        O.blk_off[q] = off + pre;
      }
      // copy the kept blocks' values, one block at a time across the warp
      unsigned todo = ball;
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int pp = base + src;
        const int l = __shfl_sync(0xffffffffu, len, src);
        const int64_t dst = off + __shfl_sync(0xffffffffu, pre, src);
        const double *from = M.vals + M.blk_off[pp];
        for (int e = lane; e < l; e += 32) O.vals[dst + e] = from[e];
      }
      g += __popc(ball);
      off += total;
    }
  }
}

cudaError_t launch_filter_count(DevMat M, double eps, DevWs ws, int nsm, cudaStream_t stream) {
  k_filter_count<<<nsm * 4, 256, 0, stream>>>(M, eps, ws);
  return cudaGetLastError();
}

cudaError_t launch_filter_fill(DevMat M, double eps, DevWs ws, DevOut O, const DevStatus *st,
                               int nsm, cudaStream_t stream) {
  k_filter_fill<<<nsm * 4, 256, 0, stream>>>(M, eps, ws, O, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// C = beta*C + alpha*A. One thread per block row merges the two sorted column
// lists (A's row and, when beta != 0, C's row).
// ---------------------------------------------------------------------------
__global__ void k_add_count(DevMat A, DevMat Cin, int use_cin, DevWs ws) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int pa = A.row_ptr[i], ea = A.row_ptr[i + 1];
    int pc = use_cin ? Cin.row_ptr[i] : 0, ec = use_cin ? Cin.row_ptr[i + 1] : 0;
    int64_t nb = 0, cols = 0;
    while (pa < ea || pc < ec) {
      const int ja = pa < ea ? A.col_idx[pa] : INT32_MAX;
      const int jc = pc < ec ? Cin.col_idx[pc] : INT32_MAX;
      const int j = min(ja, jc);
      nb++;
      cols += A.col_sizes[j];
      if (ja == j) pa++;
      if (jc == j) pc++;
    }
    ws.row_cblk[i] = (int32_t)nb;
    ws.row_nnz[i] = (int64_t)A.row_sizes[i] * cols;
    ws.row_prod[i] = 0;
    ws.row_cand[i] = 0;
    ws.row_flops[i] = 0;
  }
}

// The union pattern, each output block's sources in ws.cnt (A block or -1) and
// ws.c_cin (C_in block or -1).
__global__ void k_add_fill(DevMat A, DevMat Cin, int use_cin, DevWs ws, DevOut O,
                           const DevStatus *st) {
  if (st->overflow) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int pa = A.row_ptr[i], ea = A.row_ptr[i + 1];
    int pc = use_cin ? Cin.row_ptr[i] : 0, ec = use_cin ? Cin.row_ptr[i + 1] : 0;
    int g = O.row_ptr[i];
    int64_t off = ws.nnz_off[i];
    const int m = A.row_sizes[i];
    while (pa < ea || pc < ec) {
      const int ja = pa < ea ? A.col_idx[pa] : INT32_MAX;
      const int jc = pc < ec ? Cin.col_idx[pc] : INT32_MAX;
      const int j = min(ja, jc);
      O.col_idx[g] = j;
      O.blk_row[g] = (int32_t)i;
      O.blk_off[g] = off;
      ws.cnt[g] = (ja == j) ? pa : -1;
      ws.c_cin[g] = (jc == j) ? pc : -1;
      off += (int64_t)m * A.col_sizes[j];
      g++;
      if (ja == j) pa++;
      if (jc == j) pc++;
    }
  }
}

// Values: one warp per output block.
__global__ void k_add_values(DevMat A, DevMat Cin, double alpha, double beta, DevWs ws, DevOut O,
                             const DevStatus *st) {
  if (st->overflow) return;
  const int lane = threadIdx.x & 31;
  const int64_t n = st->nblk_c;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = w0; g < n; g += nw) {
    const int len = O.row_sizes[O.blk_row[g]] * O.col_sizes[O.col_idx[g]];
    const int sa = ws.cnt[g], sc = ws.c_cin[g];
    const double *va = sa >= 0 ? A.vals + A.blk_off[sa] : nullptr;
    const double *vc = sc >= 0 ? Cin.vals + Cin.blk_off[sc] : nullptr;
    double *out = O.vals + O.blk_off[g];
    for (int e = lane; e < len; e += 32) {
      const double base = vc ? beta * vc[e] : 0.0;
      out[e] = va ? fma(alpha, va[e], base) : base;
    }
  }
}

// ---------------------------------------------------------------------------
// Values of the result to host memory (pinned, device-mapped): C's values are
// contiguous in block order, [0, nnz).
// ---------------------------------------------------------------------------
__global__ void k_copy_out(DevOut O, const DevStatus *st) {
  if (st->overflow) return;
  const int64_t n = st->nnz_c;
  if (n > O.host_cap) return;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = t0; e < n; e += nt) O.host_vals[e] = O.vals[e];
}

cudaError_t launch_copy_out(DevOut O, const DevStatus *st, int nsm, cudaStream_t stream) {
  k_copy_out<<<nsm * 8, 256, 0, stream>>>(O, st);
  return cudaGetLastError();
}

cudaError_t launch_add(int stage, DevMat A, DevMat Cin, int use_cin, double alpha, double beta,
                       DevWs ws, DevOut O, const DevStatus *st, int nsm, cudaStream_t stream) {
  if (stage == 0)
    k_add_count<<<nsm * 2, 128, 0, stream>>>(A, Cin, use_cin, ws);
  else if (stage == 1)
    k_add_fill<<<nsm * 2, 128, 0, stream>>>(A, Cin, use_cin, ws, O, st);
  else
    k_add_values<<<nsm * 4, 256, 0, stream>>>(A, Cin, alpha, beta, ws, O, st);
  return cudaGetLastError();
}

}  // namespace bsm
