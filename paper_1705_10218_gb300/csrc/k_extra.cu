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

// Values of 32 consecutive output blocks per warp step, as one flat range:
// lane b first reads block g0 + b's length, sources and destination (one
// dependent load chain per 32 blocks instead of one per block) into shared
// memory, then the warp walks the concatenated values lane by lane, each lane
// tracking the block its element falls in. Each value is beta*C_in + alpha*A
// rounded as two separate operations (the oracle's order); copy = 1 copies A's
// values unchanged. sa / sc: the A and C_in block of each output block, or -1
// (sc may be null: no C_in). Launched with kSegWarps warps per block.
constexpr int kSegWarps = 8;

__global__ void __launch_bounds__(kSegWarps * 32)
    k_seg_values(DevMat A, DevMat Cin, double alpha, double beta,
                 const int32_t *__restrict__ sa, const int32_t *__restrict__ sc, int copy,
                 DevOut O, const DevStatus *st) {
  if (st->overflow) return;
  __shared__ int s_end[kSegWarps][32], s_len[kSegWarps][32];
  __shared__ int64_t s_oa[kSegWarps][32], s_oc[kSegWarps][32], s_od[kSegWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool alpha1 = (alpha == 1.0), beta1 = (beta == 1.0);
  const int64_t n = st->nblk_c;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g0 = w0 * 32; g0 < n; g0 += nw * 32) {
    const int64_t g = g0 + lane;
    int len = 0;
    int64_t oa = -1, oc = -1, od = 0;
    if (g < n) {
      len = O.row_sizes[O.blk_row[g]] * O.col_sizes[O.col_idx[g]];
      const int ia = sa[g];
      const int ic = sc ? sc[g] : -1;
      oa = ia >= 0 ? A.blk_off[ia] : -1;
      oc = ic >= 0 ? Cin.blk_off[ic] : -1;
      od = O.blk_off[g];
    }
    // inclusive prefix of the lengths over the 32 blocks
    int pre = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, pre, d);
      if (lane >= d) pre += y;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    s_end[warp][lane] = pre;
    s_len[warp][lane] = len;
    s_oa[warp][lane] = oa;
    s_oc[warp][lane] = oc;
    s_od[warp][lane] = od;
    __syncwarp();
    int k = 0;  // the block of this lane's element (non-decreasing in f)
    for (int f = lane; f < total; f += 32) {
      while (f >= s_end[warp][k]) k++;
      const int e = f - (s_end[warp][k] - s_len[warp][k]);
      const int64_t ka = s_oa[warp][k], kc = s_oc[warp][k];
      double v;
      if (copy) {
        v = A.vals[ka + e];
      } else {  // a product with 1 is exact: skipped (the FP64 pipe is the slow unit)
        double base = 0.0;
        if (kc >= 0) base = beta1 ? Cin.vals[kc + e] : __dmul_rn(beta, Cin.vals[kc + e]);
        v = base;
        if (ka >= 0) {
          const double x = alpha1 ? A.vals[ka + e] : __dmul_rn(alpha, A.vals[ka + e]);
          v = __dadd_rn(base, x);
        }
      }
      O.vals[s_od[warp][k] + e] = v;
    }
    __syncwarp();  // the table is read before the next step writes it
  }
}


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

// Kept blocks to their new places (same order) and their source block in
// ws.cnt. One warp per row.
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
        ws.cnt[q] = p;  // source block: the values are copied by k_seg_values
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
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  DevMat none{};
  k_seg_values<<<nsm * 8, kSegWarps * 32, 0, stream>>>(M, none, 1.0, 0.0, ws.cnt, nullptr, 1, O,
                                                        st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// C = beta*C + alpha*A. One warp per block row; the union of A's and C_in's
// sorted column lists is formed without a serial merge: a column's place in
// the union is its index in its own list plus the number of columns of the
// other list below it (binary search), minus the columns below it counted in
// both lists.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lower_bound_i32(const int32_t *__restrict__ v, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_add_count(DevMat A, DevMat Cin, int use_cin, DevWs ws) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < A.nbr; i += nw) {
    const int a0 = A.row_ptr[i], na = A.row_ptr[i + 1] - a0;
    const int c0 = use_cin ? Cin.row_ptr[i] : 0, nc = use_cin ? Cin.row_ptr[i + 1] - c0 : 0;
    const int32_t *ac = A.col_idx + a0, *cc = use_cin ? Cin.col_idx + c0 : nullptr;
    int64_t dup = 0, cols = 0;
    for (int a = lane; a < na; a += 32) {
      const int j = ac[a];
      cols += A.col_sizes[j];
      if (nc) {
        const int l = lower_bound_i32(cc, nc, j);
        dup += (l < nc && cc[l] == j);
      }
    }
    for (int c = lane; c < nc; c += 32) {
      const int j = cc[c];
      const int l = na ? lower_bound_i32(ac, na, j) : 0;
      if (!(l < na && ac[l] == j)) cols += A.col_sizes[j];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      dup += __shfl_xor_sync(0xffffffffu, dup, d);
      cols += __shfl_xor_sync(0xffffffffu, cols, d);
    }
    if (lane == 0) {
      ws.row_cblk[i] = (int32_t)(na + nc - dup);
      ws.row_nnz[i] = (int64_t)A.row_sizes[i] * cols;
      ws.row_prod[i] = 0;
      ws.row_cand[i] = 0;
      ws.row_flops[i] = 0;
    }
  }
}

// The union pattern, each output block's sources in ws.cnt (A block or -1) and
// ws.c_cin (C_in block or -1), and the blocks' value offsets.
__global__ void k_add_fill(DevMat A, DevMat Cin, int use_cin, DevWs ws, DevOut O,
                           const DevStatus *st) {
  if (st->overflow) return;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < A.nbr; i += nw) {
    const int a0 = A.row_ptr[i], na = A.row_ptr[i + 1] - a0;
    const int c0 = use_cin ? Cin.row_ptr[i] : 0, nc = use_cin ? Cin.row_ptr[i + 1] - c0 : 0;
    const int32_t *ac = A.col_idx + a0, *cc = use_cin ? Cin.col_idx + c0 : nullptr;
    const int g0 = O.row_ptr[i];
    // A's columns (with the matching C_in block, if any)
    int carry = 0;  // A columns of the earlier chunks that are also in C_in
    for (int base = 0; base < na; base += 32) {
      const int a = base + lane;
      const bool in = a < na;
      const int j = in ? ac[a] : 0;
      const int l = (in && nc) ? lower_bound_i32(cc, nc, j) : 0;
      const bool both = in && l < nc && cc[l] == j;
      const unsigned ball = __ballot_sync(0xffffffffu, both);
      if (in) {
        const int pos = a + l - (carry + __popc(ball & below));
        O.col_idx[g0 + pos] = j;
        O.blk_row[g0 + pos] = (int32_t)i;
        ws.cnt[g0 + pos] = a0 + a;
        ws.c_cin[g0 + pos] = both ? c0 + l : -1;
      }
      carry += __popc(ball);
    }
    // C_in's columns that A does not have
    carry = 0;  // C_in columns of the earlier chunks that are also in A
    for (int base = 0; base < nc; base += 32) {
      const int c = base + lane;
      const bool in = c < nc;
      const int j = in ? cc[c] : 0;
      const int l = (in && na) ? lower_bound_i32(ac, na, j) : 0;
      const bool both = in && l < na && ac[l] == j;
      const unsigned ball = __ballot_sync(0xffffffffu, both);
      if (in && !both) {
        const int pos = c + l - (carry + __popc(ball & below));
        O.col_idx[g0 + pos] = j;
        O.blk_row[g0 + pos] = (int32_t)i;
        ws.cnt[g0 + pos] = -1;
        ws.c_cin[g0 + pos] = c0 + c;
      }
      carry += __popc(ball);
    }
    __syncwarp();
    // value offsets: a scan of the union blocks' sizes in column order
    const int nb = O.row_ptr[i + 1] - g0;
    const int m = A.row_sizes[i];
    int64_t run = ws.nnz_off[i];
    for (int base = 0; base < nb; base += 32) {
      const int g = base + lane;
      const int len = g < nb ? m * A.col_sizes[O.col_idx[g0 + g]] : 0;
      int pre = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, pre, d);
        if (lane >= d) pre += y;
      }
      if (g < nb) O.blk_off[g0 + g] = run + pre - len;
      run += __shfl_sync(0xffffffffu, pre, 31);
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
    k_add_count<<<nsm * 8, 256, 0, stream>>>(A, Cin, use_cin, ws);
  else if (stage == 1)
    k_add_fill<<<nsm * 8, 256, 0, stream>>>(A, Cin, use_cin, ws, O, st);
  else
    k_seg_values<<<nsm * 8, kSegWarps * 32, 0, stream>>>(A, Cin, alpha, beta, ws.cnt, ws.c_cin,
                                                          0, O, st);
  return cudaGetLastError();
}

}  // namespace bsm
