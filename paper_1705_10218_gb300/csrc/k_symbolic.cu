// k_symbolic.cu -- block norms, symbolic phase with the on-the-fly filter,
// and the per-C-block grouping of the kept products.
//
// Sec. 2 of the paper: the result pattern is determined by the multiplication
// itself, and a block product is only performed when the product of the two
// block norms passes the threshold. Here that becomes three device passes:
//   count: per C block row, the set of columns reached by a kept product
//          (a bitmap in shared memory), the number of kept products, FLOPs;
//   scan:  exclusive sums over block rows -> C's row pointers, product and
//          value offsets, and the capacity check of the output buffers;
//   fill:  per C block row, the sorted column list of C, every C block's
//          value offset, and the kept products written grouped by C block in
//          ascending k (a per-row counting sort), so that the numeric phase
//          accumulates each C block in one place, without atomics.
#include "bsm_internal.h"

namespace bsm {

// The filter of Sec. 2: drop iff nrm(A_ik)*nrm(B_kj) < eps (a tie and NaN are kept),
// decided exactly as FP64 decides it.
__device__ __forceinline__ bool keep_product(double na, double nb, double eps) {
  return !(__dmul_rn(na, nb) < eps);
}

// The same decision with FP32 arithmetic for all but the near-ties. The FP32
// copies of the norms are within 2^-24 (relative) of the FP64 norms and lie in
// [2^-60, 2^60] (else NaN), so their FP32 product is within 3*2^-24 of the
// exact product; it is compared with eps widened by 2^-20 either way (lo, hi),
// and only a product inside that band (or a NaN) takes the FP64 test.
struct EpsBand {
  float lo, hi;
};

__device__ __forceinline__ EpsBand eps_band(double eps) {
  EpsBand b;
  if (!(eps > 0.0)) {  // eps <= 0 (or NaN eps): every non-NaN product is kept
    b.lo = -INFINITY;
    b.hi = -INFINITY;
  } else if (eps >= 0x1p-100 && eps <= 0x1p100) {
    b.lo = __double2float_rd(eps * (1.0 - 0x1p-20));
    b.hi = __double2float_ru(eps * (1.0 + 0x1p-20));
  } else {  // out of the fast test's range: always the FP64 test
    b.lo = -INFINITY;
    b.hi = INFINITY;
  }
  if (eps != eps) {
    b.lo = -INFINITY;
    b.hi = INFINITY;
  }
  return b;
}

__device__ __forceinline__ bool keep_fast(float fa, float fb, double na, double nb, double eps,
                                          const EpsBand &band) {
  const float x = fa * fb;
  if (x >= band.hi) return true;
  if (x < band.lo) return false;
  return keep_product(na, nb, eps);
}

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int lo, int hi, int key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ----------------------------------------------------------------------------
// Block norms: canonical Frobenius norm, column-major, no fused multiply-add.
// One thread per block, grid-stride; the block count is read on the device so
// a matrix produced by an earlier multiply needs no host round trip.
// ----------------------------------------------------------------------------
__global__ void k_block_norms(const int32_t *__restrict__ row_sizes,
                              const int32_t *__restrict__ col_sizes,
                              const int32_t *__restrict__ blk_row,
                              const int32_t *__restrict__ col_idx,
                              const int64_t *__restrict__ blk_off,
                              const double *__restrict__ vals, const int64_t *__restrict__ hdr,
                              double *__restrict__ norms, float *__restrict__ normsf) {
  const int64_t nblk = hdr[0];
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = (int64_t)row_sizes[blk_row[b]] * col_sizes[col_idx[b]];
    const double *x = vals + blk_off[b];
    double s = 0.0;
    for (int64_t e = 0; e < n; e++) {
      const double v = __ldg(x + e);
      s = __dadd_rn(s, __dmul_rn(v, v));
    }
    const double nrm = __dsqrt_rn(s);
    norms[b] = nrm;
    normsf[b] = (nrm >= 0x1p-60 && nrm <= 0x1p60) ? __double2float_rn(nrm) : NAN;
  }
}

cudaError_t launch_block_norms(const int32_t *row_sizes, const int32_t *col_sizes,
                               const int32_t *blk_row, const int32_t *col_idx,
                               const int64_t *blk_off, const double *vals, const int64_t *hdr,
                               double *norms, float *normsf, int grid, cudaStream_t stream) {
  k_block_norms<<<grid, 256, 0, stream>>>(row_sizes, col_sizes, blk_row, col_idx, blk_off, vals,
                                          hdr, norms, normsf);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Block-wide exclusive scan of one int64 per thread (blockDim a multiple of 32,
// at most 1024). Returns the exclusive prefix; *total gets the block sum.
// ----------------------------------------------------------------------------
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < nwarps) ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nwarps) warp_sums[lane] = w;
  }
  __syncthreads();
  const int64_t before = (warp > 0) ? warp_sums[warp - 1] : 0;
  *total = warp_sums[nwarps - 1];
  __syncthreads();
  return before + x - v;
}

__device__ int64_t block_sum(int64_t v) {
  int64_t t;
  block_exclusive_scan(v, &t);
  return t;
}

// ----------------------------------------------------------------------------
// The kept-column bitmap of C block row i over the window [w0, w0+wn):
// bit (j-w0) is set iff some kept product (i,k,j) exists, or (when use_cin)
// C_in holds block (i,j). Warps walk A's row i, lanes walk B's row k.
// With COUNT, also counts candidates, kept products and their 2mnk.
// ----------------------------------------------------------------------------
template <bool COUNT>
__device__ void row_bitmap(const DevMat &A, const DevMat &B, const DevMat &Cin, int use_cin,
                           double eps, int i, int w0, int wn, bool whole, uint32_t *bitmap,
                           int nwords, int64_t &cand, int64_t &kept, int64_t &flops) {
  for (int t = threadIdx.x; t < nwords; t += blockDim.x) bitmap[t] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int m = A.row_sizes[i];
  const int p0 = A.row_ptr[i], p1 = A.row_ptr[i + 1];
  const EpsBand band = eps_band(eps);
  for (int p = p0 + warp; p < p1; p += nwarps) {
    const int k = A.col_idx[p];
    const double na = A.norms[p];
    const float fa = A.normsf[p];
    int q0 = B.row_ptr[k], q1 = B.row_ptr[k + 1];
    if (!whole) {
      q0 = lower_bound_i32(B.col_idx, q0, q1, w0);
      q1 = lower_bound_i32(B.col_idx, q0, q1, w0 + wn);
    }
    const int64_t ms = (int64_t)m * B.row_sizes[k];
    for (int q = q0 + lane; q < q1; q += 32) {
      const int j = B.col_idx[q];
      if (COUNT) cand++;
      if (keep_fast(fa, B.normsf[q], na, B.norms[q], eps, band)) {
        const int jj = j - w0;
        atomicOr(&bitmap[jj >> 5], 1u << (jj & 31));
        if (COUNT) {
          kept++;
          flops += 2 * ms * B.col_sizes[j];
        }
      }
    }
  }
  if (use_cin) {
    int c0 = Cin.row_ptr[i], c1 = Cin.row_ptr[i + 1];
    if (!whole) {
      c0 = lower_bound_i32(Cin.col_idx, c0, c1, w0);
      c1 = lower_bound_i32(Cin.col_idx, c0, c1, w0 + wn);
    }
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
      const int jj = Cin.col_idx[c] - w0;
      atomicOr(&bitmap[jj >> 5], 1u << (jj & 31));
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// Count pass: one thread block per C block row (grid-stride).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kSymThreads) k_symbolic_count(DevMat A, DevMat B, DevMat Cin,
                                                                int use_cin, double eps,
                                                                DevWs ws) {
  extern __shared__ uint32_t smem_bits[];
  const int nbc = B.nbc;
  const bool whole = nbc <= kWindowCols;
  for (int i = blockIdx.x; i < A.nbr; i += gridDim.x) {
    int64_t cand = 0, kept = 0, flops = 0, colsum = 0, nblk = 0;
    for (int w0 = 0; w0 < nbc; w0 += kWindowCols) {
      const int wn = min(kWindowCols, nbc - w0);
      const int nwords = (wn + 31) >> 5;
      row_bitmap<true>(A, B, Cin, use_cin, eps, i, w0, wn, whole, smem_bits, nwords, cand, kept,
                       flops);
      for (int t = threadIdx.x; t < nwords; t += blockDim.x) {
        uint32_t bits = smem_bits[t];
        nblk += __popc(bits);
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          colsum += B.col_sizes[w0 + 32 * t + b];
        }
      }
      __syncthreads();
    }
    cand = block_sum(cand);
    kept = block_sum(kept);
    flops = block_sum(flops);
    colsum = block_sum(colsum);
    nblk = block_sum(nblk);
    if (threadIdx.x == 0) {
      ws.row_cblk[i] = (int32_t)nblk;
      ws.row_prod[i] = kept;
      ws.row_nnz[i] = (int64_t)A.row_sizes[i] * colsum;
      ws.row_cand[i] = cand;
      ws.row_flops[i] = flops;
    }
  }
}

cudaError_t launch_symbolic_count(DevMat A, DevMat B, DevMat Cin, int use_cin, double eps,
                                  DevWs ws, int grid, cudaStream_t stream) {
  const int nwords = (min(B.nbc, kWindowCols) + 31) / 32;
  const size_t smem = (size_t)max(nwords, 1) * sizeof(uint32_t);
  k_symbolic_count<<<grid, kSymThreads, smem, stream>>>(A, B, Cin, use_cin, eps, ws);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Scan pass: one thread block of 1024 threads. Exclusive sums over block rows,
// totals, capacity check, C's header and the sentinel of the product ranges.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_symbolic_scan(int32_t nbr, DevWs ws, DevOut C,
                                                        DevStatus *st) {
  // rows in tiles of blockDim.x, a row per thread (coalesced loads), the
  // running totals carried from tile to tile
  int64_t tb = 0, tp = 0, tn = 0, sc = 0, sf = 0;
  for (int base = 0; base < nbr; base += blockDim.x) {
    const int r = base + (int)threadIdx.x;
    const bool in = r < nbr;
    const int64_t b = in ? ws.row_cblk[r] : 0, p = in ? ws.row_prod[r] : 0;
    const int64_t n = in ? ws.row_nnz[r] : 0;
    if (in) {
      sc += ws.row_cand[r];
      sf += ws.row_flops[r];
    }
    int64_t sb, sp, sn;
    const int64_t eb = block_exclusive_scan(b, &sb);
    const int64_t ep = block_exclusive_scan(p, &sp);
    const int64_t en = block_exclusive_scan(n, &sn);
    if (in) {
      C.row_ptr[r] = (int32_t)(tb + eb);
      ws.prod_off[r] = tp + ep;
      ws.nnz_off[r] = tn + en;
    }
    tb += sb;
    tp += sp;
    tn += sn;
  }
  const int64_t tc = block_sum(sc);
  const int64_t tf = block_sum(sf);
  if (threadIdx.x == 0) {
    C.row_ptr[nbr] = (int32_t)tb;
    ws.prod_off[nbr] = tp;
    ws.nnz_off[nbr] = tn;
    const int overflow = (tb > C.cap_blk) || (tn > C.cap_nnz) || (tp > ws.cap_prod) ||
                         (tb >= (int64_t)INT32_MAX);
    st->nblk_c = tb;
    st->nnz_c = tn;
    st->nprod = tp;
    st->candidates = tc;
    st->kept = tp;
    st->flops = tf;
    st->overflow = overflow;
    st->error = 0;
    if (!overflow) {
      C.hdr[0] = tb;
      C.hdr[1] = tn;
      ws.prod_ptr[tb] = tp;
    }
  }
}

cudaError_t launch_symbolic_scan(int32_t nbr, DevWs ws, DevOut C, DevStatus *st,
                                 cudaStream_t stream) {
  k_symbolic_scan<<<1, 1024, 0, stream>>>(nbr, ws, C, st);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Fill pass helpers.
// ----------------------------------------------------------------------------
// wpre[t] = number of set bits in bitmap[0..t); returns the total.
__device__ int word_prefix(const uint32_t *bitmap, int32_t *wpre, int nwords) {
  const int per = (nwords + blockDim.x - 1) / blockDim.x;
  const int beg = min(nwords, (int)threadIdx.x * per), end = min(nwords, beg + per);
  int64_t s = 0;
  for (int t = beg; t < end; t++) s += __popc(bitmap[t]);
  int64_t total;
  int64_t run = block_exclusive_scan(s, &total);
  for (int t = beg; t < end; t++) {
    wpre[t] = (int32_t)run;
    run += __popc(bitmap[t]);
  }
  __syncthreads();
  return (int)total;
}

// Words of the per-row (C block x A block) bit matrix of the fill pass, at
// most (the launch may ask for fewer, for more resident blocks).
constexpr int kMaskWords = 8192;

// Rank of column offset jj inside the window among the set bits.
__device__ __forceinline__ int bit_rank(const uint32_t *bitmap, const int32_t *wpre, int jj) {
  return wpre[jj >> 5] + __popc(bitmap[jj >> 5] & ((1u << (jj & 31)) - 1u));
}

// ----------------------------------------------------------------------------
// Fill pass: one thread block per C block row (grid-stride).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kSymThreads) k_symbolic_fill(DevMat A, DevMat B, DevMat Cin,
                                                               int use_cin, double eps, DevWs ws,
                                                               DevOut C, const DevStatus *st,
                                                               int mask_words) {
  if (st->overflow) return;
  extern __shared__ uint32_t smem_bits[];
  const int nbc = B.nbc;
  const bool whole = nbc <= kWindowCols;
  const int nwords_max = (min(nbc, kWindowCols) + 31) >> 5;
  uint32_t *bitmap = smem_bits;
  int32_t *wpre = reinterpret_cast<int32_t *>(smem_bits + nwords_max);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int64_t dummy0 = 0, dummy1 = 0, dummy2 = 0;

  uint32_t *mask = smem_bits + 2 * nwords_max;  // mask_words words, see below
  const EpsBand band = eps_band(eps);

  for (int i = blockIdx.x; i < A.nbr; i += gridDim.x) {
    const int g0 = C.row_ptr[i], g1 = C.row_ptr[i + 1];
    if (g0 == g1) continue;
    const int m = A.row_sizes[i];
    const int p0 = A.row_ptr[i], p1 = A.row_ptr[i + 1];

    // Fast path (one column window, small enough row): a bit matrix in shared
    // memory with one bit per (C block of the row, A block of the row) says
    // which kept products exist; a product's place in its C block's list
    // (ascending k) is then the popcount of the bits before it, so every
    // product is placed at once, without a pass per A block.
    const int wps = (p1 - p0 + 31) >> 5;  // mask words per C block
    if (whole && (int64_t)(g1 - g0) * wps <= mask_words) {
      const int nwords = (nbc + 31) >> 5;
      row_bitmap<false>(A, B, Cin, use_cin, eps, i, 0, nbc, true, bitmap, nwords, dummy0, dummy1,
                        dummy2);
      word_prefix(bitmap, wpre, nwords);
      for (int t = threadIdx.x; t < nwords; t += blockDim.x) {
        uint32_t bits = bitmap[t];
        int g = g0 + wpre[t];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          C.col_idx[g] = 32 * t + b;
          C.blk_row[g] = i;
          ws.c_cin[g] = -1;
          g++;
        }
      }
      for (int t = threadIdx.x; t < (g1 - g0) * wps; t += blockDim.x) mask[t] = 0u;
      __syncthreads();
      for (int p = p0 + warp; p < p1; p += nwarps) {
        const int k = A.col_idx[p];
        const double na = A.norms[p];
        const float fa = A.normsf[p];
        const uint32_t bit = 1u << ((p - p0) & 31);
        const int wofs = (p - p0) >> 5;
        for (int q = B.row_ptr[k] + lane; q < B.row_ptr[k + 1]; q += 32) {
          if (keep_fast(fa, B.normsf[q], na, B.norms[q], eps, band)) {
            const int sl = bit_rank(bitmap, wpre, B.col_idx[q]);
            atomicOr(&mask[sl * wps + wofs], bit);
          }
        }
      }
      if (use_cin) {
        for (int c = Cin.row_ptr[i] + threadIdx.x; c < Cin.row_ptr[i + 1]; c += blockDim.x)
          ws.c_cin[g0 + bit_rank(bitmap, wpre, Cin.col_idx[c])] = c;
      }
      __syncthreads();
      // product ranges and value offsets of the row's C blocks
      int64_t carry_p = ws.prod_off[i], carry_v = ws.nnz_off[i];
      for (int base = g0; base < g1; base += blockDim.x) {
        const int g = base + threadIdx.x;
        const bool in = g < g1;
        int64_t cp = 0;
        if (in)
          for (int w = 0; w < wps; w++) cp += __popc(mask[(g - g0) * wps + w]);
        const int64_t cv = in ? (int64_t)m * C.col_sizes[C.col_idx[g]] : 0;
        int64_t tp, tv;
        const int64_t ep = block_exclusive_scan(cp, &tp);
        const int64_t ev = block_exclusive_scan(cv, &tv);
        if (in) {
          ws.prod_ptr[g] = carry_p + ep;
          C.blk_off[g] = carry_v + ev;
        }
        carry_p += tp;
        carry_v += tv;
      }
      __syncthreads();
      // every kept product straight to its place
      for (int p = p0 + warp; p < p1; p += nwarps) {
        const int k = A.col_idx[p];
        const double na = A.norms[p];
        const float fa = A.normsf[p];
        const int pi = p - p0;
        const uint32_t below = (1u << (pi & 31)) - 1u;
        for (int q = B.row_ptr[k] + lane; q < B.row_ptr[k + 1]; q += 32) {
          if (keep_fast(fa, B.normsf[q], na, B.norms[q], eps, band)) {
            const int sl = bit_rank(bitmap, wpre, B.col_idx[q]);
            const uint32_t *mk = mask + sl * wps;
            int pos = __popc(mk[pi >> 5] & below);
            for (int w = 0; w < (pi >> 5); w++) pos += __popc(mk[w]);
            ws.prods[ws.prod_ptr[g0 + sl] + pos] = make_int2(p, q);
          }
        }
      }
      __syncthreads();
      continue;
    }

    // pass 1: C blocks of the row, per-block product counts, C_in map
    int slot_base = 0;
    for (int w0 = 0; w0 < nbc; w0 += kWindowCols) {
      const int wn = min(kWindowCols, nbc - w0);
      const int nwords = (wn + 31) >> 5;
      row_bitmap<false>(A, B, Cin, use_cin, eps, i, w0, wn, whole, bitmap, nwords, dummy0, dummy1,
                        dummy2);
      const int nw = word_prefix(bitmap, wpre, nwords);
      for (int t = threadIdx.x; t < nwords; t += blockDim.x) {
        uint32_t bits = bitmap[t];
        int g = g0 + slot_base + wpre[t];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          C.col_idx[g] = w0 + 32 * t + b;
          C.blk_row[g] = i;
          ws.cnt[g] = 0;
          ws.c_cin[g] = -1;
          g++;
        }
      }
      __syncthreads();
      for (int p = p0 + warp; p < p1; p += nwarps) {
        const int k = A.col_idx[p];
        const double na = A.norms[p];
        const float fa = A.normsf[p];
        int q0 = B.row_ptr[k], q1 = B.row_ptr[k + 1];
        if (!whole) {
          q0 = lower_bound_i32(B.col_idx, q0, q1, w0);
          q1 = lower_bound_i32(B.col_idx, q0, q1, w0 + wn);
        }
        for (int q = q0 + lane; q < q1; q += 32) {
          if (keep_fast(fa, B.normsf[q], na, B.norms[q], eps, band)) {
            const int g = g0 + slot_base + bit_rank(bitmap, wpre, B.col_idx[q] - w0);
            atomicAdd(&ws.cnt[g], 1);
          }
        }
      }
      if (use_cin) {
        int c0 = Cin.row_ptr[i], c1 = Cin.row_ptr[i + 1];
        if (!whole) {
          c0 = lower_bound_i32(Cin.col_idx, c0, c1, w0);
          c1 = lower_bound_i32(Cin.col_idx, c0, c1, w0 + wn);
        }
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
          const int g = g0 + slot_base + bit_rank(bitmap, wpre, Cin.col_idx[c] - w0);
          ws.c_cin[g] = c;
        }
      }
      __syncthreads();
      slot_base += nw;
    }

    // pass 2: product ranges and value offsets of the row's C blocks
    {
      int64_t carry_p = ws.prod_off[i], carry_v = ws.nnz_off[i];
      for (int base = g0; base < g1; base += blockDim.x) {
        const int g = base + threadIdx.x;
        const bool in = g < g1;
        const int64_t cp = in ? ws.cnt[g] : 0;
        const int64_t cv = in ? (int64_t)m * C.col_sizes[C.col_idx[g]] : 0;
        int64_t tp, tv;
        const int64_t ep = block_exclusive_scan(cp, &tp);
        const int64_t ev = block_exclusive_scan(cv, &tv);
        if (in) {
          ws.prod_ptr[g] = carry_p + ep;
          C.blk_off[g] = carry_v + ev;
          ws.cnt[g] = 0;
        }
        carry_p += tp;
        carry_v += tv;
      }
      __syncthreads();
    }

    // pass 3: kept products grouped by C block, ascending k inside a block
    slot_base = 0;
    for (int w0 = 0; w0 < nbc; w0 += kWindowCols) {
      const int wn = min(kWindowCols, nbc - w0);
      const int nwords = (wn + 31) >> 5;
      int nw;
      if (!whole) {
        row_bitmap<false>(A, B, Cin, use_cin, eps, i, w0, wn, whole, bitmap, nwords, dummy0,
                          dummy1, dummy2);
        nw = word_prefix(bitmap, wpre, nwords);
      } else {
        nw = g1 - g0;
      }
      for (int p = p0; p < p1; p++) {
        const int k = A.col_idx[p];
        const double na = A.norms[p];
        const float fa = A.normsf[p];
        int q0 = B.row_ptr[k], q1 = B.row_ptr[k + 1];
        if (!whole) {
          q0 = lower_bound_i32(B.col_idx, q0, q1, w0);
          q1 = lower_bound_i32(B.col_idx, q0, q1, w0 + wn);
        }
        for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
          if (keep_fast(fa, B.normsf[q], na, B.norms[q], eps, band)) {
            const int g = g0 + slot_base + bit_rank(bitmap, wpre, B.col_idx[q] - w0);
            const int c = ws.cnt[g];
            ws.cnt[g] = c + 1;
            ws.prods[ws.prod_ptr[g] + c] = make_int2(p, q);
          }
        }
        __syncthreads();
      }
      slot_base += nw;
    }
  }
}

cudaError_t launch_symbolic_fill(DevMat A, DevMat B, DevMat Cin, int use_cin, double eps,
                                 DevWs ws, DevOut C, const DevStatus *st, int nsm, int mask_words,
                                 cudaStream_t stream) {
  const int nwords = (min(B.nbc, kWindowCols) + 31) / 32;
  const int mw = (mask_words > 0 && mask_words < kMaskWords) ? mask_words : kMaskWords;
  const size_t smem = ((size_t)max(nwords, 1) * 2 + mw) * sizeof(uint32_t);
  // one wave of resident blocks (rows taken in a grid stride): more resident
  // blocks hide more of each row's load latency, a second wave only adds a tail
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_symbolic_fill,
                                                                kSymThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
  k_symbolic_fill<<<grid, kSymThreads, smem, stream>>>(A, B, Cin, use_cin, eps, ws, C, st, mw);
  return cudaGetLastError();
}

}  // namespace bsm
