// k_split.cu -- the numeric phase in split precision: every block product
// A_ik . B_kj is carried out on the tensor cores as a sum of products of
// low-precision slices of the operands (Ozaki-style multi-term products),
// accumulated in FP32; C is formed in FP64:
//
//     C_ij = beta * C_in_ij + alpha * sum_k sum_{(p,q)} A_ik^(p) . B_kj^(q)
//
//   BF16x3: a = a1 + a2 + a3 (three BF16 slices of 8 significant bits each),
//           the six slice products with p + q <= 4 (1-based) are kept;
//   TF32x2: a = a1 + a2 (two TF32 slices of 11 significant bits),
//           the three products a1 b1, a1 b2, a2 b1 are kept.
//
// The slices are cut by integer operations on the FP64 bit pattern
// (truncation: each slice takes the next BITS significant bits of what the
// previous slices left), so no FP64 arithmetic is spent on splitting; the
// filter and the norms stay in FP64 (k_symbolic.cu).
//
// Slice layout ("fragment order"). An operand block enters an MMA either as
// the left factor (its rows are M rows, its columns the k dimension) or as the
// right factor (its rows the k dimension, its columns N columns). Each layout
// stores, per M row (left) or per N column (right), the k values of that row
// or column padded to kpad(k) and permuted inside every k-step so that one
// lane's fragment registers of a step are one aligned 8-byte (k16 / tf32 k8)
// or 4-byte (bf16 k8 tail) word:
//   BF16: k-steps of 16, and a final step of 8 when at most 8 remain; inside a
//         16-step, lane t's values k = 2t, 2t+1, 2t+8, 2t+9 sit at 4t..4t+3;
//         an 8-step keeps natural order (lane t reads 2t, 2t+1).
//   TF32: k-steps of 8; lane t's values k = t, t+4 sit at 2t, 2t+1.
// Padding is zero, so fragment loads need no predicates on k. Per block the
// layout starts at a fixed multiple of its FP64 offset blk_off[b] (48 bytes per
// value for BF16, 64 for TF32; both bound the padded size), 16-byte aligned.
#include <cstdint>

#include "bsm_internal.h"

namespace bsm {

// Padded k extent.
__host__ __device__ __forceinline__ int kpad_bf16(int k) {
  const int r = k & 15;
  return (k & ~15) + (r == 0 ? 0 : (r <= 8 ? 8 : 16));
}
__host__ __device__ __forceinline__ int kpad_tf32(int k) { return (k + 7) & ~7; }

// The k index stored at position pos (inside the padded extent of k values).
__device__ __forceinline__ int bf16_k_at(int pos, int k) {
  const int base = pos & ~15;
  const int in = pos & 15;
  if (k - base <= 8) return pos;  // the final 8-step: natural order
  const int t = in >> 2, w = in & 3;
  return base + ((w < 2) ? (2 * t + w) : (2 * t + 8 + (w - 2)));
}
__device__ __forceinline__ int tf32_k_at(int pos) {
  const int base = pos & ~7;
  const int in = pos & 7;
  return base + ((in & 1) ? (in >> 1) + 4 : (in >> 1));
}

// ---------------------------------------------------------------------------
// Splitting an FP64 value into slices of BITS significant bits (truncation).
// Zeros and FP64 subnormals give zero slices; inf/NaN go to the first slice.
// ---------------------------------------------------------------------------
template <int NS, int BITS>
struct Slices {
  uint32_t s[NS];  // bf16 in the low 16 bits, or tf32 as FP32 bits
};

template <int NS, int BITS>
__device__ __forceinline__ Slices<NS, BITS> split_value(double x) {
  Slices<NS, BITS> out;
#pragma unroll
  for (int q = 0; q < NS; q++) out.s[q] = 0u;
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return out;
  if (E == 0x7FF) {  // inf / NaN
    const bool nan = (b & 0xFFFFFFFFFFFFFull) != 0;
    out.s[0] = (BITS == 8) ? ((sign << 15) | 0x7F80u | (nan ? 0x40u : 0u))
                           : ((sign << 31) | 0x7F800000u | (nan ? 0x400000u : 0u));
    return out;
  }
  uint64_t rem = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
  const int e = E - 1023;  // value = rem * 2^(e - 52)
#pragma unroll
  for (int q = 0; q < NS; q++) {
    if (rem == 0) break;
    const int p = 63 - __clzll((long long)rem);  // leading one
    uint32_t h;
    uint64_t low;
    if (p >= BITS - 1) {
      h = (uint32_t)(rem >> (p - (BITS - 1)));
      low = rem & ((1ull << (p - (BITS - 1))) - 1ull);
    } else {
      h = (uint32_t)(rem << ((BITS - 1) - p));
      low = 0;
    }
    // slice value = h * 2^(e - 52 + p - (BITS-1)), h has BITS bits, top bit set
    const int ef = e - 52 + p + 127;  // biased exponent of the slice
    if (ef >= 1 && ef <= 254) {
      if (BITS == 8)
        out.s[q] = (sign << 15) | ((uint32_t)ef << 7) | (h & 0x7Fu);
      else
        out.s[q] = (sign << 31) | ((uint32_t)ef << 23) | ((h & 0x3FFu) << 13);
    } else if (ef > 254) {  // beyond the 8-bit exponent range: infinity
      out.s[q] = (BITS == 8) ? ((sign << 15) | 0x7F80u) : ((sign << 31) | 0x7F800000u);
      break;
    }
    rem = low;
  }
  return out;
}

// ---------------------------------------------------------------------------
// Split every block of a matrix into the left and/or right layouts. One warp
// per block (grid-stride), lanes over the padded positions of a layout.
// ---------------------------------------------------------------------------
__global__ void k_split_bf16x3(const int32_t *__restrict__ row_sizes,
                               const int32_t *__restrict__ col_sizes,
                               const int32_t *__restrict__ blk_row,
                               const int32_t *__restrict__ col_idx,
                               const int64_t *__restrict__ blk_off,
                               const double *__restrict__ vals, const int64_t *__restrict__ hdr,
                               uint16_t *__restrict__ left, uint16_t *__restrict__ right) {
  const int lane = threadIdx.x & 31;
  const int64_t nblk = hdr[0];
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = w0; b < nblk; b += nw) {
    const int r = row_sizes[blk_row[b]], c = col_sizes[col_idx[b]];
    const int64_t base = (kBf16BytesPerValue / 2) * blk_off[b];
    const double *x = vals + blk_off[b];
    if (left) {  // r rows of kpad(c), k = column index
      const int kp = kpad_bf16(c);
      const int plane = r * kp;
      for (int e = lane; e < plane; e += 32) {
        const int row = e / kp, pos = e - row * kp;
        const int k = bf16_k_at(pos, c);
        const Slices<3, 8> sl = split_value<3, 8>(k < c ? x[row + (int64_t)k * r] : 0.0);
#pragma unroll
        for (int q = 0; q < 3; q++) left[base + (int64_t)q * plane + e] = (uint16_t)sl.s[q];
      }
    }
    if (right) {  // c columns of kpad(r), k = row index
      const int kp = kpad_bf16(r);
      const int plane = c * kp;
      for (int e = lane; e < plane; e += 32) {
        const int col = e / kp, pos = e - col * kp;
        const int k = bf16_k_at(pos, r);
        const Slices<3, 8> sl = split_value<3, 8>(k < r ? x[k + (int64_t)col * r] : 0.0);
#pragma unroll
        for (int q = 0; q < 3; q++) right[base + (int64_t)q * plane + e] = (uint16_t)sl.s[q];
      }
    }
  }
}

__global__ void k_split_tf32x2(const int32_t *__restrict__ row_sizes,
                               const int32_t *__restrict__ col_sizes,
                               const int32_t *__restrict__ blk_row,
                               const int32_t *__restrict__ col_idx,
                               const int64_t *__restrict__ blk_off,
                               const double *__restrict__ vals, const int64_t *__restrict__ hdr,
                               uint32_t *__restrict__ left, uint32_t *__restrict__ right) {
  const int lane = threadIdx.x & 31;
  const int64_t nblk = hdr[0];
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = w0; b < nblk; b += nw) {
    const int r = row_sizes[blk_row[b]], c = col_sizes[col_idx[b]];
    const int64_t base = (kTf32BytesPerValue / 4) * blk_off[b];
    const double *x = vals + blk_off[b];
    if (left) {
      const int kp = kpad_tf32(c);
      const int plane = r * kp;
      for (int e = lane; e < plane; e += 32) {
        const int row = e / kp, pos = e - row * kp;
        const int k = tf32_k_at(pos);
        const Slices<2, 11> sl = split_value<2, 11>(k < c ? x[row + (int64_t)k * r] : 0.0);
#pragma unroll
        for (int q = 0; q < 2; q++) left[base + (int64_t)q * plane + e] = sl.s[q];
      }
    }
    if (right) {
      const int kp = kpad_tf32(r);
      const int plane = c * kp;
      for (int e = lane; e < plane; e += 32) {
        const int col = e / kp, pos = e - col * kp;
        const int k = tf32_k_at(pos);
        const Slices<2, 11> sl = split_value<2, 11>(k < r ? x[k + (int64_t)col * r] : 0.0);
#pragma unroll
        for (int q = 0; q < 2; q++) right[base + (int64_t)q * plane + e] = sl.s[q];
      }
    }
  }
}

cudaError_t launch_split(int precision, const int32_t *row_sizes, const int32_t *col_sizes,
                         const int32_t *blk_row, const int32_t *col_idx, const int64_t *blk_off,
                         const double *vals, const int64_t *hdr, void *left, void *right,
                         int grid, cudaStream_t stream) {
  if (precision == BSM_PREC_SPLIT_BF16X3)
    k_split_bf16x3<<<grid, 256, 0, stream>>>(row_sizes, col_sizes, blk_row, col_idx, blk_off, vals,
                                             hdr, (uint16_t *)left, (uint16_t *)right);
  else
    k_split_tf32x2<<<grid, 256, 0, stream>>>(row_sizes, col_sizes, blk_row, col_idx, blk_off, vals,
                                             hdr, (uint32_t *)left, (uint32_t *)right);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tensor-core fragments (mma.sync, FP32 accumulation).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                             uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_tf32_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                            uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Exact FP32 -> FP64 conversion with integer operations only.
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t ef = (u >> 23) & 0xFFu;
  const uint64_t man = u & 0x7FFFFFu;
  uint64_t bits;
  if (ef == 0) {
    if (man == 0) {
      bits = sign;
    } else {  // FP32 subnormal: man * 2^-149, normal in FP64
      const int p = 63 - __clzll((long long)man);
      bits = sign | ((uint64_t)(p - 149 + 1023) << 52) | ((man << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
  } else if (ef == 0xFF) {
    bits = sign | (0x7FFull << 52) | (man << 29);
  } else {
    bits = sign | ((uint64_t)(ef + 896) << 52) | (man << 29);
  }
  return __longlong_as_double((long long)bits);
}

// hi + lo += x, exactly (Knuth's TwoSum in FP32, no fused operations).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ---------------------------------------------------------------------------
// Loads of fragment words. `Sh` selects shared (32-bit addresses) or global.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.b32 {%0,%1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}

// One k-step of all slice products of a warp's MT x NT tiles.
//   L: left operand base (rows of the MMA problem, stride lstride bytes),
//   R: right operand base (columns, stride rstride bytes), plane strides in
//   bytes, kk: position of the step, k8: an 8-wide BF16 tail step. Rows /
//   columns past Mp / Np read nothing and use zero fragments.
template <int PREC, int MT, int NT, bool SH>
__device__ __forceinline__ void split_step(float (&acc)[MT][NT][4], const unsigned char *Lg,
                                           const unsigned char *Rg, uint32_t Ls, uint32_t Rs,
                                           int lstride, int rstride, int lplane, int rplane,
                                           int kk, bool k8, int Mp, int Np) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  constexpr bool BF = (PREC == BSM_PREC_SPLIT_BF16X3);
  constexpr int NSL = BF ? 3 : 2;
  constexpr int ES = BF ? 2 : 4;  // bytes per element
  // byte offset of lane's word inside a row / column of the step
  const int wofs = BF ? (k8 ? (kk + 2 * t) * ES : (kk + 4 * t) * ES) : (kk + 2 * t) * ES;
  uint32_t a[NSL][MT][4], b[NSL][NT][2];
#pragma unroll
  for (int q = 0; q < NSL; q++) {
#pragma unroll
    for (int mt = 0; mt < MT; mt++) {
      const int r0 = mt * 16 + g, r1 = r0 + 8;
      const int o0 = q * lplane + r0 * lstride + wofs, o1 = q * lplane + r1 * lstride + wofs;
      uint2 v0 = make_uint2(0u, 0u), v1 = make_uint2(0u, 0u);
      if (BF && k8) {
        if (r0 < Mp) v0.x = SH ? lds32(Ls + o0) : __ldg(reinterpret_cast<const uint32_t *>(Lg + o0));
        if (r1 < Mp) v1.x = SH ? lds32(Ls + o1) : __ldg(reinterpret_cast<const uint32_t *>(Lg + o1));
      } else {
        if (r0 < Mp) v0 = SH ? lds64(Ls + o0) : __ldg(reinterpret_cast<const uint2 *>(Lg + o0));
        if (r1 < Mp) v1 = SH ? lds64(Ls + o1) : __ldg(reinterpret_cast<const uint2 *>(Lg + o1));
      }
      // bf16 k16: {k 2t..2t+1, k 2t+8..2t+9}; tf32: {k t, k t+4}
      a[q][mt][0] = v0.x;
      a[q][mt][1] = v1.x;
      a[q][mt][2] = v0.y;
      a[q][mt][3] = v1.y;
    }
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
      const int c = nt * 8 + g;
      const int o = q * rplane + c * rstride + wofs;
      uint2 v = make_uint2(0u, 0u);
      if (c < Np) {
        if (BF && k8)
          v.x = SH ? lds32(Rs + o) : __ldg(reinterpret_cast<const uint32_t *>(Rg + o));
        else
          v = SH ? lds64(Rs + o) : __ldg(reinterpret_cast<const uint2 *>(Rg + o));
      }
      b[q][nt][0] = v.x;
      b[q][nt][1] = v.y;
    }
  }
  if (BF) {
    // slice products, smallest first: (3,1) (2,2) (1,3) (2,1) (1,2) (1,1)
    constexpr int PA[6] = {2, 1, 0, 1, 0, 0};
    constexpr int PB[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        if (mt * 16 >= Mp || nt * 8 >= Np) continue;
#pragma unroll
        for (int pq = 0; pq < 6; pq++) {
          const uint32_t *aa = a[PA[pq]][mt];
          if (k8)
            mma_bf16_k8(acc[mt][nt], aa[0], aa[1], b[PB[pq]][nt][0]);
          else
            mma_bf16_k16(acc[mt][nt], aa[0], aa[1], aa[2], aa[3], b[PB[pq]][nt][0],
                         b[PB[pq]][nt][1]);
        }
      }
  } else {
    // (2,1) (1,2) (1,1)
    constexpr int PA[3] = {1, 0, 0};
    constexpr int PB[3] = {0, 1, 0};
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        if (mt * 16 >= Mp || nt * 8 >= Np) continue;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
          const uint32_t *aa = a[PA[pq]][mt];
          mma_tf32_k8(acc[mt][nt], aa[0], aa[1], aa[2], aa[3], b[PB[pq]][nt][0],
                      b[PB[pq]][nt][1]);
        }
      }
  }
}

// The geometry of one product's operands in the layouts: byte size of a layout
// block with `rows` rows (or columns) and k values, its row stride, plane size.
template <int PREC>
__device__ __forceinline__ void layout_dims(int rows, int k, int &stride, int &plane) {
  if (PREC == BSM_PREC_SPLIT_BF16X3) {
    stride = 2 * kpad_bf16(k);
    plane = rows * stride;
  } else {
    stride = 4 * kpad_tf32(k);
    plane = rows * stride;
  }
}

template <int PREC>
__device__ __forceinline__ void run_steps_prologue(int s, int &nsteps) {
  nsteps = (PREC == BSM_PREC_SPLIT_BF16X3) ? (kpad_bf16(s) + 15) / 16 : kpad_tf32(s) / 8;
}

// Position of step st of a product with k = s: (kk, k8).
template <int PREC>
__device__ __forceinline__ void step_pos(int st, int s, int &kk, bool &k8) {
  if (PREC == BSM_PREC_SPLIT_BF16X3) {
    kk = 16 * st;
    k8 = (s - kk) <= 8;
  } else {
    kk = 8 * st;
    k8 = false;
  }
}

// Epilogue of a C block: C_ij = beta * C_in_ij + alpha * (hi + lo) in FP64 (an
// exact copy of hi + lo when alpha = 1 and beta = 0).
template <int MT, int NT>
__device__ __forceinline__ void split_epilogue(const float (&hi)[MT][NT][4],
                                               const float (&lo)[MT][NT][4], double alpha,
                                               double beta, const double *cinv, double *out,
                                               int m, bool tr, int Mp, int Np) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const bool plain = (alpha == 1.0 && beta == 0.0);
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int rr = mt * 16 + g + ((x >> 1) << 3);
        const int cc = nt * 8 + 2 * t + (x & 1);
        if (rr < Mp && cc < Np) {
          const int row = tr ? cc : rr, col = tr ? rr : cc;
          const int64_t e = (int64_t)col * m + row;
          double v = f32_to_f64_exact(hi[mt][nt][x]) + f32_to_f64_exact(lo[mt][nt][x]);
          if (!plain) {
            v = alpha * v;
            if (cinv) v = fma(beta, cinv[e], v);
          }
          out[e] = v;
        }
      }
}

// The MMA problem of C block (m x n): the block or its transpose, whichever
// needs fewer 16 x 8 tiles.
__device__ __forceinline__ void mma_problem(int m, int n, bool &tr, int &Mp, int &Np) {
  const int tiles_n = ((m + 15) >> 4) * ((n + 7) >> 3);
  const int tiles_t = ((n + 15) >> 4) * ((m + 7) >> 3);
  tr = tiles_t < tiles_n;
  Mp = tr ? n : m;
  Np = tr ? m : n;
}

// ---------------------------------------------------------------------------
// Large blocks (an MMA problem beyond 16 x 16, up to 32 x 32): fragments
// straight from global memory, 2 x 4 tiles.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(128) k_numeric_split_large(DevMat A, DevMat B, DevOut C,
                                                             DevMat Cin,
                                                             const void *__restrict__ a_left,
                                                             const void *__restrict__ b_right,
                                                             double alpha, double beta, DevWs ws,
                                                             const DevStatus *st,
                                                             const int32_t *__restrict__ items,
                                                             const int64_t *__restrict__ seg) {
  if (st->overflow) return;
  constexpr int BPV = (PREC == BSM_PREC_SPLIT_BF16X3) ? kBf16BytesPerValue : kTf32BytesPerValue;
  int64_t wb = 0, we = st->nblk_c;
  if (seg) {
    wb = seg[0];
    we = seg[1];
  }
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = wb + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); w < we;
       w += nwarp) {
    const int64_t gb = items ? items[w] : w;
    const int i = C.blk_row[gb], j = C.col_idx[gb];
    const int m = C.row_sizes[i], n = C.col_sizes[j];
    bool tr;
    int Mp, Np;
    mma_problem(m, n, tr, Mp, Np);
    if (Mp <= 16 && Np <= 16) continue;  // the pipelined kernel takes these
    float hi[2][4][4], lo[2][4][4], acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
      for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int x = 0; x < 4; x++) hi[mt][nt][x] = lo[mt][nt][x] = acc[mt][nt][x] = 0.f;
    const int64_t p0 = ws.prod_ptr[gb], p1 = ws.prod_ptr[gb + 1];
    for (int64_t p = p0; p < p1; p++) {
      const int2 pr = ws.prods[p];
      const int s = A.col_sizes[A.col_idx[pr.x]];
      const unsigned char *Al = static_cast<const unsigned char *>(a_left) + BPV * A.blk_off[pr.x];
      const unsigned char *Br = static_cast<const unsigned char *>(b_right) + BPV * B.blk_off[pr.y];
      int str, apl, bpl;
      layout_dims<PREC>(m, s, str, apl);
      layout_dims<PREC>(n, s, str, bpl);
      const unsigned char *Lg = tr ? Br : Al, *Rg = tr ? Al : Br;
      const int lplane = tr ? bpl : apl, rplane = tr ? apl : bpl;
      int nsteps;
      run_steps_prologue<PREC>(s, nsteps);
      for (int stp = 0; stp < nsteps; stp++) {
        int kk;
        bool k8;
        step_pos<PREC>(stp, s, kk, k8);
        split_step<PREC, 2, 4, false>(acc, Lg, Rg, 0u, 0u, str, str, lplane, rplane, kk, k8, Mp,
                                      Np);
      }
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
          for (int x = 0; x < 4; x++) {
            two_sum_acc(hi[mt][nt][x], lo[mt][nt][x], acc[mt][nt][x]);
            acc[mt][nt][x] = 0.f;
          }
    }
    const int cin = ws.c_cin[gb];
    split_epilogue<2, 4>(hi, lo, alpha, beta, (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr,
                         C.vals + C.blk_off[gb], m, tr, Mp, Np);
  }
}

// ---------------------------------------------------------------------------
// Blocks whose MMA problem fits 16 x 16 (the water and small-block case). Each
// warp streams the layouts of its C block's products through a ring of
// kStages shared-memory slots with 16-byte asynchronous copies (cp.async),
// kStages - 1 products ahead of the tensor-core work. The (A offset, B offset,
// k) of the products are read 32 at a time into a per-warp table in shared
// memory. The FP32 partial sum is folded into the compensated running sum
// every kFold products.
// ---------------------------------------------------------------------------
constexpr int kStages = 4;
constexpr int kPipeWarps = 4;
constexpr int kMetaEntries = 64;
constexpr int kMetaBytes = kMetaEntries * (8 + 8 + 4);
constexpr int kFold = 4;

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gptr) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bytes of one operand slot: 16 rows (or columns) of the padded largest k.
__host__ __device__ __forceinline__ int pipe_operand_bytes(int precision, int smax) {
  return precision == BSM_PREC_SPLIT_BF16X3 ? 3 * 16 * 2 * kpad_bf16(smax)
                                            : 2 * 16 * 4 * kpad_tf32(smax);
}
__host__ __device__ __forceinline__ int pipe_warp_bytes(int precision, int smax) {
  return kStages * 2 * pipe_operand_bytes(precision, smax) + kMetaBytes;
}

template <int PREC>
__global__ void __launch_bounds__(kPipeWarps * 32)
    k_numeric_split_pipe(DevMat A, DevMat B, DevOut C, DevMat Cin, const void *__restrict__ a_left,
                         const void *__restrict__ b_right, double alpha, double beta, DevWs ws,
                         const DevStatus *st, const int32_t *__restrict__ items,
                         const int64_t *__restrict__ seg, int smax, int only_small) {
  if (st->overflow) return;
  constexpr int BPV = (PREC == BSM_PREC_SPLIT_BF16X3) ? kBf16BytesPerValue : kTf32BytesPerValue;
  extern __shared__ __align__(16) unsigned char smem_pipe[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int opb = pipe_operand_bytes(PREC, smax);
  unsigned char *wbase = smem_pipe + warp * pipe_warp_bytes(PREC, smax);
  int64_t *meta_a = reinterpret_cast<int64_t *>(wbase + kStages * 2 * opb);
  int64_t *meta_b = meta_a + kMetaEntries;
  int *meta_s = reinterpret_cast<int *>(meta_b + kMetaEntries);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(wbase);

  int64_t wb = 0, we = st->nblk_c;
  if (seg) {
    wb = seg[0];
    we = seg[1];
  }
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = wb + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); w < we;
       w += nwarp) {
    const int64_t gb = items ? items[w] : w;
    const int i = C.blk_row[gb], j = C.col_idx[gb];
    const int m = C.row_sizes[i], n = C.col_sizes[j];
    bool tr;
    int Mp, Np;
    mma_problem(m, n, tr, Mp, Np);
    if (only_small && !(Mp <= 16 && Np <= 16)) continue;
    const int64_t p0 = ws.prod_ptr[gb];
    const int np = (int)(ws.prod_ptr[gb + 1] - p0);

    float hi[1][2][4], lo[1][2][4], acc[1][2][4];
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
      for (int x = 0; x < 4; x++) hi[0][nt][x] = lo[0][nt][x] = acc[0][nt][x] = 0.f;

    // copies of product q into slot q % kStages; always commits one group
    auto issue = [&](int q) {
      if (q < np) {
        if ((q & 31) == 0) {  // the next 32 products' offsets and k
          const int qq = q + lane;
          if (qq < np) {
            const int2 pr = ws.prods[p0 + qq];
            meta_a[qq & (kMetaEntries - 1)] = A.blk_off[pr.x];
            meta_b[qq & (kMetaEntries - 1)] = B.blk_off[pr.y];
            meta_s[qq & (kMetaEntries - 1)] = A.col_sizes[A.col_idx[pr.x]];
          }
          __syncwarp();
        }
        const int s = meta_s[q & (kMetaEntries - 1)];
        int str, apl, bpl;
        layout_dims<PREC>(m, s, str, apl);
        layout_dims<PREC>(n, s, str, bpl);
        const unsigned char *srcA =
            static_cast<const unsigned char *>(a_left) + BPV * meta_a[q & (kMetaEntries - 1)];
        const unsigned char *srcB =
            static_cast<const unsigned char *>(b_right) + BPV * meta_b[q & (kMetaEntries - 1)];
        const int bytesA = ((PREC == BSM_PREC_SPLIT_BF16X3) ? 3 : 2) * apl;
        const int bytesB = ((PREC == BSM_PREC_SPLIT_BF16X3) ? 3 : 2) * bpl;
        const uint32_t dst = sbase + (uint32_t)((q % kStages) * 2 * opb);
        for (int c = lane; c < (bytesA + 15) >> 4; c += 32) cp_async16(dst + 16 * c, srcA + 16 * c);
        for (int c = lane; c < (bytesB + 15) >> 4; c += 32)
          cp_async16(dst + opb + 16 * c, srcB + 16 * c);
      }
      cp_async_commit();
    };

#pragma unroll
    for (int q = 0; q < kStages - 1; q++) issue(q);
    for (int q = 0; q < np; q++) {
      cp_async_wait<kStages - 2>();
      __syncwarp();
      issue(q + kStages - 1);  // into the slot consumed by the previous product
      const int s = meta_s[q & (kMetaEntries - 1)];
      int str, apl, bpl;
      layout_dims<PREC>(m, s, str, apl);
      layout_dims<PREC>(n, s, str, bpl);
      const uint32_t sA = sbase + (uint32_t)((q % kStages) * 2 * opb), sB = sA + opb;
      const uint32_t sL = tr ? sB : sA, sR = tr ? sA : sB;
      const int lplane = tr ? bpl : apl, rplane = tr ? apl : bpl;
      int nsteps;
      run_steps_prologue<PREC>(s, nsteps);
      for (int stp = 0; stp < nsteps; stp++) {
        int kk;
        bool k8;
        step_pos<PREC>(stp, s, kk, k8);
        split_step<PREC, 1, 2, true>(acc, nullptr, nullptr, sL, sR, str, str, lplane, rplane, kk,
                                     k8, Mp, Np);
      }
      if ((q % kFold) == kFold - 1 || q == np - 1) {
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
          for (int x = 0; x < 4; x++) {
            two_sum_acc(hi[0][nt][x], lo[0][nt][x], acc[0][nt][x]);
            acc[0][nt][x] = 0.f;
          }
      }
    }
    cp_async_wait<0>();
    __syncwarp();
    const int cin = ws.c_cin[gb];
    split_epilogue<1, 2>(hi, lo, alpha, beta, (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr,
                         C.vals + C.blk_off[gb], m, tr, Mp, Np);
  }
}

cudaError_t launch_numeric_split(int precision, int sizes, DevMat A, DevMat B, DevOut C,
                                 DevMat Cin, const void *a_left, const void *b_right, double alpha,
                                 double beta, DevWs ws, const DevStatus *st, const int32_t *items,
                                 const int64_t *seg, int smax, int nsm, cudaStream_t stream) {
  if (sizes == 2) {  // blocks beyond 16 x 16
    const int grid = nsm * 2;
    if (precision == BSM_PREC_SPLIT_BF16X3)
      k_numeric_split_large<BSM_PREC_SPLIT_BF16X3><<<grid, 128, 0, stream>>>(
          A, B, C, Cin, a_left, b_right, alpha, beta, ws, st, items, seg);
    else
      k_numeric_split_large<BSM_PREC_SPLIT_TF32X2><<<grid, 128, 0, stream>>>(
          A, B, C, Cin, a_left, b_right, alpha, beta, ws, st, items, seg);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)kPipeWarps * pipe_warp_bytes(precision, smax);
  int per_sm = 1;
  cudaError_t e;
  if (precision == BSM_PREC_SPLIT_BF16X3)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_numeric_split_pipe<BSM_PREC_SPLIT_BF16X3>, kPipeWarps * 32, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_numeric_split_pipe<BSM_PREC_SPLIT_TF32X2>, kPipeWarps * 32, smem);
  if (e != cudaSuccess) return e;
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (precision == BSM_PREC_SPLIT_BF16X3)
    k_numeric_split_pipe<BSM_PREC_SPLIT_BF16X3><<<grid, kPipeWarps * 32, smem, stream>>>(
        A, B, C, Cin, a_left, b_right, alpha, beta, ws, st, items, seg, smax, sizes == 1);
  else
    k_numeric_split_pipe<BSM_PREC_SPLIT_TF32X2><<<grid, kPipeWarps * 32, smem, stream>>>(
        A, B, C, Cin, a_left, b_right, alpha, beta, ws, st, items, seg, smax, sizes == 1);
  return cudaGetLastError();
}

cudaError_t numeric_split_init() {
  // the largest slot layout: k up to 32
  const int bf = kPipeWarps * pipe_warp_bytes(BSM_PREC_SPLIT_BF16X3, 32);
  const int tf = kPipeWarps * pipe_warp_bytes(BSM_PREC_SPLIT_TF32X2, 32);
  cudaError_t e = cudaFuncSetAttribute(k_numeric_split_pipe<BSM_PREC_SPLIT_BF16X3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bf);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_numeric_split_pipe<BSM_PREC_SPLIT_TF32X2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, tf);
}

}  // namespace bsm
