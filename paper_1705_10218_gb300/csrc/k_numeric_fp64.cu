// k_numeric_fp64.cu -- the numeric phase in FP64: every C block accumulates
// its kept block products A_ik . B_kj (grouped and ordered by the symbolic
// phase, ascending k) in registers and is written once:
//
//     C_ij = beta * C_in_ij + alpha * sum_k A_ik . B_kj      (Sec. 2, Alg. 1)
//
// One warp owns one C block at a time and writes it once; no atomics. Two
// kernel families:
//   t16: 16 x 16 output tiles and k-chunks of 16; the operands of a (product,
//        chunk) step are copied to shared memory in their own layout (a
//        contiguous copy when a block fits one tile), and the next step's
//        operands are already in flight in registers while the current one is
//        multiplied. The (A offset, B offset, k) of up to 32 products are read
//        at once, one per lane, and handed out with warp shuffles. Compiled for
//        2 or 3 thread blocks of 8 warps per SM.
//   t32: 32 x 32 output tiles, synchronous staging, 4 warps per block.
// Both take an optional work list (C block indices, e.g. one shape class) and
// its [begin, end) range in device memory.
#include <cstdlib>

#include "bsm_internal.h"

namespace bsm {

// ----------------------------------------------------------------------------
// t32
// ----------------------------------------------------------------------------
constexpr int kNumWarps = 4;       // warps per thread block
constexpr int kLdA = kTile;        // sA[l * kLdA + r]
constexpr int kLdB = kTile + 1;    // sB[c * kLdB + l]
constexpr int kWarpSmem = kTile * kLdA + kTile * kLdB;  // doubles per warp

__device__ __forceinline__ void work_range(const DevStatus *st, const int64_t *seg, int64_t &b,
                                           int64_t &e) {
  if (seg) {
    b = seg[0];
    e = seg[1];
  } else {
    b = 0;
    e = st->nblk_c;
  }
}

__global__ void __launch_bounds__(kNumWarps * 32)
    k_numeric_fp64_t32(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha, double beta,
                       DevWs ws, const DevStatus *st, const int32_t *items, const int64_t *seg) {
  if (st->overflow) return;
  extern __shared__ double smem_num[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *sA = smem_num + warp * kWarpSmem;
  double *sB = sA + kTile * kLdA;
  int64_t wb, we;
  work_range(st, seg, wb, we);
  const int64_t nwarp = (int64_t)gridDim.x * kNumWarps;

  for (int64_t w = wb + (int64_t)blockIdx.x * kNumWarps + warp; w < we; w += nwarp) {
    const int64_t g = items ? items[w] : w;
    const int i = C.blk_row[g], j = C.col_idx[g];
    const int m = C.row_sizes[i], n = C.col_sizes[j];
    const int64_t p0 = ws.prod_ptr[g], p1 = ws.prod_ptr[g + 1];
    const int cin = ws.c_cin[g];
    const int64_t coff = C.blk_off[g];
    const double *cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;

    for (int r0 = 0; r0 < m; r0 += kTile) {
      for (int c0 = 0; c0 < n; c0 += kTile) {
        const int tm = min(kTile, m - r0), tn = min(kTile, n - c0);
        const int te = tm * tn;
        const int nT = (te + 31) >> 5;
        double acc[32];
        int ar[32], bc[32];
#pragma unroll
        for (int t = 0; t < 32; t++) {
          acc[t] = 0.0;
          const int e = lane + 32 * t;
          // lanes past the tile read a valid dummy element; their sums are discarded
          ar[t] = (e < te) ? e % tm : 0;
          bc[t] = (e < te) ? (e / tm) * kLdB : 0;
        }
        for (int64_t p = p0; p < p1; p++) {
          const int2 pr = ws.prods[p];
          const int k = A.col_idx[pr.x];
          const int s = A.col_sizes[k];
          const double *Ab = A.vals + A.blk_off[pr.x];  // m x s, column-major
          const double *Bb = B.vals + B.blk_off[pr.y];  // s x n, column-major
          for (int l0 = 0; l0 < s; l0 += kTile) {
            const int kc = min(kTile, s - l0);
            __syncwarp();
            for (int e = lane; e < tm * kc; e += 32) {
              const int r = e % tm, l = e / tm;
              sA[l * kLdA + r] = __ldg(Ab + (int64_t)(l0 + l) * m + r0 + r);
            }
            for (int e = lane; e < kc * tn; e += 32) {
              const int l = e % kc, c = e / kc;
              sB[c * kLdB + l] = __ldg(Bb + (int64_t)(c0 + c) * s + l0 + l);
            }
            __syncwarp();
            for (int l = 0; l < kc; l++) {
#pragma unroll
              for (int t = 0; t < 32; t++) {
                if (t >= nT) break;
                acc[t] = fma(sA[l * kLdA + ar[t]], sB[bc[t] + l], acc[t]);
              }
            }
          }
        }
        // epilogue: C_ij = beta * C_in_ij + alpha * S_ij, written once
#pragma unroll
        for (int t = 0; t < 32; t++) {
          if (t >= nT) break;
          const int e = lane + 32 * t;
          if (e < te) {
            const int r = e % tm, c = e / tm;
            const int64_t loc = (int64_t)(c0 + c) * m + r0 + r;
            double v = alpha * acc[t];
            if (cinv) v = fma(beta, cinv[loc], v);
            C.vals[coff + loc] = v;
          }
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------
// t16
// ----------------------------------------------------------------------------
constexpr int kS = 16;                 // output tile edge and k-chunk
constexpr int kSWarps = 8;             // warps per thread block
constexpr int kSElems = kS * kS / 32;  // operand elements per lane (8)

// Loads the A chunk (tm x kc, rows r0.., columns l0.. of the m x s block) and
// the B chunk (kc x tn, rows l0.., columns c0.. of the s x n block) of one
// step into registers, lane-strided in the chunks' own column-major order.
__device__ __forceinline__ void t16_load(const double *__restrict__ Ab,
                                         const double *__restrict__ Bb, int m, int s, int r0,
                                         int c0, int l0, int tm, int tn, int kc, int lane,
                                         double (&ra)[kSElems], double (&rb)[kSElems]) {
  const bool a_contig = (tm == m);  // whole columns of A: one contiguous range
  const bool b_contig = (kc == s);  // whole columns of B
#pragma unroll
  for (int u = 0; u < kSElems; u++) {
    const int e = lane + 32 * u;
    double va = 0.0, vb = 0.0;
    if (e < tm * kc) {
      const int64_t ia =
          a_contig ? (int64_t)l0 * m + e : (int64_t)(l0 + e / tm) * m + r0 + e % tm;
      va = __ldg(Ab + ia);
    }
    if (e < kc * tn) {
      const int64_t ib =
          b_contig ? (int64_t)c0 * s + e : (int64_t)(c0 + e / kc) * s + l0 + e % kc;
      vb = __ldg(Bb + ib);
    }
    ra[u] = va;
    rb[u] = vb;
  }
}

template <int MINB>
__global__ void __launch_bounds__(kSWarps * 32, MINB)
    k_numeric_fp64_t16(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha, double beta,
                       DevWs ws, const DevStatus *st, const int32_t *items, const int64_t *seg) {
  if (st->overflow) return;
  __shared__ double smem_t16[kSWarps][2 * kS * kS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *sA = smem_t16[warp];
  double *sB = sA + kS * kS;
  int64_t wb, we;
  work_range(st, seg, wb, we);
  const int64_t nwarp = (int64_t)gridDim.x * kSWarps;

  for (int64_t w = wb + (int64_t)blockIdx.x * kSWarps + warp; w < we; w += nwarp) {
    const int64_t g = items ? items[w] : w;
    const int i = C.blk_row[g], j = C.col_idx[g];
    const int m = C.row_sizes[i], n = C.col_sizes[j];
    const int64_t p0 = ws.prod_ptr[g], p1 = ws.prod_ptr[g + 1];
    const int cin = ws.c_cin[g];
    const double *cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;
    double *out = C.vals + C.blk_off[g];

    for (int r0 = 0; r0 < m; r0 += kS) {
      for (int c0 = 0; c0 < n; c0 += kS) {
        const int tm = min(kS, m - r0), tn = min(kS, n - c0);
        const int te = tm * tn;
        const int nT = (te + 31) >> 5;
        int rc[kSElems];  // (row, col) in the tile of the lane's t-th output, r | c << 8
        double acc[kSElems];
#pragma unroll
        for (int t = 0; t < kSElems; t++) {
          const int e = lane + 32 * t;
          rc[t] = (e < te) ? (e % tm) | ((e / tm) << 8) : 0;  // past the tile: a valid dummy
          acc[t] = 0.0;
        }
        for (int64_t pb = p0; pb < p1; pb += 32) {
          const int nb = (p1 - pb < 32) ? (int)(p1 - pb) : 32;
          int64_t my_a = 0, my_b = 0;
          int my_s = 1;
          if (lane < nb) {
            const int2 pr = ws.prods[pb + lane];
            my_a = A.blk_off[pr.x];
            my_b = B.blk_off[pr.y];
            my_s = A.col_sizes[A.col_idx[pr.x]];
          }
          double ra[kSElems], rb[kSElems];
          int q = 0, l0 = 0;
          int s = __shfl_sync(0xffffffffu, my_s, 0);
          t16_load(A.vals + __shfl_sync(0xffffffffu, my_a, 0),
                   B.vals + __shfl_sync(0xffffffffu, my_b, 0), m, s, r0, c0, 0, tm, tn,
                   min(kS, s), lane, ra, rb);
          while (q < nb) {
            __syncwarp();
#pragma unroll
            for (int u = 0; u < kSElems; u++) {
              sA[lane + 32 * u] = ra[u];
              sB[lane + 32 * u] = rb[u];
            }
            __syncwarp();
            const int kc = min(kS, s - l0);
            // the next step: the next k-chunk of this product, or the next product
            int nq = q, nl0 = l0 + kS;
            if (nl0 >= s) {
              nq = q + 1;
              nl0 = 0;
            }
            // warp-uniform: every lane evaluates the same (nq, nl0)
            const int ns = __shfl_sync(0xffffffffu, my_s, nq < nb ? nq : 0);
            const int64_t na = __shfl_sync(0xffffffffu, my_a, nq < nb ? nq : 0);
            const int64_t nbo = __shfl_sync(0xffffffffu, my_b, nq < nb ? nq : 0);
            if (nq < nb)
              t16_load(A.vals + na, B.vals + nbo, m, ns, r0, c0, nl0, tm, tn, min(kS, ns - nl0),
                       lane, ra, rb);
            for (int l = 0; l < kc; l++) {
#pragma unroll
              for (int t = 0; t < kSElems; t++) {
                if (t >= nT) break;
                acc[t] = fma(sA[(rc[t] & 255) + l * tm], sB[(rc[t] >> 8) * kc + l], acc[t]);
              }
            }
            q = nq;
            l0 = nl0;
            s = ns;
          }
        }
        // epilogue: C_ij = beta * C_in_ij + alpha * S_ij
#pragma unroll
        for (int t = 0; t < kSElems; t++) {
          const int e = lane + 32 * t;
          if (t < nT && e < te) {
            const int64_t loc = (int64_t)(c0 + (rc[t] >> 8)) * m + r0 + (rc[t] & 255);
            double v = alpha * acc[t];
            if (cinv) v = fma(beta, cinv[loc], v);
            out[loc] = v;
          }
        }
      }
    }
  }
}

cudaError_t launch_numeric_fp64(int variant, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                double alpha, double beta, DevWs ws, const DevStatus *st,
                                const int32_t *items, const int64_t *seg, int grid,
                                cudaStream_t stream) {
  switch (variant) {
    case kFp64T16B3:
      k_numeric_fp64_t16<3><<<grid, kSWarps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st,
                                                               items, seg);
      break;
    case kFp64T32: {
      // the shared-memory attribute is set once per device by numeric_fp64_init
      const size_t smem = (size_t)kNumWarps * kWarpSmem * sizeof(double);
      k_numeric_fp64_t32<<<grid, kNumWarps * 32, smem, stream>>>(A, B, C, Cin, alpha, beta, ws,
                                                                 st, items, seg);
      break;
    }
    default:
      k_numeric_fp64_t16<2><<<grid, kSWarps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st,
                                                               items, seg);
  }
  return cudaGetLastError();
}

int fp64_variant_blocks_per_sm(int variant) { return variant == kFp64T16B2 ? 2 : 3; }

cudaError_t numeric_fp64_init() {
  const size_t smem = (size_t)kNumWarps * kWarpSmem * sizeof(double);
  return cudaFuncSetAttribute(k_numeric_fp64_t32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

}  // namespace bsm
