// k_numeric_fp64.cu -- the numeric phase in FP64: every C block accumulates
// its kept block products A_ik . B_kj (grouped and ordered by the symbolic
// phase, ascending k) in registers and is written once:
//
//     C_ij = beta * C_in_ij + alpha * sum_k A_ik . B_kj      (Sec. 2, Alg. 1)
//
// One warp owns one C block at a time; tiles of up to 32 x 32 outputs live in
// registers (lane l owns outputs l, l+32, ... in column-major tile order), and
// each product is staged through the warp's shared-memory slice in chunks of
// up to 32 along k. No atomics: a C block is written by exactly one warp.
#include <cstdlib>

#include "bsm_internal.h"

namespace bsm {

constexpr int kNumWarps = 4;       // warps per thread block
constexpr int kLdA = kTile;        // sA[l * kLdA + r]
constexpr int kLdB = kTile + 1;    // sB[c * kLdB + l]
constexpr int kWarpSmem = kTile * kLdA + kTile * kLdB;  // doubles per warp

__global__ void __launch_bounds__(kNumWarps * 32) k_numeric_fp64(DevMat A, DevMat B, DevOut C,
                                                                 DevMat Cin, double alpha,
                                                                 double beta, DevWs ws,
                                                                 const DevStatus *st) {
  if (st->overflow) return;
  extern __shared__ double smem_num[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *sA = smem_num + warp * kWarpSmem;
  double *sB = sA + kTile * kLdA;
  const int64_t nblk = st->nblk_c;
  const int64_t gwarp = (int64_t)blockIdx.x * kNumWarps + warp;
  const int64_t nwarp = (int64_t)gridDim.x * kNumWarps;

  for (int64_t g = gwarp; g < nblk; g += nwarp) {
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
// Small-block variant: every block dimension (m, n and all k) at most 16.
// One warp per C block, 8 warps per thread block and up to three blocks per
// SM (24 warps) so the slow FP64 pipe always has ready warps. The operands of
// a product are copied to shared memory in their own column-major layout (a
// contiguous copy, no index arithmetic), and the next product's operands are
// already in flight in registers while the current one is multiplied. The
// (A offset, B offset, k) of up to 32 products are fetched at once, one per
// lane, and handed out with warp shuffles.
// ----------------------------------------------------------------------------
constexpr int kS = 16;             // largest block dimension of this variant
constexpr int kSWarps = 8;         // warps per thread block
constexpr int kSElems = kS * kS / 32;  // operand elements per lane (8)

template <int MINB>
__global__ void __launch_bounds__(kSWarps * 32, MINB)
    k_numeric_fp64_s16(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha, double beta,
                       DevWs ws, const DevStatus *st) {
  if (st->overflow) return;
  __shared__ double smem_s16[kSWarps][2 * kS * kS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *sA = smem_s16[warp];
  double *sB = sA + kS * kS;
  const int64_t nblk = st->nblk_c;
  const int64_t nwarp = (int64_t)gridDim.x * kSWarps;

  for (int64_t g = (int64_t)blockIdx.x * kSWarps + warp; g < nblk; g += nwarp) {
    const int i = C.blk_row[g], j = C.col_idx[g];
    const int m = C.row_sizes[i], n = C.col_sizes[j];
    const int64_t p0 = ws.prod_ptr[g], p1 = ws.prod_ptr[g + 1];
    const int te = m * n;
    const int nT = (te + 31) >> 5;
    int rc[kSElems];  // output (row, col) of the lane's t-th element, packed r | c << 8
    double acc[kSElems];
#pragma unroll
    for (int t = 0; t < kSElems; t++) {
      const int e = lane + 32 * t;
      rc[t] = (e < te) ? (e % m) | ((e / m) << 8) : 0;  // past the block: a valid dummy
      acc[t] = 0.0;
    }
    for (int64_t pb = p0; pb < p1; pb += 32) {
      const int nb = (p1 - pb < 32) ? (int)(p1 - pb) : 32;
      int64_t my_a = 0, my_b = 0;
      int my_s = 0;
      if (lane < nb) {
        const int2 pr = ws.prods[pb + lane];
        my_a = A.blk_off[pr.x];
        my_b = B.blk_off[pr.y];
        my_s = A.col_sizes[A.col_idx[pr.x]];
      }
      // operands of the first product of the batch
      double ra[kSElems], rb[kSElems];
      int s = __shfl_sync(0xffffffffu, my_s, 0);
      {
        const double *Ab = A.vals + __shfl_sync(0xffffffffu, my_a, 0);
        const double *Bb = B.vals + __shfl_sync(0xffffffffu, my_b, 0);
#pragma unroll
        for (int u = 0; u < kSElems; u++) {
          const int e = lane + 32 * u;
          ra[u] = (e < m * s) ? __ldg(Ab + e) : 0.0;
          rb[u] = (e < s * n) ? __ldg(Bb + e) : 0.0;
        }
      }
      for (int q = 0; q < nb; q++) {
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kSElems; u++) {
          sA[lane + 32 * u] = ra[u];
          sB[lane + 32 * u] = rb[u];
        }
        __syncwarp();
        const int sq = s;
        if (q + 1 < nb) {  // fetch the next product while this one is multiplied
          s = __shfl_sync(0xffffffffu, my_s, q + 1);
          const double *Ab = A.vals + __shfl_sync(0xffffffffu, my_a, q + 1);
          const double *Bb = B.vals + __shfl_sync(0xffffffffu, my_b, q + 1);
#pragma unroll
          for (int u = 0; u < kSElems; u++) {
            const int e = lane + 32 * u;
            ra[u] = (e < m * s) ? __ldg(Ab + e) : 0.0;
            rb[u] = (e < s * n) ? __ldg(Bb + e) : 0.0;
          }
        }
        for (int l = 0; l < sq; l++) {
#pragma unroll
          for (int t = 0; t < kSElems; t++) {
            if (t >= nT) break;
            acc[t] = fma(sA[(rc[t] & 255) + l * m], sB[(rc[t] >> 8) * sq + l], acc[t]);
          }
        }
      }
    }
    // epilogue: C_ij = beta * C_in_ij + alpha * S_ij, one coalesced write
    const int cin = ws.c_cin[g];
    const double *cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;
    double *out = C.vals + C.blk_off[g];
#pragma unroll
    for (int t = 0; t < kSElems; t++) {
      const int e = lane + 32 * t;
      if (t < nT && e < te) {
        double v = alpha * acc[t];
        if (cinv) v = fma(beta, cinv[e], v);
        out[e] = v;
      }
    }
  }
}

cudaError_t launch_numeric_fp64(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha,
                                double beta, DevWs ws, const DevStatus *st, int max_dim,
                                int nsm, cudaStream_t stream) {
  if (max_dim <= kS) {
    // blocks per SM the variant is compiled for: 2 (16 warps, no spills; 3%
    // faster on water2048) or 3 (24 warps, a few spilled registers);
    // BSM_S16_BLOCKS=3 selects the latter
    static int minb = [] {
      const char *v = getenv("BSM_S16_BLOCKS");
      return (v && atoi(v) == 3) ? 3 : 2;
    }();
    if (minb == 2)
      k_numeric_fp64_s16<2><<<nsm * 2, kSWarps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st);
    else
      k_numeric_fp64_s16<3><<<nsm * 3, kSWarps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)kNumWarps * kWarpSmem * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_numeric_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_numeric_fp64<<<nsm * 3, kNumWarps * 32, smem, stream>>>(A, B, C, Cin, alpha, beta, ws, st);
  return cudaGetLastError();
}

}  // namespace bsm
