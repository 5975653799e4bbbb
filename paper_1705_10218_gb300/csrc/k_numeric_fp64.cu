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

cudaError_t launch_numeric_fp64(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha,
                                double beta, DevWs ws, const DevStatus *st, int grid,
                                cudaStream_t stream) {
  const size_t smem = (size_t)kNumWarps * kWarpSmem * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_numeric_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_numeric_fp64<<<grid, kNumWarps * 32, smem, stream>>>(A, B, C, Cin, alpha, beta, ws, st);
  return cudaGetLastError();
}

}  // namespace bsm
