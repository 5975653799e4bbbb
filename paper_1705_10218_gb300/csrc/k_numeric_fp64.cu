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
//        2 or 3 thread blocks of 8 warps per SM; C blocks are taken one at a
//        time from a work counter.
//   t32: 32 x 32 output tiles, synchronous staging, 4 warps per block.
//   pk:  "packed" lane slots for tiles of up to 16 x 16: a lane slot is a pair
//        (output element, k-group), so a tile of te elements is computed by
//        te * G slots in nT passes of 32 lanes, with nT and G chosen per tile
//        shape so that te * G nearly fills 32 * nT (13 x 5: 65 elements, 7
//        groups in 15 passes, 95% of the slots useful, where one element per
//        slot uses 68%). The products of a C block are concatenated along k
//        (the C block is one GEMM over the concatenated k), staged in chunks
//        with 8-byte asynchronous copies, double buffered; group g sums the
//        k positions congruent to g mod G, and the G partial sums of an
//        element are added in group order at the end.
// All take an optional work list (C block indices, e.g. one shape class) and
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
                       DevWs ws, const DevStatus *st, const int32_t *items, const int64_t *seg,
                       unsigned long long *work) {
  if (st->overflow) return;
  __shared__ double smem_t16[kSWarps][2 * kS * kS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *sA = smem_t16[warp];
  double *sB = sA + kS * kS;
  int64_t wb, we;
  work_range(st, seg, wb, we);

  // C blocks come from the work counter (zero at launch), `grab` at a time:
  // one when there are few per warp, up to 8 when there are many (tiny C
  // blocks would otherwise queue on the counter)
  const int64_t per_warp = (we - wb) / ((int64_t)gridDim.x * kSWarps * 64);
  const int grab = per_warp < 1 ? 1 : (per_warp > 8 ? 8 : (int)per_warp);
  for (;;) {
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(work, (unsigned long long)grab);
    const int64_t w0 = wb + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    if (w0 >= we) break;
    const int64_t w1 = (w0 + grab < we) ? w0 + grab : we;
    for (int64_t w = w0; w < w1; w++) {
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
}

// ----------------------------------------------------------------------------
// g8: tiny C blocks with few products (semi-empirical-style matrices: blocks
// of a few rows, about one product per C block). A group of 8 lanes computes
// one C block at a time, a lane per column, the rows in registers (MR = 4, 6
// or 8 rows and GS = 4, 6 or 8 lanes per group, chosen per launch from the
// largest C block: 5 groups of 6 lanes fill 30 of a warp's 32 lanes for
// 6-wide blocks, where groups of 8 would leave a quarter of the lanes without
// a column). The groups of a warp are independent streams: each takes kG8Grab C blocks at a time from the
// work counter and walks their products one step per loop iteration, closing
// a C block (epilogue, next block's metadata) in the iteration that ends it,
// so a group whose block has more products does not hold the other groups at
// a loop exit. Lanes hold no shared state: the latency of each C block's chain
// of dependent loads is hidden by the many independent blocks in flight. A C
// block of more than MR rows or GS columns (only when the kernel is forced on
// larger blocks) is done in column and row chunks by its group.
// ----------------------------------------------------------------------------
constexpr int kG8Warps = 8;
constexpr int kG8Grab = 16;  // C blocks per group and grab

template <int MR, int GS>
__global__ void __launch_bounds__(kG8Warps * 32, 4)
    k_numeric_fp64_g8(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha, double beta,
                      DevWs ws, const DevStatus *st, const int32_t *items, const int64_t *seg,
                      unsigned long long *work) {
  if (st->overflow) return;
  const int lane = threadIdx.x & 31;
  const int grp = lane / GS, cl = lane - grp * GS;
  if (grp >= 32 / GS) return;  // lanes past the last whole group
  const unsigned gmask = ((1u << GS) - 1u) << (GS * grp);
  int64_t wb, we;
  work_range(st, seg, wb, we);
  // the second destination (host memory) when the whole result fits it
  double *hout = (C.host_vals && st->nnz_c <= C.host_cap) ? C.host_vals : nullptr;

  // the group's current grab [w, wend) and C block (group-uniform state)
  int64_t w = 0, wend = 0, p = 0, p1 = 0, cbase = 0;
  int m = 0, n = 0;
  const double *cinv = nullptr;
  double acc[MR];
  auto next_block = [&]() -> bool {
    if (w >= wend) {
      unsigned long long got = 0;
      if (cl == 0) got = atomicAdd(work, (unsigned long long)kG8Grab);
      w = wb + (int64_t)__shfl_sync(gmask, got, GS * grp);
      wend = (w + kG8Grab < we) ? w + kG8Grab : we;
      if (w >= we) return false;
    }
    const int64_t g = items ? items[w] : w;
    w++;
    m = C.row_sizes[C.blk_row[g]];
    n = C.col_sizes[C.col_idx[g]];
    p = ws.prod_ptr[g];
    p1 = ws.prod_ptr[g + 1];
    const int cin = ws.c_cin[g];
    cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;
    cbase = C.blk_off[g];
#pragma unroll
    for (int r = 0; r < MR; r++) acc[r] = 0.0;
    return true;
  };
  // rows [r0, r0 + MR) of column c of product q, added to acc
  auto product = [&](int64_t q, int c, int r0) {
    const int2 pr = ws.prods[q];
    const double *Ab = A.vals + A.blk_off[pr.x] + r0;
    const int s = A.col_sizes[A.col_idx[pr.x]];
    const double *Bb = B.vals + B.blk_off[pr.y] + (int64_t)c * s;
    for (int kk = 0; kk < s; kk++) {
      const double bv = __ldg(Bb + kk);
      const double *a = Ab + (int64_t)kk * m;
#pragma unroll
      for (int r = 0; r < MR; r++)
        if (r0 + r < m) acc[r] = fma(__ldg(a + r), bv, acc[r]);
    }
  };
  // C_ij = beta * C_in_ij + alpha * S_ij for rows [r0, r0 + MR) of column c
  auto store = [&](int c, int r0) {
#pragma unroll
    for (int r = 0; r < MR; r++) {
      if (r0 + r < m) {
        const int64_t loc = (int64_t)c * m + r0 + r;
        double v = alpha * acc[r];
        if (cinv) v = fma(beta, cinv[loc], v);
        C.vals[cbase + loc] = v;
        if (hout) hout[cbase + loc] = v;
      }
    }
  };

  bool have = next_block();
  while (have) {
    if (m > MR || n > GS) {  // column and row chunks, the products once per chunk
      for (int c = cl; c < n; c += GS)
        for (int r0 = 0; r0 < m; r0 += MR) {
#pragma unroll
          for (int r = 0; r < MR; r++) acc[r] = 0.0;
          for (int64_t q = p; q < p1; q++) product(q, c, r0);
          store(c, r0);
        }
      have = next_block();
      continue;
    }
    if (p < p1) {  // one product of the block (products in ascending k)
      if (cl < n) product(p, cl, 0);
      p++;
    }
    if (p >= p1) {  // the block is complete
      if (cl < n) store(cl, 0);
      have = next_block();
    }
  }
}

// ----------------------------------------------------------------------------
// pk
// ----------------------------------------------------------------------------
constexpr int kPkWarps = 8;          // warps per thread block (2 blocks per SM)
constexpr int kPkTile = 16;          // output tile edge
constexpr int kPkMaxSlots = 16;      // accumulator slots per lane (largest nT) of the pk16 variant
constexpr int kPkMaxG = kPkMaxGroups;  // largest number of k-groups
constexpr int kPkMaxKC = 64;         // largest chunk (k positions)
// Doubles per stage (two stages per warp; 2 blocks of 8 warps fit an SM). A
// tile of tm x tn takes chunks of KC k positions with KC * tm + tn * (KC + 1)
// within the stage.
constexpr int kPkStage = 880;
static_assert(32 * kPkMaxSlots <= kPkStage, "the slot sums must fit one stage");

size_t pk_smem_bytes() { return (size_t)kPkWarps * 2 * kPkStage * sizeof(double); }

// Slot shape of a tile of te (1..256) elements with at most `slots` slots per
// lane: the (nT, G) with nT <= slots, G <= kPkMaxG and te * G <= 32 * nT that
// maximises te * G / (32 * nT), the smallest nT among equals.
struct PkShapes {
  uint8_t nt[kPkTile * kPkTile + 1], g[kPkTile * kPkTile + 1];
};
constexpr PkShapes make_pk_shapes(int slots) {
  PkShapes tab{};
  for (int te = 1; te <= kPkTile * kPkTile; te++) {
    int bt = (te + 31) / 32, bg = 1;
    for (int t = 1; t <= slots; t++) {
      int g = (32 * t) / te;
      if (g > kPkMaxG) g = kPkMaxG;
      if (g >= 1 && g * bt > bg * t) {
        bt = t;
        bg = g;
      }
    }
    tab.nt[te] = (uint8_t)bt;
    tab.g[te] = (uint8_t)bg;
  }
  return tab;
}
__constant__ PkShapes c_pk_shapes12 = make_pk_shapes(12);
__constant__ PkShapes c_pk_shapes16 = make_pk_shapes(16);
static_assert(kPkTabEdge == kPkTile + 1, "the tuned table covers every tile shape");

void pk_formula_shape(int slots, int te, int *nt, int *g) {
  static const PkShapes s12 = make_pk_shapes(12), s16 = make_pk_shapes(16);
  const PkShapes &s = (slots == 12) ? s12 : s16;
  *nt = s.nt[te];
  *g = s.g[te];
}

// floor(x / d) as (x * r) >> 16 with r = ceil(2^16 / d): exact while
// x * (r * d - 2^16) < 2^16, i.e. for d <= 16 and x < 4096 (the error term is
// below d).
__device__ __forceinline__ uint32_t rcp16(uint32_t d) { return (65535u + d) / d; }
__device__ __forceinline__ int div16(int x, uint32_t r) { return (int)(((uint32_t)x * r) >> 16); }

__device__ __forceinline__ void cp_async8(double *sdst, const double *gsrc) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void pk_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void pk_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// C blocks a warp takes from the work counter at a time.
constexpr int kPkGrab = 1;

// `steps` steps of one chunk for a tile of NT slots per lane: slot t adds
// sA[ia_t + u * G * tm] * sB[ib_t + u * G] at step u. NT is a compile-time
// constant, so all loads of a step can be issued ahead of its FMAs; the step
// loop itself is not unrolled (with 16 instances, unrolled copies overflow the
// instruction cache on workloads with many tile shapes).
template <int NT, int SLOTS>
__device__ __forceinline__ void pk_steps(const double *__restrict__ sA,
                                         const double *__restrict__ sB,
                                         const uint32_t (&idx)[SLOTS],
                                         double (&acc)[SLOTS], int steps, int gtm, int G) {
#pragma unroll 1  // one copy of the step body per NT keeps the instruction footprint small
  for (int u = 0; u < steps; u++) {
#pragma unroll
    for (int t = 0; t < NT; t++) acc[t] = fma(sA[idx[t] & 0xFFFFu], sB[idx[t] >> 16], acc[t]);
    sA += gtm;
    sB += G;
  }
}

// work: a counter that is zero when the launch starts; warps take the next
// kPkGrab C blocks of the work range from it until the range is exhausted.
// SLOTS: accumulator slots per lane (12 or 16). Fewer slots lower the lane use
// of some tile shapes (13 x 13: 96% instead of 99%) but shorten the per-tile
// code; which wins depends on the block mix (the autotuner measures it).
template <int SLOTS>
__global__ void __launch_bounds__(kPkWarps * 32, 2)
    k_numeric_fp64_pk(DevMat A, DevMat B, DevOut C, DevMat Cin, double alpha, double beta,
                      DevWs ws, const DevStatus *st, const int32_t *items, const int64_t *seg,
                      unsigned long long *work) {
  if (st->overflow) return;
  constexpr int kStage = kPkStage;
  const PkShapes &shapes = (SLOTS == 12) ? c_pk_shapes12 : c_pk_shapes16;
  extern __shared__ double smem_pk[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *wbuf = smem_pk + warp * 2 * kStage;
  int64_t wb, we;
  work_range(st, seg, wb, we);
  // the second destination (host memory) when the whole result fits it
  double *hout = (C.host_vals && st->nnz_c <= C.host_cap) ? C.host_vals : nullptr;

  for (;;) {
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(work, (unsigned long long)kPkGrab);
    const int64_t w0 = wb + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    if (w0 >= we) break;
    const int64_t w1 = (w0 + kPkGrab < we) ? w0 + kPkGrab : we;
    for (int64_t w = w0; w < w1; w++) {
      const int64_t gblk = items ? items[w] : w;
      const int i = C.blk_row[gblk], j = C.col_idx[gblk];
      const int m = C.row_sizes[i], n = C.col_sizes[j];
      const int64_t p0 = ws.prod_ptr[gblk], p1 = ws.prod_ptr[gblk + 1];
      const int cin = ws.c_cin[gblk];
      const double *cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;
      double *out = C.vals + C.blk_off[gblk];
      double *hblk = hout ? hout + C.blk_off[gblk] : nullptr;

      for (int r0 = 0; r0 < m; r0 += kPkTile) {
        for (int c0 = 0; c0 < n; c0 += kPkTile) {
          const int tm = min(kPkTile, m - r0), tn = min(kPkTile, n - c0);
          const int te = tm * tn;
          int nT = shapes.nt[te], G = shapes.g[te];
          if (ws.pk_tab) {  // a tuned shape (validated by the host)
            const uint32_t e = ws.pk_tab[(SLOTS == 16 ? kPkTabSize : 0) + tm * kPkTabEdge + tn];
            nT = (int)(e >> 8);
            G = (int)(e & 0xFFu);
          }
          const int used = te * G;
          const uint32_t rtm = rcp16(tm), rg = rcp16(G);
          // chunk length: the largest multiple of G with KC * tm + tn * (KC + 1) <= kStage
          const int kfit = min(kPkMaxKC, (kStage - tn) / (tm + tn));
          const int KC = G * div16(kfit, rg);
          const int ldB = KC + 1;  // sB[c * ldB + kk]
          const int dq_tm = div16(32, rtm), dr_tm = 32 - dq_tm * tm;  // 32 = dq_tm * tm + dr_tm
          // slot t of this lane: z = lane + 32 t -> group g = z / te, element
          // e = z % te (row e % tm, column e / tm); its operands at step 0 are
          // sA[ia] and sB[ib], kept as ia | ib << 16 (both below 2^9)
          uint32_t idx[SLOTS];
          double acc[SLOTS];
          {
            int g = 0, e = lane;
            while (e >= te) {
              e -= te;
              g++;
            }
#pragma unroll
            for (int t = 0; t < SLOTS; t++) {
              idx[t] = 0;  // slots past te * G read valid operands; their sums are discarded
              if (g < G) {
                const int c = div16(e, rtm), r = e - c * tm;
                idx[t] = (uint32_t)(g * tm + r) | ((uint32_t)(c * ldB + g) << 16);
              }
              acc[t] = 0.0;
              e += 32;
              while (e >= te) {
                e -= te;
                g++;
              }
            }
          }

          // product cursor: batch [pb, pb + nb) of metadata, one product per lane
          int64_t pb = p0;
          int nb = 0, q = 0, lq = 0;
          int64_t my_a = 0, my_b = 0;
          int my_s = 1;
          auto load_batch = [&]() {
            nb = (p1 - pb < 32) ? (int)(p1 - pb) : 32;
            if (lane < nb) {
              const int2 pr = __ldcs(ws.prods + pb + lane);  // read once: evict first
              my_a = A.blk_off[pr.x];
              my_b = B.blk_off[pr.y];
              my_s = A.col_sizes[A.col_idx[pr.x]];
            }
          };
          if (pb < p1) load_batch();

          // Copies the next (up to) KC k positions of the concatenated products
          // into stage `buf`: sA[kk * tm + r] = A(r0 + r, k), sB[c * ldB + kk] =
          // B(k, c0 + c); zero-fills up to the next multiple of G. Returns the
          // number of steps (k positions / G) of the chunk.
          auto fill = [&](int buf) -> int {
            double *sA = wbuf + buf * kStage;
            double *sB = sA + KC * tm;
            int kk = 0;
            while (kk < KC && pb < p1) {
              const int s = __shfl_sync(0xffffffffu, my_s, q);
              const int64_t ao = __shfl_sync(0xffffffffu, my_a, q);
              const int64_t bo = __shfl_sync(0xffffffffu, my_b, q);
              const int nc = min(s - lq, KC - kk);
              const double *Ab = A.vals + ao + (int64_t)lq * m + r0;  // column lq, row r0
              const double *Bb = B.vals + bo + (int64_t)c0 * s + lq;  // row lq, column c0
              double *dA = sA + kk * tm;
              if (tm == m) {  // whole columns: one contiguous range
                for (int z = lane; z < nc * m; z += 32) cp_async8(dA + z, Ab + z);
              } else {  // (l, r) = divmod(z, tm), stepped by 32
                int l = div16(lane, rtm), r = lane - l * tm;
                for (int z = lane; z < nc * tm; z += 32) {
                  cp_async8(dA + l * tm + r, Ab + (int64_t)l * m + r);
                  l += dq_tm;
                  r += dr_tm;
                  if (r >= tm) {
                    r -= tm;
                    l++;
                  }
                }
              }
              {  // (c, l) = divmod(z, nc), stepped by 32
                const uint32_t rnc = rcp16(nc);
                const int dq = div16(32, rnc), dr = 32 - dq * nc;
                int c = div16(lane, rnc), l = lane - c * nc;
                double *dB = sB + kk;
                for (int z = lane; z < nc * tn; z += 32) {
                  cp_async8(dB + c * ldB + l, Bb + (int64_t)c * s + l);
                  c += dq;
                  l += dr;
                  if (l >= nc) {
                    l -= nc;
                    c++;
                  }
                }
              }
              kk += nc;
              lq += nc;
              if (lq == s) {
                lq = 0;
                if (++q == nb) {
                  pb += nb;
                  q = 0;
                  if (pb < p1) load_batch();
                }
              }
            }
            const int steps = div16(kk + G - 1, rg);
            const int pad = steps * G - kk;
            if (pad) {
              for (int z = lane; z < pad * tm; z += 32) sA[kk * tm + z] = 0.0;
              for (int z = lane; z < pad * tn; z += 32) {
                const int c = div16(z, rcp16(pad)), l = z - c * pad;
                sB[c * ldB + kk + l] = 0.0;
              }
            }
            return steps;
          };

          int cur = fill(0);  // steps of the current chunk
          pk_commit();
          for (int ch = 0;; ch++) {
            const int buf = ch & 1;
            const int nxt = (pb < p1) ? fill(buf ^ 1) : 0;
            pk_commit();
            pk_wait<1>();  // the current chunk has landed
            __syncwarp();
            const double *sA = wbuf + buf * kStage;
            const double *sB = sA + KC * tm;
            const int gtm = G * tm;
            switch (nT) {
#define BSM_PK_CASE(N)                                                                 \
  case N:                                                                              \
    if (N <= SLOTS) pk_steps<(N <= SLOTS ? N : 1), SLOTS>(sA, sB, idx, acc, cur, gtm, G); \
    break;
              BSM_PK_CASE(1) BSM_PK_CASE(2) BSM_PK_CASE(3) BSM_PK_CASE(4)
              BSM_PK_CASE(5) BSM_PK_CASE(6) BSM_PK_CASE(7) BSM_PK_CASE(8)
              BSM_PK_CASE(9) BSM_PK_CASE(10) BSM_PK_CASE(11) BSM_PK_CASE(12)
              BSM_PK_CASE(13) BSM_PK_CASE(14) BSM_PK_CASE(15) BSM_PK_CASE(16)
#undef BSM_PK_CASE
            }
            __syncwarp();  // the stage is read before it is filled again
            if (nxt == 0) break;
            cur = nxt;
          }
          pk_wait<0>();
          __syncwarp();

          // the G partial sums of each element, added in group order
          double *red = wbuf;
#pragma unroll
          for (int t = 0; t < SLOTS; t++) {
            const int z = lane + 32 * t;
            if (t < nT && z < used) red[z] = acc[t];
          }
          __syncwarp();
          int c = div16(lane, rtm), r = lane - c * tm;
          for (int e = lane; e < te; e += 32) {
            double v = red[e];
            for (int g = 1; g < G; g++) v += red[g * te + e];
            const int64_t loc = (int64_t)(c0 + c) * m + r0 + r;
            v = alpha * v;
            if (cinv) v = fma(beta, cinv[loc], v);
            // written once, not read by this multiply: streaming stores keep the
            // operand rows, which the next C blocks read, in L2
            __stcs(out + loc, v);
            if (hblk) __stcs(hblk + loc, v);
            c += dq_tm;
            r += dr_tm;
            if (r >= tm) {
              r -= tm;
              c++;
            }
          }
          __syncwarp();
        }
      }
    }
  }
}

cudaError_t launch_numeric_fp64(int variant, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                double alpha, double beta, DevWs ws, const DevStatus *st,
                                const int32_t *items, const int64_t *seg, int grid,
                                unsigned long long *work, int max_m, int max_n,
                                cudaStream_t stream) {
  switch (variant) {
    case kFp64G8: {
      const int mr = max_m <= 4 ? 4 : max_m <= 6 ? 6 : 8;
      const int gs = max_n <= 4 ? 4 : max_n <= 6 ? 6 : 8;
#define BSM_G8(R, G)                                                                           \
  k_numeric_fp64_g8<R, G><<<grid, kG8Warps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st, \
                                                              items, seg, work)
      if (mr == 4) {
        if (gs == 4) BSM_G8(4, 4); else if (gs == 6) BSM_G8(4, 6); else BSM_G8(4, 8);
      } else if (mr == 6) {
        if (gs == 4) BSM_G8(6, 4); else if (gs == 6) BSM_G8(6, 6); else BSM_G8(6, 8);
      } else {
        if (gs == 4) BSM_G8(8, 4); else if (gs == 6) BSM_G8(8, 6); else BSM_G8(8, 8);
      }
#undef BSM_G8
      break;
    }
    case kFp64T16B3:
      k_numeric_fp64_t16<3><<<grid, kSWarps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st,
                                                               items, seg, work);
      break;
    case kFp64T32: {
      // the shared-memory attribute is set once per device by numeric_fp64_init
      const size_t smem = (size_t)kNumWarps * kWarpSmem * sizeof(double);
      k_numeric_fp64_t32<<<grid, kNumWarps * 32, smem, stream>>>(A, B, C, Cin, alpha, beta, ws,
                                                                 st, items, seg);
      break;
    }
    case kFp64Pk12:
      k_numeric_fp64_pk<12><<<grid, kPkWarps * 32, pk_smem_bytes(), stream>>>(
          A, B, C, Cin, alpha, beta, ws, st, items, seg, work);
      break;
    case kFp64Pk16:
      k_numeric_fp64_pk<16><<<grid, kPkWarps * 32, pk_smem_bytes(), stream>>>(
          A, B, C, Cin, alpha, beta, ws, st, items, seg, work);
      break;
    default:
      k_numeric_fp64_t16<2><<<grid, kSWarps * 32, 0, stream>>>(A, B, C, Cin, alpha, beta, ws, st,
                                                               items, seg, work);
  }
  return cudaGetLastError();
}

int fp64_variant_blocks_per_sm(int variant) {
  if (variant == kFp64G8) return 4;
  return (variant == kFp64T16B3 || variant == kFp64T32) ? 3 : 2;
}

cudaError_t numeric_fp64_init() {
  const size_t smem = (size_t)kNumWarps * kWarpSmem * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_numeric_fp64_t32,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_numeric_fp64_pk<12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pk_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_numeric_fp64_pk<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pk_smem_bytes());
}

}  // namespace bsm
