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
// Slice layout. For every block b of r x c values (FP64 offset blk_off[b]),
// the slices live at a fixed multiple of the FP64 offset (no extra offset
// table). An operand is seen as `rows` rows along the k index:
//   "left" layout (the block as a left operand, k = its columns): r rows of
//         c values; "right" layout (as a right operand, k = its rows): c rows
//         (the block's columns) of r values.
// k is cut into 16-byte pieces (8 BF16 or 4 TF32 values, zero past the end),
// and a plane stores the pieces k-piece-major: piece (row, kp) at
// (kp * rows + row) * 16 bytes. Eight consecutive rows of one k-piece, the
// 8 x 8 unit of the tensor cores' fragment loads (ldmatrix), are then 128
// contiguous bytes (no shared-memory bank conflict), and a whole operand (all
// planes) is one contiguous, 16-byte aligned run for a bulk copy.
//   BF16: 3 planes of rows * ceil8(k) halfwords at halfword 24*blk_off[b];
//   TF32: 2 planes of rows * ceil4(k) words at word 8*blk_off[b].
#include <cstdint>

#include "bsm_internal.h"

namespace bsm {

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
// Split every block of a matrix into the left and/or right slice layouts.
// One warp per block (grid-stride), lanes over the positions of the block
// padded to whole pieces in both directions (ceil8(r) x ceil8(c) for BF16,
// ceil4 for TF32, column-major): each value is split once and its slices are
// written to both layouts; the padding positions write the zeros.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int round_up(int x, int q) { return (x + q - 1) / q * q; }

template <int NS, int BITS, int PIECE, typename T>
__device__ __forceinline__ void split_block(const double *__restrict__ x, int r, int c, int lane,
                                            T *__restrict__ left, T *__restrict__ right) {
  const int rp = round_up(r, PIECE), cp = round_up(c, PIECE);
  const int lplane = r * cp, rplane = c * rp;  // elements per plane
  for (int e = lane; e < rp * cp; e += 32) {
    const int yc = e / rp, xr = e - yc * rp;  // (row xr, column yc), column-major
    const bool in = xr < r && yc < c;
    const Slices<NS, BITS> sl = split_value<NS, BITS>(in ? x[xr + (int64_t)yc * r] : 0.0);
    // left: row xr along k = yc; right: row yc along k = xr; pieces k-major
    const int li = ((yc / PIECE) * r + xr) * PIECE + (yc % PIECE);
    const int ri = ((xr / PIECE) * c + yc) * PIECE + (xr % PIECE);
#pragma unroll
    for (int q = 0; q < NS; q++) {
      if (left && xr < r) left[(int64_t)q * lplane + li] = (T)sl.s[q];
      if (right && yc < c) right[(int64_t)q * rplane + ri] = (T)sl.s[q];
    }
  }
}

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
    const int64_t base = kBf16HalfwordsPerValue * blk_off[b];
    split_block<3, 8, 8>(vals + blk_off[b], row_sizes[blk_row[b]], col_sizes[col_idx[b]], lane,
                         left ? left + base : nullptr, right ? right + base : nullptr);
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
    const int64_t base = kTf32WordsPerValue * blk_off[b];
    split_block<2, 11, 4>(vals + blk_off[b], row_sizes[blk_row[b]], col_sizes[col_idx[b]], lane,
                          left ? left + base : nullptr, right ? right + base : nullptr);
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
__device__ __forceinline__ void mma_bf16_k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                             uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_tf32_k8(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                            uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Numeric kernel (below). A warp computes one C block at a time, or its
// transpose, whichever needs fewer 16x8 MMA tiles. Operands: L (Mp rows along
// k) and R (Np rows along k), both k-piece-major. Not transposed: L = A_ik (A's
// left layout), R = B_kj (B's right layout); transposed (C^T = B^T A^T): L =
// B_kj^T (B's right layout), R = A_ik^T (A's left layout). A k step is 16 (BF16;
// 8 for a last piece) or 8 (TF32) values of k with all slice products of every
// tile.
//
// Accumulation: the products are summed in FP32 by the tensor cores, a few at
// a time, then added to a running sum kept as an unevaluated pair hi + lo of
// FP32 numbers (TwoSum, error-free), so the long sum over the products of a C
// block loses no more than FP32 rounding of each partial sum; hi + lo is
// formed in FP64 at the end (FP32 -> FP64 is exact).
// ---------------------------------------------------------------------------
// hi + lo += x, exactly (Knuth's TwoSum in FP32, no fused operations).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ---------------------------------------------------------------------------
// Pipelined kernel. Two instances: C blocks whose MMA problem fits 16 x 16
// (the water and small-block case; 1x2 tiles per warp, 16-row slots), and the
// others up to 32 x 32 (2x4 tiles per warp, 32-row slots, tiles outside the
// problem skipped). Each warp streams its C blocks' products through a ring
// of STAGES shared-memory slots. For every product one lane starts two bulk
// asynchronous copies (cp.async.bulk: all slice planes of the left operand in
// one, of the right one in the other) whose completion is counted in bytes on
// the slot's mbarrier, STAGES - 1 products ahead of the tensor-core work, so
// the L2 latency of a product's operands is hidden behind the products before
// it; the fragments are read from the slot with ldmatrix, conflict-free thanks
// to the k-piece-major planes. The (A offset, B offset, k) of the products are
// read 32 at a time into a per-warp table in shared memory.
// ---------------------------------------------------------------------------
// Ring depth: deeper rings hide more copy latency, shallower ones leave room
// for more warps per SM. Measured on water (k of 5 and 13): 2 stages beat 3, 4
// and 6 (6 stages leave 8 warps per SM): each warp's chain of dependent
// fragment loads and MMAs needs many warps to fill the issue slots.
constexpr int kPipeStages = 2;
constexpr int kPipeWarps = 4;
// Products summed plainly in FP32 before each compensated fold: a partial sum
// of kFold products carries kFold times the rounding of one, still far below
// the slice truncation error, and the fold costs 6 FP32 operations per value.
constexpr int kFold = 4;
constexpr int kMetaEntries = 64;
constexpr int kMetaBytes = kMetaEntries * (8 + 8 + 4);
// A waiting thread is suspended until the phase completes or kWaitHintNs
// pass (no issue slots spent on polling); after kWaitPolls such waits (about
// a second) a warp gives up on a copy that does not land: it then raises the
// status error flag, waits (again bounded) for the copies it has in flight and
// stops.
constexpr uint32_t kWaitHintNs = 1000;
constexpr int kWaitPolls = 1 << 20;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// generic-proxy accesses of shared memory (ldmatrix reads of a slot) before
// async-proxy writes of it (the next bulk copy into the slot)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kWaitHintNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitPolls; i++)
    if (mbar_test(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                        uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

// Bytes of one row of a plane (k up to s, whole 16-byte pieces), and of one
// operand slot: all planes of at most `rows` rows (16, or 32 in the large-block
// instance) of k up to smax.
__host__ __device__ __forceinline__ int pipe_row_bytes(int precision, int s) {
  return precision == BSM_PREC_SPLIT_BF16X3 ? 2 * ((s + 7) & ~7) : 4 * ((s + 3) & ~3);
}
__host__ __device__ __forceinline__ int pipe_operand_bytes(int precision, int smax, int rows) {
  return (precision == BSM_PREC_SPLIT_BF16X3 ? 3 : 2) * rows * pipe_row_bytes(precision, smax);
}
// per warp: the slots, the product table, one mbarrier per slot (16-byte multiple)
__host__ __device__ __forceinline__ int pipe_warp_bytes(int precision, int smax, int stages,
                                                        int rows) {
  return stages * 2 * pipe_operand_bytes(precision, smax, rows) + kMetaBytes +
         ((8 * stages + 15) & ~15);
}
// The large-block instance (MMA problems up to 32x32, 2x4 tiles of 16x8 per
// warp, 32-row slots): 2 warps per thread block, 2 stages.
constexpr int kPipeWarpsBig = 2;

// A C block of the pipelined kernel's stream: gb < 0 marks the end of the work.
struct PipeBlock {
  int64_t gb, p0;
  int np, m, n;
};

// Minimum resident blocks per SM the register budget is fitted to: the kernel
// is bound by instruction issue and latency, so more resident warps pay, but
// not at the price of spills (6 blocks of the 2-stage instance spill; the
// TF32 slots are larger: 5 blocks of 2 stages fill the shared memory).
// The large-block instance: 4 blocks of 2 warps (up to 255 registers).
template <int PREC, int STAGES, bool BIG>
constexpr int pipe_min_blocks() {
  return BIG ? 4
             : PREC == BSM_PREC_SPLIT_BF16X3 ? (STAGES == 2 ? 5 : STAGES == 3 ? 5 : 4)
                                             : (STAGES == 2 ? 5 : 4);
}

// sel: 0 every C block, 1 those whose MMA problem fits 16x16, 2 the others.
template <int PREC, int STAGES, bool BIG>
__global__ void __launch_bounds__((BIG ? kPipeWarpsBig : kPipeWarps) * 32,
                                  pipe_min_blocks<PREC, STAGES, BIG>())
    k_numeric_split_pipe(DevMat A, DevMat B, DevOut C, DevMat Cin, const void *__restrict__ a_left,
                         const void *__restrict__ b_right, double alpha, double beta, DevWs ws,
                         const DevStatus *st, const int32_t *__restrict__ items,
                         const int64_t *__restrict__ seg, int smax, int sel,
                         unsigned long long *work) {
  if (st->overflow) return;
  constexpr bool BF = (PREC == BSM_PREC_SPLIT_BF16X3);
  constexpr int NSL = BF ? 3 : 2;
  constexpr int ROWS = BIG ? 32 : 16;  // slot rows
  constexpr int MT = BIG ? 2 : 1, NT = BIG ? 4 : 2;  // 16x8 tiles per warp
  constexpr int NP = NT / 2;  // pairs of 8-column tiles (one x4 fragment load)
  // slice bytes per FP64 value of an operand's offset
  constexpr int64_t kUnit = BF ? 2 * kBf16HalfwordsPerValue : 4 * kTf32WordsPerValue;
  extern __shared__ __align__(16) unsigned char smem_pipe[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int opb = pipe_operand_bytes(PREC, smax, ROWS);
  unsigned char *wbase = smem_pipe + warp * pipe_warp_bytes(PREC, smax, STAGES, ROWS);
  // the product table, a ring indexed by stream position: source addresses of
  // the two operands' slices and k
  const unsigned char **meta_a = reinterpret_cast<const unsigned char **>(wbase + STAGES * 2 * opb);
  const unsigned char **meta_b = meta_a + kMetaEntries;
  int *meta_s = reinterpret_cast<int *>(meta_b + kMetaEntries);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(wbase);
  const uint32_t bar0 = sbase + (uint32_t)(STAGES * 2 * opb + kMetaBytes);
  if (lane == 0) {
#pragma unroll
    for (int x = 0; x < STAGES; x++) mbar_init(bar0 + 8 * x, 1);
    mbar_init_fence();
  }
  __syncwarp();
  // which 8 x 8 piece (rows 0-7 or 8-15, k piece 0 or 1 of the step) this
  // lane addresses in ldmatrix: "a" order for the left operand (and for the
  // right one in BF16 k8 steps), "b" order for the right one
  const int ra = (lane & 7) + ((lane >> 3) & 1) * 8, pa = lane >> 4;
  const int rb_ = (lane & 7) + (lane >> 4) * 8, pb = (lane >> 3) & 1;

  int64_t wb = 0, we = st->nblk_c;
  if (seg) {
    wb = seg[0];
    we = seg[1];
  }
  const bool plain = (alpha == 1.0 && beta == 0.0);
  // The products of the C blocks a warp takes form one stream; stream position
  // u uses ring slot u % STAGES (mbarrier phase (u / STAGES) & 1) and table
  // entry u % kMetaEntries. Copies run STAGES - 1 positions ahead of the
  // tensor-core work, across C block boundaries (into the next block's first
  // products), so the ring does not drain between blocks.
  uint32_t u_issue = 0, u_done = 0;  // next position to copy / to compute
  bool failed = false;
  unsigned long long next = 0;  // the work counter's next index, fetched ahead
  if (lane == 0) next = atomicAdd(work, 1ull);
  PipeBlock cur, nxt;
  int cur_issued = 0, nxt_issued = 0;  // products of the block started so far
  bool have_nxt = false;

  // the next C block of this launch (warp-uniform); gb < 0: none left
  auto take = [&](PipeBlock &b) {
    for (;;) {
      const int64_t w = wb + (int64_t)__shfl_sync(0xffffffffu, next, 0);
      if (w >= we) {
        b.gb = -1;
        b.np = 0;
        return;
      }
      if (lane == 0) next = atomicAdd(work, 1ull);
      const int64_t gb = items ? items[w] : w;
      const int i = C.blk_row[gb], j = C.col_idx[gb];
      const int m = C.row_sizes[i], n = C.col_sizes[j];
      const int tiles_n = ((m + 15) >> 4) * ((n + 7) >> 3);
      const int tiles_t = ((n + 15) >> 4) * ((m + 7) >> 3);
      const bool tr = tiles_t < tiles_n;
      const int Mp = tr ? n : m, Np = tr ? m : n;
      const bool small = Mp <= 16 && Np <= 16;
      if ((sel == 1 && !small) || (sel == 2 && small)) continue;
      b.gb = gb;
      b.p0 = ws.prod_ptr[gb];
      b.np = (int)(ws.prod_ptr[gb + 1] - b.p0);
      b.m = m;
      b.n = n;
      return;
    }
  };
  // start the copies of product q of block b at stream position u_issue (all
  // lanes call; the table holds the next 32 products of b from q % 32 == 0)
  auto issue = [&](const PipeBlock &b, int q) {
    const uint32_t u = u_issue++;
    if ((q & 31) == 0) {
      const int qq = q + lane;
      if (qq < b.np) {
        const int2 pr = ws.prods[b.p0 + qq];
        const int e = (int)((u + (uint32_t)lane) & (kMetaEntries - 1));
        meta_a[e] = static_cast<const unsigned char *>(a_left) + kUnit * A.blk_off[pr.x];
        meta_b[e] = static_cast<const unsigned char *>(b_right) + kUnit * B.blk_off[pr.y];
        meta_s[e] = A.col_sizes[A.col_idx[pr.x]];
      }
      __syncwarp();
    }
    if (lane == 0) {
      const int e = (int)(u & (kMetaEntries - 1));
      const int rb = pipe_row_bytes(PREC, meta_s[e]);
      const uint32_t bytes_a = (uint32_t)(NSL * b.m * rb), bytes_b = (uint32_t)(NSL * b.n * rb);
      const uint32_t slot = u % STAGES;
      const uint32_t dst = sbase + slot * 2 * (uint32_t)opb, bar = bar0 + 8 * slot;
      fence_proxy_async_smem();
      mbar_expect_tx(bar, bytes_a + bytes_b);
      bulk_copy_g2s(dst, meta_a[e], bytes_a, bar);
      bulk_copy_g2s(dst + (uint32_t)opb, meta_b[e], bytes_b, bar);
    }
  };

  take(cur);
  while (cur_issued < cur.np && (int)(u_issue - u_done) < STAGES - 1) issue(cur, cur_issued++);
  while (cur.gb >= 0) {
    const int m = cur.m, n = cur.n;
    const int tiles_n = ((m + 15) >> 4) * ((n + 7) >> 3);
    const int tiles_t = ((n + 15) >> 4) * ((m + 7) >> 3);
    const bool tr = tiles_t < tiles_n;
    const int Mp = tr ? n : m, Np = tr ? m : n;
    const bool two = Np > 8;  // a second 8-column tile
    float hi[MT][NT][4], lo[MT][NT][4], acc[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int x = 0; x < 4; x++) hi[mt][nt][x] = lo[mt][nt][x] = acc[mt][nt][x] = 0.f;

    for (int q = 0; q < cur.np; q++) {
      const uint32_t u = u_done, slot = u % STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8 * slot, (u / STAGES) & 1u))) {
        failed = true;
        break;
      }
      u_done++;
      __syncwarp();
      // refill the slot the previous position used: the next product of this
      // block, else the first ones of the next block
      if (cur_issued < cur.np) {
        issue(cur, cur_issued++);
      } else {
        if (!have_nxt) {
          take(nxt);
          nxt_issued = 0;
          have_nxt = true;
        }
        if (nxt_issued < nxt.np) issue(nxt, nxt_issued++);
      }
      const int s = meta_s[u & (kMetaEntries - 1)];
      const int rb = pipe_row_bytes(PREC, s);
      const uint32_t sA = sbase + slot * 2 * (uint32_t)opb, sB = sA + (uint32_t)opb;
      // L (Mp rows) and R (Np rows) in the slot; plane strides rows * rb
      const uint32_t sL = tr ? sB : sA, sR = tr ? sA : sB;
      const uint32_t lpl = (uint32_t)(Mp * rb), rpl = (uint32_t)(Np * rb);
      // this lane's piece address at k step 0; a k piece column is rows * 16 bytes
      const uint32_t adL = sL + 16u * (uint32_t)(pa * Mp + ra);
      const uint32_t adR = sR + 16u * (uint32_t)(pb * Np + rb_);
      const uint32_t adR2 = sR + 16u * (uint32_t)ra;  // "a" order on R (half steps)
      if constexpr (BIG) {
        // tile (mt, nt) is live when it holds part of the Mp x Np problem
        bool live[MT][NT];
#pragma unroll
        for (int mt = 0; mt < MT; mt++)
#pragma unroll
          for (int nt = 0; nt < NT; nt++) live[mt][nt] = mt * 16 < Mp && nt * 8 < Np;
        if (BF) {
          constexpr int PA[6] = {2, 1, 0, 1, 0, 0};
          constexpr int PB[6] = {0, 1, 2, 0, 1, 0};
          for (int kk = 0; kk < s; kk += 16) {
            const uint32_t koL = 16u * (uint32_t)((kk >> 3) * Mp), koR = 16u * (uint32_t)((kk >> 3) * Np);
            if (s - kk <= 8) {  // one k piece left: m16n8k8
              uint32_t a[3][MT][2], b[3][NP][2];
#pragma unroll
              for (int q3 = 0; q3 < 3; q3++) {
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
                  ldsm_x2(a[q3][mt][0], a[q3][mt][1], adL + q3 * lpl + koL + 256u * mt);
#pragma unroll
                for (int p2 = 0; p2 < NP; p2++)
                  ldsm_x2(b[q3][p2][0], b[q3][p2][1], adR2 + q3 * rpl + koR + 256u * p2);
              }
#pragma unroll
              for (int pq = 0; pq < 6; pq++)
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
#pragma unroll
                  for (int nt = 0; nt < NT; nt++)
                    if (live[mt][nt])
                      mma_bf16_k8(acc[mt][nt], a[PA[pq]][mt][0], a[PA[pq]][mt][1],
                                  b[PB[pq]][nt >> 1][nt & 1]);
            } else {
              uint32_t a[3][MT][4], b[3][NP][4];
#pragma unroll
              for (int q3 = 0; q3 < 3; q3++) {
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
                  ldsm_x4(a[q3][mt][0], a[q3][mt][1], a[q3][mt][2], a[q3][mt][3],
                          adL + q3 * lpl + koL + 256u * mt);
#pragma unroll
                for (int p2 = 0; p2 < NP; p2++)
                  ldsm_x4(b[q3][p2][0], b[q3][p2][1], b[q3][p2][2], b[q3][p2][3],
                          adR + q3 * rpl + koR + 256u * p2);
              }
#pragma unroll
              for (int pq = 0; pq < 6; pq++)
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
#pragma unroll
                  for (int nt = 0; nt < NT; nt++)
                    if (live[mt][nt])
                      mma_bf16_k16(acc[mt][nt], a[PA[pq]][mt], b[PB[pq]][nt >> 1][2 * (nt & 1)],
                                   b[PB[pq]][nt >> 1][2 * (nt & 1) + 1]);
            }
          }
        } else {
          constexpr int PA[3] = {1, 0, 0};
          constexpr int PB[3] = {0, 1, 0};
          for (int kk = 0; kk < s; kk += 8) {
            const uint32_t koL = 16u * (uint32_t)((kk >> 2) * Mp), koR = 16u * (uint32_t)((kk >> 2) * Np);
            uint32_t a[2][MT][4], b[2][NP][4];
            if (s - kk <= 4) {  // one k piece left: the other half is zero
#pragma unroll
              for (int q2 = 0; q2 < 2; q2++) {
#pragma unroll
                for (int mt = 0; mt < MT; mt++) {
                  ldsm_x2(a[q2][mt][0], a[q2][mt][1], adL + q2 * lpl + koL + 256u * mt);
                  a[q2][mt][2] = a[q2][mt][3] = 0u;
                }
#pragma unroll
                for (int p2 = 0; p2 < NP; p2++) {
                  ldsm_x2(b[q2][p2][0], b[q2][p2][2], adR2 + q2 * rpl + koR + 256u * p2);
                  b[q2][p2][1] = b[q2][p2][3] = 0u;
                }
              }
            } else {
#pragma unroll
              for (int q2 = 0; q2 < 2; q2++) {
#pragma unroll
                for (int mt = 0; mt < MT; mt++)
                  ldsm_x4(a[q2][mt][0], a[q2][mt][1], a[q2][mt][2], a[q2][mt][3],
                          adL + q2 * lpl + koL + 256u * mt);
#pragma unroll
                for (int p2 = 0; p2 < NP; p2++)
                  ldsm_x4(b[q2][p2][0], b[q2][p2][1], b[q2][p2][2], b[q2][p2][3],
                          adR + q2 * rpl + koR + 256u * p2);
              }
            }
#pragma unroll
            for (int pq = 0; pq < 3; pq++)
#pragma unroll
              for (int mt = 0; mt < MT; mt++)
#pragma unroll
                for (int nt = 0; nt < NT; nt++)
                  if (live[mt][nt])
                    mma_tf32_k8(acc[mt][nt], a[PA[pq]][mt], b[PB[pq]][nt >> 1][2 * (nt & 1)],
                                b[PB[pq]][nt >> 1][2 * (nt & 1) + 1]);
          }
        }
      } else {
      // slice products, smallest first: (3,1) (2,2) (1,3) (2,1) (1,2) (1,1)
      // (BF16); (2,1) (1,2) (1,1) (TF32)
      if (BF) {
        constexpr int PA[6] = {2, 1, 0, 1, 0, 0};
        constexpr int PB[6] = {0, 1, 2, 0, 1, 0};
        for (int kk = 0; kk < s; kk += 16) {
          const uint32_t koL = 16u * (uint32_t)((kk >> 3) * Mp), koR = 16u * (uint32_t)((kk >> 3) * Np);
          if (s - kk <= 8) {  // one k piece left: m16n8k8
            uint32_t a[3][2], b[3][2];
#pragma unroll
            for (int q3 = 0; q3 < 3; q3++) {
              ldsm_x2(a[q3][0], a[q3][1], adL + q3 * lpl + koL);
              ldsm_x2(b[q3][0], b[q3][1], adR2 + q3 * rpl + koR);
            }
            if (two) {
#pragma unroll
              for (int pq = 0; pq < 6; pq++) {
                mma_bf16_k8(acc[0][0], a[PA[pq]][0], a[PA[pq]][1], b[PB[pq]][0]);
                mma_bf16_k8(acc[0][1], a[PA[pq]][0], a[PA[pq]][1], b[PB[pq]][1]);
              }
            } else {
#pragma unroll
              for (int pq = 0; pq < 6; pq++)
                mma_bf16_k8(acc[0][0], a[PA[pq]][0], a[PA[pq]][1], b[PB[pq]][0]);
            }
          } else {
            uint32_t a[3][4], b[3][4];
#pragma unroll
            for (int q3 = 0; q3 < 3; q3++) {
              ldsm_x4(a[q3][0], a[q3][1], a[q3][2], a[q3][3], adL + q3 * lpl + koL);
              ldsm_x4(b[q3][0], b[q3][1], b[q3][2], b[q3][3], adR + q3 * rpl + koR);
            }
            if (two) {
#pragma unroll
              for (int pq = 0; pq < 6; pq++) {
                mma_bf16_k16(acc[0][0], a[PA[pq]], b[PB[pq]][0], b[PB[pq]][1]);
                mma_bf16_k16(acc[0][1], a[PA[pq]], b[PB[pq]][2], b[PB[pq]][3]);
              }
            } else {
#pragma unroll
              for (int pq = 0; pq < 6; pq++)
                mma_bf16_k16(acc[0][0], a[PA[pq]], b[PB[pq]][0], b[PB[pq]][1]);
            }
          }
        }
      } else {
        constexpr int PA[3] = {1, 0, 0};
        constexpr int PB[3] = {0, 1, 0};
        for (int kk = 0; kk < s; kk += 8) {
          const uint32_t koL = 16u * (uint32_t)((kk >> 2) * Mp), koR = 16u * (uint32_t)((kk >> 2) * Np);
          uint32_t a[2][4], b[2][4];
          if (s - kk <= 4) {  // one k piece left: the other half is zero
#pragma unroll
            for (int q2 = 0; q2 < 2; q2++) {
              ldsm_x2(a[q2][0], a[q2][1], adL + q2 * lpl + koL);
              ldsm_x2(b[q2][0], b[q2][2], adR2 + q2 * rpl + koR);
              a[q2][2] = a[q2][3] = b[q2][1] = b[q2][3] = 0u;
            }
          } else {
#pragma unroll
            for (int q2 = 0; q2 < 2; q2++) {
              ldsm_x4(a[q2][0], a[q2][1], a[q2][2], a[q2][3], adL + q2 * lpl + koL);
              ldsm_x4(b[q2][0], b[q2][1], b[q2][2], b[q2][3], adR + q2 * rpl + koR);
            }
          }
          if (two) {
#pragma unroll
            for (int pq = 0; pq < 3; pq++) {
              mma_tf32_k8(acc[0][0], a[PA[pq]], b[PB[pq]][0], b[PB[pq]][1]);
              mma_tf32_k8(acc[0][1], a[PA[pq]], b[PB[pq]][2], b[PB[pq]][3]);
            }
          } else {
#pragma unroll
            for (int pq = 0; pq < 3; pq++)
              mma_tf32_k8(acc[0][0], a[PA[pq]], b[PB[pq]][0], b[PB[pq]][1]);
          }
        }
      }
      }
      // every kFold products (and after the last): fold the FP32 partial sum
      // into the compensated running sum
      if ((q % kFold) == kFold - 1 || q == cur.np - 1) {
#pragma unroll
        for (int mt = 0; mt < MT; mt++)
#pragma unroll
          for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int x = 0; x < 4; x++) {
              two_sum_acc(hi[mt][nt][x], lo[mt][nt][x], acc[mt][nt][x]);
              acc[mt][nt][x] = 0.f;
            }
      }
    }
    if (failed) break;

    const int64_t gb = cur.gb;
    const int cin = ws.c_cin[gb];
    const double *cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;
    double *out = C.vals + C.blk_off[gb];
    double *hblk = (C.host_vals && st->nnz_c <= C.host_cap) ? C.host_vals + C.blk_off[gb] : nullptr;
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
          // FP32 -> FP64 is exact; hi + lo rounded once in FP64
          double v = (double)hi[mt][nt][x] + (double)lo[mt][nt][x];
          if (!plain) {
            v = alpha * v;
            if (cinv) v = fma(beta, cinv[e], v);
          }
          out[e] = v;
          if (hblk) hblk[e] = v;
        }
      }

    // the next block (already begun if the ring ran into it)
    if (!have_nxt) {
      take(nxt);
      nxt_issued = 0;
    }
    cur = nxt;
    cur_issued = nxt_issued;
    have_nxt = false;
    __syncwarp();  // every lane is past its reads of the slots about to be refilled
    while (cur_issued < cur.np && (int)(u_issue - u_done) < STAGES - 1) issue(cur, cur_issued++);
  }
  if (failed && lane == 0) atomicOr(const_cast<int32_t *>(&st->error), 1);
  // copies still in flight into this warp's slots (none unless a wait gave up)
  for (uint32_t u = u_done; u < u_issue; u++)
    if (!mbar_wait(bar0 + 8 * (u % STAGES), (u / STAGES) & 1u)) break;
}

// ---------------------------------------------------------------------------
// Chunked kernel: the products of a C block concatenated along k. A warp
// computes one C block at a time (or its transpose, as the pipelined kernel
// chooses), for the C blocks whose MMA problem fits 16 x 16. The k pieces of
// the block's products, in ascending k, are staged chunk by chunk into shared
// memory. A chunk holds whole products, at most PCMAX 16-byte pieces of k, and
// each slice plane of L (and of R) is one k-piece-major plane of Mp (Np) rows
// in it, so the MMA loop runs over the chunk's pieces as over one long k
// whatever the products' boundaries: every product's pieces are zero past its
// own k. The copies are 16-byte cp.async from all lanes (one loop per operand
// and product over all its planes), double buffered as in the FP64 packed
// kernel, and the tensor cores' FP32 sums are folded into the compensated
// running sum once per chunk. Per product this leaves the copy loop and a
// table entry; the waits, the fold and the loop control come per chunk.
// ---------------------------------------------------------------------------
constexpr int kCatWarps = 4;
constexpr int kCatMeta = 32;  // product table entries (one batch)

// Bytes of one operand buffer: every plane of up to 16 rows and PCMAX pieces,
// and 256 bytes beyond, which the fragment loads of rows past Mp (or Np) in the
// last plane may touch (their results are never used).
template <int PREC, int PCMAX>
__host__ __device__ constexpr int cat_operand_bytes() {
  return (PREC == BSM_PREC_SPLIT_BF16X3 ? 3 : 2) * 16 * PCMAX * 16 + 256;
}
template <int PREC, int PCMAX>
__host__ __device__ constexpr int cat_warp_bytes() {
  return 2 * 2 * cat_operand_bytes<PREC, PCMAX>() + kCatMeta * (8 + 8 + 4);
}

__device__ __forceinline__ void cpa16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int PREC, int PCMAX>
__global__ void __launch_bounds__(kCatWarps * 32)
    k_numeric_split_cat(DevMat A, DevMat B, DevOut C, DevMat Cin, const void *__restrict__ a_left,
                        const void *__restrict__ b_right, double alpha, double beta, DevWs ws,
                        const DevStatus *st, const int32_t *__restrict__ items,
                        const int64_t *__restrict__ seg, unsigned long long *work) {
  if (st->overflow) return;
  constexpr bool BF = (PREC == BSM_PREC_SPLIT_BF16X3);
  constexpr int NSL = BF ? 3 : 2;
  constexpr int VPP = BF ? 8 : 4;  // k values per 16-byte piece
  // a product's k (at most 16 for the small instances, 32 for the others)
  // fits one chunk; the launcher picks the instance by the largest k
  static_assert(PCMAX * VPP >= 16, "a chunk must hold the longest product (k <= 16 or 32)");
  constexpr int64_t kUnit = BF ? 2 * kBf16HalfwordsPerValue : 4 * kTf32WordsPerValue;
  constexpr int OPB = cat_operand_bytes<PREC, PCMAX>();
  extern __shared__ __align__(16) unsigned char smem_cat[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  unsigned char *wbase = smem_cat + warp * cat_warp_bytes<PREC, PCMAX>();
  const unsigned char **meta_a = reinterpret_cast<const unsigned char **>(wbase + 4 * OPB);
  const unsigned char **meta_b = meta_a + kCatMeta;
  int *meta_k = reinterpret_cast<int *>(meta_b + kCatMeta);  // pieces of k
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(wbase);
  // ldmatrix lane roles (as in the pipelined kernel)
  const int ra = (lane & 7) + ((lane >> 3) & 1) * 8, pa = lane >> 4;
  const int rb_ = (lane & 7) + (lane >> 4) * 8, pb = (lane >> 3) & 1;
  int64_t wb = 0, we = st->nblk_c;
  if (seg) {
    wb = seg[0];
    we = seg[1];
  }
  const bool plain = (alpha == 1.0 && beta == 0.0);
  double *hout = (C.host_vals && st->nnz_c <= C.host_cap) ? C.host_vals : nullptr;

  for (;;) {
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(work, 1ull);
    const int64_t w = wb + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    if (w >= we) break;
    const int64_t gb = items ? items[w] : w;
    const int i = C.blk_row[gb], j = C.col_idx[gb];
    const int m = C.row_sizes[i], n = C.col_sizes[j];
    const int tiles_n = ((m + 15) >> 4) * ((n + 7) >> 3);
    const int tiles_t = ((n + 15) >> 4) * ((m + 7) >> 3);
    const bool tr = tiles_t < tiles_n;
    const int Mp = tr ? n : m, Np = tr ? m : n;
    if (Mp > 16 || Np > 16) continue;  // the large-block instance of the pipelined kernel
    const bool two = Np > 8;
    const int64_t p0 = ws.prod_ptr[gb], p1 = ws.prod_ptr[gb + 1];
    // chunk plane strides of L (Mp rows) and R (Np rows)
    const uint32_t lpl = (uint32_t)(Mp * PCMAX * 16), rpl = (uint32_t)(Np * PCMAX * 16);
    float hi[2][4], lo[2][4], acc[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
      for (int x = 0; x < 4; x++) hi[nt][x] = lo[nt][x] = acc[nt][x] = 0.f;

    // product cursor: the next product to stage and the table batch holding it
    int64_t pq = p0, tbase = p0;
    int tcount = 0;
    // all planes of one operand of a product (rows x pk pieces each,
    // contiguous, planes one after another) into the chunk at piece poff
    auto copy_operand = [&](uint32_t dst, uint32_t plane, const unsigned char *src, int rows, int pk,
                            int poff) {
      const int U = rows * pk;  // 16-byte units of one plane
      const uint32_t d0 = dst + 16u * (uint32_t)(poff * rows);
      for (int u = lane; u < NSL * U; u += 32) {
        const int q = (u >= U) + ((NSL == 3 && u >= 2 * U) ? 1 : 0);
        cpa16(d0 + (uint32_t)q * plane + 16u * (uint32_t)(u - q * U), src + 16 * (int64_t)u);
      }
    };
    // stage whole products into buffer buf while they fit; returns the pieces
    auto fill = [&](int buf) -> int {
      const uint32_t dL = sbase + (uint32_t)(buf * 2 * OPB), dR = dL + (uint32_t)OPB;
      int poff = 0;
      while (pq < p1) {
        if (pq == tbase + tcount) {  // the next batch of the product table
          tbase = pq;
          tcount = (p1 - pq < kCatMeta) ? (int)(p1 - pq) : kCatMeta;
          __syncwarp();  // every lane is past its reads of the old batch
          if (lane < tcount) {
            const int2 pr = ws.prods[pq + lane];
            meta_a[lane] = static_cast<const unsigned char *>(a_left) + kUnit * A.blk_off[pr.x];
            meta_b[lane] = static_cast<const unsigned char *>(b_right) + kUnit * B.blk_off[pr.y];
            meta_k[lane] = (A.col_sizes[A.col_idx[pr.x]] + VPP - 1) / VPP;
          }
          __syncwarp();
        }
        const int e = (int)(pq - tbase);
        const int pk = meta_k[e];
        if (pk > PCMAX) {  // longer than a chunk (the launcher rules it out): error, block skipped
          if (lane == 0) atomicOr(const_cast<int32_t *>(&st->error), 1);
          pq = p1;
          break;
        }
        if (poff + pk > PCMAX) break;
        // not transposed: L = A_ik (left layout, m rows), R = B_kj (right layout, n rows)
        const unsigned char *sa = meta_a[e], *sb = meta_b[e];
        copy_operand(dL, lpl, tr ? sb : sa, Mp, pk, poff);
        copy_operand(dR, rpl, tr ? sa : sb, Np, pk, poff);
        poff += pk;
        pq++;
      }
      return poff;
    };

    int cur = fill(0);
    cpa_commit();
    for (int ch = 0;; ch++) {
      const int buf = ch & 1;
      const int nxt = (pq < p1) ? fill(buf ^ 1) : 0;
      cpa_commit();
      cpa_wait<1>();  // the current chunk has landed
      __syncwarp();
      const uint32_t sL = sbase + (uint32_t)(buf * 2 * OPB), sR = sL + (uint32_t)OPB;
      const uint32_t adL = sL + 16u * (uint32_t)(pa * Mp + ra);
      const uint32_t adR = sR + 16u * (uint32_t)(pb * Np + rb_);
      const uint32_t adR2 = sR + 16u * (uint32_t)ra;  // "a" order on R (single pieces)
      if (BF) {
        // slice products, smallest first: (3,1) (2,2) (1,3) (2,1) (1,2) (1,1)
        constexpr int PA[6] = {2, 1, 0, 1, 0, 0};
        constexpr int PB[6] = {0, 1, 2, 0, 1, 0};
        for (int p = 0; p < cur; p += 2) {
          const uint32_t koL = 16u * (uint32_t)(p * Mp), koR = 16u * (uint32_t)(p * Np);
          if (cur - p == 1) {  // one piece left: m16n8k8
            uint32_t a[3][2], b[3][2];
#pragma unroll
            for (int q3 = 0; q3 < 3; q3++) {
              ldsm_x2(a[q3][0], a[q3][1], adL + q3 * lpl + koL);
              ldsm_x2(b[q3][0], b[q3][1], adR2 + q3 * rpl + koR);
            }
#pragma unroll
            for (int x = 0; x < 6; x++) {
              mma_bf16_k8(acc[0], a[PA[x]][0], a[PA[x]][1], b[PB[x]][0]);
              if (two) mma_bf16_k8(acc[1], a[PA[x]][0], a[PA[x]][1], b[PB[x]][1]);
            }
          } else {
            uint32_t a[3][4], b[3][4];
#pragma unroll
            for (int q3 = 0; q3 < 3; q3++) {
              ldsm_x4(a[q3][0], a[q3][1], a[q3][2], a[q3][3], adL + q3 * lpl + koL);
              ldsm_x4(b[q3][0], b[q3][1], b[q3][2], b[q3][3], adR + q3 * rpl + koR);
            }
#pragma unroll
            for (int x = 0; x < 6; x++) {
              mma_bf16_k16(acc[0], a[PA[x]], b[PB[x]][0], b[PB[x]][1]);
              if (two) mma_bf16_k16(acc[1], a[PA[x]], b[PB[x]][2], b[PB[x]][3]);
            }
          }
        }
      } else {
        // (2,1) (1,2) (1,1)
        constexpr int PA[3] = {1, 0, 0};
        constexpr int PB[3] = {0, 1, 0};
        for (int p = 0; p < cur; p += 2) {
          const uint32_t koL = 16u * (uint32_t)(p * Mp), koR = 16u * (uint32_t)(p * Np);
          uint32_t a[2][4], b[2][4];
          if (cur - p == 1) {  // one piece left: the other half of the k step is zero
#pragma unroll
            for (int q2 = 0; q2 < 2; q2++) {
              ldsm_x2(a[q2][0], a[q2][1], adL + q2 * lpl + koL);
              ldsm_x2(b[q2][0], b[q2][2], adR2 + q2 * rpl + koR);
              a[q2][2] = a[q2][3] = b[q2][1] = b[q2][3] = 0u;
            }
          } else {
#pragma unroll
            for (int q2 = 0; q2 < 2; q2++) {
              ldsm_x4(a[q2][0], a[q2][1], a[q2][2], a[q2][3], adL + q2 * lpl + koL);
              ldsm_x4(b[q2][0], b[q2][1], b[q2][2], b[q2][3], adR + q2 * rpl + koR);
            }
          }
#pragma unroll
          for (int x = 0; x < 3; x++) {
            mma_tf32_k8(acc[0], a[PA[x]], b[PB[x]][0], b[PB[x]][1]);
            if (two) mma_tf32_k8(acc[1], a[PA[x]], b[PB[x]][2], b[PB[x]][3]);
          }
        }
      }
      // the chunk's FP32 partial sums into the compensated running sum
#pragma unroll
      for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int x = 0; x < 4; x++) {
          two_sum_acc(hi[nt][x], lo[nt][x], acc[nt][x]);
          acc[nt][x] = 0.f;
        }
      __syncwarp();  // the buffer is read before it is filled again
      if (nxt == 0) break;
      cur = nxt;
    }
    cpa_wait<0>();
    __syncwarp();

    const int cin = ws.c_cin[gb];
    const double *cinv = (cin >= 0) ? Cin.vals + Cin.blk_off[cin] : nullptr;
    double *out = C.vals + C.blk_off[gb];
    double *hblk = hout ? hout + C.blk_off[gb] : nullptr;
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int rr = g + ((x >> 1) << 3);
        const int cc = nt * 8 + 2 * t + (x & 1);
        if (rr < Mp && cc < Np) {
          const int row = tr ? cc : rr, col = tr ? rr : cc;
          const int64_t e = (int64_t)col * m + row;
          // FP32 -> FP64 is exact; hi + lo rounded once in FP64
          double v = (double)hi[nt][x] + (double)lo[nt][x];
          if (!plain) {
            v = alpha * v;
            if (cinv) v = fma(beta, cinv[e], v);
          }
          out[e] = v;
          if (hblk) hblk[e] = v;
        }
      }
  }
}

// The pipelined kernel's bounded barrier wait on its own: lane 0 completes the
// phase (a plain arrive), unless never_complete; the warp then waits as the
// kernel does and records in *flag whether the wait gave up.
__global__ void k_wait_selftest(int never_complete, int32_t *flag) {
  __shared__ __align__(8) unsigned long long bar_storage;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_storage);
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncwarp();
  if (lane == 0 && !never_complete)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
  const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, 0u));
  if (lane == 0) *flag = ok ? 0 : 1;
}

cudaError_t launch_wait_selftest(int never_complete, int32_t *flag, cudaStream_t stream) {
  k_wait_selftest<<<1, 32, 0, stream>>>(never_complete, flag);
  return cudaGetLastError();
}

// [precision: BF16x3, TF32x2][0: the small-block instance, 1: the large-block one]
static const void *const (&pipe_instances())[2][2] {
  static const void *const inst[2][2] = {
      {(const void *)k_numeric_split_pipe<BSM_PREC_SPLIT_BF16X3, 2, false>,
       (const void *)k_numeric_split_pipe<BSM_PREC_SPLIT_BF16X3, 2, true>},
      {(const void *)k_numeric_split_pipe<BSM_PREC_SPLIT_TF32X2, 2, false>,
       (const void *)k_numeric_split_pipe<BSM_PREC_SPLIT_TF32X2, 2, true>}};
  return inst;
}

cudaError_t launch_numeric_split(int precision, int sizes, DevMat A, DevMat B, DevOut C,
                                 DevMat Cin, const void *a_left, const void *b_right, double alpha,
                                 double beta, DevWs ws, const DevStatus *st, const int32_t *items,
                                 const int64_t *seg, int smax, int nsm, unsigned long long *work,
                                 cudaStream_t stream) {
  const int pi = precision == BSM_PREC_SPLIT_BF16X3 ? 0 : 1;
  const bool big = sizes == 2;  // C blocks beyond 16x16: the large-block instance
  constexpr int stages = kPipeStages;
  const int warps = big ? kPipeWarpsBig : kPipeWarps;
  const size_t smem = (size_t)warps * pipe_warp_bytes(precision, smax, stages, big ? 32 : 16);
  const void *fn = pipe_instances()[pi][big ? 1 : 0];
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
  if (e != cudaSuccess) return e;
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
  const int sel = sizes;  // 0 all, 1 small C blocks only, 2 large ones only
#define BSM_SPLIT_PIPE(P, G)                                                                    \
  k_numeric_split_pipe<P, stages, G><<<grid, warps * 32, smem, stream>>>(                       \
      A, B, C, Cin, a_left, b_right, alpha, beta, ws, st, items, seg, smax, sel, work)
  if (precision == BSM_PREC_SPLIT_BF16X3) {
    if (big) BSM_SPLIT_PIPE(BSM_PREC_SPLIT_BF16X3, true);
    else BSM_SPLIT_PIPE(BSM_PREC_SPLIT_BF16X3, false);
  } else {
    if (big) BSM_SPLIT_PIPE(BSM_PREC_SPLIT_TF32X2, true);
    else BSM_SPLIT_PIPE(BSM_PREC_SPLIT_TF32X2, false);
  }
#undef BSM_SPLIT_PIPE
  return cudaGetLastError();
}

// Chunk capacity (16-byte pieces of k) of the chunked instances: the smaller
// where every k is at most 16 (the water blocks), the larger for k up to 32.
// Smaller chunks leave more warps per SM, which this kernel needs (water2048,
// BF16x3: 8 pieces 29.0 ms, 4 pieces 17.8 ms, 2 pieces 17.6 ms; TF32x2: 8
// pieces 23.4 ms, 4 pieces 18.8 ms).
constexpr int kCatPiecesBf16Small = 2, kCatPiecesBf16 = 4;
constexpr int kCatPiecesTf32Small = 4, kCatPiecesTf32 = 8;
template <int PREC, int PCMAX>
static const void *cat_fn() {
  return (const void *)k_numeric_split_cat<PREC, PCMAX>;
}

cudaError_t launch_numeric_split_cat(int precision, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                     const void *a_left, const void *b_right, double alpha,
                                     double beta, DevWs ws, const DevStatus *st,
                                     const int32_t *items, const int64_t *seg, int smax, int nsm,
                                     unsigned long long *work, cudaStream_t stream) {
  const bool bf = precision == BSM_PREC_SPLIT_BF16X3, small = smax <= 16;
  constexpr int BF = BSM_PREC_SPLIT_BF16X3, TF = BSM_PREC_SPLIT_TF32X2;
  const void *fn = bf ? (small ? cat_fn<BF, kCatPiecesBf16Small>() : cat_fn<BF, kCatPiecesBf16>())
                      : (small ? cat_fn<TF, kCatPiecesTf32Small>() : cat_fn<TF, kCatPiecesTf32>());
  const size_t smem =
      (size_t)kCatWarps * (bf ? (small ? cat_warp_bytes<BF, kCatPiecesBf16Small>() : cat_warp_bytes<BF, kCatPiecesBf16>())
                              : (small ? cat_warp_bytes<TF, kCatPiecesTf32Small>() : cat_warp_bytes<TF, kCatPiecesTf32>()));
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCatWarps * 32, smem);
  if (e != cudaSuccess) return e;
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
#define BSM_SPLIT_CAT(P, PC)                                                              \
  k_numeric_split_cat<P, PC><<<grid, kCatWarps * 32, smem, stream>>>(A, B, C, Cin, a_left, \
                                                                    b_right, alpha, beta, ws, \
                                                                    st, items, seg, work)
  if (bf) {
    if (small) BSM_SPLIT_CAT(BF, kCatPiecesBf16Small);
    else BSM_SPLIT_CAT(BF, kCatPiecesBf16);
  } else {
    if (small) BSM_SPLIT_CAT(TF, kCatPiecesTf32Small);
    else BSM_SPLIT_CAT(TF, kCatPiecesTf32);
  }
#undef BSM_SPLIT_CAT
  return cudaGetLastError();
}

cudaError_t numeric_split_init() {
  {
    constexpr int BF = BSM_PREC_SPLIT_BF16X3, TF = BSM_PREC_SPLIT_TF32X2;
    const void *fn[4] = {cat_fn<BF, kCatPiecesBf16Small>(), cat_fn<BF, kCatPiecesBf16>(),
                         cat_fn<TF, kCatPiecesTf32Small>(), cat_fn<TF, kCatPiecesTf32>()};
    const int bytes[4] = {kCatWarps * cat_warp_bytes<BF, kCatPiecesBf16Small>(),
                          kCatWarps * cat_warp_bytes<BF, kCatPiecesBf16>(),
                          kCatWarps * cat_warp_bytes<TF, kCatPiecesTf32Small>(),
                          kCatWarps * cat_warp_bytes<TF, kCatPiecesTf32>()};
    for (int x = 0; x < 4; x++) {
      cudaError_t e = cudaFuncSetAttribute(fn[x], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes[x]);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn[x], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      if (e != cudaSuccess) return e;
    }
  }
  // the largest slot layout of each instance (k up to 32), and the whole
  // shared memory of an SM for the carveout (the rings decide occupancy)
  for (int pi = 0; pi < 2; pi++)
    for (int big = 0; big < 2; big++) {
      const int prec = pi == 0 ? BSM_PREC_SPLIT_BF16X3 : BSM_PREC_SPLIT_TF32X2;
      const int bytes = big ? kPipeWarpsBig * pipe_warp_bytes(prec, 32, kPipeStages, 32)
                            : kPipeWarps * pipe_warp_bytes(prec, 32, kPipeStages, 16);
      const void *fn = pipe_instances()[pi][big];
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace bsm
