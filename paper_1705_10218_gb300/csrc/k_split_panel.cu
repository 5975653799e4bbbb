// k_split_panel.cu -- the split-precision numeric phase on the fifth-generation
// tensor cores (tcgen05): one C block row at a time as a dense panel product.
//
// The paper's local multiply is a batch of small block products (Sec. 2). For
// the split precisions (BF16x3, TF32x2; the slices are cut in k_split.cu)
// those products are regrouped here into one GEMM per C block row i:
//
//     C_i,:^T  =  B_{N(i),:}^T  .  A_i,:^T
//
//   M = the C columns of row i (the C blocks (i, j) side by side), in tiles of
//       up to 128 (whole C blocks, at most 32 of them),
//   N = r_i (the row's block size), padded to NR = 16 or 32, times the slices,
//   K = the slices' k pieces of A's row i concatenated (blocks in ascending k).
//
// The A operand of the MMA (M x K) is the transposed B panel: the pieces of the
// kept products' B_kj at (columns of j, pieces of k), zero where (k, j) is not a
// kept product (missing, or dropped by the filter: the symbolic phase's product
// lists decide, so the result pattern and the set of products are exactly those
// of the other paths). It is gathered into tensor memory (TMEM) by four warps,
// one TMEM lane per C column. The B operand (K x N) is A's row i: its slice
// pieces staged once per row (or per segment of the row, see below) in shared
// memory, the slices stacked along N so one MMA multiplies a B slice by several
// A slices at once:
//
//   BF16x3: B slice 1 x [A1 A2 A3] (N = 3 NR), B slice 2 x [A1 A2] (N = 2 NR),
//           B slice 3 x [A1] (N = NR), accumulated into three column groups of
//           the FP32 accumulator: (1,1); (2,1)+(1,2); (3,1)+(2,2)+(1,3) -- the
//           six slice products with p + q <= 4;
//   TF32x2: B slice 1 x [A1 A2] (N = 2 NR), B slice 2 x [A1] (N = NR): (1,1);
//           (2,1)+(1,2).
//
// The accumulator of a tile lives in TMEM (FP32, 128 lanes x groups x NR); the
// epilogue reads it with tcgen05.ld, adds the groups (small ones first, the last
// addition as an exact TwoSum pair), forms C in FP64 with alpha and beta, and
// writes each C column (r_i contiguous doubles of a column-major block).
//
// Roles of the ten warps of a CTA (one CTA per SM, persistent):
//   warp 9     loader: takes C block rows from a work counter, stages A's row
//              slices (bulk copies), cuts the row's C blocks into tiles and A's
//              row into chunks of at most 8 pieces, and for each (tile, chunk)
//              copies the B blocks of the kept products into a shared-memory
//              stage with bulk asynchronous copies (one per product, all slice
//              planes), with a table (C block, A block) -> stage offset;
//   warps 0-3  gather: build the chunk's A operand in TMEM from the stage
//              (16-byte shared loads, zeros for absent products, tcgen05.st);
//   warp 8     MMA: one thread issues the tcgen05.mma of each chunk and commits
//              them to mbarriers that free the TMEM stage and, after a tile's
//              last chunk, hand the accumulator to the epilogue;
//   warps 4-7  epilogue: TMEM -> registers -> FP64 C.
// Rings of mbarriers connect them: stages (loader -> gather), TMEM operand
// stages (gather -> MMA), accumulators (MMA -> epilogue, double buffered), tile
// headers (loader -> gather, epilogue). Every wait is bounded: a wait that gives
// up raises the status error flag (BSM_ERR_TIMEOUT on the host) and the warp
// leaves its loop; the others then give up too, in-flight copies and MMAs are
// waited for (bounded) and the TMEM is freed.
//
// Rows whose A pieces do not fit the shared-memory operand buffer are cut into
// segments of A blocks: each segment is a pass over all tiles of the row, the
// first one storing C and the later ones adding their partial products to it
// in FP64.
#include <cstddef>
#include <cstdint>

#include "bsm_internal.h"

namespace bsm {
namespace {

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// explicit shared-space accesses (32-bit addresses): short-latency loads
// where a generic pointer would go through the global path
__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ int lds32(uint32_t a) {
  int v;
  asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int2 lds64(uint32_t a) {
  int2 v;
  asm volatile("ld.shared.v2.b32 {%0,%1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds8(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1];\n" : "=r"(v) : "r"(a));
  return (int)v;
}
__device__ __forceinline__ void pb_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void pb_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void pb_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
// adds bytes to the pending transaction count of the current phase (no arrival)
__device__ __forceinline__ void pb_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
constexpr uint32_t kHintNs = 1000;
// about a second of suspended polling before a wait gives up
constexpr int kPolls = 1 << 20;
__device__ __forceinline__ bool pb_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kHintNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool pb_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kPolls; i++)
    if (pb_test(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// generic-proxy shared-memory writes before async-proxy reads (tensor core)
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(holder),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// D (TMEM) [+]= A (TMEM) x B (shared memory descriptor)
template <bool TF32>
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc,
                                       uint32_t acc) {
  if (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// the mbarrier completes once every tcgen05 operation this thread issued before
// has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int x = 0; x < 16; x++) r[x] = __uint_as_float(u[x]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
// Shared-memory matrix descriptor, K-major without swizzle: core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo = along
// M / N; bit 46 is the descriptor version of this architecture.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor: FP32 accumulator, A and B of type ab (1 BF16, 2
// TF32), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t ab, uint32_t n, uint32_t m) {
  return (1u << 4) | (ab << 7) | (ab << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Configuration and shared-memory layout
// ---------------------------------------------------------------------------
constexpr int kWarps = 11;
constexpr int kGatherWarp0 = 0, kEpiWarp0 = 4, kMmaWarp = 8, kLoaderWarp = 9;  // loaders: 9, 10
constexpr int kMaxSegChunks = 256;  // chunks of one segment (at most its pieces)
constexpr int kMailWords = 8;       // the loaders' shared words (multiple of 4: 16-byte layout)
constexpr int kTileCols = 128;      // MMA M: C columns per tile
constexpr int kMaxSlots = 32;       // C blocks per tile
constexpr int kChunkPieces = 8;     // K pieces (16 bytes of every slice) per chunk
static_assert(kChunkPieces % 4 == 0 && kChunkPieces <= 32, "chunk table rows of whole int4");
constexpr int kStages = 3;          // loader -> gather stages
constexpr int kStageBytes = 16384;  // B blocks of one (tile, chunk)
constexpr int kTileRing = 4;        // tile headers in flight
constexpr int kTaMax = 6;           // TMEM operand stages at most (as many as the columns allow)
constexpr int kNaMax = 512;         // A blocks per row of the panel path (longer rows: per-block kernel)
constexpr int kRecMax = kNaMax;     // so every tile has at most this many product records
constexpr uint32_t kTmemCols = 512;
constexpr int kSmemLimit = 232448;  // dynamic shared memory of one CTA (227 KB)

// flags of chunk headers, TMEM stage notes and tile headers
enum : int32_t {
  kFirstChunk = 1,    // first chunk of a tile: the accumulator starts at zero
  kLastChunk = 2,     // last chunk of a tile: the accumulator goes to the epilogue
  kFirstSegChunk = 4, // first chunk of a segment: wait for the B operand
  kLastSegChunk = 8,  // last chunk of a segment: the B operand may be replaced
  kEnd = 16,          // no more work
  kAccum = 32,        // tile of a later segment: add to C
  kLastSeg = 64       // tile of the row's last segment (host copy of C)
};

template <int PREC, int NR>
struct PanelCfg {
  static constexpr bool TF = (PREC == BSM_PREC_SPLIT_TF32X2);
  static constexpr int NSL = TF ? 2 : 3;        // slices per operand
  static constexpr int PIECE = TF ? 4 : 8;      // values per 16-byte piece
  static constexpr int64_t UNIT = TF ? 4 * kTf32WordsPerValue : 2 * kBf16HalfwordsPerValue;
  static constexpr int PB = NSL * NR * 16;      // bytes of one K piece of the B operand
  static constexpr int DC = NSL * NR;           // accumulator columns of one tile
  static constexpr int PC = 4 * kChunkPieces;   // TMEM columns of one slice plane of a stage
  static constexpr int AC = NSL * PC;           // TMEM columns of an operand stage
  static constexpr int ABASE = 2 * DC;          // operand stages follow two accumulators
  static constexpr int TA = ((int)kTmemCols - ABASE) / AC < kTaMax ? ((int)kTmemCols - ABASE) / AC : kTaMax;
  static_assert(TA >= 2 && ABASE + TA * AC <= (int)kTmemCols, "TMEM columns");
};

struct ChunkHdr {
  int32_t flags, tile, pi0, npieces;
  // per slot and K piece of a product the stage had no room for: the piece's
  // first row in B's slices in 16-byte units (the gather reads global memory)
  int32_t farb[kMaxSlots][kChunkPieces];
  // per slot and K piece of the chunk: 0 no product; else kPiecePresent |
  // (kPieceFar: in global memory, see farb) | the piece's first row in the
  // stage in 16-byte units (bits 0-10) | the slice plane stride in 16-byte
  // units (bits 11-19)
  int32_t ptab[kMaxSlots][kChunkPieces];
};
constexpr int32_t kPiecePresent = 1 << 30, kPieceFar = 1 << 29;
struct TileHdr {
  int32_t flags, r, nslots, pad;
  int32_t gb[kMaxSlots];          // C block of each slot
  uint8_t cj[kMaxSlots];          // its column count
  uint8_t mst[kMaxSlots];         // its first column in the tile
  uint8_t col_slot[kTileCols];    // slot of each column, 255: none
};
struct TaNote {
  int32_t flags, pi0, npieces, tile;
};
struct Bars {
  uint64_t stg_full[kStages], stg_empty[kStages];
  uint64_t ta_full[kTaMax], ta_empty[kTaMax];
  uint64_t d_full[2], d_empty[2];
  uint64_t tile_full[kTileRing], tile_empty[kTileRing];
  uint64_t bop_full, bop_free, fin;
  uint32_t tmem_holder, pad;
  uint4 zero;  // 16 zero bytes: what the gather reads for an absent product
};
static_assert(sizeof(ChunkHdr) % 16 == 0 && sizeof(TileHdr) % 16 == 0, "16-byte layout");

// bytes after the B operand buffer: segment block table (pmax words), stages,
// record buffers, tile entries, headers, notes, barriers
__host__ __device__ constexpr int panel_fixed_bytes(int pmax) {
  return ((pmax * 4 + 15) & ~15) + kStages * kStageBytes + 2 * kRecMax * 16 + 3 * 64 +
         kMaxSegChunks * 16 + ((pmax * 2 + 15) & ~15) + ((2 * (kMaxSegChunks + 1) + 15) & ~15) +
         kMailWords * 4 + kStages * (int)sizeof(ChunkHdr) + kTileRing * (int)sizeof(TileHdr) +
         kTaMax * (int)sizeof(TaNote) + (((int)sizeof(Bars) + 15) & ~15);
}
// the largest K pieces per segment that fit, one of them the zero pad piece
__host__ __device__ constexpr int panel_pmax(int pb) {
  int p = (kSmemLimit - panel_fixed_bytes(0)) / (pb + 4);
  while (p > 0 && p * pb + panel_fixed_bytes(p) > kSmemLimit) p--;
  return p;
}
__host__ __device__ constexpr int panel_smem_bytes(int pb) {
  return panel_pmax(pb) * pb + panel_fixed_bytes(panel_pmax(pb));
}

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  return x;
}

struct PanelSmem {
  unsigned char *bop;     // B operand: pmax pieces x PB bytes
  int32_t *sblk;          // per block of the segment: first piece << 8 | pieces
  unsigned char *stage;   // kStages x kStageBytes
  int4 *rbuf;             // 2 x kRecMax product records of tiles
  int4 *ering;            // 3 tile entries of 64 bytes
  int4 *sch;              // the segment's chunks: {first piece, pieces, first block, blocks}
  int16_t *cho;           // chunk of each block of the segment
  int16_t *crs;           // first record of each chunk of the current tile (+ end)
  int32_t *mail;          // kMailWords: the loaders' row, segment end, pieces, chunks, failed flag

  ChunkHdr *chdr;
  TileHdr *thdr;
  TaNote *note;
  Bars *bars;
};

__device__ __forceinline__ PanelSmem panel_carve(unsigned char *base, int pmax, int pb) {
  PanelSmem p;
  p.bop = base;
  unsigned char *x = base + (size_t)pmax * pb;
  p.sblk = reinterpret_cast<int32_t *>(x);
  x += (pmax * 4 + 15) & ~15;
  p.stage = x;
  x += kStages * kStageBytes;
  p.rbuf = reinterpret_cast<int4 *>(x);
  x += 2 * kRecMax * 16;
  p.ering = reinterpret_cast<int4 *>(x);
  x += 3 * 64;
  p.sch = reinterpret_cast<int4 *>(x);
  x += kMaxSegChunks * 16;
  p.cho = reinterpret_cast<int16_t *>(x);
  x += (pmax * 2 + 15) & ~15;
  p.crs = reinterpret_cast<int16_t *>(x);
  x += (2 * (kMaxSegChunks + 1) + 15) & ~15;
  p.mail = reinterpret_cast<int32_t *>(x);
  x += kMailWords * 4;
  p.chdr = reinterpret_cast<ChunkHdr *>(x);
  x += kStages * sizeof(ChunkHdr);
  p.thdr = reinterpret_cast<TileHdr *>(x);
  x += kTileRing * sizeof(TileHdr);
  p.note = reinterpret_cast<TaNote *>(x);
  x += kTaMax * sizeof(TaNote);
  p.bars = reinterpret_cast<Bars *>(x);
  return p;
}

struct PanelArgs {
  DevMat A, B, Cin;
  DevOut C;
  const unsigned char *a_left, *b_right;
  double alpha, beta;
  DevWs ws;
  PanelWs pw;
  const DevStatus *st;
  unsigned long long *work;
  int32_t pmax;
};

#define PB_BAR(field) smem_u32(&sm.bars->field)

// ---------------------------------------------------------------------------
// Tiles of a C block row: runs of whole C blocks from cb with at most 128
// columns, 32 blocks and kRecMax kept products (one block alone may exceed the
// products' limit). One warp; returns the block count, the column count and
// the first / end product record; cj: this lane's block's column count.
// ---------------------------------------------------------------------------
__device__ int panel_next_tile(const DevOut &C, const DevWs &ws, int cb, int c1, int lane,
                               int &width, int &cj, int64_t &P0, int64_t &P1) {
  const int g = cb + lane;
  cj = 0;
  int64_t pp = 0, pn = 0;
  if (g < c1) {
    cj = C.col_sizes[C.col_idx[g]];
    pp = ws.prod_ptr[g];
    pn = ws.prod_ptr[g + 1] - pp;
  }
  const int ic = warp_incl_scan(cj, lane);
  const int ip = warp_incl_scan((int)(pn < kRecMax + 1 ? pn : kRecMax + 1), lane);
  const bool fits = g < c1 && ic <= kTileCols && ip <= kRecMax;
  int ns = __popc(__ballot_sync(0xffffffffu, fits));
  if (ns == 0) ns = 1;
  width = __shfl_sync(0xffffffffu, ic, ns - 1);
  P0 = __shfl_sync(0xffffffffu, pp, 0);
  P1 = __shfl_sync(0xffffffffu, pp + pn, ns - 1);
  return ns;
}

// ---------------------------------------------------------------------------
// Prep: per C block row, its tiles and each tile's product records ordered by
// A block (a counting sort on the block position; within one position the
// order does not matter), with each record's place in its (tile, chunk) stage.
// One CTA of 256 threads per row at a time. The row's segments and chunks are
// cut by the same rule as in the loader (segments: blocks with at most pmax - 2
// pieces; chunks: blocks with at most kChunkPieces pieces, never across a
// segment).
// A record (16 bytes):
//   x = the B block's slice offset in 16-byte units;
//   y = the A block's position in the row (bits 0-11) | the C block's slot in
//       the tile (bits 12-16) | its offset in the chunk's stage in 16-byte
//       units (bits 17-26) | 1 << 27 when the stage had no room (the gather
//       reads it from global memory) | 1 << 28 on the first record of a copy
//       group;
//   z = on a group's first record: the group's length in 16-byte units (the
//       records of one A block in a tile, contiguous in B's row: one copy);
//   w = the block's first K piece in the chunk (bits 0-3) | its pieces (bits
//       4-7) | the slice plane stride in 16-byte units, columns x pieces
//       (bits 8-16).
// ---------------------------------------------------------------------------
constexpr int kPrepThreads = 256;
__device__ __forceinline__ int rec_apos(int y) { return y & 0xFFF; }
__device__ __forceinline__ int rec_slot(int y) { return (y >> 12) & 31; }
__device__ __forceinline__ int rec_off16(int y) { return (y >> 17) & 1023; }
__device__ __forceinline__ bool rec_far(int y) { return (y >> 27) & 1; }
__device__ __forceinline__ bool rec_head(int y) { return (y >> 28) & 1; }
constexpr int kRecFar = 1 << 27, kRecHead = 1 << 28;
static_assert(kNaMax <= 4096 && kMaxSlots <= 32 && kStageBytes <= 16384 && kChunkPieces <= 15,
              "record bit fields");

__global__ void __launch_bounds__(kPrepThreads) k_panel_prep(DevMat A, DevMat B, DevOut C, DevWs ws,
                                                              PanelWs pw, const DevStatus *st,
                                                              int unit16, int nsl, int piece,
                                                              int pmax) {
  if (st->overflow) return;
  __shared__ int32_t hist[kNaMax];
  __shared__ uint8_t np_s[kNaMax];
  __shared__ int16_t pi_s[kNaMax];   // a block's first piece in its segment
  __shared__ int16_t cs[kNaMax + 1];
  __shared__ int4 srec[kRecMax];
  __shared__ int64_t sstart[kMaxSlots + 1];
  __shared__ int32_t t_ns, t_width, t_nch;
  __shared__ int64_t t_P0, t_P1;
  __shared__ __align__(16) uint8_t t_cj[kMaxSlots];  // also read as two 16-byte words
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = blockIdx.x; i < A.nbr; i += gridDim.x) {
    const int32_t c0 = C.row_ptr[i], c1 = C.row_ptr[i + 1];
    const int32_t a0 = A.row_ptr[i], na = A.row_ptr[i + 1] - a0;
    if (c1 <= c0) {
      if (tid == 0) pw.row_nt[i] = 0;
      continue;
    }
    if (na > kNaMax) {  // left to the per-block kernel
      if (tid == 0) pw.row_nt[i] = -1;
      for (int g = c0 + tid; g < c1; g += kPrepThreads)
        pw.fb_items[atomicAdd(reinterpret_cast<unsigned long long *>(&pw.fb_seg[1]), 1ull)] = g;
      continue;
    }
    // pieces of the row's A blocks, and its chunks
    for (int b = tid; b < na; b += kPrepThreads)
      np_s[b] = (uint8_t)((A.col_sizes[A.col_idx[a0 + b]] + piece - 1) / piece);
    __syncthreads();
    if (tid == 0) {
      int seg = 0, chunk = 0, nch = 0;
      for (int b = 0; b < na; b++) {
        const int np = np_s[b];
        bool start = b == 0;
        if (seg + np > pmax - 2) {
          seg = 0;
          start = true;
        } else if (chunk + np > kChunkPieces) {
          start = true;
        }
        if (start) {
          cs[nch++] = (int16_t)b;
          chunk = 0;
        }
        pi_s[b] = (int16_t)seg;
        chunk += np;
        seg += np;
      }
      cs[nch] = (int16_t)na;
      t_nch = nch;
    }
    __syncthreads();
    const int nch = t_nch;
    int nt = 0;
    for (int cb = c0; cb < c1;) {
      if (warp == 0) {
        int width, cj;
        int64_t P0, P1;
        const int ns = panel_next_tile(C, ws, cb, c1, lane, width, cj, P0, P1);
        if (lane < ns) {
          t_cj[lane] = (uint8_t)cj;
          sstart[lane] = ws.prod_ptr[cb + lane] - P0;
        } else {
          t_cj[lane] = 0;
        }
        if (lane == 0) {
          sstart[ns] = P1 - P0;
          t_ns = ns;
          t_width = width;
          t_P0 = P0;
          t_P1 = P1;
        }
      }
      for (int x = tid; x < na; x += kPrepThreads) hist[x] = 0;
      __syncthreads();
      const int ns = t_ns;
      const int64_t P0 = t_P0;
      const int n = (int)(t_P1 - t_P0);  // at most kRecMax: every A row has at most kNaMax blocks
      if (tid < 4) {
        int4 w;
        if (tid == 0) w = make_int4(cb, ns, (int)(uint32_t)P0, (int)(P0 >> 32));
        else if (tid == 1) w = make_int4((int)(uint32_t)t_P1, (int)(t_P1 >> 32), t_width, 0);
        else w = reinterpret_cast<const int4 *>(t_cj)[tid - 2];
        pw.tiles[4 * ((int64_t)c0 + nt) + tid] = w;
      }
      for (int k = tid; k < n; k += kPrepThreads) atomicAdd(&hist[ws.prods[P0 + k].x - a0], 1);
      __syncthreads();
      if (warp == 0) {  // exclusive prefix of the counts over the row's A blocks
        const int per = (na + 31) / 32;
        int sum = 0;
        for (int x = lane * per; x < na && x < (lane + 1) * per; x++) sum += hist[x];
        const int incl = warp_incl_scan(sum, lane);
        int run = incl - sum;
        for (int x = lane * per; x < na && x < (lane + 1) * per; x++) {
          const int c = hist[x];
          hist[x] = run;
          run += c;
        }
      }
      __syncthreads();
      for (int k = tid; k < n; k += kPrepThreads) {
        const int2 pr = ws.prods[P0 + k];
        const int apos = pr.x - a0;
        int lo = 0, hi = ns;  // slot: the last start <= k
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sstart[mid] <= k) lo = mid;
          else hi = mid;
        }
        const int pos = atomicAdd(&hist[apos], 1);  // hist[a] ends as the start of a + 1
        srec[pos] = make_int4((int)(unit16 * B.blk_off[pr.y]), apos | (lo << 12), 0, 0);
      }
      __syncthreads();
      // within one A block, ascending B offsets: the records of a block are then
      // consecutive blocks of B's row k, one contiguous range
      for (int x = tid; x < na; x += kPrepThreads) {
        const int b0 = x == 0 ? 0 : hist[x - 1], b1 = hist[x];
        for (int u = b0 + 1; u < b1; u++) {
          const int4 key = srec[u];
          int v = u - 1;
          while (v >= b0 && srec[v].x > key.x) {
            srec[v + 1] = srec[v];
            v--;
          }
          srec[v + 1] = key;
        }
      }
      __syncthreads();
      // copy groups and stage offsets: one thread per chunk, its records in order
      for (int c = tid; c < nch; c += kPrepThreads) {
        const int r0 = cs[c] == 0 ? 0 : hist[cs[c] - 1], r1 = hist[cs[c + 1] - 1];
        const int pi0 = pi_s[cs[c]];
        int used = 0;  // 16-byte units
        for (int k = r0; k < r1;) {
          const int apos = rec_apos(srec[k].y);
          int g1 = k + 1;
          while (g1 < r1 && rec_apos(srec[g1].y) == apos) g1++;
          const int np = np_s[apos];
          const int last = g1 - 1;
          const int len = srec[last].x + nsl * (int)t_cj[rec_slot(srec[last].y)] * np - srec[k].x;
          const bool staged = (used + len) * 16 <= kStageBytes;
          for (int u = k; u < g1; u++) {
            int4 rc = srec[u];
            const int cjs = t_cj[rec_slot(rc.y)];
            rc.y |= (staged ? (used + rc.x - srec[k].x) << 17 : kRecFar) | (u == k ? kRecHead : 0);
            rc.z = (u == k && staged) ? len : 0;
            rc.w = (pi_s[apos] - pi0) | (np << 4) | ((cjs * np) << 8);
            srec[u] = rc;
          }
          if (staged) used += len;
          k = g1;
        }
      }
      __syncthreads();
      for (int k = tid; k < n; k += kPrepThreads) pw.recs[P0 + k] = srec[k];
      __syncthreads();
      cb += ns;
      nt++;
    }
    if (tid == 0) pw.row_nt[i] = nt;
  }
}

// ---------------------------------------------------------------------------
// Loader (one warp): rows, segments, tiles, chunks; all bulk copies. The
// tiles' entries and product records (from the prep kernel) come through
// asynchronous copies into shared memory one and two tiles ahead, so the loop
// over chunks touches shared memory only. Returns false when a wait gave up.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct TileEntry {
  int cb0, ns, width;
  int64_t P0, P1;
};
__device__ __forceinline__ TileEntry read_entry(const int4 *e) {
  const int4 w0 = e[0], w1 = e[1];
  TileEntry t;
  t.cb0 = w0.x;
  t.ns = w0.y;
  t.P0 = (int64_t)(uint32_t)w0.z | ((int64_t)w0.w << 32);
  t.P1 = (int64_t)(uint32_t)w1.x | ((int64_t)w1.y << 32);
  t.width = w1.z;
  return t;
}

// the two loader warps
__device__ __forceinline__ void loaders_sync() {
  __syncwarp();  // the aligned barrier wants the warp converged
  asm volatile("bar.sync 1, 64;\n" ::: "memory");
}

template <int PREC, int NR>
__device__ bool panel_loader(const PanelArgs &a, const PanelSmem &sm, int lw, int lane) {
  using Cfg = PanelCfg<PREC, NR>;
  const DevMat &A = a.A;
  const DevOut &C = a.C;
  const int pmax = a.pmax;
  uint32_t seq_base = 0, tile_seq = 0, seg_seq = 0;
  const uint32_t bop = smem_u32(sm.bop);
  const uint32_t sblk_u = smem_u32(sm.sblk);
  volatile int32_t *mail = sm.mail;  // [0] row, [1] segment end, [2] its pieces, [3] its chunks, [4] failed
  if (lw == 0 && lane == 0) mail[4] = 0;
  loaders_sync();
  bool failed = false;
  // a wait that gives up marks the loaders failed; they keep to the barrier
  // protocol (no further waits) until both leave the row loop together
  auto wait = [&](uint32_t bar, uint32_t parity) {
    if (failed) return false;
    if (pb_wait(bar, parity)) return true;
    failed = true;
    mail[4] = 1;
    return false;
  };
  for (;;) {
    if (lw == 0 && lane == 0) {
      const unsigned long long w = atomicAdd(a.work, 1ull);
      mail[0] = (int)(w < (unsigned long long)A.nbr ? w : (unsigned long long)A.nbr);
    }
    loaders_sync();
    const int i = mail[0];
    failed = mail[4] != 0;
    loaders_sync();  // both have read the mailbox before it changes
    if (i >= A.nbr || failed) break;
    const int nt = a.pw.row_nt[i];
    if (nt <= 0) continue;  // no C blocks, or left to the per-block kernel
    const int32_t c0 = C.row_ptr[i];
    const int32_t a0 = A.row_ptr[i], na = A.row_ptr[i + 1] - a0;
    const int r = A.row_sizes[i];
    if (r > NR) {  // the host routes such rows elsewhere; never silently wrong
      if (lw == 0 && lane == 0) atomicOr(const_cast<int32_t *>(&a.st->error), 2);
      continue;
    }
    int sa = 0;
    for (;;) {  // segments of A's row
      if (lw == 0) {
        // blocks [sa, sb): at most pmax - 2 pieces (pieces P and P + 1 are zero
        // pads: a chunk's last K step may reach one piece past the segment, an
        // empty row's only step two)
        int sb = sa, P = 0;
        for (;;) {
          const int b = sb + lane;
          int np = 0;
          if (b < na) np = (A.col_sizes[A.col_idx[a0 + b]] + Cfg::PIECE - 1) / Cfg::PIECE;
          const int incl = warp_incl_scan(np, lane);
          const bool fits = b < na && P + incl <= pmax - 2;
          const int k = __popc(__ballot_sync(0xffffffffu, fits));
          if (fits) sm.sblk[b - sa] = ((P + incl - np) << 8) | np;
          if (k > 0) P += __shfl_sync(0xffffffffu, incl, k - 1);
          sb += k;
          if (k < 32) break;
        }
        __syncwarp();
        // the segment's chunks: whole blocks, at most kChunkPieces pieces each
        // (the same cut as the prep kernel's)
        if (lane == 0) {
          int n = 0, cp = 0;
          for (int b = sa; b < sb; b++) {
            const int e = sm.sblk[b - sa], np = e & 255;
            if (b == sa || cp + np > kChunkPieces) {
              if (n == kMaxSegChunks) {  // cannot happen: chunks average over 4 pieces
                atomicOr(const_cast<int32_t *>(&a.st->error), 2);
                break;
              }
              if (n > 0) sm.sch[n - 1].y = cp;
              sm.sch[n] = make_int4(e >> 8, 0, b, 0);
              n++;
              cp = 0;
            }
            sm.cho[b - sa] = (int16_t)(n - 1);
            cp += np;
            sm.sch[n - 1].w++;
          }
          if (n > 0) sm.sch[n - 1].y = cp;
          if (n == 0) {  // an empty row: one chunk of no pieces per tile
            sm.sch[0] = make_int4(P, 0, sa, 0);
            n = 1;
          }
          mail[1] = sb;
          mail[2] = P;
          mail[3] = n;
        }
        // the B operand of the segment, once the previous segment's MMAs are done
        if (seg_seq > 0) wait(PB_BAR(bop_free), (seg_seq - 1) & 1u);
        if (!failed) {
          const uint4 z = make_uint4(0u, 0u, 0u, 0u);
          for (int x = lane; x < 2 * Cfg::PB / 16; x += 32)
            reinterpret_cast<uint4 *>(sm.bop + (size_t)P * Cfg::PB)[x] = z;
          fence_async_smem();
          __syncwarp();
          for (int b = sa + lane; b < sb; b += 32) {
            const int e = sm.sblk[b - sa], pi = e >> 8, np = e & 255;
            const unsigned char *src = a.a_left + Cfg::UNIT * A.blk_off[a0 + b];
            const uint32_t bytes = (uint32_t)(r * 16);
            for (int q = 0; q < Cfg::NSL; q++)
              for (int kp = 0; kp < np; kp++) {
                pb_expect_tx(PB_BAR(bop_full), bytes);
                bulk_g2s(bop + (uint32_t)((pi + kp) * Cfg::PB + q * NR * 16),
                         src + (size_t)(q * np + kp) * r * 16, bytes, PB_BAR(bop_full));
              }
          }
          __syncwarp();
          if (lane == 0) pb_arrive(PB_BAR(bop_full));
        }
      }
      loaders_sync();
      const int sb = mail[1], P = mail[2], nch = mail[3];
      failed = mail[4] != 0;
      // tiles: loader 0 fetches the tile entries two ahead and the records one
      // ahead (asynchronous copies), writes the tile header and each chunk's
      // first record; both loaders then take alternate chunks
      const int4 *entries = a.pw.tiles + 4 * (int64_t)c0;
      auto fetch_entry = [&](int t) {
        if (t < nt && lane < 4)
          cp_async16(smem_u32(sm.ering + 4 * (t % 3) + lane), entries + 4 * t + lane);
        cp_commit();
      };
      auto fetch_recs = [&](int t) {
        if (t < nt) {
          const TileEntry e = read_entry(sm.ering + 4 * (t % 3));
          const int cnt = (int)(e.P1 - e.P0);  // at most kRecMax
          int4 *dst = sm.rbuf + (t & 1) * kRecMax;
          for (int k = lane; k < cnt; k += 32) cp_async16(smem_u32(dst + k), a.pw.recs + e.P0 + k);
        }
        cp_commit();
      };
      if (lw == 0) {
        fetch_entry(0);
        fetch_entry(1);
        cp_wait1();
        __syncwarp();
        fetch_recs(0);
      }
      for (int t = 0; t < nt; t++) {
        const uint32_t rb_u = smem_u32(sm.rbuf + (t & 1) * kRecMax);
        const int tt = (int)(tile_seq % kTileRing);
        if (lw == 0) {
          fetch_entry(t + 2);
          cp_wait1();  // the records of tile t and the entry of tile t + 1 are in
          __syncwarp();
          fetch_recs(t + 1);
          const TileEntry e = read_entry(sm.ering + 4 * (t % 3));
          const uint8_t *ecj = reinterpret_cast<const uint8_t *>(sm.ering + 4 * (t % 3) + 2);
          const int nrec = (int)(e.P1 - e.P0);
          if (tile_seq >= (uint32_t)kTileRing)
            wait(PB_BAR(tile_empty[tt]), (tile_seq / kTileRing - 1) & 1u);
          TileHdr &T = sm.thdr[tt];
          const bool in = lane < e.ns;
          const int cj = in ? ecj[lane] : 0;
          const int cincl = warp_incl_scan(cj, lane);
          if (in) {
            T.gb[lane] = e.cb0 + lane;
            T.cj[lane] = (uint8_t)cj;
            T.mst[lane] = (uint8_t)(cincl - cj);
            for (int c = 0; c < cj; c++) T.col_slot[cincl - cj + c] = (uint8_t)lane;
          }
          for (int m = e.width + lane; m < kTileCols; m += 32) T.col_slot[m] = 255;
          if (lane == 0) {
            T.flags = (sa > 0 ? kAccum : 0) | (sb >= na ? kLastSeg : 0);
            T.r = r;
            T.nslots = e.ns;
          }
          // each chunk's first record: records are in ascending block order
          auto chunk_of = [&](int k) {
            const int ap = rec_apos(lds32(rb_u + 16u * (uint32_t)k + 4u));
            return ap < sa ? -1 : ap >= sb ? nch : (int)sm.cho[ap - sa];
          };
          for (int k = lane; k < nrec; k += 32) {
            const int ck = chunk_of(k), cprev = k == 0 ? -1 : chunk_of(k - 1);
            for (int cc = cprev + 1; cc <= ck && cc <= nch; cc++) sm.crs[cc] = (int16_t)k;
          }
          if (lane == 0) {  // chunks after the last record's: empty, ending at nrec
            const int clast = nrec == 0 ? -1 : chunk_of(nrec - 1);
            if (clast < nch)
              for (int cc = clast + 1; cc <= nch; cc++) sm.crs[cc] = (int16_t)nrec;
          }
          __syncwarp();
          if (lane == 0 && !failed) pb_arrive(PB_BAR(tile_full[tt]));
        }
        loaders_sync();  // the tile's header, records and chunk starts are ready
        failed = mail[4] != 0;
        for (int c = lw; c < nch && !failed; c += 2) {
          const uint32_t seq = seq_base + (uint32_t)c;
          const int sg = (int)(seq % kStages);
          if (seq >= (uint32_t)kStages && !wait(PB_BAR(stg_empty[sg]), (seq / kStages - 1) & 1u))
            break;
          const int4 ch = sm.sch[c];  // {first piece, pieces, first block, blocks}
          ChunkHdr &H = sm.chdr[sg];
          const uint32_t stage = smem_u32(sm.stage + (size_t)sg * kStageBytes);
          const uint32_t full = PB_BAR(stg_full[sg]);
#pragma unroll
          for (int x = 0; x < kChunkPieces / 4; x++)
            reinterpret_cast<int4 *>(H.ptab[lane])[x] = make_int4(0, 0, 0, 0);
          __syncwarp();
          const int r0 = sm.crs[c], r1 = sm.crs[c + 1];
          uint32_t used = 0;
          for (int k0 = r0; k0 < r1; k0 += 32) {
            const int k = k0 + lane;
            uint32_t staged = 0;
            if (k < r1) {
              const uint4 rec = lds128(rb_u + 16u * (uint32_t)k);
              const int y = (int)rec.y, w = (int)rec.w;
              const int slot = rec_slot(y), ip0 = w & 15, np = (w >> 4) & 15, pstr = (w >> 8) & 511;
              const int cjs = pstr / np;
              if (!rec_far(y)) {
                const int off16 = rec_off16(y);
                if (rec_head(y)) {
                  staged = rec.z * 16u;
                  bulk_g2s(stage + 16u * (uint32_t)off16, a.b_right + 16 * (int64_t)rec.x, staged, full);
                }
                for (int kp = 0; kp < np; kp++)
                  H.ptab[slot][ip0 + kp] = kPiecePresent | (off16 + kp * cjs) | (pstr << 11);
              } else {  // no room in the stage: the gather reads it from global memory
                for (int kp = 0; kp < np; kp++) {
                  H.ptab[slot][ip0 + kp] = kPiecePresent | kPieceFar | (pstr << 11);
                  H.farb[slot][ip0 + kp] = (int)rec.x + kp * cjs;
                }
              }
            }
            used += __reduce_add_sync(0xffffffffu, staged);
          }
          if (lane == 0) {
            H.flags = (c == 0 ? kFirstChunk : 0) | (c == nch - 1 ? kLastChunk : 0) |
                      (t == 0 && c == 0 ? kFirstSegChunk : 0) |
                      (t == nt - 1 && c == nch - 1 ? kLastSegChunk : 0);
            H.tile = (int32_t)tile_seq;
            H.pi0 = ch.x;
            H.npieces = ch.y;
          }
          __syncwarp();
          // one arrival with the chunk's staged bytes (copies that landed already
          // took the transaction count below zero; it returns to zero here)
          if (lane == 0) pb_arrive_expect_tx(full, used);
        }
        loaders_sync();  // both are done with the tile's records and chunk starts
        failed = mail[4] != 0;
        seq_base += (uint32_t)nch;
        tile_seq++;
      }
      if (lw == 0) {
        cp_wait0();
        __syncwarp();
      }
      seg_seq++;
      if (sb >= na || failed) break;
      sa = sb;
    }
  }
  if (lw != 0) return !failed;
  // no more rows: end markers for the gather (chunk) and the epilogue (tile)
  {
    const int sg = (int)(seq_base % kStages);
    if (seq_base >= (uint32_t)kStages && !wait(PB_BAR(stg_empty[sg]), (seq_base / kStages - 1) & 1u))
      return false;
    if (lane == 0) sm.chdr[sg].flags = kEnd;
    __syncwarp();
    if (lane == 0) pb_arrive(PB_BAR(stg_full[sg]));
    const int tt = (int)(tile_seq % kTileRing);
    if (tile_seq >= (uint32_t)kTileRing &&
        !wait(PB_BAR(tile_empty[tt]), (tile_seq / kTileRing - 1) & 1u))
      return false;
    if (lane == 0) sm.thdr[tt].flags = kEnd;
    __syncwarp();
    if (lane == 0) pb_arrive(PB_BAR(tile_full[tt]));
  }
  return !failed;
}

// ---------------------------------------------------------------------------
// Gather (four warps, TMEM lane = C column of the tile): the chunk's A operand.
// ---------------------------------------------------------------------------
template <int PREC, int NR>
__device__ bool panel_gather(const PanelArgs &a, const PanelSmem &sm, uint32_t tmem, int warp,
                             int lane) {
  using Cfg = PanelCfg<PREC, NR>;
  const int m = warp * 32 + lane;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (uint32_t seq = 0;; seq++) {
    const int sg = (int)(seq % kStages), ta = (int)(seq % Cfg::TA);
    if (!pb_wait(PB_BAR(stg_full[sg]), (seq / kStages) & 1u)) return false;
    const ChunkHdr &H = sm.chdr[sg];
    const int flags = H.flags;
    if (flags & kEnd) {
      // the MMA has read this stage's previous note once its MMAs completed
      if (seq >= (uint32_t)Cfg::TA &&
          !pb_wait(PB_BAR(ta_empty[ta]), (seq / Cfg::TA - 1) & 1u))
        return false;
      if (m == 0) sm.note[ta].flags = kEnd;
      __syncwarp();
      if (lane == 0) pb_arrive(PB_BAR(ta_full[ta]));
      return true;
    }
    if (seq >= (uint32_t)Cfg::TA &&
        !pb_wait(PB_BAR(ta_empty[ta]), (seq / Cfg::TA - 1) & 1u))
      return false;
    tc_after();
    const int tile = H.tile, npieces = H.npieces;
    const TileHdr &T = sm.thdr[tile % kTileRing];
    const uint32_t tbytes = smem_u32(&T);
    const int slot = lds8(tbytes + (uint32_t)offsetof(TileHdr, col_slot) + (uint32_t)m);
    int cj = 0, c = 0;
    if (slot != 255) {
      cj = lds8(tbytes + (uint32_t)offsetof(TileHdr, cj) + (uint32_t)slot);
      c = m - lds8(tbytes + (uint32_t)offsetof(TileHdr, mst) + (uint32_t)slot);
    }
    const uint32_t hb = smem_u32(&H);
    const uint32_t prow = hb + (uint32_t)offsetof(ChunkHdr, ptab) + (uint32_t)(slot & 31) * (4 * kChunkPieces);
    const uint32_t stage = smem_u32(sm.stage + (size_t)sg * kStageBytes);
    const uint32_t zero = smem_u32(&sm.bars->zero);
    const int steps = npieces > 0 ? (npieces + 1) >> 1 : 1;
    const uint32_t tbase = tmem + lane_base + (uint32_t)(Cfg::ABASE + ta * Cfg::AC);
    // this column's pieces: their stage addresses from one table row (two
    // 16-byte loads), then every piece's loads at once (an absent product
    // reads the zero line), then the stores
    int pe[kChunkPieces];
#pragma unroll
    for (int x = 0; x < kChunkPieces / 4; x++) {
      const uint4 e = slot != 255 ? lds128(prow + 16u * (uint32_t)x) : make_uint4(0u, 0u, 0u, 0u);
      pe[4 * x] = (int)e.x;
      pe[4 * x + 1] = (int)e.y;
      pe[4 * x + 2] = (int)e.z;
      pe[4 * x + 3] = (int)e.w;
    }
    constexpr int kSteps = kChunkPieces / 2;
    uint32_t v[kSteps][Cfg::NSL][8];
    bool far = false;  // a piece that did not fit the stage: read from global memory below
#pragma unroll
    for (int ip = 0; ip < kChunkPieces; ip++) {
      if (ip < 2 * steps) {
        uint32_t addr = zero, pstr = 0;
        if (pe[ip] & kPiecePresent) {
          if (pe[ip] & kPieceFar) {
            far = true;
          } else {
            addr = stage + (uint32_t)(((pe[ip] & 2047) + c) * 16);
            pstr = (uint32_t)(((pe[ip] >> 11) & 511) * 16);
          }
        }
#pragma unroll
        for (int q = 0; q < Cfg::NSL; q++) {
          const uint4 x = lds128(addr + (uint32_t)q * pstr);
          v[ip >> 1][q][4 * (ip & 1)] = x.x;
          v[ip >> 1][q][4 * (ip & 1) + 1] = x.y;
          v[ip >> 1][q][4 * (ip & 1) + 2] = x.z;
          v[ip >> 1][q][4 * (ip & 1) + 3] = x.w;
        }
      }
    }
    if (__any_sync(0xffffffffu, far)) {  // rare: the stage had no room for some products
      const uint32_t frow = hb + (uint32_t)offsetof(ChunkHdr, farb) + (uint32_t)(slot & 31) * (4 * kChunkPieces);
#pragma unroll
      for (int ip = 0; ip < kChunkPieces; ip++) {
        if ((pe[ip] & kPiecePresent) && (pe[ip] & kPieceFar)) {
          const int base = lds32(frow + 4u * (uint32_t)ip);
          const int pstr = (pe[ip] >> 11) & 511;
          const unsigned char *src = a.b_right + 16 * ((int64_t)base + c);
#pragma unroll
          for (int q = 0; q < Cfg::NSL; q++) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(src + 16 * (int64_t)q * pstr));
            v[ip >> 1][q][4 * (ip & 1)] = x.x;
            v[ip >> 1][q][4 * (ip & 1) + 1] = x.y;
            v[ip >> 1][q][4 * (ip & 1) + 2] = x.z;
            v[ip >> 1][q][4 * (ip & 1) + 3] = x.w;
          }
        }
      }
    }
#pragma unroll
    for (int st = 0; st < kSteps; st++)
      if (st < steps)
#pragma unroll
        for (int q = 0; q < Cfg::NSL; q++) tmem_st8(tbase + (uint32_t)(q * Cfg::PC + st * 8), v[st][q]);
    tmem_wait_st();
    if (m == 0) {
      TaNote &N = sm.note[ta];
      N.flags = flags;
      N.pi0 = H.pi0;
      N.npieces = npieces;
      N.tile = tile;
    }
    tc_before();
    __syncwarp();
    if (lane == 0) {
      pb_arrive(PB_BAR(ta_full[ta]));
      pb_arrive(PB_BAR(stg_empty[sg]));
      if (flags & kLastChunk) pb_arrive(PB_BAR(tile_empty[tile % kTileRing]));
    }
  }
}

// ---------------------------------------------------------------------------
// MMA (one thread): per K step of a chunk, one MMA per B slice.
// ---------------------------------------------------------------------------
template <int PREC, int NR>
__device__ bool panel_mma(const PanelSmem &sm, uint32_t tmem) {
  using Cfg = PanelCfg<PREC, NR>;
  const uint32_t ab = Cfg::TF ? 2u : 1u;
  uint32_t idesc[Cfg::NSL];
#pragma unroll
  for (int q = 0; q < Cfg::NSL; q++) idesc[q] = mma_idesc(ab, (uint32_t)((Cfg::NSL - q) * NR), 128u);
  const uint32_t bop = smem_u32(sm.bop);
  uint32_t seg = 0;
  bool ok = true;
  for (uint32_t seq = 0;; seq++) {
    const int ta = (int)(seq % Cfg::TA);
    if (!pb_wait(PB_BAR(ta_full[ta]), (seq / Cfg::TA) & 1u)) {
      ok = false;
      break;
    }
    const TaNote N = sm.note[ta];
    if (N.flags & kEnd) break;
    tc_after();
    if (N.flags & kFirstSegChunk) {
      if (!pb_wait(PB_BAR(bop_full), seg & 1u)) {
        ok = false;
        break;
      }
      seg++;
    }
    const int db = N.tile & 1;
    if ((N.flags & kFirstChunk) && N.tile >= 2) {
      if (!pb_wait(PB_BAR(d_empty[db]), ((uint32_t)N.tile / 2 - 1) & 1u)) {
        ok = false;
        break;
      }
      tc_after();
    }
    const int steps = N.npieces > 0 ? (N.npieces + 1) >> 1 : 1;
    const uint32_t dcol = tmem + (uint32_t)(db * Cfg::DC);
    const uint32_t acol = tmem + (uint32_t)(Cfg::ABASE + ta * Cfg::AC);
    for (int st = 0; st < steps; st++) {
      const uint64_t bdesc =
          smem_desc(bop + (uint32_t)((N.pi0 + 2 * st) * Cfg::PB), (uint32_t)Cfg::PB, 128u);
#pragma unroll
      for (int q = 0; q < Cfg::NSL; q++) {
        const uint32_t acc = ((N.flags & kFirstChunk) && st == 0 && q == 0) ? 0u : 1u;
        mma_ts<Cfg::TF>(dcol + (uint32_t)(q * NR), acol + (uint32_t)(q * Cfg::PC + st * 8), bdesc,
                        idesc[q], acc);
      }
    }
    mma_commit(PB_BAR(ta_empty[ta]));
    if (N.flags & kLastChunk) mma_commit(PB_BAR(d_full[db]));
    if (N.flags & kLastSegChunk) mma_commit(PB_BAR(bop_free));
  }
  // every MMA issued has completed before the TMEM is released
  mma_commit(PB_BAR(fin));
  if (!pb_wait(PB_BAR(fin), 0u)) ok = false;
  return ok;
}

// ---------------------------------------------------------------------------
// Epilogue (four warps, TMEM lane = C column): accumulator -> FP64 C.
// ---------------------------------------------------------------------------
template <int PREC, int NR>
__device__ bool panel_epilogue(const PanelArgs &a, const PanelSmem &sm, uint32_t tmem, int warp,
                               int lane) {
  using Cfg = PanelCfg<PREC, NR>;
  const int m = warp * 32 + lane;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const DevOut &C = a.C;
  const bool plain = (a.alpha == 1.0 && a.beta == 0.0);
  const bool host = C.host_vals && a.st->nnz_c <= C.host_cap;
  for (uint32_t tseq = 0;; tseq++) {
    const int tt = (int)(tseq % kTileRing), db = (int)(tseq & 1u);
    if (!pb_wait(PB_BAR(tile_full[tt]), (tseq / kTileRing) & 1u)) return false;
    const TileHdr &T = sm.thdr[tt];
    const int flags = T.flags;
    if (flags & kEnd) return true;
    if (!pb_wait(PB_BAR(d_full[db]), (tseq / 2) & 1u)) return false;
    tc_after();
    float g[Cfg::NSL][NR];
#pragma unroll
    for (int q = 0; q < Cfg::NSL; q++)
#pragma unroll
      for (int h = 0; h < NR / 16; h++) {
        float t[16];
        tmem_ld16(tmem + lane_base + (uint32_t)(db * Cfg::DC + q * NR + 16 * h), t);
#pragma unroll
        for (int x = 0; x < 16; x++) g[q][16 * h + x] = t[x];
      }
    tmem_wait_ld();
    tc_before();
    __syncwarp();
    if (lane == 0) pb_arrive(PB_BAR(d_empty[db]));
    const int slot = T.col_slot[m];
    if (slot != 255) {
      const int64_t gb = T.gb[slot];
      const int c = m - T.mst[slot], r = T.r;
      const int64_t e0 = C.blk_off[gb] + (int64_t)c * r;
      double *out = C.vals + e0;
      double *hout = (host && (flags & kLastSeg)) ? C.host_vals + e0 : nullptr;
      const double *cin = nullptr;
      if (!(flags & kAccum)) {
        const int ci = a.ws.c_cin[gb];
        if (ci >= 0) cin = a.Cin.vals + a.Cin.blk_off[ci] + (int64_t)c * r;
      }
#pragma unroll
      for (int rr = 0; rr < NR; rr++) {
        if (rr < r) {
          double v;
          if (Cfg::TF) {
            v = (double)g[0][rr] + (double)g[Cfg::NSL - 1][rr];
          } else {
            // the two small groups in FP32 (their rounding is far below the
            // slices' truncation), then an exact TwoSum with the leading one
            const float small = __fadd_rn(g[1][rr], g[Cfg::NSL - 1][rr]);
            const float hi = __fadd_rn(g[0][rr], small);
            const float bp = __fsub_rn(hi, g[0][rr]);
            const float lo =
                __fadd_rn(__fsub_rn(g[0][rr], __fsub_rn(hi, bp)), __fsub_rn(small, bp));
            v = (double)hi + (double)lo;
          }
          if (flags & kAccum) {
            v = plain ? out[rr] + v : fma(a.alpha, v, out[rr]);
          } else if (!plain) {
            v = a.alpha * v;
            if (cin) v = fma(a.beta, cin[rr], v);
          }
          out[rr] = v;
          if (hout) hout[rr] = v;
        }
      }
    }
    __syncwarp();
    if (lane == 0) pb_arrive(PB_BAR(tile_empty[tt]));
  }
}

template <int PREC, int NR>
__global__ void __launch_bounds__(kWarps * 32, 1) k_numeric_split_panel(PanelArgs a) {
  if (a.st->overflow) return;
  using Cfg = PanelCfg<PREC, NR>;
  extern __shared__ __align__(128) unsigned char panel_smem[];
  const PanelSmem sm = panel_carve(panel_smem, a.pmax, Cfg::PB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    Bars &b = *sm.bars;
    b.zero = make_uint4(0u, 0u, 0u, 0u);
    for (int x = 0; x < kStages; x++) {
      pb_init(smem_u32(&b.stg_full[x]), 1);
      pb_init(smem_u32(&b.stg_empty[x]), 4);
    }
    for (int x = 0; x < kTaMax; x++) {
      pb_init(smem_u32(&b.ta_full[x]), 4);
      pb_init(smem_u32(&b.ta_empty[x]), 1);
    }
    for (int x = 0; x < 2; x++) {
      pb_init(smem_u32(&b.d_full[x]), 1);
      pb_init(smem_u32(&b.d_empty[x]), 4);
    }
    for (int x = 0; x < kTileRing; x++) {
      pb_init(smem_u32(&b.tile_full[x]), 1);
      pb_init(smem_u32(&b.tile_empty[x]), 8);
    }
    pb_init(smem_u32(&b.bop_full), 1);
    pb_init(smem_u32(&b.bop_free), 1);
    pb_init(smem_u32(&b.fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sm.bars->tmem_holder), kTmemCols);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = sm.bars->tmem_holder;
  bool ok = true;
  if (warp >= kLoaderWarp) {
    ok = panel_loader<PREC, NR>(a, sm, warp - kLoaderWarp, lane);
  } else if (warp == kMmaWarp) {
    if (lane == 0) ok = panel_mma<PREC, NR>(sm, tmem);
  } else if (warp >= kEpiWarp0) {
    ok = panel_epilogue<PREC, NR>(a, sm, tmem, warp - kEpiWarp0, lane);
  } else {
    ok = panel_gather<PREC, NR>(a, sm, tmem, warp - kGatherWarp0, lane);
  }
  if (!ok) atomicOr(const_cast<int32_t *>(&a.st->error), 1);
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, kTmemCols);
}

#undef PB_BAR

template <int PREC, int NR>
const void *panel_fn() {
  return (const void *)k_numeric_split_panel<PREC, NR>;
}

template <int PREC, int NR>
int panel_pb() {
  return PanelCfg<PREC, NR>::PB;
}

int panel_pb_of(int precision, int max_r) {
  if (precision == BSM_PREC_SPLIT_BF16X3)
    return max_r > 16 ? panel_pb<BSM_PREC_SPLIT_BF16X3, 32>() : panel_pb<BSM_PREC_SPLIT_BF16X3, 16>();
  return max_r > 16 ? panel_pb<BSM_PREC_SPLIT_TF32X2, 32>() : panel_pb<BSM_PREC_SPLIT_TF32X2, 16>();
}

}  // namespace

cudaError_t launch_panel_prep(int precision, DevMat A, DevMat B, DevOut C, DevWs ws, PanelWs pw,
                              const DevStatus *st, int max_r, int nsm, cudaStream_t stream) {
  // B's slice offset in 16-byte units: 48 / 16 bytes per FP64 offset unit (BF16x3), 32 / 16 (TF32x2)
  const int unit16 = precision == BSM_PREC_SPLIT_BF16X3 ? (int)(2 * kBf16HalfwordsPerValue / 16)
                                                        : (int)(4 * kTf32WordsPerValue / 16);
  const bool bf = precision == BSM_PREC_SPLIT_BF16X3;
  k_panel_prep<<<nsm * 4, kPrepThreads, 0, stream>>>(A, B, C, ws, pw, st, unit16, bf ? 3 : 2,
                                                     bf ? 8 : 4, panel_pmax(panel_pb_of(precision, max_r)));
  return cudaGetLastError();
}

cudaError_t launch_numeric_split_panel(int precision, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                       const void *a_left, const void *b_right, double alpha,
                                       double beta, DevWs ws, PanelWs pw, const DevStatus *st,
                                       int max_r, int nsm, unsigned long long *work,
                                       cudaStream_t stream) {
  PanelArgs a{};
  a.pw = pw;
  a.A = A;
  a.B = B;
  a.Cin = Cin;
  a.C = C;
  a.a_left = static_cast<const unsigned char *>(a_left);
  a.b_right = static_cast<const unsigned char *>(b_right);
  a.alpha = alpha;
  a.beta = beta;
  a.ws = ws;
  a.st = st;
  a.work = work;
  const bool bf = precision == BSM_PREC_SPLIT_BF16X3;
  const bool wide = max_r > 16;
#define BSM_PANEL(P, N)                                                                         \
  do {                                                                                          \
    const int pb = PanelCfg<P, N>::PB;                                                          \
    a.pmax = panel_pmax(pb);                                                                    \
    k_numeric_split_panel<P, N><<<nsm, kWarps * 32, panel_smem_bytes(pb), stream>>>(a);         \
  } while (0)
  if (bf) {
    if (wide) BSM_PANEL(BSM_PREC_SPLIT_BF16X3, 32);
    else BSM_PANEL(BSM_PREC_SPLIT_BF16X3, 16);
  } else {
    if (wide) BSM_PANEL(BSM_PREC_SPLIT_TF32X2, 32);
    else BSM_PANEL(BSM_PREC_SPLIT_TF32X2, 16);
  }
#undef BSM_PANEL
  return cudaGetLastError();
}

cudaError_t numeric_split_panel_init() {
  const void *fns[4] = {panel_fn<BSM_PREC_SPLIT_BF16X3, 16>(), panel_fn<BSM_PREC_SPLIT_BF16X3, 32>(),
                        panel_fn<BSM_PREC_SPLIT_TF32X2, 16>(), panel_fn<BSM_PREC_SPLIT_TF32X2, 32>()};
  const int pbs[4] = {panel_pb<BSM_PREC_SPLIT_BF16X3, 16>(), panel_pb<BSM_PREC_SPLIT_BF16X3, 32>(),
                      panel_pb<BSM_PREC_SPLIT_TF32X2, 16>(), panel_pb<BSM_PREC_SPLIT_TF32X2, 32>()};
  for (int x = 0; x < 4; x++) {
    cudaError_t e = cudaFuncSetAttribute(fns[x], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         panel_smem_bytes(pbs[x]));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bsm
