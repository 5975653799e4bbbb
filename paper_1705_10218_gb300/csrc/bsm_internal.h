// bsm_internal.h -- device-side views and kernel launchers shared by the
// translation units of libbsm. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bsm.h"

namespace bsm {

// Block columns handled per pass of the per-row bitmap in the symbolic phase.
constexpr int kWindowCols = 65536;
constexpr int kSymThreads = 256;
// Largest output tile one warp accumulates in registers (32 x 32 scalars).
constexpr int kTile = 32;

// Read-only device view of a block-sparse matrix in blocked CSR form.
// Blocks of a row are sorted by column; blk_off[b] is the offset of block b's
// column-major values in vals.
struct DevMat {
  int32_t nbr, nbc;
  const int32_t *row_sizes;  // [nbr]
  const int32_t *col_sizes;  // [nbc]
  const int32_t *row_ptr;    // [nbr+1]
  const int32_t *col_idx;    // [nblk]
  const int32_t *blk_row;    // [nblk]
  const int64_t *blk_off;    // [nblk]
  const double *vals;        // [nnz]
  const double *norms;       // [nblk] canonical block norms
  const float *normsf;       // [nblk] FP32 copies for the filter's fast test (NaN: none)
  const int64_t *hdr;        // device header {nblk, nnz}
};

// Where the symbolic phase writes the result pattern of C.
struct DevOut {
  int32_t nbr, nbc;
  const int32_t *row_sizes;
  const int32_t *col_sizes;
  int32_t *row_ptr;  // [nbr+1]
  int32_t *col_idx;  // [cap_blk]
  int32_t *blk_row;  // [cap_blk]
  int64_t *blk_off;  // [cap_blk]
  double *vals;      // [cap_nnz]
  int64_t *hdr;      // {nblk, nnz}
  int64_t cap_blk, cap_nnz;
  // optional second destination of the values: pinned host memory (its device
  // address) of host_cap doubles, written only when the result fits
  double *host_vals;
  int64_t host_cap;
};

// Per-context scratch of one multiply.
struct DevWs {
  int32_t *row_cblk;   // [nbr] C blocks per row
  int64_t *row_prod;   // [nbr] kept products per row
  int64_t *row_nnz;    // [nbr] C scalars per row
  int64_t *row_cand;   // [nbr] candidate products per row
  int64_t *row_flops;  // [nbr] 2mnk of kept products per row
  int64_t *prod_off;   // [nbr+1] first product of each row
  int64_t *nnz_off;    // [nbr+1] first C scalar of each row
  int32_t *cnt;        // [cap_blk] per-C-block product counter / cursor
  int32_t *c_cin;      // [cap_blk] index of the matching C_in block or -1
  int64_t *prod_ptr;   // [cap_blk+1] first product of each C block
  int2 *prods;         // [cap_prod] (A block, B block) per kept product
  int64_t cap_prod;
  int64_t cap_rows;
  // slot shapes of the packed kernels per tile (tm, tn): entry
  // (slots == 16) * kPkTabSize + tm * kPkTabEdge + tn = nT << 8 | G (tuned), or
  // null: the built-in formula
  const uint16_t *pk_tab;
};
constexpr int kPkTabEdge = 17;
constexpr int kPkTabSize = kPkTabEdge * kPkTabEdge;

// Device status of one multiply (written by the device, copied to pinned host).
struct DevStatus {
  int64_t nblk_c;
  int64_t nnz_c;
  int64_t nprod;
  int64_t candidates;
  int64_t kept;
  int64_t flops;    // sum of 2*m*n*k over kept products (exact integer)
  int32_t overflow; // 1: a capacity was too small; later phases skipped
  int32_t error;    // nonzero: a device-side check failed
};

// ---- launchers (each enqueues on `stream`, returns cudaGetLastError()) ----
cudaError_t launch_block_norms(const int32_t *row_sizes, const int32_t *col_sizes,
                               const int32_t *blk_row, const int32_t *col_idx,
                               const int64_t *blk_off, const double *vals, const int64_t *hdr,
                               double *norms, float *normsf, int grid, cudaStream_t stream);

cudaError_t launch_symbolic_count(DevMat A, DevMat B, DevMat Cin, int use_cin, double eps,
                                  DevWs ws, int grid, cudaStream_t stream);

cudaError_t launch_symbolic_scan(int32_t nbr, DevWs ws, DevOut C, DevStatus *st,
                                 cudaStream_t stream);

// mask_words: words of the per-row bit matrix of the placement (a bound on C
// blocks per row times the words per A row; rows beyond it take the slower
// per-window passes); 0: the largest (8192).
cudaError_t launch_symbolic_fill(DevMat A, DevMat B, DevMat Cin, int use_cin, double eps,
                                 DevWs ws, DevOut C, const DevStatus *st, int nsm, int mask_words,
                                 cudaStream_t stream);

// FP64 numeric kernel variants (k_numeric_fp64.cu).
enum {
  kFp64T16B2 = 0,
  kFp64T16B3 = 1,
  kFp64T32 = 2,
  kFp64Pk12 = 3,
  kFp64Pk16 = 4,
  kFp64G8 = 5,
  kFp64NumVariants = 6
};
int fp64_variant_blocks_per_sm(int variant);
// The packed kernel's built-in slot shape (nT, G) of a tile of te elements
// (1..256) with at most `slots` (12 or 16) slots per lane.
void pk_formula_shape(int slots, int te, int *nt, int *g);
// Largest number of k-groups of the packed kernel.
constexpr int kPkMaxGroups = 8;
// Per-device kernel attributes (call with the device current, outside capture).
cudaError_t numeric_fp64_init();

// items: optional work list of C block indices; seg: optional device [begin,
// end) into it (default: all C blocks of the multiply, in row order).
// work: a device counter that must be zero when the launch starts (the t16 and
// pk variants hand out C blocks dynamically; may be null for t32).
// max_m, max_n: the largest C block row and column sizes of the launch (the
// g8 variant sizes its register rows and lane groups by them).
cudaError_t launch_numeric_fp64(int variant, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                double alpha, double beta, DevWs ws, const DevStatus *st,
                                const int32_t *items, const int64_t *seg, int grid,
                                unsigned long long *work, int max_m, int max_n,
                                cudaStream_t stream);
inline bool fp64_variant_uses_work(int variant) { return variant != kFp64T32; }

// Shape classes (k_classes.cu): class of C block g = row_cls[row] * ncc +
// col_cls[col]; items receives the C blocks grouped by class, segs[2c..2c+1]
// the [begin, end) of class c. counts/cursor: ncls int32 of scratch.
constexpr int kMaxClasses = 1024;
cudaError_t launch_class_sort(DevOut C, const int32_t *row_cls, const int32_t *col_cls, int ncc,
                              int ncls, const DevStatus *st, int32_t *counts, int32_t *cursor,
                              int64_t *segs, int32_t *items, int nsm, cudaStream_t stream);

// C blocks in the order of a permutation of C's block rows (k_classes.cu):
// row_order[p] = the row at position p, row_pos[r] = the position of row r;
// items[nblk_c] receives the blocks row by row in that order, start[nbr] is
// scratch. Two launches.
cudaError_t launch_order_items(DevOut C, const int32_t *row_order, const int32_t *row_pos,
                               int32_t nbr, const DevStatus *st, int32_t *start, int32_t *items,
                               int nsm, cudaStream_t stream);
// segs[2s..2s+1] = the s-th of n consecutive ranges of the multiply's C blocks
// (one thread block; n <= 64).
cudaError_t launch_slice_segs(const DevStatus *st, int n, int64_t *segs, cudaStream_t stream);

// Split precision (k_split.cu). left/right: slice layouts of the operand as a
// left (row-major) or right (column-major) MMA operand; either may be null.
// One warp waits (bounded) on an mbarrier that it completes itself, or that
// nothing completes (never_complete); *flag = 1 when the wait gave up.
cudaError_t launch_wait_selftest(int never_complete, int32_t *flag, cudaStream_t stream);

cudaError_t launch_split(int precision, const int32_t *row_sizes, const int32_t *col_sizes,
                         const int32_t *blk_row, const int32_t *col_idx, const int64_t *blk_off,
                         const double *vals, const int64_t *hdr, void *left, void *right,
                         int grid, cudaStream_t stream);

// The chunked split kernel: the C blocks whose MMA problem fits 16 x 16, each
// block's products concatenated along k in shared-memory chunks (the others
// are skipped: the large-block instance of launch_numeric_split takes them).
// smax: the largest k of the launch (at most 32; picks the chunk size).
cudaError_t launch_numeric_split_cat(int precision, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                     const void *a_left, const void *b_right, double alpha,
                                     double beta, DevWs ws, const DevStatus *st,
                                     const int32_t *items, const int64_t *seg, int smax, int nsm,
                                     unsigned long long *work, cudaStream_t stream);

// sizes: 0 = every block's MMA problem fits 16 x 16 (one launch covers all);
// 1 = only the blocks that fit 16 x 16; 2 = only the larger ones (<= 32 x 32).
// smax: the largest k (column size of A) the launch can meet, at most 32.
cudaError_t launch_numeric_split(int precision, int sizes, DevMat A, DevMat B, DevOut C,
                                 DevMat Cin, const void *a_left, const void *b_right, double alpha,
                                 double beta, DevWs ws, const DevStatus *st, const int32_t *items,
                                 const int64_t *seg, int smax, int nsm, unsigned long long *work,
                                 cudaStream_t stream);
// The row-panel split kernel (k_split_panel.cu). Its work of a multiply:
//   tiles:  per C block row, its tiles (runs of whole C blocks, at most 128
//           columns and 32 blocks) as 64-byte entries at the row's first C
//           block index: {first C block, blocks, first record (int64)},
//           {end record (int64), columns, 0}, the blocks' column sizes (32 bytes);
//   row_nt: tiles per row, -1 for a row left to the per-block kernel (more A
//           blocks than the record sort handles);
//   recs:   the kept products of each tile ordered by A block, with their
//           places in the staged copies (16-byte records, see k_split_panel.cu);
//   fb_items, fb_seg: C blocks of the rows left to the per-block kernel and
//           {0, their count} (fb_seg[1] must be zero before the prep kernel).
struct PanelWs {
  int4 *recs;       // [cap_prod]
  int4 *tiles;      // [4 * cap C blocks]
  int32_t *row_nt;  // [rows]
  int32_t *fb_items;
  int64_t *fb_seg;
};
cudaError_t launch_panel_prep(int precision, DevMat A, DevMat B, DevOut C, DevWs ws, PanelWs pw,
                              const DevStatus *st, int max_r, int nsm, cudaStream_t stream);
// max_r: the largest block row size of A (at most 32). work: a device counter
// that must be zero when the launch starts.
cudaError_t launch_numeric_split_panel(int precision, DevMat A, DevMat B, DevOut C, DevMat Cin,
                                       const void *a_left, const void *b_right, double alpha,
                                       double beta, DevWs ws, PanelWs pw, const DevStatus *st,
                                       int max_r, int nsm, unsigned long long *work,
                                       cudaStream_t stream);
cudaError_t numeric_split_panel_init();

// Post filter and block-sparse add (k_extra.cu).
cudaError_t launch_filter_count(DevMat M, double eps, DevWs ws, int nsm, cudaStream_t stream);
cudaError_t launch_filter_fill(DevMat M, double eps, DevWs ws, DevOut O, const DevStatus *st,
                               int nsm, cudaStream_t stream);
// stage 0: per-row union counts; 1: union pattern and sources; 2: values
// Copies C's values (nnz from the status) to O.host_vals when they fit host_cap
// and the multiply did not overflow.
cudaError_t launch_copy_out(DevOut O, const DevStatus *st, int nsm, cudaStream_t stream);
inline bool fp64_variant_writes_host(int variant) {
  return variant == kFp64Pk12 || variant == kFp64Pk16 || variant == kFp64G8;
}

cudaError_t launch_add(int stage, DevMat A, DevMat Cin, int use_cin, double alpha, double beta,
                       DevWs ws, DevOut O, const DevStatus *st, int nsm, cudaStream_t stream);

// Per-device kernel attributes of the split kernels (outside capture).
cudaError_t numeric_split_init();

// Slice storage of an operand block b starts at a fixed multiple of its FP64
// offset blk_off[b], 16-byte aligned so whole blocks can be copied with bulk
// asynchronous copies. Each slice plane of an r x c block is stored as rows
// with k contiguous, every row padded with zeros to 16 bytes: BF16x3 at
// halfword 24*blk_off (3 planes of r rows of ceil8(c) halfwords take at most
// 24 per value, reached for c = 1), TF32x2 at word 8*blk_off (2 planes of
// ceil4(c) words per row, at most 8 per value).
constexpr int64_t kBf16HalfwordsPerValue = 24;
constexpr int64_t kTf32WordsPerValue = 8;
inline int64_t split_bytes_per_value(int precision) {
  return precision == BSM_PREC_SPLIT_BF16X3 ? 2 * kBf16HalfwordsPerValue : 4 * kTf32WordsPerValue;
}

// One diagonal part of a block-diagonal matrix (the request loop's batches).
struct DiagPart {
  int32_t nbr;                 // block rows of the part (= its block columns)
  const int32_t *sizes;        // [nbr]
  int64_t nblk;                // blocks, sorted by (row, col), no duplicates
  const int32_t *brow, *bcol;  // [nblk] indices within the part
  const double *vals;          // column-major values in list order (page-locked: DMA)
};

// diag(P_0, ..., P_{n-1}) as one square matrix on ctx: the block rows and
// columns of part p follow those of the parts before it. Each part's values go
// to the device with one copy of their own (no host-side concatenation).
// INVALID_ARG for a null argument, a non-positive size or a part whose blocks
// are not strictly sorted; OUT_OF_RANGE for an index outside its part.
int mat_create_diag(bsm_ctx ctx, int nparts, const DiagPart *parts, bsm_mat *out);

// A host function called between the slices of a sliced numeric phase
// (opts.numeric_slices > 1) of an uncaptured multiply on ctx, after the slice
// before it has finished on the device; it may block (the request loop holds a
// large multiply's next slice there while small multiplies run). nullptr: none.
using SliceGate = void (*)(void *arg);
int set_slice_gate(bsm_ctx ctx, SliceGate gate, void *arg);

}  // namespace bsm
