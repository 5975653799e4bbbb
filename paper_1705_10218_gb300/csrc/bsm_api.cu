// bsm_api.cu -- host runtime behind include/bsm.h: contexts, matrices, the
// multiply pipeline (norms -> symbolic count -> scan -> fill -> numeric), the
// result-buffer capacities, and error mapping.
//
// Result buffers follow the reuse rule the paper gives for its panel buffers
// (Sec. 3): they are kept between multiplies and only reallocated when the
// needed size exceeds the current one. The device checks the sizes itself (the
// scan pass compares the totals with the capacities), so a multiply into a C
// whose buffers are already large enough needs no host round trip: it is one
// stream-ordered sequence of launches. When a buffer is too small, later passes
// skip their work, and the host grows the buffers and reruns the multiply when
// it next looks at the result.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <numeric>
#include <unordered_map>
#include <thread>
#include <vector>

#include "bsm_internal.h"

using namespace bsm;

namespace {

thread_local char g_cuda_err[256] = "";

// Host threads for the checks and offsets of long block lists.
constexpr int kHostThreads = 8;

int cuda_fail(cudaError_t e, const char *where) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return BSM_ERR_NOMEM;
  return BSM_ERR_CUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// Device memory. cudaFree synchronises the whole device (every stream of every
// context), so the library keeps freed blocks in a per-device cache and
// reuses them instead. Every caller frees a block only after the work that
// used it has finished (after synchronising the owning context's streams), so
// a cached block can go to any context and any stream. Sizes are rounded up
// to classes 1/8 of a power of two apart (under 12.5% slack); the cache holds
// at most kCacheCap bytes per device (beyond that blocks are freed), a failed
// cudaMalloc empties it and retries, and it is emptied when the last context
// on the device is destroyed.
// ---------------------------------------------------------------------------
constexpr int kCacheDevices = 64;
constexpr size_t kCacheCap = 16ull << 30;

struct DevCache {
  std::mutex mu;
  std::multimap<size_t, void *> free_blocks;     // class -> block
  std::unordered_map<void *, size_t> block_size;  // every block the cache handed out
  size_t cached = 0;
  size_t held = 0;  // bytes of all blocks in block_size (handed out or cached)
  int contexts = 0;
};

// Device bytes the library may hold per device: BSM_DEVICE_MEMORY_CAP=<bytes>
// (read once; unset or 0: no cap). An allocation beyond it fails as if the
// device were out of memory (BSM_ERR_NOMEM), which simulates a full device.
size_t device_memory_cap() {
  static const size_t cap = [] {
    const char *v = getenv("BSM_DEVICE_MEMORY_CAP");
    return v ? (size_t)strtoull(v, nullptr, 10) : (size_t)0;
  }();
  return cap;
}
DevCache g_cache[kCacheDevices];

size_t size_class(size_t b) {
  if (b <= 256) return 256;
  const int p = 63 - __builtin_clzll((unsigned long long)(b - 1));  // 2^p <= b - 1 < 2^(p+1)
  const size_t step = (size_t)1 << (p - 3);
  return (b + step - 1) & ~(step - 1);
}

DevCache *cache_of_current() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCacheDevices) return nullptr;
  return &g_cache[dev];
}

// Frees every cached block (the caller holds c.mu).
void cache_flush_locked(DevCache &c) {
  for (auto &kv : c.free_blocks) {
    c.block_size.erase(kv.second);
    cudaFree(kv.second);
  }
  c.free_blocks.clear();
  c.held -= c.cached;
  c.cached = 0;
}

cudaError_t cache_alloc(void **p, size_t bytes) {
  *p = nullptr;
  DevCache *c = cache_of_current();
  const size_t cls = size_class(bytes);
  if (!c) return cudaMalloc(p, cls);
  std::lock_guard<std::mutex> lock(c->mu);
  auto it = c->free_blocks.find(cls);
  if (it != c->free_blocks.end()) {
    *p = it->second;
    c->free_blocks.erase(it);
    c->cached -= cls;
    return cudaSuccess;
  }
  const size_t cap = device_memory_cap();
  if (cap && c->held + cls > cap && c->cached > 0) cache_flush_locked(*c);
  if (cap && c->held + cls > cap) return cudaErrorMemoryAllocation;  // simulated full device
  cudaError_t e = cudaMalloc(p, cls);
  if (e == cudaErrorMemoryAllocation && c->cached > 0) {  // give the cache back, retry
    cudaGetLastError();
    cache_flush_locked(*c);
    e = cudaMalloc(p, cls);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  c->block_size[*p] = cls;
  c->held += cls;
  return cudaSuccess;
}

void cache_free(void *p) {
  if (!p) return;
  DevCache *c = cache_of_current();
  if (!c) {
    cudaFree(p);
    return;
  }
  std::lock_guard<std::mutex> lock(c->mu);
  auto it = c->block_size.find(p);
  if (it == c->block_size.end()) {  // not from the cache (another device current): plain free
    cudaFree(p);
    return;
  }
  const size_t cls = it->second;
  if (c->cached + cls <= kCacheCap) {
    c->free_blocks.emplace(cls, p);
    c->cached += cls;
  } else {
    c->block_size.erase(it);
    c->held -= cls;
    cudaFree(p);
  }
}

template <class T>
int dev_alloc(T **p, int64_t n) {
  if (n <= 0) n = 1;
  void *q = nullptr;
  cudaError_t e = cache_alloc(&q, (size_t)n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc");
  }
  *p = static_cast<T *>(q);
  return BSM_OK;
}

template <class T>
void dev_free(T *&p) {
  cache_free((void *)p);
  p = nullptr;
}

}  // namespace

// One set of pattern + value buffers of a matrix.
struct Buf {
  int32_t *row_ptr = nullptr;  // [nbr+1]
  int32_t *col_idx = nullptr;  // [cap_blk]
  int32_t *blk_row = nullptr;  // [cap_blk]
  int64_t *blk_off = nullptr;  // [cap_blk]
  double *norms = nullptr;     // [cap_blk]
  float *normsf = nullptr;     // [cap_blk] FP32 copies for the filter's fast test
  double *vals = nullptr;      // [cap_nnz]
  int64_t *hdr = nullptr;      // {nblk, nnz}
  int64_t cap_blk = -1, cap_nnz = -1;  // -1: never sized

  void release() {
    dev_free(row_ptr);
    dev_free(col_idx);
    dev_free(blk_row);
    dev_free(blk_off);
    dev_free(norms);
    dev_free(normsf);
    dev_free(vals);
    dev_free(hdr);
    cap_blk = cap_nnz = -1;
  }
};

struct Pending {
  bool active = false;
  bsm_mat A = nullptr, B = nullptr;
  double alpha = 0, beta = 0, eps = 0;
  bsm_opts opts{};
  int slot = -1;
};

struct bsm_mat_s {
  bsm_ctx ctx = nullptr;
  // recorded after every multiply that reads or writes the matrix: the work
  // to wait for before its contents change (filter, add and the getters
  // finish their own work before they return)
  cudaEvent_t ev_use = nullptr;
  int32_t nbr = 0, nbc = 0;
  std::vector<int32_t> h_row_sizes, h_col_sizes;
  int32_t max_row = 0, max_col = 0;  // largest block row / column size
  int64_t max_row_blocks = -1;  // most blocks in one block row (-1: unknown, the
                                // pattern was made on the device)
  // shape kinds: the distinct block row / column sizes (at most 32; more are
  // folded into one kind) and each block row's / column's kind index
  std::vector<int32_t> row_kinds, col_kinds;
  bool kinds_exact = true;  // every kind is one size (not folded)
  int32_t *row_cls = nullptr, *col_cls = nullptr;
  // slices of the values for the split precisions (left / right operand layouts)
  void *split_left = nullptr, *split_right = nullptr;
  int64_t cap_left = 0, cap_right = 0;  // bytes
  int32_t *row_sizes = nullptr, *col_sizes = nullptr;
  Buf front, back;
  int64_t nblk = 0, nnz = 0;  // valid when !pend.active
  int64_t hint_blk = 0, hint_nnz = 0;  // sizes of the last result computed into it
  // a breadth-first order of the block rows over the pattern ([2 nbr]: the row
  // at each position, then each row's position), the order in which the
  // numeric phase takes the C blocks of a multiply with this matrix on the left;
  // valid while order_id != 0. A result inherits the order of its left operand
  // (same block rows).
  int32_t *row_order = nullptr;
  uint64_t order_id = 0;
  // the pattern (row pointers, column indices) the order was computed from: an
  // upload of the same pattern keeps the order without a new search
  std::vector<int32_t> order_ptr, order_col;
  Pending pend;
};

constexpr int kSlots = 64;

struct bsm_ctx_s {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_last = nullptr;   // last work of this context (any stream)
  // matrix uploads (bsm_mat_create / bsm_mat_assign): a stream of their own, so
  // that an upload runs while a multiply of other matrices is on the device
  cudaStream_t up_stream = nullptr;
  cudaEvent_t ev_up = nullptr;
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
  DevStatus *d_status = nullptr;
  unsigned long long *d_work = nullptr;  // work counter of the dynamically scheduled kernels
  DevStatus *h_slots = nullptr;    // pinned ring of status copies
  unsigned char *h_stage = nullptr;  // pinned staging of uploaded index arrays
  size_t h_stage_cap = 0;
  cudaEvent_t slot_ev[kSlots] = {};
  bsm_mat slot_owner[kSlots] = {};
  int next_slot = 0;
  // workspace
  DevWs ws{};
  int64_t cap_rows = 0, cap_cblk = -1;
  int64_t hint_prod = 0;
  std::vector<bsm_mat> mats;
  // profiling
  bool prof = false;
  cudaEvent_t prof_ev[kSlots][4] = {};
  bool prof_pending[kSlots] = {};
  bsm_profile prof_tot{};
  int last_fp64 = -1;  // BSM_FP64_* of the last FP64 numeric launch
  int last_split = -1;  // BSM_SPLIT_* of the last split-precision numeric launch
  int64_t launches = 0;
  int64_t launches_at_enable = 0;
  // shape-class grouping (per-stack launches)
  int32_t *cls_items = nullptr;  // [cap_cblk]
  int32_t *ord_start = nullptr;  // [cap_rows] first item of each position of a row order
  // work of the row-panel split kernel (records, tile entries, tiles per row);
  // its fallback list reuses cls_items / cls_segs
  PanelWs pw{};
  int64_t cap_pw_recs = 0, cap_pw_tiles = 0, cap_pw_rows = 0;
  int32_t *cls_counts = nullptr, *cls_cursor = nullptr;  // [kMaxClasses]
  int64_t *cls_segs = nullptr;   // [2 * kMaxClasses]
  // captured multiplies (opts.graph), keyed by every kernel argument
  struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    uint64_t used = 0;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  // autotuner: key -> FP64 variant, or for a tile key the packed kernel's
  // slot shape nT << 8 | G
  std::map<std::string, int> tune;
  // slot shapes of the packed kernels (12 slots, then 16) per tile (tm, tn):
  // the formula's, replaced by tuned ones; on the device once one is tuned
  // (ws.pk_tab)
  uint16_t pk_tab[2 * kPkTabSize] = {};
  uint16_t *d_pk_tab = nullptr;
  std::string tune_path;
  uint64_t tune_version = 0;
  // between the slices of a sliced numeric phase (uncaptured multiplies only):
  // the previous slice is waited for, then gate(gate_arg) is called
  bsm::SliceGate gate = nullptr;
  void *gate_arg = nullptr;
  cudaEvent_t ev_gate = nullptr;
};

constexpr int kMaxKinds = 32;
constexpr int kMaxGraphs = 8;

// Add the phase times of slot s to the totals (once per recorded multiply).
static int prof_collect(bsm_ctx ctx, int s) {
  if (!ctx->prof_pending[s]) return BSM_OK;
  ctx->prof_pending[s] = false;
  CK(cudaEventSynchronize(ctx->prof_ev[s][3]));
  float a = 0, b = 0, c = 0, t = 0;
  CK(cudaEventElapsedTime(&a, ctx->prof_ev[s][0], ctx->prof_ev[s][1]));
  CK(cudaEventElapsedTime(&b, ctx->prof_ev[s][1], ctx->prof_ev[s][2]));
  CK(cudaEventElapsedTime(&c, ctx->prof_ev[s][2], ctx->prof_ev[s][3]));
  CK(cudaEventElapsedTime(&t, ctx->prof_ev[s][0], ctx->prof_ev[s][3]));
  ctx->prof_tot.ms_norms += a;
  ctx->prof_tot.ms_symbolic += b;
  ctx->prof_tot.ms_numeric += c;
  ctx->prof_tot.ms_total += t;
  ctx->prof_tot.multiplies += 1;
  return BSM_OK;
}

static int ctx_set_device(bsm_ctx ctx) {
  CK(cudaSetDevice(ctx->device));
  return BSM_OK;
}

// ---------------------------------------------------------------------------
// workspace sizing
// ---------------------------------------------------------------------------
static int ws_rows(bsm_ctx ctx, int64_t nrows) {
  if (ctx->cap_rows >= nrows + 1) return BSM_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  DevWs &w = ctx->ws;
  dev_free(w.row_cblk);
  dev_free(w.row_prod);
  dev_free(w.row_nnz);
  dev_free(w.row_cand);
  dev_free(w.row_flops);
  dev_free(w.prod_off);
  dev_free(w.nnz_off);
  dev_free(ctx->ord_start);
  const int64_t n = std::max<int64_t>(nrows + 1, 1024);
  int rc;
  if ((rc = dev_alloc(&w.row_cblk, n)) || (rc = dev_alloc(&w.row_prod, n)) ||
      (rc = dev_alloc(&w.row_nnz, n)) || (rc = dev_alloc(&w.row_cand, n)) ||
      (rc = dev_alloc(&w.row_flops, n)) || (rc = dev_alloc(&w.prod_off, n)) ||
      (rc = dev_alloc(&w.nnz_off, n)) || (rc = dev_alloc(&ctx->ord_start, n))) {
    ctx->cap_rows = 0;
    return rc;
  }
  ctx->cap_rows = n;
  w.cap_rows = n;
  return BSM_OK;
}

static int ws_grow(bsm_ctx ctx, int64_t nblk_c, int64_t nprod) {
  DevWs &w = ctx->ws;
  if (ctx->cap_cblk < nblk_c + 1) {
    CK(cudaStreamSynchronize(ctx->stream));
    dev_free(w.cnt);
    dev_free(w.c_cin);
    dev_free(w.prod_ptr);
    dev_free(ctx->cls_items);
    const int64_t n = nblk_c + nblk_c / 8 + 1024;
    int rc;
    if ((rc = dev_alloc(&w.cnt, n)) || (rc = dev_alloc(&w.c_cin, n)) ||
        (rc = dev_alloc(&w.prod_ptr, n + 1)) || (rc = dev_alloc(&ctx->cls_items, n))) {
      ctx->cap_cblk = -1;
      return rc;
    }
    ctx->cap_cblk = n;
  }
  if (w.cap_prod < nprod) {
    CK(cudaStreamSynchronize(ctx->stream));
    dev_free(w.prods);
    const int64_t n = nprod + nprod / 8 + 1024;
    int rc;
    if ((rc = dev_alloc(&w.prods, n))) {
      w.cap_prod = 0;
      return rc;
    }
    w.cap_prod = n;
  }
  return BSM_OK;
}

// The row-panel kernel's work buffers, sized to the workspace's capacities.
// Buffers are freed (returned to the cache) only once the multiplies that may
// still read them have finished.
static int panel_ws(bsm_ctx ctx, int64_t nrows) {
  int rc;
  if (ctx->cap_pw_recs < ctx->ws.cap_prod || ctx->cap_pw_tiles < ctx->cap_cblk ||
      ctx->cap_pw_rows < nrows)
    CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->cap_pw_recs < ctx->ws.cap_prod) {
    dev_free(ctx->pw.recs);
    ctx->cap_pw_recs = 0;
    if ((rc = dev_alloc(&ctx->pw.recs, ctx->ws.cap_prod))) return rc;
    ctx->cap_pw_recs = ctx->ws.cap_prod;
  }
  if (ctx->cap_pw_tiles < ctx->cap_cblk) {
    dev_free(ctx->pw.tiles);
    ctx->cap_pw_tiles = 0;
    if ((rc = dev_alloc(&ctx->pw.tiles, 4 * ctx->cap_cblk))) return rc;
    ctx->cap_pw_tiles = ctx->cap_cblk;
  }
  if (ctx->cap_pw_rows < nrows) {
    dev_free(ctx->pw.row_nt);
    ctx->cap_pw_rows = 0;
    if ((rc = dev_alloc(&ctx->pw.row_nt, nrows))) return rc;
    ctx->cap_pw_rows = nrows;
  }
  ctx->pw.fb_items = ctx->cls_items;
  ctx->pw.fb_seg = ctx->cls_segs;
  return BSM_OK;
}

// Buffers sized for (nblk, nnz); row arrays for nbr rows.
static int buf_grow(bsm_mat M, Buf &b, int64_t nblk, int64_t nnz, bool exact) {
  if (!b.row_ptr) {
    int rc;
    if ((rc = dev_alloc(&b.row_ptr, (int64_t)M->nbr + 1)) || (rc = dev_alloc(&b.hdr, 2))) return rc;
    cudaStream_t s = M->ctx->stream;
    CK(cudaMemsetAsync(b.row_ptr, 0, ((size_t)M->nbr + 1) * sizeof(int32_t), s));
    CK(cudaMemsetAsync(b.hdr, 0, 2 * sizeof(int64_t), s));
  }
  if (b.cap_blk < nblk) {
    CK(cudaStreamSynchronize(M->ctx->stream));
    dev_free(b.col_idx);
    dev_free(b.blk_row);
    dev_free(b.blk_off);
    dev_free(b.norms);
    dev_free(b.normsf);
    const int64_t n = exact ? nblk : nblk + nblk / 8 + 64;
    int rc;
    if ((rc = dev_alloc(&b.col_idx, n)) || (rc = dev_alloc(&b.blk_row, n)) ||
        (rc = dev_alloc(&b.blk_off, n)) || (rc = dev_alloc(&b.norms, n)) ||
        (rc = dev_alloc(&b.normsf, n))) {
      b.cap_blk = -1;
      return rc;
    }
    b.cap_blk = n;
  }
  if (b.cap_nnz < nnz) {
    CK(cudaStreamSynchronize(M->ctx->stream));
    dev_free(b.vals);
    const int64_t n = exact ? nnz : nnz + nnz / 8 + 1024;
    int rc;
    if ((rc = dev_alloc(&b.vals, n))) {
      b.cap_nnz = -1;
      return rc;
    }
    b.cap_nnz = n;
  }
  return BSM_OK;
}

static DevMat dev_view(bsm_mat M) {
  DevMat v{};
  v.nbr = M->nbr;
  v.nbc = M->nbc;
  v.row_sizes = M->row_sizes;
  v.col_sizes = M->col_sizes;
  v.row_ptr = M->front.row_ptr;
  v.col_idx = M->front.col_idx;
  v.blk_row = M->front.blk_row;
  v.blk_off = M->front.blk_off;
  v.vals = M->front.vals;
  v.norms = M->front.norms;
  v.normsf = M->front.normsf;
  v.hdr = M->front.hdr;
  return v;
}

static DevOut dev_out(bsm_mat M, Buf &b) {
  DevOut o{};
  o.nbr = M->nbr;
  o.nbc = M->nbc;
  o.row_sizes = M->row_sizes;
  o.col_sizes = M->col_sizes;
  o.row_ptr = b.row_ptr;
  o.col_idx = b.col_idx;
  o.blk_row = b.blk_row;
  o.blk_off = b.blk_off;
  o.vals = b.vals;
  o.hdr = b.hdr;
  o.cap_blk = std::max<int64_t>(b.cap_blk, 0);
  o.cap_nnz = std::max<int64_t>(b.cap_nnz, 0);
  return o;
}

static int resolve(bsm_mat M, bsm_stats *timed = nullptr);

// ---------------------------------------------------------------------------
// the multiply pipeline
// ---------------------------------------------------------------------------
static int enqueue_norms(bsm_ctx ctx, bsm_mat M, cudaStream_t s) {
  const int grid = ctx->nsm * 8;
  CK(launch_block_norms(M->row_sizes, M->col_sizes, M->front.blk_row, M->front.col_idx,
                        M->front.blk_off, M->front.vals, M->front.hdr, M->front.norms,
                        M->front.normsf, grid, s));
  return BSM_OK;
}

// Slice buffers of M for the given layouts, sized for its current values.
static int split_buffers(bsm_mat M, int precision, bool left, bool right) {
  const int64_t need = std::max<int64_t>(M->nnz, 1) * split_bytes_per_value(precision);
  auto grow = [&](void *&p, int64_t &cap) -> int {
    if (cap >= need) return BSM_OK;
    if (p) {  // earlier multiplies may still read the slices
      CK(cudaStreamSynchronize(M->ctx->stream));
      cache_free(p);
    }
    p = nullptr;
    cap = 0;
    cudaError_t e = cache_alloc(&p, (size_t)need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "cudaMalloc(slices)");
    }
    cap = need;
    return BSM_OK;
  };
  int rc;
  if (left && (rc = grow(M->split_left, M->cap_left))) return rc;
  if (right && (rc = grow(M->split_right, M->cap_right))) return rc;
  return BSM_OK;
}

static int take_slot(bsm_ctx ctx, bsm_mat owner) {
  const int s = ctx->next_slot;
  ctx->next_slot = (ctx->next_slot + 1) % kSlots;
  if (ctx->prof_pending[s]) {
    int rc = prof_collect(ctx, s);
    if (rc) return -1000 + rc;
  }
  if (ctx->slot_owner[s] && ctx->slot_owner[s]->pend.active && ctx->slot_owner[s]->pend.slot == s) {
    int rc = resolve(ctx->slot_owner[s]);
    if (rc) return -1000 + rc;
  }
  ctx->slot_owner[s] = owner;
  return s;
}

// ---------------------------------------------------------------------------
// autotuner: FP64 numeric variants per shape class (per-stack launches) or for
// the whole class mix (one persistent launch), timed on the real data the first
// time a key is met and kept in a text file (BSM_AUTOTUNE_CACHE) across runs.
// ---------------------------------------------------------------------------
static std::string tune_key_class(int m, int n) {
  return "fp64/class/" + std::to_string(m) + "x" + std::to_string(n);
}

static std::string tune_key_tile(int slots, int m, int n) {
  return "pk" + std::to_string(slots) + "tile:" + std::to_string(m) + "x" + std::to_string(n);
}

// A slot shape the packed kernel with `slots` slots per lane can run for a
// tile of te elements.
static bool pk_shape_ok(int slots, int te, int nt, int g) {
  return nt >= 1 && nt <= slots && g >= 1 && g <= kPkMaxGroups && te * g <= 32 * nt;
}
static int pk_slots(int variant) { return variant == kFp64Pk16 ? 16 : 12; }
static int pk_tab_at(int slots, int m, int n) {
  return (slots == 16 ? kPkTabSize : 0) + m * kPkTabEdge + n;
}

static std::string tune_key_all(bsm_mat A, bsm_mat B) {
  std::string k = "fp64/all/";
  for (int32_t r : A->row_kinds) k += std::to_string(r) + ",";
  k += "|";
  for (int32_t c : A->col_kinds) k += std::to_string(c) + ",";
  k += "|";
  for (int32_t c : B->col_kinds) k += std::to_string(c) + ",";
  return k;
}

// Entries of the cache file: "key value ms" per line; lines starting with '#'
// are notes. A tile entry sets the packed kernel's slot shape of that tile.
static void tune_load(bsm_ctx ctx) {
  const char *p = getenv("BSM_AUTOTUNE_CACHE");
  if (!p || !*p) return;
  ctx->tune_path = p;
  FILE *f = fopen(p, "r");
  if (!f) return;
  char line[640], key[512];
  int v, m, n;
  double ms;
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || sscanf(line, "%511s %d %lf", key, &v, &ms) != 3) continue;
    int slots = 0;
    if (sscanf(key, "pk%dtile:%dx%d", &slots, &m, &n) == 3) {
      if ((slots == 12 || slots == 16) && m >= 1 && m < kPkTabEdge && n >= 1 && n < kPkTabEdge &&
          v >= 0 && pk_shape_ok(slots, m * n, v >> 8, v & 0xFF)) {
        ctx->tune[key] = v;
        ctx->pk_tab[pk_tab_at(slots, m, n)] = (uint16_t)v;
      }
    } else if (v >= 0 && v < kFp64NumVariants) {
      ctx->tune[key] = v;
    }
  }
  fclose(f);
}

// A note line in the cache file (kept for the record, ignored when loading).
static void tune_note(bsm_ctx ctx, const std::string &text) {
  if (ctx->tune_path.empty()) return;
  FILE *f = fopen(ctx->tune_path.c_str(), "a");
  if (!f) return;
  fprintf(f, "# %s\n", text.c_str());
  fclose(f);
}

static void tune_save(bsm_ctx ctx, const std::string &key, int v, double ms) {
  ctx->tune[key] = v;
  ctx->tune_version++;
  if (ctx->tune_path.empty()) return;
  FILE *f = fopen(ctx->tune_path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s %d %.6f\n", key.c_str(), v, ms);
  fclose(f);
}

// A packed kernel's slot shapes are tuned per (m, n) class of C blocks that
// are one tile (m, n <= 16), where the shape kinds are exact.
static bool tiles_need_tuning(bsm_ctx ctx, bsm_mat A, bsm_mat B, int variant) {
  if ((variant != kFp64Pk12 && variant != kFp64Pk16) || !A->kinds_exact || !B->kinds_exact)
    return false;
  for (int32_t m : A->row_kinds)
    for (int32_t n : B->col_kinds)
      if (m < kPkTabEdge && n < kPkTabEdge &&
          !ctx->tune.count(tune_key_tile(pk_slots(variant), m, n)))
        return true;
  return false;
}

static bool needs_tuning(bsm_ctx ctx, bsm_mat A, bsm_mat B, const bsm_opts &o) {
  if (!o.autotune || o.precision != BSM_PREC_FP64 || o.fp64_kernel) return false;
  if (o.launch != BSM_LAUNCH_PER_STACK) {
    auto it = ctx->tune.find(tune_key_all(A, B));
    return it == ctx->tune.end() || tiles_need_tuning(ctx, A, B, it->second);
  }
  for (int32_t m : A->row_kinds)
    for (int32_t n : B->col_kinds)
      if (!ctx->tune.count(tune_key_class(m, n))) return true;
  return false;
}

static_assert((int)kFp64T16B2 == (int)BSM_FP64_T16_B2 && (int)kFp64T16B3 == (int)BSM_FP64_T16_B3 &&
                  (int)kFp64T32 == (int)BSM_FP64_T32 && (int)kFp64Pk12 == (int)BSM_FP64_PK12 &&
                  (int)kFp64Pk16 == (int)BSM_FP64_PK16 && (int)kFp64G8 == (int)BSM_FP64_G8 &&
                  (int)kFp64NumVariants == (int)BSM_FP64_NUM_KERNELS,
              "public and internal FP64 kernel numbers differ");

// The default FP64 kernel for a result C: the packed kernel, unless the last
// multiply into C had fewer than 4 block products per C block (the sizes of
// the previous result, or of this one once the symbolic totals were read).
static int fp64_default(bsm_ctx ctx, bsm_mat C) {
  if (C->hint_blk > 0 && ctx->hint_prod < 4 * C->hint_blk)  // few products per C block
    return (C->max_row <= 8 && C->max_col <= 8) ? kFp64G8 : kFp64T16B2;
  return kFp64Pk12;
}

// The forced kernel, else the tuned one, else the default.
static int variant_or_default(bsm_ctx ctx, bsm_mat C, const bsm_opts &o,
                              const std::string &key) {
  if (o.fp64_kernel > 0) return o.fp64_kernel - 1;
  auto it = ctx->tune.find(key);
  return it == ctx->tune.end() ? fp64_default(ctx, C) : it->second;
}

// The split-precision kernel of a multiply: the forced one, else the per-block
// kernel (measured faster on the water and amorphous systems); the per-block
// kernel also when B's slice offsets do not fit the panel's 32-bit records
// (16-byte units).
static int split_kernel_of(const bsm_opts &o, bsm_mat B) {
  const int64_t unit16 = o.precision == BSM_PREC_SPLIT_BF16X3 ? 3 : 2;
  if (B && B->nnz * unit16 >= (int64_t)INT32_MAX) return BSM_SPLIT_BLOCKS;
  return o.split_kernel > 0 ? o.split_kernel - 1 : BSM_SPLIT_BLOCKS;
}

struct Launch {
  bsm_ctx ctx;
  bsm_mat A, B, C;
  double alpha, beta, eps;
  bsm_opts o;
  int slot;
  cudaStream_t s;
  bool use_cin, split, prof;
  bool host_written;  // every numeric launch so far stored the host copy itself
  bool gated;         // call the context's slice gate between numeric slices
  DevMat dA, dB, dC;
  DevWs ws;
  DevOut out;
};

// norms, operand slices, symbolic count and scan
static int stage_a(Launch &L, bool record) {
  bsm_ctx ctx = L.ctx;
  int rc;
  if (L.prof && record) CK(cudaEventRecord(ctx->prof_ev[L.slot][0], L.s));
  if ((rc = enqueue_norms(ctx, L.A, L.s))) return rc;
  ctx->launches++;
  if (L.B != L.A) {
    if ((rc = enqueue_norms(ctx, L.B, L.s))) return rc;
    ctx->launches++;
  }
  if (L.split) {  // operand slices for the tensor-core products
    const int grid = ctx->nsm * 16;
    bsm_mat A = L.A, B = L.B;
    CK(launch_split(L.o.precision, A->row_sizes, A->col_sizes, A->front.blk_row, A->front.col_idx,
                    A->front.blk_off, A->front.vals, A->front.hdr, A->split_left,
                    B == A ? A->split_right : nullptr, grid, L.s));
    ctx->launches++;
    if (B != A) {
      CK(launch_split(L.o.precision, B->row_sizes, B->col_sizes, B->front.blk_row,
                      B->front.col_idx, B->front.blk_off, B->front.vals, B->front.hdr, nullptr,
                      B->split_right, grid, L.s));
      ctx->launches++;
    }
  }
  if (L.prof && record) CK(cudaEventRecord(ctx->prof_ev[L.slot][1], L.s));
  CK(launch_symbolic_count(L.dA, L.dB, L.dC, L.use_cin ? 1 : 0, L.eps, L.ws, ctx->nsm * 6, L.s));
  ctx->launches++;
  CK(launch_symbolic_scan(L.A->nbr, L.ws, L.out, ctx->d_status, L.s));
  ctx->launches++;
  return BSM_OK;
}

// max_m, max_n: the largest C block row / column size the launch can meet
// (they pick the split-precision tile paths).
static int launch_numeric(Launch &L, int variant, const int32_t *items, const int64_t *seg,
                          int max_m, int max_n) {
  bsm_ctx ctx = L.ctx;
  if (L.split) {
    const int smax = L.A->max_col;
    if (split_kernel_of(L.o, L.B) == BSM_SPLIT_CHUNKS) {
      ctx->last_split = BSM_SPLIT_CHUNKS;
      // the C blocks whose MMA problem fits 16 x 16; the others (if any) to
      // the large-block instance of the per-block kernel
      CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
      CK(launch_numeric_split_cat(L.o.precision, L.dA, L.dB, L.out, L.dC, L.A->split_left,
                                  L.B->split_right, L.alpha, L.beta, L.ws, ctx->d_status, items,
                                  seg, smax, ctx->nsm, ctx->d_work, L.s));
      if (!(max_m <= 16 && max_n <= 16)) {
        ctx->launches++;
        CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
        CK(launch_numeric_split(L.o.precision, 2, L.dA, L.dB, L.out, L.dC, L.A->split_left,
                                L.B->split_right, L.alpha, L.beta, L.ws, ctx->d_status, items,
                                seg, smax, ctx->nsm, ctx->d_work, L.s));
      }
      ctx->launches++;
      return BSM_OK;
    }
    ctx->last_split = BSM_SPLIT_BLOCKS;
    if (max_m <= 16 && max_n <= 16) {
      CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
      CK(launch_numeric_split(L.o.precision, 0, L.dA, L.dB, L.out, L.dC, L.A->split_left,
                              L.B->split_right, L.alpha, L.beta, L.ws, ctx->d_status, items, seg,
                              smax, ctx->nsm, ctx->d_work, L.s));
    } else {
      CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
      CK(launch_numeric_split(L.o.precision, 1, L.dA, L.dB, L.out, L.dC, L.A->split_left,
                              L.B->split_right, L.alpha, L.beta, L.ws, ctx->d_status, items, seg,
                              smax, ctx->nsm, ctx->d_work, L.s));
      ctx->launches++;
      CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
      CK(launch_numeric_split(L.o.precision, 2, L.dA, L.dB, L.out, L.dC, L.A->split_left,
                              L.B->split_right, L.alpha, L.beta, L.ws, ctx->d_status, items, seg,
                              smax, ctx->nsm, ctx->d_work, L.s));
    }
  } else {
    if (fp64_variant_uses_work(variant))
      CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
    ctx->last_fp64 = variant;
    L.host_written = L.host_written && fp64_variant_writes_host(variant);
    CK(launch_numeric_fp64(variant, L.dA, L.dB, L.out, L.dC, L.alpha, L.beta, L.ws,
                           ctx->d_status, items, seg,
                           ctx->nsm * fp64_variant_blocks_per_sm(variant), ctx->d_work, max_m,
                           max_n, L.s));
  }
  ctx->launches++;
  return BSM_OK;
}

// Time `variant` over a work range (blocking; only while tuning).
static int time_variant(Launch &L, int variant, const int32_t *items, const int64_t *seg,
                        int max_m, int max_n, double *ms_out) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e30;
  int rc = BSM_OK;
  for (int rep = 0; rep < 3 && rc == BSM_OK; rep++) {
    cudaEventRecord(e0, L.s);
    rc = launch_numeric(L, variant, items, seg, max_m, max_n);
    cudaEventRecord(e1, L.s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = BSM_ERR_CUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, (double)ms);  // the first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return rc;
}

// Fewest C blocks of a class for its slot shape to be timed (below, the
// formula's shape is kept and recorded).
constexpr int64_t kTileTuneMinBlocks = 256;

// Tune the packed kernel's (variant: 12 or 16 slots) slot shape (nT, G) of
// every one-tile class (m, n <= 16) of this multiply that has no entry yet: the
// C blocks are grouped by class, and each candidate -- every G up to the
// largest with the fewest passes nT = ceil(m n G / 32) <= slots -- is timed on
// the class's blocks alone
// (best of two runs after one warm-up) with the table entry set to it. The
// fastest is kept in the table the persistent launch reads (and in the cache
// file, with the formula's time beside it as a note). Blocking.
static int tune_pk_tiles(Launch &L, int variant) {
  bsm_ctx ctx = L.ctx;
  const int slots = pk_slots(variant);
  const int ncc = (int)L.B->col_kinds.size();
  const int ncls = (int)L.A->row_kinds.size() * ncc;
  if (ncls > kMaxClasses) return BSM_OK;
  CK(launch_class_sort(L.out, L.A->row_cls, L.B->col_cls, ncc, ncls, ctx->d_status,
                       ctx->cls_counts, ctx->cls_cursor, ctx->cls_segs, ctx->cls_items, ctx->nsm,
                       L.s));
  ctx->launches += 3;
  std::vector<int64_t> segs(2 * (size_t)ncls);
  CK(cudaMemcpyAsync(segs.data(), ctx->cls_segs, segs.size() * sizeof(int64_t),
                     cudaMemcpyDeviceToHost, L.s));
  CK(cudaStreamSynchronize(L.s));
  L.ws.pk_tab = ctx->d_pk_tab;
  for (int c = 0; c < ncls; c++) {
    const int m = L.A->row_kinds[c / ncc], n = L.B->col_kinds[c % ncc];
    const std::string key = tune_key_tile(slots, m, n);
    if (m >= kPkTabEdge || n >= kPkTabEdge || ctx->tune.count(key)) continue;
    const int idx = pk_tab_at(slots, m, n), te = m * n;
    const uint16_t formula = ctx->pk_tab[idx];
    uint16_t best = formula;
    double best_ms = 0, formula_ms = 0;
    std::string tried;  // "nT/G/ms" of every candidate, for the note
    if (segs[2 * c + 1] - segs[2 * c] >= kTileTuneMinBlocks) {
      best_ms = 1e30;
      for (int g = 1; g <= kPkMaxGroups; g++) {
        const int nt = (te * g + 31) / 32;
        if (nt > slots) break;
        if (!pk_shape_ok(slots, te, nt, g)) continue;
        const uint16_t v = (uint16_t)(nt << 8 | g);
        CK(cudaMemcpyAsync(ctx->d_pk_tab + idx, &v, sizeof(v), cudaMemcpyHostToDevice, L.s));
        double ms;
        int rc = time_variant(L, variant, ctx->cls_items, ctx->cls_segs + 2 * c, m, n, &ms);
        if (rc) return rc;
        if (v == formula) formula_ms = ms;
        if (ms < best_ms) best_ms = ms, best = v;
        char one[48];
        snprintf(one, sizeof(one), " %d/%d/%.4f", nt, g, ms);
        tried += one;
      }
      char note[160];
      snprintf(note, sizeof(note), "%s %lld blocks: formula nT=%d G=%d %.4f ms, tuned nT=%d G=%d %.4f ms;",
               key.c_str(), (long long)(segs[2 * c + 1] - segs[2 * c]), formula >> 8, formula & 0xFF,
               formula_ms, best >> 8, best & 0xFF, best_ms);
      tune_note(ctx, std::string(note) + " nT/G/ms:" + tried);
    }
    ctx->pk_tab[idx] = best;
    CK(cudaMemcpyAsync(ctx->d_pk_tab + idx, &ctx->pk_tab[idx], sizeof(uint16_t),
                       cudaMemcpyHostToDevice, L.s));
    CK(cudaStreamSynchronize(L.s));
    tune_save(ctx, key, best, best_ms);
  }
  ctx->ws.pk_tab = ctx->d_pk_tab;
  return BSM_OK;
}

// Words of the fill pass's per-row bit matrix: a bound on a C block row's
// blocks (B's block columns, and A's longest row times B's) times the words of
// A's longest row; 0 (the largest) where a pattern was made on the device or C
// enters (beta != 0). Smaller matrices leave room for more resident blocks of
// the latency-bound placement on very sparse inputs; a row beyond the bound
// takes the slower per-window passes.
static int fill_mask_words(const Launch &L) {
  if (L.use_cin || L.A->max_row_blocks < 0 || L.B->max_row_blocks < 0) return 0;
  const int64_t cblk = std::min<int64_t>(L.B->nbc, L.A->max_row_blocks * L.B->max_row_blocks);
  const int64_t words = cblk * ((L.A->max_row_blocks + 31) / 32);
  return (int)std::min<int64_t>(std::max<int64_t>((words + 31) & ~31ll, 32), 8192);
}

// fill, shape-class grouping (per-stack), numeric
static int stage_b(Launch &L, bool record, bool may_tune) {
  bsm_ctx ctx = L.ctx;
  int rc;
  L.host_written = true;  // the split kernels store it; FP64 launches update this
  CK(launch_symbolic_fill(L.dA, L.dB, L.dC, L.use_cin ? 1 : 0, L.eps, L.ws, L.out, ctx->d_status,
                          ctx->nsm, fill_mask_words(L), L.s));
  ctx->launches++;
  if (L.prof && record) CK(cudaEventRecord(ctx->prof_ev[L.slot][2], L.s));
  if (L.split && split_kernel_of(L.o, L.B) == BSM_SPLIT_PANEL) {
    // the row-panel kernel takes every C block row in one launch, whatever the
    // launch mode (its work unit is a row, not a shape class): the prep kernel
    // orders each tile's products by A block, the panel kernel multiplies, and
    // the per-block kernel takes the rows the prep left to it (none unless a
    // row of A has more than 1024 blocks)
    if ((rc = panel_ws(ctx, L.A->nbr))) return rc;
    CK(cudaMemsetAsync(ctx->cls_segs, 0, 2 * sizeof(int64_t), L.s));
    CK(launch_panel_prep(L.o.precision, L.dA, L.dB, L.out, L.ws, ctx->pw, ctx->d_status,
                         L.A->max_row, ctx->nsm, L.s));
    ctx->launches++;
    CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), L.s));
    CK(launch_numeric_split_panel(L.o.precision, L.dA, L.dB, L.out, L.dC, L.A->split_left,
                                  L.B->split_right, L.alpha, L.beta, L.ws, ctx->pw,
                                  ctx->d_status, L.A->max_row, ctx->nsm, ctx->d_work, L.s));
    ctx->launches++;
    if ((rc = launch_numeric(L, 0, ctx->cls_items, ctx->cls_segs, L.A->max_row, L.B->max_col)))
      return rc;
    ctx->last_split = BSM_SPLIT_PANEL;
  } else if (L.o.launch == BSM_LAUNCH_PER_STACK) {
    const int ncc = (int)L.B->col_kinds.size();
    const int ncls = (int)L.A->row_kinds.size() * ncc;
    CK(launch_class_sort(L.out, L.A->row_cls, L.B->col_cls, ncc, ncls, ctx->d_status,
                         ctx->cls_counts, ctx->cls_cursor, ctx->cls_segs, ctx->cls_items, ctx->nsm,
                         L.s));
    ctx->launches += 3;
    for (int c = 0; c < ncls; c++) {
      const int m = L.A->row_kinds[c / ncc], n = L.B->col_kinds[c % ncc];
      const std::string key = tune_key_class(m, n);
      const int64_t *seg = ctx->cls_segs + 2 * c;
      if (may_tune && L.o.autotune && !L.o.fp64_kernel && !L.split && !ctx->tune.count(key)) {
        int best = fp64_default(ctx, L.C);
        double best_ms = 1e30;
        for (int v = 0; v < kFp64NumVariants; v++) {
          double ms;
          if ((rc = time_variant(L, v, ctx->cls_items, seg, m, n, &ms))) return rc;
          if (ms < best_ms) best_ms = ms, best = v;
        }
        tune_save(ctx, key, best, best_ms);
      }
      if ((rc = launch_numeric(L, variant_or_default(ctx, L.C, L.o, key), ctx->cls_items, seg, m, n)))
        return rc;
    }
  } else {
    const std::string key = tune_key_all(L.A, L.B);
    if (may_tune && L.o.autotune && !L.o.fp64_kernel && !L.split && !ctx->tune.count(key)) {
      int best = fp64_default(ctx, L.C);
      double best_ms = 1e30;
      for (int v = 0; v < kFp64NumVariants; v++) {
        double ms;
        if ((rc = time_variant(L, v, nullptr, nullptr, L.A->max_row, L.B->max_col, &ms)))
          return rc;
        if (ms < best_ms) best_ms = ms, best = v;
      }
      tune_save(ctx, key, best, best_ms);
    }
    const int variant = variant_or_default(ctx, L.C, L.o, key);
    if (may_tune && L.o.autotune && !L.o.fp64_kernel && !L.split &&
        tiles_need_tuning(ctx, L.A, L.B, variant) && (rc = tune_pk_tiles(L, variant)))
      return rc;
    // C blocks in A's row order where A has one, else in C's row order
    const int32_t *items = nullptr;
    if (L.A->order_id) {
      CK(launch_order_items(L.out, L.A->row_order, L.A->row_order + L.A->nbr, L.A->nbr,
                            ctx->d_status, ctx->ord_start, ctx->cls_items, ctx->nsm, L.s));
      ctx->launches += 2;
      items = ctx->cls_items;
    }
    if (!L.split && L.o.numeric_slices > 1) {
      // consecutive ranges of the C blocks (of the work list) in launches of their own
      const int n = L.o.numeric_slices;
      CK(launch_slice_segs(ctx->d_status, n, ctx->cls_segs, L.s));
      ctx->launches++;
      for (int x = 0; x < n; x++) {
        if (L.gated && x > 0) {  // the slice before done, then the gate
          CK(cudaEventRecord(ctx->ev_gate, L.s));
          CK(cudaEventSynchronize(ctx->ev_gate));
          ctx->gate(ctx->gate_arg);
        }
        if ((rc = launch_numeric(L, variant, items, ctx->cls_segs + 2 * x, L.A->max_row,
                                 L.B->max_col)))
          return rc;
      }
    } else if ((rc = launch_numeric(L, variant, items, nullptr, L.A->max_row, L.B->max_col))) {
      return rc;
    }
  }
  // the host copy of the values, where a numeric kernel did not store it
  if (L.out.host_vals && !L.host_written) {
    CK(launch_copy_out(L.out, ctx->d_status, ctx->nsm, L.s));
    ctx->launches++;
  }
  if (L.prof && record) {
    CK(cudaEventRecord(ctx->prof_ev[L.slot][3], L.s));
    ctx->prof_pending[L.slot] = true;
  }
  return BSM_OK;
}

static void graph_key(const Launch &L, std::vector<uint64_t> &k) {
  auto put = [&](const void *p) { k.push_back((uint64_t)(uintptr_t)p); };
  auto num = [&](int64_t v) { k.push_back((uint64_t)v); };
  auto dbl = [&](double v) {
    uint64_t u;
    memcpy(&u, &v, 8);
    k.push_back(u);
  };
  for (bsm_mat M : {L.A, L.B, L.C}) {
    const Buf *bs[2] = {&M->front, &M->back};
    for (const Buf *b : bs) {
      put(b->row_ptr), put(b->col_idx), put(b->blk_row), put(b->blk_off), put(b->norms);
      put(b->normsf);
      put(b->vals), put(b->hdr), num(b->cap_blk), num(b->cap_nnz);
    }
    put(M->split_left), put(M->split_right), put(M->row_sizes), put(M->col_sizes);
    put(M->row_cls), put(M->col_cls), num(M->nbr), num(M->nbc);
  }
  const DevWs &w = L.ws;
  put(w.row_cblk), put(w.row_prod), put(w.row_nnz), put(w.row_cand), put(w.row_flops);
  put(w.prod_off), put(w.nnz_off), put(w.cnt), put(w.c_cin), put(w.prod_ptr), put(w.prods);
  num(w.cap_prod), num(L.out.cap_blk), num(L.out.cap_nnz);
  put(L.ctx->cls_items), put(L.ctx->ord_start), put(L.s);
  put(L.A->row_order), num((int64_t)L.A->order_id);
  put(L.ctx->pw.recs), put(L.ctx->pw.tiles), put(L.ctx->pw.row_nt);
  dbl(L.alpha), dbl(L.beta), dbl(L.eps);
  num(L.o.precision), num(L.o.launch), num(L.o.fp64_kernel), num((int64_t)L.ctx->tune_version);
  num(L.o.split_kernel), num(L.o.numeric_slices);
  put(L.out.host_vals), num(L.out.host_cap);
  num(fp64_default(L.ctx, L.C));
}

// Enqueue one multiply. sync_sizes: read the totals back after the scan and
// size the buffers exactly before the fill and numeric passes.
static int run_multiply(bsm_ctx ctx, double alpha, bsm_mat A, bsm_mat B, double beta, bsm_mat C,
                        double eps, const bsm_opts &o, bool sync_sizes, int slot,
                        bsm_stats *stats) {
  Launch L{};
  L.ctx = ctx;
  L.A = A, L.B = B, L.C = C;
  L.alpha = alpha, L.beta = beta, L.eps = eps;
  L.o = o;
  L.slot = slot;
  L.s = o.stream ? (cudaStream_t)o.stream : ctx->stream;
  L.use_cin = (beta != 0.0);
  L.split = o.precision != BSM_PREC_FP64;
  if (L.s != ctx->stream) CK(cudaStreamWaitEvent(L.s, ctx->ev_last, 0));
  int rc;
  if ((rc = ws_rows(ctx, A->nbr))) return rc;
  if ((rc = buf_grow(C, C->back, 0, 0, true))) return rc;
  if (ctx->cap_cblk < 0 && (rc = ws_grow(ctx, 0, 0))) return rc;
  if (L.split) {
    if ((rc = split_buffers(A, o.precision, true, B == A))) return rc;
    if (B != A && (rc = split_buffers(B, o.precision, false, true))) return rc;
  }
  // C's block rows are A's: C inherits A's row order (a hint for the multiply
  // that takes C on the left next)
  if (A->order_id && C->order_id != A->order_id && C->nbr == A->nbr) {
    if (!C->row_order && (rc = dev_alloc(&C->row_order, 2 * (int64_t)C->nbr))) return rc;
    CK(cudaMemcpyAsync(C->row_order, A->row_order, 2 * (size_t)C->nbr * sizeof(int32_t),
                       cudaMemcpyDeviceToDevice, L.s));
    C->order_id = A->order_id;
    C->order_ptr.clear();  // not computed from C's own pattern
    C->order_col.clear();
  }
  L.dA = dev_view(A), L.dB = dev_view(B), L.dC = dev_view(C);
  C->max_row_blocks = -1;  // the result's pattern is made on the device
  double *host_dev = nullptr;  // device address of o.host_values
  if (o.host_values) {
    cudaPointerAttributes pa{};
    CK(cudaPointerGetAttributes(&pa, o.host_values));
    host_dev = static_cast<double *>(pa.devicePointer);
  }
  auto make_out = [&]() {
    L.ws = ctx->ws;
    L.out = dev_out(C, C->back);
    L.out.host_vals = host_dev;
    L.out.host_cap = o.host_values ? o.host_cap : 0;
    // capacities of the per-C-block scratch cap the block count as well
    L.out.cap_blk = std::min<int64_t>(L.out.cap_blk, std::max<int64_t>(ctx->cap_cblk - 1, 0));
  };
  make_out();
  // the panel kernel's work buffers before any capture (no allocation inside one)
  if (L.split && split_kernel_of(o, B) == BSM_SPLIT_PANEL && (rc = panel_ws(ctx, A->nbr)))
    return rc;
  const bool use_graph = o.graph && !sync_sizes;
  L.prof = ctx->prof && !use_graph;
  if (stats) CK(cudaEventRecord(ctx->ev_t0, L.s));

  if (use_graph) {
    std::vector<uint64_t> key;
    graph_key(L, key);
    bsm_ctx_s::GraphEntry *hit = nullptr;
    for (auto &g : ctx->graphs)
      if (g.key == key) hit = &g;
    if (!hit) {
      // a multiply with new arguments: capture it once (tuning already done)
      if (needs_tuning(ctx, A, B, o)) {
        // run uncaptured first so that the missing tuner entries are filled
        if ((rc = stage_a(L, false)) || (rc = stage_b(L, false, true))) return rc;
        graph_key(L, key);  // the tuner may have changed the table version
        for (auto &g : ctx->graphs)
          if (g.key == key) hit = &g;
      }
    }
    if (!hit) {
      const int64_t l0 = ctx->launches;
      CK(cudaStreamBeginCapture(L.s, cudaStreamCaptureModeThreadLocal));
      rc = stage_a(L, false);
      if (rc == BSM_OK) rc = stage_b(L, false, false);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(L.s, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
      cudaGraphExec_t exec = nullptr;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
      if ((int)ctx->graphs.size() >= kMaxGraphs) {  // evict the least recently used
        auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                    [](const bsm_ctx_s::GraphEntry &a,
                                       const bsm_ctx_s::GraphEntry &b) { return a.used < b.used; });
        cudaGraphExecDestroy(lru->exec);
        ctx->graphs.erase(lru);
      }
      bsm_ctx_s::GraphEntry e;
      e.key = key;
      e.exec = exec;
      e.launches = (int)(ctx->launches - l0);
      ctx->launches = l0;  // counted when the graph runs
      ctx->graphs.push_back(e);
      hit = &ctx->graphs.back();
    }
    hit->used = ++ctx->graph_clock;
    CK(cudaGraphLaunch(hit->exec, L.s));
    ctx->launches += hit->launches;
  } else {
    L.gated = ctx->gate != nullptr;
    if ((rc = stage_a(L, true))) return rc;
    if (sync_sizes) {
      DevStatus h{};
      CK(cudaMemcpyAsync(&h, ctx->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, L.s));
      CK(cudaStreamSynchronize(L.s));
      C->hint_blk = h.nblk_c;
      C->hint_nnz = h.nnz_c;
      ctx->hint_prod = std::max(ctx->hint_prod, h.nprod);
      if (h.overflow) {
        if (h.nblk_c >= (int64_t)INT32_MAX) return BSM_ERR_UNSUPPORTED;
        if ((rc = buf_grow(C, C->back, h.nblk_c, h.nnz_c, false))) return rc;
        if ((rc = ws_grow(ctx, h.nblk_c, h.nprod))) return rc;
        make_out();
        CK(launch_symbolic_scan(A->nbr, L.ws, L.out, ctx->d_status, L.s));
        ctx->launches++;
      }
    }
    if ((rc = stage_b(L, true, true))) return rc;
  }
  if (stats) CK(cudaEventRecord(ctx->ev_t1, L.s));
  CK(cudaMemcpyAsync(&ctx->h_slots[slot], ctx->d_status, sizeof(DevStatus),
                     cudaMemcpyDeviceToHost, L.s));
  CK(cudaEventRecord(ctx->slot_ev[slot], L.s));
  CK(cudaEventRecord(ctx->ev_last, L.s));
  if (L.s != ctx->stream) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_last, 0));
  return BSM_OK;
}

// Wait for M's pending result; on overflow, grow and recompute (blocking).
static int resolve(bsm_mat M, bsm_stats *timed) {
  if (!M->pend.active) return BSM_OK;
  bsm_ctx ctx = M->ctx;
  Pending p = M->pend;
  CK(cudaEventSynchronize(ctx->slot_ev[p.slot]));
  DevStatus h = ctx->h_slots[p.slot];
  M->pend.active = false;
  if (h.error) {  // a bounded device-side wait gave up: the result is incomplete
    M->nblk = M->nnz = 0;
    return BSM_ERR_TIMEOUT;
  }
  M->hint_blk = std::max(M->hint_blk, h.nblk_c);
  M->hint_nnz = std::max(M->hint_nnz, h.nnz_c);
  ctx->hint_prod = std::max(ctx->hint_prod, h.nprod);
  if (!h.overflow) {
    M->nblk = h.nblk_c;
    M->nnz = h.nnz_c;
    return BSM_OK;
  }
  if (timed) timed->retries++;
  // undo the swap (front = the previous contents), then recompute with exact sizes
  std::swap(M->front, M->back);
  if (p.A->pend.active) {
    int rc = resolve(p.A);
    if (rc) return rc;
  }
  if (p.B->pend.active) {
    int rc = resolve(p.B);
    if (rc) return rc;
  }
  int rc = run_multiply(ctx, p.alpha, p.A, p.B, p.beta, M, p.eps, p.opts, true, p.slot, timed);
  if (rc) {  // nothing of the recompute may still run once M's operands change
    cudaStreamSynchronize(p.opts.stream ? (cudaStream_t)p.opts.stream : ctx->stream);
    return rc;
  }
  CK(cudaEventSynchronize(ctx->slot_ev[p.slot]));
  h = ctx->h_slots[p.slot];
  if (h.overflow) return BSM_ERR_NOMEM;
  std::swap(M->front, M->back);
  M->nblk = h.nblk_c;
  M->nnz = h.nnz_c;
  return BSM_OK;
}

// ---------------------------------------------------------------------------
// public API
// ---------------------------------------------------------------------------
extern "C" {

const char *bsm_strerror(int code) {
  switch (code) {
    case BSM_OK: return "ok";
    case BSM_ERR_INVALID_ARG: return "invalid argument";
    case BSM_ERR_DIM_MISMATCH: return "block sizes of the operands do not match";
    case BSM_ERR_DUPLICATE_BLOCK: return "duplicate block in the block list";
    case BSM_ERR_OUT_OF_RANGE: return "block index out of range";
    case BSM_ERR_ALIAS: return "C aliases A or B";
    case BSM_ERR_NOMEM: return "out of device or pinned host memory";
    case BSM_ERR_CUDA: return "CUDA runtime error";
    case BSM_ERR_TIMEOUT: return "device-side wait timed out";
    case BSM_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown error";
  }
}

const char *bsm_last_cuda_error(void) { return g_cuda_err; }

int bsm_ctx_create(int device, bsm_ctx *out) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return BSM_ERR_INVALID_ARG;
  bsm_ctx ctx = new (std::nothrow) bsm_ctx_s();
  if (!ctx) return BSM_ERR_NOMEM;
  ctx->device = device;
  if (device < kCacheDevices) {  // the device-memory cache lives while a context does
    std::lock_guard<std::mutex> lock(g_cache[device].mu);
    g_cache[device].contexts++;
  }
  int rc = BSM_OK;
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device)) !=
          cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&ctx->ev_up, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&ctx->ev_last, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreate(&ctx->ev_t0)) != cudaSuccess ||
      (e = cudaEventCreate(&ctx->ev_t1)) != cudaSuccess ||
      (e = cache_alloc((void **)&ctx->d_status, sizeof(DevStatus))) != cudaSuccess ||
      (e = cache_alloc((void **)&ctx->d_work, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMallocHost((void **)&ctx->h_slots, kSlots * sizeof(DevStatus))) != cudaSuccess) {
    rc = cuda_fail(e, "bsm_ctx_create");
  }
  for (int i = 0; rc == BSM_OK && i < kSlots; i++) {
    if ((e = cudaEventCreateWithFlags(&ctx->slot_ev[i], cudaEventDisableTiming)) != cudaSuccess)
      rc = cuda_fail(e, "cudaEventCreate");
  }
  if (rc == BSM_OK) {
    if ((e = numeric_fp64_init()) != cudaSuccess) rc = cuda_fail(e, "numeric_fp64_init");
    else if ((e = numeric_split_init()) != cudaSuccess) rc = cuda_fail(e, "numeric_split_init");
    else if ((e = numeric_split_panel_init()) != cudaSuccess)
      rc = cuda_fail(e, "numeric_split_panel_init");
  }
  if (rc == BSM_OK) {
    rc = dev_alloc(&ctx->cls_counts, kMaxClasses);
    if (rc == BSM_OK) rc = dev_alloc(&ctx->cls_cursor, kMaxClasses);
    if (rc == BSM_OK) rc = dev_alloc(&ctx->cls_segs, 2 * kMaxClasses);
  }
  if (rc == BSM_OK) {  // the packed kernel's slot shapes: the formula, then tuned entries
    for (int slots : {12, 16})
      for (int tm = 1; tm < kPkTabEdge; tm++)
        for (int tn = 1; tn < kPkTabEdge; tn++) {
          int nt, g;
          pk_formula_shape(slots, tm * tn, &nt, &g);
          ctx->pk_tab[pk_tab_at(slots, tm, tn)] = (uint16_t)(nt << 8 | g);
        }
    tune_load(ctx);
    rc = dev_alloc(&ctx->d_pk_tab, 2 * kPkTabSize);
    if (rc == BSM_OK && (e = cudaMemcpy(ctx->d_pk_tab, ctx->pk_tab, sizeof(ctx->pk_tab),
                                        cudaMemcpyHostToDevice)) != cudaSuccess)
      rc = cuda_fail(e, "slot shape table");
    for (auto &kv : ctx->tune)
      if (rc == BSM_OK && kv.first.find("tile:") != std::string::npos) ctx->ws.pk_tab = ctx->d_pk_tab;
  }
  if (rc == BSM_OK) {
    memset(ctx->h_slots, 0, kSlots * sizeof(DevStatus));
    e = cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset");
  }
  if (rc != BSM_OK) {
    bsm_ctx_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return BSM_OK;
}

int bsm_mat_destroy(bsm_mat m);

int bsm_ctx_destroy(bsm_ctx ctx) {
  if (!ctx) return BSM_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->up_stream) cudaStreamSynchronize(ctx->up_stream);
  while (!ctx->mats.empty()) {
    bsm_mat m = ctx->mats.back();
    m->pend.active = false;
    bsm_mat_destroy(m);
  }
  DevWs &w = ctx->ws;
  dev_free(w.row_cblk);
  dev_free(w.row_prod);
  dev_free(w.row_nnz);
  dev_free(w.row_cand);
  dev_free(w.row_flops);
  dev_free(w.prod_off);
  dev_free(w.nnz_off);
  dev_free(w.cnt);
  dev_free(w.c_cin);
  dev_free(w.prod_ptr);
  dev_free(w.prods);
  dev_free(ctx->d_status);
  dev_free(ctx->d_work);
  dev_free(ctx->cls_items);
  dev_free(ctx->ord_start);
  dev_free(ctx->d_pk_tab);
  dev_free(ctx->pw.recs);
  dev_free(ctx->pw.tiles);
  dev_free(ctx->pw.row_nt);
  dev_free(ctx->cls_counts);
  dev_free(ctx->cls_cursor);
  dev_free(ctx->cls_segs);
  for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  if (ctx->h_slots) cudaFreeHost(ctx->h_slots);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  for (int i = 0; i < kSlots; i++) {
    if (ctx->slot_ev[i]) cudaEventDestroy(ctx->slot_ev[i]);
    for (int e = 0; e < 4; e++)
      if (ctx->prof_ev[i][e]) cudaEventDestroy(ctx->prof_ev[i][e]);
  }
  if (ctx->ev_last) cudaEventDestroy(ctx->ev_last);
  if (ctx->ev_t0) cudaEventDestroy(ctx->ev_t0);
  if (ctx->ev_t1) cudaEventDestroy(ctx->ev_t1);
  if (ctx->ev_gate) cudaEventDestroy(ctx->ev_gate);
  if (ctx->ev_up) cudaEventDestroy(ctx->ev_up);
  if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->device < kCacheDevices) {
    DevCache &c = g_cache[ctx->device];
    std::lock_guard<std::mutex> lock(c.mu);
    if (--c.contexts == 0) cache_flush_locked(c);
  }
  delete ctx;
  return BSM_OK;
}

}  // extern "C"

// Validates a block list against M's block sizes, builds the blocked CSR
// arrays (sorted by row, then column) in the context's pinned staging memory
// and uploads them with the values into M's front buffers (grown when they are
// too small). Synchronises the context stream before returning, so the
// caller's arrays may be reused at once.
// Page-locked staging of an upload's index arrays: row_ptr | col | row | off,
// each part 16-byte aligned.
struct StageLayout {
  size_t b_ptr, b_col, b_off, b_hdr, need;
};
static StageLayout stage_layout(int64_t nbrows, int64_t nblocks) {
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  StageLayout L;
  L.b_ptr = al(((size_t)nbrows + 1) * 4);
  L.b_col = al((size_t)nblocks * 4);
  L.b_off = al(((size_t)nblocks + 1) * 8);
  L.b_hdr = 16;  // the (blocks, values) header, last
  L.need = L.b_ptr + 2 * L.b_col + L.b_off + L.b_hdr;
  return L;
}

// The context's staging, at least `need` bytes, once the copies of an earlier
// upload that may still read it are done. The uploads that use it finish their
// copies (synchronise their stream) before they return, also when they fail;
// the upload stream is synchronised here all the same, which costs nothing
// when it is idle. A multiply still running on the context's stream is not
// waited for.
static int stage_reserve(bsm_ctx ctx, size_t need) {
  CK(cudaStreamSynchronize(ctx->up_stream));
  if (ctx->h_stage_cap < need) {
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_cap = 0;
    const size_t cap = need + need / 4 + 4096;
    if (cudaMallocHost((void **)&ctx->h_stage, cap) != cudaSuccess) {
      cudaGetLastError();
      return BSM_ERR_NOMEM;
    }
    ctx->h_stage_cap = cap;
  }
  return BSM_OK;
}

// Square matrices of at least this many block rows get a row order (below it
// the operands of a multiply stay in L2 in any order).
constexpr int32_t kOrderMinRows = 1024;

// Breadth-first order of the block rows of a square pattern in blocked CSR
// (row i adjacent to the rows named by its column indices): each component
// from its lowest unvisited row, neighbours in column order. order[p] is the
// row at position p, pos[r] the position of row r. O(rows + blocks).
static void bfs_row_order(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *order,
                          int32_t *pos) {
  std::fill(pos, pos + n, -1);
  int32_t head = 0, tail = 0;
  for (int32_t s = 0; s < n; s++) {
    if (pos[s] >= 0) continue;
    pos[s] = tail;
    order[tail++] = s;
    while (head < tail) {
      const int32_t v = order[head++];
      for (int32_t b = row_ptr[v]; b < row_ptr[v + 1]; b++) {
        const int32_t k = col[b];
        if (pos[k] < 0) {
          pos[k] = tail;
          order[tail++] = k;
        }
      }
    }
  }
}

static uint64_t next_order_id() {
  static std::atomic<uint64_t> ids{0};
  return ++ids;
}

static int upload_contents(bsm_mat M, int64_t nblocks, const int32_t *blk_row,
                           const int32_t *blk_col, const double *values, bool exact) {
  bsm_ctx ctx = M->ctx;
  const int32_t nbrows = M->nbr, nbcols = M->nbc;
  const int32_t *row_sizes = M->h_row_sizes.data(), *col_sizes = M->h_col_sizes.data();
  if (nblocks < 0 || (nblocks > 0 && (!blk_row || !blk_col))) return BSM_ERR_INVALID_ARG;
  if (nblocks >= (int64_t)INT32_MAX) return BSM_ERR_UNSUPPORTED;
  // pinned staging: row_ptr | col | row | off (16-byte aligned parts)
  const StageLayout L = stage_layout(nbrows, nblocks);
  int rc0 = stage_reserve(ctx, L.need);
  if (rc0) return rc0;
  const size_t b_ptr = L.b_ptr, b_col = L.b_col;
  int32_t *h_row_ptr = reinterpret_cast<int32_t *>(ctx->h_stage);
  int32_t *h_col = reinterpret_cast<int32_t *>(ctx->h_stage + b_ptr);
  int32_t *h_row = reinterpret_cast<int32_t *>(ctx->h_stage + b_ptr + b_col);
  int64_t *h_off = reinterpret_cast<int64_t *>(ctx->h_stage + b_ptr + 2 * b_col);
  // range check, sortedness and the offsets of the blocks in list order, on
  // several host threads for long lists (the values' copy waits for nnz)
  const int nth = nblocks >= (1 << 17) ? kHostThreads : 1;
  std::vector<int64_t> part(nth + 1, 0);
  std::vector<char> bad(nth, 0), unsorted(nth, 0);
  auto chunk = [&](int t, int64_t &b0, int64_t &b1) {
    b0 = nblocks * t / nth;
    b1 = nblocks * (t + 1) / nth;
  };
  auto check = [&](int t) {  // range, order and the chunk's value count
    int64_t b0, b1, sum = 0;
    chunk(t, b0, b1);
    for (int64_t b = b0; b < b1; b++) {
      const int32_t i = blk_row[b], j = blk_col[b];
      if (i < 0 || i >= nbrows || j < 0 || j >= nbcols) {
        bad[t] = 1;
        return;
      }
      sum += (int64_t)row_sizes[i] * col_sizes[j];
      if (b > 0 && (blk_row[b - 1] > i || (blk_row[b - 1] == i && blk_col[b - 1] >= j)))
        unsorted[t] = 1;
    }
    part[t + 1] = sum;
  };
  auto offsets = [&](int t) {
    int64_t b0, b1;
    chunk(t, b0, b1);
    int64_t o = part[t];
    for (int64_t b = b0; b < b1; b++) {
      h_off[b] = o;
      o += (int64_t)row_sizes[blk_row[b]] * col_sizes[blk_col[b]];
    }
  };
  auto run = [&](auto &&fn) {
    if (nth == 1) {
      fn(0);
      return;
    }
    std::vector<std::thread> th;
    int t = 1;
    try {
      for (; t < nth; t++) th.emplace_back(fn, t);
    } catch (...) {  // no thread could be started: the rest inline
    }
    for (int u = t; u < nth; u++) fn(u);
    fn(0);
    for (auto &x : th) x.join();
  };
  run(check);
  bool sorted = true;
  for (int t = 0; t < nth; t++) {
    if (bad[t]) return BSM_ERR_OUT_OF_RANGE;
    sorted = sorted && !unsorted[t];
    part[t + 1] += part[t];
  }
  run(offsets);
  h_off[nblocks] = part[nth];
  const int64_t nnz = h_off[nblocks];
  std::vector<int64_t> order, list_off;
  if (!sorted) {
    order.resize(nblocks);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      return blk_row[a] != blk_row[b] ? blk_row[a] < blk_row[b] : blk_col[a] < blk_col[b];
    });
    for (int64_t p = 1; p < nblocks; p++)
      if (blk_row[order[p]] == blk_row[order[p - 1]] && blk_col[order[p]] == blk_col[order[p - 1]])
        return BSM_ERR_DUPLICATE_BLOCK;
    list_off.assign(h_off, h_off + nblocks + 1);
  }
  int rc;
  const bool fresh = !M->front.row_ptr;  // buf_grow zeroes new buffers on the context's stream
  if ((rc = buf_grow(M, M->front, nblocks, nnz, exact))) return rc;
  cudaStream_t st = ctx->up_stream;
  cudaError_t e;
  if (fresh && ((e = cudaEventRecord(ctx->ev_up, ctx->stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, ctx->ev_up, 0)) != cudaSuccess))
    return cuda_fail(e, "matrix upload order");
  auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  auto up_fail = [&](cudaError_t err, const char *where) {  // nothing left in flight
    cudaStreamSynchronize(st);
    return cuda_fail(err, where);
  };
  // values in sorted order: start their copy now, it runs while the index
  // arrays are staged
  if (sorted && values && (e = cp(M->front.vals, values, (size_t)nnz * 8)) != cudaSuccess)
    return up_fail(e, "matrix upload values");
  std::vector<double> staged;
  if (sorted) {
    memcpy(h_row, blk_row, (size_t)nblocks * 4);
    memcpy(h_col, blk_col, (size_t)nblocks * 4);
    memset(h_row_ptr, 0, ((size_t)nbrows + 1) * 4);
    for (int64_t b = 0; b < nblocks; b++) h_row_ptr[blk_row[b] + 1]++;
  } else {
    memset(h_row_ptr, 0, ((size_t)nbrows + 1) * 4);
    if (values) staged.resize((size_t)nnz);
    int64_t acc = 0;
    for (int64_t p = 0; p < nblocks; p++) {
      const int64_t b = order[p];
      h_row[p] = blk_row[b];
      h_col[p] = blk_col[b];
      h_off[p] = acc;
      const int64_t len = list_off[b + 1] - list_off[b];
      if (values) memcpy(&staged[acc], values + list_off[b], (size_t)len * sizeof(double));
      acc += len;
      h_row_ptr[blk_row[b] + 1]++;
    }
  }
  M->max_row_blocks = 0;
  for (int32_t i = 0; i < nbrows; i++)
    M->max_row_blocks = std::max<int64_t>(M->max_row_blocks, h_row_ptr[i + 1]);
  for (int32_t i = 0; i < nbrows; i++) h_row_ptr[i + 1] += h_row_ptr[i];
  // the row order of the numeric phase (host BFS over the sorted pattern),
  // kept as it is when the pattern is the one it was computed from (an
  // iteration that assigns new values to the same pattern)
  std::vector<int32_t> h_order;
  if (nbrows == nbcols && nbrows >= kOrderMinRows) {
    const bool same = M->order_id && M->order_ptr.size() == (size_t)nbrows + 1 &&
                      M->order_col.size() == (size_t)nblocks &&
                      !memcmp(M->order_ptr.data(), h_row_ptr, ((size_t)nbrows + 1) * 4) &&
                      (nblocks == 0 || !memcmp(M->order_col.data(), h_col, (size_t)nblocks * 4));
    if (!same) {
      M->order_id = 0;
      h_order.resize(2 * (size_t)nbrows);
      bfs_row_order(nbrows, h_row_ptr, h_col, h_order.data(), h_order.data() + nbrows);
      if (!M->row_order && (rc = dev_alloc(&M->row_order, 2 * (int64_t)nbrows))) {
        cudaStreamSynchronize(st);
        return rc;
      }
      if ((e = cp(M->row_order, h_order.data(), h_order.size() * 4)) != cudaSuccess)
        return up_fail(e, "matrix upload row order");
      M->order_ptr.assign(h_row_ptr, h_row_ptr + nbrows + 1);
      M->order_col.assign(h_col, h_col + nblocks);
      M->order_id = next_order_id();
    }
  } else {
    M->order_id = 0;
  }
  // page-locked like the rest: a copy from pageable memory may wait for other work
  int64_t *hdr = reinterpret_cast<int64_t *>(ctx->h_stage + L.need - L.b_hdr);
  hdr[0] = nblocks;
  hdr[1] = nnz;
  if ((e = cp(M->front.row_ptr, h_row_ptr, ((size_t)nbrows + 1) * 4)) != cudaSuccess ||
      (e = cp(M->front.col_idx, h_col, (size_t)nblocks * 4)) != cudaSuccess ||
      (e = cp(M->front.blk_row, h_row, (size_t)nblocks * 4)) != cudaSuccess ||
      (e = cp(M->front.blk_off, h_off, (size_t)nblocks * 8)) != cudaSuccess ||
      (e = cp(M->front.hdr, hdr, 2 * sizeof(int64_t))) != cudaSuccess)
    return up_fail(e, "matrix upload");
  if (!sorted && values) {
    if ((e = cp(M->front.vals, staged.data(), (size_t)nnz * 8)) != cudaSuccess)
      return up_fail(e, "matrix upload values");
  } else if (!values && nnz > 0) {
    if ((e = cudaMemsetAsync(M->front.vals, 0, (size_t)nnz * 8, st)) != cudaSuccess)
      return up_fail(e, "matrix upload zero");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "matrix upload sync");
  M->nblk = nblocks;
  M->nnz = nnz;
  return BSM_OK;
}

// Records M's use event on stream s after the work enqueued there.
static int mark_use(bsm_mat M, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!M->ev_use) e = cudaEventCreateWithFlags(&M->ev_use, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(M->ev_use, s);
  if (e != cudaSuccess) {
    // an event that was never recorded would let an upload overwrite M early
    cudaStreamSynchronize(s);
    return cuda_fail(e, "matrix use event");
  }
  return BSM_OK;
}

// Work that reads M as an input, or writes it, must be finished (and any
// recompute that would read M done) before M's contents change. Only
// multiplies leave work on the device after they return; each records M's
// use event, so other work still running (a multiply of other matrices) is
// not waited for.
static int quiesce(bsm_mat m) {
  bsm_ctx ctx = m->ctx;
  if (m->ev_use) CK(cudaEventSynchronize(m->ev_use));
  for (bsm_mat o : std::vector<bsm_mat>(ctx->mats))
    if (o != m && o->pend.active && (o->pend.A == m || o->pend.B == m)) {
      int rc = resolve(o);
      if (rc) return rc;
    }
  return BSM_OK;
}

extern "C" {

int bsm_mat_create(bsm_ctx ctx, int32_t nbrows, const int32_t *row_sizes, int32_t nbcols,
                   const int32_t *col_sizes, int64_t nblocks, const int32_t *blk_row,
                   const int32_t *blk_col, const double *values, bsm_mat *out) {
  if (!ctx || !out || nbrows < 0 || nbcols < 0 || nblocks < 0) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  if ((nbrows > 0 && !row_sizes) || (nbcols > 0 && !col_sizes)) return BSM_ERR_INVALID_ARG;
  if (nblocks > 0 && (!blk_row || !blk_col)) return BSM_ERR_INVALID_ARG;
  if (nblocks >= (int64_t)INT32_MAX) return BSM_ERR_UNSUPPORTED;
  for (int32_t i = 0; i < nbrows; i++)
    if (row_sizes[i] <= 0) return BSM_ERR_INVALID_ARG;
  for (int32_t j = 0; j < nbcols; j++)
    if (col_sizes[j] <= 0) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(ctx);
  if (rc) return rc;
  bsm_mat M = new (std::nothrow) bsm_mat_s();
  if (!M) return BSM_ERR_NOMEM;
  M->ctx = ctx;
  M->nbr = nbrows;
  M->nbc = nbcols;
  M->h_row_sizes.assign(row_sizes, row_sizes + nbrows);
  M->h_col_sizes.assign(col_sizes, col_sizes + nbcols);
  for (int32_t v : M->h_row_sizes) M->max_row = std::max(M->max_row, v);
  for (int32_t v : M->h_col_sizes) M->max_col = std::max(M->max_col, v);
  // shape kinds of the block rows and columns
  auto kinds = [&](const std::vector<int32_t> &sizes, std::vector<int32_t> &kind,
                   std::vector<int32_t> &cls) {
    kind = sizes;
    std::sort(kind.begin(), kind.end());
    kind.erase(std::unique(kind.begin(), kind.end()), kind.end());
    cls.resize(sizes.size());
    if ((int)kind.size() > kMaxKinds) {  // too many sizes: one kind, keyed by the largest
      kind = {kind.back()};
      M->kinds_exact = false;
      std::fill(cls.begin(), cls.end(), 0);
      return;
    }
    for (size_t i = 0; i < sizes.size(); i++)
      cls[i] = (int32_t)(std::lower_bound(kind.begin(), kind.end(), sizes[i]) - kind.begin());
  };
  std::vector<int32_t> h_row_cls, h_col_cls;
  kinds(M->h_row_sizes, M->row_kinds, h_row_cls);
  kinds(M->h_col_sizes, M->col_kinds, h_col_cls);
  ctx->mats.push_back(M);
  auto fail = [&](int code) {
    bsm_mat_destroy(M);
    return code;
  };
  if ((rc = dev_alloc(&M->row_sizes, nbrows)) || (rc = dev_alloc(&M->col_sizes, nbcols)) ||
      (rc = dev_alloc(&M->row_cls, nbrows)) || (rc = dev_alloc(&M->col_cls, nbcols)))
    return fail(rc);
  cudaStream_t s = ctx->stream;
  auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  cudaError_t e;
  if ((e = cp(M->row_sizes, row_sizes, (size_t)nbrows * 4)) != cudaSuccess ||
      (e = cp(M->col_sizes, col_sizes, (size_t)nbcols * 4)) != cudaSuccess ||
      (e = cp(M->row_cls, h_row_cls.data(), (size_t)nbrows * 4)) != cudaSuccess ||
      (e = cp(M->col_cls, h_col_cls.data(), (size_t)nbcols * 4)) != cudaSuccess)
    return fail(cuda_fail(e, "bsm_mat_create copy"));
  if ((rc = upload_contents(M, nblocks, blk_row, blk_col, values, true))) return fail(rc);
  *out = M;
  return BSM_OK;
}

int bsm_mat_assign(bsm_mat m, int64_t nblocks, const int32_t *blk_row, const int32_t *blk_col,
                   const double *values) {
  if (!m) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(m->ctx);
  if (rc || (rc = quiesce(m))) return rc;
  m->pend.active = false;  // a result computed into m is replaced, not read
  const void *before[2] = {m->front.col_idx, m->front.vals};
  rc = upload_contents(m, nblocks, blk_row, blk_col, values, false);
  if (before[0] != m->front.col_idx || before[1] != m->front.vals) {
    // captured multiplies may name the old buffers
    for (auto &g : m->ctx->graphs) cudaGraphExecDestroy(g.exec);
    m->ctx->graphs.clear();
  }
  const bool validation = rc == BSM_ERR_INVALID_ARG || rc == BSM_ERR_OUT_OF_RANGE ||
                          rc == BSM_ERR_DUPLICATE_BLOCK || rc == BSM_ERR_UNSUPPORTED;
  if (rc && !validation) {  // the old contents may be partly overwritten: leave m empty
    m->nblk = m->nnz = 0;
    int64_t z[2] = {0, 0};
    if (m->front.hdr) cudaMemcpy(m->front.hdr, z, sizeof(z), cudaMemcpyHostToDevice);
    if (m->front.row_ptr)
      cudaMemset(m->front.row_ptr, 0, ((size_t)m->nbr + 1) * sizeof(int32_t));
  }
  return rc;
}

int bsm_mat_destroy(bsm_mat m) {
  if (!m) return BSM_ERR_INVALID_ARG;
  bsm_ctx ctx = m->ctx;
  cudaSetDevice(ctx->device);
  // any pending multiply may read this matrix, an upload may write it: finish
  // all work first
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->up_stream);
  for (bsm_mat o : ctx->mats)
    if (o != m && o->pend.active && (o->pend.A == m || o->pend.B == m)) resolve(o);
  for (int i = 0; i < kSlots; i++)
    if (ctx->slot_owner[i] == m) ctx->slot_owner[i] = nullptr;
  m->front.release();
  m->back.release();
  cache_free(m->split_left);
  cache_free(m->split_right);
  dev_free(m->row_sizes);
  dev_free(m->col_sizes);
  dev_free(m->row_cls);
  dev_free(m->col_cls);
  dev_free(m->row_order);
  if (m->ev_use) cudaEventDestroy(m->ev_use);
  // captured multiplies may name this matrix's buffers
  for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  auto &v = ctx->mats;
  v.erase(std::remove(v.begin(), v.end(), m), v.end());
  delete m;
  return BSM_OK;
}

int bsm_multiply(bsm_ctx ctx, double alpha, bsm_mat A, bsm_mat B, double beta, bsm_mat C,
                 double eps, const bsm_opts *opts, bsm_stats *stats) {
  if (!ctx || !A || !B || !C) return BSM_ERR_INVALID_ARG;
  if (A->ctx != ctx || B->ctx != ctx || C->ctx != ctx) return BSM_ERR_INVALID_ARG;
  if (C == A || C == B) return BSM_ERR_ALIAS;
  bsm_opts o{};
  if (opts) o = *opts;
  if (o.precision != BSM_PREC_FP64 && o.precision != BSM_PREC_SPLIT_BF16X3 &&
      o.precision != BSM_PREC_SPLIT_TF32X2)
    return BSM_ERR_INVALID_ARG;
  if (o.launch != BSM_LAUNCH_PERSISTENT && o.launch != BSM_LAUNCH_PER_STACK)
    return BSM_ERR_INVALID_ARG;
  if (o.fp64_kernel < 0 || o.fp64_kernel > BSM_FP64_NUM_KERNELS) return BSM_ERR_INVALID_ARG;
  if (o.split_kernel < 0 || o.split_kernel > BSM_SPLIT_NUM_KERNELS) return BSM_ERR_INVALID_ARG;
  if (o.numeric_slices < 0 || o.numeric_slices > 64) return BSM_ERR_INVALID_ARG;
  if (o.host_values) {  // must be device-mapped page-locked host memory
    if (o.host_cap < 0) return BSM_ERR_INVALID_ARG;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, o.host_values) != cudaSuccess ||
        pa.type != cudaMemoryTypeHost || !pa.devicePointer) {
      cudaGetLastError();
      return BSM_ERR_INVALID_ARG;
    }
  }
  if (A->nbc != B->nbr || A->h_col_sizes != B->h_row_sizes) return BSM_ERR_DIM_MISMATCH;
  if (C->nbr != A->nbr || C->nbc != B->nbc || C->h_row_sizes != A->h_row_sizes ||
      C->h_col_sizes != B->h_col_sizes)
    return BSM_ERR_DIM_MISMATCH;
  // the split-precision kernels cover blocks of up to 32 x 32
  if (o.precision != BSM_PREC_FP64 &&
      std::max(A->max_row, std::max(A->max_col, B->max_col)) > 32)
    return BSM_ERR_UNSUPPORTED;
  int rc = ctx_set_device(ctx);
  if (rc) return rc;
  if ((rc = resolve(A)) || (rc = resolve(B))) return rc;
  if (beta != 0.0) {
    if ((rc = resolve(C))) return rc;
  } else {
    C->pend.active = false;  // superseded: the previous result is not read
  }
  const int slot = take_slot(ctx, C);
  if (slot < 0) return slot + 1000;
  // size the buffers exactly now when the last result computed into C (or the
  // workspace's product count) would not fit; otherwise the device checks itself
  const bool sync_sizes = C->back.cap_blk < 0 || C->back.cap_blk < C->hint_blk ||
                          C->back.cap_nnz < C->hint_nnz || ctx->ws.cap_prod <= 0 ||
                          ctx->ws.cap_prod < ctx->hint_prod || ctx->cap_cblk <= C->hint_blk;
  if (stats) stats->retries = 0;
  rc = run_multiply(ctx, alpha, A, B, beta, C, eps, o, sync_sizes, slot, stats);
  {  // whatever was enqueued, also on an error part way
    const cudaStream_t s = o.stream ? (cudaStream_t)o.stream : ctx->stream;
    int ru = mark_use(A, s);  // a failure synchronises s: nothing left to mark
    if (!ru) ru = mark_use(B, s);
    if (!ru) ru = mark_use(C, s);
    if (!rc) rc = ru;
  }
  if (rc) return rc;
  std::swap(C->front, C->back);
  C->pend.active = true;
  C->pend.A = A;
  C->pend.B = B;
  C->pend.alpha = alpha;
  C->pend.beta = beta;
  C->pend.eps = eps;
  C->pend.opts = o;
  C->pend.slot = slot;
  if (o.blocking || stats) {
    if ((rc = resolve(C, stats))) return rc;
  }
  if (stats) {
    const DevStatus &h = ctx->h_slots[slot];
    stats->candidates = h.candidates;
    stats->kept = h.kept;
    stats->dropped = h.candidates - h.kept;
    stats->c_blocks = h.nblk_c;
    stats->c_nnz = h.nnz_c;
    stats->flops = (double)h.flops;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev_t0, ctx->ev_t1));
    stats->ms_total = ms;
    stats->reserved = 0;
  }
  return BSM_OK;
}

int bsm_mat_nblocks(bsm_mat m, int64_t *nblocks, int64_t *nnz) {
  if (!m || !nblocks || !nnz) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(m->ctx);
  if (rc || (rc = resolve(m))) return rc;
  *nblocks = m->nblk;
  *nnz = m->nnz;
  return BSM_OK;
}

int bsm_mat_get_pattern(bsm_mat m, int64_t cap, int32_t *blk_row, int32_t *blk_col) {
  if (!m) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(m->ctx);
  if (rc || (rc = resolve(m))) return rc;
  if (cap < m->nblk || (m->nblk > 0 && (!blk_row || !blk_col))) return BSM_ERR_INVALID_ARG;
  if (m->nblk == 0) return BSM_OK;
  cudaStream_t s = m->ctx->stream;
  CK(cudaMemcpyAsync(blk_row, m->front.blk_row, (size_t)m->nblk * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(blk_col, m->front.col_idx, (size_t)m->nblk * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return BSM_OK;
}

int bsm_mat_get_values(bsm_mat m, int64_t cap, double *values) {
  if (!m) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(m->ctx);
  if (rc || (rc = resolve(m))) return rc;
  if (cap < m->nnz || (m->nnz > 0 && !values)) return BSM_ERR_INVALID_ARG;
  if (m->nnz == 0) return BSM_OK;
  cudaStream_t s = m->ctx->stream;
  CK(cudaMemcpyAsync(values, m->front.vals, (size_t)m->nnz * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return BSM_OK;
}

int bsm_mat_filter(bsm_mat M, double eps) {
  if (!M) return BSM_ERR_INVALID_ARG;
  bsm_ctx ctx = M->ctx;
  int rc = ctx_set_device(ctx);
  if (rc || (rc = resolve(M))) return rc;
  cudaStream_t s = ctx->stream;
  if ((rc = ws_rows(ctx, M->nbr)) || (rc = buf_grow(M, M->back, M->nblk, M->nnz, false)) ||
      (rc = ws_grow(ctx, M->nblk, 0)))
    return rc;
  if ((rc = enqueue_norms(ctx, M, s))) return rc;
  DevMat dM = dev_view(M);
  DevWs ws = ctx->ws;
  DevOut out = dev_out(M, M->back);
  CK(launch_filter_count(dM, eps, ws, ctx->nsm, s));
  CK(launch_symbolic_scan(M->nbr, ws, out, ctx->d_status, s));
  CK(launch_filter_fill(dM, eps, ws, out, ctx->d_status, ctx->nsm, s));
  ctx->launches += 5;
  DevStatus h{};
  CK(cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h.overflow) return BSM_ERR_NOMEM;  // cannot happen: the back buffer holds all blocks
  std::swap(M->front, M->back);
  M->nblk = h.nblk_c;
  M->nnz = h.nnz_c;
  return BSM_OK;
}

int bsm_mat_add(bsm_ctx ctx, double alpha, bsm_mat A, double beta, bsm_mat C) {
  if (!ctx || !A || !C || A->ctx != ctx || C->ctx != ctx) return BSM_ERR_INVALID_ARG;
  if (A == C) return BSM_ERR_ALIAS;
  if (A->h_row_sizes != C->h_row_sizes || A->h_col_sizes != C->h_col_sizes)
    return BSM_ERR_DIM_MISMATCH;
  int rc = ctx_set_device(ctx);
  if (rc || (rc = resolve(A))) return rc;
  const bool use_cin = beta != 0.0;
  if (use_cin) {
    if ((rc = resolve(C))) return rc;
  } else {
    C->pend.active = false;
  }
  const int64_t nb = A->nblk + (use_cin ? C->nblk : 0);
  const int64_t nz = A->nnz + (use_cin ? C->nnz : 0);
  cudaStream_t s = ctx->stream;
  if ((rc = ws_rows(ctx, A->nbr)) || (rc = buf_grow(C, C->back, nb, nz, false)) ||
      (rc = ws_grow(ctx, nb, 0)))
    return rc;
  DevMat dA = dev_view(A), dC = dev_view(C);
  DevWs ws = ctx->ws;
  DevOut out = dev_out(C, C->back);
  CK(launch_add(0, dA, dC, use_cin, alpha, beta, ws, out, ctx->d_status, ctx->nsm, s));
  CK(launch_symbolic_scan(A->nbr, ws, out, ctx->d_status, s));
  CK(launch_add(1, dA, dC, use_cin, alpha, beta, ws, out, ctx->d_status, ctx->nsm, s));
  CK(launch_add(2, dA, dC, use_cin, alpha, beta, ws, out, ctx->d_status, ctx->nsm, s));
  ctx->launches += 4;
  DevStatus h{};
  CK(cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h.overflow) return BSM_ERR_NOMEM;
  std::swap(C->front, C->back);
  C->nblk = h.nblk_c;
  C->nnz = h.nnz_c;
  C->hint_blk = std::max(C->hint_blk, h.nblk_c);
  C->hint_nnz = std::max(C->hint_nnz, h.nnz_c);
  // the union of the two patterns (or A's alone)
  C->max_row_blocks = !use_cin ? A->max_row_blocks
                      : (A->max_row_blocks < 0 || C->max_row_blocks < 0)
                          ? -1
                          : A->max_row_blocks + C->max_row_blocks;
  return BSM_OK;
}

int bsm_ctx_profile(bsm_ctx ctx, int enable) {
  if (!ctx) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(ctx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int s = 0; s < kSlots; s++) {
    ctx->prof_pending[s] = false;
    if (enable && !ctx->prof_ev[s][0])
      for (int e = 0; e < 4; e++) CK(cudaEventCreate(&ctx->prof_ev[s][e]));
  }
  ctx->prof = enable != 0;
  ctx->prof_tot = bsm_profile{};
  ctx->launches_at_enable = ctx->launches;
  return BSM_OK;
}

int bsm_ctx_profile_read(bsm_ctx ctx, bsm_profile *out) {
  if (!ctx || !out) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(ctx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int s = 0; s < kSlots; s++)
    if ((rc = prof_collect(ctx, s))) return rc;
  *out = ctx->prof_tot;
  out->launches = ctx->launches - ctx->launches_at_enable;
  out->last_fp64_kernel = ctx->last_fp64;
  out->last_split_kernel = ctx->last_split;
  return BSM_OK;
}

int bsm_selftest_wait(bsm_ctx ctx, int never_complete) {
  if (!ctx) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(ctx);
  if (rc) return rc;
  int32_t *d_flag = nullptr, h_flag = -1;
  CK(cudaMalloc((void **)&d_flag, sizeof(int32_t)));
  cudaError_t e = launch_wait_selftest(never_complete ? 1 : 0, d_flag, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_flag, d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_flag);
  if (e != cudaSuccess) return cuda_fail(e, "wait selftest");
  return h_flag == 0 ? BSM_OK : BSM_ERR_TIMEOUT;
}

int bsm_sync(bsm_ctx ctx) {
  if (!ctx) return BSM_ERR_INVALID_ARG;
  int rc = ctx_set_device(ctx);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  for (bsm_mat m : std::vector<bsm_mat>(ctx->mats))
    if (m->pend.active && (rc = resolve(m))) return rc;
  return BSM_OK;
}

}  // extern "C"

namespace bsm {

int mat_create_diag(bsm_ctx ctx, int nparts, const DiagPart *parts, bsm_mat *out) {
  if (!ctx || !out || nparts < 0 || (nparts > 0 && !parts)) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  // the parts' first block row, block and value in the whole matrix
  std::vector<int64_t> row0(nparts + 1, 0), blk0(nparts + 1, 0), val0(nparts + 1, 0);
  std::vector<int32_t> sizes;
  for (int p = 0; p < nparts; p++) {
    const DiagPart &P = parts[p];
    if (P.nbr < 0 || P.nblk < 0 || (P.nbr > 0 && !P.sizes) ||
        (P.nblk > 0 && (!P.brow || !P.bcol || !P.vals)))
      return BSM_ERR_INVALID_ARG;
    for (int32_t i = 0; i < P.nbr; i++)
      if (P.sizes[i] <= 0) return BSM_ERR_INVALID_ARG;
    int64_t nv = 0;
    for (int64_t b = 0; b < P.nblk; b++) {
      const int32_t i = P.brow[b], j = P.bcol[b];
      if (i < 0 || i >= P.nbr || j < 0 || j >= P.nbr) return BSM_ERR_OUT_OF_RANGE;
      if (b > 0 && (P.brow[b - 1] > i || (P.brow[b - 1] == i && P.bcol[b - 1] >= j)))
        return BSM_ERR_INVALID_ARG;
      nv += (int64_t)P.sizes[i] * P.sizes[j];
    }
    row0[p + 1] = row0[p] + P.nbr;
    blk0[p + 1] = blk0[p] + P.nblk;
    val0[p + 1] = val0[p] + nv;
    if (row0[p + 1] >= (int64_t)INT32_MAX || blk0[p + 1] >= (int64_t)INT32_MAX)
      return BSM_ERR_UNSUPPORTED;
    sizes.insert(sizes.end(), P.sizes, P.sizes + P.nbr);
  }
  const int32_t nbr = (int32_t)row0[nparts];
  const int64_t nblk = blk0[nparts], nnz = val0[nparts];
  bsm_mat M = nullptr;
  int rc = bsm_mat_create(ctx, nbr, sizes.data(), nbr, sizes.data(), 0, nullptr, nullptr, nullptr, &M);
  if (rc) return rc;
  auto fail = [&](int code) {
    bsm_mat_destroy(M);
    return code;
  };
  const StageLayout L = stage_layout(nbr, nblk);
  if ((rc = stage_reserve(ctx, L.need))) return fail(rc);
  int32_t *h_row_ptr = reinterpret_cast<int32_t *>(ctx->h_stage);
  int32_t *h_col = reinterpret_cast<int32_t *>(ctx->h_stage + L.b_ptr);
  int32_t *h_row = reinterpret_cast<int32_t *>(ctx->h_stage + L.b_ptr + L.b_col);
  int64_t *h_off = reinterpret_cast<int64_t *>(ctx->h_stage + L.b_ptr + 2 * L.b_col);
  memset(h_row_ptr, 0, ((size_t)nbr + 1) * 4);
  int64_t g = 0, off = 0;
  for (int p = 0; p < nparts; p++) {
    const DiagPart &P = parts[p];
    const int32_t r0 = (int32_t)row0[p];
    for (int64_t b = 0; b < P.nblk; b++, g++) {
      h_row[g] = r0 + P.brow[b];
      h_col[g] = r0 + P.bcol[b];
      h_off[g] = off;
      off += (int64_t)P.sizes[P.brow[b]] * P.sizes[P.bcol[b]];
      h_row_ptr[h_row[g] + 1]++;
    }
  }
  M->max_row_blocks = 0;
  for (int32_t i = 0; i < nbr; i++)
    M->max_row_blocks = std::max<int64_t>(M->max_row_blocks, h_row_ptr[i + 1]);
  for (int32_t i = 0; i < nbr; i++) h_row_ptr[i + 1] += h_row_ptr[i];
  if ((rc = buf_grow(M, M->front, nblk, nnz, true))) return fail(rc);
  cudaStream_t st = ctx->stream;
  auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  int64_t hdr[2] = {nblk, nnz};
  cudaError_t e;
  for (int p = 0; p < nparts; p++)
    if ((e = cp(M->front.vals + val0[p], parts[p].vals, (size_t)(val0[p + 1] - val0[p]) * 8)) !=
        cudaSuccess)
      return fail(cuda_fail(e, "diagonal upload values"));
  if ((e = cp(M->front.row_ptr, h_row_ptr, ((size_t)nbr + 1) * 4)) != cudaSuccess ||
      (e = cp(M->front.col_idx, h_col, (size_t)nblk * 4)) != cudaSuccess ||
      (e = cp(M->front.blk_row, h_row, (size_t)nblk * 4)) != cudaSuccess ||
      (e = cp(M->front.blk_off, h_off, (size_t)nblk * 8)) != cudaSuccess ||
      (e = cp(M->front.hdr, hdr, sizeof(hdr))) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(cuda_fail(e, "diagonal upload"));
  M->nblk = nblk;
  M->nnz = nnz;
  *out = M;
  return BSM_OK;
}

int set_slice_gate(bsm_ctx ctx, SliceGate gate, void *arg) {
  if (!ctx) return BSM_ERR_INVALID_ARG;
  if (gate && !ctx->ev_gate) {
    cudaSetDevice(ctx->device);
    const cudaError_t e = cudaEventCreateWithFlags(&ctx->ev_gate, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      ctx->ev_gate = nullptr;
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  ctx->gate = gate;
  ctx->gate_arg = arg;
  return BSM_OK;
}

}  // namespace bsm
