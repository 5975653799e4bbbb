// bsm_server.cu -- a request loop over the filtered multiply: independent
// multiplies C = A.A of differently sized systems arrive one by one and are run
// with continuous batching.
//
// The server owns `slots` lanes, each a libbsm context (own stream and
// workspace) driven by a worker thread of its own. A free lane takes the next
// batch from the queue as soon as its device-memory footprint (an upper bound
// computed at submission) fits the budget next to the requests already held.
// Admission is earliest deadline first: a request's deadline is its submission
// time plus kStretch times its estimated run time (from the exact count of its
// unfiltered multiply-adds). Small requests therefore pass large ones that
// arrived a little earlier, while a large one is never passed by requests that
// arrive after its deadline. Large requests (kLargeMs) run one at a time (two
// for a backlog of large ones only), their numeric phase in slices; small
// batches launch on a high-priority stream, and a large one's next slice waits
// while they are on the device.
// A batch is the earliest-deadline request plus, when it is small (kMergeMs),
// the other small queued requests of the same eps in deadline order, within the
// batch limits below. The batch runs as one multiply of the
// block-diagonal matrix diag(A_1, ..., A_n) (one norm, symbolic and numeric
// launch sequence over all the batch's blocks). diag(A_1..A_n)^2 =
// diag(A_1^2..A_n^2): the kernels compute every C block from its own product list
// alone, in an order fixed by that list, so each request's part of the result is
// bit for bit the result of the request run alone. The lanes run their batches
// concurrently on the device (at most kMaxSmall small ones), and a request that
// arrives while others run starts the moment a lane and memory free up. Inputs
// are copied at submission into page-locked host memory (large copies on
// several threads) and uploaded from there by DMA, one copy per
// request into the batch's matrix. Results go to page-locked host memory (the
// multiply stores the values there directly when they fit) and wait there
// until taken or released.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/bsm.h"
#include "bsm_internal.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

enum { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
  int64_t id = 0;
  std::vector<int32_t> sizes, brow, bcol;  // blocks sorted by (row, col)
  double *vals = nullptr;  // page-locked copy of the values, in block order
  const double *in_vals = nullptr;  // what the lane uploads: vals, or the caller's (borrowed)
  int64_t nvals = 0;
  double eps = 0;
  int64_t footprint = 0;     // bytes held on the device while admitted
  int64_t c_vals_bound = 0;  // upper bound of the result's value count
  double est_ms = 0;         // estimated run time alone
  double deadline = 0;       // admission order: t_submit + kStretch * est_ms
  int state = kQueued;       // under the server's lock
  int err = BSM_OK;
  int slot = -1;
  double t_submit = 0, t_queued = 0, t_start = 0, t_done = 0;
  // written by the lane's worker while running; read by others once done
  int64_t nblk = 0, nnz = 0;
  // the result: page-locked host blocks of the server's pool
  int32_t *res_row = nullptr, *res_col = nullptr;
  double *res_val = nullptr;
};

// Admission and batching. A request's deadline is its submission time plus
// kStretch times its estimated run time; requests estimated at most kMergeMs
// share a multiply with other such requests, up to kMaxBatch requests and a total
// estimate of kBatchMs, and never more than kStretch times the estimate of the
// batch's first request (the batch finishes as one, so that request still makes
// its deadline). The estimate is a fixed cost per multiply plus the exact count of
// unfiltered multiply-adds at a nominal rate per precision: it orders the queue,
// it is not a prediction the server relies on.
constexpr double kStretch = 4.0;
constexpr double kMergeMs = 4.0;
constexpr double kBatchMs = 8.0;
constexpr int kMaxBatch = 16;
// A large request (estimated at least kLargeMs) fills every SM on its own: at
// most one large request runs, so that the small ones get the SMs between its
// slices, unless a backlog of large requests waits and no small one does (the
// tail of a burst): then two may run, the second's upload and read-back
// overlapping the first's products (a 100-request water replay: 84.6 requests/s
// with 4 lanes free to run large ones together, 94.4 with 2 lanes).
constexpr double kLargeMs = 8.0;
constexpr int kMaxLarge = 1, kMaxLargeAlone = 2;
// Small batches running at once: more share the SMs (each runs slower), fewer
// queue (and merge) the small requests behind one another. (100 and 200 water
// requests, 4 lanes: at most 2 gave the highest burst rate, 92-100 requests/s
// against 80-95 with 4, at the same Poisson p50.)
constexpr int kMaxSmall = 2;
// A large request's numeric phase runs in slices of about kSliceMs of
// estimated work (consecutive ranges of its C blocks, each a launch of its
// own), and small batches run on a stream of the highest priority: a small
// request that arrives while a large one runs gets SMs at the next slice
// boundary instead of after the whole multiply.
constexpr double kSliceMs = 2.0;
// Between two slices the large request's lane waits for the slice to finish,
// then, while small batches run, holds the next slice back (at most kGateMs per
// slice, so that a stream of small requests cannot stall a large one): a small
// multiply's dependent launches then find the SMs free instead of taking turns
// with the large one's persistent slices. (100 water requests, Poisson
// arrivals at 0.8 x the sequential rate: p50 14 ms without the hold, 10-11 ms
// with it; a longer hold lowers the burst rate, 2 to 8 ms per slice gave
// 97 to 92 requests/s.)
constexpr double kGateMs = 4.0;
constexpr double kFixedMs = 0.15;
double est_run_ms(int64_t macs, int precision) {
  const double flop_per_ms = precision == BSM_PREC_FP64 ? 1.0e9 : 2.5e9;
  return kFixedMs + 2.0 * (double)macs / flop_per_ms;
}

// Page-locked host memory for results: the lanes read results back into it at
// the DMA rate (pageable memory goes through the driver's staging copies), and
// a result can be handed to the caller without a copy. Freed blocks are kept
// for reuse (cudaHostAlloc is slow), up to kPinnedCap bytes.
constexpr size_t kPinnedCap = 16ull << 30;
constexpr int64_t kHostValuesCap = 128ll << 20;  // values (1 GiB) a lane's multiply stores directly

struct PinnedPool {
  std::mutex mu;
  std::multimap<size_t, void *> free_blocks;
  std::map<void *, size_t> block_size;
  size_t cached = 0;

  static size_t size_class(size_t b) {
    if (b <= 4096) return 4096;
    const int p = 63 - __builtin_clzll((unsigned long long)(b - 1));
    const size_t step = (size_t)1 << (p - 3);
    return (b + step - 1) & ~(step - 1);
  }
  void *get(size_t bytes) {
    const size_t cls = size_class(bytes);
    std::lock_guard<std::mutex> lk(mu);
    auto it = free_blocks.find(cls);
    if (it != free_blocks.end()) {
      void *p = it->second;
      free_blocks.erase(it);
      cached -= cls;
      return p;
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, cls, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    block_size[p] = cls;
    return p;
  }
  void put(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu);
    auto it = block_size.find(p);
    if (it == block_size.end()) return;
    if (cached + it->second <= kPinnedCap) {
      free_blocks.emplace(it->second, p);
      cached += it->second;
    } else {
      block_size.erase(it);
      cudaFreeHost(p);
    }
  }
  void clear() {
    std::lock_guard<std::mutex> lk(mu);
    for (auto &kv : block_size) cudaFreeHost(kv.first);
    block_size.clear();
    free_blocks.clear();
    cached = 0;
  }
};

// A lane: a context and the worker thread that runs one batch at a time on
// it; small batches launch on the lane's high-priority stream.
struct Slot {
  bsm_ctx ctx = nullptr;
  cudaStream_t hi = nullptr;
  std::thread worker;
};

// memcpy in pieces of at least kCopyPiece bytes on up to kCopyThreads threads
// (the caller's among them): one thread copies into page-locked memory at a
// fraction of the host's memory bandwidth, and the copy is part of every
// request's latency.
constexpr size_t kCopyPiece = 4u << 20;
constexpr int kCopyThreads = 6;
void copy_parallel(void *dst, const void *src, size_t bytes) {
  const int nt = (int)std::min<size_t>(kCopyThreads, bytes / kCopyPiece);
  if (nt <= 1) {
    memcpy(dst, src, bytes);
    return;
  }
  const size_t per = (bytes / nt + 63) & ~(size_t)63;
  auto piece = [&](int t) {
    const size_t a = std::min(bytes, per * (size_t)t), b = std::min(bytes, a + per);
    if (b > a) memcpy(static_cast<char *>(dst) + a, static_cast<const char *>(src) + a, b - a);
  };
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  try {
    for (int t = 1; t < nt; t++) th.emplace_back(piece, t);
  } catch (const std::system_error &) {  // no thread to be had: the rest here
    for (int t = 1 + (int)th.size(); t < nt; t++) piece(t);
  }
  piece(0);
  for (std::thread &x : th) x.join();
}

// Upper bound of the device bytes a request C = A.A can hold; also the bound
// of its result's value count and its unfiltered multiply-adds.
int64_t footprint_bound(const Request &r, int precision, int64_t *c_vals_bound, int64_t *macs) {
  const int64_t nbr = (int64_t)r.sizes.size();
  std::vector<int64_t> row_nblk(nbr, 0), row_cols(nbr, 0);
  for (size_t b = 0; b < r.brow.size(); b++) {
    row_nblk[r.brow[b]]++;
    row_cols[r.brow[b]] += r.sizes[r.bcol[b]];
  }
  int64_t dim = 0;
  for (int32_t s : r.sizes) dim += s;
  int64_t cand = 0, cand_vals = 0, mac = 0;
  for (size_t b = 0; b < r.brow.size(); b++) {
    cand += row_nblk[r.bcol[b]];
    cand_vals += (int64_t)r.sizes[r.brow[b]] * row_cols[r.bcol[b]];
    mac += (int64_t)r.sizes[r.brow[b]] * r.sizes[r.bcol[b]] * row_cols[r.bcol[b]];
  }
  if (macs) *macs = mac;
  const int64_t a_bytes = 8 * r.nvals + 32 * (int64_t)r.brow.size();
  const int64_t c_blocks = std::min<int64_t>(nbr * nbr, cand);
  const int64_t c_vals = std::min<int64_t>(dim * dim, cand_vals);
  if (c_vals_bound) *c_vals_bound = c_vals;
  // the split precisions keep A's slices in both operand layouts
  const int64_t slice_bytes =
      precision == BSM_PREC_FP64 ? 0 : 2 * bsm::split_bytes_per_value(precision) * r.nvals;
  // A, C twice (front/back), per-block metadata, product records
  return 4 * a_bytes + slice_bytes + 2 * (8 * c_vals + 32 * c_blocks) + 8 * cand + 64 * nbr +
         (1 << 20);
}

}  // namespace

struct bsm_server_s {
  int device = 0;
  int precision = BSM_PREC_FP64;
  int64_t budget = 0;
  std::vector<Slot> slots;
  PinnedPool pinned;
  // everything below, and each request's state, under `mu`; `cv` wakes the
  // workers when a request arrives, memory is released or the server stops
  std::mutex mu;
  std::condition_variable cv;
  int64_t in_use = 0, peak = 0;
  std::deque<Request *> queue;
  std::map<int64_t, Request *> reqs;
  int64_t next_id = 1;
  int64_t completed = 0, reported = 0;
  int64_t running = 0;
  int64_t running_large = 0;  // large requests running (at most kMaxLarge)
  int64_t running_small = 0;  // small batches running (at most kMaxSmall)
  int64_t small_on_gpu = 0;   // small batches between upload and multiply's end
  int64_t batches = 0;  // multiplies run (a batch of one or more requests each)
  bool stop = false;
};

static void drop_result(bsm_server s, Request *r) {
  s->pinned.put(r->res_row);
  s->pinned.put(r->res_col);
  s->pinned.put(r->res_val);
  r->res_row = r->res_col = nullptr;
  r->res_val = nullptr;
}

// Hand the part of the batch's result that belongs to request p (block rows
// [r0, r1) of the whole) to the request, in page-locked blocks of its own.
// rows/cols/vals: the whole result (pattern sorted by (row, col)).
static int split_result(bsm_server s, Request *r, int32_t r0, int32_t r1, const int32_t *rows,
                        const int32_t *cols, const double *vals, int64_t nblk,
                        const std::vector<int64_t> &voff) {
  const int64_t b0 = std::lower_bound(rows, rows + nblk, r0) - rows;
  const int64_t b1 = std::lower_bound(rows, rows + nblk, r1) - rows;
  r->nblk = b1 - b0;
  r->nnz = voff[b1] - voff[b0];
  r->res_row = static_cast<int32_t *>(s->pinned.get(4 * (size_t)r->nblk));
  r->res_col = static_cast<int32_t *>(s->pinned.get(4 * (size_t)r->nblk));
  r->res_val = static_cast<double *>(s->pinned.get(8 * (size_t)r->nnz));
  if (!r->res_row || !r->res_col || !r->res_val) return BSM_ERR_NOMEM;
  for (int64_t b = b0; b < b1; b++) {  // block-diagonal: the columns lie in [r0, r1) too
    r->res_row[b - b0] = rows[b] - r0;
    r->res_col[b - b0] = cols[b] - r0;
  }
  std::copy(vals + voff[b0], vals + voff[b1], r->res_val);
  return BSM_OK;
}

// The large requests' lanes call this between two numeric slices, once the
// slice before has finished: it returns when no small batch is on the device,
// after kGateMs at most, or when the server stops.
static void slice_gate(void *arg) {
  bsm_server s = static_cast<bsm_server>(arg);
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait_for(lk, std::chrono::microseconds((int64_t)(kGateMs * 1000.0)),
                 [&] { return s->stop || s->small_on_gpu == 0; });
}

static void small_on_gpu_add(bsm_server s, int d) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->small_on_gpu += d;
  }
  if (d < 0) s->cv.notify_all();
}

// One batch on a lane, in the lane's worker thread: the block-diagonal matrix of
// the batch's requests uploaded, one multiply, each request's part of the
// result to host memory, device memory released.
static void run_batch(bsm_server s, Slot &sl, const std::vector<Request *> &batch) {
  const int n = (int)batch.size();
  const bool small = batch[0]->est_ms < kLargeMs;
  if (small) small_on_gpu_add(s, 1);  // until its multiply has finished
  std::vector<bsm::DiagPart> parts(n);
  std::vector<int32_t> sizes, row0(n + 1, 0);
  int64_t vals_bound = 0;
  for (int p = 0; p < n; p++) {
    const Request *r = batch[p];
    parts[p] = {(int32_t)r->sizes.size(), r->sizes.data(), (int64_t)r->brow.size(), r->brow.data(),
                r->bcol.data(), r->in_vals};
    sizes.insert(sizes.end(), r->sizes.begin(), r->sizes.end());
    row0[p + 1] = row0[p] + (int32_t)r->sizes.size();
    vals_bound += r->c_vals_bound;
  }
  const int32_t nbr = row0[n];
  bsm_mat A = nullptr, C = nullptr;
  int rc = bsm::mat_create_diag(sl.ctx, n, parts.data(), &A);
  if (rc == BSM_OK)
    rc = bsm_mat_create(sl.ctx, nbr, sizes.data(), nbr, sizes.data(), 0, nullptr, nullptr,
                        nullptr, &C);
  // the values go straight to page-locked host memory while the multiply runs,
  // into a block sized by the bound on the result (up to kHostValuesCap values);
  // a larger result is read back after the multiply
  const int64_t hv_cap = std::min<int64_t>(std::max<int64_t>(vals_bound, 1), kHostValuesCap);
  double *hv = (rc == BSM_OK) ? static_cast<double *>(s->pinned.get(8 * (size_t)hv_cap)) : nullptr;
  if (rc == BSM_OK) {
    bsm_opts o{};
    o.precision = s->precision;
    o.blocking = 1;
    o.host_values = hv;
    o.host_cap = hv ? hv_cap : 0;
    if (small)
      o.stream = sl.hi;
    else  // a large request runs alone, sliced
      o.numeric_slices = (int)std::min(64.0, std::ceil(batch[0]->est_ms / kSliceMs));
    rc = bsm_multiply(sl.ctx, 1.0, A, A, 0.0, C, batch[0]->eps, &o, nullptr);
  }
  if (small) small_on_gpu_add(s, -1);  // blocking: its kernels have finished
  int64_t nblk = 0, nnz = 0;
  if (rc == BSM_OK) rc = bsm_mat_nblocks(C, &nblk, &nnz);
  int32_t *rows = nullptr, *cols = nullptr;
  double *vals = nullptr;
  const bool direct = rc == BSM_OK && hv && nnz <= hv_cap;  // values already in host memory
  if (rc == BSM_OK) {
    rows = static_cast<int32_t *>(s->pinned.get(4 * (size_t)nblk));
    cols = static_cast<int32_t *>(s->pinned.get(4 * (size_t)nblk));
    if (direct) {
      vals = hv;
      hv = nullptr;
    } else {
      vals = static_cast<double *>(s->pinned.get(8 * (size_t)nnz));
    }
    if (!rows || !cols || !vals) rc = BSM_ERR_NOMEM;
    if (rc == BSM_OK) rc = bsm_mat_get_pattern(C, nblk, rows, cols);
    if (rc == BSM_OK && !direct) rc = bsm_mat_get_values(C, nnz, vals);
  }
  if (rc == BSM_OK && n == 1) {  // the whole result is the request's: no copies
    Request *r = batch[0];
    r->nblk = nblk;
    r->nnz = nnz;
    r->res_row = rows;
    r->res_col = cols;
    r->res_val = vals;
    rows = cols = nullptr;
    vals = nullptr;
  } else if (rc == BSM_OK) {
    std::vector<int64_t> voff((size_t)nblk + 1, 0);  // first value of each result block
    for (int64_t b = 0; b < nblk; b++) voff[b + 1] = voff[b] + (int64_t)sizes[rows[b]] * sizes[cols[b]];
    for (int p = 0; p < n && rc == BSM_OK; p++)
      rc = split_result(s, batch[p], row0[p], row0[p + 1], rows, cols, vals, nblk, voff);
  }
  s->pinned.put(rows);
  s->pinned.put(cols);
  s->pinned.put(vals);
  s->pinned.put(hv);
  if (A) bsm_mat_destroy(A);
  if (C) bsm_mat_destroy(C);
  const double t = now_ms();
  for (Request *r : batch) {
    if (rc != BSM_OK) drop_result(s, r);
    s->pinned.put(r->vals);  // the host copy of the input is no longer needed
    r->vals = nullptr;
    r->in_vals = nullptr;  // a borrowed input is no longer read
    r->err = rc;
    r->t_done = t;
  }
}

// The next batch, under the server's lock: the earliest-deadline request that
// may start -- a large one only while fewer than kMaxLarge large ones run
// (kMaxLargeAlone when only large requests, two or more, wait), a small one
// while fewer than kMaxSmall small batches run --
// once it fits the budget (it waits for memory rather than be passed by later
// requests), and, when it is small, the other small queued requests of the same
// eps in deadline order, as far as the work and memory limits allow. The batch
// leaves the queue. False (batch empty) when nothing can start.
static bool pick_batch(bsm_server s, std::vector<Request *> &batch) {
  batch.clear();
  if (s->queue.empty()) return false;
  std::vector<Request *> order(s->queue.begin(), s->queue.end());
  std::stable_sort(order.begin(), order.end(),
                   [](const Request *a, const Request *b) { return a->deadline < b->deadline; });
  int small_waiting = 0, large_waiting = 0;
  for (const Request *r : order) (r->est_ms < kLargeMs ? small_waiting : large_waiting)++;
  const int max_large = (small_waiting == 0 && large_waiting >= 2) ? kMaxLargeAlone : kMaxLarge;
  Request *head = nullptr;
  for (Request *r : order)
    if (r->est_ms < kLargeMs ? s->running_small < kMaxSmall : s->running_large < max_large) {
      head = r;
      break;
    }
  if (!head || s->in_use + head->footprint > s->budget) return false;
  batch.push_back(head);
  int64_t held = head->footprint;
  double work = head->est_ms;
  if (head->est_ms <= kMergeMs) {
    const double limit = std::min(kBatchMs, kStretch * head->est_ms);
    for (size_t q = 0; q < order.size() && (int)batch.size() < kMaxBatch; q++) {
      Request *r = order[q];
      if (r == head || r->eps != head->eps || r->est_ms > kMergeMs || work + r->est_ms > limit ||
          s->in_use + held + r->footprint > s->budget)
        continue;
      batch.push_back(r);
      held += r->footprint;
      work += r->est_ms;
    }
  }
  for (Request *r : batch) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
  return true;
}

// A lane's worker: takes the next batch once it fits the budget, runs it, and
// returns its memory to the budget.
static void worker_loop(bsm_server s, int lane) {
  cudaSetDevice(s->device);
  std::vector<Request *> batch;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return s->stop || pick_batch(s, batch); });
    if (s->stop) {  // queued requests are dropped by bsm_server_destroy
      for (Request *r : batch) s->queue.push_front(r);
      return;
    }
    int64_t held = 0;
    const double t = now_ms();
    for (Request *r : batch) {
      held += r->footprint;
      r->state = kRunning;
      r->slot = lane;
      r->t_start = t;
    }
    const bool large = batch[0]->est_ms >= kLargeMs;  // a large request runs alone
    s->in_use += held;
    s->peak = std::max(s->peak, s->in_use);
    s->running += (int64_t)batch.size();
    s->running_large += large ? 1 : 0;
    s->running_small += large ? 0 : 1;
    s->batches++;
    lk.unlock();
    run_batch(s, s->slots[lane], batch);
    lk.lock();
    s->in_use -= held;  // the lane released the batch's device memory
    for (Request *r : batch) {
      r->footprint = 0;
      r->state = r->err == BSM_OK ? kDone : kFailed;
    }
    s->running -= (int64_t)batch.size();
    s->running_large -= large ? 1 : 0;
    s->running_small -= large ? 0 : 1;
    s->completed += (int64_t)batch.size();
    batch.clear();
    s->cv.notify_all();  // a head that waited for memory may fit now
  }
}

static void forget(bsm_server s, Request *r) {
  drop_result(s, r);
  s->pinned.put(r->vals);
  delete r;
}

extern "C" {

int bsm_server_create(int device, const bsm_server_opts *opts, bsm_server *out) {
  if (!out) return BSM_ERR_INVALID_ARG;
  *out = nullptr;
  bsm_server_opts o{};
  if (opts) o = *opts;
  if (o.slots <= 0) o.slots = 4;
  if (o.slots > 64) return BSM_ERR_INVALID_ARG;
  if (o.hbm_budget <= 0) o.hbm_budget = 8ll << 30;
  if (o.precision != BSM_PREC_FP64 && o.precision != BSM_PREC_SPLIT_BF16X3 &&
      o.precision != BSM_PREC_SPLIT_TF32X2)
    return BSM_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return BSM_ERR_INVALID_ARG;
  bsm_server s = new (std::nothrow) bsm_server_s();
  if (!s) return BSM_ERR_NOMEM;
  s->device = device;
  s->precision = o.precision;
  s->budget = o.hbm_budget;
  s->slots = std::vector<Slot>(o.slots);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (Slot &sl : s->slots) {
    int rc = bsm_ctx_create(device, &sl.ctx);
    if (rc == BSM_OK) rc = bsm::set_slice_gate(sl.ctx, slice_gate, s);
    if (rc == BSM_OK &&
        cudaStreamCreateWithPriority(&sl.hi, cudaStreamNonBlocking, greatest) != cudaSuccess) {
      cudaGetLastError();
      sl.hi = nullptr;
      rc = BSM_ERR_CUDA;
    }
    if (rc != BSM_OK) {
      bsm_server_destroy(s);
      return rc;
    }
  }
  for (int i = 0; i < o.slots; i++) s->slots[i].worker = std::thread(worker_loop, s, i);
  *out = s;
  return BSM_OK;
}

int bsm_server_destroy(bsm_server s) {
  if (!s) return BSM_ERR_INVALID_ARG;
  cudaSetDevice(s->device);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (Slot &sl : s->slots)  // a running request is finished first
    if (sl.worker.joinable()) sl.worker.join();
  for (auto &kv : s->reqs) forget(s, kv.second);
  s->reqs.clear();
  s->queue.clear();
  for (Slot &sl : s->slots) {
    if (sl.ctx) bsm_ctx_destroy(sl.ctx);
    if (sl.hi) cudaStreamDestroy(sl.hi);
  }
  s->pinned.clear();
  delete s;
  return BSM_OK;
}

// borrow: the caller's values are uploaded as they are (sorted block lists
// only), without the copy into page-locked memory.
static int submit_request(bsm_server s, int32_t nbrows, const int32_t *sizes, int64_t nblocks,
                          const int32_t *blk_row, const int32_t *blk_col, const double *values,
                          double eps, bool borrow, int64_t *id) {
  // the request arrives now: its latency and deadline count from here, not from
  // the end of the copies below (which may wait for page-locked memory)
  const double t_arrive = now_ms();
  if (!s || !id || nbrows < 0 || nblocks < 0 || (nbrows > 0 && !sizes) ||
      (nblocks > 0 && (!blk_row || !blk_col || !values)))
    return BSM_ERR_INVALID_ARG;
  for (int32_t b = 0; b < nbrows; b++)
    if (sizes[b] <= 0) return BSM_ERR_INVALID_ARG;
  int64_t nv = 0;
  for (int64_t b = 0; b < nblocks; b++) {
    if (blk_row[b] < 0 || blk_row[b] >= nbrows || blk_col[b] < 0 || blk_col[b] >= nbrows)
      return BSM_ERR_OUT_OF_RANGE;
    nv += (int64_t)sizes[blk_row[b]] * sizes[blk_col[b]];
  }
  // the copies are made before the lock: a large request does not hold up the
  // lanes. The blocks are kept sorted by (row, col), the order the batch's
  // matrix is assembled in; the values go to page-locked memory, from where the
  // lane uploads them by DMA (a borrowed submission's from the caller's array).
  bool sorted = true;
  for (int64_t b = 1; b < nblocks && sorted; b++)
    sorted = blk_row[b - 1] < blk_row[b] || (blk_row[b - 1] == blk_row[b] && blk_col[b - 1] < blk_col[b]);
  if (borrow && !sorted) return BSM_ERR_INVALID_ARG;
  Request *r = new (std::nothrow) Request();
  if (!r) return BSM_ERR_NOMEM;
  r->nvals = nv;
  if (borrow) {
    r->in_vals = values;
  } else {
    r->vals = static_cast<double *>(s->pinned.get(8 * (size_t)std::max<int64_t>(nv, 1)));
    if (!r->vals) {
      delete r;
      return BSM_ERR_NOMEM;
    }
    r->in_vals = r->vals;
  }
  try {
    r->sizes.assign(sizes, sizes + nbrows);
    if (sorted) {
      r->brow.assign(blk_row, blk_row + nblocks);
      r->bcol.assign(blk_col, blk_col + nblocks);
      if (nv && !borrow) copy_parallel(r->vals, values, (size_t)nv * sizeof(double));
    } else {
      std::vector<int64_t> order((size_t)nblocks), off((size_t)nblocks + 1, 0);
      for (int64_t b = 0; b < nblocks; b++) {
        order[b] = b;
        off[b + 1] = off[b] + (int64_t)sizes[blk_row[b]] * sizes[blk_col[b]];
      }
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return blk_row[a] != blk_row[b] ? blk_row[a] < blk_row[b] : blk_col[a] < blk_col[b];
      });
      r->brow.resize((size_t)nblocks);
      r->bcol.resize((size_t)nblocks);
      int64_t at = 0;
      for (int64_t p = 0; p < nblocks; p++) {
        const int64_t b = order[p];
        if (p > 0 && blk_row[b] == r->brow[p - 1] && blk_col[b] == r->bcol[p - 1]) {
          forget(s, r);
          return BSM_ERR_DUPLICATE_BLOCK;
        }
        r->brow[p] = blk_row[b];
        r->bcol[p] = blk_col[b];
        memcpy(r->vals + at, values + off[b], (size_t)(off[b + 1] - off[b]) * sizeof(double));
        at += off[b + 1] - off[b];
      }
    }
  } catch (const std::bad_alloc &) {
    forget(s, r);
    return BSM_ERR_NOMEM;
  }
  r->eps = eps;
  int64_t macs = 0;
  r->footprint = footprint_bound(*r, s->precision, &r->c_vals_bound, &macs);
  r->est_ms = est_run_ms(macs, s->precision);
  if (r->footprint > s->budget) {  // could never be admitted
    forget(s, r);
    return BSM_ERR_NOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = t_arrive;
    r->t_queued = now_ms();
    r->deadline = r->t_submit + kStretch * r->est_ms;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *id = r->id;
  }
  s->cv.notify_all();
  return BSM_OK;
}

int bsm_server_submit(bsm_server s, int32_t nbrows, const int32_t *sizes, int64_t nblocks,
                      const int32_t *blk_row, const int32_t *blk_col, const double *values,
                      double eps, int64_t *id) {
  return submit_request(s, nbrows, sizes, nblocks, blk_row, blk_col, values, eps, false, id);
}

int bsm_server_submit_borrowed(bsm_server s, int32_t nbrows, const int32_t *sizes,
                               int64_t nblocks, const int32_t *blk_row, const int32_t *blk_col,
                               const double *values, double eps, int64_t *id) {
  return submit_request(s, nbrows, sizes, nblocks, blk_row, blk_col, values, eps, true, id);
}

int bsm_server_progress(bsm_server s, int32_t *completed) {
  if (!s) return BSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = (int32_t)(s->completed - s->reported);
  s->reported = s->completed;
  return BSM_OK;
}

int bsm_server_poll(bsm_server s, int64_t id, int32_t *state, double *latency_ms,
                    int64_t *nblocks, int64_t *nnz) {
  if (!s || !state) return BSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return BSM_ERR_INVALID_ARG;
  const Request *r = it->second;
  const bool fin = r->state >= kDone;
  *state = r->state;
  if (latency_ms) *latency_ms = fin ? r->t_done - r->t_submit : -1.0;
  if (nblocks) *nblocks = fin ? r->nblk : 0;
  if (nnz) *nnz = fin ? r->nnz : 0;
  return r->state == kFailed ? r->err : BSM_OK;
}

int bsm_server_timing(bsm_server s, int64_t id, double *submit_ms, double *wait_ms,
                      double *run_ms) {
  if (!s) return BSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->state < kDone) return BSM_ERR_INVALID_ARG;
  const Request *r = it->second;
  if (submit_ms) *submit_ms = r->t_queued - r->t_submit;
  if (wait_ms) *wait_ms = r->t_start - r->t_queued;
  if (run_ms) *run_ms = r->t_done - r->t_start;
  return BSM_OK;
}

int bsm_server_take(bsm_server s, int64_t id, int64_t cap_blk, int32_t *blk_row,
                    int32_t *blk_col, int64_t cap_nnz, double *values) {
  if (!s) return BSM_ERR_INVALID_ARG;
  Request *r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BSM_ERR_INVALID_ARG;
    r = it->second;
    if (r->state == kFailed) {
      const int err = r->err;
      s->reqs.erase(it);
      forget(s, r);
      return err;
    }
    if (r->state != kDone) return BSM_ERR_INVALID_ARG;
    if (((blk_row || blk_col) && cap_blk < r->nblk) || (values && cap_nnz < r->nnz))
      return BSM_ERR_INVALID_ARG;  // the result stays until taken
    s->reqs.erase(it);  // from here on only this call sees the request
  }
  if (blk_row) std::copy(r->res_row, r->res_row + r->nblk, blk_row);
  if (blk_col) std::copy(r->res_col, r->res_col + r->nblk, blk_col);
  if (values) std::copy(r->res_val, r->res_val + r->nnz, values);
  forget(s, r);
  return BSM_OK;
}

int bsm_server_result(bsm_server s, int64_t id, const int32_t **blk_row, const int32_t **blk_col,
                      const double **values, int64_t *nblocks, int64_t *nnz) {
  if (!s) return BSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->state != kDone) return BSM_ERR_INVALID_ARG;
  const Request *r = it->second;
  if (blk_row) *blk_row = r->res_row;
  if (blk_col) *blk_col = r->res_col;
  if (values) *values = r->res_val;
  if (nblocks) *nblocks = r->nblk;
  if (nnz) *nnz = r->nnz;
  return BSM_OK;
}

int bsm_server_release(bsm_server s, int64_t id) {
  if (!s) return BSM_ERR_INVALID_ARG;
  Request *r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second->state < kDone) return BSM_ERR_INVALID_ARG;
    r = it->second;
    s->reqs.erase(it);
  }
  forget(s, r);
  return BSM_OK;
}

int bsm_server_get_info(bsm_server s, bsm_server_info *out) {
  if (!s || !out) return BSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int64_t)s->queue.size();
  out->running = s->running;
  out->completed = s->completed;
  out->bytes_in_use = s->in_use;
  out->bytes_peak = s->peak;
  out->budget = s->budget;
  out->batches = s->batches;
  return BSM_OK;
}

}  // extern "C"
