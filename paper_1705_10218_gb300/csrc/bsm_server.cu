// bsm_server.cu -- a request loop over the filtered multiply: independent
// multiplies C = A.A of differently sized systems arrive one by one and are run
// with continuous batching.
//
// The server owns `slots` lanes, each a libbsm context with its own stream and
// workspace. A request waits in a FIFO queue until a lane is free and its
// device-memory footprint fits the budget next to the requests already held;
// it is then uploaded and its multiply enqueued on that lane, while the other
// lanes' multiplies keep running: requests of different sizes overlap on the
// device, and a request that arrives while others run starts as soon as a lane
// and memory free up (no waiting for a batch to drain). The footprint is an
// upper bound before the multiply (A, a dense-or-candidate bound on C, the
// product records) and the exact result size after it; results stay on the
// device until taken. Everything goes through the public C ABI, so a request's
// result is computed by exactly the kernels a lone bsm_multiply uses.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "../../include/bsm.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

enum { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
  int64_t id = 0;
  std::vector<int32_t> sizes, brow, bcol;
  std::vector<double> vals;
  double eps = 0;
  int64_t footprint = 0;  // bytes held on the device while admitted
  int state = kQueued;
  int err = BSM_OK;
  int slot = -1;
  double t_submit = 0, t_start = 0, t_done = 0;
  bsm_mat A = nullptr, C = nullptr;
  int64_t nblk = 0, nnz = 0;
};

struct Slot {
  bsm_ctx ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Request *req = nullptr;
};

// Upper bound of the device bytes a request C = A.A can hold.
int64_t footprint_bound(const Request &r) {
  const int64_t nbr = (int64_t)r.sizes.size();
  std::vector<int64_t> row_nblk(nbr, 0), row_cols(nbr, 0);
  for (size_t b = 0; b < r.brow.size(); b++) {
    row_nblk[r.brow[b]]++;
    row_cols[r.brow[b]] += r.sizes[r.bcol[b]];
  }
  int64_t dim = 0;
  for (int32_t s : r.sizes) dim += s;
  int64_t cand = 0, cand_vals = 0;
  for (size_t b = 0; b < r.brow.size(); b++) {
    cand += row_nblk[r.bcol[b]];
    cand_vals += (int64_t)r.sizes[r.brow[b]] * row_cols[r.bcol[b]];
  }
  const int64_t a_bytes = 8 * (int64_t)r.vals.size() + 32 * (int64_t)r.brow.size();
  const int64_t c_blocks = std::min<int64_t>(nbr * nbr, cand);
  const int64_t c_vals = std::min<int64_t>(dim * dim, cand_vals);
  // A (+ slices for the split precisions), C twice (front/back), per-block
  // metadata, product records
  return 4 * a_bytes + 2 * (8 * c_vals + 32 * c_blocks) + 8 * cand + 64 * nbr + (1 << 20);
}

}  // namespace

struct bsm_server_s {
  int device = 0;
  int precision = BSM_PREC_FP64;
  int64_t budget = 0, in_use = 0, peak = 0;
  std::vector<Slot> slots;
  std::deque<Request *> queue;
  std::map<int64_t, Request *> reqs;
  int64_t next_id = 1;
  int64_t completed = 0;
};

static void release(bsm_server s, Request *r) {
  if (r->A) bsm_mat_destroy(r->A);
  if (r->C) bsm_mat_destroy(r->C);
  r->A = r->C = nullptr;
  s->in_use -= r->footprint;
  r->footprint = 0;
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
  s->slots.resize(o.slots);
  for (Slot &sl : s->slots) {
    int rc = bsm_ctx_create(device, &sl.ctx);
    if (rc == BSM_OK && (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess))
      rc = BSM_ERR_CUDA;
    if (rc != BSM_OK) {
      bsm_server_destroy(s);
      return rc;
    }
  }
  *out = s;
  return BSM_OK;
}

int bsm_server_destroy(bsm_server s) {
  if (!s) return BSM_ERR_INVALID_ARG;
  cudaSetDevice(s->device);
  for (Slot &sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  }
  for (auto &kv : s->reqs) {
    release(s, kv.second);
    delete kv.second;
  }
  s->reqs.clear();
  for (Slot &sl : s->slots) {
    if (sl.ctx) bsm_ctx_destroy(sl.ctx);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
  return BSM_OK;
}

int bsm_server_submit(bsm_server s, int32_t nbrows, const int32_t *sizes, int64_t nblocks,
                      const int32_t *blk_row, const int32_t *blk_col, const double *values,
                      double eps, int64_t *id) {
  if (!s || !id || nbrows < 0 || nblocks < 0 || (nbrows > 0 && !sizes) ||
      (nblocks > 0 && (!blk_row || !blk_col || !values)))
    return BSM_ERR_INVALID_ARG;
  Request *r = new (std::nothrow) Request();
  if (!r) return BSM_ERR_NOMEM;
  r->sizes.assign(sizes, sizes + nbrows);
  r->brow.assign(blk_row, blk_row + nblocks);
  r->bcol.assign(blk_col, blk_col + nblocks);
  int64_t nv = 0;
  for (int64_t b = 0; b < nblocks; b++) {
    if (blk_row[b] < 0 || blk_row[b] >= nbrows || blk_col[b] < 0 || blk_col[b] >= nbrows) {
      delete r;
      return BSM_ERR_OUT_OF_RANGE;
    }
    nv += (int64_t)sizes[blk_row[b]] * sizes[blk_col[b]];
  }
  for (int32_t v : r->sizes)
    if (v <= 0) {
      delete r;
      return BSM_ERR_INVALID_ARG;
    }
  r->vals.assign(values, values + nv);
  r->eps = eps;
  r->footprint = footprint_bound(*r);
  if (r->footprint > s->budget) {  // could never be admitted
    delete r;
    return BSM_ERR_NOMEM;
  }
  r->id = s->next_id++;
  r->t_submit = now_ms();
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  *id = r->id;
  return BSM_OK;
}

int bsm_server_progress(bsm_server s, int32_t *completed) {
  if (!s) return BSM_ERR_INVALID_ARG;
  if (cudaSetDevice(s->device) != cudaSuccess) return BSM_ERR_CUDA;
  int32_t done = 0;
  // 1. retire finished lanes
  for (Slot &sl : s->slots) {
    Request *r = sl.req;
    if (!r) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) {
      r->err = BSM_ERR_CUDA;
    } else {
      r->err = bsm_mat_nblocks(r->C, &r->nblk, &r->nnz);  // completes the result
    }
    r->t_done = now_ms();
    r->state = r->err == BSM_OK ? kDone : kFailed;
    if (r->A) bsm_mat_destroy(r->A);
    r->A = nullptr;
    // from the bound to what the result really holds (front and back buffers)
    const int64_t held = r->err == BSM_OK ? 2 * (8 * r->nnz + 32 * r->nblk) : 0;
    s->in_use += held - r->footprint;
    r->footprint = held;
    if (r->err != BSM_OK && r->C) {
      bsm_mat_destroy(r->C);
      r->C = nullptr;
      s->in_use -= r->footprint;
      r->footprint = 0;
    }
    sl.req = nullptr;
    s->completed++;
    done++;
  }
  // 2. admit from the head of the queue while a lane and memory are free
  for (Slot &sl : s->slots) {
    if (sl.req || s->queue.empty()) continue;
    Request *r = s->queue.front();
    if (s->in_use + r->footprint > s->budget) break;  // FIFO: wait for memory
    s->queue.pop_front();
    s->in_use += r->footprint;
    s->peak = std::max(s->peak, s->in_use);
    const int32_t nbr = (int32_t)r->sizes.size();
    int rc = bsm_mat_create(sl.ctx, nbr, r->sizes.data(), nbr, r->sizes.data(),
                            (int64_t)r->brow.size(), r->brow.data(), r->bcol.data(),
                            r->vals.data(), &r->A);
    if (rc == BSM_OK)
      rc = bsm_mat_create(sl.ctx, nbr, r->sizes.data(), nbr, r->sizes.data(), 0, nullptr, nullptr,
                          nullptr, &r->C);
    if (rc == BSM_OK) {
      bsm_opts o{};
      o.precision = s->precision;
      o.stream = sl.stream;
      rc = bsm_multiply(sl.ctx, 1.0, r->A, r->A, 0.0, r->C, r->eps, &o, nullptr);
    }
    if (rc == BSM_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = BSM_ERR_CUDA;
    r->t_start = now_ms();
    r->slot = (int)(&sl - s->slots.data());
    if (rc != BSM_OK) {
      r->err = rc;
      r->state = kFailed;
      r->t_done = r->t_start;
      release(s, r);
      s->completed++;
      done++;
      continue;
    }
    r->state = kRunning;
    sl.req = r;
    // the host copies are no longer needed
    std::vector<double>().swap(r->vals);
  }
  if (completed) *completed = done;
  return BSM_OK;
}

int bsm_server_poll(bsm_server s, int64_t id, int32_t *state, double *latency_ms,
                    int64_t *nblocks, int64_t *nnz) {
  if (!s || !state) return BSM_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return BSM_ERR_INVALID_ARG;
  Request *r = it->second;
  *state = r->state;
  if (latency_ms) *latency_ms = (r->state >= kDone) ? r->t_done - r->t_submit : -1.0;
  if (nblocks) *nblocks = r->nblk;
  if (nnz) *nnz = r->nnz;
  return r->state == kFailed ? r->err : BSM_OK;
}

int bsm_server_take(bsm_server s, int64_t id, int64_t cap_blk, int32_t *blk_row,
                    int32_t *blk_col, int64_t cap_nnz, double *values) {
  if (!s) return BSM_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return BSM_ERR_INVALID_ARG;
  Request *r = it->second;
  if (r->state == kFailed) {
    const int err = r->err;
    s->reqs.erase(it);
    release(s, r);
    delete r;
    return err;
  }
  if (r->state != kDone) return BSM_ERR_INVALID_ARG;
  int rc = BSM_OK;
  if (blk_row || blk_col) rc = bsm_mat_get_pattern(r->C, cap_blk, blk_row, blk_col);
  if (rc == BSM_OK && values) rc = bsm_mat_get_values(r->C, cap_nnz, values);
  if (rc != BSM_OK) return rc;  // e.g. a small cap: the result stays until taken
  s->reqs.erase(it);
  release(s, r);
  delete r;
  return BSM_OK;
}

int bsm_server_get_info(bsm_server s, bsm_server_info *out) {
  if (!s || !out) return BSM_ERR_INVALID_ARG;
  out->queued = (int64_t)s->queue.size();
  int64_t running = 0;
  for (const Slot &sl : s->slots) running += sl.req ? 1 : 0;
  out->running = running;
  out->completed = s->completed;
  out->bytes_in_use = s->in_use;
  out->bytes_peak = s->peak;
  out->budget = s->budget;
  return BSM_OK;
}

}  // extern "C"
