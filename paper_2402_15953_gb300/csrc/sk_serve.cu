// Continuous-batching request loop over live sketch sets resident on one GPU
// (sk_server_*): the serving form of the update (Algorithm 2) and the estimate
// (Algorithm 3 and the median over rows).
//
// Scheduling
//  - Every set keeps its requests in arrival order.  An estimate of a set sees exactly
//    the updates of that set that arrived before it; updates that arrive after it wait
//    until it has read the counters.  Results are therefore identical to running the
//    requests one by one (counter updates are exact integer additions).
//  - Across sets nothing is serialised: the scheduler thread admits the head request of
//    each set, oldest first, as soon as an update slot (a bounded number of in-flight
//    update batches) or an estimate worker is free and its device memory fits the HBM
//    budget, so newly arrived work joins the work already running on the device.
//  - Updates are coalesced: every update admitted in one scheduling pass (across sets, and
//    consecutive updates of one set) forms one batch.  Its host columns are copied into one
//    stream-ordered staging buffer on the copy stream, then ONE persistent multi-item
//    launch on the update stream applies all of the batch's plain updates (sketches are
//    linear, Section 2.2: the counters receive the same sums in any order or grouping);
//    updates that declare key domains run as their own sk_sketch_update_batch calls, so a
//    large one can take the key tables.  An event marks the batch's end and each touched
//    set's last admitted update; a pass that meets an estimate launches its batch first.
//  - Estimates: one worker thread per estimate stream takes up to kEstBatch admitted
//    estimates at a time (of distinct
//    sets: a set has one admitted estimate at most), its stream waits for each set's
//    last update, and one many-set estimate runs them (fused sets of one width share
//    their transforms).
//  - A retire thread waits on the oldest in-flight batch's event (batches complete in
//    launch order on the single update stream) and releases its slot and memory; the
//    scheduler sleeps on a condition variable until a submission, a retired update or a
//    finished estimate changes what can be admitted.  No thread polls.
//  - Memory: the counters of every registered set, the staging buffers of in-flight
//    updates and a per-estimate scratch allowance are charged against the budget; a
//    request that does not fit waits.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "sk_internal.h"

using sk::set_status_from_cuda;

namespace {

constexpr int kEstBatch = 8;    // estimates a worker runs together
constexpr int kUpdBatch = 64;   // updates coalesced into one batch at most
struct SvRequest {
  int64_t id = 0;
  bool is_estimate = false;
  int32_t set_id = 0;
  int32_t relation = 0;
  int64_t n = 0;
  const int64_t* cols = nullptr;   // host, attribute-major, stride `stride`
  int64_t stride = 0;
  const int64_t* w = nullptr;      // host or null
  std::vector<int64_t> domain;     // declared key domains (empty: none)
  size_t bytes = 0;                // memory charged while admitted
  double arrival = 0.0, done = 0.0;
  bool finished = false;
  sk_status status = SK_OK;
  sk_estimate est;
};

// Updates admitted together: one staging buffer, one multi-item launch (plus one call per
// update with declared domains), one completion event.
struct SvBatch {
  std::vector<SvRequest*> reqs;
  size_t bytes = 0;                // charged against the budget (sum of the requests')
  cudaEvent_t ev = nullptr;
  int slot = -1;                   // pinned descriptor slot
};

struct SvSet {
  sk_set* set = nullptr;
  size_t counter_bytes = 0;
  size_t est_bytes = 0;
  std::deque<SvRequest*> queue;
  bool estimating = false;
  bool has_update = false;
  cudaEvent_t last_update = nullptr;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct sk_server {
  int device = 0;
  size_t budget = 0, used = 0;
  size_t resident = 0;               // counters of the registered sets (charged for good)
  int slots = 1;
  int est_free = 1;
  std::chrono::steady_clock::time_point t0;
  cudaStream_t copy_stream = nullptr, update_stream = nullptr;
  std::vector<cudaStream_t> est_streams;
  std::mutex mu;
  std::condition_variable cv;        // scheduler, retire thread, waiters
  std::condition_variable est_cv;    // estimate workers
  std::map<int32_t, SvSet> sets;
  std::map<int64_t, std::unique_ptr<SvRequest>> reqs;
  std::deque<SvBatch*> inflight;     // launched update batches, launch order
  char* desc_host = nullptr;         // pinned blocks, one per slot: zeroed work counter + descriptors
  size_t desc_block = 0;             // bytes per block
  std::vector<cudaEvent_t> ev_copied, ev_done;   // per slot, reused by its batches
  std::vector<int> free_desc;        // free slots
  sk_update_plan_config cfg{};       // launch configuration of the batches
  uint64_t batches = 0, batched_updates = 0;
  std::deque<SvRequest*> est_queue;  // admitted estimates
  int64_t next_id = 1;
  int64_t unfinished = 0;
  bool changed = false;
  bool stop = false;
  bool hold = false;                 // admission paused (requests still queue)
  std::vector<std::thread> threads;
};

namespace {

// Device bytes an admitted update holds: its staged columns and weights.
size_t update_bytes(const sk_set* s, int relation, int64_t n, bool weights) {
  return (size_t)n * 8 * ((size_t)s->num_join_attrs[relation] + (weights ? 1 : 0));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

void finish(sk_server* sv, SvRequest* q, sk_status st) {
  q->status = st;
  q->done = now_s(sv->t0);
  q->finished = true;
  sv->unfinished--;
  sv->changed = true;
}

// Launches one batch of admitted updates (called with the lock held).  Layout of its staging
// buffer: work counter (256 B) | descriptors | per request: columns, weights (256-aligned).
// The work counter's zero and the descriptors come from the slot's pinned block in one copy.
// A batch of one update without declared domains is a plain sk_sketch_update_batch call.
sk_status launch_batch(sk_server* sv, SvBatch* b) {
  const size_t dsz = sk::multi_item_size();
  const size_t head = 256 + align256(dsz * b->reqs.size());
  size_t total = head;
  for (SvRequest* q : b->reqs) total += align256(q->bytes);
  char* buf = nullptr;
  // from the library's pool, which keeps its memory mapped between batches (the device's
  // default pool would return it at every synchronisation and map it again for the next)
  cudaError_t e = sk::pool_malloc_async((void**)&buf, total, sv->copy_stream);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  std::vector<sk_update_item> items;
  std::vector<std::pair<SvRequest*, std::pair<int64_t*, int64_t*>>> direct;   // own calls
  size_t off = head;
  const bool single = b->reqs.size() == 1;
  for (SvRequest* q : b->reqs) {
    sk_set* s = sv->sets[q->set_id].set;
    const int a = s->num_join_attrs[q->relation];
    int64_t* dc = (int64_t*)(buf + off);
    int64_t* dw = q->w ? dc + (size_t)q->n * a : nullptr;
    off += align256(q->bytes);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dc, (size_t)q->n * 8, q->cols, (size_t)q->stride * 8, (size_t)q->n * 8, (size_t)a,
                            cudaMemcpyHostToDevice, sv->copy_stream);
    if (e == cudaSuccess && dw) e = cudaMemcpyAsync(dw, q->w, (size_t)q->n * 8, cudaMemcpyHostToDevice, sv->copy_stream);
    if (single || !q->domain.empty() || a > 5) direct.push_back({q, {dc, dw}});
    else items.push_back(sk_update_item{s, q->relation, q->n, dc, q->n, dw});
  }
  int64_t chunks = 0;
  int coef_words = 0;
  size_t smem = 0;
  char* blk = sv->desc_host + (size_t)b->slot * sv->desc_block;
  sk_status st = set_status_from_cuda(e);
  if (st == SK_OK && !items.empty()) {
    std::memset(blk, 0, 256);
    st = sk::multi_describe(items.data(), (int)items.size(), sv->cfg, blk + 256, &chunks, &coef_words, &smem);
    if (st == SK_OK)
      st = set_status_from_cuda(cudaMemcpyAsync(buf, blk, 256 + dsz * items.size(), cudaMemcpyHostToDevice,
                                                sv->copy_stream));
  }
  const cudaEvent_t copied = sv->ev_copied[b->slot];
  if (st == SK_OK) st = set_status_from_cuda(cudaEventRecord(copied, sv->copy_stream));
  if (st == SK_OK) st = set_status_from_cuda(cudaStreamWaitEvent(sv->update_stream, copied, 0));
  if (st == SK_OK && !items.empty())
    st = sk::multi_launch(buf + 256, (int)items.size(), chunks, sv->cfg, coef_words, smem,
                          (unsigned long long*)buf, sv->update_stream, false);
  for (auto& dq : direct) {
    if (st != SK_OK) break;
    SvRequest* q = dq.first;
    st = sk_sketch_update_batch(sv->sets[q->set_id].set, q->relation, q->n, dq.second.first, q->n,
                                dq.second.second, q->domain.empty() ? nullptr : q->domain.data(), sv->update_stream);
  }
  const cudaError_t ef = cudaFreeAsync(buf, sv->update_stream);
  if (st == SK_OK) st = set_status_from_cuda(ef);
  b->ev = sv->ev_done[b->slot];
  if (st == SK_OK) st = set_status_from_cuda(cudaEventRecord(b->ev, sv->update_stream));
  for (SvRequest* q : b->reqs) {
    SvSet& ss = sv->sets[q->set_id];
    if (st == SK_OK) st = set_status_from_cuda(cudaEventRecord(ss.last_update, sv->update_stream));
    if (st == SK_OK) ss.has_update = true;
  }
  sv->batches++;
  sv->batched_updates += b->reqs.size();
  return st;
}

// Launches the pass's batch, if any (lock held); on failure its requests finish with the error.
void flush_batch(sk_server* sv, SvBatch*& b) {
  if (!b) return;
  const sk_status st = launch_batch(sv, b);
  if (st != SK_OK) {
    sv->used -= b->bytes;
    for (SvRequest* q : b->reqs) finish(sv, q, st);
    sv->free_desc.push_back(b->slot);
    delete b;
  } else {
    sv->inflight.push_back(b);
  }
  b = nullptr;
}

// One scheduling pass (lock held): heads of the sets' queues in global arrival order.
void admit(sk_server* sv) {
  std::vector<std::pair<int64_t, int32_t>> heads;
  for (auto& kv : sv->sets)
    if (!kv.second.queue.empty() && !kv.second.estimating) heads.push_back({kv.second.queue.front()->id, kv.first});
  std::sort(heads.begin(), heads.end());
  SvBatch* b = nullptr;
  for (const auto& h : heads) {
    SvSet& ss = sv->sets[h.second];
    while (!ss.queue.empty() && !ss.estimating) {
      SvRequest* q = ss.queue.front();
      if (!q->is_estimate) {
        if (!b && sv->free_desc.empty()) break;                      // every update slot in flight
        if (b && (int)b->reqs.size() >= kUpdBatch) break;
        if (sv->used + q->bytes > sv->budget) break;
        if (!b) {
          b = new (std::nothrow) SvBatch();
          if (!b) return;
          b->slot = sv->free_desc.back();
          sv->free_desc.pop_back();
        }
        ss.queue.pop_front();
        sv->used += q->bytes;
        b->bytes += q->bytes;
        b->reqs.push_back(q);
      } else {
        if (sv->est_free == 0 || sv->used + ss.est_bytes > sv->budget) break;
        // the estimate waits for this set's last update event: launch the pending batch first
        flush_batch(sv, b);
        ss.queue.pop_front();
        q->bytes = ss.est_bytes;
        sv->used += q->bytes;
        sv->est_free--;
        ss.estimating = true;
        sv->est_queue.push_back(q);
        sv->est_cv.notify_one();
        break;
      }
    }
  }
  flush_batch(sv, b);
}

void scheduler(sk_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] { return (sv->changed && !sv->hold) || sv->stop; });
    if (sv->stop) return;
    sv->changed = false;
    admit(sv);
    sv->cv.notify_all();   // new in-flight updates for the retire thread
  }
}

void retirer(sk_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] { return !sv->inflight.empty() || sv->stop; });
    if (sv->inflight.empty()) return;   // stop with nothing in flight
    SvBatch* b = sv->inflight.front();
    lk.unlock();
    const cudaError_t e = cudaEventSynchronize(b->ev);
    lk.lock();
    sv->inflight.pop_front();
    sv->used -= b->bytes;
    for (SvRequest* q : b->reqs) finish(sv, q, set_status_from_cuda(e));
    sv->free_desc.push_back(b->slot);
    delete b;
    sv->cv.notify_all();
  }
}

void estimator(sk_server* sv, cudaStream_t stream) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  std::vector<SvRequest*> batch;
  std::vector<sk_set*> sets;
  std::vector<cudaEvent_t> waits;
  std::vector<sk_estimate> outs;
  for (;;) {
    sv->est_cv.wait(lk, [&] { return !sv->est_queue.empty() || sv->stop; });
    if (sv->est_queue.empty()) return;
    batch.clear();
    sets.clear();
    waits.clear();
    while (!sv->est_queue.empty() && (int)batch.size() < kEstBatch) {
      SvRequest* q = sv->est_queue.front();
      sv->est_queue.pop_front();
      SvSet& ss = sv->sets[q->set_id];
      batch.push_back(q);
      sets.push_back(ss.set);
      if (ss.has_update) waits.push_back(ss.last_update);
    }
    lk.unlock();
    sk_status st = SK_OK;
    for (cudaEvent_t ev : waits)
      if (st == SK_OK) st = set_status_from_cuda(cudaStreamWaitEvent(stream, ev, 0));
    if (st == SK_OK) {
      if (batch.size() == 1) {
        st = sk_estimate_join(sets[0], &batch[0]->est, stream);
      } else {
        outs.assign(batch.size(), sk_estimate());
        st = sk::run_estimate_many(sets.data(), (int)sets.size(), outs.data(), stream);
        for (size_t i = 0; i < batch.size(); i++) batch[i]->est = outs[i];
      }
    }
    lk.lock();
    for (SvRequest* q : batch) {
      sv->sets[q->set_id].estimating = false;
      sv->est_free++;
      sv->used -= q->bytes;
      finish(sv, q, st);
    }
    sv->cv.notify_all();
  }
}

}  // namespace

extern "C" {

sk_status sk_server_create(int64_t hbm_budget_bytes, int32_t update_slots, int32_t estimate_workers,
                           int32_t estimate_priority, sk_server** out) {
  if (!out || hbm_budget_bytes <= 0 || update_slots < 1 || estimate_workers < 1 || estimate_workers > 64)
    return SK_ERR_INVALID_ARG;
  *out = nullptr;
  sk_server* sv = new (std::nothrow) sk_server();
  if (!sv) return SK_ERR_NO_MEMORY;
  sv->budget = (size_t)hbm_budget_bytes;
  sv->slots = update_slots;
  sv->est_free = estimate_workers * kEstBatch;
  sv->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&sv->device);
  int lo = 0, hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->update_stream, cudaStreamNonBlocking);
  // pinned descriptor blocks, one per update slot (a batch's descriptors are copied from
  // its block asynchronously, so the block stays reserved until the batch retires)
  sv->desc_block = 256 + align256(kUpdBatch * sk::multi_item_size());
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&sv->desc_host, (size_t)update_slots * sv->desc_block, cudaHostAllocDefault);
  for (int i = 0; i < update_slots && e == cudaSuccess; i++) {
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
    if (a) sv->ev_copied.push_back(a);
    if (b) sv->ev_done.push_back(b);
  }
  for (int i = 0; i < update_slots; i++) sv->free_desc.push_back(update_slots - 1 - i);
  // batches: chunks of 16384 tuples, 6 CTAs per SM, int32 shared sub-sketches up to 16384
  // counters (the plan defaults of sk_update_plan_create but with smaller chunks: serving
  // batches are 1e3..1e6 tuples)
  sv->cfg = sk_update_plan_config{16384, 256, 6, 16384, 0};
  for (int i = 0; i < estimate_workers && e == cudaSuccess; i++) {
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, estimate_priority ? hi : lo);
    if (e == cudaSuccess) sv->est_streams.push_back(s);
  }
  if (e != cudaSuccess) {
    for (cudaStream_t s : sv->est_streams) cudaStreamDestroy(s);
    if (sv->copy_stream) cudaStreamDestroy(sv->copy_stream);
    if (sv->update_stream) cudaStreamDestroy(sv->update_stream);
    if (sv->desc_host) cudaFreeHost(sv->desc_host);
    for (cudaEvent_t x : sv->ev_copied) cudaEventDestroy(x);
    for (cudaEvent_t x : sv->ev_done) cudaEventDestroy(x);
    delete sv;
    return set_status_from_cuda(e);
  }
  sv->threads.emplace_back(scheduler, sv);
  sv->threads.emplace_back(retirer, sv);
  for (cudaStream_t s : sv->est_streams) sv->threads.emplace_back(estimator, sv, s);
  *out = sv;
  return SK_OK;
}

sk_status sk_server_register_set(sk_server* sv, int32_t set_id, sk_set* set) {
  if (!sv || !set) return SK_ERR_INVALID_ARG;
  const size_t cb = (size_t)set->r * set->d * set->m * 8;
  const size_t slots = (size_t)std::max(2, set->r);
  const size_t est = (slots + 1) * set->d * set->m * 32 + 2 * (size_t)set->d * 4 * set->m * 16 + (size_t)(set->m / 2) * 16;
  cudaEvent_t ev = nullptr;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->sets.count(set_id)) return SK_ERR_INVALID_ARG;
  if (sv->used + cb > sv->budget) return SK_ERR_OVER_BUDGET;
  const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  SvSet& ss = sv->sets[set_id];
  ss.set = set;
  ss.counter_bytes = cb;
  ss.est_bytes = est;
  ss.last_update = ev;
  sv->used += cb;
  sv->resident += cb;
  return SK_OK;
}

sk_status sk_server_submit_update(sk_server* sv, int32_t set_id, int32_t relation, int64_t n_rows,
                                  const int64_t* host_cols, int64_t col_stride, const int64_t* host_weights,
                                  const int64_t* domain_hint, int64_t* request_id) {
  if (!sv || !request_id || n_rows < 0) return SK_ERR_INVALID_ARG;
  std::unique_ptr<SvRequest> q(new (std::nothrow) SvRequest());
  if (!q) return SK_ERR_NO_MEMORY;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sets.find(set_id);
  if (it == sv->sets.end()) return SK_ERR_INVALID_ARG;
  sk_set* s = it->second.set;
  if (relation < 0 || relation >= s->r || (n_rows > 0 && (!host_cols || col_stride < n_rows)))
    return SK_ERR_INVALID_ARG;
  q->id = sv->next_id++;
  q->set_id = set_id;
  q->relation = relation;
  q->n = n_rows;
  q->cols = host_cols;
  q->stride = col_stride;
  q->w = host_weights;
  if (domain_hint) q->domain.assign(domain_hint, domain_hint + s->num_join_attrs[relation]);
  q->bytes = update_bytes(s, relation, n_rows, host_weights != nullptr);
  q->arrival = now_s(sv->t0);
  *request_id = q->id;
  SvRequest* raw = q.get();
  sv->reqs[q->id] = std::move(q);
  sv->unfinished++;
  if (n_rows == 0) {   // no tuples: nothing to order against, finished at once
    finish(sv, raw, SK_OK);
    sv->cv.notify_all();
    return SK_OK;
  }
  if (raw->bytes > sv->budget - sv->resident) {   // could never be admitted
    finish(sv, raw, SK_ERR_OVER_BUDGET);
    sv->cv.notify_all();
    return SK_OK;
  }
  it->second.queue.push_back(raw);
  sv->changed = true;
  sv->cv.notify_all();
  return SK_OK;
}

sk_status sk_server_submit_estimate(sk_server* sv, int32_t set_id, int64_t* request_id) {
  if (!sv || !request_id) return SK_ERR_INVALID_ARG;
  std::unique_ptr<SvRequest> q(new (std::nothrow) SvRequest());
  if (!q) return SK_ERR_NO_MEMORY;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sets.find(set_id);
  if (it == sv->sets.end()) return SK_ERR_INVALID_ARG;
  q->id = sv->next_id++;
  q->is_estimate = true;
  q->set_id = set_id;
  q->arrival = now_s(sv->t0);
  *request_id = q->id;
  SvRequest* raw = q.get();
  sv->reqs[q->id] = std::move(q);
  sv->unfinished++;
  if (it->second.est_bytes > sv->budget - sv->resident) {   // could never be admitted
    finish(sv, raw, SK_ERR_OVER_BUDGET);
    sv->cv.notify_all();
    return SK_OK;
  }
  it->second.queue.push_back(raw);
  sv->changed = true;
  sv->cv.notify_all();
  return SK_OK;
}

sk_status sk_server_result(sk_server* sv, int64_t request_id, int32_t wait, int32_t* finished, sk_status* status,
                           sk_estimate* est, double* arrival_s, double* done_s) {
  if (!sv || !finished) return SK_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(request_id);
  if (it == sv->reqs.end()) return SK_ERR_INVALID_ARG;
  SvRequest* q = it->second.get();
  if (wait) sv->cv.wait(lk, [&] { return q->finished; });
  *finished = q->finished ? 1 : 0;
  if (!q->finished) return SK_OK;
  if (status) *status = q->status;
  if (est) {
    if (q->is_estimate) *est = q->est;
    else std::memset(est, 0, sizeof(*est));
  }
  if (arrival_s) *arrival_s = q->arrival;
  if (done_s) *done_s = q->done;
  sv->reqs.erase(it);
  return SK_OK;
}

sk_status sk_server_hold(sk_server* sv, int32_t on) {
  if (!sv) return SK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->hold = on != 0;
  if (!sv->hold) {
    sv->changed = true;
    sv->cv.notify_all();
  }
  return SK_OK;
}

sk_status sk_server_pending(sk_server* sv, int64_t* n) {
  if (!sv || !n) return SK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  *n = sv->unfinished;
  return SK_OK;
}

sk_status sk_server_drain(sk_server* sv) {
  if (!sv) return SK_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv.wait(lk, [&] { return sv->unfinished == 0; });
  return SK_OK;
}

sk_status sk_server_destroy(sk_server* sv) {
  if (!sv) return SK_OK;
  sk_server_hold(sv, 0);
  sk_server_drain(sv);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
    sv->est_cv.notify_all();
  }
  for (std::thread& t : sv->threads) t.join();
  cudaStreamSynchronize(sv->update_stream);
  for (cudaStream_t s : sv->est_streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  cudaStreamDestroy(sv->copy_stream);
  cudaStreamDestroy(sv->update_stream);
  for (auto& kv : sv->sets)
    if (kv.second.last_update) cudaEventDestroy(kv.second.last_update);
  cudaFreeHost(sv->desc_host);
  for (cudaEvent_t x : sv->ev_copied) cudaEventDestroy(x);
  for (cudaEvent_t x : sv->ev_done) cudaEventDestroy(x);
  delete sv;
  return SK_OK;
}

sk_status sk_server_stats(sk_server* sv, int64_t* batches, int64_t* batched_updates) {
  if (!sv) return SK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (batches) *batches = (int64_t)sv->batches;
  if (batched_updates) *batched_updates = (int64_t)sv->batched_updates;
  return SK_OK;
}

}  // extern "C"
