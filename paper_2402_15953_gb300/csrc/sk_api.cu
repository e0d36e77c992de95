// Host side of the C ABI: query validation and canonical numbering (Section 2.6
// notation), hash-function sampling (Algorithm 1, its sampling step), the Algorithm 3
// schedule, and dispatch to the update / merge / estimate kernels.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <set>

#include "sk_internal.h"

#include <atomic>

namespace sk {

static std::atomic<int64_t> g_launches{0};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t allow_dynamic_smem(const void* func) {
  static const int optin = [] {   // thread-safe one-time initialisation
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return x > 0 ? x : 48 * 1024;
  }();
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t fit_dynamic_smem(const void* func, size_t dynamic_bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  if (fa.sharedSizeBytes + dynamic_bytes <= (size_t)48 * 1024) return cudaSuccess;   // the default limit
  return allow_dynamic_smem(func);
}

// Stream-ordered device memory pool of this library (one per device, created on first use)
// for update scratch: key tables and the partitioned update's planes.  Up to
// SK_POOL_KEEP_MB (default 4096) MiB stay reserved between calls, so a batch's scratch of a
// few GB is not mapped again for every call; anything above that is returned to the
// device at the next synchronisation.
namespace {
constexpr int kPoolMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kPoolMaxDevices] = {};
}  // namespace

cudaError_t pool_malloc_async(void** ptr, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kPoolMaxDevices) return cudaMallocAsync(ptr, bytes, st);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pools[dev], &props);
      if (e != cudaSuccess) {
        g_pools[dev] = nullptr;
        return e;
      }
      const char* v = std::getenv("SK_POOL_KEEP_MB");
      const long long mb = v ? std::atoll(v) : 4096;
      uint64_t keep = (uint64_t)(mb < 0 ? 0 : mb) << 20;
      cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

sk_status set_status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SK_OK;
  if (e == cudaErrorMemoryAllocation) return SK_ERR_NO_MEMORY;
  return SK_ERR_CUDA;
}

namespace {

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): state advances by the golden-ratio increment and the
// output is the state passed through the variant-13 finaliser.
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // Uniform element of GF(2^61 - 1): the top 61 bits, 2^61 - 1 itself rejected.
  uint64_t field_element() {
    for (;;) {
      uint64_t v = next() >> 3;
      if (v != kP61) return v;
    }
  }
};

using Canon = QueryInfo;

int find_root(std::vector<int>& parent, int x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

// Validates the query and numbers attributes relation by relation; joins are
// stored as (u, v) with u < v and sorted; components are numbered in order of
// their smallest attribute.  The relations joined by the edges must form a tree.
sk_status canonicalize(const sk_query* q, Canon* c) {
  if (!q || q->num_relations < 2 || !q->num_join_attrs || (q->num_edges > 0 && !q->edges))
    return SK_ERR_INVALID_ARG;
  const int r = q->num_relations;
  c->r = r;
  c->offsets.assign(r, 0);
  int w = 0;
  for (int k = 0; k < r; k++) {
    const int a = q->num_join_attrs[k];
    if (a < 1 || a > kMaxAttrs) return SK_ERR_INVALID_ARG;
    c->num_join_attrs.push_back(a);
    c->offsets[k] = w;
    for (int t = 0; t < a; t++) c->rel_of.push_back(k);
    w += a;
  }
  std::set<std::pair<int, int>> es;
  for (int i = 0; i < q->num_edges; i++) {
    const sk_edge& e = q->edges[i];
    if (e.rel_a < 0 || e.rel_a >= r || e.rel_b < 0 || e.rel_b >= r) return SK_ERR_INVALID_ARG;
    if (e.attr_a < 0 || e.attr_a >= c->num_join_attrs[e.rel_a] || e.attr_b < 0 ||
        e.attr_b >= c->num_join_attrs[e.rel_b])
      return SK_ERR_INVALID_ARG;
    if (e.rel_a == e.rel_b) return SK_ERR_SELF_EDGE;
    const int u = c->offsets[e.rel_a] + e.attr_a, v = c->offsets[e.rel_b] + e.attr_b;
    const std::pair<int, int> p(std::min(u, v), std::max(u, v));
    if (es.count(p)) return SK_ERR_INVALID_ARG;
    es.insert(p);
  }
  c->edges.assign(es.begin(), es.end());
  std::vector<int> parent(r);
  for (int k = 0; k < r; k++) parent[k] = k;
  for (auto& e : c->edges) {
    const int a = find_root(parent, c->rel_of[e.first]), b = find_root(parent, c->rel_of[e.second]);
    if (a == b) return SK_ERR_CYCLIC_QUERY;
    parent[a] = b;
  }
  const int root0 = find_root(parent, 0);
  for (int k = 1; k < r; k++)
    if (find_root(parent, k) != root0) return SK_ERR_DISCONNECTED_QUERY;
  c->gamma.assign(w, {});
  c->incident.assign(w, {});
  for (int i = 0; i < (int)c->edges.size(); i++) {
    const auto& e = c->edges[i];
    c->gamma[e.first].push_back(e.second);
    c->gamma[e.second].push_back(e.first);
    c->incident[e.first].push_back(i);
    c->incident[e.second].push_back(i);
  }
  for (int u = 0; u < w; u++) {
    if (c->gamma[u].empty() || (int)c->gamma[u].size() > kMaxDegree) return SK_ERR_INVALID_ARG;
    std::sort(c->gamma[u].begin(), c->gamma[u].end());
  }
  c->comp_of.assign(w, -1);
  c->n_comp = 0;
  for (int s = 0; s < w; s++) {
    if (c->comp_of[s] >= 0) continue;
    std::vector<int> stack{s};
    c->comp_of[s] = c->n_comp;
    while (!stack.empty()) {
      const int x = stack.back();
      stack.pop_back();
      for (int y : c->gamma[x])
        if (c->comp_of[y] < 0) {
          c->comp_of[y] = c->n_comp;
          stack.push_back(y);
        }
    }
    c->n_comp++;
  }
  return SK_OK;
}

// Unrolls Algorithm 3 (CombineSketches from the root attribute) into a schedule
// over vector slots.  A freshly initialised all-ones vector multiplied by its
// first factor is just that factor, so no slot ever holds the ones vector.
void build_plan(sk_set* s) {
  std::vector<sk::EstOp> ops;
  std::vector<int> free_slots;
  int n_slots = 0;
  int corr = 0;
  auto alloc = [&]() {
    if (!free_slots.empty()) {
      int x = free_slots.back();
      free_slots.pop_back();
      return x;
    }
    return n_slots++;
  };
  auto release = [&](int x) { free_slots.push_back(x); };
  std::vector<char> visited(s->rel_of.size(), 0);
  std::function<int(int)> combine = [&](int u) -> int {
    const int k = s->rel_of[u];
    const int x = alloc();
    ops.push_back({OP_LEAF, x, -1, k});
    visited[u] = 1;
    for (int t = 0; t < s->num_join_attrs[k]; t++) {
      const int u2 = s->offsets[k] + t;
      if (u2 == u) continue;
      visited[u2] = 1;
      int a = -1;
      for (int v : s->gamma[u2]) {
        const int y = combine(v);
        if (a < 0) {
          a = y;
        } else {
          ops.push_back({OP_HAD, a, y, -1});
          release(y);
        }
      }
      ops.push_back({OP_CORR, x, a, -1});
      corr++;
      release(a);
    }
    for (int v : s->gamma[u]) {
      if (visited[v]) continue;
      const int y = combine(v);
      ops.push_back({OP_HAD, x, y, -1});
      release(y);
    }
    return x;
  };
  const int root = combine(0);
  ops.push_back({OP_SUM, root, root, -1});
  s->plan = ops;
  s->n_slots = n_slots;
  s->corr_steps = corr;
}

sk_status upload_relation_plans(sk_set* s) {
  s->rel.assign(s->r, sk::RelPlan());
  for (int k = 0; k < s->r; k++) {
    sk::RelPlan& rp = s->rel[k];
    rp.a = s->num_join_attrs[k];
    int len = 0;
    for (int t = 0; t < rp.a; t++) {
      const int u = s->offsets[k] + t;
      rp.deg[t] = (int)s->incident[u].size();
      len += 2 + 4 * rp.deg[t];
    }
    rp.coef_row_len = len;
    std::vector<uint64_t> packed((size_t)s->d * len);
    for (int row = 0; row < s->d; row++) {
      const uint64_t* cr = s->h_coef.data() + (size_t)row * s->coef_row_len;
      uint64_t* o = packed.data() + (size_t)row * len;
      for (int t = 0; t < rp.a; t++) {
        const int u = s->offsets[k] + t;
        *o++ = cr[2 * s->comp_of[u]];
        *o++ = cr[2 * s->comp_of[u] + 1];
        for (int e : s->incident[u])
          for (int c = 0; c < 4; c++) *o++ = cr[2 * s->n_comp + 4 * e + c];
      }
    }
    if (!rp.d_coef) {
      cudaError_t e = cudaMalloc(&rp.d_coef, packed.size() * sizeof(uint64_t));
      if (e != cudaSuccess) return set_status_from_cuda(e);
    }
    cudaError_t e = cudaMemcpy(rp.d_coef, packed.data(), packed.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_status_from_cuda(e);
  }
  return SK_OK;
}

void free_set(sk_set* s) {
  if (!s) return;
  for (auto& rp : s->rel)
    if (rp.d_coef) cudaFree(rp.d_coef);
  if (s->d_status) cudaFree(s->d_status);
  sk::free_estimator(s);
  delete s;
}

}  // namespace

sk_status query_info(const sk_query* q, QueryInfo* out) { return canonicalize(q, out); }

std::vector<uint64_t> draw_coefficients(uint64_t seed, int d, int row_len) {
  SplitMix64 rng{seed};
  std::vector<uint64_t> v((size_t)d * row_len);
  for (auto& x : v) x = rng.field_element();
  return v;
}

sk_status make_estimation_set(const QueryInfo& c, int64_t m, int d, uint64_t seed, std::vector<uint64_t> h_coef,
                              std::vector<int64_t*> rel_ctr, sk_set** out) {
  *out = nullptr;
  if ((int)rel_ctr.size() != c.r) return SK_ERR_INVALID_ARG;
  sk_set* s = new (std::nothrow) sk_set();
  if (!s) return SK_ERR_NO_MEMORY;
  s->r = c.r;
  s->m = m;
  s->d = d;
  s->seed = seed;
  s->num_join_attrs = c.num_join_attrs;
  s->offsets = c.offsets;
  s->rel_of = c.rel_of;
  s->comp_of = c.comp_of;
  s->edges = c.edges;
  s->gamma = c.gamma;
  s->incident = c.incident;
  s->n_comp = c.n_comp;
  s->coef_row_len = 2 * c.n_comp + 4 * (int)c.edges.size();
  s->h_coef = std::move(h_coef);
  s->rel_ctr = std::move(rel_ctr);
  cudaGetDevice(&s->device);
  cudaError_t e = cudaMalloc(&s->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_set(s);
    return set_status_from_cuda(e);
  }
  build_plan(s);
  *out = s;
  return SK_OK;
}

void destroy_set(sk_set* s) { free_set(s); }

}  // namespace sk

using namespace sk;

extern "C" {

const char* sk_status_string(sk_status status) {
  switch (status) {
    case SK_OK: return "SK_OK";
    case SK_ERR_INVALID_ARG: return "SK_ERR_INVALID_ARG";
    case SK_ERR_CYCLIC_QUERY: return "SK_ERR_CYCLIC_QUERY";
    case SK_ERR_DISCONNECTED_QUERY: return "SK_ERR_DISCONNECTED_QUERY";
    case SK_ERR_SELF_EDGE: return "SK_ERR_SELF_EDGE";
    case SK_ERR_UNSUPPORTED_WIDTH: return "SK_ERR_UNSUPPORTED_WIDTH";
    case SK_ERR_BUFFER_TOO_SMALL: return "SK_ERR_BUFFER_TOO_SMALL";
    case SK_ERR_MISMATCH: return "SK_ERR_MISMATCH";
    case SK_ERR_KEY_OUT_OF_DOMAIN: return "SK_ERR_KEY_OUT_OF_DOMAIN";
    case SK_ERR_TIMEOUT: return "SK_ERR_TIMEOUT";
    case SK_ERR_CUDA: return "SK_ERR_CUDA";
    case SK_ERR_OVERFLOW: return "SK_ERR_OVERFLOW";
    case SK_ERR_INEXACT: return "SK_ERR_INEXACT";
    case SK_ERR_NO_MEMORY: return "SK_ERR_NO_MEMORY";
    case SK_ERR_SCRATCH_TOO_SMALL: return "SK_ERR_SCRATCH_TOO_SMALL";
    case SK_ERR_OVER_BUDGET: return "SK_ERR_OVER_BUDGET";
    default: return "SK_ERR_UNKNOWN";
  }
}

sk_status sk_sketch_bytes(const sk_query* query, int64_t m, int32_t d, size_t* bytes) {
  if (!bytes) return SK_ERR_INVALID_ARG;
  Canon c;
  sk_status st = canonicalize(query, &c);
  if (st != SK_OK) return st;
  if (m < 1 || m > (1ll << 30)) return SK_ERR_UNSUPPORTED_WIDTH;
  if (d < 1 || d > SK_MAX_ROWS) return SK_ERR_INVALID_ARG;
  *bytes = (size_t)c.r * (size_t)d * (size_t)m * sizeof(int64_t);
  return SK_OK;
}

sk_status sk_sketch_create(const sk_query* query, int64_t m, int32_t d, uint64_t seed, void* dev_counters,
                           size_t bytes, void* cuda_stream, sk_set** out) {
  if (!out || !dev_counters) return SK_ERR_INVALID_ARG;
  *out = nullptr;
  size_t need = 0;
  sk_status st = sk_sketch_bytes(query, m, d, &need);
  if (st != SK_OK) return st;
  if (bytes < need) return SK_ERR_BUFFER_TOO_SMALL;
  Canon c;
  canonicalize(query, &c);
  sk_set* s = new (std::nothrow) sk_set();
  if (!s) return SK_ERR_NO_MEMORY;
  s->r = c.r;
  s->m = m;
  s->d = d;
  s->seed = seed;
  s->num_join_attrs = c.num_join_attrs;
  s->offsets = c.offsets;
  s->rel_of = c.rel_of;
  s->comp_of = c.comp_of;
  s->edges = c.edges;
  s->gamma = c.gamma;
  s->incident = c.incident;
  s->n_comp = c.n_comp;
  s->coef_row_len = 2 * c.n_comp + 4 * (int)c.edges.size();
  s->counters = (int64_t*)dev_counters;
  s->counter_bytes = need;
  for (int k = 0; k < c.r; k++) s->rel_ctr.push_back(s->counters + (size_t)k * d * m);
  cudaGetDevice(&s->device);
  // Algorithm 1, SampleBinHashes / SampleSignHashes: per row, (b0, b1) for every
  // component, then (s0, s1, s2, s3) for every join, in canonical order.
  s->h_coef = draw_coefficients(seed, d, s->coef_row_len);
  cudaError_t e = cudaMalloc(&s->d_status, sizeof(int));
  if (e != cudaSuccess) {
    free_set(s);
    return set_status_from_cuda(e);
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  e = cudaMemsetAsync(s->d_status, 0, sizeof(int), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_counters, 0, need, stream);
  if (e != cudaSuccess) {
    free_set(s);
    return set_status_from_cuda(e);
  }
  st = upload_relation_plans(s);
  if (st != SK_OK) {
    free_set(s);
    return st;
  }
  build_plan(s);
  // Default: the fused arithmetic (exact by construction: CRT primes, or Algorithm 3's steps
  // modulo them; GF(q) steps beyond nine primes).  SK_ESTIMATOR picks another at creation.
  s->estimator = SK_ESTIMATOR_FUSED;
  const char* ev = std::getenv("SK_ESTIMATOR");
  if (ev && std::strcmp(ev, "ntt") == 0) s->estimator = SK_ESTIMATOR_NTT;
  if (ev && std::strcmp(ev, "fft64") == 0) s->estimator = SK_ESTIMATOR_FFT64;
  *out = s;
  return SK_OK;
}

sk_status sk_sketch_update_batch(sk_set* set, int32_t relation, int64_t n_rows, const int64_t* dev_cols,
                                 int64_t col_stride, const int64_t* dev_weights, const int64_t* domain_hint,
                                 void* cuda_stream) {
  if (!set || relation < 0 || relation >= set->r || n_rows < 0) return SK_ERR_INVALID_ARG;
  if (n_rows == 0) return SK_OK;
  if (!dev_cols || col_stride < n_rows) return SK_ERR_INVALID_ARG;
  return launch_update(set, relation, n_rows, dev_cols, col_stride, dev_weights, domain_hint,
                       (cudaStream_t)cuda_stream);
}

sk_status sk_sketch_merge(sk_set* dst, const sk_set* src, void* cuda_stream) {
  if (!dst || !src) return SK_ERR_INVALID_ARG;
  if (dst->r != src->r || dst->m != src->m || dst->d != src->d || dst->seed != src->seed ||
      dst->num_join_attrs != src->num_join_attrs || dst->edges != src->edges || dst->h_coef != src->h_coef)
    return SK_ERR_MISMATCH;
  if (dst == src || dst->counters == src->counters) return SK_ERR_INVALID_ARG;
  return launch_merge(dst->counters, src->counters, (int64_t)(dst->counter_bytes / sizeof(int64_t)),
                      (cudaStream_t)cuda_stream);
}

sk_status sk_estimate_join(sk_set* set, sk_estimate* out, void* cuda_stream) {
  if (!set || !out) return SK_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  const bool pow2 = (set->m & (set->m - 1)) == 0;
  if (set->m < 2 || set->m > (pow2 ? (1ll << 22) : (1ll << 21))) return SK_ERR_UNSUPPORTED_WIDTH;
  return run_estimate(set, out, (cudaStream_t)cuda_stream);
}

sk_status sk_estimate_many(sk_set* const* sets, int32_t n, sk_estimate* out, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!sets || !out))) return SK_ERR_INVALID_ARG;
  std::vector<sk_set*> v(n);
  for (int i = 0; i < n; i++) {
    sk_set* s = sets[i];
    if (!s) return SK_ERR_INVALID_ARG;
    const bool pow2 = (s->m & (s->m - 1)) == 0;
    if (s->m < 2 || s->m > (pow2 ? (1ll << 22) : (1ll << 21))) return SK_ERR_UNSUPPORTED_WIDTH;
    for (int j = 0; j < i; j++)
      if (v[j] == s) return SK_ERR_INVALID_ARG;   // a set once per call (it owns one scratch)
    v[i] = s;
  }
  if (n == 0) return SK_OK;
  std::memset(out, 0, sizeof(sk_estimate) * n);
  return run_estimate_many(v.data(), n, out, (cudaStream_t)cuda_stream);
}

sk_status sk_estimate_join_noalloc(sk_set* set, sk_estimate* out, void* cuda_stream) {
  if (!set || !out) return SK_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (set->m < 2 || set->m > (1ll << 22) || (set->m & (set->m - 1))) return SK_ERR_UNSUPPORTED_WIDTH;
  return run_estimate_noalloc(set, out, (cudaStream_t)cuda_stream);
}

sk_status sk_sketch_set_estimator(sk_set* set, int32_t estimator) {
  if (!set || estimator < SK_ESTIMATOR_FFT64 || estimator > SK_ESTIMATOR_FUSED) return SK_ERR_INVALID_ARG;
  set->estimator = estimator;
  return SK_OK;
}

sk_status sk_sketch_reset(sk_set* set, void* cuda_stream) {
  if (!set) return SK_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemsetAsync(set->counters, 0, set->counter_bytes, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(set->d_status, 0, sizeof(int), stream);
  return set_status_from_cuda(e);
}

int64_t sk_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

sk_status sk_sync(sk_set* set, void* cuda_stream) {
  if (!set) return SK_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, set->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  if (h != 0) {
    e = cudaMemsetAsync(set->d_status, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return set_status_from_cuda(e);
  }
  return (sk_status)h;
}

sk_status sk_sketch_destroy(sk_set* set) {
  if (!set) return SK_OK;
  free_set(set);
  return SK_OK;
}

sk_status sk_sketch_info(const sk_set* set, int32_t* r, int64_t* m, int32_t* d, int32_t* n_components,
                         int32_t* n_joins) {
  if (!set) return SK_ERR_INVALID_ARG;
  if (r) *r = set->r;
  if (m) *m = set->m;
  if (d) *d = set->d;
  if (n_components) *n_components = set->n_comp;
  if (n_joins) *n_joins = (int32_t)set->edges.size();
  return SK_OK;
}

sk_status sk_get_coefficients(const sk_set* set, uint64_t* host_out, size_t count) {
  if (!set || !host_out || count < set->h_coef.size()) return SK_ERR_INVALID_ARG;
  std::memcpy(host_out, set->h_coef.data(), set->h_coef.size() * sizeof(uint64_t));
  return SK_OK;
}

sk_status sk_set_coefficients(sk_set* set, const uint64_t* host_coeffs, size_t count, void* cuda_stream) {
  if (!set || !host_coeffs || count != set->h_coef.size()) return SK_ERR_INVALID_ARG;
  for (size_t i = 0; i < count; i++)
    if (host_coeffs[i] >= kP61) return SK_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  std::memcpy(set->h_coef.data(), host_coeffs, count * sizeof(uint64_t));
  return upload_relation_plans(set);
}

}  // extern "C"
