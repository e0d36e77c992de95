// Batched update: one persistent launch applies many update batches (items), each
// an Algorithm 2 pass over one relation of one sketch set.  CTAs pull chunks of
// tuples from a device work counter in item order; a CTA reloads an item's hash
// coefficients and arguments into shared memory only when it moves to another item.  Items with
// a small d x m accumulate each chunk in an int32 shared-memory sub-sketch that is
// flushed into the int64 counters at the end of the chunk; items up to twice as large
// can use 16-bit counters packed two per word instead (see sk_update_plan_config).
#include <dlfcn.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sk_hash.cuh"
#include "sk_internal.h"

namespace sk {
namespace {

using namespace dev;

constexpr int kMaxMultiAttrs = 5;   // joined attributes per relation in a batched plan

struct MultiItem {
  UpdArgs args;
  int64_t chunk0;   // first global chunk of this item
  int pow2;
  int use_smem;     // 0 global counters, 1 int32 shared sub-sketch, 2 packed 16-bit one
  int deg1;         // every attribute in exactly one join
};

template <int A, bool POW2, bool DEG1>
__device__ __forceinline__ void multi_chunk(const UpdArgs& p, int use_smem, const uint64_t* s_coef, int* s_sub,
                                            int64_t t0, int64_t t1) {
  if (use_smem == 1) {
    const int64_t dm = (int64_t)p.d * (int64_t)p.m;
    for (int64_t j = threadIdx.x; j < dm; j += blockDim.x) s_sub[j] = 0;
    __syncthreads();
    for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x)
      update_tuple<A, POW2, true, false, DEG1>(p, s_coef, s_sub, i);
    __syncthreads();
    for (int64_t j = threadIdx.x; j < dm; j += blockDim.x) {
      const int v = s_sub[j];
      if (v != 0) red_add_global(p.ctr + j, (unsigned long long)(int64_t)v);
    }
  } else if (use_smem == 2) {
    // 16-bit counters biased by 2^15, two per word (counter j in half j & 1 of word j / 2)
    const int64_t dm = (int64_t)p.d * (int64_t)p.m, words = (dm + 1) >> 1;
    unsigned int* w = (unsigned int*)s_sub;
    for (int64_t k = threadIdx.x; k < words; k += blockDim.x) w[k] = 0x80008000u;
    __syncthreads();
    for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x)
      update_tuple<A, POW2, true, false, DEG1>(p, s_coef, s_sub, i);
    __syncthreads();
    for (int64_t k = threadIdx.x; k < words; k += blockDim.x) {
      const unsigned int x = w[k];
      const int lo = (int)(x & 0xffffu) - 32768, hi = (int)(x >> 16) - 32768;
      if (lo != 0) red_add_global(p.ctr + 2 * k, (unsigned long long)(int64_t)lo);
      if (hi != 0 && 2 * k + 1 < dm) red_add_global(p.ctr + 2 * k + 1, (unsigned long long)(int64_t)hi);
    }
  } else {
    for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x)
      update_tuple<A, POW2, false, false, DEG1>(p, s_coef, s_sub, i);
  }
}

template <bool POW2, bool DEG1>
__device__ __forceinline__ void multi_dispatch(const UpdArgs& p, int use_smem, const uint64_t* s_coef, int* s_sub,
                                               int64_t t0, int64_t t1) {
  switch (p.a) {
    case 1: multi_chunk<1, POW2, DEG1>(p, use_smem, s_coef, s_sub, t0, t1); break;
    case 2: multi_chunk<2, POW2, DEG1>(p, use_smem, s_coef, s_sub, t0, t1); break;
    case 3: multi_chunk<3, POW2, DEG1>(p, use_smem, s_coef, s_sub, t0, t1); break;
    case 4: multi_chunk<4, POW2, DEG1>(p, use_smem, s_coef, s_sub, t0, t1); break;
    default: multi_chunk<5, POW2, DEG1>(p, use_smem, s_coef, s_sub, t0, t1); break;
  }
}

__global__ void __launch_bounds__(256, 4) k_update_multi(const MultiItem* __restrict__ items, int n_items, int64_t total_chunks,
                               int64_t chunk, int coef_words, unsigned long long* queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_c;
  __shared__ int s_item;
  // the current item's arguments: read in the tuple loop from shared memory rather than
  // from the item array (global memory the counter updates could alias)
  __shared__ UpdArgs s_args;
  __shared__ int s_pow2, s_smem, s_deg1;
  uint64_t* s_coef = (uint64_t*)smem_raw;
  int* s_sub = (int*)(s_coef + coef_words);
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t c = (int64_t)atomicAdd(queue, 1ull);
      s_c = c;
      if (c < total_chunks) {
        int lo = 0, hi = n_items - 1;   // last item with chunk0 <= c
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].chunk0 <= c) lo = mid; else hi = mid - 1;
        }
        s_item = lo;
      }
    }
    __syncthreads();
    const int64_t c = s_c;
    if (c >= total_chunks) break;
    const int it = s_item;
    if (it != cur) {
      const MultiItem& mi = items[it];
      if (threadIdx.x == 0) {
        s_args = mi.args;
        s_pow2 = mi.pow2;
        s_smem = mi.use_smem;
        s_deg1 = mi.deg1;
      }
      const int nc = mi.args.d * mi.args.row_len;
      for (int j = threadIdx.x; j < nc; j += blockDim.x) s_coef[j] = mi.args.coef[j];
      cur = it;
      __syncthreads();
    }
    const UpdArgs& p = s_args;
    const int64_t t0 = (c - items[it].chunk0) * chunk;
    const int64_t t1 = min(p.n, t0 + chunk);
    if (s_pow2) {
      if (s_deg1) multi_dispatch<true, true>(p, s_smem, s_coef, s_sub, t0, t1);
      else multi_dispatch<true, false>(p, s_smem, s_coef, s_sub, t0, t1);
    } else {
      if (s_deg1) multi_dispatch<false, true>(p, s_smem, s_coef, s_sub, t0, t1);
      else multi_dispatch<false, false>(p, s_smem, s_coef, s_sub, t0, t1);
    }
    __syncthreads();
  }
}

// Zeroes the counter block of every item (d x m int64 words each; an item repeated for
// several batches of one relation is zeroed more than once, harmlessly).  Grid row y takes
// items y, y + gridDim.y, ...; its blocks stride over the item's words with 16-byte stores
// (a block starting at an odd word, as a later relation's block with d m odd does, first
// clears that word on its own).
__global__ void k_zero_multi(const MultiItem* __restrict__ items, int n_items) {
  for (int it = blockIdx.y; it < n_items; it += gridDim.y) {
    unsigned long long* c = items[it].args.ctr;
    const int64_t words = (int64_t)items[it].args.d * (int64_t)items[it].args.m;
    const int head = ((uintptr_t)c & 15u) ? 1 : 0;   // counters are 8-byte aligned
    if (head && words > 0 && blockIdx.x == 0 && threadIdx.x == 0) c[0] = 0ull;
    const int64_t rest = words - head;
    ulonglong2* v = (ulonglong2*)(c + head);
    const int64_t pairs = rest > 0 ? rest >> 1 : 0;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < pairs; j += step)
      v[j] = make_ulonglong2(0ull, 0ull);
    if (rest > 0 && (rest & 1) && blockIdx.x == 0 && threadIdx.x == 0) c[head + rest - 1] = 0ull;
  }
}

int sms() {
  static const int n = [] {   // thread-safe one-time initialisation
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, dev);
    return x > 0 ? x : 1;
  }();
  return n;
}

}  // namespace

size_t multi_item_size() { return sizeof(MultiItem); }

sk_status multi_describe(const sk_update_item* items, int n, const sk_update_plan_config& cfg, void* desc,
                         int64_t* total_chunks, int* coef_words_out, size_t* smem_bytes) {
  MultiItem* out = (MultiItem*)desc;
  int64_t chunk0 = 0;
  int coef_words = 0;
  int64_t sub_words = 0;
  for (int i = 0; i < n; i++) {
    const sk_update_item& it = items[i];
    sk_set* s = it.set;
    const RelPlan& rp = s->rel[it.relation];
    MultiItem mi;
    std::memset(&mi, 0, sizeof(mi));
    UpdArgs& a = mi.args;
    a.cols = it.dev_cols;
    a.stride = it.col_stride;
    a.w = it.dev_weights;
    a.n = it.n_rows;
    a.ctr = (unsigned long long*)(s->counters + (size_t)it.relation * s->d * s->m);
    a.coef = rp.d_coef;
    a.row_len = rp.coef_row_len;
    a.d = s->d;
    a.a = rp.a;
    for (int t = 0; t < kMaxAttrs; t++) a.deg[t] = rp.deg[t];
    a.m = (uint64_t)s->m;
    a.mrec = ~0ull / a.m;
    a.has_dom = 0;
    a.status = s->d_status;
    a.agg = 0;
    mi.pow2 = (s->m & (s->m - 1)) == 0;
    mi.deg1 = 1;
    for (int t = 0; t < rp.a; t++)
      if (rp.deg[t] != 1) mi.deg1 = 0;
    const int64_t dm = (int64_t)s->d * s->m;
    // the sub-sketch must also fit in shared memory next to the coefficients
    const bool fits32 = cfg.smem_max_counters > 0 && dm <= cfg.smem_max_counters && dm * 4 <= 160 * 1024;
    const bool fits16 = !fits32 && cfg.smem16_max_counters > 0 && dm <= cfg.smem16_max_counters &&
                        dm * 2 <= 160 * 1024;
    mi.use_smem = fits32 ? 1 : (fits16 ? 2 : 0);
    a.s16 = mi.use_smem == 2 ? 1 : 0;
    // |Delta| below which a tuple goes to the sub-sketch: a chunk's sum per counter then
    // stays within int32 (1) or within +-32767 (2, the 16-bit halves never carry)
    a.smem_wmax = (int64_t)(mi.use_smem == 2 ? 0x7fff : 0x7fffffff) / std::max<int64_t>(cfg.chunk_tuples, 1);
    mi.chunk0 = chunk0;
    chunk0 += (it.n_rows + cfg.chunk_tuples - 1) / cfg.chunk_tuples;
    coef_words = std::max(coef_words, s->d * rp.coef_row_len);
    if (mi.use_smem) sub_words = std::max(sub_words, mi.use_smem == 1 ? dm : (dm + 1) / 2);
    out[i] = mi;
  }
  *total_chunks = chunk0;
  *coef_words_out = (coef_words + 1) & ~1;
  *smem_bytes = (size_t)(*coef_words_out) * 8 + (size_t)sub_words * 4;
  return *smem_bytes > 200 * 1024 ? SK_ERR_INVALID_ARG : SK_OK;
}

sk_status multi_launch(const void* d_desc, int n, int64_t total_chunks, const sk_update_plan_config& cfg,
                       int coef_words, size_t smem_bytes, unsigned long long* d_queue, cudaStream_t st,
                       bool zero_queue) {
  if (total_chunks == 0) return SK_OK;
  cudaError_t e = zero_queue ? cudaMemsetAsync(d_queue, 0, sizeof(unsigned long long), st) : cudaSuccess;
  if (e != cudaSuccess) return set_status_from_cuda(e);
  e = allow_dynamic_smem((const void*)k_update_multi);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(total_chunks, (int64_t)sms() * cfg.ctas_per_sm));
  k_update_multi<<<grid, cfg.threads, smem_bytes, st>>>((const MultiItem*)d_desc, n, total_chunks, cfg.chunk_tuples,
                                                        coef_words, d_queue);
  count_launch();
  return set_status_from_cuda(cudaGetLastError());
}

}  // namespace sk

using namespace sk;

struct sk_update_plan {
  std::vector<sk_update_item> items;
  std::vector<MultiItem> host;
  sk_update_plan_config cfg{};
  MultiItem* d_items = nullptr;
  unsigned long long* d_queue = nullptr;
  int n_active = 0;
  int64_t total_chunks = 0;
  int coef_words = 0;
  size_t smem_bytes = 0;
};

namespace {

sk_status plan_build(sk_update_plan* pl) {
  pl->host.clear();
  std::vector<sk_update_item> active;
  for (const sk_update_item& it : pl->items)
    if (it.n_rows > 0) active.push_back(it);
  pl->host.resize(active.size());
  sk_status st = multi_describe(active.data(), (int)active.size(), pl->cfg, pl->host.data(), &pl->total_chunks,
                                &pl->coef_words, &pl->smem_bytes);
  if (st != SK_OK) return st;
  pl->n_active = (int)active.size();
  if (pl->d_items) {
    cudaFree(pl->d_items);
    pl->d_items = nullptr;
  }
  if (pl->n_active > 0) {
    cudaError_t e = cudaMalloc(&pl->d_items, sizeof(MultiItem) * pl->n_active);
    if (e != cudaSuccess) return set_status_from_cuda(e);
    e = cudaMemcpy(pl->d_items, pl->host.data(), sizeof(MultiItem) * pl->n_active, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_status_from_cuda(e);
  }
  return SK_OK;
}

// ---------------------------------------------------------------------------
// Persistent autotuning choices.  A plan's key is the device's SM count and the sorted
// shapes of its items ((m, d, attributes) with their counts, and the log2 of its tuple
// count); sk_update_plan_autotune looks the key up in a JSON-lines file (one object per line:
// key, chunk_tuples, threads, ctas_per_sm, smem_max_counters, smem16_max_counters, ms) and
// times its configuration grid only on a miss, appending the winner.  File:
// SK_AUTOTUNE_CACHE, else autotune.json beside libsketch.so; SK_AUTOTUNE_CACHE=off disables it.
// ---------------------------------------------------------------------------
std::string tune_key(const sk_update_plan* pl) {
  std::map<std::tuple<int64_t, int, int>, int> shapes;
  int64_t tuples = 0;
  for (const sk_update_item& it : pl->items) {
    if (it.n_rows == 0) continue;
    shapes[std::make_tuple(it.set->m, it.set->d, it.set->rel[it.relation].a)]++;
    tuples += it.n_rows;
  }
  int lg = 0;
  while (lg < 62 && ((int64_t)1 << (lg + 1)) <= tuples) lg++;
  std::string k = "sms=" + std::to_string(sms()) + ";tuples=2^" + std::to_string(lg) + ";";
  for (const auto& kv : shapes)
    k += "m" + std::to_string(std::get<0>(kv.first)) + ".d" + std::to_string(std::get<1>(kv.first)) + ".a" +
         std::to_string(std::get<2>(kv.first)) + "x" + std::to_string(kv.second) + ",";
  return k;
}

std::string tune_cache_path() {
  const char* v = std::getenv("SK_AUTOTUNE_CACHE");
  if (v && std::strcmp(v, "off") == 0) return std::string();
  if (v && v[0]) return std::string(v);
  Dl_info info;
  if (dladdr((const void*)&tune_cache_path, &info) && info.dli_fname) {
    std::string lib(info.dli_fname);
    const size_t slash = lib.rfind('/');
    if (slash != std::string::npos) return lib.substr(0, slash + 1) + "autotune.json";
  }
  return std::string();
}

std::mutex g_tune_mu;

bool tune_cache_find(const std::string& path, const std::string& key, sk_update_plan_config* cfg, double* ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return false;
  char line[4096];
  bool found = false;
  const std::string want = "{\"key\": \"" + key + "\", ";
  while (std::fgets(line, sizeof(line), f)) {
    if (std::strncmp(line, want.c_str(), want.size()) != 0) continue;
    sk_update_plan_config c{};
    double t = 0.0;
    if (std::sscanf(line + want.size(),
                    "\"chunk_tuples\": %d, \"threads\": %d, \"ctas_per_sm\": %d, \"smem_max_counters\": %d, "
                    "\"smem16_max_counters\": %d, \"ms\": %lf",
                    &c.chunk_tuples, &c.threads, &c.ctas_per_sm, &c.smem_max_counters, &c.smem16_max_counters, &t) == 6) {
      *cfg = c;   // the last matching line wins
      *ms = t;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void tune_cache_store(const std::string& path, const std::string& key, const sk_update_plan_config& c, double ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;   // read-only location: tuning still applies to this plan
  std::fprintf(f,
               "{\"key\": \"%s\", \"chunk_tuples\": %d, \"threads\": %d, \"ctas_per_sm\": %d, "
               "\"smem_max_counters\": %d, \"smem16_max_counters\": %d, \"ms\": %.6f}\n",
               key.c_str(), c.chunk_tuples, c.threads, c.ctas_per_sm, c.smem_max_counters, c.smem16_max_counters, ms);
  std::fclose(f);
}

}  // namespace

extern "C" {

sk_status sk_update_plan_create(const sk_update_item* items, int32_t n_items, sk_update_plan** out) {
  if (!out || n_items < 0 || (n_items > 0 && !items)) return SK_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n_items; i++) {
    const sk_update_item& it = items[i];
    if (!it.set || it.relation < 0 || it.relation >= it.set->r || it.n_rows < 0) return SK_ERR_INVALID_ARG;
    if (it.n_rows > 0 && (!it.dev_cols || it.col_stride < it.n_rows)) return SK_ERR_INVALID_ARG;
    if (it.set->rel[it.relation].a > kMaxMultiAttrs) return SK_ERR_INVALID_ARG;
  }
  sk_update_plan* pl = new (std::nothrow) sk_update_plan();
  if (!pl) return SK_ERR_NO_MEMORY;
  pl->items.assign(items, items + n_items);
  pl->cfg.chunk_tuples = 32768;
  pl->cfg.threads = 256;
  pl->cfg.ctas_per_sm = 6;
  pl->cfg.smem_max_counters = 16384;
  cudaError_t e = cudaMalloc(&pl->d_queue, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    delete pl;
    return set_status_from_cuda(e);
  }
  sk_status st = plan_build(pl);
  if (st != SK_OK) {
    sk_update_plan_destroy(pl);
    return st;
  }
  *out = pl;
  return SK_OK;
}

sk_status sk_update_plan_run(sk_update_plan* pl, void* cuda_stream) {
  if (!pl) return SK_ERR_INVALID_ARG;
  return multi_launch(pl->d_items, pl->n_active, pl->total_chunks, pl->cfg, pl->coef_words, pl->smem_bytes,
                      pl->d_queue, (cudaStream_t)cuda_stream, true);
}

sk_status sk_update_plan_zero(sk_update_plan* pl, void* cuda_stream) {
  if (!pl) return SK_ERR_INVALID_ARG;
  if (pl->n_active == 0) return SK_OK;
  const dim3 grid(8, (unsigned)std::min(pl->n_active, 65535));
  k_zero_multi<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(pl->d_items, pl->n_active);
  count_launch();
  return set_status_from_cuda(cudaGetLastError());
}

sk_status sk_update_plan_get_config(const sk_update_plan* pl, sk_update_plan_config* out) {
  if (!pl || !out) return SK_ERR_INVALID_ARG;
  *out = pl->cfg;
  return SK_OK;
}

sk_status sk_update_plan_set_config(sk_update_plan* pl, const sk_update_plan_config* c) {
  if (!pl || !c) return SK_ERR_INVALID_ARG;
  if (c->chunk_tuples < 256 || c->threads < 32 || c->threads > 256 || (c->threads & 31) || c->ctas_per_sm < 1 ||
      c->ctas_per_sm > 32 || c->smem_max_counters < 0 || c->smem16_max_counters < 0)
    return SK_ERR_INVALID_ARG;
  const sk_update_plan_config old = pl->cfg;
  pl->cfg = *c;
  sk_status st = plan_build(pl);
  if (st != SK_OK) {
    pl->cfg = old;
    plan_build(pl);
  }
  return st;
}

sk_status sk_update_plan_autotune(sk_update_plan* pl, void* cuda_stream, sk_update_plan_config* best,
                                  double* best_ms) {
  if (!pl) return SK_ERR_INVALID_ARG;
  const std::string key = tune_key(pl);
  const std::string path = tune_cache_path();
  sk_update_plan_config cached;
  double cached_ms = 0.0;
  if (!path.empty() && tune_cache_find(path, key, &cached, &cached_ms) && sk_update_plan_set_config(pl, &cached) == SK_OK) {
    if (best) *best = cached;
    if (best_ms) *best_ms = cached_ms;
    return SK_OK;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int chunks[] = {8192, 32768, 131072};
  const int ctas[] = {4, 8};
  const int smem[] = {0, 8192, 32768};
  const int smem16[] = {0, 32768};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SK_ERR_CUDA;
  sk_update_plan_config bestc = pl->cfg;
  float bestt = 1e30f;
  sk_status rs = SK_OK;
  for (int ch : chunks)
    for (int ct : ctas)
      for (int sm : smem)
        for (int s16 : smem16) {
          if (s16 && s16 <= sm) continue;   // nothing would use the 16-bit sub-sketch
          sk_update_plan_config c{ch, 256, ct, sm, s16};
          if (sk_update_plan_set_config(pl, &c) != SK_OK) continue;
          if ((rs = sk_update_plan_run(pl, st)) != SK_OK) break;   // warm-up
          float total = 0.f;
          for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, st);
            if ((rs = sk_update_plan_run(pl, st)) != SK_OK) break;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
          }
          if (rs != SK_OK) break;
          if (total / 3 < bestt) {
            bestt = total / 3;
            bestc = c;
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != SK_OK) return rs;
  sk_status s2 = sk_update_plan_set_config(pl, &bestc);
  if (best) *best = bestc;
  if (best_ms) *best_ms = bestt;
  if (s2 == SK_OK && !path.empty()) tune_cache_store(path, key, bestc, bestt);
  return s2;
}

sk_status sk_update_plan_destroy(sk_update_plan* pl) {
  if (!pl) return SK_OK;
  if (pl->d_items) cudaFree(pl->d_items);
  if (pl->d_queue) cudaFree(pl->d_queue);
  delete pl;
  return SK_OK;
}

}  // extern "C"
