// Sub-query families (Section 3.4): the sketches of many sub-queries of one query Q,
// built in one pass per relation, with one sketch per distinct view of a relation.
//
// Hash functions.  Q's functions are drawn as for a plain set.  A sub-query S inherits
// them: a component of S takes the bin function of the component of Q containing it; a
// component of S with one join takes the sign function of the first join of its Q
// component; a component with several joins takes each join's own sign function.  Q's
// relations form a tree, so a connected S has at most one component inside any component
// of Q and the functions of different joins of S stay independent (Theorem 3.1 holds).
//
// Views.  For relation R_k in S, every attribute u that S joins is hashed with its
// component's bin function and with a set F_u of sign functions (its S-joins, or its Q
// component's first join).  The view {(u, F_u)} determines R_k's sketch for S, so
// sub-queries with the same view share it.  Per relation, the sign functions any view
// uses are numbered as "slots": for attribute t, its Q joins (canonical order), then its
// component's first join if that join is not one of them.
//
// Update.  k_update_views hashes a tuple once per row (per attribute: the bin value and
// one parity bit per slot) and adds it to every view: bin = sum of the view's attribute
// bins mod m, sign = parity of the view's slot bits.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <thread>

#include "sk_hash.cuh"
#include "sk_internal.h"

namespace sk {
namespace {

using namespace dev;

struct ViewArgs {
  int nv;
  uint32_t amask[SK_MAX_VIEWS];            // attributes of the relation the view joins
  unsigned long long jmask[SK_MAX_VIEWS];  // sign slots the view multiplies
  unsigned long long* ctr[SK_MAX_VIEWS];   // the view's [d][m] counters
};

// Per row, attribute t's bin (mod 2^32 for power-of-two m, else mod m) and its slot
// parities; cr points at t's coefficients in the row: (b0, b1), then (s0..s3) per slot.
template <bool POW2>
__device__ __forceinline__ uint32_t attr_row(const UpdArgs& p, const uint64_t* cr, int nsl, uint64_t x, bool narrow,
                                             int slot0, unsigned long long* pbits) {
  uint32_t h;
  if (narrow) {
    const uint32_t x32 = (uint32_t)x;
    const uint64_t v = mac_narrow(cr[1], x32, cr[0]);
    h = POW2 ? (uint32_t)v + mersenne_q1(v) : (uint32_t)mod_m(reduce_lazy(v), p.m, p.mrec);
    for (int e = 0; e < nsl; e++) {
      const uint64_t* sc = cr + 2 + 4 * e;
      uint64_t acc = mac_narrow(sc[3], x32, sc[2]);
      acc = mac_narrow(acc, x32, sc[1]);
      acc = mac_narrow(acc, x32, sc[0]);
      *pbits |= (unsigned long long)(((uint32_t)acc ^ mersenne_q1(acc)) & 1u) << (slot0 + e);
    }
  } else {
    const uint64_t hv = addmod(mulmod(cr[1], x), cr[0]);
    h = POW2 ? (uint32_t)hv : (uint32_t)mod_m(hv, p.m, p.mrec);
    for (int e = 0; e < nsl; e++) {
      const uint64_t* sc = cr + 2 + 4 * e;
      uint64_t acc = sc[3];
      acc = addmod(mulmod(acc, x), sc[2]);
      acc = addmod(mulmod(acc, x), sc[1]);
      acc = addmod(mulmod(acc, x), sc[0]);
      *pbits |= (unsigned long long)(acc & 1u) << (slot0 + e);
    }
  }
  return h;
}

// p.deg[t] = slots of attribute t; p.coef = the relation's family table [d][row_len].
template <int A, bool POW2>
__global__ void __launch_bounds__(256) k_update_views(UpdArgs p, ViewArgs v) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* s_coef = (uint64_t*)smem_raw;
  const int ncoef = p.d * p.row_len;
  for (int i = threadIdx.x; i < ncoef; i += blockDim.x) s_coef[i] = p.coef[i];
  __syncthreads();
  constexpr int AM = A > 0 ? A : kMaxAttrs;
  const int na = A > 0 ? A : p.a;
  const uint32_t m32 = (uint32_t)p.m;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += step) {
    uint64_t x[AM];
    bool ok = true, narrow = true;
#pragma unroll
    for (int t = 0; t < AM; t++) {
      if (A == 0 && t >= na) break;
      const int64_t key = __ldg(p.cols + (int64_t)t * p.stride + i);
      if (p.has_dom && (key < 0 || key >= p.dom[t])) ok = false;
      x[t] = field_of(key);
      narrow = narrow && (x[t] >> 32) == 0;
    }
    if (!ok) {
      record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
      continue;
    }
    const int64_t delta = p.w ? __ldg(p.w + i) : 1;
    const uint64_t* cr = s_coef;
    for (int row = 0; row < p.d; row++, cr += p.row_len) {
      uint32_t h[AM];
      unsigned long long bits = 0;
      int off = 0, slot = 0;
#pragma unroll
      for (int t = 0; t < AM; t++) {
        if (A == 0 && t >= na) break;
        h[t] = attr_row<POW2>(p, cr + off, p.deg[t], x[t], narrow, slot, &bits);
        off += 2 + 4 * p.deg[t];
        slot += p.deg[t];
      }
      for (int vi = 0; vi < v.nv; vi++) {
        const uint32_t am = v.amask[vi];
        uint32_t b = 0;
#pragma unroll
        for (int t = 0; t < AM; t++) {
          if (A == 0 && t >= na) break;
          if ((am >> t) & 1u) {
            b += h[t];
            if (!POW2 && b >= m32) b -= m32;
          }
        }
        const uint32_t bin = POW2 ? (b & (m32 - 1)) : b;
        const int64_t val = (__popcll(bits & v.jmask[vi]) & 1) ? -delta : delta;
        red_add_global(v.ctr[vi] + (int64_t)row * p.m + bin, (unsigned long long)val);
      }
    }
  }
}

template <int A, bool POW2>
cudaError_t launch_views(const UpdArgs& a, const ViewArgs& v, size_t smem, cudaStream_t st) {
  auto kern = k_update_views<A, POW2>;
  cudaError_t e = fit_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>((a.n + 255) / 256, 0x7fffffff);
  kern<<<(int)grid, 256, smem, st>>>(a, v);
  count_launch();
  return cudaGetLastError();
}

template <bool POW2>
cudaError_t dispatch_views(const UpdArgs& a, const ViewArgs& v, size_t smem, cudaStream_t st) {
  switch (a.a) {
    case 1: return launch_views<1, POW2>(a, v, smem, st);
    case 2: return launch_views<2, POW2>(a, v, smem, st);
    case 3: return launch_views<3, POW2>(a, v, smem, st);
    case 4: return launch_views<4, POW2>(a, v, smem, st);
    default: return launch_views<0, POW2>(a, v, smem, st);
  }
}

// One relation of Q inside the family.
struct FamRel {
  int a = 0;
  std::vector<std::vector<int>> slot_join;   // per attribute: the Q join of each slot
  int row_len = 0;                           // sum over attributes of 2 + 4 slots
  uint64_t* d_coef = nullptr;                // [d][row_len]
  std::vector<uint32_t> amask;               // per view
  std::vector<unsigned long long> jmask;     // per view
  std::vector<int> view_id;                  // per view: index into the family's counters
};

// One sub-query: its relations (Q indices, ascending) and the view of each.
struct FamSub {
  std::vector<int> q_rel;
  std::vector<int> view;      // family-wide view index per S relation
  sk_set* est = nullptr;      // estimation set over the shared counters
};

int find_root(std::vector<int>& parent, int x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

int env_workers() {
  const char* v = std::getenv("SK_FAMILY_WORKERS");
  const int x = v ? std::atoi(v) : 4;
  return x < 1 ? 1 : (x > 16 ? 16 : x);
}

}  // namespace
}  // namespace sk

struct sk_family {
  int device = 0;
  int64_t m = 0;
  int d = 0;
  uint64_t seed = 0;
  sk::QueryInfo q;
  std::vector<uint64_t> h_coef;            // Q's functions [d][2 n_comp + 4 |E|]
  std::vector<sk::FamRel> rel;             // per relation of Q
  std::vector<sk::FamSub> sub;
  int n_views = 0;
  int64_t* d_counters = nullptr;           // [n_views][d][m]
  int* d_status = nullptr;
  std::vector<cudaStream_t> workers;
};

namespace sk {
namespace {

void free_family(sk_family* f) {
  if (!f) return;
  for (auto& s : f->sub)
    if (s.est) destroy_set(s.est);
  for (auto& r : f->rel)
    if (r.d_coef) cudaFree(r.d_coef);
  if (f->d_counters) cudaFree(f->d_counters);
  if (f->d_status) cudaFree(f->d_status);
  for (cudaStream_t w : f->workers) cudaStreamDestroy(w);
  delete f;
}

}  // namespace
}  // namespace sk

using namespace sk;

extern "C" {

sk_status sk_family_create(const sk_query* query, int32_t n_sub, const int32_t* sub_offsets,
                           const int32_t* sub_edges, int64_t m, int32_t d, uint64_t seed, void* cuda_stream,
                           sk_family** out) {
  if (!out) return SK_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_sub < 1 || !sub_offsets || !sub_edges || sub_offsets[0] != 0) return SK_ERR_INVALID_ARG;
  if (d < 1 || d > SK_MAX_ROWS) return SK_ERR_INVALID_ARG;
  const bool pow2 = m >= 1 && (m & (m - 1)) == 0;
  if (m < 2 || m > (pow2 ? (1ll << 22) : (1ll << 21))) return SK_ERR_UNSUPPORTED_WIDTH;
  QueryInfo q;
  sk_status st = query_info(query, &q);
  if (st != SK_OK) return st;
  const int nE = (int)q.edges.size();
  // the user's join i -> Q's canonical join index
  std::vector<int> canon_of(query->num_edges);
  for (int i = 0; i < query->num_edges; i++) {
    const sk_edge& e = query->edges[i];
    const int u = q.offsets[e.rel_a] + e.attr_a, v = q.offsets[e.rel_b] + e.attr_b;
    const std::pair<int, int> pr(std::min(u, v), std::max(u, v));
    canon_of[i] = (int)(std::lower_bound(q.edges.begin(), q.edges.end(), pr) - q.edges.begin());
  }
  // first join of every component of Q
  std::vector<int> first_join(q.n_comp, -1);
  for (int j = 0; j < nE; j++) {
    const int c = q.comp_of[q.edges[j].first];
    if (first_join[c] < 0) first_join[c] = j;
  }
  sk_family* f = new (std::nothrow) sk_family();
  if (!f) return SK_ERR_NO_MEMORY;
  cudaGetDevice(&f->device);
  f->m = m;
  f->d = d;
  f->seed = seed;
  f->q = q;
  f->h_coef = draw_coefficients(seed, d, 2 * q.n_comp + 4 * nE);
  f->rel.assign(q.r, FamRel());
  // slots of every attribute: its Q joins, then its component's first join
  for (int k = 0; k < q.r; k++) {
    FamRel& fr = f->rel[k];
    fr.a = q.num_join_attrs[k];
    fr.slot_join.assign(fr.a, {});
    int nslots = 0;
    for (int t = 0; t < fr.a; t++) {
      const int u = q.offsets[k] + t;
      fr.slot_join[t] = q.incident[u];
      const int fj = first_join[q.comp_of[u]];
      if (std::find(fr.slot_join[t].begin(), fr.slot_join[t].end(), fj) == fr.slot_join[t].end())
        fr.slot_join[t].push_back(fj);
      nslots += (int)fr.slot_join[t].size();
      fr.row_len += 2 + 4 * (int)fr.slot_join[t].size();
    }
    if (nslots > SK_MAX_SLOTS) {
      free_family(f);
      return SK_ERR_INVALID_ARG;
    }
  }
  // views and sub-queries
  std::vector<std::map<std::pair<uint32_t, unsigned long long>, int>> view_index(q.r);
  for (int si = 0; si < n_sub; si++) {
    const int b = sub_offsets[si], e = sub_offsets[si + 1];
    if (e <= b) {
      free_family(f);
      return SK_ERR_INVALID_ARG;
    }
    std::vector<int> joins;   // Q canonical indices
    for (int i = b; i < e; i++) {
      const int ui = sub_edges[i];
      if (ui < 0 || ui >= query->num_edges) {
        free_family(f);
        return SK_ERR_INVALID_ARG;
      }
      joins.push_back(canon_of[ui]);
    }
    std::sort(joins.begin(), joins.end());
    if (std::adjacent_find(joins.begin(), joins.end()) != joins.end()) {
      free_family(f);
      return SK_ERR_INVALID_ARG;
    }
    // relations and connectivity
    std::vector<int> parent(q.r);
    for (int k = 0; k < q.r; k++) parent[k] = k;
    std::vector<char> in_s(q.r, 0);
    for (int j : joins) {
      const int ra = q.rel_of[q.edges[j].first], rb = q.rel_of[q.edges[j].second];
      in_s[ra] = in_s[rb] = 1;
      parent[find_root(parent, ra)] = find_root(parent, rb);
    }
    FamSub fs;
    for (int k = 0; k < q.r; k++)
      if (in_s[k]) fs.q_rel.push_back(k);
    for (int k : fs.q_rel)
      if (find_root(parent, k) != find_root(parent, fs.q_rel[0])) {
        free_family(f);
        return SK_ERR_INVALID_ARG;
      }
    // components of S over Q attributes, and their join counts
    const int W = (int)q.rel_of.size();
    std::vector<int> ap(W);
    for (int u = 0; u < W; u++) ap[u] = u;
    for (int j : joins) ap[find_root(ap, q.edges[j].first)] = find_root(ap, q.edges[j].second);
    std::vector<int> comp_joins(W, 0);
    for (int j : joins) comp_joins[find_root(ap, q.edges[j].first)]++;
    std::vector<char> joined(W, 0);
    for (int j : joins) joined[q.edges[j].first] = joined[q.edges[j].second] = 1;
    // sign functions of every joined attribute
    auto sign_set = [&](int u) {
      std::vector<int> fu;
      if (comp_joins[find_root(ap, u)] == 1) {
        fu.push_back(first_join[q.comp_of[u]]);
      } else {
        for (int j : q.incident[u])
          if (std::binary_search(joins.begin(), joins.end(), j)) fu.push_back(j);
      }
      return fu;
    };
    // the view of each relation
    for (int k : fs.q_rel) {
      FamRel& fr = f->rel[k];
      uint32_t am = 0;
      unsigned long long jm = 0;
      int slot = 0;
      for (int t = 0; t < fr.a; t++) {
        const int u = q.offsets[k] + t;
        if (joined[u]) {
          am |= 1u << t;
          for (int j : sign_set(u)) {
            const auto it = std::find(fr.slot_join[t].begin(), fr.slot_join[t].end(), j);
            jm |= 1ull << (slot + (int)(it - fr.slot_join[t].begin()));
          }
        }
        slot += (int)fr.slot_join[t].size();
      }
      auto key = std::make_pair(am, jm);
      auto it = view_index[k].find(key);
      int vid;
      if (it == view_index[k].end()) {
        if ((int)fr.amask.size() >= SK_MAX_VIEWS) {
          free_family(f);
          return SK_ERR_INVALID_ARG;
        }
        vid = f->n_views++;
        view_index[k][key] = (int)fr.amask.size();
        fr.amask.push_back(am);
        fr.jmask.push_back(jm);
        fr.view_id.push_back(vid);
      } else {
        vid = fr.view_id[it->second];
      }
      fs.view.push_back(vid);
    }
    f->sub.push_back(fs);
  }
  // counters, status, coefficient tables
  const size_t vbytes = (size_t)d * (size_t)m * sizeof(int64_t);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  cudaError_t ce = cudaMalloc(&f->d_counters, vbytes * f->n_views);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(f->d_counters, 0, vbytes * f->n_views, stream);
  if (ce == cudaSuccess) ce = cudaMalloc(&f->d_status, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemsetAsync(f->d_status, 0, sizeof(int), stream);
  const int qrow = 2 * q.n_comp + 4 * nE;
  for (int k = 0; k < q.r && ce == cudaSuccess; k++) {
    FamRel& fr = f->rel[k];
    if (fr.amask.empty()) continue;
    std::vector<uint64_t> tab((size_t)d * fr.row_len);
    for (int row = 0; row < d; row++) {
      const uint64_t* cr = f->h_coef.data() + (size_t)row * qrow;
      uint64_t* o = tab.data() + (size_t)row * fr.row_len;
      for (int t = 0; t < fr.a; t++) {
        const int c = q.comp_of[q.offsets[k] + t];
        *o++ = cr[2 * c];
        *o++ = cr[2 * c + 1];
        for (int j : fr.slot_join[t])
          for (int z = 0; z < 4; z++) *o++ = cr[2 * q.n_comp + 4 * j + z];
      }
    }
    if ((size_t)d * fr.row_len * sizeof(uint64_t) > 200 * 1024) {
      free_family(f);
      return SK_ERR_INVALID_ARG;
    }
    ce = cudaMalloc(&fr.d_coef, tab.size() * sizeof(uint64_t));
    if (ce == cudaSuccess)
      ce = cudaMemcpy(fr.d_coef, tab.data(), tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
  }
  if (ce != cudaSuccess) {
    free_family(f);
    return set_status_from_cuda(ce);
  }
  // estimation sets: S's own canonical numbering over the shared view counters
  for (int si = 0; si < n_sub; si++) {
    FamSub& fs = f->sub[si];
    std::vector<int> joins;
    for (int i = sub_offsets[si]; i < sub_offsets[si + 1]; i++) joins.push_back(canon_of[sub_edges[i]]);
    std::sort(joins.begin(), joins.end());
    std::vector<char> joined(q.rel_of.size(), 0);
    for (int j : joins) joined[q.edges[j].first] = joined[q.edges[j].second] = 1;
    std::vector<int> pos(q.rel_of.size(), -1);   // Q attribute -> position in its S relation
    std::vector<int32_t> attrs;
    for (int k : fs.q_rel) {
      int a = 0;
      for (int t = 0; t < q.num_join_attrs[k]; t++)
        if (joined[q.offsets[k] + t]) pos[q.offsets[k] + t] = a++;
      attrs.push_back(a);
    }
    std::vector<int> rel_new(q.r, -1);
    for (int i = 0; i < (int)fs.q_rel.size(); i++) rel_new[fs.q_rel[i]] = i;
    std::vector<sk_edge> sedges;
    for (int j : joins) {
      const int u = q.edges[j].first, v = q.edges[j].second;
      sedges.push_back({rel_new[q.rel_of[u]], pos[u], rel_new[q.rel_of[v]], pos[v]});
    }
    sk_query sq{(int32_t)fs.q_rel.size(), attrs.data(), (int32_t)sedges.size(), sedges.data()};
    QueryInfo si_info;
    st = query_info(&sq, &si_info);
    if (st != SK_OK) {
      free_family(f);
      return SK_ERR_INVALID_ARG;
    }
    // S's functions in S's layout (kept for inspection; the estimate reads only counters)
    const int srow = 2 * si_info.n_comp + 4 * (int)si_info.edges.size();
    std::vector<int> q_attr_of;   // S global attribute -> Q attribute
    for (int k : fs.q_rel)
      for (int t = 0; t < q.num_join_attrs[k]; t++)
        if (joined[q.offsets[k] + t]) q_attr_of.push_back(q.offsets[k] + t);
    std::vector<int> sjoins_in_comp(si_info.n_comp, 0);
    for (auto& ed : si_info.edges) sjoins_in_comp[si_info.comp_of[ed.first]]++;
    std::vector<uint64_t> hs((size_t)d * srow);
    for (int row = 0; row < d; row++) {
      const uint64_t* cr = f->h_coef.data() + (size_t)row * qrow;
      uint64_t* o = hs.data() + (size_t)row * srow;
      for (int c = 0; c < si_info.n_comp; c++) {
        int us = 0;
        while (si_info.comp_of[us] != c) us++;
        const int cq = q.comp_of[q_attr_of[us]];
        o[2 * c] = cr[2 * cq];
        o[2 * c + 1] = cr[2 * cq + 1];
      }
      for (int j = 0; j < (int)si_info.edges.size(); j++) {
        const int u = q_attr_of[si_info.edges[j].first], v = q_attr_of[si_info.edges[j].second];
        int jq;
        if (sjoins_in_comp[si_info.comp_of[si_info.edges[j].first]] == 1) {
          jq = first_join[q.comp_of[u]];
        } else {
          const std::pair<int, int> pr(std::min(u, v), std::max(u, v));
          jq = (int)(std::lower_bound(q.edges.begin(), q.edges.end(), pr) - q.edges.begin());
        }
        for (int z = 0; z < 4; z++) o[2 * si_info.n_comp + 4 * j + z] = cr[2 * q.n_comp + 4 * jq + z];
      }
    }
    std::vector<int64_t*> rc;
    for (int vid : fs.view) rc.push_back(f->d_counters + (size_t)vid * d * m);
    st = make_estimation_set(si_info, m, d, seed, std::move(hs), std::move(rc), &fs.est);
    if (st != SK_OK) {
      free_family(f);
      return st;
    }
    const char* ev = std::getenv("SK_ESTIMATOR");
    if (ev && std::strcmp(ev, "ntt") == 0) fs.est->estimator = SK_ESTIMATOR_NTT;
    if (ev && std::strcmp(ev, "fft64") == 0) fs.est->estimator = SK_ESTIMATOR_FFT64;
  }
  const int nw = std::min(env_workers(), n_sub);
  for (int w = 0; w < nw; w++) {
    cudaStream_t s = nullptr;
    ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      free_family(f);
      return set_status_from_cuda(ce);
    }
    f->workers.push_back(s);
  }
  *out = f;
  return SK_OK;
}

sk_status sk_family_update_batch(sk_family* fam, int32_t relation, int64_t n_rows, const int64_t* dev_cols,
                                 int64_t col_stride, const int64_t* dev_weights, const int64_t* domain_hint,
                                 void* cuda_stream) {
  if (!fam || relation < 0 || relation >= fam->q.r || n_rows < 0) return SK_ERR_INVALID_ARG;
  if (n_rows == 0) return SK_OK;
  if (!dev_cols || col_stride < n_rows) return SK_ERR_INVALID_ARG;
  const FamRel& fr = fam->rel[relation];
  if (fr.amask.empty()) return SK_OK;
  UpdArgs a;
  a.cols = dev_cols;
  a.stride = col_stride;
  a.w = dev_weights;
  a.n = n_rows;
  a.ctr = nullptr;
  a.coef = fr.d_coef;
  a.row_len = fr.row_len;
  a.d = fam->d;
  a.a = fr.a;
  for (int t = 0; t < kMaxAttrs; t++) a.deg[t] = t < fr.a ? (int)fr.slot_join[t].size() : 0;
  a.m = (uint64_t)fam->m;
  a.mrec = ~0ull / a.m;
  a.has_dom = domain_hint != nullptr;
  for (int t = 0; t < kMaxAttrs; t++) a.dom[t] = (domain_hint && t < fr.a) ? domain_hint[t] : 0;
  a.status = fam->d_status;
  a.smem_wmax = 0;
  a.agg = 0;
  a.s16 = 0;
  ViewArgs v;
  v.nv = (int)fr.amask.size();
  for (int i = 0; i < v.nv; i++) {
    v.amask[i] = fr.amask[i];
    v.jmask[i] = fr.jmask[i];
    v.ctr[i] = (unsigned long long*)(fam->d_counters + (size_t)fr.view_id[i] * fam->d * fam->m);
  }
  const size_t smem = (size_t)fam->d * fr.row_len * sizeof(uint64_t);
  const bool pow2 = (fam->m & (fam->m - 1)) == 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (domain_hint && !dev_weights) {
    bool done = false;
    const sk_status ps = family_partitioned_update(a, v.nv, v.amask, v.jmask, v.ctr, st, &done);
    if (done || ps != SK_OK) return ps;
  }
  cudaError_t e = pow2 ? dispatch_views<true>(a, v, smem, st) : dispatch_views<false>(a, v, smem, st);
  return set_status_from_cuda(e);
}

sk_status sk_family_estimate(sk_family* fam, sk_estimate* out, void* cuda_stream) {
  if (!fam || !out) return SK_ERR_INVALID_ARG;
  const int n = (int)fam->sub.size();
  std::memset(out, 0, sizeof(sk_estimate) * n);
  cudaStream_t caller = (cudaStream_t)cuda_stream;
  // Fused estimator throughout: the sub-queries go to the many-set estimate, which
  // transforms the rows of all sub-queries of one width together (chains and stars; the
  // others run on its worker streams).
  bool all_fused = n > 0;
  for (const auto& sq : fam->sub) all_fused = all_fused && sq.est->estimator == SK_ESTIMATOR_FUSED;
  if (all_fused) {
    std::vector<sk_set*> v(n);
    for (int i = 0; i < n; i++) v[i] = fam->sub[i].est;
    return run_estimate_many(v.data(), n, out, caller);
  }
  cudaEvent_t ready;
  cudaError_t ce = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (ce != cudaSuccess) return set_status_from_cuda(ce);
  ce = cudaEventRecord(ready, caller);
  for (cudaStream_t w : fam->workers)
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(w, ready, 0);
  if (ce != cudaSuccess) {
    cudaEventDestroy(ready);
    return set_status_from_cuda(ce);
  }
  const int nw = (int)fam->workers.size();
  std::vector<sk_status> status(n, SK_OK);
  auto work = [&](int w) {
    cudaSetDevice(fam->device);
    for (int i = w; i < n; i += nw) status[i] = run_estimate(fam->sub[i].est, &out[i], fam->workers[w]);
  };
  std::vector<std::thread> threads;
  for (int w = 1; w < nw; w++) threads.emplace_back(work, w);
  work(0);
  for (auto& t : threads) t.join();
  // the caller's stream continues after every worker's work
  for (cudaStream_t w : fam->workers) {
    if (ce == cudaSuccess) ce = cudaEventRecord(ready, w);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(caller, ready, 0);
  }
  cudaEventDestroy(ready);
  for (int i = 0; i < n; i++)
    if (status[i] != SK_OK) return status[i];
  return set_status_from_cuda(ce);
}

sk_status sk_family_set_estimator(sk_family* fam, int32_t estimator) {
  if (!fam || estimator < SK_ESTIMATOR_FFT64 || estimator > SK_ESTIMATOR_FUSED) return SK_ERR_INVALID_ARG;
  for (auto& s : fam->sub) s.est->estimator = estimator;
  return SK_OK;
}

sk_status sk_family_info(const sk_family* fam, int32_t* n_sub, int32_t* n_views, size_t* counter_bytes) {
  if (!fam) return SK_ERR_INVALID_ARG;
  if (n_sub) *n_sub = (int32_t)fam->sub.size();
  if (n_views) *n_views = fam->n_views;
  if (counter_bytes) *counter_bytes = (size_t)fam->n_views * fam->d * fam->m * sizeof(int64_t);
  return SK_OK;
}

sk_status sk_family_view(const sk_family* fam, int32_t sub, int32_t rel_s, int32_t* q_relation, int32_t* view) {
  if (!fam || sub < 0 || sub >= (int)fam->sub.size()) return SK_ERR_INVALID_ARG;
  const FamSub& fs = fam->sub[sub];
  if (rel_s < 0 || rel_s >= (int)fs.q_rel.size()) return SK_ERR_INVALID_ARG;
  if (q_relation) *q_relation = fs.q_rel[rel_s];
  if (view) *view = fs.view[rel_s];
  return SK_OK;
}

sk_status sk_family_copy_sketch(const sk_family* fam, int32_t sub, int32_t rel_s, int64_t* host_out,
                                void* cuda_stream) {
  int32_t vid = 0;
  sk_status st = sk_family_view(fam, sub, rel_s, nullptr, &vid);
  if (st != SK_OK) return st;
  if (!host_out) return SK_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = (size_t)fam->d * fam->m * sizeof(int64_t);
  cudaError_t e = cudaMemcpyAsync(host_out, fam->d_counters + (size_t)vid * fam->d * fam->m, bytes,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return set_status_from_cuda(e);
}

sk_status sk_family_reset(sk_family* fam, void* cuda_stream) {
  if (!fam) return SK_ERR_INVALID_ARG;
  const size_t bytes = (size_t)fam->n_views * fam->d * fam->m * sizeof(int64_t);
  return set_status_from_cuda(cudaMemsetAsync(fam->d_counters, 0, bytes, (cudaStream_t)cuda_stream));
}

sk_status sk_family_sync(sk_family* fam, void* cuda_stream) {
  if (!fam) return SK_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, fam->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  if (h != 0) {
    e = cudaMemsetAsync(fam->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_status_from_cuda(e);
  }
  return (sk_status)h;
}

sk_status sk_family_destroy(sk_family* fam) {
  free_family(fam);
  return SK_OK;
}

}  // extern "C"
