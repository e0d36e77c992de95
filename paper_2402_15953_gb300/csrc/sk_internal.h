// Internal declarations shared by the translation units of libsketch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sketch.h"

namespace sk {

constexpr uint64_t kP61 = (1ull << 61) - 1;   // the Mersenne prime 2^61 - 1
constexpr int kMaxAttrs = 16;                  // joined attributes per relation handled by the update kernel
constexpr int kMaxDegree = 16;                 // joins per attribute
constexpr int kMaxLimbs = 40;                  // limbs per correlation operand

// Update-kernel description of one relation: for every row, for each attribute u in
// column order, (b0, b1) of u's component bin function followed by (s0..s3) of each
// join incident to u.  coef_row_len = sum_u (2 + 4 deg(u)).
struct RelPlan {
  int a = 0;                        // |Omega(R_k)|
  int deg[kMaxAttrs] = {0};         // |Gamma(u)| per attribute
  int coef_row_len = 0;
  uint64_t* d_coef = nullptr;       // device [d][coef_row_len]
};

enum OpKind { OP_LEAF = 0, OP_HAD = 1, OP_CORR = 2, OP_SUM = 3 };

// One step of Algorithm 3, unrolled on the host into a fixed schedule over
// vector slots (each slot holds d rows of m signed 256-bit integers).
struct EstOp {
  OpKind kind;
  int dst;   // slot written (LEAF, HAD: dst = dst o src, CORR: dst = src (star) dst, SUM: slot summed)
  int src;   // slot read
  int rel;   // LEAF: relation
};

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Canonical numbering of a query (Section 2.6 notation): attributes numbered relation by
// relation, joins (u, v) with u < v sorted, components numbered by smallest attribute.
struct QueryInfo {
  int r = 0;
  std::vector<int> num_join_attrs, offsets, rel_of, comp_of;
  std::vector<std::pair<int, int>> edges;
  std::vector<std::vector<int>> gamma, incident;
  int n_comp = 0;
};

}  // namespace sk

struct sk_set {
  int r = 0;
  int64_t m = 0;
  int d = 0;
  uint64_t seed = 0;
  int device = 0;
  std::vector<int> num_join_attrs, offsets, rel_of, comp_of;
  std::vector<std::pair<int, int>> edges;     // canonical joins {u, v}, u < v, sorted
  std::vector<std::vector<int>> gamma, incident;
  int n_comp = 0;
  int coef_row_len = 0;                        // 2 * n_comp + 4 * n_edges
  std::vector<uint64_t> h_coef;                // [d][coef_row_len]
  std::vector<sk::RelPlan> rel;                // per relation
  int64_t* counters = nullptr;                 // caller-owned int64 [r][d][m]
  std::vector<int64_t*> rel_ctr;               // per relation: its d x m counters (the estimator reads these)
  size_t counter_bytes = 0;
  int* d_status = nullptr;                     // first device-side error, 0 = none
  std::vector<sk::EstOp> plan;                 // Algorithm 3 schedule
  int n_slots = 0;
  int corr_steps = 0;
  sk::Scratch scratch;                         // estimator slots and small buffers
  sk::Scratch fft_scratch;                     // estimator FFT buffers (grown on demand)
  double* d_twiddle = nullptr;                 // FFT twiddles for width m
  int64_t twiddle_m = 0;
  int estimator = SK_ESTIMATOR_FUSED;          // correlation backend
  uint64_t* d_gl_tw = nullptr;                 // GF(q) twiddles [w^t | w^-t] for the NTT length
  int64_t gl_m = 0;
  uint64_t gl_r4 = 1, gl_r4inv = 1, gl_minv = 1;
  uint64_t eval_draws = 0;                     // evaluation points drawn for certificates
  uint32_t* d_fu_tw = nullptr;                 // fused estimator: per prime [w^t | w^-t], t < m/2
  int64_t fu_m = 0;                            // width the fused twiddles are for
  int fu_np = 0;                               // primes they cover
  const int64_t** d_fu_rel = nullptr;          // fused estimator: device copy of rel_ctr
};

namespace sk {

// sk_update.cu
sk_status launch_update(sk_set* s, int relation, int64_t n, const int64_t* cols, int64_t col_stride,
                        const int64_t* weights, const int64_t* domain, cudaStream_t st);
sk_status launch_merge(int64_t* dst, const int64_t* src, int64_t count, cudaStream_t st);

// sk_multi.cu: the persistent multi-item update behind sk_update_plan_* and the serving loop.
size_t multi_item_size();   // bytes of one device descriptor
// Fills n descriptors (n * multi_item_size() bytes of host memory at desc) for items whose
// n_rows are all > 0, under cfg; the launch's chunk count, coefficient words and dynamic
// shared memory come back.  SK_ERR_INVALID_ARG when the shared memory would exceed 200 KB.
sk_status multi_describe(const sk_update_item* items, int n, const sk_update_plan_config& cfg, void* desc,
                         int64_t* total_chunks, int* coef_words, size_t* smem_bytes);
// One persistent launch over n descriptors already in device memory (d_queue: an 8-byte
// work counter, zeroed here on st when zero_queue, else already zero).
sk_status multi_launch(const void* d_desc, int n, int64_t total_chunks, const sk_update_plan_config& cfg,
                       int coef_words, size_t smem_bytes, unsigned long long* d_queue, cudaStream_t st,
                       bool zero_queue);

// sk_estimate.cu
sk_status run_estimate(sk_set* s, sk_estimate* out, cudaStream_t st);
sk_status run_estimate_noalloc(sk_set* s, sk_estimate* out, cudaStream_t st);
sk_status run_estimate_many(sk_set** sets, int n, sk_estimate* out, cudaStream_t st);
void free_estimator(sk_set* s);

// sk_api.cu
sk_status set_status_from_cuda(cudaError_t e);
void count_launch(int n = 1);   // adds to the process-wide kernel-launch counter
// Raises kernel func's dynamic shared-memory limit to the most it can have: the device's
// opt-in limit per block less the kernel's static shared memory.  Every kernel always gets
// this one value: the attribute is process-wide per kernel, so per-call sizes would let a
// concurrent caller (estimate worker threads) lower it between another thread's set and
// launch, failing that launch.  Launches still request only what they use.
cudaError_t allow_dynamic_smem(const void* func);
// Raises func's dynamic shared-memory limit when its static shared memory plus
// dynamic_bytes exceed the default 48 KB.
cudaError_t fit_dynamic_smem(const void* func, size_t dynamic_bytes);
sk_status query_info(const sk_query* q, QueryInfo* out);   // validation + canonical numbering
// Stream-ordered allocation from the library's device pool (update scratch); release with
// cudaFreeAsync on a stream ordered after the last use.
cudaError_t pool_malloc_async(void** ptr, size_t bytes, cudaStream_t st);
// Algorithm 1's draw: d rows of row_len field elements from SplitMix64(seed)
std::vector<uint64_t> draw_coefficients(uint64_t seed, int d, int row_len);
// A set used only for estimation: its relations' counters are rel_ctr (owned elsewhere).
sk_status make_estimation_set(const QueryInfo& c, int64_t m, int d, uint64_t seed, std::vector<uint64_t> h_coef,
                              std::vector<int64_t*> rel_ctr, sk_set** out);
void destroy_set(sk_set* s);
namespace dev {
struct UpdArgs;
}
// Sub-query family views of one relation through the partitioned update when the batch and
// the views allow it (sk_update.cu); *done = false when it launched nothing.
sk_status family_partitioned_update(const dev::UpdArgs& a, int nv, const uint32_t* amask,
                                    const unsigned long long* jmask, unsigned long long* const* ctr, cudaStream_t st,
                                    bool* done);

}  // namespace sk
