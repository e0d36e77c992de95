/*
 * sketch.h -- C ABI of a GB300 (sm_103a) implementation of the convolved
 * Count sketch of Heddes, Nunes, Givargis and Nicolau, "Convolution and
 * Cross-Correlation of Count Sketches Enables Fast Cardinality Estimation of
 * Multi-Join Queries" (PACMMOD 2024).
 *
 * The library keeps, for one join query over relations R_0 .. R_{r-1}, one
 * Count sketch per relation and per median row (d rows), updates them from
 * batches of tuples on the GPU (Algorithm 2), and estimates the query's
 * cardinality by combining the sketches with circular cross-correlation and
 * Hadamard products (Algorithm 3), taking the median over rows (Section 3.3).
 *
 * Conventions for every function
 *   - Returns an sk_status: SK_OK (0) or a negative error code; never throws,
 *     never aborts.  sk_status_string() names a code.
 *   - "dev_" pointers are CUDA device pointers on the current device, managed
 *     memory, or page-locked host memory (cudaHostAlloc / registered), which the
 *     kernels then read across the host link; every other pointer is host memory.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it and is asynchronous unless stated.
 *   - The caller owns every buffer it passes (counters, columns, weights) and
 *     keeps it alive until the stream work that uses it has completed.  The
 *     library owns the sk_set handle, its hash-coefficient table, its status
 *     word and its estimator scratch; sk_sketch_destroy frees them.
 *   - Errors found on the device (a key outside a declared domain, an
 *     estimator overflow) are recorded in the set's status word and reported
 *     by the next sk_sync or sk_estimate_join.
 *   - A handle may be used from one host thread at a time.
 */
#ifndef SK_SKETCH_H
#define SK_SKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sk_status;

enum {
  SK_OK = 0,
  SK_ERR_INVALID_ARG = -1,        /* null pointer, bad size, relation out of range ... */
  SK_ERR_CYCLIC_QUERY = -2,       /* the joins close a cycle (Section 2.6: joins are non-cyclic) */
  SK_ERR_DISCONNECTED_QUERY = -3, /* the relations do not form one connected join graph */
  SK_ERR_SELF_EDGE = -4,          /* a join inside one relation (use a fictitious copy, Section 2.6) */
  SK_ERR_UNSUPPORTED_WIDTH = -5,  /* m out of range for the requested operation */
  SK_ERR_BUFFER_TOO_SMALL = -6,   /* counters buffer smaller than sk_sketch_bytes */
  SK_ERR_MISMATCH = -7,           /* merge of sets with different query, m, d or seed */
  SK_ERR_KEY_OUT_OF_DOMAIN = -8,  /* a key fell outside the declared domain_hint (tuple skipped) */
  SK_ERR_TIMEOUT = -9,            /* a bounded device wait gave up */
  SK_ERR_CUDA = -10,              /* a CUDA runtime call failed */
  SK_ERR_OVERFLOW = -11,          /* an exact intermediate would leave the signed 256-bit range */
  SK_ERR_INEXACT = -12,           /* an FFT correlation could not be certified exact */
  SK_ERR_NO_MEMORY = -13,         /* device allocation failed */
  SK_ERR_SCRATCH_TOO_SMALL = -14, /* the allocation-free estimator's fixed scratch cannot hold this set */
  SK_ERR_OVER_BUDGET = -15        /* a serving request or set does not fit the server's HBM budget */
};

/* Largest number of median rows d a set may have. */
#define SK_MAX_ROWS 64

/* One join {u, v} between attribute attr_a of relation rel_a and attribute
 * attr_b of relation rel_b (Section 2.6 notation: an edge of the join graph). */
typedef struct {
  int32_t rel_a, attr_a, rel_b, attr_b;
} sk_edge;

/* A join query Q(R_0, ..., R_{r-1}).  num_join_attrs[k] = |Omega(R_k)| >= 1; the
 * attributes of R_k are numbered 0 .. |Omega(R_k)|-1 and are the columns of
 * that relation's update batches, in that order.  The joins must make the
 * relations one tree (connected, r - 1 joins, no cycle), and every attribute
 * must take part in at least one join.  Components Psi are the connected
 * components of the attribute graph; each gets one bin function, each join
 * one sign function (Section 3.2, Initialization). */
typedef struct {
  int32_t num_relations;
  const int32_t* num_join_attrs;
  int32_t num_edges;
  const sk_edge* edges;
} sk_query;

/* Opaque handle: a query, its hash functions and its counters. */
typedef struct sk_set sk_set;

/* Signed 256-bit two's-complement integer, little-endian 64-bit limbs. */
typedef struct {
  uint64_t limb[4];
} sk_i256;

/* Result of sk_estimate_join.  row[i] is median row i's estimate X (Eq. 5,
 * computed by Algorithm 3), exact.  median is the lower median of the d rows,
 * row[(d-1)/2] of the sorted values (Section 3.3, median trick). */
typedef struct {
  sk_i256 median;
  int64_t median_i64;    /* == median when fits_i64 */
  int32_t fits_i64;
  int32_t d;
  double median_f64;     /* median rounded to double */
  double mid_mean_f64;   /* mean of the two middle rows (the middle row if d is odd) */
  double max_residual;   /* max |y - round(y)| over every FFT output rounded to an integer */
  int32_t max_limbs;     /* largest number of limbs an operand of a correlation was split into */
  int32_t limb_bits;     /* limb width B of the last correlation step */
  int32_t corr_steps;    /* correlation steps per row (Algorithm 3's FFT-based correlations) */
  int32_t retries;       /* steps redone with narrower limbs after a failed certificate */
  sk_i256 row[SK_MAX_ROWS];
} sk_estimate;

/* ---------------------------------------------------------------------------
 * sk_sketch_bytes: size in bytes of the counters buffer for (query, m, d):
 * r * d * m int64 counters, laid out [relation][row][bucket].
 * Errors: SK_ERR_INVALID_ARG, query validation codes. */
sk_status sk_sketch_bytes(const sk_query* query, int64_t m, int32_t d, size_t* bytes);

/* ---------------------------------------------------------------------------
 * sk_sketch_create: the sampling step of Algorithm 1 and the initialisation of Section 3.2.
 * Validates the query, draws per row one bin function per component and one sign
 * function per join (SplitMix64 from `seed`, each coefficient an element of
 * GF(2^61 - 1)), uploads them, and zeroes the caller's counters buffer
 * (dev_counters, `bytes` >= sk_sketch_bytes) on cuda_stream.
 * 1 <= m <= 2^30 (the estimator needs 2 <= m <= 2^22, or <= 2^21 when m is not a
 * power of two);
 * 1 <= d <= SK_MAX_ROWS.  *out receives the handle.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_CYCLIC_QUERY, SK_ERR_DISCONNECTED_QUERY,
 * SK_ERR_SELF_EDGE, SK_ERR_UNSUPPORTED_WIDTH, SK_ERR_BUFFER_TOO_SMALL,
 * SK_ERR_CUDA, SK_ERR_NO_MEMORY. */
sk_status sk_sketch_create(const sk_query* query, int64_t m, int32_t d, uint64_t seed,
                           void* dev_counters, size_t bytes, void* cuda_stream, sk_set** out);

/* ---------------------------------------------------------------------------
 * sk_sketch_update_batch: Algorithm 2 for n_rows tuples of relation `relation`.
 * Tuple i has key dev_cols[a * col_stride + i] for its attribute a (int64,
 * attribute-major, col_stride >= n_rows) and frequency change
 * Delta_i = dev_weights[i] (NULL: Delta = 1).  For every median row the tuple's
 * bin is (sum over its attributes u of h_Psi(u)(key_u)) mod m (Eq. 3) and its
 * sign the product of s_{u,v}(key_u) over its joins (Eq. 2); counter
 * [relation][row][bin] += sign * Delta in wrapping int64 (Eq. 4).  A key maps to
 * the field as (uint64)key mod (2^61 - 1).  domain_hint (host array of |Omega|
 * exclusive upper bounds, or NULL) declares 0 <= key < bound; tuples with a key
 * outside it are skipped and SK_ERR_KEY_OUT_OF_DOMAIN is recorded.
 * With declared domains whose bounds are at most 2^31, the call may first hash
 * every domain key once per attribute into a table (per key and row: the bin
 * and the sign parity, 16 or 32 bits) and then update by table lookups; it does
 * so when the domains are small against the batch (sum of bounds * 4 <=
 * n_rows * |Omega|) and the relation's d * m * 8-byte sketch is at most 32 MiB
 * (environment: SK_KEY_TABLE=0 never, =1 whenever the bounds allow).  The table
 * (sum of bounds * 16 or 32 bytes when m <= 2^16 and d <= 14; 24 bytes for the
 * two-phase update below when d <= 9; 4 d rounded up to 16 bytes otherwise) comes
 * from the device's stream-ordered pool and is released on cuda_stream at the end
 * of the call; if it cannot be allocated the call hashes per tuple.  Unit-weight
 * batches (dev_weights NULL) into a power-of-two 1024 <= m <= 2^16 with d <= 14, at
 * most 5 attributes, at least 16 m rows and a d * m int32 sketch too large for one
 * CTA's shared memory update in two phases through the table: per-tuple bins
 * written as 16-bit items (2 d bytes per row of staging from the same pool, in
 * windows of at most 2^30 rows), then added per half row in shared memory.
 * Unit-weight batches into a power-of-two 2^17 <= m <= 2^24 with d <= 16, at most 5
 * attributes, at least m rows and a sketch larger than 32 MiB take the table too
 * (the lookups then replace one L2 reduction per counter update that would miss
 * L2) and sort each row's bins by part of 2^15 bins before adding them in shared
 * memory (6 d bytes per row of staging, windows of at most 2^24 rows).
 * SK_PART_UPDATE=0 keeps the one-phase table update and the per-tuple update for
 * both.  Results are identical on every path.
 * Asynchronous on cuda_stream; the columns and weights must stay valid until it
 * completes.  n_rows == 0 is a no-op.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA. */
sk_status sk_sketch_update_batch(sk_set* set, int32_t relation, int64_t n_rows, const int64_t* dev_cols,
                                 int64_t col_stride, const int64_t* dev_weights,
                                 const int64_t* domain_hint, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched update: many (set, relation, batch) items in one persistent launch.
 *
 * sk_update_plan_create records n_items update batches (each exactly what one
 * sk_sketch_update_batch call would take: Algorithm 2 for that relation of that
 * set) and uploads a descriptor table.  sk_update_plan_run then applies all of
 * them with ONE kernel launch (plus a 8-byte memset of its work counter) on
 * cuda_stream: CTAs take chunks of tuples from a device work queue in item order,
 * so small batches share the GPU instead of each paying a launch.  The counters
 * receive exactly the same values as the item-by-item calls (integer addition is
 * order independent).  A run is capturable in a CUDA graph.  The plan keeps the
 * items' pointers: the caller may change the buffers' contents between runs, not
 * their addresses or sizes.  Items of one plan must not target the same counters
 * from different plans running concurrently.  Key domains are not checked.  A
 * relation in a plan may have at most 5 joined attributes.
 *
 * sk_update_plan_config: chunk_tuples (tuples per work item), threads (per CTA),
 * ctas_per_sm, smem_max_counters (items with d*m at most this, and at most 40960,
 * use a per-chunk int32 shared-memory sub-sketch; 0 = never), smem16_max_counters
 * (other items with d*m at most this, and at most 81920, use a per-chunk sub-sketch
 * of 16-bit counters, two per 32-bit word, each biased by 2^15; only tuples with
 * |Delta| <= 32767 / chunk_tuples go there, so no counter leaves [0, 2^16) within a
 * chunk and the packed adds are exact; the others update global memory; 0 = never).
 * sk_update_plan_autotune times a set of configurations on the plan itself (every
 * timed run updates the counters: reset them afterwards) and keeps the fastest.  The
 * choice is persisted: keyed by the device's SM count, the plan's item shapes (m, d and
 * attribute count, with their counts) and the log2 of its tuple count, it is appended to a
 * JSON-lines file (SK_AUTOTUNE_CACHE, else autotune.json beside libsketch.so;
 * SK_AUTOTUNE_CACHE=off disables it), and a later autotune of a plan with the same key takes
 * the stored configuration without timing (or updating the counters); *best_ms is then the
 * stored time.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA, SK_ERR_NO_MEMORY. */
typedef struct {
  sk_set* set;
  int32_t relation;
  int64_t n_rows;
  const int64_t* dev_cols;
  int64_t col_stride;
  const int64_t* dev_weights;
} sk_update_item;

typedef struct {
  int32_t chunk_tuples;
  int32_t threads;
  int32_t ctas_per_sm;
  int32_t smem_max_counters;
  int32_t smem16_max_counters;
} sk_update_plan_config;

typedef struct sk_update_plan sk_update_plan;

sk_status sk_update_plan_create(const sk_update_item* items, int32_t n_items, sk_update_plan** out);
sk_status sk_update_plan_run(sk_update_plan* plan, void* cuda_stream);
/* sk_update_plan_zero: sets to zero, in one launch on cuda_stream, the int64[d][m]
 * counters of every (set, relation) that the plan's items write (the other relations
 * of those sets are left as they are): the batched form of sk_sketch_reset for a plan
 * that re-sketches its relations.  Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA. */
sk_status sk_update_plan_zero(sk_update_plan* plan, void* cuda_stream);
sk_status sk_update_plan_get_config(const sk_update_plan* plan, sk_update_plan_config* out);
sk_status sk_update_plan_set_config(sk_update_plan* plan, const sk_update_plan_config* config);
sk_status sk_update_plan_autotune(sk_update_plan* plan, void* cuda_stream, sk_update_plan_config* best,
                                  double* best_ms);
sk_status sk_update_plan_destroy(sk_update_plan* plan);

/* ---------------------------------------------------------------------------
 * sk_sketch_merge: dst += src, counter by counter (Section 2.2: linear sketches
 * combine by addition).  Both sets must have the same query, m, d and seed.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_MISMATCH, SK_ERR_CUDA. */
sk_status sk_sketch_merge(sk_set* dst, const sk_set* src, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * sk_estimate_join: Algorithm 3 for every median row, then the lower median.
 * Root attribute: attribute 0 of relation 0.  Every row is the exact integer of Eq. 5;
 * the arithmetic that computes each circular cross-correlation IFFT(conj(FFT(a)) o FFT(x))
 * exactly is the set's estimator (sk_sketch_set_estimator; default SK_ESTIMATOR_FUSED,
 * exact by construction); Hadamard products and sums are exact signed 256-bit
 * integers.  2 <= m <= 2^22 for a power of two m; any other
 * 2 <= m <= 2^21 is handled with zero-padded transforms of the next power of two >= 2m - 1
 * (the circular correlation mod m is the padded linear correlation folded back).
 * Synchronises cuda_stream and fills *out (host memory).
 * Errors: SK_ERR_UNSUPPORTED_WIDTH, SK_ERR_OVERFLOW, SK_ERR_INEXACT,
 * SK_ERR_KEY_OUT_OF_DOMAIN (from earlier updates), SK_ERR_CUDA, SK_ERR_NO_MEMORY. */
sk_status sk_estimate_join(sk_set* set, sk_estimate* out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * sk_estimate_many: sk_estimate_join for n distinct sets in one call; out[i] is
 * set i's estimate, identical to what sk_estimate_join would give.  Sets using
 * SK_ESTIMATOR_FUSED whose queries qualify are grouped by width and estimated
 * together (each set takes the number of CRT primes its own bound needs; per prime:
 * one load, one batch of transforms and one product-sum over the rows of every set
 * that needs that prime); the others are estimated concurrently on
 * internal worker streams (SK_MANY_WORKERS, default 4), which first wait for the
 * work already queued on cuda_stream, and cuda_stream continues after them.  The
 * call returns when every estimate is on the host; grouped work takes one
 * stream-ordered device block for the call.  Returns the first error of any set.
 * Errors: SK_ERR_INVALID_ARG (null, or a set twice), SK_ERR_UNSUPPORTED_WIDTH,
 * and those of sk_estimate_join. */
sk_status sk_estimate_many(sk_set* const* sets, int32_t n, sk_estimate* out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * sk_sketch_set_estimator: selects how sk_estimate_join computes each circular
 * cross-correlation (Definition 3.1); all give the identical exact result.
 * Default (sk_sketch_create): SK_ESTIMATOR_FUSED.
 *   SK_ESTIMATOR_FFT64: the paper's transform, FP64 FFTs on signed limbs, outputs
 *     rounded to integers.  The limb width B is the widest for which an a priori bound
 *     on the FFT rounding error -- Percival's bound for FFT convolution (Math. Comp. 72,
 *     2003), extended to the packing of two limbs per transform and the sums over limb
 *     pairs, with the twiddle table's measured error -- is at most 1/4, so every rounded
 *     output is exact by that bound; each step is also checked a posteriori (largest
 *     distance to an integer <= 1/4, the exact row-sum identity sum z = (sum a)(sum x)
 *     mod 2^64 and, for power-of-two m, Z(w) = A(1/w) X(w) modulo q = 2^64 - 2^32 + 1
 *     at a random primitive m-th root of unity w) and redone with narrower limbs if a
 *     check fails.  The other two arithmetics need no certificate;
 *   SK_ESTIMATOR_NTT: number-theoretic transforms over GF(2^64 - 2^32 + 1) on signed
 *     limbs narrow enough that every output lies below q/2 in magnitude, exact by
 *     construction (GB300's integer pipes are much faster than its FP64 pipe);
 *   SK_ESTIMATOR_FUSED: for queries whose components all have exactly two attributes
 *     (chains, stars) and power-of-two m, no correlation steps at all: with the
 *     relations two-coloured along the components, X = (1/m) sum_nu prod_k C_k(+-nu)
 *     (C_k the DFT of relation k's row), evaluated modulo 31-bit primes c 2^22 + 1
 *     and recombined by the Chinese remainder theorem, with enough primes that their
 *     product exceeds 8 prod_k ||c_k||_1 >= 8 |X| (exact: correlation, Hadamard
 *     product and sum are all submultiplicative in the l1 norm).  Other queries (a
 *     component of three or more attributes, Figure 3) and widths run Algorithm 3's
 *     correlation steps modulo the same primes (one transform per operand, no limbs;
 *     widths that are not powers of two zero-padded to a power of two >= 2m - 1 and
 *     folded back) and recombine the row sums by CRT; only bounds beyond 9 primes
 *     are estimated as with SK_ESTIMATOR_NTT.  In the result, max_limbs is the
 *     number of primes and limb_bits 0.
 * The environment variable SK_ESTIMATOR=ntt (or =fft64) selects that arithmetic for
 * sets created after it is set.  Errors: SK_ERR_INVALID_ARG. */
enum { SK_ESTIMATOR_FFT64 = 0, SK_ESTIMATOR_NTT = 1, SK_ESTIMATOR_FUSED = 2 };
sk_status sk_sketch_set_estimator(sk_set* set, int32_t estimator);

/* ---------------------------------------------------------------------------
 * sk_estimate_join_noalloc: the estimate of sk_estimate_join without any device
 * allocation, for callers that cannot allocate device memory while they estimate --
 * e.g. code running in a host callback or driver hook that must not enter the CUDA
 * allocator, a process whose device memory is fully held by another pool, or a
 * latency-critical path that forbids allocation.  No counterpart in the paper.
 * It always uses FP64 FFTs (whatever the set's estimator) with the limb width and
 * checks described for SK_ESTIMATOR_FFT64 -- the a priori bound, then the residual,
 * exact per-row sums and the evaluation at a random root of unity, each step redone up
 * to three times with narrower limbs -- so rows, median, fits_i64, median_i64,
 * median_f64 and mid_mean_f64 equal those of
 * sk_estimate_join; the diagnostics (max_residual, max_limbs, limb_bits, retries)
 * describe this call's own arithmetic.  Only power-of-two m (2 <= m <= 2^22) is
 * accepted; other widths return SK_ERR_UNSUPPORTED_WIDTH.  The set's device must be
 * the current device (else SK_ERR_INVALID_ARG).
 * It calls no cudaMalloc/cudaFree and no allocating library routine: all scratch
 * lives in one static device array of 32 MiB (SK_NOALLOC_SCRATCH_BYTES) that every
 * GPU loading this library holds until the process exits.  The array's device
 * address is looked up on the first call on each device (with that device
 * current), so make that first call before any stream capture.  Every call shares
 * the array and leaves its contents behind; calls whose GPU work overlaps (other
 * streams or threads) race on it and must be serialised by the caller.  The
 * handle itself must have been created earlier (sk_sketch_create allocates).
 * Limits: the estimator's vector slots ((schedule slots + 1) * d * m * 32 bytes),
 * twiddles (m * 8 bytes) and small buffers must fit in the array, or the call
 * returns SK_ERR_SCRATCH_TOO_SMALL before any GPU work; the FFT buffers of each
 * correlation step (2 * d * ceil(limbs / 2) * m * 16 bytes) must fit in what is
 * left, or the call returns SK_ERR_SCRATCH_TOO_SMALL at that step.
 * Synchronises cuda_stream and fills *out.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_UNSUPPORTED_WIDTH, SK_ERR_SCRATCH_TOO_SMALL,
 * SK_ERR_OVERFLOW, SK_ERR_INEXACT, SK_ERR_KEY_OUT_OF_DOMAIN (from earlier updates),
 * SK_ERR_CUDA. */
#define SK_NOALLOC_SCRATCH_BYTES (32ull << 20)
sk_status sk_estimate_join_noalloc(sk_set* set, sk_estimate* out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * sk_sketch_reset: zeroes every counter of the set and its device status word on
 * cuda_stream (the "set a block of memory to zeros" initialisation of Section
 * 2.2, without redrawing the hash functions).
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA. */
sk_status sk_sketch_reset(sk_set* set, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * sk_sync: synchronises cuda_stream and returns (then clears) the first error
 * recorded on the device for this set since the last sk_sync. */
sk_status sk_sync(sk_set* set, void* cuda_stream);

/* sk_sketch_destroy: frees the handle, its coefficient table, status word and
 * scratch.  Does not touch the caller's counters.  NULL is a no-op. */
sk_status sk_sketch_destroy(sk_set* set);

/* sk_status_string: static, human-readable name of a status code. */
const char* sk_status_string(sk_status status);

/* ---------------------------------------------------------------------------
 * Introspection and test hooks.
 *
 * sk_sketch_info: r, m, d, number of components and of joins of a set.
 * sk_get_coefficients: copies the hash coefficients to host memory:
 *   uint64 [d][2*components + 4*joins]; per row (b0, b1) of each component's bin
 *   function h(x) = ((b1 x + b0) mod p) mod m, then (s0, s1, s2, s3) of each
 *   join's sign function s(x) = +1 if (s0 + s1 x + s2 x^2 + s3 x^3) mod p is even,
 *   else -1; components are numbered by their smallest attribute, joins sorted
 *   by their endpoints (attributes numbered relation by relation).
 *   `count` is the number of uint64 the host buffer holds.
 * sk_set_coefficients: replaces the table (same layout; every value < 2^61 - 1),
 *   e.g. to run the method with chosen hash functions.  Enqueued on cuda_stream.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA. */
sk_status sk_sketch_info(const sk_set* set, int32_t* r, int64_t* m, int32_t* d, int32_t* n_components,
                         int32_t* n_joins);
sk_status sk_get_coefficients(const sk_set* set, uint64_t* host_out, size_t count);
sk_status sk_set_coefficients(sk_set* set, const uint64_t* host_coeffs, size_t count, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving (sk_server_*): a continuous-batching request loop over live sets resident on
 * the current device, run by native threads (a scheduler, a retire thread and one
 * worker per estimate stream).  Every set keeps its requests in arrival order: an
 * estimate sees exactly the updates of that set submitted before it, and later
 * updates of the set wait until it has read the counters, so each result equals
 * running the set's requests one by one.  Across sets the scheduler admits the
 * oldest head request as soon as an update slot or an estimate worker is free and its
 * memory fits the budget; updates are staged from host memory on a copy stream and
 * run on an update stream, estimates on their worker's stream, overlapping on the
 * device.  Charged against hbm_budget_bytes: the counters of every registered set
 * (r * d * m * 8 bytes), the staged columns and weights of every in-flight update and
 * an allowance per running estimate of (max(2, r) + 1) * d * m * 32 + 128 * d * m +
 * 8 * m bytes.
 *
 * sk_server_create: update_slots in-flight update batches (>= 1), estimate_workers
 *   estimate threads and streams (1..64), each running up to 8 admitted estimates of
 *   distinct sets together (as sk_estimate_many), estimate streams at the device's
 *   highest priority when estimate_priority != 0.
 * sk_server_register_set: makes `set` (created and owned by the caller, alive until
 *   sk_server_destroy) a live set named set_id; SK_ERR_OVER_BUDGET when its counters
 *   do not fit.  Sets must not be updated or estimated outside the server meanwhile.
 * sk_server_submit_update: queues Algorithm 2 for n_rows tuples of `relation` from
 *   host memory (int64 attribute-major columns with col_stride >= n_rows, optional
 *   int64 weights; page-locked memory lets the copy overlap; domain_hint: NULL or the
 *   relation's |Omega| exclusive key bounds, copied at submission, as for
 *   sk_sketch_update_batch).  The host buffers must stay valid until the request has
 *   finished.  *request_id names the request.  The updates admitted in one scheduling
 *   pass are coalesced: one staging buffer and one persistent multi-item launch for those
 *   without declared domains (up to 64 per batch, at most update_slots batches in
 *   flight), one sk_sketch_update_batch call each for those with declared domains (so a
 *   large batch can take the key tables); results are the same as one launch per update.
 *   A request that could never fit (more memory than the budget leaves beside the
 *   registered sets' counters) finishes at once with status SK_ERR_OVER_BUDGET, and an
 *   update of zero rows finishes at once with SK_OK.
 * sk_server_submit_estimate: queues Algorithm 3 and the median for set set_id.
 * sk_server_result: the state of a request (wait != 0 blocks until it finishes).
 *   When *finished is 1 it also returns its status, the estimate (zeroed for an
 *   update), its submission and completion times in seconds since sk_server_create,
 *   and forgets the request (a later call with the same id is SK_ERR_INVALID_ARG).
 * sk_server_hold: on != 0 pauses admission (submissions still queue; work already on the
 *   device finishes), on == 0 resumes it; e.g. to queue a batch of requests and release
 *   them at once.  sk_server_drain on a held server with queued requests does not return.
 * sk_server_pending: the number of submitted requests not yet finished.
 * sk_server_drain: blocks until every submitted request has finished.
 * sk_server_stats: update batches launched so far and the update requests they held.
 * sk_server_destroy: drains, stops the threads and releases the server (not the sets).
 * Errors: SK_ERR_INVALID_ARG (null, unknown set or request, bad relation or sizes),
 * SK_ERR_OVER_BUDGET, SK_ERR_CUDA, SK_ERR_NO_MEMORY; a request's own status carries
 * the errors of its update or estimate. */
typedef struct sk_server sk_server;
sk_status sk_server_create(int64_t hbm_budget_bytes, int32_t update_slots, int32_t estimate_workers,
                           int32_t estimate_priority, sk_server** out);
sk_status sk_server_register_set(sk_server* server, int32_t set_id, sk_set* set);
sk_status sk_server_submit_update(sk_server* server, int32_t set_id, int32_t relation, int64_t n_rows,
                                  const int64_t* host_cols, int64_t col_stride, const int64_t* host_weights,
                                  const int64_t* domain_hint, int64_t* request_id);
sk_status sk_server_submit_estimate(sk_server* server, int32_t set_id, int64_t* request_id);
sk_status sk_server_result(sk_server* server, int64_t request_id, int32_t wait, int32_t* finished,
                           sk_status* status, sk_estimate* est, double* arrival_s, double* done_s);
sk_status sk_server_hold(sk_server* server, int32_t on);
sk_status sk_server_pending(sk_server* server, int64_t* n);
sk_status sk_server_drain(sk_server* server);
sk_status sk_server_stats(sk_server* server, int64_t* batches, int64_t* batched_updates);
sk_status sk_server_destroy(sk_server* server);

/* sk_launch_count: number of CUDA kernels this library has launched in this process
 * (all sets, all devices), for accounting of GPU work. */
int64_t sk_launch_count(void);

/* ---------------------------------------------------------------------------
 * Sub-query families (Section 3.4, integration with query optimizers).  A plan
 * enumerator needs the cardinality of many sub-queries of one query Q; the
 * sketches of all of them are built in one pass over each relation's tuples, and
 * a relation's sketch is shared by every sub-query that sees the same view of it.
 *
 * A sub-query S is a non-empty subset of Q's joins (indices into query->edges)
 * whose relations are connected.  Its relations are those its joins touch (in
 * ascending order of their index in Q, which is S's relation numbering in the
 * results), each keeping the attributes S joins (ascending).  Hash functions are
 * drawn for Q exactly as sk_sketch_create draws them from `seed`, and S inherits
 * them: each component of S takes the bin function of the component of Q that
 * contains it; a component of S with one join takes the sign function of the
 * first join (lowest canonical index) of its component of Q; a component of S
 * with several joins takes each join's own sign function.  (With this choice the
 * two-way sub-queries {0,1} and {1,3} of Figure 3 share relation R1's sketch, as
 * the paper describes; S = Q gives exactly sk_sketch_create's functions.)  The
 * view of relation R_k in S is, for every attribute S joins, the set of sign
 * functions its value is hashed with; sub-queries with equal views of R_k share
 * one d x m sketch.  The library owns the family's counters (views x d x m int64
 * in device memory).
 * ------------------------------------------------------------------------- */
typedef struct sk_family sk_family;

/* Largest number of views one relation may have in a family, and of sign
 * functions ("slots": its joins plus its component's first join) its attributes
 * may use together. */
#define SK_MAX_VIEWS 64
#define SK_MAX_SLOTS 64

/* sk_family_create: n_sub sub-queries; sub-query i is the joins
 * sub_edges[sub_offsets[i] .. sub_offsets[i+1]) (indices into query->edges,
 * sub_offsets has n_sub + 1 entries, sub_offsets[0] = 0).  m, d, seed as for
 * sk_sketch_create (the estimate needs 2 <= m <= 2^22, or <= 2^21 when m is not
 * a power of two).  The counters are zeroed on cuda_stream.
 * Errors: SK_ERR_INVALID_ARG (empty, repeated or out-of-range joins, a
 * disconnected sub-query, too many views or slots), query validation codes,
 * SK_ERR_UNSUPPORTED_WIDTH, SK_ERR_NO_MEMORY, SK_ERR_CUDA. */
sk_status sk_family_create(const sk_query* query, int32_t n_sub, const int32_t* sub_offsets,
                           const int32_t* sub_edges, int64_t m, int32_t d, uint64_t seed, void* cuda_stream,
                           sk_family** out);

/* sk_family_update_batch: Algorithm 2 for a batch of Q's relation `relation`,
 * laid out as for sk_sketch_update_batch (all |Omega(R_k)| columns of Q).  One
 * pass hashes every tuple once per row and adds it to every view of R_k (each
 * view with its own bin sum and sign product).  When every attribute of R_k has
 * one sign slot (each in one join of Q), the batch has unit weights and declared
 * domains, m is a power of two in [1024, 2^16], d <= 9, views have at most 5
 * attributes and the batch at least 16 m rows, the call instead builds one key
 * table over R_k's attributes (24 bytes per domain key) and runs the two-phase
 * update of sk_sketch_update_batch once per view (staging from the same pool;
 * SK_PART_UPDATE=0 keeps the one-pass update).  A tuple with any key outside its
 * domain is left out of every view.  A relation in no sub-query is a no-op.
 * Domain violations are recorded and reported by sk_family_sync.  Results are
 * identical on both paths.
 * Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA. */
sk_status sk_family_update_batch(sk_family* fam, int32_t relation, int64_t n_rows, const int64_t* dev_cols,
                                 int64_t col_stride, const int64_t* dev_weights, const int64_t* domain_hint,
                                 void* cuda_stream);

/* sk_family_estimate: Algorithm 3 and the median for every sub-query; out has
 * n_sub entries, entry i for sub-query i (as sk_estimate_join).  With
 * SK_ESTIMATOR_FUSED on every sub-query they are estimated as sk_estimate_many
 * does (qualifying sub-queries of one width transformed together); otherwise
 * concurrently on the family's worker streams.  Either way the work starts after
 * the work already queued on cuda_stream, and the call returns when every
 * estimate is on the host.  Returns the first error of any sub-query.
 * Errors: as sk_estimate_join. */
sk_status sk_family_estimate(sk_family* fam, sk_estimate* out, void* cuda_stream);

/* sk_family_set_estimator: the correlation arithmetic of every sub-query (as
 * sk_sketch_set_estimator). */
sk_status sk_family_set_estimator(sk_family* fam, int32_t estimator);

/* sk_family_info: number of sub-queries, total views (distinct sketches) and the
 * bytes of counters they take.  Any output may be NULL. */
sk_status sk_family_info(const sk_family* fam, int32_t* n_sub, int32_t* n_views, size_t* counter_bytes);

/* sk_family_view: for relation rel_s of sub-query sub (S's numbering), the
 * relation of Q it is and the index of its view (the same index for every
 * sub-query sharing that sketch).  Errors: SK_ERR_INVALID_ARG. */
sk_status sk_family_view(const sk_family* fam, int32_t sub, int32_t rel_s, int32_t* q_relation, int32_t* view);

/* sk_family_copy_sketch: copies the d x m counters of relation rel_s of
 * sub-query sub into host_out (int64 [d][m]) after the work queued on
 * cuda_stream; synchronous.  Errors: SK_ERR_INVALID_ARG, SK_ERR_CUDA. */
sk_status sk_family_copy_sketch(const sk_family* fam, int32_t sub, int32_t rel_s, int64_t* host_out,
                                void* cuda_stream);

/* sk_family_reset: zeroes every view on cuda_stream.  sk_family_sync: waits for
 * cuda_stream and returns (and clears) the first device-side error of the
 * family's updates.  sk_family_destroy: frees the family. */
sk_status sk_family_reset(sk_family* fam, void* cuda_stream);
sk_status sk_family_sync(sk_family* fam, void* cuda_stream);
sk_status sk_family_destroy(sk_family* fam);

#ifdef __cplusplus
}
#endif

#endif /* SK_SKETCH_H */
