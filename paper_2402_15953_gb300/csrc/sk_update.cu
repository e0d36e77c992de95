// Sketch update (Algorithm 2, Eqs. 2-4) and merge (Section 2.2) kernels.
//
// Every tuple of relation R_k is hashed for all d median rows: for each of its
// joined attributes u the key is mapped into GF(p), p = 2^61 - 1, the bin
// function of u's component h(x) = ((b1 x + b0) mod p) mod m and the sign
// functions of u's joins s(x) = +-1 from the parity of (s0 + s1 x + s2 x^2 +
// s3 x^3) mod p are evaluated; the tuple's bin is the sum of the bins mod m and
// its sign the product of the signs; sign * Delta is added to that counter.
//
// Two scatter targets:
//   - SMEM: the d x m sub-sketch fits in shared memory; each CTA accumulates
//     into block-private int32 counters (exact: the host bounds |Delta| times
//     the tuples a CTA sees below 2^31, larger weights go straight to global
//     memory) and flushes the non-zero counters into the int64 sketch with
//     64-bit atomics at the end;
//   - GLOBAL: 64-bit atomic adds straight into the int64 sketch (resident in
//     L2 when d * m * 8 bytes is small against the 126 MiB L2).
// Counters wrap like two's-complement int64 (additions are done on uint64).
#include <algorithm>
#include <cstdlib>

#include "sk_hash.cuh"
#include "sk_internal.h"

namespace sk {
namespace {

using namespace dev;


template <int A, bool POW2, bool SMEM, bool DEG1>
__global__ void __launch_bounds__(256) k_update(UpdArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* s_coef = (uint64_t*)smem_raw;
  const int ncoef = p.d * p.row_len;
  int* s_sub = (int*)(s_coef + ncoef);
  const int64_t dm = (int64_t)p.d * (int64_t)p.m;
  for (int i = threadIdx.x; i < ncoef; i += blockDim.x) s_coef[i] = p.coef[i];
  if (SMEM)
    for (int64_t i = threadIdx.x; i < dm; i += blockDim.x) s_sub[i] = 0;
  __syncthreads();

  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  if (SMEM && p.agg) {
    // warp-uniform loop: every lane of a warp runs the same iterations (collectives inside)
    const int lane = threadIdx.x & 31;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x - lane); b < p.n; b += step)
      update_tuple<A, POW2, SMEM, true, DEG1>(p, s_coef, s_sub, b + lane, b + lane < p.n);
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += step)
      update_tuple<A, POW2, SMEM, false, DEG1>(p, s_coef, s_sub, i);
  }
  if (SMEM) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < dm; i += blockDim.x) {
      const int v = s_sub[i];
      if (v != 0) atomicAdd(p.ctr + i, (unsigned long long)(int64_t)v);
    }
  }
}

// Key-table records for every declared domain key of every attribute (one thread per key).
template <bool POW2, bool DEG1>
__global__ void __launch_bounds__(256) k_key_table(UpdArgs p, TabArgs t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* s_coef = (uint64_t*)smem_raw;
  const int ncoef = p.d * p.row_len;
  for (int i = threadIdx.x; i < ncoef; i += blockDim.x) s_coef[i] = p.coef[i];
  __syncthreads();
  const int64_t total = t.base[p.a];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    int u = 0;
    while (u + 1 < p.a && g >= t.base[u + 1]) u++;
    key_record<POW2, DEG1>(p, t, s_coef, u, (uint32_t)(g - t.base[u]), t.tbl + g * 4 * t.rvec);
  }
}

// Algorithm 2 through the key tables; scatter targets as in k_update.  The instances with
// 32-byte narrow records and a power-of-two width fit 48 registers without spills, which
// gives five CTAs per SM and more gathers in flight (star F update 5.63 -> 5.50 ms).
template <int A, bool POW2, bool SMEM, bool NARROW, bool V8>
__global__ void __launch_bounds__(256, (A > 0 && V8 && NARROW && POW2) ? 5 : 1) k_update_tab(UpdArgs p, TabArgs t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* s_sub = (int*)smem_raw;
  const int64_t dm = (int64_t)p.d * (int64_t)p.m;
  if (SMEM) {
    for (int64_t i = threadIdx.x; i < dm; i += blockDim.x) s_sub[i] = 0;
    __syncthreads();
  }
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += step)
    update_tuple_tab<A, POW2, SMEM, NARROW, V8>(p, t, s_sub, i);
  if (SMEM) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < dm; i += blockDim.x) {
      const int v = s_sub[i];
      if (v != 0) atomicAdd(p.ctr + i, (unsigned long long)(int64_t)v);
    }
  }
}

// ---------------------------------------------------------------------------
// Partitioned update through the key tables (unit weights, power-of-two 1024 <= m <= 2^16,
// d <= 14, at most 5 attributes: the star fact table).  k_update_tab adds each (tuple, row)
// to the L2-resident int64 sketch with one 64-bit reduction, and the L2 lookup rate bounds it
// (9 reductions per tuple at d = 9, about half of them forwarded between the two dies' L2
// halves).  Shared-memory atomics run about ten times faster than L2 reductions on GB300,
// but a d x m int32 sketch of 9 x 2^16 does not fit in one SM.  So the update runs in two
// phases over windows of the batch.  Each row's bins are split into S = m / 2^L parts of
// 2^L bins, L = min(log2 m, 15), so S is 1 or 2.
//   1. k_tab_items: per tuple the key-table gathers and each row's bin sum and sign product
//      (Eqs. 2-3).  Each warp of this persistent kernel owns one region of C item slots per
//      row (C = 32 x its tile count) and appends its tiles' items there: the part-0 items
//      from the region's start upward, the part-1 items from its end downward (each item the
//      bin's offset within its part in bits 0..14 and the sign in bit 15).  At the end the warp
//      writes each row's part-0 count and its count of valid tuples.  A tuple with a key
//      outside its declared domain is left out (and reported, as in every other path).
//      Stores carry an L2 evict-first hint, so the items do not push the key tables' records
//      out of L2.
//   2. k_part_accum: a CTA owns part h of one row as 2^L int32 counters in shared memory
//      (at most 128 KB) over the regions of a range of phase-1 warps; its warps take pieces of
//      those regions, each lane 8 items (one 16-byte load) at a time, and add the signs with
//      shared-memory atomics, reading only part h's items; the CTA finally adds each counter
//      into the int64 sketch with one 64-bit reduction.
// Every counter receives the same sum as in k_update_tab (integer addition in any order);
// a CTA's int32 counter holds at most its range's tuple count in magnitude, kept below 2^31.
//
// Records for this path (32 bytes, built by k_key_table_l20 for d <= 9): row r's bin in bits
// 20 (r mod 3) .. 20 (r mod 3) + 15 of 64-bit word r / 3 (words 0..2), the d sign bits in
// 32-bit word 7.  Summing the A <= 5 records word by word in 64 bits gives every row's exact
// bin sum (below A 2^16 < 2^20: no carry between lanes).  For 10 <= d <= 14 the narrow
// 16-bit records of k_key_table are used (row pairs summed as described at k_tab_items).
// ---------------------------------------------------------------------------
constexpr int kPartMaxCtasPerSm = 8;   // phase-1 CTAs of 256 threads per SM, at most

struct PartArgs {
  uint16_t* items;               // phase-1 warp w, row j: region items + (w d + j) C
  uint32_t* cnts;                // phase-1 warp w: [16 w + j] part-0 items of row j, [16 w + 15] valid tuples
  const int64_t* col[5];         // column u of the window's first tuple
  int64_t W;                     // window capacity, a multiple of 256
  int64_t cnt;                   // tuples in the window, <= W
  int64_t C;                     // item slots per (warp, row) region: 32 x tiles per warp
  int nwarps;                    // warps of the phase-1 grid
  int logL;                      // part width 2^L
  const uint32_t* vbits;         // nullptr, or bit (i mod 32) of word i / 32: window tuple i is kept
};

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void st_u16_hint(uint16_t* ptr, uint16_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(ptr), "h"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ int64_t ld_key_policy(const int64_t* ptr, uint64_t pol) {
  int64_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
  return v;
}

// Key-table records in the 20-bit lane format above (d <= 9, one thread per domain key).
template <bool DEG1>
__global__ void __launch_bounds__(256) k_key_table_l20(UpdArgs p, TabArgs t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* s_coef = (uint64_t*)smem_raw;
  const int ncoef = p.d * p.row_len;
  for (int i = threadIdx.x; i < ncoef; i += blockDim.x) s_coef[i] = p.coef[i];
  __syncthreads();
  const int64_t total = t.base[p.a];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    int u = 0;
    while (u + 1 < p.a && g >= t.base[u + 1]) u++;
    const uint32_t x = (uint32_t)(g - t.base[u]);
    const uint64_t* cr = s_coef + t.off[u];
    uint64_t lane[3] = {0, 0, 0};
    uint32_t mask = 0;
#pragma unroll
    for (int r = 0; r < 9; r++) {
      if (r >= p.d) break;
      uint32_t par;
      const uint32_t b = key_row_hash<true, DEG1>(p, cr + (int64_t)r * p.row_len, p.deg[u], x, &par);
      lane[r / 3] |= (uint64_t)b << (20 * (r % 3));
      mask |= par << r;
    }
    uint4* out = (uint4*)(t.tbl + g * 8);
    out[0] = make_uint4((uint32_t)lane[0], (uint32_t)(lane[0] >> 32), (uint32_t)lane[1], (uint32_t)(lane[1] >> 32));
    out[1] = make_uint4((uint32_t)lane[2], (uint32_t)(lane[2] >> 32), 0u, mask);
  }
}

// Key-table records of 24 bytes (d <= 9, one thread per domain key): rows 3w .. 3w + 2 in
// 64-bit word w (w = 0, 1, 2), row r's lane at bit 22 (r mod 3): its bin (below 2^16) in the
// lane's bits 0..15 and its sign bit at lane bit 19.  Summing A <= 5 records word by word in
// 64 bits: the bins add up to below 5 2^16 < 2^19 in lane bits 0..18, so they never reach
// bit 19, and lane bit 19 of the sum is the parity of the signs (their sum, at most 5, fills
// lane bits 19..21; for the top lane, bits 63 and beyond, the carries leave the word).  So a
// row's bin sum mod m is (word >> 22 (r mod 3)) & (m - 1) and its sign product the bit above
// it at 19.  Five tables over 10^6 keys take 120 MB against 160 MB for 32-byte records, which
// keeps more of the Zipf tail in L2.  Record k (global index, 8-byte aligned) starts at 24 k:
// for even k its words 0 and 1 form the 16-byte-aligned pair and word 2 follows; for odd k
// the first 8 bytes hold word 2 and the aligned pair after it words 0 and 1, so a reader
// always takes words 0 and 1 with one 16-byte load and word 2 with one 8-byte load.
template <bool DEG1>
__global__ void __launch_bounds__(256) k_key_table_l24(UpdArgs p, TabArgs t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* s_coef = (uint64_t*)smem_raw;
  const int ncoef = p.d * p.row_len;
  for (int i = threadIdx.x; i < ncoef; i += blockDim.x) s_coef[i] = p.coef[i];
  __syncthreads();
  const int64_t total = t.base[p.a];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  uint64_t* tbl = (uint64_t*)t.tbl;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    int u = 0;
    while (u + 1 < p.a && g >= t.base[u + 1]) u++;
    const uint32_t x = (uint32_t)(g - t.base[u]);
    const uint64_t* cr = s_coef + t.off[u];
    uint64_t lane[3] = {0, 0, 0};
#pragma unroll
    for (int r = 0; r < 9; r++) {
      if (r >= p.d) break;
      uint32_t par;
      const uint32_t b = key_row_hash<true, DEG1>(p, cr + (int64_t)r * p.row_len, p.deg[u], x, &par);
      lane[r / 3] |= ((uint64_t)b | ((uint64_t)par << 19)) << (22 * (r % 3));
    }
    const bool odd = (g & 1) != 0;
    uint64_t* out = tbl + 3 * g;
    out[odd ? 1 : 0] = lane[0];
    out[odd ? 2 : 1] = lane[1];
    out[odd ? 0 : 2] = lane[2];
  }
}

// Words 0, 1 and 2 of 24-byte record k (layout above): one 16-byte and one 8-byte load.
__device__ __forceinline__ void ld_record24(const uint64_t* tbl, uint64_t k, uint64_t& w0, uint64_t& w1,
                                            uint64_t& w2) {
  const uint64_t odd = k & 1u;
  const uint64_t* r = tbl + 3 * k;
  asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(r + odd));
  asm("ld.global.nc.u64 %0, [%1];" : "=l"(w2) : "l"(r + 2 - 2 * odd));
}

// FMT 0: 20-bit lane records (d <= 9); FMT 2: 24-byte records (d <= 9, k_key_table_l24);
// FMT 1: narrow 16-bit records of 32 bytes (d <= 14):
// per record word holding the bins of rows 2j and 2j + 1, lo[j] adds the low halves (below
// 5 * 2^16: no overflow) and all[j] the whole words mod 2^32, so row 2j's sum is lo[j] mod
// 2^16 and row 2j + 1's is ((all[j] - lo[j]) >> 16) mod 2^16 (m divides 2^16).
// Persistent: each thread walks the window with the grid's stride, loading the keys of its
// next tuple before it gathers the records of the current one, so the key stream's latency
// overlaps the gathers.  Lanes of a warp take consecutive tuples (one tile) and iterate
// together (the ballots need the whole warp).  Four CTAs per SM (64 registers): with the
// running counts five (48 registers) spilled and took the star's F update from 3.10 to 3.84 ms;
// six for the instances of one or two attributes (40 registers, no spills) took a sub-query
// family's update from 8.45 to 9.22 ms.
template <int A, int FMT>
__global__ void __launch_bounds__(256, 4) k_tab_items(UpdArgs p, TabArgs t, PartArgs q) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int64_t gend = (q.cnt + 31) & ~(int64_t)31;
  const uint32_t mask = (uint32_t)p.m - 1u;
  const uint32_t low = (1u << q.logL) - 1u;
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  const int d = p.d;
  const uint64_t pol = policy_evict_first();
  const uint4* tbl = (const uint4*)t.tbl;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t rb = (uint32_t)(g >> 5) * (uint32_t)d;     // this warp's row-0 region index
  const uint32_t C = (uint32_t)q.C;
  // counts so far: lane j < d holds row j's part-0 items, lane 15 the valid tuples
  uint32_t cw = 0;
  // keys of the thread's next tuple, checked against their domains as they arrive: the
  // in-domain keys (< 2^31) as 32-bit values, bit u of okm set when key u is in its domain
  uint32_t kx[A], okm = 0;
#pragma unroll
  for (int u = 0; u < A; u++) {
    const int64_t k = g < q.cnt ? ld_key_policy(q.col[u] + g, pol) : -1;
    const bool kin = (uint64_t)k < (uint64_t)p.dom[u];
    okm |= (uint32_t)kin << u;
    kx[u] = kin ? (uint32_t)k : 0u;
  }
  for (; g < gend; g += step) {
    const bool in = g < q.cnt;
    const bool ok = in && okm == (1u << A) - 1u && (!q.vbits || ((q.vbits[g >> 5] >> lane) & 1u));
    uint32_t kg[A];   // global record indices (the host keeps this path's tables below 2^32 records)
#pragma unroll
    for (int u = 0; u < A; u++) kg[u] = (uint32_t)t.base[u] + kx[u];
    if (in && !ok) record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);   // left out of the tile below
    const int64_t gn = g + step;
    okm = 0;
#pragma unroll
    for (int u = 0; u < A; u++) {
      const int64_t k = gn < q.cnt ? ld_key_policy(q.col[u] + gn, pol) : -1;
      const bool kin = (uint64_t)k < (uint64_t)p.dom[u];
      okm |= (uint32_t)kin << u;
      kx[u] = kin ? (uint32_t)k : 0u;
    }
    const uint32_t vb = __ballot_sync(0xffffffffu, ok);
    const uint32_t nv = __popc(vb), rv = __popc(vb & lt);   // valid tuples in the tile / before this lane
    const uint32_t nval = __shfl_sync(0xffffffffu, cw, 15);  // valid tuples before the tile
    uint32_t add = nv;   // this tile's part-0 items of row `lane` (lane < d), its valid tuples (lane 15)
    // one row: with r1 the part-1 tuples before this lane, a part-0 tuple goes to slot
    // (part-0 items so far) + rv - r1 and a part-1 one to C - 1 - (part-1 items so far) - r1
    auto put = [&](int j, uint32_t bin, uint32_t neg) {
      const bool hi = (bin >> q.logL) != 0;
      const uint32_t hb = __ballot_sync(0xffffffffu, ok && hi);
      const uint32_t n1 = __popc(hb), r1 = __popc(hb & lt);
      const uint32_t c0 = __shfl_sync(0xffffffffu, cw, j);
      const uint32_t pos = hi ? C - 1u - (nval - c0) - r1 : c0 + rv - r1;
      // slot (rb + j) C + pos, formed here rather than kept as d row pointers across the
      // loop (registers)
      uint64_t slot;
      asm volatile("{\n\t.reg .u32 r;\n\tadd.u32 r, %1, %2;\n\tmad.wide.u32 %0, r, %3, %4;\n\t}"
                   : "=l"(slot) : "r"(rb), "r"((uint32_t)j), "r"(C), "l"((uint64_t)pos));
      if (ok) st_u16_hint(q.items + slot, (uint16_t)((bin & low) | (neg << 15)), pol);
      if (lane == (unsigned)j) add = nv - n1;
    };
    uint32_t sg = 0;
    if (FMT == 0) {
      uint64_t acc0 = 0, acc1 = 0, acc2 = 0;
      if (ok) {
#pragma unroll
        for (int u = 0; u < A; u++) {
          uint32_t w[8];
          ld_record32(tbl + (uint64_t)kg[u] * 2, w);
          acc0 += ((uint64_t)w[1] << 32) | w[0];
          acc1 += ((uint64_t)w[3] << 32) | w[2];
          acc2 += ((uint64_t)w[5] << 32) | w[4];
          sg ^= w[7];
        }
      }
#pragma unroll
      for (int j = 0; j < 9; j++) {
        if (j >= d) break;
        const uint64_t acc = j < 3 ? acc0 : (j < 6 ? acc1 : acc2);
        put(j, (uint32_t)(acc >> (20 * (j % 3))) & mask, (sg >> j) & 1u);
      }
    } else if (FMT == 2) {
      uint64_t acc0 = 0, acc1 = 0, acc2 = 0;
      if (ok) {
#pragma unroll
        for (int u = 0; u < A; u++) {
          uint64_t w0, w1, w2;
          ld_record24((const uint64_t*)t.tbl, kg[u], w0, w1, w2);
          acc0 += w0;
          acc1 += w1;
          acc2 += w2;
        }
      }
#pragma unroll
      for (int j = 0; j < 9; j++) {
        if (j >= d) break;
        const uint64_t acc = j < 3 ? acc0 : (j < 6 ? acc1 : acc2);
        const int sh = 22 * (j % 3);
        put(j, (uint32_t)(acc >> sh) & mask, (uint32_t)(acc >> (sh + 19)) & 1u);
      }
    } else {
      uint32_t lo[7], all[7];
#pragma unroll
      for (int j = 0; j < 7; j++) lo[j] = all[j] = 0;
      if (ok) {
#pragma unroll
        for (int u = 0; u < A; u++) {
          uint32_t w[8];
          ld_record32(tbl + (uint64_t)kg[u] * 2, w);
          sg ^= w[7];
#pragma unroll
          for (int j = 0; j < 7; j++) {
            lo[j] += w[j] & 0xffffu;
            all[j] += w[j];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 14; j++) {
        if (j >= d) break;
        const uint32_t sum = (j & 1) ? (all[j >> 1] - lo[j >> 1]) >> 16 : lo[j >> 1];
        put(j, sum & mask, (sg >> j) & 1u);
      }
    }
    cw += add;   // after the rows: their shuffles all read the counts before the tile
  }
  // the warp's counts: lane j < d row j's part-0 items, lane 15 the valid tuples
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (lane < (unsigned)d || lane == 15u) q.cnts[wg * 16 + lane] = cw;
}

// shared counter at saddr += v when x < n (unsigned): one compare, one predicated reduction
__device__ __forceinline__ void red_shared_if_lt(uint32_t saddr, int v, uint32_t x, uint32_t n) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %2, %3;\n\t@q red.shared.add.s32 [%0], %1;\n\t}"
               ::"r"(saddr), "r"(v), "r"(x), "r"(n) : "memory");
}

__device__ __forceinline__ void red_shared(uint32_t saddr, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

// The 8 items of one 16-byte chunk (two per 32-bit word: bin offset in bits 0..14, sign in
// bit 15) added into the shared counters at sbase; slots b .. b + 7 counted from the run's
// first item, those at or beyond n skipped.  A chunk wholly inside the run (every chunk but
// a run's first and last) goes without the per-slot compare.
__device__ __forceinline__ void add_chunk(uint32_t sbase, uint4 v, uint32_t b, uint32_t n) {
  const uint32_t e[4] = {v.x, v.y, v.z, v.w};
  if (n >= 8u && b <= n - 8u) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint32_t it = e[k >> 1] >> (16 * (k & 1));
      int neg;   // 0 or -1 from the item's sign bit
      asm("bfe.s32 %0, %1, 15, 1;" : "=r"(neg) : "r"(it));
      red_shared(sbase + ((it & 0x7fffu) << 2), neg | 1);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint32_t it = e[k >> 1] >> (16 * (k & 1));
      int neg;
      asm("bfe.s32 %0, %1, 15, 1;" : "=r"(neg) : "r"(it));
      red_shared_if_lt(sbase + ((it & 0x7fffu) << 2), neg | 1, b + (uint32_t)k, n);
    }
  }
}

// blockIdx.x = h + S (row + d c), S = m >> logL: part h of row `row` over the regions of the
// phase-1 warps [c R, min(c R + R, nwarps)), each region's part-h chunks (8 items, one 16-byte
// load) split into 2^logP pieces.  Warp k of the CTA takes pieces k, k + 32, ...; lane l of a
// warp takes the piece's chunks l, l + 32, ..., two per iteration, loads first.
__global__ void __launch_bounds__(1024) k_part_accum(PartArgs q, unsigned long long* ctr, int64_t m, int d,
                                                     int logL, int R, int logP) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* cnt = (int*)smem_raw;
  const int S = (int)(m >> logL);
  const int h = (int)(blockIdx.x % (unsigned)S);
  const int rest = (int)(blockIdx.x / (unsigned)S);
  const int row = rest % d;
  const int c = rest / d;
  const int L = 1 << logL;
  for (int k = threadIdx.x; k < L; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(cnt);
  const uint32_t lane = threadIdx.x & 31u;
  const int w0 = c * R;
  const int w1 = min(w0 + R, q.nwarps);
  const int npc = (w1 - w0) << logP;
  const uint32_t C = (uint32_t)q.C;
  // slots b .. b + 7 counted from the part's first item: add the signs of those below n
  auto unit = [&](uint4 v, uint32_t b, uint32_t n) { add_chunk(sbase, v, b, n); };
  for (int pc = (int)(threadIdx.x >> 5); pc < npc; pc += (int)(blockDim.x >> 5)) {
    const int w = w0 + (pc >> logP);
    const uint32_t piece = (uint32_t)pc & ((1u << logP) - 1u);
    const uint32_t n0 = q.cnts[(int64_t)w * 16 + row], nv = q.cnts[(int64_t)w * 16 + 15];
    const uint32_t n = h ? nv - n0 : n0;         // part h's items in this region
    const uint32_t lo = h ? C - n : 0u;          // and the first of them
    const uint32_t kb = lo >> 3, nk = ((lo + n + 7) >> 3) - kb;
    const uint32_t ke = kb + (uint32_t)(((uint64_t)nk * (piece + 1)) >> logP);
    uint32_t k = kb + (uint32_t)(((uint64_t)nk * piece) >> logP) + lane;
    const uint16_t* rg = q.items + ((int64_t)w * d + row) * q.C;
    for (; k + 32 < ke; k += 64) {
      const uint4 v1 = *(const uint4*)(rg + 8 * k);
      const uint4 v2 = *(const uint4*)(rg + 8 * (k + 32));
      unit(v1, 8 * k - lo, n);
      unit(v2, 8 * (k + 32) - lo, n);
    }
    if (k < ke) unit(*(const uint4*)(rg + 8 * k), 8 * k - lo, n);
  }
  __syncthreads();
  unsigned long long* out = ctr + (int64_t)row * m + ((int64_t)h << logL);
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const int v = cnt[k];
    if (v != 0) red_add_global(out + k, (unsigned long long)(int64_t)v);
  }
}

// CTAs of k_tab_items<A, FMT> per SM (no shared memory: the whole unified array is left to
// L1, which caches the hot records).
template <int A, int FMT>
cudaError_t tab_items_per_sm(int* per_sm) {
  auto kern = k_tab_items<A, FMT>;
  cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, 256, 0);
  *per_sm = std::max(1, std::min(*per_sm, kPartMaxCtasPerSm));
  return e;
}

template <int FMT>
cudaError_t tab_items_occupancy(int A, int* per_sm) {
  switch (A) {
    case 1: return tab_items_per_sm<1, FMT>(per_sm);
    case 2: return tab_items_per_sm<2, FMT>(per_sm);
    case 3: return tab_items_per_sm<3, FMT>(per_sm);
    case 4: return tab_items_per_sm<4, FMT>(per_sm);
    default: return tab_items_per_sm<5, FMT>(per_sm);
  }
}

template <int FMT>
cudaError_t dispatch_tab_items(const UpdArgs& a, const TabArgs& t, const PartArgs& q, int grid, cudaStream_t st) {
  switch (a.a) {
    case 1: k_tab_items<1, FMT><<<grid, 256, 0, st>>>(a, t, q); break;
    case 2: k_tab_items<2, FMT><<<grid, 256, 0, st>>>(a, t, q); break;
    case 3: k_tab_items<3, FMT><<<grid, 256, 0, st>>>(a, t, q); break;
    case 4: k_tab_items<4, FMT><<<grid, 256, 0, st>>>(a, t, q); break;
    default: k_tab_items<5, FMT><<<grid, 256, 0, st>>>(a, t, q); break;
  }
  count_launch();
  return cudaGetLastError();
}

// SK_PART_UPDATE=0 keeps the single-phase k_update_tab (and the per-tuple update) for batches
// the partitioned updates could take; =2 gives the wide partitioned update every batch whose
// width, rows, arity and weights it accepts, whatever the sketch's size and the batch length.
// SK_PART_WINDOW caps the tuples per window (default and largest: 2^30, which keeps every
// shared-memory counter of k_part_accum below 2^31 in magnitude; 2^24 for the wide update).
int part_update_mode() {
  const char* v = std::getenv("SK_PART_UPDATE");
  return (v && v[0] == '0') ? 0 : ((v && v[0] == '2') ? 2 : 1);
}

// SK_PART_RECORD=32 takes the 32-byte 20-bit lane records instead of the 24-byte ones for d <= 9.
int part_record_bytes() {
  const char* v = std::getenv("SK_PART_RECORD");
  return (v && std::atoi(v) == 32) ? 32 : 24;
}

int64_t part_window(int64_t n) {
  const char* v = std::getenv("SK_PART_WINDOW");
  const long long x = v ? std::atoll(v) : 0;
  const int64_t cap = (x > 0 && x < (1ll << 30)) ? (int64_t)x : ((int64_t)1 << 30);
  return std::min<int64_t>((n + 255) / 256 * 256, (cap + 255) / 256 * 256);
}

// Regions of a window of W tuples: the phase-1 grid has at most sms x kPartMaxCtasPerSm CTAs
// of 256 threads, so its warps' regions hold at most W + that many threads' tiles per row.
size_t part_items_bytes(int d, int64_t W, int sms) {
  const int64_t threads = (int64_t)sms * kPartMaxCtasPerSm * 256;
  return ((size_t)d * (size_t)(W + threads) * sizeof(uint16_t) + 255) & ~(size_t)255;
}

size_t part_staging_bytes(int d, int64_t W, int sms) {
  return part_items_bytes(d, W, sms) + (size_t)sms * kPartMaxCtasPerSm * 8 * 16 * sizeof(uint32_t);
}

// Both phases over every window of the batch; staging (part_staging_bytes) is caller-owned.
// colp: the first tuple's key of each of the a.a attributes (nullptr: a.cols + u a.stride).
// vbits: nullptr, or one bit per batch tuple (bit i mod 32 of word i / 32) that must be set
// for the tuple to be added.
cudaError_t run_partitioned(const UpdArgs& a, const TabArgs& t, int fmt, void* staging, int sms, cudaStream_t st,
                            const int64_t* const* colp = nullptr, const uint32_t* vbits = nullptr) {
  const int64_t n = a.n;
  int tab_per_sm = 1;
  cudaError_t e = fmt == 0   ? tab_items_occupancy<0>(a.a, &tab_per_sm)
                  : fmt == 2 ? tab_items_occupancy<2>(a.a, &tab_per_sm)
                             : tab_items_occupancy<1>(a.a, &tab_per_sm);
  if (e != cudaSuccess) return e;
  const int64_t full_grid = (int64_t)sms * tab_per_sm;
  const int64_t W = part_window(n);
  PartArgs q;
  q.items = (uint16_t*)staging;
  q.cnts = (uint32_t*)((char*)staging + part_items_bytes(a.d, W, sms));
  q.W = W;
  int logm = 0;
  while (((int64_t)1 << logm) < (int64_t)a.m) logm++;
  const int logL = std::min(logm, 15);
  q.logL = logL;
  const int S = (int)(a.m >> logL);
  const size_t smem = (size_t)4 << logL;
  e = allow_dynamic_smem((const void*)k_part_accum);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_part_accum, 1024, smem);
  const int64_t slots = (int64_t)sms * std::max(1, per_sm);
  const int64_t units = (int64_t)S * a.d;
  for (int64_t i0 = 0; i0 < n && e == cudaSuccess; i0 += W) {
    q.cnt = std::min(W, n - i0);
    for (int u = 0; u < 5; u++)
      q.col[u] = u < a.a ? (colp ? colp[u] : a.cols + (int64_t)u * a.stride) + i0 : nullptr;
    q.vbits = vbits ? vbits + i0 / 32 : nullptr;   // windows start at multiples of 256
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((q.cnt + 255) / 256, full_grid));
    const int64_t gend = (q.cnt + 31) / 32 * 32;
    q.C = 32 * ((gend + (int64_t)grid * 256 - 1) / ((int64_t)grid * 256));
    q.nwarps = grid * 8;
    e = fmt == 0   ? dispatch_tab_items<0>(a, t, q, grid, st)
        : fmt == 2 ? dispatch_tab_items<2>(a, t, q, grid, st)
                   : dispatch_tab_items<1>(a, t, q, grid, st);
    if (e != cudaSuccess) break;
    // ranges of phase-1 warps per (row, part): the grid a whole number of waves when that
    // takes 2..64 waves; pieces per region so that a CTA's 32 warps get equal shares
    int64_t nr = 0;
    for (int64_t k = 2; k <= 64 && !nr; k++)
      if ((k * slots) % units == 0) nr = k * slots / units;
    if (!nr) nr = (4 * slots + units - 1) / units;
    nr = std::max<int64_t>(1, std::min<int64_t>(nr, q.nwarps));
    const int R = (int)((q.nwarps + nr - 1) / nr);
    nr = (q.nwarps + R - 1) / R;
    int logP = 3;
    for (int lp = 0; lp < 3; lp++) {
      const int64_t pcs = (int64_t)R << lp;
      if ((pcs + 31) / 32 * 32 * 100 <= pcs * 105) {
        logP = lp;
        break;
      }
    }
    k_part_accum<<<(unsigned)(units * nr), 1024, smem, st>>>(q, a.ctr, (int64_t)a.m, a.d, logL, R, logP);
    count_launch();
    e = cudaGetLastError();
  }
  return e;
}

// ---------------------------------------------------------------------------
// Partitioned update for wide sketches (unit weights, power-of-two 2^17 <= m <= 2^24, d <= 16,
// at most 5 attributes, declared domains: the chain of eight relations at m = 2^20).  A d x m
// int64 sketch of 128 MB does not stay in L2, and one 64-bit reduction per (tuple, row) then
// waits on DRAM.  Each row's bins are split into S = m / 2^15 parts of 2^15 bins (the int32
// counters of one part fill 128 KB of one SM's shared memory); the items of a window are
// sorted by part in four steps:
//   1. k_wide_items: one CTA per chunk of kWideChunk tuples gathers the A key-table records
//      (wide format: one 32-bit word per row, bin in bits 0..30, sign in bit 31) of each tuple,
//      writes row j's item (bin mod m | sign << 31; 0x7fffffff for a tuple left out for a key
//      outside its domain) to plane[j][i] and counts each row's items per part in shared
//      memory; the counts go to H[(j S + b) nchunk + c];
//   2. an exclusive scan of H (k_scan_*) into OFF: OFF[(j S + b) nchunk + c] is the first
//      position of chunk c's part-b items of row j in the sorted item array, whose row-major,
//      part-major order the flat scan gives;
//   3. k_wide_scatter: per (chunk, row) the chunk's items ranked within their parts in shared
//      memory (16-bit: offset within the part | sign << 15) and written out part by part,
//      each part's run contiguous;
//   4. k_wide_plan lists the phase-2 CTAs (heavy parts split over several), and in
//      k_wide_accum a CTA owns part b of row j as 2^15 int32 counters over a range of that
//      part's items, adds with shared-memory atomics and adds each counter into the int64
//      sketch with one 64-bit reduction.
// Every counter receives the same integer sum as with one reduction per (tuple, row).
// ---------------------------------------------------------------------------
constexpr int kWideChunk = 4096;   // tuples per phase-1 CTA (256 threads x 16; 2048: chain8 update 9.04 vs 8.72 ms)
constexpr int kWideMaxRows = 16;
constexpr int kWideMaxParts = 512;  // m <= 2^24

struct WideArgs {
  uint32_t* plane;     // [d][W] 32-bit items of the window
  uint16_t* sorted;    // [d W + 8] 16-bit items, row-major then part-major
  uint32_t* H;         // [d][S][nchunk] per-chunk part counts
  uint32_t* OFF;       // [d][S][nchunk] their exclusive scan: first position in `sorted`
  uint32_t* bsum;      // scan block sums
  uint4* plan;         // phase-2 work: per CTA (row j * S + part b, first item, end, heavy); plan_n[0] CTAs
  uint32_t* plan_n;
  int64_t W;           // window capacity
  int64_t cnt;         // tuples in the window
  const int64_t* col[5];
  int nchunk;
  int S;
};

// Per tuple the A records' vectors are all loaded before any is summed (up to 4 x A vectors
// in flight; A <= 2, the chain's relations), and the next tuple's keys are loaded before this
// tuple's records.
template <int A>
__global__ void __launch_bounds__(256) k_wide_items(UpdArgs p, TabArgs t, WideArgs q) {
  __shared__ uint32_t hist[kWideMaxRows * kWideMaxParts];
  constexpr int VH = A <= 2 ? 4 : 1;   // vectors loaded together per record
  const int d = p.d, S = q.S;
  for (int k = threadIdx.x; k < d * S; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const uint32_t mask = (uint32_t)p.m - 1u;
  const int rv = (d + 3) >> 2;   // 16-byte vectors per record
  const int64_t c0 = (int64_t)blockIdx.x * kWideChunk;
  const int64_t cend = c0 + kWideChunk < q.cnt ? c0 + kWideChunk : q.cnt;
  int64_t i = c0 + threadIdx.x;
  int64_t key[A];
#pragma unroll
  for (int u = 0; u < A; u++) key[u] = i < cend ? ld_key_stream(q.col[u] + i) : 0;
  for (; i < cend; i += 256) {
    bool ok = true;
    const uint4* rec[A];
#pragma unroll
    for (int u = 0; u < A; u++) {
      const bool kin = (uint64_t)key[u] < (uint64_t)p.dom[u];
      ok = ok && kin;
      rec[u] = (const uint4*)t.tbl + ((uint64_t)t.base[u] + (kin ? (uint64_t)key[u] : 0ull)) * (uint64_t)t.rvec;
    }
    const int64_t inext = i + 256;
#pragma unroll
    for (int u = 0; u < A; u++) key[u] = inext < cend ? ld_key_stream(q.col[u] + inext) : 0;
    if (!ok) record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
    for (int v0 = 0; v0 < rv; v0 += VH) {
      uint4 w[VH][A];
#pragma unroll
      for (int vh = 0; vh < VH; vh++)
#pragma unroll
        for (int u = 0; u < A; u++)
          w[vh][u] = (ok && v0 + vh < rv) ? __ldg(rec[u] + v0 + vh) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int vh = 0; vh < VH; vh++) {
        uint32_t acc[4] = {0, 0, 0, 0}, sg[4] = {0, 0, 0, 0};
#pragma unroll
        for (int u = 0; u < A; u++) {
          const uint32_t e[4] = {w[vh][u].x, w[vh][u].y, w[vh][u].z, w[vh][u].w};
#pragma unroll
          for (int h = 0; h < 4; h++) {
            acc[h] += e[h] & 0x7fffffffu;
            sg[h] ^= e[h] >> 31;
          }
        }
#pragma unroll
        for (int h = 0; h < 4; h++) {
          const int j = 4 * (v0 + vh) + h;
          if (j < d) {
            const uint32_t bin = acc[h] & mask;
            q.plane[(int64_t)j * q.W + i] = ok ? (bin | (sg[h] << 31)) : 0x7fffffffu;
            if (ok) atomicAdd(&hist[j * S + (int)(bin >> 15)], 1u);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d * S; k += blockDim.x) q.H[(int64_t)k * q.nchunk + blockIdx.x] = hist[k];
}

// Exclusive scan of n uint32: k_scan_blocks scans blocks of 4096 of `in` (4 per thread) into
// `out` and leaves each block's total in bsum; k_scan_sums scans bsum (one CTA); k_scan_add
// adds the scanned totals to `out`.
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31u) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < (blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= (unsigned)o) s += y;
    }
    s_warp[lane] = s;   // inclusive warp totals
  }
  __syncthreads();
  const uint32_t before = wid ? s_warp[wid - 1] : 0u;
  *total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* bsum) {
  __shared__ uint32_t s_warp[32];
  const int64_t base = (int64_t)blockIdx.x * 4096 + (int64_t)threadIdx.x * 4;
  uint32_t v[4], sum = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    v[k] = base + k < n ? in[base + k] : 0u;
    sum += v[k];
  }
  uint32_t total;
  uint32_t run = block_excl_scan_1024(sum, s_warp, &total);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t* bsum, int nb) {
  __shared__ uint32_t s_warp[32];
  uint32_t carry = 0;
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int i = b0 + (int)threadIdx.x;
    const uint32_t v = i < nb ? bsum[i] : 0u;
    uint32_t total;
    const uint32_t x = block_excl_scan_1024(v, s_warp, &total);
    if (i < nb) bsum[i] = carry + x;
    carry += total;
  }
}

__global__ void __launch_bounds__(1024) k_scan_add(uint32_t* a, int64_t n, const uint32_t* bsum) {
  const int64_t base = (int64_t)blockIdx.x * 4096;
  const uint32_t off = bsum[blockIdx.x];
  for (int k = threadIdx.x; k < 4096; k += blockDim.x)
    if (base + k < n) a[base + k] += off;
}

// blockIdx.x = chunk c, blockIdx.y = row j.  Chunk c's items of row j ranked within their
// parts (a shared-memory counter per part), staged in part order, then written part by part.
__global__ void __launch_bounds__(256) k_wide_scatter(WideArgs q, int64_t m) {
  __shared__ uint32_t lstart[kWideMaxParts], rank[kWideMaxParts], gpos[kWideMaxParts];
  __shared__ uint32_t s_pk[kWideChunk];   // item | part << 16
  __shared__ uint32_t s_warp[32];
  const int c = blockIdx.x, j = blockIdx.y, S = q.S;
  // this chunk's part counts (S <= 512: two per thread), their exclusive scan
  uint32_t n2[2] = {0u, 0u};
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int b = 2 * (int)threadIdx.x + h;
    if (b < S) {
      const int64_t k = ((int64_t)j * S + b) * q.nchunk + c;
      n2[h] = q.H[k];
      gpos[b] = q.OFF[k];
    }
  }
  uint32_t total;
  const uint32_t ex = block_excl_scan_1024(n2[0] + n2[1], s_warp, &total);
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int b = 2 * (int)threadIdx.x + h;
    if (b < S) {
      lstart[b] = ex + (h ? n2[0] : 0u);
      rank[b] = 0u;
    }
  }
  __syncthreads();
  const int64_t i0 = (int64_t)c * kWideChunk;
  const uint32_t low = (1u << 15) - 1u;
  for (int k = threadIdx.x; k < kWideChunk; k += blockDim.x) {
    const int64_t i = i0 + k;
    if (i >= q.cnt) break;
    const uint32_t it = q.plane[(int64_t)j * q.W + i];
    const uint32_t bin = it & 0x7fffffffu;
    if (bin < (uint32_t)m) {
      const uint32_t b = bin >> 15;
      const uint32_t lp = lstart[b] + atomicAdd(&rank[b], 1u);
      s_pk[lp] = (bin & low) | ((it >> 31) << 15) | (b << 16);
    }
  }
  __syncthreads();
  for (uint32_t lp = threadIdx.x; lp < total; lp += blockDim.x) {
    const uint32_t pk = s_pk[lp], b = pk >> 16;
    q.sorted[gpos[b] + (lp - lstart[b])] = (uint16_t)pk;
  }
}

// Phase-2 work list: part b of row j gets ceil(items / B) CTAs over equal ranges of its items
// (B = twice the mean part's items, at least 2^16), so a part that a heavy bin makes large is
// spread over several SMs; a CTA of such a part is marked heavy.  One CTA of 1024 threads:
// entries e = j S + b, scanned in rounds of 1024.
__global__ void __launch_bounds__(1024) k_wide_plan(WideArgs q, int d, uint32_t B, uint32_t maxc) {
  __shared__ uint32_t s_warp[32];
  const int64_t ne = (int64_t)d * q.S;
  const int64_t last = ne * q.nchunk - 1;
  uint32_t carry = 0;
  for (int64_t e0 = 0; e0 < ne; e0 += 1024) {
    const int64_t e = e0 + threadIdx.x;
    uint32_t P0 = 0, P1 = 0, k = 0;
    if (e < ne) {
      P0 = q.OFF[e * q.nchunk];
      P1 = e + 1 < ne ? q.OFF[(e + 1) * q.nchunk] : q.OFF[last] + q.H[last];
      k = (P1 - P0 + B - 1) / B;
    }
    uint32_t total;
    const uint32_t first = carry + block_excl_scan_1024(k, s_warp, &total);
    for (uint32_t r = 0; r < k; r++) {
      if (first + r >= maxc) break;
      const uint32_t lo = P0 + (uint32_t)(((uint64_t)(P1 - P0) * r) / k);
      const uint32_t hi = P0 + (uint32_t)(((uint64_t)(P1 - P0) * (r + 1)) / k);
      q.plan[first + r] = make_uint4((uint32_t)e, lo, hi, k > 1 ? 1u : 0u);
    }
    carry += total;
  }
  if (threadIdx.x == 0) q.plan_n[0] = carry < maxc ? carry : maxc;
}

// One CTA per work-list entry (CTAs past the list's length return at once): part b of row j as
// 2^15 int32 counters over its items [lo, hi) of `sorted`.  Lanes take consecutive 8-item
// chunks, two per iteration.  In a heavy CTA each lane first merges runs of equal items among
// its 8 (a heavy bin's items make most of such a part) and adds each run with one atomic.
__global__ void __launch_bounds__(1024) k_wide_accum(WideArgs q, unsigned long long* ctr, int64_t m) {
  if (blockIdx.x >= q.plan_n[0]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* cnt = (int*)smem_raw;
  const uint4 wk = q.plan[blockIdx.x];
  const int S = q.S;
  const int j = (int)(wk.x / (uint32_t)S), b = (int)(wk.x % (uint32_t)S);
  const uint32_t lo = wk.y, hi = wk.z;
  const bool heavy = wk.w != 0;
  constexpr int L = 1 << 15;
  for (int k = threadIdx.x; k < L; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  const uint32_t n = hi - lo;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(cnt);
  // slots bo .. bo + 7 counted from lo: add those below n
  auto unit = [&](uint4 v, uint32_t bo) { add_chunk(sbase, v, bo, n); };
  auto unit_merge = [&](uint4 v, uint32_t bo) {
    const uint32_t e[4] = {v.x, v.y, v.z, v.w};
    uint32_t prev = 0xffffffffu;   // no item has bits 16..31 set
    int run = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint32_t it = (e[k >> 1] >> (16 * (k & 1))) & 0xffffu;
      const bool valid = bo + (uint32_t)k < n;
      const int sv = (it >> 15) ? -1 : 1;
      if (valid && it == prev) {
        run += sv;
      } else if (valid) {
        if (run != 0) atomicAdd(cnt + (prev & 0x7fffu), run);
        prev = it;
        run = sv;
      }
    }
    if (run != 0) atomicAdd(cnt + (prev & 0x7fffu), run);
  };
  const uint32_t ke = (hi + 7) >> 3;
  uint32_t k = (lo >> 3) + threadIdx.x;
  if (heavy) {
    for (; k < ke; k += blockDim.x) unit_merge(*(const uint4*)(q.sorted + 8 * (size_t)k), 8 * k - lo);
  } else {
    for (; k + blockDim.x < ke; k += 2 * blockDim.x) {
      const uint4 v1 = *(const uint4*)(q.sorted + 8 * (size_t)k);
      const uint4 v2 = *(const uint4*)(q.sorted + 8 * (size_t)(k + blockDim.x));
      unit(v1, 8 * k - lo);
      unit(v2, 8 * (k + blockDim.x) - lo);
    }
    if (k < ke) unit(*(const uint4*)(q.sorted + 8 * (size_t)k), 8 * k - lo);
  }
  __syncthreads();
  unsigned long long* out = ctr + (int64_t)j * m + ((int64_t)b << 15);
  for (int x = threadIdx.x; x < L; x += blockDim.x) {
    const int v = cnt[x];
    if (v != 0) red_add_global(out + x, (unsigned long long)(int64_t)v);
  }
}

// Window capacity of the wide partitioned update: positions in `sorted` stay below 2^28.
int64_t wide_window(int64_t n) {
  const char* v = std::getenv("SK_PART_WINDOW");
  const long long x = v ? std::atoll(v) : 0;
  const int64_t cap = (x > 0 && x < (1ll << 24)) ? (int64_t)x : ((int64_t)1 << 24);
  return std::min<int64_t>((n + 255) / 256 * 256, (cap + 255) / 256 * 256);
}

struct WideLayout {
  size_t plane, sorted, H, OFF, bsum, plan, plan_n, total;
  uint32_t maxc;   // phase-2 work-list capacity
};

WideLayout wide_layout(int d, int64_t m, int64_t W) {
  const int S = (int)(m >> 15);
  const int64_t nchunk = (W + kWideChunk - 1) / kWideChunk;
  const int64_t N = (int64_t)d * S * nchunk;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  WideLayout L;
  L.plane = 0;
  L.sorted = L.plane + al((size_t)d * W * sizeof(uint32_t));
  L.H = L.sorted + al(((size_t)d * W + 8) * sizeof(uint16_t));
  L.OFF = L.H + al((size_t)N * sizeof(uint32_t));
  L.bsum = L.OFF + al((size_t)N * sizeof(uint32_t));
  L.plan = L.bsum + al((size_t)((N + 4095) / 4096) * sizeof(uint32_t));
  // at most one CTA per (row, part) plus one per 2^16 items
  L.maxc = (uint32_t)((int64_t)d * S + ((int64_t)d * W >> 16) + 1);
  L.plan_n = L.plan + al((size_t)L.maxc * sizeof(uint4));
  L.total = L.plan_n + 256;
  return L;
}

template <int A>
void launch_wide_items(const UpdArgs& a, const TabArgs& t, const WideArgs& q, cudaStream_t st) {
  k_wide_items<A><<<q.nchunk, 256, 0, st>>>(a, t, q);
}

// All four steps over every window of the batch; staging (wide_layout(...).total bytes for
// the window wide_window(n)) is caller-owned.
cudaError_t run_wide_partitioned(const UpdArgs& a, const TabArgs& t, void* staging, int sms, cudaStream_t st) {
  const int64_t n = a.n;
  const int64_t W = wide_window(n);
  const WideLayout Ly = wide_layout(a.d, (int64_t)a.m, W);
  char* base = (char*)staging;
  WideArgs q;
  q.plane = (uint32_t*)(base + Ly.plane);
  q.sorted = (uint16_t*)(base + Ly.sorted);
  q.H = (uint32_t*)(base + Ly.H);
  q.OFF = (uint32_t*)(base + Ly.OFF);
  q.bsum = (uint32_t*)(base + Ly.bsum);
  q.plan = (uint4*)(base + Ly.plan);
  q.plan_n = (uint32_t*)(base + Ly.plan_n);
  q.W = W;
  q.S = (int)(a.m >> 15);
  const size_t smem = (size_t)4 << 15;
  cudaError_t e = allow_dynamic_smem((const void*)k_wide_accum);
  const int64_t units = (int64_t)q.S * a.d;
  (void)sms;
  for (int64_t i0 = 0; i0 < n && e == cudaSuccess; i0 += W) {
    q.cnt = std::min(W, n - i0);
    for (int u = 0; u < 5; u++) q.col[u] = u < a.a ? a.cols + (int64_t)u * a.stride + i0 : nullptr;
    q.nchunk = (int)((q.cnt + kWideChunk - 1) / kWideChunk);
    switch (a.a) {
      case 1: launch_wide_items<1>(a, t, q, st); break;
      case 2: launch_wide_items<2>(a, t, q, st); break;
      case 3: launch_wide_items<3>(a, t, q, st); break;
      case 4: launch_wide_items<4>(a, t, q, st); break;
      default: launch_wide_items<5>(a, t, q, st); break;
    }
    const int64_t N = units * q.nchunk;
    const int nb = (int)((N + 4095) / 4096);
    k_scan_blocks<<<nb, 1024, 0, st>>>(q.H, q.OFF, N, q.bsum);
    k_scan_sums<<<1, 1024, 0, st>>>(q.bsum, nb);
    k_scan_add<<<nb, 1024, 0, st>>>(q.OFF, N, q.bsum);
    k_wide_scatter<<<dim3((unsigned)q.nchunk, (unsigned)a.d), 256, 0, st>>>(q, (int64_t)a.m);
    // phase-2 work: B = twice the mean part's items (at least 2^16) per CTA
    const uint32_t B = (uint32_t)std::max<int64_t>((int64_t)1 << 16, 2 * (q.cnt * a.d) / std::max<int64_t>(1, units));
    const uint32_t maxc = (uint32_t)std::min<int64_t>((int64_t)Ly.maxc, units + ((int64_t)a.d * q.cnt) / B + 1);
    k_wide_plan<<<1, 1024, 0, st>>>(q, a.d, B, maxc);
    k_wide_accum<<<maxc, 1024, smem, st>>>(q, a.ctr, (int64_t)a.m);
    count_launch(7);
    e = cudaGetLastError();
  }
  return e;
}

// SK_TAB_V8=0 reads 32-byte key-table records as two 16-byte loads instead of one.
bool tab_v8_enabled() {
  const char* v = std::getenv("SK_TAB_V8");
  return !(v && v[0] == '0');
}

template <int A, bool POW2, bool SMEM>
cudaError_t launch_tab(const UpdArgs& a, const TabArgs& t, int grid, size_t smem, cudaStream_t st) {
  const bool v8 = t.rvec == 2 && tab_v8_enabled();
  auto kern = t.narrow ? (v8 ? k_update_tab<A, POW2, SMEM, true, true> : k_update_tab<A, POW2, SMEM, true, false>)
                       : (v8 ? k_update_tab<A, POW2, SMEM, false, true> : k_update_tab<A, POW2, SMEM, false, false>);
  cudaError_t e = fit_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, smem, st>>>(a, t);
  count_launch();
  return cudaGetLastError();
}

template <bool POW2, bool SMEM>
cudaError_t dispatch_tab(const UpdArgs& a, const TabArgs& t, int grid, size_t smem, cudaStream_t st) {
  switch (a.a) {
    case 1: return launch_tab<1, POW2, SMEM>(a, t, grid, smem, st);
    case 2: return launch_tab<2, POW2, SMEM>(a, t, grid, smem, st);
    case 3: return launch_tab<3, POW2, SMEM>(a, t, grid, smem, st);
    case 4: return launch_tab<4, POW2, SMEM>(a, t, grid, smem, st);
    case 5: return launch_tab<5, POW2, SMEM>(a, t, grid, smem, st);
    default: return launch_tab<0, POW2, SMEM>(a, t, grid, smem, st);
  }
}

// CTAs per SM of the global-atomic update grid.  Default: one tuple per thread (a grid of
// n / 256 CTAs), which measured fastest on the 1e8-row star fact table (12.18 ms, against
// 13.01 / 12.80 / 12.45 / 12.28 ms for 6 / 8 / 16 / 32 grid-stride CTAs per SM);
// SK_UPDATE_GRID=<n> caps the grid at n CTAs per SM instead.
int update_grid_per_sm(int resident) {
  (void)resident;
  const char* v = std::getenv("SK_UPDATE_GRID");
  const int x = v ? std::atoi(v) : 0;
  return x <= 0 ? (1 << 30) / 64 : x;
}

// true when each of the relation's A attributes is in exactly one join
bool all_deg1(const UpdArgs& a) {
  if (a.a < 1) return false;
  for (int u = 0; u < a.a; u++)
    if (a.deg[u] != 1) return false;
  return true;
}

// grid <= 0 sizes the grid with update_grid_per_sm.
template <int A, bool POW2, bool SMEM>
cudaError_t launch_one(const UpdArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = (A > 0 && all_deg1(a)) ? k_update<A, POW2, SMEM, (A > 0)> : k_update<A, POW2, SMEM, false>;
  cudaError_t e = allow_dynamic_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  if (grid <= 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (a.n + 255) / 256;
    const int mult = update_grid_per_sm(std::max(1, per_sm));
    const int64_t cap = std::min<int64_t>((int64_t)mult * std::max(1, sms), 0x7fffffff);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
  }
  kern<<<grid, 256, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <bool POW2, bool SMEM>
cudaError_t dispatch_a(const UpdArgs& a, int grid, size_t smem, cudaStream_t st) {
  switch (a.a) {
    case 1: return launch_one<1, POW2, SMEM>(a, grid, smem, st);
    case 2: return launch_one<2, POW2, SMEM>(a, grid, smem, st);
    case 3: return launch_one<3, POW2, SMEM>(a, grid, smem, st);
    case 4: return launch_one<4, POW2, SMEM>(a, grid, smem, st);
    case 5: return launch_one<5, POW2, SMEM>(a, grid, smem, st);
    default: return launch_one<0, POW2, SMEM>(a, grid, smem, st);
  }
}

// ---------------------------------------------------------------------------
// Hot-key cached update (power-of-two m, d <= 32, global atomics).
//
// Skewed key columns (the Zipf-like columns of Figure 5) repeat a few keys very
// often.  Each CTA keeps, per attribute, a direct-mapped table of S keys with
// their per-row results (bin value mod m and sign parity).  The table is filled
// from the CTA's first tuples (first come, first kept; no eviction), then frozen.
// A warp works on 32 tuples at a time: attributes whose key is in the table take
// the stored results; the other (tuple, attribute) pairs are queued and hashed by
// the whole warp densely, one pair per lane, their per-row results accumulated
// into per-tuple shared-memory partial sums.  Every counter update is identical to
// the uncached kernel's.
// ---------------------------------------------------------------------------
constexpr uint64_t kEmptyKey = ~0ull;

__device__ __forceinline__ uint32_t cache_slot(uint64_t x, int log2s) {
  return (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> (64 - log2s));
}

struct CacheLayout {
  int log2s;        // table slots per attribute = 2^log2s
  int fill_groups;  // 32-tuple groups per warp used to fill the table
};

template <int A, bool FILL>
__device__ __forceinline__ void cached_group(const UpdArgs& p, const CacheLayout& c, int64_t i0, int64_t i1,
                                             const uint64_t* s_coef, const int* s_off, uint64_t* cx,
                                             uint32_t* cdata, uint32_t* sbin, uint32_t* ssign, uint64_t* qx,
                                             uint16_t* qtu) {
  const int lane = threadIdx.x & 31;
  const int d = p.d;
  const int S = 1 << c.log2s;
  const int64_t i = i0 + lane;
  bool valid = i < i1;
  uint64_t x[A];
#pragma unroll
  for (int u = 0; u < A; u++) {
    const int64_t key = valid ? __ldg(p.cols + (int64_t)u * p.stride + i) : 0;
    if (valid && p.has_dom && (key < 0 || key >= p.dom[u])) {
      record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
      valid = false;
    }
    x[u] = field_of(key);
  }
  const int64_t delta = valid ? (p.w ? __ldg(p.w + i) : 1) : 0;
  uint32_t slot[A];
  uint32_t hitmask = 0;
#pragma unroll
  for (int u = 0; u < A; u++) {
    slot[u] = cache_slot(x[u], c.log2s);
    if (!FILL && valid && cx[u * S + slot[u]] == x[u]) hitmask |= 1u << u;
  }
  uint32_t* my_bin = sbin + lane * d;
  for (int r = 0; r < d; r++) my_bin[r] = 0;
  ssign[lane] = 0;
  int qn = 0;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int u = 0; u < A; u++) {
    const bool miss = valid && !((hitmask >> u) & 1u);
    const uint32_t bal = __ballot_sync(0xffffffffu, miss);
    if (miss) {
      const int pos = qn + __popc(bal & lt);
      qx[pos] = x[u];
      qtu[pos] = (uint16_t)(lane | (u << 5));
    }
    qn += __popc(bal);
  }
  __syncwarp();
  for (int j = lane; j < qn; j += 32) {
    const uint64_t xv = qx[j];
    const int t = qtu[j] & 31, u = qtu[j] >> 5;
    const uint32_t sl = cache_slot(xv, c.log2s);
    const bool claim = FILL && atomicCAS((unsigned long long*)&cx[u * S + sl], kEmptyKey, xv) == kEmptyKey;
    const int off = s_off[u];
    const int deg = p.deg[u];
    uint32_t* tb = sbin + t * d;
    uint32_t* cd = cdata + ((size_t)u * S + sl) * d;
    uint32_t sbits = 0;
    const bool narrow = (xv >> 32) == 0;
    const uint32_t x32 = (uint32_t)xv;
#pragma unroll 3
    for (int r = 0; r < d; r++) {
      const uint64_t* cr = s_coef + r * p.row_len + off;
      uint32_t hv, par = 0;
      if (narrow) {
        const uint64_t v = mac_narrow(cr[1], x32, cr[0]);
        hv = (uint32_t)v + mersenne_q(v);
        for (int e = 0; e < deg; e++) {
          const uint64_t* sc = cr + 2 + 4 * e;
          uint64_t acc = mac_narrow(sc[3], x32, sc[2]);
          acc = mac_narrow(acc, x32, sc[1]);
          acc = mac_narrow(acc, x32, sc[0]);
          par ^= ((uint32_t)acc ^ mersenne_q(acc)) & 1u;
        }
      } else {
        hv = (uint32_t)addmod(mulmod(cr[1], xv), cr[0]);
        for (int e = 0; e < deg; e++) {
          const uint64_t* sc = cr + 2 + 4 * e;
          uint64_t acc = sc[3];
          acc = addmod(mulmod(acc, xv), sc[2]);
          acc = addmod(mulmod(acc, xv), sc[1]);
          acc = addmod(mulmod(acc, xv), sc[0]);
          par ^= (uint32_t)(acc & 1u);
        }
      }
      atomicAdd(tb + r, hv);
      sbits |= par << r;
      if (claim) cd[r] = (hv & (uint32_t)(p.m - 1)) | (par << 31);
    }
    atomicXor(ssign + t, sbits);
  }
  __syncwarp();
  if (valid) {
    uint32_t sm = ssign[lane];
    for (int r = 0; r < d; r++) {
      uint32_t b = my_bin[r];
#pragma unroll
      for (int u = 0; u < A; u++) {
        if ((hitmask >> u) & 1u) {
          const uint32_t cv = cdata[((size_t)u * S + slot[u]) * d + r];
          b += cv & 0x7fffffffu;
          sm ^= (cv >> 31) << r;
        }
      }
      const uint32_t bin = b & (uint32_t)(p.m - 1);
      const int64_t v = ((sm >> r) & 1u) ? -delta : delta;
      atomicAdd(p.ctr + (int64_t)r * p.m + bin, (unsigned long long)v);
    }
  }
  __syncwarp();
}

template <int A>
__global__ void __launch_bounds__(512) k_update_cached(UpdArgs p, CacheLayout c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = p.d;
  const int S = 1 << c.log2s;
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  __shared__ int s_off[A];
  uint64_t* s_coef = (uint64_t*)smem_raw;
  const int ncoef = d * p.row_len;
  uint64_t* cx = s_coef + ncoef;
  uint32_t* cdata = (uint32_t*)(cx + (size_t)A * S);
  uint32_t* sbin = cdata + (size_t)A * S * d;
  uint32_t* ssign = sbin + (size_t)W * 32 * d;
  uint64_t* qx = (uint64_t*)(ssign + W * 32 + ((W * 32) & 1));
  uint16_t* qtu = (uint16_t*)(qx + (size_t)W * 32 * A);
  for (int t = threadIdx.x; t < ncoef; t += blockDim.x) s_coef[t] = p.coef[t];
  for (int t = threadIdx.x; t < A * S; t += blockDim.x) cx[t] = kEmptyKey;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int u = 0; u < A; u++) {
      s_off[u] = o;
      o += 2 + 4 * p.deg[u];
    }
  }
  __syncthreads();
  uint32_t* wb = sbin + (size_t)warp * 32 * d;
  uint32_t* ws = ssign + warp * 32;
  uint64_t* wq = qx + (size_t)warp * 32 * A;
  uint16_t* wt = qtu + (size_t)warp * 32 * A;
  const int64_t per = ((p.n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t c0 = (int64_t)blockIdx.x * per;
  const int64_t c1 = min(p.n, c0 + per);
  const int64_t ngroups = c1 > c0 ? (c1 - c0 + 31) / 32 : 0;
  for (int it = 0; it < c.fill_groups; it++) {
    const int64_t g = warp + (int64_t)W * it;
    cached_group<A, true>(p, c, c0 + g * 32, g < ngroups ? c1 : c0, s_coef, s_off, cx, cdata, wb, ws, wq, wt);
  }
  __syncthreads();
  for (int64_t g = warp + (int64_t)W * c.fill_groups; g < ngroups; g += W)
    cached_group<A, false>(p, c, c0 + g * 32, c1, s_coef, s_off, cx, cdata, wb, ws, wq, wt);
}

size_t cached_smem_bytes(int A, int d, int row_len, int log2s, int warps) {
  const size_t S = (size_t)1 << log2s;
  size_t b = (size_t)d * row_len * 8 + (size_t)A * S * 8 + (size_t)A * S * d * 4 + (size_t)warps * 32 * d * 4 +
             (size_t)warps * 32 * 4 + 4 + (size_t)warps * 32 * A * 8 + (size_t)warps * 32 * A * 2;
  return (b + 15) & ~(size_t)15;
}

template <int A>
cudaError_t launch_cached(const UpdArgs& a, int grid, int threads, size_t smem, CacheLayout c, cudaStream_t st) {
  auto kern = k_update_cached<A>;
  cudaError_t e = allow_dynamic_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(a, c);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_merge(unsigned long long* dst, const unsigned long long* src, int64_t count) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += step) dst[i] += src[i];
}

// SK_WARP_AGG=1 turns on the warp aggregation of shared-memory counter updates (off by
// default: on GB300 it measured 2.4-4x slower than plain shared-memory atomics for
// 1- and 2-attribute Zipf(1.1 and 1.4) relations with m = 256..4096).
bool warp_agg_enabled() {
  const char* v = std::getenv("SK_WARP_AGG");
  return v && v[0] == '1';
}

// Tuning knobs (environment): SK_UPDATE_CACHE=1 enables the hot-key cached kernel
// (off by default: on the Zipf(1.1) star fact table it measured slower than the plain
// kernel, 14.5 vs 13.8 ms per 1e8 tuples), SK_CACHE_LOG2S sets its table size per
// attribute (default 2^8 slots).
bool cache_disabled() {
  const char* v = std::getenv("SK_UPDATE_CACHE");
  return !(v && v[0] == '1');
}

int cache_log2s() {
  const char* v = std::getenv("SK_CACHE_LOG2S");
  const int x = v ? std::atoi(v) : 8;
  return x < 4 ? 4 : (x > 12 ? 12 : x);
}

// Key tables (declared domains): SK_KEY_TABLE=0 never uses them, =1 uses them whenever
// the domains allow it (tests), otherwise (default) when the domains are small against the
// batch (sum of domains * 4 <= tuples * attributes) and the relation's sketch is at most
// 32 MiB.  SK_KEY_TABLE_MAX_MB caps the table (default 1024 MiB).
int key_table_mode() {
  const char* v = std::getenv("SK_KEY_TABLE");
  if (!v || !v[0]) return 2;
  return v[0] == '0' ? 0 : (v[0] == '1' ? 1 : 2);
}

// Share of L2 for the counters one per-tuple update pass writes (SK_ROW_PASS_MB, default
// 64 MiB, half of GB300's L2; 0 = never split the rows).  8 x 1e7 rows into 16 x 2^20
// counters (128 MiB per relation): one pass 22.9 ms, two passes of 64 MiB 19.3 ms, three
// of 43 MiB 23.6 ms, four of 32 MiB 27.5 ms (each pass reads the keys again).
size_t row_pass_bytes() {
  const char* v = std::getenv("SK_ROW_PASS_MB");
  const long long x = v ? std::atoll(v) : 64;
  return (size_t)(x < 0 ? 0 : x) << 20;
}

size_t key_table_max_bytes() {
  const char* v = std::getenv("SK_KEY_TABLE_MAX_MB");
  const long long x = v ? std::atoll(v) : 1024;
  return (size_t)(x < 0 ? 0 : x) << 20;
}

int sm_count() {
  static const int n = [] {   // thread-safe one-time initialisation
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, dev);
    return x > 0 ? x : 1;
  }();
  return n;
}

}  // namespace

// CTAs for the shared-memory sub-sketch kernels: 16 tuples per thread (4096 per CTA of 256),
// or for small batches up to one CTA per SM with at least max(256, m) tuples each, so that a
// CTA's flush of its m-counter rows stays below its own counter updates and a batch of a few
// thousand tuples does not run on a handful of SMs.
int64_t smem_grid_want(int64_t n, int64_t m, int sms) {
  const int64_t per = std::max<int64_t>(256, std::min<int64_t>(m, 4096));
  return std::max<int64_t>((n + 4095) / 4096, std::min<int64_t>(sms, (n + per - 1) / per));
}

sk_status launch_update(sk_set* s, int relation, int64_t n, const int64_t* cols, int64_t col_stride,
                        const int64_t* weights, const int64_t* domain, cudaStream_t st) {
  const RelPlan& rp = s->rel[relation];
  UpdArgs a;
  a.cols = cols;
  a.stride = col_stride;
  a.w = weights;
  a.n = n;
  a.ctr = (unsigned long long*)(s->counters + (size_t)relation * s->d * s->m);
  a.coef = rp.d_coef;
  a.row_len = rp.coef_row_len;
  a.d = s->d;
  a.a = rp.a;
  for (int t = 0; t < kMaxAttrs; t++) a.deg[t] = rp.deg[t];
  a.m = (uint64_t)s->m;
  a.mrec = ~0ull / a.m;
  a.has_dom = domain != nullptr;
  for (int t = 0; t < kMaxAttrs; t++) a.dom[t] = (domain && t < rp.a) ? domain[t] : 0;
  a.status = s->d_status;
  a.agg = warp_agg_enabled() ? 1 : 0;
  a.s16 = 0;
  const bool pow2 = (s->m & (s->m - 1)) == 0;
  const size_t coef_bytes = (size_t)s->d * rp.coef_row_len * sizeof(uint64_t);
  const size_t sub_bytes = (size_t)s->d * (size_t)s->m * sizeof(int);
  const int sms = sm_count();
  if (coef_bytes > 200 * 1024) return SK_ERR_INVALID_ARG;   // hash table must fit in shared memory
  const bool use_smem = coef_bytes + sub_bytes <= 200 * 1024 && (int64_t)(s->d * s->m) <= n;
  cudaError_t e;
  const int ktm = key_table_mode();
  if (domain && ktm != 0 && n > 0 && rp.a >= 1 && s->d <= SK_MAX_ROWS && s->m <= (1ll << 30)) {
    TabArgs t;
    bool fits = true;
    int64_t total = 0;
    int off = 0;
    for (int u = 0; u < rp.a; u++) {
      if (domain[u] < 1 || domain[u] > (1ll << 31)) fits = false;
      t.base[u] = total;
      t.off[u] = off;
      total += fits ? domain[u] : 0;
      off += 2 + 4 * rp.deg[u];
    }
    t.base[rp.a] = total;
    t.narrow = s->m <= 65536 && s->d <= 32;
    t.rvec = key_record_vectors(s->d, t.narrow);
    // The two-phase partitioned update (unit weights, power-of-two 1024 <= m <= 2^16, d <= 14,
    // at most 5 attributes, sketch too large for one CTA's shared memory, at least 16 tuples
    // per counter of a row, fewer than 2^32 table records) takes 24-byte records for d <= 9
    // (the 32-byte 20-bit lane ones with SK_PART_RECORD=32) and the narrow 32-byte format
    // otherwise.
    bool part = part_update_mode() != 0 && pow2 && weights == nullptr && rp.a <= 5 && !use_smem && s->m >= 1024 &&
                s->m <= 65536 && s->d <= 14 && n >= (int64_t)s->m * 16 && total < ((int64_t)1 << 32);
    const int part_fmt = s->d <= 9 ? (part_record_bytes() == 32 ? 0 : 2) : 1;
    // The wide partitioned update (unit weights, power-of-two 2^17 <= m <= 2^24, d <= 16, at most
    // 5 attributes, at least m tuples, a sketch larger than 32 MiB, whose counter updates would
    // leave L2) takes the wide records (one 32-bit word per row).
    const size_t sketch_bytes = (size_t)s->d * (size_t)s->m * sizeof(int64_t);
    const int pum = part_update_mode();
    bool wide = pum != 0 && pow2 && weights == nullptr && rp.a <= 5 && s->m >= ((int64_t)1 << 17) &&
                s->m <= ((int64_t)1 << 24) && s->d <= kWideMaxRows && total < ((int64_t)1 << 32) &&
                (pum == 2 || (n >= (int64_t)s->m && sketch_bytes > ((size_t)32 << 20)));
    // Automatic choice: the tables replace per-tuple hashing by gathers, which pays when
    // the domains are small against a batch of at least 2^16 tuples (below that the table's
    // launch and allocation cost more than the hashing) and the counter updates hit L2 (for a sketch
    // much larger than L2 the update is bound by its atomics either way and the gathers
    // only add traffic: 27.7 vs 24.7 ms for 8 x 1e7 rows into 128 MB sketches), unless the
    // wide partitioned update takes the batch: it replaces those atomics.
    const bool worth = ktm == 1 || (n >= ((int64_t)1 << 16) && total * 4 <= n * (int64_t)rp.a &&
                                    (sketch_bytes <= ((size_t)32 << 20) || wide));
    void* staging = nullptr;
    if (fits && worth && total > 0 && part) {
      e = pool_malloc_async(&staging, part_staging_bytes(s->d, part_window(n), sms), st);
      if (e != cudaSuccess) {
        cudaGetLastError();   // no room for the planes: single-phase update
        staging = nullptr;
        part = false;
      }
    } else if (fits && worth && total > 0 && wide) {
      e = pool_malloc_async(&staging, wide_layout(s->d, s->m, wide_window(n)).total, st);
      if (e != cudaSuccess) {
        cudaGetLastError();   // no room for the planes: per-tuple update
        staging = nullptr;
        wide = false;
      }
    } else {
      wide = false;
    }
    if (part) t.rvec = 2;
    const size_t bytes = (size_t)total * (part && part_fmt == 2 ? 24 : (size_t)t.rvec * 16);
    if (fits && worth && total > 0 && bytes <= key_table_max_bytes()) {
      void* buf = nullptr;
      e = pool_malloc_async(&buf, bytes, st);
      if (e != cudaSuccess) {
        cudaGetLastError();   // not enough memory for the table: hash per tuple instead
        if (staging) cudaFreeAsync(staging, st);
      } else {
        t.tbl = (uint32_t*)buf;
        a.smem_wmax = 0;
        const bool d1 = all_deg1(a);
        auto kb = (part && part_fmt == 2)   ? (d1 ? k_key_table_l24<true> : k_key_table_l24<false>)
                  : (part && part_fmt == 0) ? (d1 ? k_key_table_l20<true> : k_key_table_l20<false>)
                  : pow2 ? (d1 ? k_key_table<true, true> : k_key_table<true, false>)
                         : (d1 ? k_key_table<false, true> : k_key_table<false, false>);
        e = cudaSuccess;
        e = fit_dynamic_smem((const void*)kb, coef_bytes);
        if (e == cudaSuccess) {
          const int bgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 32);
          kb<<<bgrid, 256, coef_bytes, st>>>(a, t);
          count_launch();
          e = cudaGetLastError();
        }
        if (e == cudaSuccess && part) {
          e = run_partitioned(a, t, part_fmt, staging, sms, st);
        } else if (e == cudaSuccess && wide) {
          e = run_wide_partitioned(a, t, staging, sms, st);
        } else if (e == cudaSuccess) {
          if (use_smem) {
            const int per_sm = sub_bytes <= 48 * 1024 ? 4 : (sub_bytes <= 100 * 1024 ? 2 : 1);
            const int64_t want = smem_grid_want(n, s->m, sms);
            const int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)sms * per_sm);
            const int64_t tpc = (n + (int64_t)grid * 256 - 1) / ((int64_t)grid * 256) * 256;
            a.smem_wmax = (int64_t)0x7fffffff / std::max<int64_t>(tpc, 1);
            e = pow2 ? dispatch_tab<true, true>(a, t, grid, sub_bytes, st)
                     : dispatch_tab<false, true>(a, t, grid, sub_bytes, st);
          } else {
            const int grid = (int)std::min<int64_t>((n + 255) / 256, 0x7fffffff);
            e = pow2 ? dispatch_tab<true, false>(a, t, grid, 0, st) : dispatch_tab<false, false>(a, t, grid, 0, st);
          }
        }
        cudaError_t ef = cudaFreeAsync(buf, st);
        if (staging) {
          const cudaError_t es = cudaFreeAsync(staging, st);
          if (ef == cudaSuccess) ef = es;
        }
        return set_status_from_cuda(e != cudaSuccess ? e : ef);
      }
    } else if (staging) {
      cudaFreeAsync(staging, st);
    }
  }
  const bool cache_ok = !use_smem && pow2 && s->d <= 32 && rp.a >= 1 && rp.a <= 5 && s->m <= (1ll << 30) &&
                        n >= (int64_t)1 << 17 && !cache_disabled();
  if (cache_ok) {
    const int threads = 512, warps = threads / 32;
    int log2s = cache_log2s();
    size_t smem = cached_smem_bytes(rp.a, s->d, rp.coef_row_len, log2s, warps);
    while (log2s > 6 && smem > 200 * 1024) smem = cached_smem_bytes(rp.a, s->d, rp.coef_row_len, --log2s, warps);
    if (smem <= 200 * 1024) {
      const int per_sm = smem <= 110 * 1024 ? 2 : 1;
      const int grid = (int)std::min<int64_t>((int64_t)sms * per_sm, std::max<int64_t>(1, n / (threads * 8)));
      CacheLayout c{log2s, 8};
      a.smem_wmax = 0;
      switch (rp.a) {
        case 1: e = launch_cached<1>(a, grid, threads, smem, c, st); break;
        case 2: e = launch_cached<2>(a, grid, threads, smem, c, st); break;
        case 3: e = launch_cached<3>(a, grid, threads, smem, c, st); break;
        case 4: e = launch_cached<4>(a, grid, threads, smem, c, st); break;
        default: e = launch_cached<5>(a, grid, threads, smem, c, st); break;
      }
      return set_status_from_cuda(e);
    }
  }
  if (use_smem) {
    const size_t smem = coef_bytes + sub_bytes;
    const int per_sm = smem <= 48 * 1024 ? 4 : (smem <= 100 * 1024 ? 2 : 1);
    int64_t want = smem_grid_want(n, s->m, sms);
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)sms * per_sm);
    const int64_t tpc = (n + (int64_t)grid * 256 - 1) / ((int64_t)grid * 256) * 256;
    a.smem_wmax = (int64_t)0x7fffffff / std::max<int64_t>(tpc, 1);
    e = pow2 ? dispatch_a<true, true>(a, grid, smem, st) : dispatch_a<false, true>(a, grid, smem, st);
  } else {
    // Counters in global memory.  When the relation's d x m int64 counters exceed the share
    // of L2 given by row_pass_bytes(), the rows are split into passes over the whole batch
    // (each pass hashes only its rows; the keys are read once per pass), so that the
    // counter updates of a pass stay in L2.
    a.smem_wmax = 0;
    const size_t row_bytes = (size_t)s->m * sizeof(int64_t);
    const size_t budget = row_pass_bytes();
    int rows = s->d;
    if (budget > 0 && (size_t)s->d * row_bytes > budget) rows = (int)std::max<size_t>(1, budget / row_bytes);
    const int passes = (s->d + rows - 1) / rows;
    rows = (s->d + passes - 1) / passes;   // even split
    e = cudaSuccess;
    for (int r0 = 0; r0 < s->d && e == cudaSuccess; r0 += rows) {
      UpdArgs b = a;
      b.d = std::min(rows, s->d - r0);
      b.coef = a.coef + (size_t)r0 * rp.coef_row_len;
      b.ctr = a.ctr + (size_t)r0 * s->m;
      const size_t cb = (size_t)b.d * rp.coef_row_len * sizeof(uint64_t);
      e = pow2 ? dispatch_a<true, false>(b, 0, cb, st) : dispatch_a<false, false>(b, 0, cb, st);
    }
  }
  return set_status_from_cuda(e);
}

sk_status launch_merge(int64_t* dst, const int64_t* src, int64_t count, cudaStream_t st) {
  if (count == 0) return SK_OK;
  const int grid = (int)std::min<int64_t>((count + 255) / 256, (int64_t)sm_count() * 8);
  k_merge<<<grid, 256, 0, st>>>((unsigned long long*)dst, (const unsigned long long*)src, count);
  count_launch();
  return set_status_from_cuda(cudaGetLastError());
}

// One bit per tuple: all of the relation's keys inside their declared domains (a tuple with a
// key outside is reported and left out of every view).
__global__ void __launch_bounds__(256) k_valid_bits(UpdArgs p, uint32_t* bits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = i < p.n;
  if (ok)
    for (int u = 0; u < p.a; u++) {
      const int64_t key = ld_key_stream(p.cols + (int64_t)u * p.stride + i);
      if ((uint64_t)key >= (uint64_t)p.dom[u]) ok = false;
    }
  if (i < p.n && !ok) record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
  const uint32_t b = __ballot_sync(0xffffffffu, ok);
  if ((threadIdx.x & 31u) == 0 && i < p.n) bits[i >> 5] = b;
}

// Sub-query family views of one relation through the two-phase partitioned update (see
// run_partitioned): when every attribute has exactly one sign slot, a view's sign is the
// product of its attributes' slot-0 signs and its bin the sum of their bins, so one 24-byte
// key table over the relation's attributes (built once) serves every view, and each view's
// counters get both phases over the view's attributes (a validity pass over all of the
// relation's keys first: a tuple is left out of every view when any key is outside its
// domain, as in the per-tuple view update).  Taken for unit weights with declared
// domains, power-of-two 1024 <= m <= 2^16, d <= 9, views of at most 5 attributes, at least
// 16 m tuples and views too large for one CTA's shared memory; *done = false (nothing
// launched) otherwise, and the caller runs its per-tuple view update.
sk_status family_partitioned_update(const UpdArgs& a, int nv, const uint32_t* amask, const unsigned long long* jmask,
                                    unsigned long long* const* ctr, cudaStream_t st, bool* done) {
  *done = false;
  const int64_t n = a.n;
  const bool pow2 = (a.m & (a.m - 1)) == 0;
  if (part_update_mode() == 0 || key_table_mode() == 0 || !a.has_dom || a.w != nullptr || !pow2 || a.m < 1024 ||
      a.m > 65536 || a.d > 9 || a.a < 1 || a.a > kMaxAttrs || n < (int64_t)a.m * 16 ||
      (size_t)a.d * a.m * sizeof(int) <= 200 * 1024 || !all_deg1(a))
    return SK_OK;
  TabArgs t;
  int64_t total = 0;
  int off = 0;
  for (int u = 0; u < a.a; u++) {
    if (a.dom[u] < 1 || a.dom[u] > (1ll << 31)) return SK_OK;
    t.base[u] = total;
    t.off[u] = off;
    total += a.dom[u];
    off += 2 + 4 * a.deg[u];
  }
  t.base[a.a] = total;
  t.narrow = 1;
  t.rvec = 2;
  if (total >= ((int64_t)1 << 32) || (key_table_mode() != 1 && total * 4 > n * (int64_t)a.a)) return SK_OK;
  for (int v = 0; v < nv; v++) {
    // slot i is attribute i's only slot: a view's signs are those of its attributes
    if (__builtin_popcount(amask[v]) > 5 || (unsigned long long)amask[v] != jmask[v]) return SK_OK;
  }
  const size_t tbytes = (size_t)total * 24;
  if (tbytes > key_table_max_bytes()) return SK_OK;
  const int sms = sm_count();
  void* tbl = nullptr;
  void* staging = nullptr;
  if (pool_malloc_async(&tbl, tbytes, st) != cudaSuccess) {
    cudaGetLastError();
    return SK_OK;
  }
  const size_t sbytes = part_staging_bytes(a.d, part_window(n), sms);
  const size_t vbytes = (size_t)(n + 31) / 32 * sizeof(uint32_t);
  if (pool_malloc_async(&staging, sbytes + ((vbytes + 255) & ~(size_t)255), st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(tbl, st);
    return SK_OK;
  }
  *done = true;
  uint32_t* vbits = (uint32_t*)((char*)staging + sbytes);
  t.tbl = (uint32_t*)tbl;
  const size_t coef_bytes = (size_t)a.d * a.row_len * sizeof(uint64_t);
  cudaError_t e = fit_dynamic_smem((const void*)k_key_table_l24<true>, coef_bytes);
  if (e == cudaSuccess) {
    const int bgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 32);
    k_key_table_l24<true><<<bgrid, 256, coef_bytes, st>>>(a, t);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_valid_bits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, vbits);
    count_launch();
    e = cudaGetLastError();
  }
  for (int v = 0; v < nv && e == cudaSuccess; v++) {
    UpdArgs av = a;
    TabArgs tv = t;
    const int64_t* colp[5];
    int k = 0;
    for (int u = 0; u < a.a; u++) {
      if (!((amask[v] >> u) & 1u)) continue;
      av.dom[k] = a.dom[u];
      av.deg[k] = a.deg[u];
      tv.base[k] = t.base[u];
      colp[k] = a.cols + (int64_t)u * a.stride;
      k++;
    }
    if (k == 0) continue;
    av.a = k;
    tv.base[k] = total;
    av.ctr = ctr[v];
    e = run_partitioned(av, tv, 2, staging, sms, st, colp, vbits);
  }
  cudaError_t ef = cudaFreeAsync(tbl, st);
  const cudaError_t es = cudaFreeAsync(staging, st);
  if (ef == cudaSuccess) ef = es;
  return set_status_from_cuda(e != cudaSuccess ? e : ef);
}

}  // namespace sk
