// Device-side hashing shared by the update kernels: the GF(2^61 - 1) arithmetic and
// the per-tuple body of Algorithm 2 (Eqs. 2-4).  Included by sk_update.cu and
// sk_multi.cu only.
#pragma once

#include "sk_internal.h"

namespace sk {
namespace dev {

struct UpdArgs {
  const int64_t* cols;
  int64_t stride;
  const int64_t* w;
  int64_t n;
  unsigned long long* ctr;   // this relation's [d][m]
  const uint64_t* coef;      // [d][row_len], see RelPlan
  int row_len;
  int d;
  int a;
  int deg[kMaxAttrs];
  uint64_t m;
  uint64_t mrec;             // floor((2^64 - 1) / m), for reductions mod m when m is not a power of two
  int has_dom;
  int64_t dom[kMaxAttrs];
  int* status;
  int64_t smem_wmax;         // |Delta| <= smem_wmax goes to the int32 sub-sketch
  int agg;                   // warp-aggregate shared-memory counter updates
  int s16;                   // shared sub-sketch of biased 16-bit counters, two per 32-bit word
};

__device__ __forceinline__ uint64_t field_of(int64_t key) {
  const uint64_t k = (uint64_t)key;
  const uint64_t x = (k & kP61) + (k >> 61);   // 2^61 == 1 (mod p)
  return x >= kP61 ? x - kP61 : x;
}

// a * b mod p for a, b < p: the 122-bit product split at bit 61, the high part
// folded onto the low part (2^61 == 1 mod p), one conditional subtraction.
__device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b) {
  const uint64_t lo = a * b;
  const uint64_t hi = __umul64hi(a, b);
  const uint64_t r = (lo & kP61) + ((lo >> 61) | (hi << 3));
  return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ uint64_t addmod(uint64_t a, uint64_t b) {
  const uint64_t r = a + b;
  return r >= kP61 ? r - kP61 : r;
}

// Narrow-key arithmetic, used when every key of a tuple lies in [0, 2^32) (then the
// field element is the key itself): Horner steps with a 32-bit multiplier whose
// results stay "lazy" (congruent mod p, below 2^61 + 2^35) until one final
// reduction per polynomial.
//
// acc * x + c mod p, lazily, for any acc < 2^64, x < 2^32 and c < 2^61; the result is
// below 2^61 + 2^35.  The 96-bit value acc x + c is formed from two 32x32+32 -> 64
// multiply-adds, T = lo32(acc) x + lo32(c) and U = hi32(acc) x + hi32(c) (neither
// overflows), as s 2^32 + lo32(T) with s = U + (T >> 32) < 2^64; folding at bit 61
// (2^61 == 1 mod p) leaves ((s mod 2^29) 2^32 + lo32(T)) + (s >> 29).
__device__ __forceinline__ uint64_t mac_narrow(uint64_t acc, uint32_t x, uint64_t c) {
  const uint64_t T = (uint64_t)(uint32_t)acc * x + (uint32_t)c;
  const uint64_t U = (uint64_t)(uint32_t)(acc >> 32) * x + (uint32_t)(c >> 32);
  const uint64_t sv = U + (T >> 32);
  const uint32_t s0 = (uint32_t)sv, s1 = (uint32_t)(sv >> 32);
  const uint32_t fl = __funnelshift_r(s0, s1, 29);
  const uint32_t fh = s1 >> 29;
  uint32_t r0, r1;
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;"
      : "=r"(r0), "=r"(r1)
      : "r"((uint32_t)T), "r"(fl), "r"(s0 & ((1u << 29) - 1u)), "r"(fh));
  return ((uint64_t)r1 << 32) | r0;
}

// floor(v / p) for v < 2^63: with v = a 2^61 + b, v / p = a + (a + b) / p and a + b < 2^61 + 4,
// so the quotient is a or a + 1, and it is a + 1 exactly when b + a + 1 reaches 2^61.
__device__ __forceinline__ uint32_t mersenne_q(uint64_t v) { return (uint32_t)((v + (v >> 61) + 1) >> 61); }

// floor(v / p) for the outputs of mac_narrow (v < 2^61 + 2^35 < 2p): 1 exactly when
// v >= p, i.e. when v + 1 reaches 2^61.
__device__ __forceinline__ uint32_t mersenne_q1(uint64_t v) { return (uint32_t)((v + 1) >> 61); }

// v < 2^63 -> v mod p
__device__ __forceinline__ uint64_t reduce_lazy(uint64_t v) {
  const uint64_t r = (v & kP61) + (v >> 61);
  return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ void record(int* status, int code) { atomicCAS(status, 0, code); }

// counter += v as a global-memory reduction (no return value).  The pointer may come from
// memory the compiler cannot trace to a kernel argument (the batched plan's items), where
// atomicAdd would be issued as a generic atomic with a return value.
__device__ __forceinline__ void red_add_global(unsigned long long* ptr, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(ptr)), "l"(v));
}

// Key-column load for the update kernels: the columns are streamed once, so they are
// kept out of L1 and marked first to leave L2 (the tables and the sketch stay cached).
__device__ __forceinline__ int64_t ld_key_stream(const int64_t* ptr) {
  int64_t v;
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
  return v;
}

// v mod m for any v < 2^64 and m >= 1, with mrec = floor((2^64 - 1) / m): the quotient
// estimate hi64(v mrec) lies between floor(v / m) - 2 and floor(v / m), so at most two
// subtractions of m give the remainder exactly (no division instruction sequence).
__device__ __forceinline__ uint64_t mod_m(uint64_t v, uint64_t m, uint64_t mrec) {
  uint64_t r = v - __umul64hi(v, mrec) * m;
  if (r >= m) r -= m;
  if (r >= m) r -= m;
  return r;
}

template <bool POW2>
__device__ __forceinline__ uint64_t reduce_m(uint64_t v, uint64_t m, uint64_t mrec) {
  return POW2 ? (v & (m - 1)) : mod_m(v, m, mrec);
}

// A = number of attributes when known at compile time (1..4), 0 = runtime a.
// Algorithm 2 for tuple i: all d rows hashed in registers, one counter update per row
// (int32 shared-memory sub-sketch when SMEM and |Delta| is small, int64 global otherwise).
//
// AGG (shared-memory path only): the whole warp calls this for 32 consecutive tuples,
// `live` false past the end; lanes that add to the same shared counter are grouped with
// __match_any_sync and their values summed with __reduce_add_sync, so each distinct
// counter receives one atomic per warp (hot keys of skewed columns otherwise serialise
// on one shared-memory address).  Lanes past the end or with a key outside the declared
// domain take part with Delta = 0.
//
// DEG1: every attribute of the relation is in exactly one join (chains, stars), so each
// attribute has one sign polynomial and the loop over its joins disappears.
template <int A, bool POW2, bool SMEM, bool AGG = false, bool DEG1 = false>
__device__ __forceinline__ void update_tuple(const UpdArgs& p, const uint64_t* s_coef, int* s_sub, int64_t i,
                                             bool live = true) {
  const int na = A > 0 ? A : p.a;
  uint64_t x[A > 0 ? A : kMaxAttrs];
  bool ok = true;
#pragma unroll
  for (int u = 0; u < (A > 0 ? A : kMaxAttrs); u++) {
    if (A == 0 && u >= na) break;
    const int64_t key = (!AGG || live) ? ld_key_stream(p.cols + (int64_t)u * p.stride + i) : 0;
    if (p.has_dom && (!AGG || live) && (key < 0 || key >= p.dom[u])) ok = false;
    x[u] = field_of(key);
  }
  if (!ok) {
    record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
    if (!AGG) return;
  }
  const int64_t delta = (AGG && (!live || !ok)) ? 0 : (p.w ? __ldg(p.w + i) : 1);
  const bool small = SMEM && (delta <= p.smem_wmax && delta >= -p.smem_wmax);
  bool narrow = true;
#pragma unroll
  for (int u = 0; u < (A > 0 ? A : kMaxAttrs); u++) {
    if (A == 0 && u >= na) break;
    narrow = narrow && (x[u] >> 32) == 0;
  }
  const uint64_t* cr = s_coef;
  for (int row = 0; row < p.d; row++, cr += p.row_len) {
    uint64_t bin = 0;
    uint32_t sbit = 0;
    int off = 0;
    if (narrow) {
      // Coefficient pairs are 16-byte aligned: the table starts 16-byte aligned and every
      // attribute block (2 + 4 deg words) and row (a sum of those) has an even length.
      uint32_t bin32 = 0, sx = 0;
#pragma unroll
      for (int u = 0; u < (A > 0 ? A : kMaxAttrs); u++) {
        if (A == 0 && u >= na) break;
        const uint32_t xu = (uint32_t)x[u];
        const ulonglong2 bc = *(const ulonglong2*)(cr + off);
        const uint64_t v = mac_narrow(bc.y, xu, bc.x);
        if (POW2) {
          bin32 += (uint32_t)v + mersenne_q1(v);   // == h(x) mod 2^32
        } else {
          bin += mod_m(reduce_lazy(v), p.m, p.mrec);
        }
        off += 2;
        const int deg = DEG1 ? 1 : p.deg[u];
        for (int e = 0; e < deg; e++, off += 4) {
          const ulonglong2 s01 = *(const ulonglong2*)(cr + off);
          const ulonglong2 s23 = *(const ulonglong2*)(cr + off + 2);
          uint64_t acc = mac_narrow(s23.y, xu, s23.x);
          acc = mac_narrow(acc, xu, s01.y);
          acc = mac_narrow(acc, xu, s01.x);
          sx ^= (uint32_t)acc ^ mersenne_q1(acc);   // bit 0: parity of acc mod p
        }
      }
      sbit = sx & 1u;
      if (POW2) bin = bin32;
    } else {
#pragma unroll
      for (int u = 0; u < (A > 0 ? A : kMaxAttrs); u++) {
        if (A == 0 && u >= na) break;
        const uint64_t xu = x[u];
        const uint64_t h = addmod(mulmod(cr[off + 1], xu), cr[off]);
        bin += reduce_m<POW2>(h, p.m, p.mrec);
        off += 2;
        const int deg = DEG1 ? 1 : p.deg[u];
        for (int e = 0; e < deg; e++, off += 4) {
          uint64_t acc = cr[off + 3];
          acc = addmod(mulmod(acc, xu), cr[off + 2]);
          acc = addmod(mulmod(acc, xu), cr[off + 1]);
          acc = addmod(mulmod(acc, xu), cr[off]);
          sbit ^= (uint32_t)(acc & 1u);
        }
      }
    }
    bin = reduce_m<POW2>(bin, p.m, p.mrec);
    const int64_t v = sbit ? -delta : delta;
    if (AGG) {
      const unsigned lane = threadIdx.x & 31u;
      const unsigned key = small ? (unsigned)(row * p.m + bin) : 0xffffffffu - lane;
      const unsigned same = __match_any_sync(0xffffffffu, key);
      const int sum = __reduce_add_sync(same, small ? (int)v : 0);
      if (small && lane == (unsigned)(__ffs(same) - 1) && sum != 0) atomicAdd(s_sub + key, sum);
      if (!small && v != 0) red_add_global(p.ctr + (int64_t)row * p.m + bin, (unsigned long long)v);
    } else if (SMEM && small) {
      if (p.s16) {   // counter j in half (j & 1) of word j / 2; the bias keeps it from carrying
        const int64_t j = (int64_t)row * p.m + bin;
        const uint32_t add = (uint32_t)(int32_t)v << (16 * (uint32_t)(j & 1));
        atomicAdd((unsigned int*)s_sub + (j >> 1), add);
      } else {
        atomicAdd(s_sub + (int64_t)row * p.m + bin, (int)v);
      }
    } else {
      red_add_global(p.ctr + (int64_t)row * p.m + bin, (unsigned long long)v);
    }
  }
}

// ---------------------------------------------------------------------------
// Key tables.  When a relation's keys come with declared domains [0, dom_u) and the
// batch is much longer than the domains, the per-attribute hash results are computed
// once per domain key instead of once per tuple.  The record of (attribute u, key x)
// holds, for every row, the bin h_comp(u)(x) mod m and the parity of the product of
// the signs of u's joins (set = sign -1).  A tuple then combines its A records with the
// same sum-mod-m and sign product as update_tuple (Eqs. 2-3), so every counter update
// is identical.  Two record formats:
//   - narrow (m <= 2^16, d <= 32): d uint16 bins from byte 0, the d sign bits in the
//     record's last 32-bit word; round_up(2d + 4, 16) bytes (32 for d <= 14);
//   - wide: d uint32 words, bin in bits 0..30 and sign in bit 31, zero-padded to a
//     multiple of 16 bytes.
// ---------------------------------------------------------------------------
struct TabArgs {
  uint32_t* tbl;                 // [sum_u dom_u][rvec * 4] 32-bit words
  int64_t base[kMaxAttrs + 1];   // first record of attribute u; base[a] = total records
  int off[kMaxAttrs];            // coefficient offset of attribute u within a row
  int rvec;                      // record length in 16-byte vectors
  int narrow;                    // record format
};

__host__ __device__ inline int key_record_vectors(int d, bool narrow) {
  return narrow ? (2 * d + 4 + 15) / 16 : (4 * d + 15) / 16;
}

// bin mod m and sign parity of attribute u's functions for one row at key x (< 2^32)
template <bool POW2, bool DEG1 = false>
__device__ __forceinline__ uint32_t key_row_hash(const UpdArgs& p, const uint64_t* c, int deg, uint32_t x,
                                                 uint32_t* parity) {
  const ulonglong2 bc = *(const ulonglong2*)c;
  const uint64_t v = mac_narrow(bc.y, x, bc.x);
  uint32_t h;
  if (POW2) h = ((uint32_t)v + mersenne_q1(v)) & (uint32_t)(p.m - 1);
  else h = (uint32_t)mod_m(reduce_lazy(v), p.m, p.mrec);
  uint32_t sx = 0;
  if (DEG1) deg = 1;
  for (int k = 0; k < deg; k++) {
    const ulonglong2 s01 = *(const ulonglong2*)(c + 2 + 4 * k);
    const ulonglong2 s23 = *(const ulonglong2*)(c + 4 + 4 * k);
    uint64_t acc = mac_narrow(s23.y, x, s23.x);
    acc = mac_narrow(acc, x, s01.y);
    acc = mac_narrow(acc, x, s01.x);
    sx ^= (uint32_t)acc ^ mersenne_q1(acc);
  }
  *parity = sx & 1u;
  return h;
}

// Record of attribute u for key x (< 2^31: the field element is the key itself).
template <bool POW2, bool DEG1 = false>
__device__ __forceinline__ void key_record(const UpdArgs& p, const TabArgs& t, const uint64_t* s_coef, int u,
                                           uint32_t x, uint32_t* out) {
  const int deg = p.deg[u];
  const uint64_t* cr = s_coef + t.off[u];
  const int nw = 4 * t.rvec;
  uint32_t mask = 0;
  for (int w0 = 0; w0 < nw; w0 += 4) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int wi = w0 + j;
      uint32_t e = 0;
      if (t.narrow) {
        if (wi == nw - 1) {
          e = mask;
        } else {
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const int row = 2 * wi + h;
            if (row < p.d) {
              uint32_t par;
              const uint32_t b = key_row_hash<POW2, DEG1>(p, cr + (int64_t)row * p.row_len, deg, x, &par);
              e |= b << (16 * h);
              mask |= par << row;
            }
          }
        }
      } else if (wi < p.d) {
        uint32_t par;
        const uint32_t b = key_row_hash<POW2, DEG1>(p, cr + (int64_t)wi * p.row_len, deg, x, &par);
        e = b | (par << 31);
      }
      w[j] = e;
    }
    *(uint4*)(out + w0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <bool SMEM>
__device__ __forceinline__ void scatter_row(const UpdArgs& p, int* s_sub, bool small, int row, uint32_t bin,
                                            int64_t v) {
  if (SMEM && small) atomicAdd(s_sub + (int64_t)row * p.m + bin, (int)v);
  else red_add_global(p.ctr + (int64_t)row * p.m + bin, (unsigned long long)v);
}

// Lane-wise sum of two pairs of 16-bit values (each half mod 2^16, no carry across halves):
// the low 15 bits of each half add normally, bit 15 is the XOR of both inputs' bit 15 with
// the carry into it.
__device__ __forceinline__ uint32_t add16x2(uint32_t a, uint32_t b) {
  return ((a & 0x7fff7fffu) + (b & 0x7fff7fffu)) ^ ((a ^ b) & 0x80008000u);
}

// One 32-byte record with a single 256-bit load.  Only for records of exactly two
// 16-byte vectors: the table base is 256-byte aligned, so every record is 32-byte aligned.
__device__ __forceinline__ void ld_record32(const uint4* ptr, uint32_t (&w)[8]) {
  asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
      : "l"(ptr));
}

// Algorithm 2 for tuple i through the key tables (declared domains are required).
// V8: records are 32 bytes (rvec == 2) and each is read with one load.
template <int A, bool POW2, bool SMEM, bool NARROW, bool V8 = false>
__device__ __forceinline__ void update_tuple_tab(const UpdArgs& p, const TabArgs& t, int* s_sub, int64_t i) {
  const int na = A > 0 ? A : p.a;
  constexpr int AM = A > 0 ? A : kMaxAttrs;
  const uint4* rec[AM];
  bool ok = true;
#pragma unroll
  for (int u = 0; u < AM; u++) {
    if (A == 0 && u >= na) break;
    const int64_t key = ld_key_stream(p.cols + (int64_t)u * p.stride + i);
    if (key < 0 || key >= p.dom[u]) ok = false;
    rec[u] = (const uint4*)t.tbl + (t.base[u] + (ok ? key : 0)) * t.rvec;
  }
  if (!ok) {
    record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
    return;
  }
  const int64_t delta = p.w ? __ldg(p.w + i) : 1;
  const bool small = SMEM && (delta <= p.smem_wmax && delta >= -p.smem_wmax);
  const uint32_t m32 = (uint32_t)p.m;
  if (V8 && NARROW) {
    // d <= 14: bins in words 0..6, sign mask in word 7
    if (POW2) {
      // m divides 2^16, so each bin sum is needed mod 2^16 only: two rows per 32-bit word,
      // added lane-wise without a carry between the 16-bit halves
      uint32_t b2[7] = {0, 0, 0, 0, 0, 0, 0}, sg = 0;
#pragma unroll
      for (int u = 0; u < AM; u++) {
        if (A == 0 && u >= na) break;
        uint32_t w[8];
        ld_record32(rec[u], w);
        sg ^= w[7];
#pragma unroll
        for (int j = 0; j < 7; j++) b2[j] = add16x2(b2[j], w[j]);
      }
#pragma unroll
      for (int j = 0; j < 14; j++) {
        if (j >= p.d) break;
        const uint32_t bin = (b2[j >> 1] >> (16 * (j & 1))) & (m32 - 1);
        scatter_row<SMEM>(p, s_sub, small, j, bin, ((sg >> j) & 1u) ? -delta : delta);
      }
    } else {
      uint32_t b[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, sg = 0;
#pragma unroll
      for (int u = 0; u < AM; u++) {
        if (A == 0 && u >= na) break;
        uint32_t w[8];
        ld_record32(rec[u], w);
        sg ^= w[7];
#pragma unroll
        for (int j = 0; j < 14; j++) {
          b[j] += (w[j >> 1] >> (16 * (j & 1))) & 0xffffu;
          if (b[j] >= m32) b[j] -= m32;
        }
      }
#pragma unroll
      for (int j = 0; j < 14; j++) {
        if (j >= p.d) break;
        scatter_row<SMEM>(p, s_sub, small, j, b[j], ((sg >> j) & 1u) ? -delta : delta);
      }
    }
  } else if (V8) {
    // d <= 8: one word per row
    uint32_t b[8] = {0, 0, 0, 0, 0, 0, 0, 0}, sg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int u = 0; u < AM; u++) {
      if (A == 0 && u >= na) break;
      uint32_t w[8];
      ld_record32(rec[u], w);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        if (POW2) {
          b[j] += w[j];
        } else {
          b[j] += w[j] & 0x7fffffffu;
          if (b[j] >= m32) b[j] -= m32;
        }
        sg[j] ^= w[j];
      }
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (j >= p.d) break;
      const uint32_t bin = POW2 ? (b[j] & (m32 - 1)) : b[j];
      scatter_row<SMEM>(p, s_sub, small, j, bin, (sg[j] >> 31) ? -delta : delta);
    }
  } else if (NARROW) {
    // the last vector of every record carries the sign mask; keep it
    const int last = t.rvec - 1;
    uint4 tail[AM];
    uint32_t sg = 0;
#pragma unroll
    for (int u = 0; u < AM; u++) {
      if (A == 0 && u >= na) break;
      tail[u] = __ldg(rec[u] + last);
      sg ^= tail[u].w;
    }
    for (int c = 0; c <= last; c++) {
      uint32_t b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int u = 0; u < AM; u++) {
        if (A == 0 && u >= na) break;
        const uint4 q = c == last ? tail[u] : __ldg(rec[u] + c);
        const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const uint32_t e = (wd[j >> 1] >> (16 * (j & 1))) & 0xffffu;
          if (POW2) {
            b[j] += e;
          } else {
            b[j] += e;
            if (b[j] >= m32) b[j] -= m32;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int row = 8 * c + j;
        if (row >= p.d) break;
        const uint32_t bin = POW2 ? (b[j] & (m32 - 1)) : b[j];
        scatter_row<SMEM>(p, s_sub, small, row, bin, ((sg >> row) & 1u) ? -delta : delta);
      }
    }
  } else {
    for (int c = 0; c < t.rvec; c++) {
      uint32_t b[4] = {0, 0, 0, 0}, sg[4] = {0, 0, 0, 0};
#pragma unroll
      for (int u = 0; u < AM; u++) {
        if (A == 0 && u >= na) break;
        const uint4 q = __ldg(rec[u] + c);
        const uint32_t e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
          if (POW2) {
            b[j] += e[j];   // sign bits carry out above the masked bin bits
          } else {
            b[j] += e[j] & 0x7fffffffu;
            if (b[j] >= m32) b[j] -= m32;
          }
          sg[j] ^= e[j];
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int row = 4 * c + j;
        if (row >= p.d) break;
        const uint32_t bin = POW2 ? (b[j] & (m32 - 1)) : b[j];
        scatter_row<SMEM>(p, s_sub, small, row, bin, (sg[j] >> 31) ? -delta : delta);
      }
    }
  }
}

}  // namespace dev
}  // namespace sk
