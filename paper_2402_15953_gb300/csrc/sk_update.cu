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

#include "sk_internal.h"

namespace sk {
namespace {

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
  int has_dom;
  int64_t dom[kMaxAttrs];
  int* status;
  int64_t smem_wmax;         // |Delta| <= smem_wmax goes to the int32 sub-sketch
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

template <bool POW2>
__device__ __forceinline__ uint64_t reduce_m(uint64_t v, uint64_t m) {
  return POW2 ? (v & (m - 1)) : (v % m);
}

// A = number of attributes when known at compile time (1..4), 0 = runtime a.
// Algorithm 2 for tuple i: all d rows hashed in registers, one counter update per row
// (int32 shared-memory sub-sketch when SMEM and |Delta| is small, int64 global otherwise).
template <int A, bool POW2, bool SMEM>
__device__ __forceinline__ void update_tuple(const UpdArgs& p, const uint64_t* s_coef, int* s_sub, int64_t i) {
  const int na = A > 0 ? A : p.a;
  uint64_t x[A > 0 ? A : kMaxAttrs];
  bool ok = true;
#pragma unroll
  for (int u = 0; u < (A > 0 ? A : kMaxAttrs); u++) {
    if (A == 0 && u >= na) break;
    const int64_t key = __ldg(p.cols + (int64_t)u * p.stride + i);
    if (p.has_dom && (key < 0 || key >= p.dom[u])) ok = false;
    x[u] = field_of(key);
  }
  if (!ok) {
    record(p.status, SK_ERR_KEY_OUT_OF_DOMAIN);
    return;
  }
  const int64_t delta = p.w ? __ldg(p.w + i) : 1;
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
          bin += reduce_lazy(v) % p.m;
        }
        off += 2;
        for (int e = 0; e < p.deg[u]; e++, off += 4) {
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
        bin += reduce_m<POW2>(h, p.m);
        off += 2;
        for (int e = 0; e < p.deg[u]; e++, off += 4) {
          uint64_t acc = cr[off + 3];
          acc = addmod(mulmod(acc, xu), cr[off + 2]);
          acc = addmod(mulmod(acc, xu), cr[off + 1]);
          acc = addmod(mulmod(acc, xu), cr[off]);
          sbit ^= (uint32_t)(acc & 1u);
        }
      }
    }
    bin = reduce_m<POW2>(bin, p.m);
    const int64_t v = sbit ? -delta : delta;
    if (SMEM && small) {
      atomicAdd(s_sub + (int64_t)row * p.m + bin, (int)v);
    } else {
      atomicAdd(p.ctr + (int64_t)row * p.m + bin, (unsigned long long)v);
    }
  }
}

template <int A, bool POW2, bool SMEM>
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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += step) {
    update_tuple<A, POW2, SMEM>(p, s_coef, s_sub, i);
  }
  if (SMEM) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < dm; i += blockDim.x) {
      const int v = s_sub[i];
      if (v != 0) atomicAdd(p.ctr + i, (unsigned long long)(int64_t)v);
    }
  }
}

template <int A, bool POW2, bool SMEM>
cudaError_t launch_one(const UpdArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = k_update<A, POW2, SMEM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
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
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(a, c);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_merge(unsigned long long* dst, const unsigned long long* src, int64_t count) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += step) dst[i] += src[i];
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

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

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
  a.has_dom = domain != nullptr;
  for (int t = 0; t < kMaxAttrs; t++) a.dom[t] = (domain && t < rp.a) ? domain[t] : 0;
  a.status = s->d_status;
  const bool pow2 = (s->m & (s->m - 1)) == 0;
  const size_t coef_bytes = (size_t)s->d * rp.coef_row_len * sizeof(uint64_t);
  const size_t sub_bytes = (size_t)s->d * (size_t)s->m * sizeof(int);
  const int sms = sm_count();
  if (coef_bytes > 200 * 1024) return SK_ERR_INVALID_ARG;   // hash table must fit in shared memory
  const bool use_smem = coef_bytes + sub_bytes <= 200 * 1024 && (int64_t)(s->d * s->m) <= n;
  cudaError_t e;
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
    int64_t want = (n + 256 * 16 - 1) / (256 * 16);
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)sms * per_sm);
    const int64_t tpc = (n + (int64_t)grid * 256 - 1) / ((int64_t)grid * 256) * 256;
    a.smem_wmax = (int64_t)0x7fffffff / std::max<int64_t>(tpc, 1);
    e = pow2 ? dispatch_a<true, true>(a, grid, smem, st) : dispatch_a<false, true>(a, grid, smem, st);
  } else {
    a.smem_wmax = 0;
    int64_t want = (n + 255) / 256;
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)sms * 8);
    e = pow2 ? dispatch_a<true, false>(a, grid, coef_bytes, st)
             : dispatch_a<false, false>(a, grid, coef_bytes, st);
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

}  // namespace sk
