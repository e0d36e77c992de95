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
// field element is the key itself).  Values are kept "lazy": congruent mod p and
// below 2^63, reduced once at the end.  acc * x for acc < 2^63, x < 2^32 is
// p1 2^32 + p0 with p0 = lo32(acc) x < 2^64 and p1 = hi32(acc) x < 2^63; since
// 2^61 == 1, p1 2^32 == (p1 >> 29) + ((p1 mod 2^29) << 32) and p0 == (p0 mod 2^61) +
// (p0 >> 61).  The four terms sum below 2^62 + 2^35, so adding a coefficient
// (< 2^61) keeps the result below 2^63.
__device__ __forceinline__ uint64_t mul_narrow(uint64_t acc, uint32_t x) {
  const uint64_t p0 = (uint64_t)(uint32_t)acc * x;
  const uint64_t p1 = (uint64_t)(uint32_t)(acc >> 32) * x;
  return (p1 >> 29) + ((p1 & ((1ull << 29) - 1)) << 32) + (p0 & kP61) + (p0 >> 61);
}

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

  const int na = A > 0 ? A : p.a;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += step) {
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
      continue;
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
#pragma unroll
        for (int u = 0; u < (A > 0 ? A : kMaxAttrs); u++) {
          if (A == 0 && u >= na) break;
          const uint32_t xu = (uint32_t)x[u];
          const uint64_t h = reduce_lazy(mul_narrow(cr[off + 1], xu) + cr[off]);
          bin += reduce_m<POW2>(h, p.m);
          off += 2;
          for (int e = 0; e < p.deg[u]; e++, off += 4) {
            uint64_t acc = mul_narrow(cr[off + 3], xu) + cr[off + 2];
            acc = mul_narrow(acc, xu) + cr[off + 1];
            acc = mul_narrow(acc, xu) + cr[off];
            sbit ^= (uint32_t)(reduce_lazy(acc) & 1u);
          }
        }
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

__global__ void k_merge(unsigned long long* dst, const unsigned long long* src, int64_t count) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += step) dst[i] += src[i];
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
