// Estimator (Algorithm 3, Eq. 5) and median over rows (Section 3.3).
//
// The host has unrolled Algorithm 3 into a schedule over vector slots (see
// build_plan); every slot holds d rows of m signed 256-bit integers, so every
// intermediate of the algorithm is kept exactly.  The steps:
//   LEAF  slot <- relation sketch (int64 counters, sign-extended)
//   HAD   x <- y o x                   Hadamard product, exact (overflow checked)
//   CORR  x <- a (star) x              circular cross-correlation, Definition 3.1,
//                                      via IFFT(conj(FFT(a)) o FFT(x))
//   SUM   per-row sum, then the lower median of the d row values
//
// CORR splits both operands into L signed B-bit limbs (v = sum_l v_l 2^(B l),
// v_l in [-2^(B-1), 2^(B-1))), runs FP64 FFTs on the limbs (two real limbs
// packed per complex transform), forms for every limb-sum s the spectrum
// sum_{l + l' = s} conj(A_l) X_l', inverts it, rounds every output to the
// nearest integer and recombines z = sum_s 2^(B s) round(y_s) exactly.  B is
// the widest limb for which Percival's a priori bound on the FFT's rounding error
// (with the twiddle table's measured error, see fp64_step_bound) stays at or below
// 1/4, so every rounding is exact by that bound; each step is also checked a
// posteriori: the largest distance of an output to its nearest integer must be
// <= 1/4, per row the exact identity sum_j z_j = (sum_j a_j)(sum_j x_j) must hold
// mod 2^64 and, for power-of-two m, Z(w) = A(1/w) X(w) mod 2^64 - 2^32 + 1 at a
// random primitive m-th root of unity w.  A failed check redoes the step with
// narrower limbs.
//
// FFTs: radix-2 decimation-in-time in shared memory; widths up to 2^12 in one
// pass, wider ones (up to 2^22) as a four-step transform m = R x C (column FFTs
// with the twiddle W_m^(n2 k1) fused, then row FFTs).  Twiddles come from
// sincospi.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "sk_internal.h"

namespace sk {
namespace {

// ---------------------------------------------------------------------------
// signed 256-bit integers (two's complement, little-endian words)
// ---------------------------------------------------------------------------
struct I256 {
  uint64_t w[4];
};

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ I256 i256_from_i64(int64_t v) {
  const uint64_t f = v < 0 ? ~0ull : 0ull;
  return I256{{(uint64_t)v, f, f, f}};
}

__host__ __device__ __forceinline__ I256 i256_add(const I256& a, const I256& b) {
  I256 r;
  uint64_t c = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint64_t s = a.w[k] + b.w[k];
    const uint64_t c1 = s < a.w[k];
    const uint64_t t = s + c;
    const uint64_t c2 = t < s;
    r.w[k] = t;
    c = c1 | c2;
  }
  return r;
}

__host__ __device__ __forceinline__ I256 i256_neg(const I256& a) {
  I256 r;
  uint64_t c = 1;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint64_t t = ~a.w[k] + c;
    c = (c && t == 0) ? 1 : 0;
    r.w[k] = t;
  }
  return r;
}

__host__ __device__ __forceinline__ bool i256_neg_p(const I256& a) { return (int64_t)a.w[3] < 0; }

__host__ __device__ __forceinline__ bool i256_eq(const I256& a, const I256& b) {
  return a.w[0] == b.w[0] && a.w[1] == b.w[1] && a.w[2] == b.w[2] && a.w[3] == b.w[3];
}

// a < b (signed)
__host__ __device__ __forceinline__ bool i256_lt(const I256& a, const I256& b) {
  if (a.w[3] != b.w[3]) return (int64_t)a.w[3] < (int64_t)b.w[3];
  for (int k = 2; k >= 0; k--)
    if (a.w[k] != b.w[k]) return a.w[k] < b.w[k];
  return false;
}

// bit length of |a| (0 for a = 0)
__host__ __device__ __forceinline__ int i256_bits(const I256& a) {
  const I256 m = i256_neg_p(a) ? i256_neg(a) : a;
  for (int k = 3; k >= 0; k--) {
    if (m.w[k]) {
#ifdef __CUDA_ARCH__
      return 64 * k + 64 - __clzll((long long)m.w[k]);
#else
      return 64 * k + 64 - __builtin_clzll(m.w[k]);
#endif
    }
  }
  return 0;
}

// low 256 bits of a * b: the exact product whenever it fits
__host__ __device__ __forceinline__ I256 i256_mul(const I256& a, const I256& b) {
  uint64_t r[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 4; i++) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; i + j < 4; j++) {
      const uint64_t lo = a.w[i] * b.w[j];
      const uint64_t hi = mulhi64(a.w[i], b.w[j]);
      uint64_t s = r[i + j] + lo;
      uint64_t c = s < lo;
      const uint64_t s2 = s + carry;
      c += s2 < s;
      r[i + j] = s2;
      carry = hi + c;
    }
  }
  return I256{{r[0], r[1], r[2], r[3]}};
}

// (int64) v << sh, sign-extended, modulo 2^256; 0 <= sh < 256
__device__ __forceinline__ I256 i256_shl_i64(int64_t v, int sh) {
  const I256 x = i256_from_i64(v);
  const int q = sh >> 6, b = sh & 63;
  I256 r{{0, 0, 0, 0}};
#pragma unroll
  for (int k = 3; k >= 0; k--) {
    const int src = k - q;
    uint64_t val = 0;
    if (src >= 0) {
      val = x.w[src] << b;
      if (b && src - 1 >= 0) val |= x.w[src - 1] >> (64 - b);
    }
    r.w[k] = val;
  }
  return r;
}

// arithmetic shift right by 0 < b < 64
__device__ __forceinline__ I256 i256_sar(const I256& a, int b) {
  I256 r;
#pragma unroll
  for (int k = 0; k < 3; k++) r.w[k] = (a.w[k] >> b) | (a.w[k + 1] << (64 - b));
  r.w[3] = (uint64_t)((int64_t)a.w[3] >> b);
  return r;
}

__device__ __forceinline__ void record(int* status, int code) { atomicCAS(status, 0, code); }

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
// max over the block's values of `bits`, added to *out with atomicMax (out may be null)
__device__ __forceinline__ void block_max_bits(int bits, int* out) {
  if (!out) return;
  for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
  if ((threadIdx.x & 31) == 0 && bits > 0) atomicMax(out, bits);
}

__global__ void k_leaf(I256* __restrict__ dst, const int64_t* __restrict__ src, int64_t n, int* bits_out) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    const int64_t v = src[i];
    const uint64_t a = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
    best = max(best, a ? 64 - __clzll((long long)a) : 0);
    dst[i] = i256_from_i64(v);
  }
  block_max_bits(best, bits_out);
}

__global__ void k_hadamard(I256* __restrict__ x, const I256* __restrict__ y, int64_t n, int* status,
                           int* bits_out) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    const I256 a = x[i], b = y[i];
    if (i256_bits(a) + i256_bits(b) > 255) record(status, SK_ERR_OVERFLOW);
    const I256 z = i256_mul(a, b);
    best = max(best, i256_bits(z));
    x[i] = z;
  }
  block_max_bits(best, bits_out);
}

__global__ void k_maxbits(const I256* __restrict__ v, int64_t n, int* out) {
  int best = 0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step)
    best = max(best, i256_bits(v[i]));
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(out, best);
}

// per-row exact sums: one block per row, four independent accumulators per thread
__global__ void k_rowsum(const I256* __restrict__ v, int64_t m, I256* out) {
  __shared__ I256 part[32];
  const I256* row = v + (int64_t)blockIdx.x * m;
  I256 acc{{0, 0, 0, 0}}, acc1{{0, 0, 0, 0}}, acc2{{0, 0, 0, 0}}, acc3{{0, 0, 0, 0}};
  const int64_t step = blockDim.x;
  int64_t j = threadIdx.x;
  for (; j + 3 * step < m; j += 4 * step) {
    acc = i256_add(acc, row[j]);
    acc1 = i256_add(acc1, row[j + step]);
    acc2 = i256_add(acc2, row[j + 2 * step]);
    acc3 = i256_add(acc3, row[j + 3 * step]);
  }
  for (; j < m; j += step) acc = i256_add(acc, row[j]);
  acc = i256_add(i256_add(acc, acc1), i256_add(acc2, acc3));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    I256 t;
#pragma unroll
    for (int k = 0; k < 4; k++) t.w[k] = __shfl_xor_sync(0xffffffffu, acc.w[k], o);
    acc = i256_add(acc, t);
  }
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    I256 s{{0, 0, 0, 0}};
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s = i256_add(s, part[w]);
    out[blockIdx.x] = s;
  }
}

// sorted copy of the d row estimates (the lower median is sorted[(d-1)/2])
__global__ void k_sort_rows(const I256* __restrict__ rows, int d, I256* sorted) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < d; i++) {
    const I256 v = rows[i];
    int j = i - 1;
    while (j >= 0 && i256_lt(v, sorted[j])) {
      sorted[j + 1] = sorted[j];
      j--;
    }
    sorted[j + 1] = v;
  }
}

// ---------------------------------------------------------------------------
// FFT
// ---------------------------------------------------------------------------
__global__ void k_twiddle(double2* tw, int64_t n) {
  const int64_t half = n >> 1;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += step) {
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_double2(c, -s);   // W_n^t = exp(-2 pi i t / n)
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------------------
// Arithmetic of the Goldilocks prime field GF(q), q = 2^64 - 2^32 + 1, used by the
// number-theoretic transform.  2^64 = 2^32 - 1 and 2^96 = -1 (mod q), so a 128-bit
// product hi 2^64 + lo with hi = hh 2^32 + hl reduces to lo - hh + hl (2^32 - 1).
// Inputs are canonical (< q); outputs are canonical.
// ---------------------------------------------------------------------------
constexpr uint64_t kGL = 0xFFFFFFFF00000001ull;
constexpr uint64_t kGLEps = 0xFFFFFFFFull;   // 2^64 mod q

__host__ __device__ __forceinline__ uint64_t gl_add(uint64_t a, uint64_t b) {
  uint64_t s = a + b;
  if (s < a) s += kGLEps;               // wrapped past 2^64: add 2^64 mod q
  return s >= kGL ? s - kGL : s;
}

__host__ __device__ __forceinline__ uint64_t gl_sub(uint64_t a, uint64_t b) {
  uint64_t d = a - b;
  if (a < b) d -= kGLEps;               // borrowed 2^64: subtract 2^64 - q
  return d;
}

__host__ __device__ __forceinline__ uint64_t gl_mul(uint64_t a, uint64_t b) {
  const uint64_t lo = a * b;
  const uint64_t hi = mulhi64(a, b);
  const uint64_t hh = hi >> 32, hl = hi & kGLEps;
  uint64_t t = lo - hh;
  if (lo < hh) t -= kGLEps;
  const uint64_t u = hl * kGLEps;
  uint64_t r = t + u;
  if (r < u) r += kGLEps;
  return r >= kGL ? r - kGL : r;
}

__host__ __device__ __forceinline__ uint64_t gl_pow(uint64_t b, uint64_t e) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = gl_mul(r, b);
    b = gl_mul(b, b);
    e >>= 1;
  }
  return r;
}

// ---------------------------------------------------------------------------
// Transforms.  One radix-2 DIT machinery serves two arithmetics:
//   CplxOps: complex FP64, twiddles W_n^t = exp(-2 pi i t / n) (inverse: conjugates);
//   GlOps:   GF(q), twiddles w^t for a primitive n-th root of unity w (the inverse
//            transform is handed the table of w^-t).
// Both satisfy W^(n/2) = -1, which the four-step twiddle uses.
// ---------------------------------------------------------------------------
struct CplxOps {
  using T = double2;
  static constexpr bool kExact = false;   // rounding: twiddles always come from the table
  static constexpr bool kReg = false;     // transforms through smem_dif_il
  static __device__ __forceinline__ T mul(T a, T b) { return cmul(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ T sub(T a, T b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ T neg(T a) { return make_double2(-a.x, -a.y); }
  static __device__ __forceinline__ T tw(const T* tab, int64_t i, bool inv) {
    T w = tab[i];
    if (inv) w.y = -w.y;
    return w;
  }
  // W_4h^(pos + h) = W_4h^pos * W_4^1: -i times w (forward), +i times w (inverse)
  static __device__ __forceinline__ T rot4(T w, bool inv, T) {
    return inv ? make_double2(-w.y, w.x) : make_double2(w.y, -w.x);
  }
};

struct GlOps {
  using T = uint64_t;
  static constexpr bool kExact = true;
  static constexpr bool kReg = false;   // transforms through smem_dif_il
  static __device__ __forceinline__ T mul(T a, T b) { return gl_mul(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return gl_add(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return gl_sub(a, b); }
  static __device__ __forceinline__ T neg(T a) { return a ? kGL - a : 0; }
  static __device__ __forceinline__ T tw(const T* tab, int64_t i, bool) { return tab[i]; }
  static __device__ __forceinline__ T rot4(T w, bool, T r4) { return gl_mul(w, r4); }
};

// w^e for 0 <= e < n from the half table
template <class Ops>
__device__ __forceinline__ typename Ops::T twid(const typename Ops::T* __restrict__ tw, int64_t e, int64_t half,
                                                bool inv) {
  return e < half ? Ops::tw(tw, e, inv) : Ops::neg(Ops::tw(tw, e - half, inv));
}

// In-place radix-2 DIT transforms of `cnt` vectors of length 2^logL stored back to back
// in shared memory, input already in bit-reversed order.  tw is the half table of the
// length-N transform; a length-L transform uses w_L^e = w_N^(e * N / L), twstride = N / L.
// r4 is w_N^(N/4) (GlOps only; complex uses -i).
template <class Ops>
__device__ void smem_xform(typename Ops::T* s, int cnt, int logL, const typename Ops::T* __restrict__ tw,
                           int64_t twstride, bool inv, typename Ops::T r4) {
  using T = typename Ops::T;
  const int L = 1 << logL;
  const int halfL = L >> 1;
  const int total = cnt * halfL;
  int st = 0;
  // Pairs of radix-2 stages (half sizes h and 2h) fused: the four elements b, b+h, b+2h,
  // b+3h (b = group * 4h + pos, pos < h) are closed under both stages.  Stage one
  // pairs (b, b+h), (b+2h, b+3h) with w_2h^pos; stage two pairs (b, b+2h) with
  // w_4h^pos and (b+h, b+3h) with w_4h^(pos+h) = w_4h^pos * w_4.
  if (logL >= 2) {
    const int quarterL = L >> 2;
    const int total4 = cnt * quarterL;
    for (; st + 1 < logL; st += 2) {
      const int h = 1 << st;
      const int64_t t1 = (int64_t)(L >> (st + 1)) * twstride;   // w_2h^pos = tw[pos * t1]
      const int64_t t2 = (int64_t)(L >> (st + 2)) * twstride;   // w_4h^pos = tw[pos * t2]
      for (int b4 = threadIdx.x; b4 < total4; b4 += blockDim.x) {
        const int v = b4 >> (logL - 2);
        const int jj = b4 & (quarterL - 1);
        const int grp = jj >> st, pos = jj & (h - 1);
        const int i0 = v * L + grp * 4 * h + pos;
        const T w1 = Ops::tw(tw, (int64_t)pos * t1, inv);
        const T w2 = Ops::tw(tw, (int64_t)pos * t2, inv);
        const T w3 = Ops::rot4(w2, inv, r4);
        const T a0 = s[i0], a1 = s[i0 + h], a2 = s[i0 + 2 * h], a3 = s[i0 + 3 * h];
        const T t01 = Ops::mul(a1, w1), t23 = Ops::mul(a3, w1);
        const T b0 = Ops::add(a0, t01), b1 = Ops::sub(a0, t01);
        const T b2 = Ops::add(a2, t23), b3 = Ops::sub(a2, t23);
        const T u2 = Ops::mul(b2, w2), u3 = Ops::mul(b3, w3);
        s[i0] = Ops::add(b0, u2);
        s[i0 + 2 * h] = Ops::sub(b0, u2);
        s[i0 + h] = Ops::add(b1, u3);
        s[i0 + 3 * h] = Ops::sub(b1, u3);
      }
      __syncthreads();
    }
  }
  for (; st < logL; st++) {
    const int h = 1 << st;
    const int64_t tstep = (int64_t)(L >> (st + 1)) * twstride;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int v = b >> (logL - 1);
      const int jj = b & (halfL - 1);
      const int grp = jj >> st, pos = jj & (h - 1);
      const int i0 = v * L + grp * 2 * h + pos;
      const int i1 = i0 + h;
      const T w = Ops::tw(tw, (int64_t)pos * tstep, inv);
      const T a = s[i0];
      const T t = Ops::mul(s[i1], w);
      s[i0] = Ops::add(a, t);
      s[i1] = Ops::sub(a, t);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int i, int bits) { return (int)(__brev((unsigned)i) >> (32 - bits)); }

// whole transforms of length L = 2^logL <= 4096, vpc vectors per block
template <class Ops>
__global__ void k_xf_small(const typename Ops::T* __restrict__ in, typename Ops::T* __restrict__ out, int64_t batch,
                           int logL, int vpc, const typename Ops::T* __restrict__ tw, int64_t twstride, bool inv,
                           typename Ops::T r4) {
  using T = typename Ops::T;
  extern __shared__ __align__(16) unsigned char xf_smem[];
  T* sm = (T*)xf_smem;
  const int L = 1 << logL;
  const int64_t v0 = (int64_t)blockIdx.x * vpc;
  const int64_t rem = batch - v0;
  const int cnt = (int)(rem < (int64_t)vpc ? rem : (int64_t)vpc);
  for (int idx = threadIdx.x; idx < cnt * L; idx += blockDim.x) {
    const int v = idx >> logL, i = idx & (L - 1);
    sm[v * L + bitrev(i, logL)] = in[(v0 + v) * L + i];
  }
  __syncthreads();
  smem_xform<Ops>(sm, cnt, logL, tw, twstride, inv, r4);
  for (int idx = threadIdx.x; idx < cnt * L; idx += blockDim.x) out[(v0 * L) + idx] = sm[idx];
}

// In-place radix-2 decimation-in-frequency transforms (natural-order input, output in
// bit-reversed order) of `cnt` vectors of length 2^logL held interleaved in shared
// memory: element i of vector v at s[i * S + v] with S = cnt + 1 (odd, so that the
// transposing loads of the row pass and the bit-reversed reads stay conflict-free).
// Consecutive threads take consecutive vectors of the same butterfly: every access of a
// warp is a contiguous run and the butterfly's twiddle is the same across it.  Pairs of
// stages (half sizes 2q and q) are fused on the four elements i0 + {0, q, 2q, 3q}.
// tw is the half table of the length-N transform, twstride = N / L; r4 as in smem_xform.
template <class Ops>
__device__ void smem_dif_il(typename Ops::T* s, int cnt, int S, int logL, const typename Ops::T* __restrict__ tw,
                            int64_t twstride, bool inv, typename Ops::T r4) {
  using T = typename Ops::T;
  const int L = 1 << logL;
  const int lc = __ffs(cnt) - 1;   // cnt is a power of two: indices by shifts, not divisions
  int lh = logL - 1;   // log2 of the larger half size of the pair
  for (; lh >= 1; lh -= 2) {
    const int q = 1 << (lh - 1);
    const int64_t s4 = (int64_t)(L >> (lh + 1)) * twstride;   // w_4q^pos = tw[pos * s4]
    const int64_t s2 = (int64_t)(L >> lh) * twstride;         // w_2q^pos = tw[pos * s2]
    const int total4 = cnt * (L >> 2);
    const int qS = q * S;
    for (int b = threadIdx.x; b < total4; b += blockDim.x) {
      const int v = b & (cnt - 1), jj = b >> lc;
      const int grp = jj >> (lh - 1), pos = jj & (q - 1);
      T* e = s + (grp * 4 * q + pos) * S + v;
      const T w4 = Ops::tw(tw, (int64_t)pos * s4, inv);
      const T w4b = Ops::rot4(w4, inv, r4);                    // w_4q^(pos + q)
      const T w2 = Ops::tw(tw, (int64_t)pos * s2, inv);
      const T e0 = e[0], e1 = e[qS], e2 = e[2 * qS], e3 = e[3 * qS];
      const T u0 = Ops::add(e0, e2), u2 = Ops::mul(Ops::sub(e0, e2), w4);
      const T u1 = Ops::add(e1, e3), u3 = Ops::mul(Ops::sub(e1, e3), w4b);
      e[0] = Ops::add(u0, u1);
      e[qS] = Ops::mul(Ops::sub(u0, u1), w2);
      e[2 * qS] = Ops::add(u2, u3);
      e[3 * qS] = Ops::mul(Ops::sub(u2, u3), w2);
    }
    __syncthreads();
  }
  if (lh == 0) {   // odd logL: the last stage, half size 1 (twiddle 1)
    const int total = cnt * (L >> 1);
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int v = b & (cnt - 1), g = b >> lc;
      T* e = s + (2 * g) * S + v;
      const T a0 = e[0], a1 = e[S];
      e[0] = Ops::add(a0, a1);
      e[S] = Ops::sub(a0, a1);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Register transforms (exact arithmetics only, lengths L = 2^6..2^10).  A length-L DFT in
// natural order is taken as A x B (L = A B): with x_i at i = B a + b and X_k at k = c + A e,
//   X[c + A e] = sum_b w_B^(b e) (w_L^(b c) sum_a x[B a + b] w_A^(a c)),
// so step 1 gives each thread one b: the A-point DFT over a of its stride-B elements, held in
// registers, times w_L^(b c), written back to the same positions B c + b; step 2 gives each
// thread one c: the B-point DFT over b of the contiguous block B c .. B c + B - 1, written
// to the positions c + A e.  Every twiddle is a power of w_L, read from an L-entry table in
// shared memory (the same entry across the threads of one vector: broadcast reads).
// ---------------------------------------------------------------------------
template <int LOG>
__host__ __device__ constexpr int bitrev_const(int k) {
  int r = 0;
  for (int i = 0; i < LOG; i++) r |= ((k >> i) & 1) << (LOG - 1 - i);
  return r;
}

// 2^LOG-point DFT of x (natural order in and out); wt[j] = w_N^j for j < N / 2.  Radix-2
// decimation in frequency (stage s pairs j and j + N / 2^(s+1) with the twiddle
// w_N^(j 2^s)), then the bit reversal as a renaming of registers.
template <class Ops, int LOG>
__device__ __forceinline__ void reg_dft(typename Ops::T (&x)[1 << LOG], const typename Ops::T (&wt)[(1 << LOG) / 2]) {
  using T = typename Ops::T;
  constexpr int N = 1 << LOG;
#pragma unroll
  for (int st = 0; st < LOG; st++) {
    const int h = N >> (st + 1);
#pragma unroll
    for (int blk = 0; blk < N; blk += 2 * h) {
#pragma unroll
      for (int j = 0; j < h; j++) {
        const T u = x[blk + j], v = x[blk + j + h];
        x[blk + j] = Ops::add(u, v);
        const T dl = Ops::sub(u, v);
        x[blk + j + h] = j == 0 ? dl : Ops::mul(dl, wt[j << st]);
      }
    }
  }
  T y[N];
#pragma unroll
  for (int k = 0; k < N; k++) y[k] = x[bitrev_const<LOG>(k)];
#pragma unroll
  for (int k = 0; k < N; k++) x[k] = y[k];
}

// In-place natural-order DFTs of `cnt` (a power of two) vectors of length L = 2^(LA + LB),
// element i of vector v at s[i S + v]; stw[e] = w_L^e for e < L.  Needs cnt 2^max(LA, LB)
// <= blockDim.x (one A- or B-point DFT per thread and step).  Ends with a barrier.
template <class Ops, int LA, int LB>
__device__ void smem_ntt_2lvl(typename Ops::T* s, int cnt, int S, const typename Ops::T* stw) {
  using T = typename Ops::T;
  constexpr int A = 1 << LA, B = 1 << LB;
  const int lc = __ffs(cnt) - 1;
  const int t = threadIdx.x;
  {
    T w[A / 2];
#pragma unroll
    for (int j = 0; j < A / 2; j++) w[j] = stw[B * j];   // w_A^j
    if (t < cnt * B) {
      const int v = t & (cnt - 1), b = t >> lc;
      T x[A];
#pragma unroll
      for (int a = 0; a < A; a++) x[a] = s[(B * a + b) * S + v];
      reg_dft<Ops, LA>(x, w);
#pragma unroll
      for (int c = 1; c < A; c++) x[c] = Ops::mul(x[c], stw[b * c]);
#pragma unroll
      for (int c = 0; c < A; c++) s[(B * c + b) * S + v] = x[c];
    }
  }
  __syncthreads();
  {
    T w[B / 2];
#pragma unroll
    for (int j = 0; j < B / 2; j++) w[j] = stw[A * j];   // w_B^j
    const bool act = t < cnt * A;
    const int v = t & (cnt - 1), c = t >> lc;
    T x[B];
    if (act) {
#pragma unroll
      for (int b = 0; b < B; b++) x[b] = s[(B * c + b) * S + v];
    }
    __syncthreads();   // every block read before any position c + A e is written
    if (act) {
      reg_dft<Ops, LB>(x, w);
#pragma unroll
      for (int e = 0; e < B; e++) s[(c + A * e) * S + v] = x[e];
    }
  }
  __syncthreads();
}

// The register transform for length 2^logL when this arithmetic has one (kReg) and the tile
// of cnt vectors fits it; fills stw (L entries) from the length-N half table first.  false:
// nothing done (the caller takes smem_dif_il, bit-reversed output).
template <class Ops>
__device__ bool smem_ntt_reg(typename Ops::T* s, int cnt, int S, int logL, const typename Ops::T* __restrict__ tw,
                             int64_t twstride, int64_t N, bool inv, typename Ops::T* stw) {
  if constexpr (Ops::kReg) {
    if (logL < 6 || logL > 10 || (cnt << (logL - logL / 2)) > (int)blockDim.x) return false;
    const int L = 1 << logL;
    for (int e = threadIdx.x; e < L; e += blockDim.x) stw[e] = twid<Ops>(tw, ((int64_t)e * twstride) & (N - 1), N >> 1, inv);
    __syncthreads();
    switch (logL) {
      case 6: smem_ntt_2lvl<Ops, 3, 3>(s, cnt, S, stw); break;
      case 7: smem_ntt_2lvl<Ops, 3, 4>(s, cnt, S, stw); break;
      case 8: smem_ntt_2lvl<Ops, 4, 4>(s, cnt, S, stw); break;
      case 9: smem_ntt_2lvl<Ops, 4, 5>(s, cnt, S, stw); break;
      default: smem_ntt_2lvl<Ops, 5, 5>(s, cnt, S, stw); break;
    }
    return true;
  } else {
    return false;
  }
}

// loads each thread of the four-step passes keeps in flight while filling its tile (16
// measured no faster than 8 for 32-bit residues)
template <class T>
constexpr int kLoadBatchOf = 8;

// four-step, pass 1: length-R transforms down the columns of the R x C view
// (element n1 * C + n2), then the twiddle w_N^(n2 k1); in place.  Tile: cb columns.
template <class Ops>
__global__ void __launch_bounds__(512, 2) k_xf_cols(typename Ops::T* __restrict__ buf, int logR, int logC, int cb,
                          const typename Ops::T* __restrict__ tw, bool inv, typename Ops::T r4) {
  using T = typename Ops::T;
  extern __shared__ __align__(16) unsigned char xf_smem[];
  T* sm = (T*)xf_smem;
  const int R = 1 << logR, C = 1 << logC;
  const int S = cb + 1;
  const int64_t N = (int64_t)R * C;
  const int lcb = __ffs(cb) - 1;   // cb is a power of two
  const int blocks_per_vec = C >> lcb;
  const int64_t vec = blockIdx.x >> (logC - lcb);
  const int c0 = (blockIdx.x & (blocks_per_vec - 1)) * cb;
  T* v = buf + vec * N;
  // the tile: kLoadBatch loads per thread in flight before their shared-memory stores
  constexpr int kLoadBatch = kLoadBatchOf<T>;
  for (int i0 = threadIdx.x; i0 < R * cb; i0 += kLoadBatch * blockDim.x) {
    T tmp[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; u++) {
      const int idx = i0 + u * (int)blockDim.x;
      if (idx < R * cb) tmp[u] = v[(int64_t)(idx >> lcb) * C + c0 + (idx & (cb - 1))];
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; u++) {
      const int idx = i0 + u * (int)blockDim.x;
      if (idx < R * cb) sm[(idx >> lcb) * S + (idx & (cb - 1))] = tmp[u];
    }
  }
  __syncthreads();
  // natural-order register transform where it applies (its twiddle table after the tile),
  // else the radix-2 one with bit-reversed output
  const bool nat = smem_ntt_reg<Ops>(sm, cb, S, logR, tw, C, N, inv, sm + (int64_t)R * S);
  if (!nat) smem_dif_il<Ops>(sm, cb, S, logR, tw, C, inv, r4);
  const int64_t half = N >> 1;
  if (Ops::kExact && (blockDim.x & (cb - 1)) == 0) {
    // each thread keeps one column n2 and walks rows k1 = k1_0 + j kstep: the twiddle
    // w^(n2 k1) advances by the factor w^(n2 kstep) (exact modular products), instead of a
    // table load per element at the scattered index n2 k1
    const int c = threadIdx.x & (cb - 1), kstep = blockDim.x >> lcb;
    const int64_t n2 = c0 + c;
    T w = twid<Ops>(tw, (n2 * (threadIdx.x >> lcb)) & (N - 1), half, inv);
    const T ws = twid<Ops>(tw, (n2 * kstep) & (N - 1), half, inv);
    for (int k1 = threadIdx.x >> lcb; k1 < R; k1 += kstep) {
      v[(int64_t)k1 * C + n2] = Ops::mul(sm[(nat ? k1 : bitrev(k1, logR)) * S + c], w);
      w = Ops::mul(w, ws);
    }
  } else {
    for (int idx = threadIdx.x; idx < R * cb; idx += blockDim.x) {
      const int c = idx & (cb - 1), k1 = idx >> lcb;
      const int64_t n2 = c0 + c;
      const T w = twid<Ops>(tw, (n2 * k1) & (N - 1), half, inv);
      v[(int64_t)k1 * C + n2] = Ops::mul(sm[(nat ? k1 : bitrev(k1, logR)) * S + c], w);
    }
  }
}

// four-step, pass 2: length-C transforms along the rows k1, written to the
// natural-order output X[k1 + R k2]; out of place.  Tile: rb rows.
template <class Ops>
__global__ void __launch_bounds__(512, 2) k_xf_rows(const typename Ops::T* __restrict__ in, typename Ops::T* __restrict__ out, int logR,
                          int logC, int rb, const typename Ops::T* __restrict__ tw, bool inv, typename Ops::T r4) {
  using T = typename Ops::T;
  extern __shared__ __align__(16) unsigned char xf_smem[];
  T* sm = (T*)xf_smem;
  const int R = 1 << logR, C = 1 << logC;
  const int S = rb + 1;
  const int64_t N = (int64_t)R * C;
  const int lrb = __ffs(rb) - 1;   // rb is a power of two
  const int blocks_per_vec = R >> lrb;
  const int64_t vec = blockIdx.x >> (logR - lrb);
  const int r0 = (blockIdx.x & (blocks_per_vec - 1)) * rb;
  const T* vi = in + vec * N;
  T* vo = out + vec * N;
  constexpr int kLoadBatch = kLoadBatchOf<T>;
  for (int i0 = threadIdx.x; i0 < C * rb; i0 += kLoadBatch * blockDim.x) {
    T tmp[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; u++) {
      const int idx = i0 + u * (int)blockDim.x;
      if (idx < C * rb) tmp[u] = vi[(int64_t)(r0 + (idx >> logC)) * C + (idx & (C - 1))];
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; u++) {
      const int idx = i0 + u * (int)blockDim.x;
      if (idx < C * rb) sm[(idx & (C - 1)) * S + (idx >> logC)] = tmp[u];
    }
  }
  __syncthreads();
  const bool nat = smem_ntt_reg<Ops>(sm, rb, S, logC, tw, R, N, inv, sm + (int64_t)C * S);
  if (!nat) smem_dif_il<Ops>(sm, rb, S, logC, tw, R, inv, r4);
  for (int idx = threadIdx.x; idx < C * rb; idx += blockDim.x) {
    const int rr = idx & (rb - 1), k2 = idx >> lrb;
    vo[(int64_t)(r0 + rr) + (int64_t)R * k2] = sm[(nat ? k2 : bitrev(k2, logC)) * S + rr];
  }
}

// ---------------------------------------------------------------------------
// Evaluation certificate of an FP64 correlation step (power-of-two m).  For z = a star x
// (Definition 3.1) and any m-th root of unity w in GF(q), q = 2^64 - 2^32 + 1,
//   sum_j z_j w^j = sum_i a_i w^-i * sum_k x_k w^k        (w^m = 1, k = i + j mod m),
// so Z(w) = A(1/w) X(w).  With w a random primitive m-th root, a wrong z_j passes with
// probability at most (m - 1) / q.  Each block sums one chunk of one row (consecutive
// threads read consecutive elements); k_eval_final adds the chunks.
// ---------------------------------------------------------------------------
struct EvalArgs {
  const I256* a;
  const I256* x;
  const I256* z;
  int64_t m;
  int nchunk;
  uint64_t w, winv;            // w and 1/w
  uint64_t wstep, winvstep;    // w^blockDim and its inverse
  uint64_t e1, e2, e3, e4;     // 2^64k mod q, k = 1..4
  uint64_t* part;              // [d][nchunk][3]
};

__device__ __forceinline__ uint64_t gl_canon(uint64_t v) { return v >= kGL ? v - kGL : v; }

// a signed 256-bit value mod q
__device__ __forceinline__ uint64_t i256_mod_gl(const I256& v, const EvalArgs& p) {
  uint64_t r = gl_canon(v.w[0]);
  r = gl_add(r, gl_mul(gl_canon(v.w[1]), p.e1));
  r = gl_add(r, gl_mul(gl_canon(v.w[2]), p.e2));
  r = gl_add(r, gl_mul(gl_canon(v.w[3]), p.e3));
  if ((int64_t)v.w[3] < 0) r = gl_sub(r, p.e4);   // two's complement: value = unsigned - 2^256
  return r;
}

__global__ void __launch_bounds__(256) k_eval_partial(EvalArgs p) {
  __shared__ uint64_t red[3][256];
  const int row = blockIdx.x / p.nchunk, c = blockIdx.x % p.nchunk;
  const int64_t clen = p.m / p.nchunk;
  const int64_t j0 = (int64_t)c * clen + threadIdx.x;
  const int64_t j1 = (int64_t)(c + 1) * clen;
  uint64_t sa = 0, sx = 0, sz = 0;
  if (j0 < j1) {
    uint64_t pw = gl_pow(p.w, (uint64_t)j0), pi = gl_pow(p.winv, (uint64_t)j0);
    const int64_t base = (int64_t)row * p.m;
    for (int64_t j = j0; j < j1; j += blockDim.x) {
      sa = gl_add(sa, gl_mul(i256_mod_gl(p.a[base + j], p), pi));
      sx = gl_add(sx, gl_mul(i256_mod_gl(p.x[base + j], p), pw));
      sz = gl_add(sz, gl_mul(i256_mod_gl(p.z[base + j], p), pw));
      pw = gl_mul(pw, p.wstep);
      pi = gl_mul(pi, p.winvstep);
    }
  }
  red[0][threadIdx.x] = sa;
  red[1][threadIdx.x] = sx;
  red[2][threadIdx.x] = sz;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int k = 0; k < 3; k++) red[k][threadIdx.x] = gl_add(red[k][threadIdx.x], red[k][threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x < 3) p.part[((int64_t)row * p.nchunk + c) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// out[row * 3 + k] = sum over chunks of part[row][chunk][k] (k: A(1/w), X(w), Z(w))
__global__ void k_eval_final(const uint64_t* part, int d, int nchunk, unsigned long long* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * d) return;
  const int row = t / 3, k = t % 3;
  uint64_t sum = 0;
  for (int c = 0; c < nchunk; c++) sum = gl_add(sum, part[((int64_t)row * nchunk + c) * 3 + k]);
  out[row * 3 + k] = sum;
}

// GF(q) twiddle tables for a length-n transform: tw[t] = w^t and itw[t] = w^-t, t < n/2.
__global__ void k_gl_twiddle(uint64_t* tw, uint64_t* itw, int64_t n, uint64_t w, uint64_t winv) {
  const int64_t half = n >> 1;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += step) {
    tw[t] = gl_pow(w, (uint64_t)t);
    itw[t] = gl_pow(winv, (uint64_t)t);
  }
}

// ---------------------------------------------------------------------------
// limb split, spectral products, recombination
// ---------------------------------------------------------------------------
struct CorrArgs {
  const I256* a;     // [d][m]
  const I256* x;     // [d][m]
  I256* z;           // [d][m] output
  double2* F;        // packed forward buffer [d][nf][m]
  double2* G;        // packed inverse buffer [d][ni][m]
  int64_t m;
  int logm;
  int d;
  int B;             // limb bits
  int La, Lx;        // limbs of a and x
  int nf, ni;
  int* status;
  unsigned long long* residual;   // max |y - rint(y)| as double bits
  unsigned long long* sums;       // optional [d][3]: row sums mod 2^64 of a, x, z
  int* zbits;                     // optional: bit length of max |z|
  int64_t M;                      // FFT length: m for power-of-two m, else a power of two >= 2m - 1
};

// Adds v (one value of row `row`) to sums[row * 3 + col] mod 2^64.  With warp_rows the
// caller guarantees that the 32 lanes of every warp are active and in one row, and the
// warp reduces first.
__device__ __forceinline__ void row_sum_add(unsigned long long* sums, bool warp_rows, int64_t row, int col,
                                            unsigned long long v) {
  if (warp_rows) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sums + row * 3 + col, v);
  } else {
    atomicAdd(sums + row * 3 + col, v);
  }
}

// Real vector number q of the forward batch: q < La -> limb q of a, else limb q-La of x.
// Packed complex vector t holds real vectors 2t (real part) and 2t+1 (imaginary part).
// Limb split over the FFT length M: positions j >= m (zero padding when m is not a
// power of two) get zero limbs.
__global__ void k_split(CorrArgs p) {
  const int64_t total = (int64_t)p.d * p.M;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int64_t half = 1ll << (p.B - 1), full = 1ll << p.B;
  const int lM = __ffsll((unsigned long long)p.M) - 1;   // M is a power of two
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, j = g & (p.M - 1);
    double2* F = p.F + (row * p.nf) * p.M + j;
    const bool in = j < p.m;
    const int64_t e = row * p.m + j;
    if (p.sums) {
      row_sum_add(p.sums, p.M >= 32, row, 0, in ? p.a[e].w[0] : 0ull);
      row_sum_add(p.sums, p.M >= 32, row, 1, in ? p.x[e].w[0] : 0ull);
    }
    if (!in) {
      const int nreal = p.La + p.Lx;
      for (int t = 0; t < (nreal + 1) / 2; t++) F[(int64_t)t * p.M] = make_double2(0.0, 0.0);
      continue;
    }
    for (int which = 0; which < 2; which++) {
      I256 v = which == 0 ? p.a[e] : p.x[e];
      const int L = which == 0 ? p.La : p.Lx;
      const int base = which == 0 ? 0 : p.La;
      for (int l = 0; l < L; l++) {
        int64_t dig = (int64_t)(v.w[0] & (uint64_t)(full - 1));
        if (dig >= half) dig -= full;
        v = i256_add(v, i256_from_i64(-dig));
        v = i256_sar(v, p.B);
        const int q = base + l;
        double* slot = (double*)(F + (int64_t)(q >> 1) * p.M) + (q & 1);
        *slot = (double)dig;
      }
      if (v.w[0] | v.w[1] | v.w[2] | v.w[3]) record(p.status, SK_ERR_OVERFLOW);
    }
    const int nreal = p.La + p.Lx;
    if (nreal & 1) ((double*)(F + (int64_t)(nreal >> 1) * p.M))[1] = 0.0;
  }
}

__global__ void k_product(CorrArgs p) {
  const int64_t total = (int64_t)p.d * p.M;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int lM = __ffsll((unsigned long long)p.M) - 1;   // M is a power of two
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, k = g & (p.M - 1);
    const int64_t mk = (p.M - k) & (p.M - 1);
    const double2* F = p.F + (row * p.nf) * p.M;
    double2 A[kMaxLimbs], X[kMaxLimbs];
    const int nreal = p.La + p.Lx;
    for (int q = 0; q < nreal; q++) {
      const int t = q >> 1;
      const double2 zk = F[(int64_t)t * p.M + k];
      const double2 zm = F[(int64_t)t * p.M + mk];
      // Z = FFT(u + i v): U[k] = (Z[k] + conj Z[-k]) / 2, V[k] = (Z[k] - conj Z[-k]) / (2i)
      double2 s;
      if ((q & 1) == 0) {
        s = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
      } else {
        const double dr = zk.x - zm.x, di = zk.y + zm.y;
        s = make_double2(0.5 * di, -0.5 * dr);
      }
      if (q < p.La) A[q] = s; else X[q - p.La] = s;
    }
    double2* G = p.G + (row * p.ni) * p.M + k;
    const int ns = p.La + p.Lx - 1;
    for (int t = 0; t < p.ni; t++) {
      double2 P[2];
      for (int h = 0; h < 2; h++) {
        const int s = 2 * t + h;
        double re = 0.0, im = 0.0;
        if (s < ns) {
          const int l0 = max(0, s - (p.Lx - 1)), l1 = min(s, p.La - 1);
          for (int l = l0; l <= l1; l++) {
            const double2 a = A[l], x = X[s - l];
            // conj(a) * x
            re += a.x * x.x + a.y * x.y;
            im += a.x * x.y - a.y * x.x;
          }
        }
        P[h] = make_double2(re, im);
      }
      // pack the two real-output spectra: IFFT(P0 + i P1) = y0 + i y1
      G[(int64_t)t * p.M] = make_double2(P[0].x - P[1].y, P[0].y + P[1].x);
    }
  }
}

__global__ void k_recombine(CorrArgs p, const double2* __restrict__ Y) {
  const int64_t total = (int64_t)p.d * p.m;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const double inv_m = 1.0 / (double)p.M;
  const bool warp_rows = (p.m & 31) == 0;
  const bool padded = p.M != p.m;
  const int ns = p.La + p.Lx - 1;
  double worst = 0.0;
  int zb = 0;
  const bool mp2 = (p.m & (p.m - 1)) == 0;
  const int lm = __ffsll((unsigned long long)p.m) - 1;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = mp2 ? g >> lm : g / p.m, j = g - row * p.m;
    const double2* y = Y + (row * p.ni) * p.M + j;
    I256 z{{0, 0, 0, 0}};
    for (int s = 0; s < ns; s++) {
      const double2 c = y[(int64_t)(s >> 1) * p.M];
      double v = ((s & 1) ? c.y : c.x) * inv_m;
      if (padded && j > 0) {   // circular lag j = linear lag j plus linear lag j - m
        const double2 c2 = y[(int64_t)(s >> 1) * p.M + (p.M - p.m)];
        v += ((s & 1) ? c2.y : c2.x) * inv_m;
      }
      const double rv = rint(v);
      worst = fmax(worst, fabs(v - rv));
      // beyond 2^52 a double no longer resolves integers: fail this step's certificate (the
      // residual check), so the step is redone with narrower limbs
      if (fabs(rv) >= 4503599627370496.0) worst = 1.0;   // 2^52
      z = i256_add(z, i256_shl_i64((int64_t)rv, p.B * s));
    }
    p.z[g] = z;
    if (p.sums) row_sum_add(p.sums, warp_rows, row, 2, z.w[0]);
    zb = max(zb, i256_bits(z));
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(p.residual, (unsigned long long)__double_as_longlong(worst));
  block_max_bits(zb, p.zbits);
}

// ---------------------------------------------------------------------------
// Exact correlation by number-theoretic transform over GF(q), q = 2^64 - 2^32 + 1.
// Operands are split into signed B-bit limbs as for the FP64 path; each limb vector is
// transformed (w a primitive M-th root of unity); for every limb sum s the product
// sum_{l + l' = s} A_l(w^-k) X_l'(w^k) is formed (A at index M - k) and transformed
// back.  B is chosen so that every output satisfies |y_s| <= pairs m 2^(2B-2) < 2^62 <
// q / 2, so the residue determines y_s exactly: no rounding, exact by construction.
// ---------------------------------------------------------------------------
struct NttArgs {
  const I256* a;
  const I256* x;
  I256* z;
  uint64_t* F;       // [d][nl][M] limb residues / spectra
  uint64_t* G;       // [d][ns][M] products / outputs
  int64_t m, M;
  int d, B, La, Lx, nl, ns;
  int* status;
  unsigned long long* sums;   // [d][3] row sums mod 2^64 of a, x, z
  int* zbits;
  uint64_t minv;              // M^-1 mod q
};

__global__ void k_nsplit(NttArgs p) {
  const int64_t total = (int64_t)p.d * p.M;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int64_t half = 1ll << (p.B - 1), full = 1ll << p.B;
  const int lM = __ffsll((unsigned long long)p.M) - 1;   // M is a power of two
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, j = g & (p.M - 1);
    uint64_t* F = p.F + (row * p.nl) * p.M + j;
    const bool in = j < p.m;
    const int64_t e = row * p.m + j;
    row_sum_add(p.sums, p.M >= 32, row, 0, in ? p.a[e].w[0] : 0ull);
    row_sum_add(p.sums, p.M >= 32, row, 1, in ? p.x[e].w[0] : 0ull);
    if (!in) {
      for (int t = 0; t < p.nl; t++) F[(int64_t)t * p.M] = 0;
      continue;
    }
    for (int which = 0; which < 2; which++) {
      I256 v = which == 0 ? p.a[e] : p.x[e];
      const int L = which == 0 ? p.La : p.Lx;
      const int base = which == 0 ? 0 : p.La;
      for (int l = 0; l < L; l++) {
        int64_t dig = (int64_t)(v.w[0] & (uint64_t)(full - 1));
        if (dig >= half) dig -= full;
        v = i256_add(v, i256_from_i64(-dig));
        v = i256_sar(v, p.B);
        F[(int64_t)(base + l) * p.M] = dig >= 0 ? (uint64_t)dig : kGL - (uint64_t)(-dig);
      }
      if (v.w[0] | v.w[1] | v.w[2] | v.w[3]) record(p.status, SK_ERR_OVERFLOW);
    }
  }
}

__global__ void k_nproduct(NttArgs p) {
  const int64_t total = (int64_t)p.d * p.M;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int lM = __ffsll((unsigned long long)p.M) - 1;   // M is a power of two
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, k = g & (p.M - 1);
    const int64_t mk = (p.M - k) & (p.M - 1);
    const uint64_t* F = p.F + (row * p.nl) * p.M;
    uint64_t A[kMaxLimbs], X[kMaxLimbs];
    for (int l = 0; l < p.La; l++) A[l] = F[(int64_t)l * p.M + mk];
    for (int l = 0; l < p.Lx; l++) X[l] = F[(int64_t)(p.La + l) * p.M + k];
    uint64_t* G = p.G + (row * p.ns) * p.M + k;
    for (int s = 0; s < p.ns; s++) {
      const int l0 = max(0, s - (p.Lx - 1)), l1 = min(s, p.La - 1);
      uint64_t acc = 0;
      for (int l = l0; l <= l1; l++) acc = gl_add(acc, gl_mul(A[l], X[s - l]));
      G[(int64_t)s * p.M] = gl_mul(acc, p.minv);
    }
  }
}

__global__ void k_nrecombine(NttArgs p, const uint64_t* __restrict__ Y) {
  const int64_t total = (int64_t)p.d * p.m;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const bool warp_rows = (p.m & 31) == 0;
  const bool padded = p.M != p.m;
  int zb = 0;
  const bool mp2 = (p.m & (p.m - 1)) == 0;
  const int lm = __ffsll((unsigned long long)p.m) - 1;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = mp2 ? g >> lm : g / p.m, j = g - row * p.m;
    const uint64_t* y = Y + (row * p.ns) * p.M + j;
    I256 z{{0, 0, 0, 0}};
    for (int s = 0; s < p.ns; s++) {
      uint64_t r = y[(int64_t)s * p.M];
      if (padded && j > 0) r = gl_add(r, y[(int64_t)s * p.M + (p.M - p.m)]);
      const int64_t v = r > (kGL >> 1) ? -(int64_t)(kGL - r) : (int64_t)r;
      z = i256_add(z, i256_shl_i64(v, p.B * s));
    }
    p.z[g] = z;
    row_sum_add(p.sums, warp_rows, row, 2, z.w[0]);
    zb = max(zb, i256_bits(z));
  }
  block_max_bits(zb, p.zbits);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
int num_sms() {
  static const int sms = [] {   // thread-safe one-time initialisation
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, dev);
    return x > 0 ? x : 1;
  }();
  return sms;
}

int grid_for(int64_t n, int threads = 256) {
  const int sms = num_sms();
  int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

int ilog2(int64_t v) {
  int r = 0;
  while ((1ll << r) < v) r++;
  return r;
}

// ---------------------------------------------------------------------------
// A priori error bound of one FP64 correlation step, after Percival (Math. Comp. 72 (2003),
// Theorem 5.1): a cyclic convolution of length N = 2^n computed with radix-2 FFTs in floating
// point (unit roundoff eps), with precomputed roots of unity off by at most beta, errs in every
// output by at most |x|_2 |y|_2 ((1 + eps)^(3n) (1 + eps sqrt5)^(3n+1) (1 + beta)^(3n) - 1).
// The step here differs from that computation in ways that each add a bounded factor:
//   - every transform has S = n stages, plus one more above 2^12 (the four-step split multiplies
//     by the inter-pass twiddle from the same table): S replaces n;
//   - two real limb vectors share one complex forward transform; the separation after it (one
//     complex addition, an exact halving) maps the packed spectrum's error onto the two limbs'
//     spectra without growing its l2 norm, and the packed input has |w|_2^2 = |u|_2^2 + |v|_2^2;
//   - the npairs limb products of one limb sum are added (npairs - 1 additions) and two limb sums
//     share one inverse transform (one addition), whose output error is bounded by the packed
//     input's norm: at most twice a single sum's;
//   - for widths that are not powers of two the circular output adds two linear outputs.
// Every addition stage contributes a factor (1 + eps).  A limb vector has at most m non-zero
// signed B-bit digits, so a packed forward vector has |w|_2 <= sqrt(2 m) 2^(B-1), and
//   error <= fold * 2 * npairs * 2 m 2^(2B-2) * E,
//   E = (1 + eps)^(3S + 2 + npairs) (1 + eps sqrt5)^(3S + 1) (1 + beta)^(3S) - 1.
// The limb width is the largest B with that bound at most 1/4 (rounding to the nearest integer
// is then exact, with margin) and every output below 2^51 in magnitude.  beta is measured on
// the twiddle table itself (twiddle_error), so the bound holds for the roots actually used.
// ---------------------------------------------------------------------------
double fp64_step_bound(int64_t m, int64_t M, int npairs, int B, double beta) {
  int n = 0;
  while (((int64_t)1 << n) < M) n++;
  const int S = n + (M > 4096 ? 1 : 0);
  const double eps = std::ldexp(1.0, -53);
  const double lg = (3.0 * S + 2 + npairs) * std::log1p(eps) + (3.0 * S + 1) * std::log1p(std::sqrt(5.0) * eps) +
                    3.0 * S * std::log1p(beta);
  const double E = std::expm1(lg) * (1.0 + 1e-9);   // margin for the rounding of this evaluation
  const double fold = M != m ? 2.0 : 1.0;
  return fold * 2.0 * npairs * 2.0 * (double)m * std::ldexp(1.0, 2 * B - 2) * E;
}

int limb_bits_for(int64_t m, int64_t M, int npairs, double beta) {
  const double fold = M != m ? 2.0 : 1.0;
  for (int B = 24; B >= 2; B--) {
    const double mag = fold * (double)npairs * (double)m * std::ldexp(1.0, 2 * B - 2);
    if (fp64_step_bound(m, M, npairs, B, beta) <= 0.25 && mag < std::ldexp(1.0, 51)) return B;
  }
  return 2;
}

// Largest deviation |w' - w| of the length-M twiddle table (M / 2 entries W_M^t =
// exp(-2 pi i t / M) in device memory) from the exact roots, computed on the host in long
// double (the reference's own error, far below 1e-17, is covered by the added 1e-17).  The
// table for a length comes from one deterministic kernel, so the value is cached per length.
double twiddle_error(int64_t M, const double2* d_tw, cudaStream_t st) {
  static std::mutex mu;
  static std::map<int64_t, double> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(M);
    if (it != cache.end()) return it->second;
  }
  std::vector<double2> h((size_t)(M / 2));
  if (M >= 2) {
    if (cudaMemcpyAsync(h.data(), d_tw, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return 1.0;   // unknown: a bound that admits no limb width, so the step reports inexact
  }
  const long double pi = acosl(-1.0L);
  double worst = 0.0;
  for (int64_t t = 0; t < M / 2; t++) {
    const long double a = 2.0L * pi * (long double)t / (long double)M;
    const long double dc = (long double)h[(size_t)t].x - cosl(a), ds = (long double)h[(size_t)t].y + sinl(a);
    worst = std::max(worst, (double)sqrtl(dc * dc + ds * ds));
  }
  const double beta = worst + 1e-17;
  std::lock_guard<std::mutex> lk(mu);
  cache[M] = beta;
  return beta;
}

// Grows a scratch buffer with the stream-ordered allocator: the old buffer is only
// ever used by earlier work of this estimate on the same stream (sk_estimate_join
// synchronises its stream before returning), so freeing and reallocating in stream
// order needs no device-wide synchronisation.
// (Re)allocates a per-set table on the stream (stream-ordered: no device-wide
// synchronisation, which cudaFree would impose on every other stream, e.g. a server's update
// streams, the first time a set is estimated at a width).
cudaError_t table_alloc(void** p, size_t bytes, cudaStream_t st) {
  if (*p) {
    cudaError_t e = cudaFreeAsync(*p, st);
    if (e != cudaSuccess) return e;
    *p = nullptr;
  }
  return cudaMallocAsync(p, bytes, st);
}

// The device copy of the set's relation counter pointers (stream-ordered, once per set).
cudaError_t fu_rel_table(sk_set* s, cudaStream_t st) {
  if (s->d_fu_rel) return cudaSuccess;
  cudaError_t e = cudaMallocAsync((void**)&s->d_fu_rel, sizeof(int64_t*) * s->r, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_fu_rel, s->rel_ctr.data(), sizeof(int64_t*) * s->r, cudaMemcpyHostToDevice, st);
  return e;
}

cudaError_t ensure(Scratch& s, size_t bytes, cudaStream_t st) {
  if (s.bytes >= bytes) return cudaSuccess;
  if (s.ptr) {
    cudaError_t e = cudaFreeAsync(s.ptr, st);
    if (e != cudaSuccess) return e;
    s.ptr = nullptr;
    s.bytes = 0;
  }
  cudaError_t e = cudaMallocAsync(&s.ptr, bytes, st);
  if (e == cudaSuccess) s.bytes = bytes;
  return e;
}

#define SK_CK(x)                                        \
  do {                                                  \
    cudaError_t _e = (x);                               \
    if (_e != cudaSuccess) return set_status_from_cuda(_e); \
  } while (0)

#define SK_CK_ST(x)                \
  do {                             \
    const sk_status _s = (x);      \
    if (_s != SK_OK) return _s;    \
  } while (0)

// Forward (inv = false) or inverse (unnormalised) transform of `batch` vectors of
// length m held in src; the result is written to dst, src is clobbered.  Complex FP64
// with the W table (conjugated for the inverse), or GF(q) with the w^t / w^-t table.
template <class Ops>
sk_status xform(typename Ops::T* src, typename Ops::T* dst, int64_t batch, int64_t m, const typename Ops::T* tw,
                bool inv, typename Ops::T r4, cudaStream_t st) {
  using T = typename Ops::T;
  const int logm = ilog2(m);
  const int esz = (int)sizeof(T);
  if (logm <= 12) {
    const int L = (int)m;
    const int vpc = (int)std::max<int64_t>(1, std::min<int64_t>(4096 / L, batch));
    const int64_t grid = (batch + vpc - 1) / vpc;
    const size_t smem = (size_t)vpc * L * esz;
    SK_CK(allow_dynamic_smem((const void*)k_xf_small<Ops>));
    k_xf_small<Ops><<<(unsigned)grid, 256, smem, st>>>(src, dst, batch, logm, vpc, tw, 1, inv, r4);
    count_launch();
    return set_status_from_cuda(cudaGetLastError());
  }
  const int logR = logm / 2, logC = logm - logR;
  const int R = 1 << logR, C = 1 << logC;
  // 64 KB tiles: two or three CTAs per SM (measured against 128 KB at m = 2^20, one CTA per SM:
  // chain8 estimate 36 -> 24 ms fused, 57 -> 45 ms GF(q), 214 -> 196 ms FP64; 32 KB: no gain)
  const int budget = 64 << 10;
  int cb = std::max(1, std::min(C, budget / (R * esz)));
  int rb = std::max(1, std::min(R, budget / (C * esz)));
  // narrower tiles until the grid gives every SM two CTAs (a small batch of vectors would
  // otherwise leave SMs idle); at least 4 columns per tile keep the column loads sector-wide
  const int64_t want = 2 * (int64_t)num_sms();
  while (cb > 4 && batch * (C / cb) < want) cb >>= 1;
  while (rb > 1 && batch * (R / rb) < want) rb >>= 1;
  if ((cb & (cb - 1)) || (rb & (rb - 1))) return SK_ERR_INVALID_ARG;   // the kernels index by shifts
  // the register transform (exact arithmetics, lengths 2^6..2^10) takes one A- or B-point DFT
  // per thread: at most 512 >> max(log A, log B) vectors per tile; plus its twiddle table
  size_t smc_tw = 0, smr_tw = 0;
  if (Ops::kReg) {
    if (logR >= 6 && logR <= 10) {
      cb = std::min(cb, 512 >> (logR - logR / 2));
      smc_tw = (size_t)R * esz;
    }
    if (logC >= 6 && logC <= 10) {
      rb = std::min(rb, 512 >> (logC - logC / 2));
      smr_tw = (size_t)C * esz;
    }
  }
  const size_t smc = (size_t)(cb + 1) * R * esz + smc_tw, smr = (size_t)(rb + 1) * C * esz + smr_tw;   // padded tiles
  SK_CK(allow_dynamic_smem((const void*)k_xf_cols<Ops>));
  SK_CK(allow_dynamic_smem((const void*)k_xf_rows<Ops>));
  k_xf_cols<Ops><<<(unsigned)(batch * (C / cb)), 512, smc, st>>>(src, logR, logC, cb, tw, inv, r4);
  count_launch();
  SK_CK(cudaGetLastError());
  k_xf_rows<Ops><<<(unsigned)(batch * (R / rb)), 512, smr, st>>>(src, dst, logR, logC, rb, tw, inv, r4);
  count_launch();
  return set_status_from_cuda(cudaGetLastError());
}

sk_status fft(double2* src, double2* dst, int64_t batch, int64_t m, const double2* tw, bool inv, cudaStream_t st) {
  return xform<CplxOps>(src, dst, batch, m, tw, inv, make_double2(0.0, 0.0), st);
}

struct HostI256 {
  static I256 mul(const I256& a, const I256& b) { return i256_mul(a, b); }
};

}  // namespace

void free_estimator(sk_set* s) {
  if (s->d_fu_tw) cudaFree(s->d_fu_tw);
  if (s->d_fu_rel) cudaFree(s->d_fu_rel);
  s->d_fu_tw = nullptr;
  s->d_fu_rel = nullptr;
  s->fu_m = 0;
  s->fu_np = 0;
  if (s->scratch.ptr) cudaFree(s->scratch.ptr);
  if (s->fft_scratch.ptr) cudaFree(s->fft_scratch.ptr);
  if (s->d_twiddle) cudaFree(s->d_twiddle);
  if (s->d_gl_tw) cudaFree(s->d_gl_tw);
  s->d_gl_tw = nullptr;
  s->gl_m = 0;
  s->scratch = Scratch();
  s->fft_scratch = Scratch();
  s->d_twiddle = nullptr;
  s->twiddle_m = 0;
}

// One exact correlation step z = a (star) x through the GF(q) transform.
sk_status corr_ntt(sk_set* s, const I256* a, const I256* x, I256* z, int* zbits, unsigned long long* cert, int bits_a,
                   int bits_x, int64_t m, int64_t M, cudaStream_t st, int* max_limbs, int* last_B) {
  const int d = s->d;
  const int logM = ilog2(M);
  if (s->gl_m != M) {
    SK_CK(table_alloc((void**)&s->d_gl_tw, (size_t)M * sizeof(uint64_t), st));   // [w^t | w^-t], t < M/2
    const uint64_t w = gl_pow(7, (kGL - 1) / (uint64_t)M);          // 7 generates GF(q)*
    if (M >= 2 && gl_pow(w, (uint64_t)M / 2) != kGL - 1) return SK_ERR_INEXACT;   // not a primitive root
    const uint64_t winv = gl_pow(w, kGL - 2);
    s->gl_r4 = M >= 4 ? gl_pow(w, (uint64_t)M / 4) : 1;
    s->gl_r4inv = M >= 4 ? gl_pow(winv, (uint64_t)M / 4) : 1;
    s->gl_minv = gl_pow((uint64_t)M, kGL - 2);
    k_gl_twiddle<<<grid_for(M / 2), 256, 0, st>>>(s->d_gl_tw, s->d_gl_tw + M / 2, M, w, winv);
    count_launch();
    SK_CK(cudaGetLastError());
    s->gl_m = M;
  }
  // widest limbs with every output below 2^62: pairs * m * 2^(2B-2) < 2^62
  int B = 30, La = 0, Lx = 0;
  for (; B >= 2; B--) {
    La = (bits_a + 2 + B - 1) / B;
    Lx = (bits_x + 2 + B - 1) / B;
    const int pairs = std::min(La, Lx);
    if (ilog2(pairs) + ilog2(m) + 2 * B - 2 <= 61) break;
  }
  if (La > kMaxLimbs || Lx > kMaxLimbs || B < 2) return SK_ERR_INEXACT;
  NttArgs p;
  p.a = a;
  p.x = x;
  p.z = z;
  p.m = m;
  p.M = M;
  p.d = d;
  p.B = B;
  p.La = La;
  p.Lx = Lx;
  p.nl = La + Lx;
  p.ns = La + Lx - 1;
  p.status = s->d_status;
  p.sums = cert + 1;
  p.zbits = zbits;
  p.minv = s->gl_minv;
  const size_t words = (size_t)d * p.nl * M;
  SK_CK(ensure(s->fft_scratch, 2 * words * sizeof(uint64_t), st));
  uint64_t* bufA = (uint64_t*)s->fft_scratch.ptr;
  uint64_t* bufB = bufA + words;
  const int egM = grid_for((int64_t)d * M);
  p.F = bufA;
  SK_CK(cudaMemsetAsync(zbits, 0, sizeof(int), st));
  k_nsplit<<<egM, 256, 0, st>>>(p);
  count_launch();
  SK_CK(cudaGetLastError());
  sk_status fs = xform<GlOps>(bufA, bufB, (int64_t)d * p.nl, M, s->d_gl_tw, false, s->gl_r4, st);
  if (fs != SK_OK) return fs;
  p.F = bufB;
  p.G = bufA;
  k_nproduct<<<egM, 128, 0, st>>>(p);
  count_launch();
  SK_CK(cudaGetLastError());
  fs = xform<GlOps>(bufA, bufB, (int64_t)d * p.ns, M, s->d_gl_tw + M / 2, true, s->gl_r4inv, st);
  if (fs != SK_OK) return fs;
  k_nrecombine<<<grid_for((int64_t)d * m), 256, 0, st>>>(p, bufB);
  count_launch();
  SK_CK(cudaGetLastError());
  *max_limbs = std::max(*max_limbs, std::max(La, Lx));
  *last_B = B;
  (void)logM;
  return SK_OK;
}

// Fills *out from the d row values and their sorted copy.
void fill_estimate(sk_estimate* out, const I256* rows, const I256* sorted, int d) {
  auto to_double = [](const I256& v) {
    const bool neg = i256_neg_p(v);
    const I256 a = neg ? i256_neg(v) : v;
    double r = 0.0;
    for (int k = 3; k >= 0; k--) r = r * 18446744073709551616.0 + (double)a.w[k];
    return neg ? -r : r;
  };
  out->d = d;
  for (int r = 0; r < d; r++) std::memcpy(&out->row[r], &rows[r], sizeof(sk_i256));
  const I256 med = sorted[(d - 1) / 2];
  std::memcpy(&out->median, &med, sizeof(sk_i256));
  const bool fits = (med.w[1] == med.w[2] && med.w[2] == med.w[3] &&
                     (med.w[3] == 0 ? (int64_t)med.w[0] >= 0 : (med.w[3] == ~0ull && (int64_t)med.w[0] < 0)));
  out->fits_i64 = fits ? 1 : 0;
  out->median_i64 = fits ? (int64_t)med.w[0] : 0;
  out->median_f64 = to_double(med);
  out->mid_mean_f64 = (d & 1) ? to_double(sorted[d / 2])
                              : 0.5 * (to_double(sorted[d / 2 - 1]) + to_double(sorted[d / 2]));
}

// ===========================================================================
// Fused estimator for queries whose components all have exactly two attributes
// (chains, stars).  Writing each sketch through its DFT over an m-th root of unity w,
// the sum over all components' bins in Eq. 5 leaves one free frequency: with the
// relations two-coloured along the tree of components (s_k = +1 / -1),
//     X = (1/m) sum_nu prod_k C_k(s_k nu),     C_k(nu) = sum_t c_k[t] w^(nu t).
// That identity is evaluated exactly modulo several primes p = c 2^22 + 1 in
// (2^30, 2^31) and the row values are recombined by the Chinese remainder theorem.
// |X| <= prod_k ||c_k||_1 (each choice of one counter per relation meets at most one
// bin assignment, by peeling leaf relations), so primes whose product exceeds eight
// times that bound give X exactly.  Arithmetic mod p is Montgomery with R = 2^32.
// ===========================================================================
constexpr int kFuMaxPrimes = 9;            // 9 x 30+ bits covers any signed 256-bit result
__constant__ uint32_t c_fu_p[kFuMaxPrimes];
__constant__ uint32_t c_fu_pinv[kFuMaxPrimes];   // -p^-1 mod 2^32

struct FuPrime {
  uint32_t p, pinv, r2, r3;   // r2 = 2^64 mod p, r3 = 2^96 mod p
  uint64_t g;                 // a quadratic non-residue mod p
  double log2p;
};

uint64_t fu_powmod(uint64_t b, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  b %= p;
  for (; e; e >>= 1) {
    if (e & 1) r = (uint64_t)((unsigned __int128)r * b % p);
    b = (uint64_t)((unsigned __int128)b * b % p);
  }
  return r;
}

// the primes c 2^22 + 1 in (2^30, 2^31), largest first (trial division suffices below 2^31)
const std::vector<FuPrime>& fu_primes() {
  static const std::vector<FuPrime> v = [] {
    std::vector<FuPrime> out;
    for (uint64_t c = ((1ull << 31) - 1) >> 22; c >= (1ull << 8) && (int)out.size() < kFuMaxPrimes; c--) {
      const uint64_t p = (c << 22) + 1;
      if (p >= (1ull << 31) || p <= (1ull << 30)) continue;
      bool prime = true;
      for (uint64_t f = 3; f * f <= p; f += 2)
        if (p % f == 0) {
          prime = false;
          break;
        }
      if (!prime) continue;
      FuPrime fp;
      fp.p = (uint32_t)p;
      uint32_t inv = 1;   // p^-1 mod 2^32 by Newton's iteration (correct bits double each step)
      for (int k = 0; k < 5; k++) inv *= 2u - (uint32_t)p * inv;
      fp.pinv = 0u - inv;
      const uint64_t R = (1ull << 32) % p;
      fp.r2 = (uint32_t)((unsigned __int128)R * R % p);
      fp.r3 = (uint32_t)((unsigned __int128)fp.r2 * R % p);
      fp.g = 0;
      for (uint64_t g = 3; g < p; g++)
        if (fu_powmod(g, (p - 1) / 2, p) == p - 1) {
          fp.g = g;
          break;
        }
      fp.log2p = std::log2((double)p);
      out.push_back(fp);
    }
    return out;
  }();
  return v;
}

// a * b / 2^32 mod p for a, b < p < 2^31 (Montgomery reduction; the sum below stays < 2^64)
__device__ __forceinline__ uint32_t mont32(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t q = (uint32_t)t * pinv;
  const uint64_t u = (t + (uint64_t)q * p) >> 32;
  return (uint32_t)(u >= p ? u - p : u);
}

template <int PI>
struct MontOps {
  using T = uint32_t;
  static constexpr bool kExact = true;
  static constexpr bool kReg = true;    // lengths 2^6..2^10 through smem_ntt_2lvl
  static __device__ __forceinline__ T mul(T a, T b) { return mont32(a, b, c_fu_p[PI], c_fu_pinv[PI]); }
  static __device__ __forceinline__ T add(T a, T b) {
    const uint32_t p = c_fu_p[PI], s = a + b;
    return s >= p ? s - p : s;
  }
  static __device__ __forceinline__ T sub(T a, T b) { return a >= b ? a - b : a + c_fu_p[PI] - b; }
  static __device__ __forceinline__ T neg(T a) { return a ? c_fu_p[PI] - a : 0; }
  static __device__ __forceinline__ T tw(const T* tab, int64_t i, bool) { return tab[i]; }
  static __device__ __forceinline__ T rot4(T w, bool, T r4) { return mul(w, r4); }
};

// tw[t] = w^t, itw[t] = w^-t for t < n/2 (Montgomery form; one is R mod p)
template <int PI>
__global__ void k_fu_twiddle(uint32_t* tw, uint32_t* itw, int64_t n, uint32_t w, uint32_t winv, uint32_t one) {
  const int64_t half = n >> 1;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += step) {
    uint32_t r = one, ri = one, b = w, bi = winv;
    for (int64_t e = t; e; e >>= 1) {
      if (e & 1) {
        r = MontOps<PI>::mul(r, b);
        ri = MontOps<PI>::mul(ri, bi);
      }
      b = MontOps<PI>::mul(b, b);
      bi = MontOps<PI>::mul(bi, bi);
    }
    tw[t] = r;
    itw[t] = ri;
  }
}

// Partial norms: vector v (= blockIdx.x / nch) is base[v / per] + (v % per) m; block
// (v, ch) writes part[2 (v nch + ch)] = sum |c[j]| and part[2 (v nch + ch) + 1] = sum c[j]^2
// over the ch-th of nch chunks of ceil(m / nch) elements (the last one shorter).  The
// host adds a vector's partials in order (double; the bounds carry a safety margin).
__global__ void __launch_bounds__(256) k_fu_norms(const int64_t* const* base, int per, int64_t m, int nch,
                                                  double* part) {
  // Each thread sums 8 loaded values at a time in FP32, as |c| 2^-32 and (|c| 2^-32)^2 (the
  // scaling keeps the square of 2^63 inside the float range), and adds each 8-term sum into
  // double accumulators: GB300's FP64 rate would bound a loop of double operations per
  // element.  A term is within 2^-22 of its value and an 8-term float sum within 7 2^-24
  // more, so the partials are within a relative 2^-19 of the exact sums (the double
  // additions add nothing comparable), inside the 2^-10 margin fu_row_bits applies.
  __shared__ double red1[256], red2[256];
  const int64_t v = blockIdx.x / nch, ch = blockIdx.x % nch, len = (m + nch - 1) / nch;
  const int64_t j0 = ch * len, j1 = j0 + len < m ? j0 + len : m;
  const int64_t* c = base[v / per] + (v % per) * m;
  double s1 = 0.0, s2 = 0.0;
  constexpr int U = 8;   // loads in flight per thread
  for (int64_t j = j0 + threadIdx.x; j < j1; j += U * (int64_t)blockDim.x) {
    int64_t x[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t jj = j + u * (int64_t)blockDim.x;
      x[u] = jj < j1 ? __ldg(c + jj) : 0;
    }
    float f1 = 0.0f, f2 = 0.0f;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint64_t mag = x[u] < 0 ? 0ull - (uint64_t)x[u] : (uint64_t)x[u];
      // |c| 2^-32 = hi + lo 2^-32
      const float a = fmaf((float)(uint32_t)mag, 2.3283064365386963e-10f, (float)(uint32_t)(mag >> 32));
      f1 += a;
      f2 = fmaf(a, a, f2);
    }
    s1 += (double)f1;
    s2 += (double)f2;
  }
  red1[threadIdx.x] = s1;
  red2[threadIdx.x] = s2;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      red1[threadIdx.x] += red1[threadIdx.x + h];
      red2[threadIdx.x] += red2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * (int64_t)blockIdx.x] = red1[0] * 4294967296.0;                 // sum |c|
    part[2 * (int64_t)blockIdx.x + 1] = red2[0] * 18446744073709551616.0;   // sum c^2
  }
}

// chunks per vector for k_fu_norms: at least 2048 elements each, about four waves of blocks
int fu_l1_chunks(int64_t nvec, int64_t m) {
  int nch = 1;
  while (m / (nch * 2) >= 2048 && nvec * nch < 4 * (int64_t)num_sms()) nch *= 2;
  return nch;
}

// Launches k_fu_norms and reads the nvec l1 and l2 norms back (synchronises st).  d_part
// holds 2 nvec nch doubles.
sk_status fu_norms(const int64_t* const* base, int per, int64_t nvec, int64_t m, double* d_part, int nch,
                   std::vector<double>& l1, std::vector<double>& l2, cudaStream_t st) {
  k_fu_norms<<<(unsigned)(nvec * nch), 256, 0, st>>>(base, per, m, nch, d_part);
  count_launch();
  SK_CK(cudaGetLastError());
  std::vector<double> part((size_t)2 * nvec * nch);
  SK_CK(cudaMemcpyAsync(part.data(), d_part, part.size() * 8, cudaMemcpyDeviceToHost, st));
  SK_CK(cudaStreamSynchronize(st));
  l1.assign((size_t)nvec, 0.0);
  l2.assign((size_t)nvec, 0.0);
  for (int64_t v = 0; v < nvec; v++) {
    double sq = 0.0;
    for (int c = 0; c < nch; c++) {
      l1[v] += part[2 * ((size_t)v * nch + c)];
      sq += part[2 * ((size_t)v * nch + c) + 1];
    }
    l2[v] = std::sqrt(sq);
  }
  return SK_OK;
}

// log2 of an upper bound on |X_row| from the norms of the row's r relation vectors
// (l1[k * stride], l2[k * stride]); -1 when one of them is zero (then X_row = 0).  Any
// schedule: prod_k ||c_k||_1 (correlation, Hadamard product and sum are submultiplicative
// in the l1 norm).  Pairwise product of spectra, X = (1/m) sum_nu prod_k C_k(+-nu): with
// |C_k| <= ||c_k||_1 for all but two relations a, b, Cauchy-Schwarz and Parseval
// (sum_nu |C|^2 = m ||c||_2^2) give ||c_a||_2 ||c_b||_2 prod_{k != a, b} ||c_k||_1; a and b
// are the two relations with the largest l1 / l2 ratio.  Each factor carries a relative
// margin of 1e-9 for the rounding of the double sums.
double fu_row_bits(const double* l1, const double* l2, int r, int64_t stride, bool pairwise) {
  double b = 0.0, best1 = 0.0, best2 = 0.0;
  // the norms come from k_fu_norms's FP32 partial sums: within a relative 2^-19 of the exact
  // ones, so scaling l1 up by 2^-10 keeps b an upper bound; l2 scaled up only lowers the savings
  constexpr double kUp = 1.0 + 1.0 / 1024.0;
  for (int k = 0; k < r; k++) {
    const double v1 = l1[k * stride], v2 = l2[k * stride];
    if (v1 <= 0.0) return -1.0;
    b += std::log2(v1 * kUp);
    const double save = std::log2(v1) - std::log2(v2 * kUp);
    if (save > best1) {
      best2 = best1;
      best1 = save;
    } else if (save > best2) {
      best2 = save;
    }
  }
  return pairwise && r >= 2 ? b - best1 - best2 : b;
}

// out[(k d + row) m + j] = c_k[row][j] mod p, Montgomery form (|c| = h 2^32 + l)
template <int PI>
__global__ void k_fu_load(const int64_t* const* rel, int r, int d, int64_t m, uint32_t r2, uint32_t r3, uint32_t* out) {
  using O = MontOps<PI>;
  const int64_t dm = (int64_t)d * m;
  const uint32_t p = c_fu_p[PI];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int k = blockIdx.y;            // relation: its d x m counters are contiguous
  const int64_t* src = rel[k];
  out += (int64_t)k * dm;
  constexpr int U = 4;   // loads in flight per thread
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g0 < dm; g0 += U * step) {
    int64_t cv[U];
#pragma unroll
    for (int u = 0; u < U; u++) cv[u] = g0 + u * step < dm ? src[g0 + u * step] : 0;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t g = g0 + u * step;
      if (g >= dm) break;
      const int64_t c = cv[u];
      const uint64_t mag = c < 0 ? 0ull - (uint64_t)c : (uint64_t)c;
      uint32_t h = (uint32_t)(mag >> 32);
      if (h >= p) h -= p;
      const uint32_t v = O::add(O::mul(h, r3), O::mul((uint32_t)mag, r2));
      out[g] = c < 0 ? O::neg(v) : v;
    }
  }
}

// part[row * nchunk + chunk] = sum over the chunk's nu of prod_k C_k(s_k nu)
template <int PI>
__global__ void __launch_bounds__(256) k_fu_reduce(const uint32_t* W, int r, int d, int64_t M, unsigned long long negmask,
                                                   int nchunk, uint32_t* part) {
  using O = MontOps<PI>;
  __shared__ uint32_t red[256];
  const int row = blockIdx.x / nchunk, c = blockIdx.x % nchunk;
  const int64_t clen = M / nchunk;
  uint32_t s = 0;
  constexpr int KR = 8;   // factors loaded before their products
  for (int64_t nu = (int64_t)c * clen + threadIdx.x; nu < (int64_t)(c + 1) * clen; nu += blockDim.x) {
    const int64_t neg_nu = (M - nu) & (M - 1);
    uint32_t f[KR];
#pragma unroll
    for (int k = 0; k < KR; k++)
      if (k < r) f[k] = W[((int64_t)k * d + row) * M + (((negmask >> k) & 1ull) ? neg_nu : nu)];
    uint32_t prod = f[0];
#pragma unroll
    for (int k = 1; k < KR; k++)
      if (k < r) prod = O::mul(prod, f[k]);
    for (int k = KR; k < r; k++)
      prod = O::mul(prod, W[((int64_t)k * d + row) * M + (((negmask >> k) & 1ull) ? neg_nu : nu)]);
    s = O::add(s, prod);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = O::add(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// res[row * np + PI] = (sum of the row's chunks) / m, back from Montgomery form
template <int PI>
__global__ void k_fu_final(const uint32_t* part, int d, int nchunk, uint32_t minv_mont, uint32_t* res, int np) {
  using O = MontOps<PI>;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d) return;
  uint32_t s = 0;
  for (int c = 0; c < nchunk; c++) s = O::add(s, part[row * nchunk + c]);
  res[row * np + PI] = O::mul(O::mul(s, minv_mont), 1u);
}

// host: Montgomery form of v (< p)
uint32_t fu_to_mont(uint64_t v, uint32_t p) { return (uint32_t)(((unsigned __int128)v << 32) % p); }

// Per-width constants of prime i, computed once per width M (modular exponentiations are
// host work that every estimate would otherwise repeat): w, a root of unity of order exactly
// M, its inverse, and in Montgomery form w, w^-1, w^(M/4), w^(-M/4), M^-1 and 1.
struct FuWidth {
  uint64_t w = 1, winv = 1;
  uint32_t w_m = 0, winv_m = 0, r4 = 0, r4i = 0, minv = 0, one = 0;
};

const FuWidth& fu_width(int i, int64_t M) {
  static std::mutex mu;
  static std::map<int64_t, std::vector<FuWidth>> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(M);
  if (it == cache.end()) {
    const std::vector<FuPrime>& pr = fu_primes();
    std::vector<FuWidth> v(kFuMaxPrimes);
    for (int k = 0; k < kFuMaxPrimes && k < (int)pr.size(); k++) {
      const uint64_t p = pr[k].p;
      FuWidth& f = v[k];
      f.w = fu_powmod(pr[k].g, (p - 1) / (uint64_t)M, p);
      f.winv = fu_powmod(f.w, p - 2, p);
      f.one = fu_to_mont(1, pr[k].p);
      f.w_m = fu_to_mont(f.w, pr[k].p);
      f.winv_m = fu_to_mont(f.winv, pr[k].p);
      f.r4 = M >= 4 ? fu_to_mont(fu_powmod(f.w, (uint64_t)M / 4, p), pr[k].p) : f.one;
      f.r4i = M >= 4 ? fu_to_mont(fu_powmod(f.winv, (uint64_t)M / 4, p), pr[k].p) : f.one;
      f.minv = fu_to_mont(fu_powmod((uint64_t)M % p, p - 2, p), pr[k].p);
    }
    it = cache.emplace(M, std::move(v)).first;
  }
  return it->second[i];
}

// One prime's pass (twiddles already in place): load, forward transform, product-sum.
template <int PI>
sk_status fu_prime_pass(sk_set* s, const FuPrime& fp, int64_t M, uint32_t* V, uint32_t* W, uint32_t* part,
                        int nchunk, uint32_t* res, int np, unsigned long long negmask, cudaStream_t st) {
  const int r = s->r, d = s->d;
  uint32_t* tw = s->d_fu_tw + (size_t)PI * M;
  const FuWidth& fw = fu_width(PI, M);
  const uint32_t r4 = fw.r4;
  k_fu_load<PI><<<dim3((unsigned)std::max(1, grid_for((int64_t)r * d * M) / r), (unsigned)r), 256, 0, st>>>(
      s->d_fu_rel, r, d, M, fp.r2, fp.r3, V);
  count_launch();
  SK_CK(cudaGetLastError());
  sk_status fs = xform<MontOps<PI>>(V, W, (int64_t)r * d, M, tw, false, r4, st);
  if (fs != SK_OK) return fs;
  k_fu_reduce<PI><<<d * nchunk, 256, 0, st>>>(W, r, d, M, negmask, nchunk, part);
  k_fu_final<PI><<<(d + 63) / 64, 64, 0, st>>>(part, d, nchunk, fw.minv, res, np);
  count_launch(2);
  return set_status_from_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Small widths (m <= 4096, every relation's row in one CTA's shared memory): the whole
// pairwise fused estimate in one launch and one host synchronisation.  CTA (row, prime)
// first bounds its row as fu_row_bits does (l1 and l2 norms of the row's r counter vectors,
// |X_row| <= prod_k ||c_k||_1 with the two largest l1/l2 savings of the pairwise form) and
// takes the row's own number of primes, the fewest whose product exceeds 8 times the bound
// (one for a row with an all-zero vector, whose estimate is 0; none when nine do not
// reach it); a CTA whose prime is beyond that count returns.  The others reduce the
// vectors mod the prime, transform them in shared memory, form sum_nu prod_k C_k(s_k nu)
// and write the row's residue.  Every CTA of a row computes the same count (same data,
// same reduction order).
// ---------------------------------------------------------------------------
struct FuSmallArgs {
  const int64_t* const* rel;     // r relation counter blocks [d][m]
  const uint32_t* tw;            // twiddle tables [prime][m] (w^t | w^-t, Montgomery form)
  uint32_t r2[kFuMaxPrimes], r3[kFuMaxPrimes], r4[kFuMaxPrimes], minv[kFuMaxPrimes];
  double log2p[kFuMaxPrimes];
  int r, d, logm;
  unsigned long long negmask;
  uint32_t* res;                 // [d][kFuMaxPrimes] residues, then [d] prime counts (int)
};

// The number of primes row `row` needs (all threads of the CTA get it; 256 threads).
__device__ int fu_small_row_primes(const FuSmallArgs& a, int row, double (*wsum)[8], int* s_np) {
  const int m = 1 << a.logm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double b = 0.0, best1 = 0.0, best2 = 0.0;   // thread 0's running bound (fu_row_bits)
  bool zero = false;
  for (int k = 0; k < a.r; k++) {
    const int64_t* src = a.rel[k] + (int64_t)row * m;
    double s1 = 0.0, s2 = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const int64_t c = src[j];
      const double x = (double)(c < 0 ? 0ull - (uint64_t)c : (uint64_t)c);
      s1 += x;
      s2 += x * x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      wsum[0][warp] = s1;
      wsum[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v1 = 0.0, sq = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        v1 += wsum[0][w];
        sq += wsum[1][w];
      }
      if (v1 <= 0.0) {
        zero = true;
      } else if (!zero) {
        const double v2 = sqrt(sq);
        b += log2(v1 * (1.0 + 1e-9));
        const double save = log2(v1 * (1.0 + 1e-9)) - log2(v2 * (1.0 + 1e-9));
        if (save > best1) {
          best2 = best1;
          best1 = save;
        } else if (save > best2) {
          best2 = save;
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int np = 1;
    if (!zero) {
      const double bits = a.r >= 2 ? b - best1 - best2 : b;
      double cover = 0.0;
      np = 0;
      while (np < kFuMaxPrimes && cover < bits + 3.0) cover += a.log2p[np++];
      if (cover < bits + 3.0) np = 0;
    }
    *s_np = np;
  }
  __syncthreads();
  return *s_np;
}

template <int PI>
__device__ __forceinline__ void fu_small_body(const FuSmallArgs& a, int row, uint32_t* V, uint32_t* red) {
  using O = MontOps<PI>;
  const int m = 1 << a.logm;
  const uint32_t p = c_fu_p[PI];
  for (int idx = threadIdx.x; idx < a.r * m; idx += blockDim.x) {
    const int k = idx >> a.logm, j = idx & (m - 1);
    const int64_t c = a.rel[k][(int64_t)row * m + j];
    const uint64_t mag = c < 0 ? 0ull - (uint64_t)c : (uint64_t)c;
    uint32_t h = (uint32_t)(mag >> 32);
    if (h >= p) h -= p;
    const uint32_t v = O::add(O::mul(h, a.r3[PI]), O::mul((uint32_t)mag, a.r2[PI]));
    V[k * m + bitrev(j, a.logm)] = c < 0 ? O::neg(v) : v;
  }
  __syncthreads();
  smem_xform<O>(V, a.r, a.logm, a.tw + (int64_t)PI * m, 1, false, a.r4[PI]);
  uint32_t sum = 0;
  for (int nu = threadIdx.x; nu < m; nu += blockDim.x) {
    const int neg_nu = (m - nu) & (m - 1);
    uint32_t prod = V[(a.negmask & 1ull) ? neg_nu : nu];
    for (int k = 1; k < a.r; k++) prod = O::mul(prod, V[k * m + (((a.negmask >> k) & 1ull) ? neg_nu : nu)]);
    sum = O::add(sum, prod);
  }
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = O::add(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) a.res[row * kFuMaxPrimes + PI] = O::mul(O::mul(red[0], a.minv[PI]), 1u);
}

// grid (d, kFuMaxPrimes), 256 threads, r m 4 bytes of dynamic shared memory
__global__ void __launch_bounds__(256) k_fu_small(FuSmallArgs a) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  __shared__ uint32_t red[256];
  __shared__ double wsum[2][8];
  __shared__ int s_np;
  const int row = blockIdx.x, pi = blockIdx.y;
  const int np = fu_small_row_primes(a, row, wsum, &s_np);
  if (pi == 0 && threadIdx.x == 0) ((int*)(a.res + (int64_t)a.d * kFuMaxPrimes))[row] = np;
  if (pi >= np) return;   // uniform across the CTA
  uint32_t* V = (uint32_t*)fs_smem;
  switch (pi) {
    case 0: fu_small_body<0>(a, row, V, red); break;
    case 1: fu_small_body<1>(a, row, V, red); break;
    case 2: fu_small_body<2>(a, row, V, red); break;
    case 3: fu_small_body<3>(a, row, V, red); break;
    case 4: fu_small_body<4>(a, row, V, red); break;
    case 5: fu_small_body<5>(a, row, V, red); break;
    case 6: fu_small_body<6>(a, row, V, red); break;
    case 7: fu_small_body<7>(a, row, V, red); break;
    default: fu_small_body<8>(a, row, V, red); break;
  }
}

// Garner's mixed-radix reconstruction of the integer with the given residues, taken in
// [-P/2, P/2) with P the product of the primes; false when it needs more than 255 bits.
// Garner's coefficients: c_i = (p_0 p_1 ... p_{i-1})^-1 mod p_i, computed once.
const std::vector<uint64_t>& fu_garner() {
  static const std::vector<uint64_t> c = [] {
    const std::vector<FuPrime>& pr = fu_primes();
    std::vector<uint64_t> v(pr.size(), 1);
    for (size_t i = 0; i < pr.size(); i++) {
      const uint64_t p = pr[i].p;
      uint64_t q = 1;
      for (size_t k = 0; k < i; k++) q = q * (pr[k].p % p) % p;   // all below 2^31: products fit 64 bits
      v[i] = fu_powmod(q, p - 2, p);
    }
    return v;
  }();
  return c;
}

bool fu_crt(const uint32_t* res, int np, const std::vector<FuPrime>& pr, I256* out) {
  constexpr int W = 6;   // 384-bit accumulators
  const std::vector<uint64_t>& cg = fu_garner();
  // mixed-radix digits: X = t_0 + t_1 p_0 + t_2 p_0 p_1 + ..., 0 <= t_i < p_i, with
  // t_i = (res_i - (t_0 + t_1 p_0 + ... + t_{i-1} p_0 ... p_{i-2})) c_i mod p_i, the bracket
  // evaluated mod p_i by Horner (every operand below 2^31)
  uint64_t t[kFuMaxPrimes];
  for (int i = 0; i < np; i++) {
    const uint64_t p = pr[i].p;
    uint64_t acc = 0;
    for (int j = i - 1; j >= 0; j--) acc = (acc * (pr[j].p % p) + t[j]) % p;
    t[i] = ((uint64_t)res[i] % p + p - acc) % p * cg[i] % p;
  }
  auto mul_add = [](uint64_t* acc, const uint64_t* a, uint64_t f) {   // acc += a * f
    unsigned __int128 carry = 0;
    for (int i = 0; i < W; i++) {
      const unsigned __int128 v = (unsigned __int128)a[i] * f + acc[i] + carry;
      acc[i] = (uint64_t)v;
      carry = v >> 64;
    }
  };
  uint64_t X[W] = {0}, Q[W] = {1, 0, 0, 0, 0, 0};
  for (int i = 0; i < np; i++) {
    mul_add(X, Q, t[i]);
    uint64_t Qn[W] = {0};
    mul_add(Qn, Q, pr[i].p);
    std::memcpy(Q, Qn, sizeof(Q));
  }
  // negative when 2X >= Q
  uint64_t X2[W];
  uint64_t carry = 0;
  for (int i = 0; i < W; i++) {
    X2[i] = (X[i] << 1) | carry;
    carry = X[i] >> 63;
  }
  bool neg = false;
  for (int i = W - 1; i >= 0; i--)
    if (X2[i] != Q[i]) {
      neg = X2[i] > Q[i];
      break;
    } else if (i == 0) {
      neg = true;
    }
  uint64_t mag[W];
  if (neg) {   // mag = Q - X
    uint64_t borrow = 0;
    for (int i = 0; i < W; i++) {
      const unsigned __int128 v = (unsigned __int128)Q[i] - X[i] - borrow;
      mag[i] = (uint64_t)v;
      borrow = (uint64_t)(v >> 64) ? 1 : 0;
    }
  } else {
    std::memcpy(mag, X, sizeof(mag));
  }
  if (mag[4] || mag[5] || (mag[3] >> 63)) return false;
  I256 v;
  for (int i = 0; i < 4; i++) v.w[i] = mag[i];
  *out = neg ? i256_neg(v) : v;
  return true;
}

// true when every component has exactly two attributes (then the components, as edges,
// make the relations a tree); signs: bit k of *negmask set when s_k = -1
bool fu_eligible(const sk_set* s, unsigned long long* negmask) {
  if (s->r > 64) return false;
  std::vector<std::vector<int>> members(s->n_comp);
  for (int u = 0; u < (int)s->comp_of.size(); u++) members[s->comp_of[u]].push_back(u);
  for (const auto& mb : members)
    if (mb.size() != 2) return false;
  std::vector<int> sign(s->r, 0);
  sign[0] = 1;
  for (bool changed = true; changed;) {
    changed = false;
    for (const auto& mb : members) {
      const int ka = s->rel_of[mb[0]], kb = s->rel_of[mb[1]];
      if (sign[ka] && !sign[kb]) sign[kb] = -sign[ka], changed = true;
      if (sign[kb] && !sign[ka]) sign[ka] = -sign[kb], changed = true;
    }
  }
  unsigned long long nm = 0;
  for (int k = 0; k < s->r; k++) {
    if (!sign[k]) return false;
    if (sign[k] < 0) nm |= 1ull << k;
  }
  *negmask = nm;
  return true;
}

std::mutex g_fu_const_mutex;
bool g_fu_const_ready[64] = {false};

// Uploads the primes' constants to the current device once; *ready false when the fused
// form cannot run here (fewer primes than needed, device index beyond the table).
cudaError_t fu_constants(bool* ready) {
  *ready = false;
  const std::vector<FuPrime>& pr = fu_primes();
  if ((int)pr.size() < kFuMaxPrimes) return cudaSuccess;
  std::lock_guard<std::mutex> lk(g_fu_const_mutex);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaSuccess;
  if (!g_fu_const_ready[dev]) {
    uint32_t ps[kFuMaxPrimes], pis[kFuMaxPrimes];
    for (int i = 0; i < kFuMaxPrimes; i++) {
      ps[i] = pr[i].p;
      pis[i] = pr[i].pinv;
    }
    cudaError_t e = cudaMemcpyToSymbol(c_fu_p, ps, sizeof(ps));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_fu_pinv, pis, sizeof(pis));
    if (e != cudaSuccess) return e;
    g_fu_const_ready[dev] = true;
  }
  *ready = true;
  return cudaSuccess;
}

// Scratch, bound and primes shared by both fused forms.  The row estimate of Algorithm 3 is
// built from the counters by correlations, Hadamard products and one sum, each of which
// satisfies ||f(a, x)||_1 <= ||a||_1 ||x||_1, so |X_row| <= prod_k ||c_k[row]||_1.  np is
// the number of CRT primes whose product exceeds 8 times the largest such bound (0 when
// nine primes do not reach it); the twiddle tables are kept for transform length M.
struct FuSetup {
  uint32_t* d_res = nullptr;    // [d][kFuMaxPrimes] residues of the row estimates
  uint32_t* d_part = nullptr;   // [d][nchunk] partial sums
  int nchunk = 1;
  int np = 0;
};

sk_status fu_setup(sk_set* s, int64_t M, bool pairwise, cudaStream_t st, FuSetup* f) {
  const int64_t m = s->m;
  const int r = s->r, d = s->d;
  const std::vector<FuPrime>& pr = fu_primes();
  SK_CK(fu_rel_table(s, st));
  // scratch: norm partials [r][d][l1ch][2] doubles | residues [d][9] | partials [d][nchunk]
  int nchunk = 1;
  while ((int64_t)nchunk * 2 * 256 <= M && (int64_t)d * nchunk * 2 <= 4096) nchunk *= 2;
  const int l1ch = fu_l1_chunks((int64_t)r * d, m);
  const size_t l1_bytes = ((size_t)r * d * l1ch * 16 + 255) & ~(size_t)255;
  const size_t res_bytes = ((size_t)d * kFuMaxPrimes * 4 + 255) & ~(size_t)255;
  const size_t part_bytes = ((size_t)d * nchunk * 4 + 255) & ~(size_t)255;
  SK_CK(ensure(s->scratch, l1_bytes + res_bytes + part_bytes, st));
  double* d_l1 = (double*)s->scratch.ptr;
  f->d_res = (uint32_t*)((char*)s->scratch.ptr + l1_bytes);
  f->d_part = (uint32_t*)((char*)f->d_res + res_bytes);
  f->nchunk = nchunk;
  std::vector<double> l1, l2;
  const sk_status ls = fu_norms(s->d_fu_rel, d, (int64_t)r * d, m, d_l1, l1ch, l1, l2, st);
  if (ls != SK_OK) return ls;
  double bits = 0.0;   // log2 of the largest row bound
  for (int row = 0; row < d; row++) bits = std::max(bits, fu_row_bits(&l1[row], &l2[row], r, d, pairwise));
  int np = 0;
  double cover = 0.0;
  while (np < kFuMaxPrimes && cover < bits + 3.0) cover += pr[np++].log2p;
  f->np = cover < bits + 3.0 ? 0 : np;
  if (f->np && (s->fu_m != M || !s->d_fu_tw)) {
    s->fu_np = 0;
    SK_CK(table_alloc((void**)&s->d_fu_tw, (size_t)kFuMaxPrimes * M * sizeof(uint32_t), st));
    s->fu_m = M;
  }
  return SK_OK;
}

// Reads the residues back, reconstructs each row by CRT and fills *out.
sk_status fu_finish(sk_set* s, const FuSetup& f, sk_estimate* out, cudaStream_t st) {
  const int d = s->d;
  const std::vector<FuPrime>& pr = fu_primes();
  s->fu_np = std::max(s->fu_np, f.np);
  std::vector<uint32_t> res((size_t)d * kFuMaxPrimes);
  SK_CK(cudaMemcpyAsync(res.data(), f.d_res, res.size() * 4, cudaMemcpyDeviceToHost, st));
  SK_CK(cudaStreamSynchronize(st));
  I256 rows[SK_MAX_ROWS], sorted[SK_MAX_ROWS];
  for (int row = 0; row < d; row++)
    if (!fu_crt(res.data() + (size_t)row * kFuMaxPrimes, f.np, pr, &rows[row])) return SK_ERR_OVERFLOW;
  std::memcpy(sorted, rows, sizeof(I256) * d);
  std::sort(sorted, sorted + d, [](const I256& a, const I256& b) { return i256_lt(a, b); });
  fill_estimate(out, rows, sorted, d);
  out->max_residual = 0.0;
  out->max_limbs = f.np;      // CRT primes
  out->limb_bits = 0;
  out->corr_steps = s->corr_steps;
  out->retries = 0;
  return SK_OK;
}

// Twiddles of prime PI for length M (once per set and length).
template <int PI>
sk_status fu_twiddles(sk_set* s, const FuPrime& fp, int64_t M, cudaStream_t st) {
  if (s->fu_np > PI) return SK_OK;
  const FuWidth& fw = fu_width(PI, M);
  (void)fp;
  uint32_t* tw = s->d_fu_tw + (size_t)PI * M;
  k_fu_twiddle<PI><<<grid_for(M / 2), 256, 0, st>>>(tw, tw + M / 2, M, fw.w_m, fw.winv_m, fw.one);
  count_launch();
  return set_status_from_cuda(cudaGetLastError());
}

// The fused estimate for queries whose components all join two attributes and a
// power-of-two width: one product of spectra per prime.  *done false when it does not
// apply.
// The small-width form (see k_fu_small): twiddles for every prime once per set, then each
// row's bound and residues in one launch, one read-back.  *done false when a row's bound
// needs more than kFuMaxPrimes primes (the caller then takes the general path).
sk_status run_estimate_pairwise_small(sk_set* s, sk_estimate* out, unsigned long long negmask, cudaStream_t st,
                                      bool* done) {
  *done = false;
  const int64_t m = s->m;
  const int r = s->r, d = s->d;
  const std::vector<FuPrime>& pr = fu_primes();
  SK_CK(fu_rel_table(s, st));
  if (s->fu_m != m || !s->d_fu_tw) {
    s->fu_np = 0;
    SK_CK(table_alloc((void**)&s->d_fu_tw, (size_t)kFuMaxPrimes * m * sizeof(uint32_t), st));
    s->fu_m = m;
  }
  if (s->fu_np < kFuMaxPrimes) {
    sk_status ts = SK_OK;
#define SK_FU_TW(I) if (ts == SK_OK) ts = fu_twiddles<I>(s, pr[I], m, st);
    SK_FU_TW(0) SK_FU_TW(1) SK_FU_TW(2) SK_FU_TW(3) SK_FU_TW(4) SK_FU_TW(5) SK_FU_TW(6) SK_FU_TW(7) SK_FU_TW(8)
#undef SK_FU_TW
    if (ts != SK_OK) return ts;
    s->fu_np = kFuMaxPrimes;
  }
  // scratch: residues [d][kFuMaxPrimes], then each row's prime count
  const size_t out_words = (size_t)d * kFuMaxPrimes + d;
  SK_CK(ensure(s->scratch, out_words * 4, st));
  FuSmallArgs a;
  a.rel = s->d_fu_rel;
  a.tw = s->d_fu_tw;
  int logm = 0;
  while (((int64_t)1 << logm) < m) logm++;
  for (int i = 0; i < kFuMaxPrimes; i++) {
    const FuWidth& fw = fu_width(i, m);
    a.r2[i] = pr[i].r2;
    a.r3[i] = pr[i].r3;
    a.r4[i] = fw.r4;
    a.minv[i] = fw.minv;
    a.log2p[i] = pr[i].log2p;
  }
  a.r = r;
  a.d = d;
  a.logm = logm;
  a.negmask = negmask;
  a.res = (uint32_t*)s->scratch.ptr;
  const size_t smem = (size_t)r * m * sizeof(uint32_t);
  SK_CK(fit_dynamic_smem((const void*)k_fu_small, smem));
  k_fu_small<<<dim3((unsigned)d, kFuMaxPrimes), 256, smem, st>>>(a);
  count_launch();
  SK_CK(cudaGetLastError());
  std::vector<uint32_t> res(out_words);
  SK_CK(cudaMemcpyAsync(res.data(), a.res, out_words * 4, cudaMemcpyDeviceToHost, st));
  SK_CK(cudaStreamSynchronize(st));
  const int* np = (const int*)(res.data() + (size_t)d * kFuMaxPrimes);
  int npmax = 0;
  for (int row = 0; row < d; row++) {
    if (np[row] == 0) return SK_OK;   // a row beyond nine primes: the general path
    npmax = std::max(npmax, np[row]);
  }
  I256 rows[SK_MAX_ROWS], sorted[SK_MAX_ROWS];
  for (int row = 0; row < d; row++)
    if (!fu_crt(res.data() + (size_t)row * kFuMaxPrimes, np[row], pr, &rows[row])) return SK_ERR_OVERFLOW;
  std::memcpy(sorted, rows, sizeof(I256) * d);
  std::sort(sorted, sorted + d, [](const I256& x, const I256& y) { return i256_lt(x, y); });
  fill_estimate(out, rows, sorted, d);
  out->max_residual = 0.0;
  out->max_limbs = npmax;   // CRT primes of the widest row
  out->limb_bits = 0;
  out->corr_steps = s->corr_steps;
  out->retries = 0;
  *done = true;
  return SK_OK;
}

// SK_FUSED_SMALL=0 keeps small widths on the general fused path.
bool fused_small_enabled() {
  const char* v = std::getenv("SK_FUSED_SMALL");
  return !(v && v[0] == '0');
}

sk_status run_estimate_pairwise(sk_set* s, sk_estimate* out, cudaStream_t st, bool* done) {
  *done = false;
  const int64_t m = s->m;
  unsigned long long negmask = 0;
  if ((m & (m - 1)) != 0 || m < 2 || m > (1ll << 22) || !fu_eligible(s, &negmask)) return SK_OK;
  if (m <= 4096 && (int64_t)s->r * m * 4 <= 96 * 1024 && fused_small_enabled()) {
    SK_CK_ST(run_estimate_pairwise_small(s, out, negmask, st, done));
    if (*done) return SK_OK;
  }
  FuSetup f;
  SK_CK_ST(fu_setup(s, m, true, st, &f));
  if (!f.np) return SK_OK;   // beyond nine primes: the GF(q) steps handle it
  const std::vector<FuPrime>& pr = fu_primes();
  const size_t words = (size_t)s->r * s->d * m;
  SK_CK(ensure(s->fft_scratch, 2 * words * sizeof(uint32_t), st));
  uint32_t* V = (uint32_t*)s->fft_scratch.ptr;
  uint32_t* Wb = V + words;
  for (int i = 0; i < f.np; i++) {
    sk_status ps;
    switch (i) {
#define SK_FU_CASE(I)                                                                                      \
  case I:                                                                                                  \
    ps = fu_twiddles<I>(s, pr[I], m, st);                                                                  \
    if (ps == SK_OK)                                                                                       \
      ps = fu_prime_pass<I>(s, pr[I], m, V, Wb, f.d_part, f.nchunk, f.d_res, kFuMaxPrimes, negmask, st);   \
    break;
      SK_FU_CASE(0) SK_FU_CASE(1) SK_FU_CASE(2) SK_FU_CASE(3) SK_FU_CASE(4) SK_FU_CASE(5) SK_FU_CASE(6)
      SK_FU_CASE(7) default: SK_FU_CASE(8)
#undef SK_FU_CASE
    }
    if (ps != SK_OK) return ps;
  }
  SK_CK_ST(fu_finish(s, f, out, st));
  *done = true;
  return SK_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 3 step by step modulo each CRT prime, for every query shape (components of
// three or more attributes, Figure 3) and every width.  The schedule is the one the
// stepwise estimate runs; the row estimate is a polynomial in the counters, so running it
// in Z/p for each prime and reconstructing by CRT (np from the l1 bound above) gives it
// exactly, with one transform per operand of a correlation and no limbs.  Slots hold d
// rows of M residues (Montgomery form), zero beyond m.
// ---------------------------------------------------------------------------
template <int PI>
__global__ void k_crt_leaf(const int64_t* __restrict__ c, int d, int64_t m, int64_t M, uint32_t r2, uint32_t r3,
                           uint32_t* __restrict__ out) {
  using O = MontOps<PI>;
  const uint32_t p = c_fu_p[PI];
  const int64_t total = (int64_t)d * M, step = (int64_t)gridDim.x * blockDim.x;
  const int lM = __ffsll((unsigned long long)M) - 1;   // M is a power of two
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, j = g - row * M;
    uint32_t v = 0;
    if (j < m) {
      const int64_t x = c[row * m + j];
      const uint64_t mag = x < 0 ? 0ull - (uint64_t)x : (uint64_t)x;
      uint32_t h = (uint32_t)(mag >> 32);
      if (h >= p) h -= p;
      v = O::add(O::mul(h, r3), O::mul((uint32_t)mag, r2));
      if (x < 0) v = O::neg(v);
    }
    out[g] = v;
  }
}

template <int PI>
__global__ void k_crt_had(uint32_t* __restrict__ x, const uint32_t* __restrict__ y, int64_t n) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += step)
    x[g] = MontOps<PI>::mul(x[g], y[g]);
}

// X[row][k] <- A[row][-k mod M] X[row][k] / M: the spectrum of z = a (star) x, since
// sum_j z_j w^jk = sum_i a_i w^-ik sum_t x_t w^tk (Definition 3.1, t = i + j mod M)
template <int PI>
__global__ void k_crt_product(const uint32_t* __restrict__ A, uint32_t* __restrict__ X, int d, int64_t M,
                              uint32_t minv) {
  using O = MontOps<PI>;
  const int64_t total = (int64_t)d * M, step = (int64_t)gridDim.x * blockDim.x;
  const int lM = __ffsll((unsigned long long)M) - 1;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, k = g - row * M;
    X[g] = O::mul(O::mul(A[row * M + ((M - k) & (M - 1))], X[g]), minv);
  }
}

// x[row][j] = L[row][j] + L[row][j - m mod M] for j < m, 0 beyond: the circular correlation
// mod m from the length-M one of the zero-padded rows (M >= 2m - 1)
template <int PI>
__global__ void k_crt_fold(const uint32_t* __restrict__ L, uint32_t* __restrict__ x, int d, int64_t m, int64_t M) {
  const int64_t total = (int64_t)d * M, step = (int64_t)gridDim.x * blockDim.x;
  const int lM = __ffsll((unsigned long long)M) - 1;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t row = g >> lM, j = g - row * M;
    x[g] = j < m ? MontOps<PI>::add(L[g], L[row * M + M - m + j]) : 0u;
  }
}

// part[row * nchunk + c] = sum of the c-th chunk of row `row` (mod p)
template <int PI>
__global__ void __launch_bounds__(256) k_crt_rowsum(const uint32_t* __restrict__ x, int64_t M, int nchunk,
                                                    uint32_t* part) {
  using O = MontOps<PI>;
  __shared__ uint32_t red[256];
  const int row = blockIdx.x / nchunk, c = blockIdx.x % nchunk;
  const int64_t clen = M / nchunk;
  const uint32_t* v = x + (int64_t)row * M + (int64_t)c * clen;
  uint32_t s = 0;
  for (int64_t j = threadIdx.x; j < clen; j += blockDim.x) s = O::add(s, v[j]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = O::add(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// One prime's run of the schedule; the row sums' residues go to f.d_res[row][PI].
template <int PI>
sk_status crt_prime_pass(sk_set* s, const FuPrime& fp, int64_t M, uint32_t* slots, uint32_t* T1, uint32_t* T2,
                         const FuSetup& f, cudaStream_t st) {
  using O = MontOps<PI>;
  const int d = s->d;
  const int64_t m = s->m, dM = (int64_t)d * M;
  const FuWidth& fw = fu_width(PI, M);
  const uint32_t one = fw.one, r4 = fw.r4, r4i = fw.r4i, minv = fw.minv;
  const uint32_t* tw = s->d_fu_tw + (size_t)PI * M;
  auto slot = [&](int i) { return slots + (size_t)i * dM; };
  const int eg = grid_for(dM);
  for (const EstOp& op : s->plan) {
    if (op.kind == OP_LEAF) {
      k_crt_leaf<PI><<<eg, 256, 0, st>>>(s->rel_ctr[op.rel], d, m, M, fp.r2, fp.r3, slot(op.dst));
      count_launch();
    } else if (op.kind == OP_HAD) {
      k_crt_had<PI><<<eg, 256, 0, st>>>(slot(op.dst), slot(op.src), dM);
      count_launch();
    } else if (op.kind == OP_CORR) {
      // src (a) is not read after its correlation, so its slot may be clobbered
      sk_status e = xform<O>(slot(op.src), T1, d, M, tw, false, r4, st);
      if (e == SK_OK) e = xform<O>(slot(op.dst), T2, d, M, tw, false, r4, st);
      if (e != SK_OK) return e;
      k_crt_product<PI><<<eg, 256, 0, st>>>(T1, T2, d, M, minv);
      count_launch();
      SK_CK(cudaGetLastError());
      if (M == m) {
        e = xform<O>(T2, slot(op.dst), d, M, tw + M / 2, true, r4i, st);
        if (e != SK_OK) return e;
      } else {
        e = xform<O>(T2, T1, d, M, tw + M / 2, true, r4i, st);
        if (e != SK_OK) return e;
        k_crt_fold<PI><<<eg, 256, 0, st>>>(T1, slot(op.dst), d, m, M);
        count_launch();
      }
    } else {   // OP_SUM
      k_crt_rowsum<PI><<<d * f.nchunk, 256, 0, st>>>(slot(op.dst), M, f.nchunk, f.d_part);
      k_fu_final<PI><<<(d + 63) / 64, 64, 0, st>>>(f.d_part, d, f.nchunk, one, f.d_res, kFuMaxPrimes);
      count_launch(2);
    }
    SK_CK(cudaGetLastError());
  }
  return SK_OK;
}

// The stepwise CRT estimate; *done false when nine primes do not cover the bound.
sk_status run_estimate_crt(sk_set* s, sk_estimate* out, cudaStream_t st, bool* done) {
  *done = false;
  const int64_t m = s->m;
  const int64_t M = (m & (m - 1)) == 0 ? m : (int64_t)1 << ilog2(2 * m - 1);
  if (M < 2 || M > (1ll << 22) || s->n_slots + 1 > 64) return SK_OK;
  FuSetup f;
  SK_CK_ST(fu_setup(s, M, false, st, &f));
  if (!f.np) return SK_OK;
  const std::vector<FuPrime>& pr = fu_primes();
  const size_t dM = (size_t)s->d * M;
  SK_CK(ensure(s->fft_scratch, (size_t)(s->n_slots + 2) * dM * sizeof(uint32_t), st));
  uint32_t* slots = (uint32_t*)s->fft_scratch.ptr;
  uint32_t* T1 = slots + (size_t)s->n_slots * dM;
  uint32_t* T2 = T1 + dM;
  for (int i = 0; i < f.np; i++) {
    sk_status ps;
    switch (i) {
#define SK_CRT_CASE(I)                                                   \
  case I:                                                                \
    ps = fu_twiddles<I>(s, pr[I], M, st);                                \
    if (ps == SK_OK) ps = crt_prime_pass<I>(s, pr[I], M, slots, T1, T2, f, st); \
    break;
      SK_CRT_CASE(0) SK_CRT_CASE(1) SK_CRT_CASE(2) SK_CRT_CASE(3) SK_CRT_CASE(4) SK_CRT_CASE(5) SK_CRT_CASE(6)
      SK_CRT_CASE(7) default: SK_CRT_CASE(8)
#undef SK_CRT_CASE
    }
    if (ps != SK_OK) return ps;
  }
  SK_CK_ST(fu_finish(s, f, out, st));
  *done = true;
  return SK_OK;
}

// The fused estimate: the product of spectra where it applies, else the schedule modulo
// the CRT primes; *done false when neither applies (the caller then runs the GF(q) steps).
sk_status run_estimate_fused(sk_set* s, sk_estimate* out, cudaStream_t st, bool* done) {
  *done = false;
  bool ready = false;
  SK_CK(fu_constants(&ready));
  if (!ready) return SK_OK;
  SK_CK_ST(run_estimate_pairwise(s, out, st, done));
  if (*done) return SK_OK;
  return run_estimate_crt(s, out, st, done);
}

// Evaluation point of one certificate: a random primitive m-th root of unity w in GF(q)
// (power-of-two m dividing 2^32), (7^((q-1)/m))^r with r odd, drawn from the set's seed and
// a per-set counter, so that successive estimates use fresh points.
EvalArgs draw_eval_point(sk_set* s, int64_t m, int nchunk, uint64_t* part) {
  EvalArgs ev;
  uint64_t z = s->seed ^ (0x9E3779B97F4A7C15ull * (++s->eval_draws));
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const uint64_t r = (z % (uint64_t)m) | 1ull;
  const uint64_t wm = gl_pow(7, (kGL - 1) / (uint64_t)m);
  ev.w = gl_pow(wm, r);
  ev.winv = gl_pow(ev.w, kGL - 2);
  ev.wstep = gl_pow(ev.w, 256);
  ev.winvstep = gl_pow(ev.winv, 256);
  ev.e1 = kGLEps;
  ev.e2 = gl_mul(ev.e1, ev.e1);
  ev.e3 = gl_mul(ev.e2, ev.e1);
  ev.e4 = gl_mul(ev.e3, ev.e1);
  ev.m = m;
  ev.nchunk = nchunk;
  ev.part = part;
  return ev;
}

// Chunks per row of the evaluation certificate: the d rows give up to 1024 blocks of 256
// threads, each chunk at least 512 elements.
int eval_chunks(int64_t m, int d) {
  int nchunk = 1;
  while ((int64_t)nchunk * 2 * 256 <= m && (int64_t)d * nchunk * 2 <= 1024) nchunk *= 2;
  return nchunk;
}

// Algorithm 3 over the schedule.  One host round trip per correlation step: before a
// step the host reads the bit lengths of its two operands (written by the kernels that
// produced them) together with the previous step's certificate (largest rounding
// residual, the row sums of a, x and z modulo 2^64, whose identity
// sum z = (sum a)(sum x) holds exactly in Z/2^64, and the row evaluations A(1/w), X(w),
// Z(w) modulo q for power-of-two m).  A failed certificate restarts the
// schedule with narrower limbs for that step.
sk_status run_estimate(sk_set* s, sk_estimate* out, cudaStream_t st) {
  if (s->estimator == SK_ESTIMATOR_FUSED) {
    bool done = false;
    const sk_status fs = run_estimate_fused(s, out, st, &done);
    if (fs != SK_OK || done) return fs;
  }
  const int64_t m = s->m;
  const int d = s->d;
  const int64_t dm = (int64_t)d * m;
  const int logm = ilog2(m);
  // FFT length: m itself when it is a power of two (circular correlation directly), else a
  // power of two >= 2m - 1 holding the zero-padded linear correlation, folded back mod m.
  const int64_t M = (m & (m - 1)) == 0 ? m : (int64_t)1 << ilog2(2 * m - 1);
  const int nslots = s->n_slots + 1;
  const int ncorr = std::max(1, s->corr_steps);
  const size_t slot_bytes = (size_t)dm * sizeof(I256);
  const size_t small_off = slot_bytes * nslots;
  // small buffers: rows, sorted rows (I256 [64] each) | slot bits (int [nslots]) | per step:
  // residual (u64), row sums (u64 [d][3]) and row evaluations (u64 [d][3]) | evaluation
  // partials (u64 [d][nchunk][3], at most 3 * 1024)
  const size_t cw = 1 + 6 * (size_t)d;   // certificate words per step
  const size_t cert_words = (size_t)ncorr * cw;
  const size_t small_bytes = 2 * SK_MAX_ROWS * sizeof(I256) + 256 + cert_words * 8 + 3 * 1024 * 8 + 64;
  SK_CK(ensure(s->scratch, small_off + small_bytes, st));
  if (s->twiddle_m != M) {
    SK_CK(table_alloc((void**)&s->d_twiddle, (size_t)(M / 2) * sizeof(double2), st));
    s->twiddle_m = M;
    k_twiddle<<<grid_for(M / 2), 256, 0, st>>>((double2*)s->d_twiddle, M);
    count_launch();
    SK_CK(cudaGetLastError());
  }
  const double2* tw = (const double2*)s->d_twiddle;
  const double beta = s->estimator == SK_ESTIMATOR_FFT64 ? twiddle_error(M, tw, st) : 0.0;
  char* base = (char*)s->scratch.ptr;
  I256* d_rows = (I256*)(base + small_off);
  I256* d_sorted = d_rows + SK_MAX_ROWS;
  int* d_bits = (int*)(d_sorted + SK_MAX_ROWS);                           // [nslots] (<= 64)
  unsigned long long* d_cert = (unsigned long long*)((char*)d_bits + 256);  // [ncorr][cw]
  uint64_t* d_part = (uint64_t*)(d_cert + cert_words);                       // [d][nchunk][3]
  const int eg = grid_for(dm);
  if (nslots > 64) return SK_ERR_INVALID_ARG;
  // evaluation certificate: FP64 path with a power-of-two m (an m-th root of unity exists in
  // GF(q) for m | 2^32); chunks per row so that the d rows give up to 1024 blocks
  const bool eval_cert = s->estimator == SK_ESTIMATOR_FFT64 && M == m && logm <= 32;
  const int nchunk = eval_chunks(m, d);

  std::vector<int> bmax(ncorr, 64);     // per-step cap on the limb width (lowered on failure)
  std::vector<unsigned long long> cert(cert_words);
  int retries = 0;
  for (int attempt = 0; attempt < 4; attempt++) {
    EvalArgs ev;
    if (eval_cert) ev = draw_eval_point(s, m, nchunk, d_part);
    std::vector<int> phys(nslots);
    for (int i = 0; i < nslots; i++) phys[i] = i;
    auto slot = [&](int i) { return (I256*)(base + slot_bytes * phys[i]); };
    const int spare = nslots - 1;
    SK_CK(cudaMemsetAsync(d_bits, 0, 256, st));
    SK_CK(cudaMemsetAsync(d_cert, 0, cert_words * 8, st));
    std::vector<int> step_B(ncorr, 0);
    double max_resid = 0.0;
    int max_limbs = 0, last_B = 0, corr = 0;
    int failed = -1;
    // checks the certificate of every step < upto whose values are in `cert`: residual,
    // row sums mod 2^64 and (FP64, power-of-two m) Z(w) = A(1/w) X(w) mod q per row; an
    // uncertified step (GF(q), zero operands) holds zeros there, which pass
    auto check = [&](int upto) {
      for (int t = 0; t < upto && failed < 0; t++) {
        const unsigned long long* c = cert.data() + (size_t)t * cw;
        double resid;
        std::memcpy(&resid, &c[0], sizeof(resid));
        max_resid = std::max(max_resid, resid);
        bool ok = resid <= 0.25;
        for (int r = 0; r < d && ok; r++) ok = c[1 + 3 * r + 2] == c[1 + 3 * r] * c[1 + 3 * r + 1];
        const unsigned long long* e = c + 1 + 3 * d;
        for (int r = 0; r < d && ok; r++)
          ok = e[3 * r + 2] == (unsigned long long)(((unsigned __int128)e[3 * r] * e[3 * r + 1]) % kGL);
        if (!ok) failed = t;
      }
    };
    for (const EstOp& op : s->plan) {
      if (failed >= 0) break;
      if (op.kind == OP_LEAF) {
        SK_CK(cudaMemsetAsync(d_bits + phys[op.dst], 0, sizeof(int), st));
        k_leaf<<<eg, 256, 0, st>>>(slot(op.dst), s->rel_ctr[op.rel], dm, d_bits + phys[op.dst]);
        count_launch();
        SK_CK(cudaGetLastError());
      } else if (op.kind == OP_HAD) {
        SK_CK(cudaMemsetAsync(d_bits + phys[op.dst], 0, sizeof(int), st));
        k_hadamard<<<eg, 256, 0, st>>>(slot(op.dst), slot(op.src), dm, s->d_status, d_bits + phys[op.dst]);
        count_launch();
        SK_CK(cudaGetLastError());
      } else if (op.kind == OP_CORR) {
        I256* x = slot(op.dst);
        I256* a = slot(op.src);
        int hb[64];
        SK_CK(cudaMemcpyAsync(hb, d_bits, sizeof(int) * nslots, cudaMemcpyDeviceToHost, st));
        if (corr > 0)
          SK_CK(cudaMemcpyAsync(cert.data(), d_cert, (size_t)corr * cw * 8, cudaMemcpyDeviceToHost, st));
        SK_CK(cudaStreamSynchronize(st));
        check(corr);
        if (failed >= 0) break;
        const int bits_a = hb[phys[op.src]], bits_x = hb[phys[op.dst]];
        unsigned long long* cert_t = d_cert + (size_t)corr * cw;
        if (bits_a == 0 || bits_x == 0) {
          SK_CK(cudaMemsetAsync(x, 0, slot_bytes, st));
          SK_CK(cudaMemsetAsync(d_bits + phys[op.dst], 0, sizeof(int), st));
          corr++;                       // an all-zero step certifies trivially (sums 0, residual 0)
          continue;
        }
        if (bits_a + bits_x + logm + 1 > 255) return SK_ERR_OVERFLOW;
        if (s->estimator != SK_ESTIMATOR_FFT64) {   // GF(q) transforms (also the fused fallback)
          sk_status ns = corr_ntt(s, a, x, slot(spare), d_bits + phys[spare], cert_t, bits_a, bits_x, m, M, st,
                                  &max_limbs, &last_B);
          if (ns != SK_OK) return ns;
          std::swap(phys[op.dst], phys[spare]);
          step_B[corr] = last_B;
          corr++;
          continue;
        }
        int B = std::min(limb_bits_for(m, M, 1, beta), bmax[corr]);
        int La = 0, Lx = 0;
        for (;;) {
          La = (bits_a + 2 + B - 1) / B;
          Lx = (bits_x + 2 + B - 1) / B;
          const int nb = std::min(limb_bits_for(m, M, std::min(La, Lx), beta), bmax[corr]);
          if (nb >= B) break;
          B = nb;
        }
        if (La > kMaxLimbs || Lx > kMaxLimbs) return SK_ERR_INEXACT;
        CorrArgs p;
        p.a = a;
        p.x = x;
        p.z = slot(spare);
        p.m = m;
        p.logm = logm;
        p.d = d;
        p.B = B;
        p.La = La;
        p.Lx = Lx;
        p.nf = (La + Lx + 1) / 2;
        p.ni = (La + Lx) / 2;
        p.status = s->d_status;
        p.residual = cert_t;
        p.sums = cert_t + 1;
        p.zbits = d_bits + phys[spare];
        p.M = M;
        const size_t fbytes = (size_t)d * p.nf * M * sizeof(double2);
        SK_CK(ensure(s->fft_scratch, 2 * fbytes, st));
        double2* bufA = (double2*)s->fft_scratch.ptr;
        double2* bufB = bufA + (size_t)d * p.nf * M;
        p.F = bufA;
        SK_CK(cudaMemsetAsync(p.zbits, 0, sizeof(int), st));
        const int egM = grid_for((int64_t)d * M);
        k_split<<<egM, 256, 0, st>>>(p);
        count_launch();
        SK_CK(cudaGetLastError());
        sk_status fs = fft(bufA, bufB, (int64_t)d * p.nf, M, tw, false, st);
        if (fs != SK_OK) return fs;
        p.F = bufB;
        p.G = bufA;
        k_product<<<egM, 128, 0, st>>>(p);
        count_launch();
        SK_CK(cudaGetLastError());
        fs = fft(bufA, bufB, (int64_t)d * p.ni, M, tw, true, st);
        if (fs != SK_OK) return fs;
        k_recombine<<<eg, 256, 0, st>>>(p, bufB);
        count_launch();
        SK_CK(cudaGetLastError());
        if (eval_cert) {
          ev.a = a;
          ev.x = x;
          ev.z = p.z;
          k_eval_partial<<<d * nchunk, 256, 0, st>>>(ev);
          k_eval_final<<<(3 * d + 255) / 256, 256, 0, st>>>(d_part, d, nchunk, cert_t + 1 + 3 * d);
          count_launch(2);
          SK_CK(cudaGetLastError());
        }
        std::swap(phys[op.dst], phys[spare]);
        step_B[corr] = B;
        max_limbs = std::max(max_limbs, std::max(La, Lx));
        last_B = B;
        corr++;
      } else {  // OP_SUM
        k_rowsum<<<d, 1024, 0, st>>>(slot(op.dst), m, d_rows);
        count_launch();
        k_sort_rows<<<1, 32, 0, st>>>(d_rows, d, d_sorted);
        count_launch();
        SK_CK(cudaGetLastError());
      }
    }
    if (failed < 0) {
      I256 rows[SK_MAX_ROWS], sorted[SK_MAX_ROWS];
      int status = 0;
      SK_CK(cudaMemcpyAsync(rows, d_rows, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
      SK_CK(cudaMemcpyAsync(sorted, d_sorted, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
      SK_CK(cudaMemcpyAsync(&status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      if (corr > 0)
        SK_CK(cudaMemcpyAsync(cert.data(), d_cert, (size_t)corr * cw * 8, cudaMemcpyDeviceToHost, st));
      SK_CK(cudaStreamSynchronize(st));
      check(corr);
      if (failed < 0) {
        if (status != 0) {
          SK_CK(cudaMemsetAsync(s->d_status, 0, sizeof(int), st));
          SK_CK(cudaStreamSynchronize(st));
          return (sk_status)status;
        }
        fill_estimate(out, rows, sorted, d);
        out->max_residual = max_resid;
        out->max_limbs = max_limbs;
        out->limb_bits = last_B;
        out->corr_steps = s->corr_steps;
        out->retries = retries;
        return SK_OK;
      }
    }
    // a step failed its certificate: redo everything with narrower limbs there
    retries++;
    bmax[failed] = std::max(2, (step_B[failed] ? step_B[failed] : limb_bits_for(m, M, 1, beta)) - 3);
  }
  return SK_ERR_INEXACT;
}

// ===========================================================================
// Many sets at once (sk_estimate_many).  Sets that use the fused form and qualify are
// grouped by width; each group is estimated with one load, one transform pass and one
// product-sum per prime over all of its (set, relation, row) vectors, with a descriptor
// per output row.  The other sets run their own estimates concurrently on worker streams.
// ===========================================================================
struct FuOut {
  int64_t base;                 // first vector of the set; vector (base + k d + row)
  int r, d, row;
  unsigned long long negmask;   // relations with s_k = -1
};

// out[v * m + j] = rows[v][j] mod p, Montgomery form
template <int PI>
__global__ void k_fu_load_rows(const int64_t* const* rows, int64_t nvec, int logm, uint32_t r2, uint32_t r3,
                               uint32_t* out) {
  using O = MontOps<PI>;
  const int64_t m = (int64_t)1 << logm, total = nvec * m;
  const uint32_t p = c_fu_p[PI];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int64_t c = rows[g >> logm][g & (m - 1)];
    const uint64_t mag = c < 0 ? 0ull - (uint64_t)c : (uint64_t)c;
    uint32_t h = (uint32_t)(mag >> 32);
    if (h >= p) h -= p;
    const uint32_t v = O::add(O::mul(h, r3), O::mul((uint32_t)mag, r2));
    out[g] = c < 0 ? O::neg(v) : v;
  }
}

template <int PI>
__global__ void __launch_bounds__(256) k_fu_reduce_many(const uint32_t* W, const FuOut* outs, int64_t M, int nchunk,
                                                        uint32_t* part) {
  using O = MontOps<PI>;
  __shared__ uint32_t red[256];
  const FuOut f = outs[blockIdx.x / nchunk];
  const int c = blockIdx.x % nchunk;
  const int64_t clen = M / nchunk;
  uint32_t s = 0;
  constexpr int KR = 8;   // factors loaded before their products
  for (int64_t nu = (int64_t)c * clen + threadIdx.x; nu < (int64_t)(c + 1) * clen; nu += blockDim.x) {
    const int64_t neg_nu = (M - nu) & (M - 1);
    uint32_t fk[KR];
#pragma unroll
    for (int k = 0; k < KR; k++)
      if (k < f.r) fk[k] = W[(f.base + (int64_t)k * f.d + f.row) * M + (((f.negmask >> k) & 1ull) ? neg_nu : nu)];
    uint32_t prod = fk[0];
#pragma unroll
    for (int k = 1; k < KR; k++)
      if (k < f.r) prod = O::mul(prod, fk[k]);
    for (int k = KR; k < f.r; k++)
      prod = O::mul(prod, W[(f.base + (int64_t)k * f.d + f.row) * M + (((f.negmask >> k) & 1ull) ? neg_nu : nu)]);
    s = O::add(s, prod);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = O::add(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// One prime over a group: twiddles, load, forward transforms, product-sums, row values.
template <int PI>
sk_status fu_group_pass(const FuPrime& fp, int64_t M, const int64_t* const* d_rows, int64_t nvec, const FuOut* d_outs,
                        int nout, uint32_t* tw, uint32_t* V, uint32_t* W, uint32_t* part, int nchunk, uint32_t* res,
                        cudaStream_t st) {
  const FuWidth& fw = fu_width(PI, M);
  k_fu_twiddle<PI><<<grid_for(std::max<int64_t>(1, M / 2)), 256, 0, st>>>(tw, tw + M / 2, M, fw.w_m, fw.winv_m,
                                                                           fw.one);
  k_fu_load_rows<PI><<<grid_for(nvec * M), 256, 0, st>>>(d_rows, nvec, ilog2(M), fp.r2, fp.r3, V);
  count_launch(2);
  SK_CK(cudaGetLastError());
  sk_status fs = xform<MontOps<PI>>(V, W, nvec, M, tw, false, fw.r4, st);
  if (fs != SK_OK) return fs;
  k_fu_reduce_many<PI><<<nout * nchunk, 256, 0, st>>>(W, d_outs, M, nchunk, part);
  k_fu_final<PI><<<(nout + 63) / 64, 64, 0, st>>>(part, nout, nchunk, fw.minv, res, kFuMaxPrimes);
  count_launch(2);
  return set_status_from_cuda(cudaGetLastError());
}

// The fused estimates of one group of sets of width M (all eligible); done[i] is set for
// every set estimated here (a group whose bound needs more than 9 primes is left to the
// caller).
sk_status fu_group(sk_set** sets, const std::vector<int>& idx, int64_t M, sk_estimate* out, std::vector<char>& done,
                   cudaStream_t st) {
  const std::vector<FuPrime>& pr = fu_primes();
  std::vector<const int64_t*> rows;
  std::vector<FuOut> outs;
  for (int i : idx) {
    sk_set* s = sets[i];
    unsigned long long negmask = 0;
    fu_eligible(s, &negmask);
    const int64_t base = (int64_t)rows.size();
    for (int k = 0; k < s->r; k++)
      for (int row = 0; row < s->d; row++) rows.push_back(s->rel_ctr[k] + (int64_t)row * M);
    for (int row = 0; row < s->d; row++) outs.push_back({base, s->r, s->d, row, negmask});
  }
  const int64_t nvec = (int64_t)rows.size();
  const int nout = (int)outs.size();
  int nchunk = 1;
  while ((int64_t)nchunk * 2 * 256 <= M && (int64_t)nout * nchunk * 2 <= 4096) nchunk *= 2;
  // one stream-ordered block: row pointers | descriptors | l1 | residues | partials |
  // twiddles | V | W (freed at the end of the call)
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const int l1ch = fu_l1_chunks(nvec, M);
  const size_t b_rows = al(nvec * sizeof(void*)), b_outs = al(nout * sizeof(FuOut)),
               b_l1 = al((size_t)nvec * l1ch * 16), b_res = al((size_t)nout * kFuMaxPrimes * 4), b_part = al((size_t)nout * nchunk * 4),
               b_tw = al((size_t)M * 4), b_v = al((size_t)nvec * M * 4);
  char* blk = nullptr;
  SK_CK(pool_malloc_async((void**)&blk, b_rows + b_outs + b_l1 + b_res + b_part + b_tw + 2 * b_v, st));
  const int64_t** d_rows = (const int64_t**)blk;
  FuOut* d_outs = (FuOut*)(blk + b_rows);
  double* d_l1 = (double*)(blk + b_rows + b_outs);
  uint32_t* d_res = (uint32_t*)(blk + b_rows + b_outs + b_l1);
  uint32_t* d_part = (uint32_t*)((char*)d_res + b_res);
  uint32_t* d_tw = (uint32_t*)((char*)d_part + b_part);
  uint32_t* V = (uint32_t*)((char*)d_tw + b_tw);
  uint32_t* W = (uint32_t*)((char*)V + b_v);
  sk_status status = SK_OK;
  auto fail = [&](sk_status x) {
    if (status == SK_OK) status = x;
  };
  std::vector<double> l1, l2;
  std::vector<uint32_t> res((size_t)nout * kFuMaxPrimes);
  // per set: the primes its own rows' bound needs; sets are then ordered by that count,
  // largest first, so that prime i only loads, transforms and reduces the leading sets
  // that need more than i primes
  const int nset = (int)idx.size();
  std::vector<int> set_np(nset, 0), order;
  std::vector<int64_t> nvec_at(kFuMaxPrimes, 0);
  std::vector<int> nout_at(kFuMaxPrimes, 0);
  int np = 0;
  do {
    cudaError_t e = cudaMemcpyAsync(d_rows, rows.data(), nvec * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { fail(set_status_from_cuda(e)); break; }
    const sk_status ls = fu_norms(d_rows, 1, nvec, M, d_l1, l1ch, l1, l2, st);
    if (ls != SK_OK) { fail(ls); break; }
    int o = 0;
    for (int t = 0; t < nset; t++) {
      const sk_set* s = sets[idx[t]];
      double bits = 0.0;
      for (int row = 0; row < s->d; row++, o++)
        bits = std::max(bits, fu_row_bits(&l1[outs[o].base + row], &l2[outs[o].base + row], s->r, s->d, true));
      int k = 0;
      double cover = 0.0;
      while (k < kFuMaxPrimes && cover < bits + 3.0) cover += pr[k++].log2p;
      set_np[t] = cover < bits + 3.0 ? 0 : k;   // 0: beyond nine primes, left to the caller
      if (set_np[t] > 0) order.push_back(t);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return set_np[x] > set_np[y]; });
    if (order.empty()) break;
    np = set_np[order[0]];
    // rows and outputs again in that order
    std::vector<const int64_t*> rows2;
    std::vector<FuOut> outs2;
    for (int t : order) {
      const sk_set* s = sets[idx[t]];
      unsigned long long negmask = 0;
      fu_eligible(s, &negmask);
      const int64_t base = (int64_t)rows2.size();
      for (int k = 0; k < s->r; k++)
        for (int row = 0; row < s->d; row++) rows2.push_back(s->rel_ctr[k] + (int64_t)row * M);
      for (int row = 0; row < s->d; row++) outs2.push_back({base, s->r, s->d, row, negmask});
      for (int i = 0; i < set_np[t]; i++) {
        nvec_at[i] = (int64_t)rows2.size();
        nout_at[i] = (int)outs2.size();
      }
    }
    e = cudaMemcpyAsync(d_rows, rows2.data(), rows2.size() * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_outs, outs2.data(), outs2.size() * sizeof(FuOut), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { fail(set_status_from_cuda(e)); break; }
    for (int i = 0; i < np && status == SK_OK; i++) {
      const int64_t nv = nvec_at[i];
      const int no = nout_at[i];
      sk_status ps;
      switch (i) {
#define SK_GP_CASE(I)                                                                                     \
  case I:                                                                                                 \
    ps = fu_group_pass<I>(pr[I], M, d_rows, nv, d_outs, no, d_tw, V, W, d_part, nchunk, d_res, st);        \
    break;
        SK_GP_CASE(0) SK_GP_CASE(1) SK_GP_CASE(2) SK_GP_CASE(3) SK_GP_CASE(4) SK_GP_CASE(5) SK_GP_CASE(6)
        SK_GP_CASE(7) default: SK_GP_CASE(8)
#undef SK_GP_CASE
      }
      fail(ps);
    }
    if (status != SK_OK) break;
    e = cudaMemcpyAsync(res.data(), d_res, res.size() * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) fail(set_status_from_cuda(e));
  } while (false);
  const cudaError_t ef = cudaFreeAsync(blk, st);
  if (status != SK_OK) return status;
  if (ef != cudaSuccess) return set_status_from_cuda(ef);
  if (np == 0) return SK_OK;
  int o = 0;
  for (int t : order) {
    const int i = idx[t];
    sk_set* s = sets[i];
    I256 r_rows[SK_MAX_ROWS], sorted[SK_MAX_ROWS];
    for (int row = 0; row < s->d; row++, o++)
      if (!fu_crt(res.data() + (size_t)o * kFuMaxPrimes, set_np[t], pr, &r_rows[row])) return SK_ERR_OVERFLOW;
    std::memcpy(sorted, r_rows, sizeof(I256) * s->d);
    std::sort(sorted, sorted + s->d, [](const I256& a, const I256& b) { return i256_lt(a, b); });
    fill_estimate(&out[i], r_rows, sorted, s->d);
    out[i].max_residual = 0.0;
    out[i].max_limbs = set_np[t];
    out[i].limb_bits = 0;
    out[i].corr_steps = s->corr_steps;
    out[i].retries = 0;
    done[i] = 1;
  }
  return SK_OK;
}

int many_workers() {
  const char* v = std::getenv("SK_MANY_WORKERS");
  const int x = v ? std::atoi(v) : 4;
  return x < 1 ? 1 : (x > 16 ? 16 : x);
}

sk_status run_estimate_many(sk_set** sets, int n, sk_estimate* out, cudaStream_t st) {
  std::vector<char> done(n, 0);
  std::vector<sk_status> status(n, SK_OK);
  // fused groups by width, on the caller's stream
  std::map<int64_t, std::vector<int>> groups;
  bool ready = false;
  SK_CK(fu_constants(&ready));
  for (int i = 0; i < n; i++) {
    sk_set* s = sets[i];
    unsigned long long nm = 0;
    const int64_t m = s->m;
    if (ready && s->estimator == SK_ESTIMATOR_FUSED && (m & (m - 1)) == 0 && m >= 2 && m <= (1ll << 22) &&
        fu_eligible(s, &nm))
      groups[m].push_back(i);
  }
  for (auto& g : groups) {
    const sk_status gs = fu_group(sets, g.second, g.first, out, done, st);
    if (gs != SK_OK) return gs;
  }
  // everything else: per-set estimates on worker streams, after the caller's queued work
  std::vector<int> rest;
  for (int i = 0; i < n; i++)
    if (!done[i]) rest.push_back(i);
  if (rest.empty()) return SK_OK;
  const int nw = std::min<int>(many_workers(), (int)rest.size());
  std::vector<cudaStream_t> ws(nw, nullptr);
  cudaEvent_t ev = nullptr;
  cudaError_t ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev, st);
  for (int w = 0; w < nw && ce == cudaSuccess; w++) {
    ce = cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ws[w], ev, 0);
  }
  if (ce == cudaSuccess) {
    int dev = 0;
    cudaGetDevice(&dev);
    auto work = [&](int w) {
      cudaSetDevice(dev);
      for (size_t j = w; j < rest.size(); j += nw) {
        const int i = rest[j];
        status[i] = run_estimate(sets[i], &out[i], ws[w]);
      }
    };
    std::vector<std::thread> th;
    for (int w = 1; w < nw; w++) th.emplace_back(work, w);
    work(0);
    for (auto& t : th) t.join();
    for (int w = 0; w < nw && ce == cudaSuccess; w++) {   // the caller's stream continues after them
      ce = cudaEventRecord(ev, ws[w]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, ev, 0);
    }
  }
  for (cudaStream_t w : ws)
    if (w) cudaStreamDestroy(w);
  if (ev) cudaEventDestroy(ev);
  if (ce != cudaSuccess) return set_status_from_cuda(ce);
  for (int i : rest)
    if (status[i] != SK_OK) return status[i];
  return SK_OK;
}

// ===========================================================================
// Estimation without device allocation (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc while they estimate: code running inside
// a host callback or a driver-level hook where the CUDA allocator must not be
// entered, processes whose device memory is fully reserved by another pool, or
// latency-critical paths that forbid allocation.  sk_estimate_join_noalloc runs
// the same Algorithm 3 schedule with the same kernels as sk_estimate_join, but
// carves every scratch buffer (vector slots, FFT buffers, twiddles, small
// result buffers) out of one file-scope device array of kNoAllocScratchBytes.
// That array lives in every GPU that loads this library until the process
// exits.  Its device address is looked up once per device (the first call on
// that device, with that device current) with cudaGetSymbolAddress; the host-
// side name of the array is only a stand-in and is never passed to a kernel.
// All calls share the array: two calls whose work overlaps on the GPU (other
// streams, other threads) race on it.  Every buffer that must start at zero is
// cleared on the call's stream before use.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = SK_NOALLOC_SCRATCH_BYTES;   // 32 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::atomic<void*> g_noalloc_addr[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device, which must be the set's
// device (the set's counters and the scratch must live on the same GPU).  The first call
// on a device looks it up (under a lock; later calls read the cached address).
sk_status noalloc_base(const sk_set* s, char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_status_from_cuda(e);
  if (dev < 0 || dev >= kNoAllocMaxDevices || dev != s->device) return SK_ERR_INVALID_ARG;
  void* ptr = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    ptr = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!ptr) {
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return set_status_from_cuda(e);
      g_noalloc_addr[dev].store(ptr, std::memory_order_release);
    }
  }
  *out = (char*)ptr;
  return SK_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// Every correlation step is accepted on three checks, as in run_estimate's FP64 path: the
// largest distance of an output to its integer (<= 1/4), the exact per-row identity
// sum z = (sum a)(sum x) (here in signed 256-bit arithmetic), and Z(w) = A(1/w) X(w) modulo
// q = 2^64 - 2^32 + 1 per row at a freshly drawn random primitive m-th root of unity w.
// A step that fails is redone with narrower limbs (up to three times).
sk_status run_estimate_noalloc(sk_set* s, sk_estimate* out, cudaStream_t st) {
  const int64_t m = s->m;
  const int d = s->d;
  const int64_t dm = (int64_t)d * m;
  const int logm = ilog2(m);
  const int nslots = s->n_slots + 1;
  if (nslots > 64) return SK_ERR_SCRATCH_TOO_SMALL;
  const int nchunk = eval_chunks(m, d);
  // layout: small buffers | twiddles | slots | FFT A | FFT B.  Small buffers: row sums of
  // a, x, z and the sorted rows (I256 [64] each) | bit lengths (int [4]) | residual (u64) |
  // evaluation partials (u64 [d][nchunk][3]) | row evaluations (u64 [d][3])
  const size_t part_words = (size_t)d * nchunk * 3;
  const size_t small_bytes = align256(4 * SK_MAX_ROWS * sizeof(I256) + 64 + part_words * 8 + 3 * SK_MAX_ROWS * 8);
  const size_t tw_bytes = align256((size_t)(m / 2) * sizeof(double2));
  const size_t slot_bytes = align256((size_t)dm * sizeof(I256));
  const size_t fixed = small_bytes + tw_bytes + slot_bytes * nslots;
  if (fixed > kNoAllocScratchBytes) return SK_ERR_SCRATCH_TOO_SMALL;
  const size_t fft_room = kNoAllocScratchBytes - fixed;
  char* base = nullptr;
  sk_status bs = noalloc_base(s, &base);
  if (bs != SK_OK) return bs;
  I256* d_sa = (I256*)base;
  I256* d_sx = d_sa + SK_MAX_ROWS;
  I256* d_sz = d_sx + SK_MAX_ROWS;
  I256* d_sorted = d_sz + SK_MAX_ROWS;
  int* d_bits = (int*)(d_sorted + SK_MAX_ROWS);
  unsigned long long* d_resid = (unsigned long long*)(d_bits + 4);
  uint64_t* d_part = (uint64_t*)((char*)d_bits + 64);            // after the 64-byte block of bits + residual
  unsigned long long* d_eval = (unsigned long long*)(d_part + part_words);
  double2* tw = (double2*)(base + small_bytes);
  char* slot_base = base + small_bytes + tw_bytes;
  int phys[64];
  for (int i = 0; i < nslots; i++) phys[i] = i;
  auto slot = [&](int i) { return (I256*)(slot_base + slot_bytes * phys[i]); };
  const int spare = nslots - 1;

  SK_CK(cudaMemsetAsync(base, 0, small_bytes, st));
  k_twiddle<<<grid_for(m / 2), 256, 0, st>>>(tw, m);
  count_launch();
  SK_CK(cudaGetLastError());
  const double beta = twiddle_error(m, tw, st);

  double max_resid = 0.0;
  int max_limbs = 0, last_B = 0, retries = 0;
  const int eg = grid_for(dm);
  I256 sa[SK_MAX_ROWS], sx[SK_MAX_ROWS], sz[SK_MAX_ROWS];
  unsigned long long evals[3 * SK_MAX_ROWS];

  for (const EstOp& op : s->plan) {
    if (op.kind == OP_LEAF) {
      k_leaf<<<eg, 256, 0, st>>>(slot(op.dst), s->rel_ctr[op.rel], dm, nullptr);
      count_launch();
      SK_CK(cudaGetLastError());
    } else if (op.kind == OP_HAD) {
      k_hadamard<<<eg, 256, 0, st>>>(slot(op.dst), slot(op.src), dm, s->d_status, nullptr);
      count_launch();
      SK_CK(cudaGetLastError());
    } else if (op.kind == OP_CORR) {
      I256* x = slot(op.dst);
      I256* a = slot(op.src);
      SK_CK(cudaMemsetAsync(d_bits, 0, 2 * sizeof(int), st));
      k_maxbits<<<eg, 256, 0, st>>>(a, dm, d_bits);
      count_launch();
      k_maxbits<<<eg, 256, 0, st>>>(x, dm, d_bits + 1);
      count_launch();
      k_rowsum<<<d, 1024, 0, st>>>(a, m, d_sa);
      count_launch();
      k_rowsum<<<d, 1024, 0, st>>>(x, m, d_sx);
      count_launch();
      SK_CK(cudaGetLastError());
      int hb[2];
      SK_CK(cudaMemcpyAsync(hb, d_bits, sizeof(hb), cudaMemcpyDeviceToHost, st));
      SK_CK(cudaMemcpyAsync(sa, d_sa, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
      SK_CK(cudaMemcpyAsync(sx, d_sx, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
      SK_CK(cudaStreamSynchronize(st));
      if (hb[0] == 0 || hb[1] == 0) {
        SK_CK(cudaMemsetAsync(x, 0, (size_t)dm * sizeof(I256), st));
        continue;
      }
      if (hb[0] + hb[1] + logm + 1 > 255) return SK_ERR_OVERFLOW;
      int B = limb_bits_for(m, m, 1, beta);
      bool done = false;
      for (int attempt = 0; attempt < 4 && !done; attempt++) {
        int La = 0, Lx = 0;
        for (;;) {
          La = (hb[0] + 2 + B - 1) / B;
          Lx = (hb[1] + 2 + B - 1) / B;
          const int nb = limb_bits_for(m, m, std::min(La, Lx), beta);
          if (nb >= B) break;
          B = nb;
        }
        if (attempt > 0) {
          B = std::max(2, B - 3 * attempt);
          La = (hb[0] + 2 + B - 1) / B;
          Lx = (hb[1] + 2 + B - 1) / B;
        }
        if (La > kMaxLimbs || Lx > kMaxLimbs) return SK_ERR_INEXACT;
        CorrArgs p;
        p.a = a;
        p.x = x;
        p.z = slot(spare);
        p.m = m;
        p.logm = logm;
        p.d = d;
        p.B = B;
        p.La = La;
        p.Lx = Lx;
        p.nf = (La + Lx + 1) / 2;
        p.ni = (La + Lx) / 2;
        p.status = s->d_status;
        p.residual = d_resid;
        p.sums = nullptr;
        p.zbits = nullptr;
        p.M = m;
        const size_t fbytes = align256((size_t)d * p.nf * m * sizeof(double2));
        if (2 * fbytes > fft_room) return SK_ERR_SCRATCH_TOO_SMALL;
        double2* bufA = (double2*)(slot_base + slot_bytes * nslots);
        double2* bufB = (double2*)((char*)bufA + fbytes);
        p.F = bufA;
        SK_CK(cudaMemsetAsync(d_resid, 0, sizeof(unsigned long long), st));
        k_split<<<eg, 256, 0, st>>>(p);
        count_launch();
        SK_CK(cudaGetLastError());
        sk_status fs = fft(bufA, bufB, (int64_t)d * p.nf, m, tw, false, st);
        if (fs != SK_OK) return fs;
        p.F = bufB;
        p.G = bufA;
        k_product<<<eg, 128, 0, st>>>(p);
        count_launch();
        SK_CK(cudaGetLastError());
        fs = fft(bufA, bufB, (int64_t)d * p.ni, m, tw, true, st);
        if (fs != SK_OK) return fs;
        k_recombine<<<eg, 256, 0, st>>>(p, bufB);
        count_launch();
        k_rowsum<<<d, 1024, 0, st>>>(p.z, m, d_sz);
        count_launch();
        EvalArgs ev = draw_eval_point(s, m, nchunk, d_part);
        ev.a = a;
        ev.x = x;
        ev.z = p.z;
        k_eval_partial<<<d * nchunk, 256, 0, st>>>(ev);
        k_eval_final<<<(3 * d + 255) / 256, 256, 0, st>>>(d_part, d, nchunk, d_eval);
        count_launch(2);
        SK_CK(cudaGetLastError());
        unsigned long long rbits = 0;
        SK_CK(cudaMemcpyAsync(&rbits, d_resid, sizeof(rbits), cudaMemcpyDeviceToHost, st));
        SK_CK(cudaMemcpyAsync(sz, d_sz, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
        SK_CK(cudaMemcpyAsync(evals, d_eval, 3 * d * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        SK_CK(cudaStreamSynchronize(st));
        double resid;
        std::memcpy(&resid, &rbits, sizeof(resid));
        bool ok = resid <= 0.25;
        for (int r = 0; r < d && ok; r++) ok = i256_eq(sz[r], HostI256::mul(sa[r], sx[r]));
        for (int r = 0; r < d && ok; r++)
          ok = evals[3 * r + 2] == (unsigned long long)(((unsigned __int128)evals[3 * r] * evals[3 * r + 1]) % kGL);
        if (ok) {
          max_resid = std::max(max_resid, resid);
          max_limbs = std::max(max_limbs, std::max(La, Lx));
          last_B = B;
          std::swap(phys[op.dst], phys[spare]);
          done = true;
        } else {
          retries++;
        }
      }
      if (!done) return SK_ERR_INEXACT;
    } else {  // OP_SUM
      k_rowsum<<<d, 1024, 0, st>>>(slot(op.dst), m, d_sz);
      count_launch();
      k_sort_rows<<<1, 32, 0, st>>>(d_sz, d, d_sorted);
      count_launch();
      SK_CK(cudaGetLastError());
    }
  }
  I256 rows[SK_MAX_ROWS], sorted[SK_MAX_ROWS];
  int status = 0;
  SK_CK(cudaMemcpyAsync(rows, d_sz, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
  SK_CK(cudaMemcpyAsync(sorted, d_sorted, d * sizeof(I256), cudaMemcpyDeviceToHost, st));
  SK_CK(cudaMemcpyAsync(&status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SK_CK(cudaStreamSynchronize(st));
  if (status != 0) {
    SK_CK(cudaMemsetAsync(s->d_status, 0, sizeof(int), st));
    SK_CK(cudaStreamSynchronize(st));
    return (sk_status)status;
  }
  fill_estimate(out, rows, sorted, d);
  out->max_residual = max_resid;
  out->max_limbs = max_limbs;
  out->limb_bits = last_B;
  out->corr_steps = s->corr_steps;
  out->retries = retries;
  return SK_OK;
}

}  // namespace sk
