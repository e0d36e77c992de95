/*
 * Plain CPU oracle for the convolved Count-sketch method of Heddes, Nunes,
 * Givargis and Nicolau, "Convolution and Cross-Correlation of Count Sketches
 * Enables Fast Cardinality Estimation of Multi-Join Queries" (PACMMOD 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code with the CUDA implementation: the field
 * arithmetic below is written with unsigned __int128 and the C `%` operator
 * only (no Mersenne-prime folding), and the exact integer correlation is a
 * direct O(m^2) double loop.
 *
 * Contents
 *   - field map and polynomial hashes over GF(p), p = 2^61 - 1, the
 *     "random polynomials over a Mersenne prime field" of Section 4: a
 *     degree-1 polynomial for the 2-wise independent bin function and a
 *     degree-3 polynomial for the 4-wise independent sign function
 *     (Definition 2.1; Count sketch, Section 2.4);
 *   - sketch creation, Algorithm 2 / Eq. 4: per tuple the bin is the sum of
 *     the per-attribute bins mod m (Eq. 3) and the sign is the product of the
 *     per-join signs (Eq. 2); the counter at that bin receives sign * Delta;
 *   - circular cross-correlation, Definition 3.1, for real integer vectors:
 *     z_j = sum_i a_i x_{(j+i) mod m}, computed exactly, in two forms:
 *     int64 inputs with an int128 accumulator (used only when the caller has
 *     shown that no intermediate can leave the int128 range), and a signed
 *     256-bit two's-complement type for everything else.
 */
#include <stdint.h>
#include <string.h>

typedef unsigned __int128 or_u128;
typedef __int128 or_i128;

#define OR_P ((((uint64_t)1) << 61) - 1u)

/* x -> (uint64)x mod p: how an int64 join key becomes a field element. */
uint64_t or_field(int64_t key) { return ((uint64_t)key) % OR_P; }

uint64_t or_mulmod(uint64_t a, uint64_t b) { return (uint64_t)(((or_u128)a * (or_u128)b) % OR_P); }

/* sum_{t<k} c[t] x^t mod p, by Horner's rule; every step reduced with `%`. */
uint64_t or_poly(const uint64_t* c, int k, uint64_t x) {
  or_u128 acc = c[k - 1] % OR_P;
  for (int t = k - 2; t >= 0; t--) acc = (acc * (or_u128)x + (or_u128)c[t]) % OR_P;
  return (uint64_t)acc;
}

/* Bin function h(x) = ((b1 x + b0) mod p) mod m. */
int64_t or_bin(const uint64_t* b, uint64_t x, int64_t m) { return (int64_t)(or_poly(b, 2, x) % (uint64_t)m); }

/* Sign function s(x) = +1 if (s3 x^3 + s2 x^2 + s1 x + s0) mod p is even, else -1. */
int or_sign(const uint64_t* s, uint64_t x) { return (or_poly(s, 4, x) & 1u) ? -1 : +1; }

/*
 * Algorithm 2 (CreateSketch), all d median rows, accumulated into out[d][m].
 *
 * Relation R_k has a_k joined attributes; attribute u reads its key of tuple i
 * at cols[u * col_stride + i].  attr_comp[u] is the graph component Psi(u);
 * attr_edges[attr_edge_off[u] .. attr_edge_off[u+1]) are the indices of the
 * join edges {u, v}, v in Gamma(u).  Row `row` of the coefficient table is
 * coeffs[row * (2*n_comp + 4*n_edges) ...]: first (b0, b1) for each component,
 * then (s0, s1, s2, s3) for each edge.  weights == NULL means Delta = 1.
 * Counters are int64 with two's-complement wrap-around (done in uint64).
 */
void or_sketch(int64_t n, int a_k, const int64_t* cols, int64_t col_stride, const int64_t* weights,
               int d, int64_t m, const int32_t* attr_comp, const int32_t* attr_edge_off,
               const int32_t* attr_edges, int n_comp, int n_edges, const uint64_t* coeffs,
               int64_t* out) {
  const int64_t row_len = 2 * (int64_t)n_comp + 4 * (int64_t)n_edges;
  for (int64_t i = 0; i < n; i++) {
    const int64_t delta = weights ? weights[i] : 1;
    for (int row = 0; row < d; row++) {
      const uint64_t* cr = coeffs + row * row_len;
      int64_t j = 0;   /* accumulation of bins */
      int64_t x = 1;   /* accumulation of signs */
      for (int u = 0; u < a_k; u++) {
        const uint64_t key = or_field(cols[(int64_t)u * col_stride + i]);
        j += or_bin(cr + 2 * attr_comp[u], key, m);
        for (int t = attr_edge_off[u]; t < attr_edge_off[u + 1]; t++)
          x *= or_sign(cr + 2 * (int64_t)n_comp + 4 * (int64_t)attr_edges[t], key);
      }
      j %= m;
      uint64_t* c = (uint64_t*)(out + (int64_t)row * m + j);
      *c += (uint64_t)x * (uint64_t)delta;
    }
  }
}

/* Per-tuple (bin, sign) for every row: the two quantities of Eqs. 2-3. */
void or_tuple_hash(int a_k, const int64_t* keys, int d, int64_t m, const int32_t* attr_comp,
                   const int32_t* attr_edge_off, const int32_t* attr_edges, int n_comp, int n_edges,
                   const uint64_t* coeffs, int64_t* bins, int32_t* signs) {
  const int64_t row_len = 2 * (int64_t)n_comp + 4 * (int64_t)n_edges;
  for (int row = 0; row < d; row++) {
    const uint64_t* cr = coeffs + row * row_len;
    int64_t j = 0;
    int x = 1;
    for (int u = 0; u < a_k; u++) {
      const uint64_t key = or_field(keys[u]);
      j += or_bin(cr + 2 * attr_comp[u], key, m);
      for (int t = attr_edge_off[u]; t < attr_edge_off[u + 1]; t++)
        x *= or_sign(cr + 2 * (int64_t)n_comp + 4 * (int64_t)attr_edges[t], key);
    }
    bins[row] = j % m;
    signs[row] = x;
  }
}

/* ---- exact correlation, Definition 3.1 ---------------------------------- */

/* z[j - j0] = sum_i a[i] x[(j+i) mod m] for j in [j0, j1); the caller guarantees
 * max|a| * max|x| * m < 2^127, so the int128 sum is exact.  z is written as
 * (lo, hi) uint64 pairs. */
void or_correlate_i64(const int64_t* a, const int64_t* x, int64_t m, int64_t j0, int64_t j1,
                      uint64_t* z) {
  for (int64_t j = j0; j < j1; j++) {
    or_i128 acc = 0;
    for (int64_t i = 0; i < m; i++) acc += (or_i128)a[i] * (or_i128)x[(j + i) % m];
    z[2 * (j - j0)] = (uint64_t)(or_u128)acc;
    z[2 * (j - j0) + 1] = (uint64_t)((or_u128)acc >> 64);
  }
}

/* Signed 256-bit two's-complement integers, four little-endian 64-bit words. */
typedef struct { uint64_t w[4]; } or_i256;

static or_i256 i256_add(or_i256 a, or_i256 b) {
  or_i256 r;
  or_u128 carry = 0;
  for (int k = 0; k < 4; k++) {
    or_u128 s = (or_u128)a.w[k] + b.w[k] + carry;
    r.w[k] = (uint64_t)s;
    carry = s >> 64;
  }
  return r;
}

/* product modulo 2^256, which is the exact product whenever it fits */
static or_i256 i256_mul(or_i256 a, or_i256 b) {
  uint64_t r[4] = {0, 0, 0, 0};
  for (int i = 0; i < 4; i++) {
    or_u128 carry = 0;
    for (int j = 0; i + j < 4; j++) {
      or_u128 t = (or_u128)a.w[i] * b.w[j] + r[i + j] + carry;
      r[i + j] = (uint64_t)t;
      carry = t >> 64;
    }
  }
  or_i256 out;
  memcpy(out.w, r, sizeof r);
  return out;
}

void or_correlate_i256(const uint64_t* a, const uint64_t* x, int64_t m, int64_t j0, int64_t j1,
                       uint64_t* z) {
  const or_i256* A = (const or_i256*)a;
  const or_i256* X = (const or_i256*)x;
  for (int64_t j = j0; j < j1; j++) {
    or_i256 acc = {{0, 0, 0, 0}};
    for (int64_t i = 0; i < m; i++) acc = i256_add(acc, i256_mul(A[i], X[(j + i) % m]));
    memcpy(z + 4 * (j - j0), acc.w, sizeof acc.w);
  }
}
