"""Plain CPU oracle for Heddes et al., "Convolution and Cross-Correlation of
Count Sketches Enables Fast Cardinality Estimation of Multi-Join Queries"
(PACMMOD 2024).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  The library
(`paper_2402_15953_gb300`) never imports it and shares no code with it: the
hash arithmetic lives in `cs_oracle.c` (unsigned __int128 and `%`), the query
handling and Algorithm 3 are plain Python with Python integers, so every
estimate here is exact.

What each function follows:
  canonical_query      Section 2.6 notation (Omega, Gamma, Psi, E) and the
                       initialisation paragraph of Section 3.2
  draw_coefficients    Algorithm 1 (SampleSignHashes, SampleBinHashes)
  sketch_relation      Algorithm 2 / Eq. 4 (hashes per Eqs. 2-3)
  correlate            Definition 3.1 (direct O(m^2) sum, exact)
  estimate_row         Algorithm 3 (GetQueryEstimate / CombineSketches)
  brute_force_row      Eq. 5 (sum over J = [m]^components)
  median_lower         median trick of Section 3.3 and the l = 5 medians of
                       Section 4.1
  exact_join_size      E[X] of Theorem 3.1 (the true join cardinality)
  subquery             Section 3.4 (sub-queries for plan enumeration; sketch reuse)

Every row of every estimate uses its own, independently drawn hash functions
("l i.i.d. estimates", Section 3.3).
"""
from __future__ import annotations

import ctypes
import dataclasses
import itertools
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

P61 = (1 << 61) - 1
MASK64 = (1 << 64) - 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcs_oracle.so")
_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile cs_oracle.c into oracle/_build/libcs_oracle.so (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lib_lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64, i64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int
            vp = ctypes.c_void_p
            L.or_field.restype = u64; L.or_field.argtypes = [i64]
            L.or_mulmod.restype = u64; L.or_mulmod.argtypes = [u64, u64]
            L.or_poly.restype = u64; L.or_poly.argtypes = [vp, i32, u64]
            L.or_bin.restype = i64; L.or_bin.argtypes = [vp, u64, i64]
            L.or_sign.restype = i32; L.or_sign.argtypes = [vp, u64]
            L.or_sketch.restype = None
            L.or_sketch.argtypes = [i64, i32, vp, i64, vp, i32, i64, vp, vp, vp, i32, i32, vp, vp]
            L.or_tuple_hash.restype = None
            L.or_tuple_hash.argtypes = [i32, vp, i32, i64, vp, vp, vp, i32, i32, vp, vp, vp]
            L.or_correlate_i64.restype = None
            L.or_correlate_i64.argtypes = [vp, vp, i64, i64, i64, vp]
            L.or_correlate_i256.restype = None
            L.or_correlate_i256.argtypes = [vp, vp, i64, i64, i64, vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# query graph (Section 2.6 notation; Section 3.2 initialisation)
# --------------------------------------------------------------------------

class QueryError(ValueError):
    """Invalid query graph; .code is one of INVALID, SELF_EDGE, CYCLIC, DISCONNECTED."""

    def __init__(self, code: str, msg: str):
        super().__init__(f"{code}: {msg}")
        self.code = code


@dataclasses.dataclass
class Query:
    num_join_attrs: List[int]          # |Omega(R_k)|
    offsets: List[int]                 # global id of attribute 0 of R_k
    rel_of: List[int]                  # relation of each global attribute
    edges: List[Tuple[int, int]]       # joins {u, v}, u < v, sorted
    comp_of: List[int]                 # Psi(u)
    n_comp: int
    gamma: List[List[int]]             # Gamma(u), sorted
    incident: List[List[int]]          # indices of the edges {u, v}, sorted

    @property
    def r(self) -> int:
        return len(self.num_join_attrs)

    @property
    def w(self) -> int:
        return len(self.rel_of)

    def omega(self, k: int) -> List[int]:
        return list(range(self.offsets[k], self.offsets[k] + self.num_join_attrs[k]))

    def attr(self, k: int, a: int) -> int:
        return self.offsets[k] + a

    def attr_plan(self, k: int):
        """(attr_comp, attr_edge_off, attr_edges) int32 arrays for relation k."""
        us = self.omega(k)
        comp = np.array([self.comp_of[u] for u in us], dtype=np.int32)
        off = [0]
        lst: List[int] = []
        for u in us:
            lst.extend(self.incident[u])
            off.append(len(lst))
        return comp, np.array(off, dtype=np.int32), np.array(lst if lst else [0], dtype=np.int32)


def canonical_query(num_join_attrs: Sequence[int], edges: Sequence[Tuple[int, int, int, int]]) -> Query:
    """Attributes are (relation, attribute) pairs numbered relation-major; a join
    {u, v} is stored with u < v and the list is sorted.  Components Psi are the
    connected components of the attribute graph, numbered in order of their
    smallest attribute.  The query must be acyclic (Section 2.6: joins are
    non-cyclic, a self-join uses a fictitious copy) and connected: its
    relations joined by its edges form a tree, so |E| = r - 1."""
    r = len(num_join_attrs)
    if r < 2:
        raise QueryError("INVALID", "a join query needs at least two relations")
    if any(int(a) < 1 for a in num_join_attrs):
        raise QueryError("INVALID", "every relation needs at least one joined attribute")
    offsets = [0]
    for a in num_join_attrs:
        offsets.append(offsets[-1] + int(a))
    w = offsets[-1]
    rel_of = [k for k in range(r) for _ in range(int(num_join_attrs[k]))]
    es = set()
    for (ra, aa, rb, ab) in edges:
        if not (0 <= ra < r and 0 <= rb < r and 0 <= aa < num_join_attrs[ra] and 0 <= ab < num_join_attrs[rb]):
            raise QueryError("INVALID", f"edge {(ra, aa, rb, ab)} out of range")
        if ra == rb:
            raise QueryError("SELF_EDGE", f"edge {(ra, aa, rb, ab)} joins a relation with itself")
        u, v = offsets[ra] + aa, offsets[rb] + ab
        e = (min(u, v), max(u, v))
        if e in es:
            raise QueryError("INVALID", f"duplicate edge {e}")
        es.add(e)
    elist = sorted(es)
    # relation-level tree check
    parent = list(range(r))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for (u, v) in elist:
        a, b = find(rel_of[u]), find(rel_of[v])
        if a == b:
            raise QueryError("CYCLIC", f"join {(u, v)} closes a cycle")
        parent[a] = b
    if len({find(k) for k in range(r)}) != 1:
        raise QueryError("DISCONNECTED", "the join graph is not connected")
    gamma: List[List[int]] = [[] for _ in range(w)]
    incident: List[List[int]] = [[] for _ in range(w)]
    for idx, (u, v) in enumerate(elist):
        gamma[u].append(v)
        gamma[v].append(u)
        incident[u].append(idx)
        incident[v].append(idx)
    for u in range(w):
        if not gamma[u]:
            raise QueryError("INVALID", f"attribute {u} takes part in no join")
        gamma[u].sort()
    # components of the attribute graph, numbered by smallest member
    comp_of = [-1] * w
    n_comp = 0
    for s in range(w):
        if comp_of[s] >= 0:
            continue
        stack = [s]
        comp_of[s] = n_comp
        while stack:
            x = stack.pop()
            for y in gamma[x]:
                if comp_of[y] < 0:
                    comp_of[y] = n_comp
                    stack.append(y)
        n_comp += 1
    return Query([int(a) for a in num_join_attrs], offsets[:-1], rel_of, elist, comp_of, n_comp, gamma, incident)


# --------------------------------------------------------------------------
# hash functions (Algorithm 1: SampleSignHashes, SampleBinHashes)
# --------------------------------------------------------------------------

def splitmix64(state: int) -> Tuple[int, int]:
    """One SplitMix64 step (Steele, Lea and Flood, OOPSLA 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def draw_coefficients(seed: int, d: int, n_comp: int, n_edges: int) -> np.ndarray:
    """uint64 [d][2*n_comp + 4*n_edges]: per median row, (b0, b1) for each component's bin
    function, then (s0, s1, s2, s3) for each join's sign function; each an element of
    GF(2^61 - 1) drawn as the top 61 bits of a SplitMix64 output, 2^61 - 1 rejected."""
    st = int(seed) & MASK64
    out = np.zeros((d, 2 * n_comp + 4 * n_edges), dtype=np.uint64)
    for row in range(d):
        for c in range(out.shape[1]):
            while True:
                st, z = splitmix64(st)
                v = z >> 3
                if v != P61:
                    break
            out[row, c] = v
    return out


def identity_coefficients(q: Query, d: int, radices: Sequence[int]) -> np.ndarray:
    """Test-only hash functions: bin h_q(x) = x * R_q (R_q = product of the domains of the
    earlier components) and sign s = +1.  With every key below its domain and m at least
    the product of all domains, each relation's sketch is an injective histogram and the
    estimate equals the exact join size."""
    out = np.zeros((d, 2 * q.n_comp + 4 * len(q.edges)), dtype=np.uint64)
    rad = 1
    for c in range(q.n_comp):
        out[:, 2 * c + 1] = rad
        rad *= int(radices[c])
    return out


# --------------------------------------------------------------------------
# Algorithm 2 / Eq. 4
# --------------------------------------------------------------------------

def field(key: int) -> int:
    return int(lib().or_field(int(key)))


def poly(coeffs: Sequence[int], x: int) -> int:
    c = np.asarray(coeffs, dtype=np.uint64)
    return int(lib().or_poly(_ptr(c), len(c), int(x)))


def tuple_hash(q: Query, coeffs: np.ndarray, k: int, keys: Sequence[int], m: int):
    """(bins int64[d], signs int32[d]) of one tuple of relation k (Eqs. 2-3)."""
    d = coeffs.shape[0]
    comp, off, lst = q.attr_plan(k)
    kk = np.ascontiguousarray(np.asarray(keys, dtype=np.int64))
    bins = np.zeros(d, dtype=np.int64)
    signs = np.zeros(d, dtype=np.int32)
    co = np.ascontiguousarray(coeffs, dtype=np.uint64)
    lib().or_tuple_hash(len(kk), _ptr(kk), d, m, _ptr(comp), _ptr(off), _ptr(lst), q.n_comp, len(q.edges),
                        _ptr(co), _ptr(bins), _ptr(signs))
    return bins, signs


def sketch_relation(q: Query, coeffs: np.ndarray, k: int, cols: np.ndarray, weights: Optional[np.ndarray],
                    m: int, threads: int = 1) -> np.ndarray:
    """int64 [d][m] sketch of relation k over the tuples cols[:, i] (Algorithm 2).  With
    threads > 1 the tuples are split into chunks whose partial sketches are added,
    which gives the same counters because sketches are linear (Section 2.2)."""
    d = coeffs.shape[0]
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    a_k, n = cols.shape
    assert a_k == q.num_join_attrs[k]
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.int64)
    comp, off, lst = q.attr_plan(k)
    co = np.ascontiguousarray(coeffs, dtype=np.uint64)
    L = lib()

    def run(i0: int, i1: int) -> np.ndarray:
        out = np.zeros((d, m), dtype=np.int64)
        if i1 > i0:
            sub = np.ascontiguousarray(cols[:, i0:i1])
            wp = None if w is None else _ptr(w[i0:i1])
            L.or_sketch(i1 - i0, a_k, _ptr(sub), i1 - i0, wp, d, m, _ptr(comp), _ptr(off), _ptr(lst),
                        q.n_comp, len(q.edges), _ptr(co), _ptr(out))
        return out

    if threads <= 1 or n < 4096:
        return run(0, n)
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda t: run(int(bounds[t]), int(bounds[t + 1])), range(threads)))
    acc = np.zeros((d, m), dtype=np.uint64)
    for p in parts:
        acc += p.view(np.uint64)
    return acc.view(np.int64)


def sketch_from_hashes(bins: Sequence[int], signs: Sequence[int], weights: Sequence[int], m: int) -> List[int]:
    """Eq. 4 with the per-tuple bin H and sign S given: c_j = sum over tuples with H = j of S * Delta."""
    c = [0] * m
    for b, s, w in zip(bins, signs, weights):
        c[int(b) % m] += int(s) * int(w)
    return c


# --------------------------------------------------------------------------
# Definition 3.1 and Algorithm 3
# --------------------------------------------------------------------------

def _to_i256(v: Sequence[int]) -> np.ndarray:
    out = np.zeros((len(v), 4), dtype=np.uint64)
    for i, x in enumerate(v):
        x &= (1 << 256) - 1
        out[i, 0] = x & MASK64
        out[i, 1] = (x >> 64) & MASK64
        out[i, 2] = (x >> 128) & MASK64
        out[i, 3] = (x >> 192) & MASK64
    return out


def _from_words(w: np.ndarray, bits: int) -> List[int]:
    res = []
    half = 1 << (bits - 1)
    full = 1 << bits
    for row in w.tolist():
        x = 0
        for k, word in enumerate(row):
            x |= int(word) << (64 * k)
        res.append(x - full if x >= half else x)
    return res


def correlate(a: Sequence[int], x: Sequence[int], threads: int = 0,
              bins: Optional[Sequence[int]] = None) -> List[int]:
    """Circular cross-correlation of Definition 3.1 for real integer vectors:
    z_j = sum_i a_i * x_{(j+i) mod m}, by the direct double sum, exactly.
    `bins` restricts the output to those j (returned in that order)."""
    m = len(a)
    assert len(x) == m
    js = list(range(m)) if bins is None else [int(j) for j in bins]
    if m == 0:
        return []
    ma = max(abs(int(v)) for v in a)
    mx = max(abs(int(v)) for v in x)
    bound = ma * mx * m
    if bound >= 1 << 255:
        raise OverflowError("correlation result may exceed the signed 256-bit range")
    small = ma < (1 << 63) and mx < (1 << 63) and bound < (1 << 126)
    L = lib()
    if small:
        A = np.asarray([int(v) for v in a], dtype=np.int64)
        X = np.asarray([int(v) for v in x], dtype=np.int64)
        words = 2
    else:
        A = _to_i256(a)
        X = _to_i256(x)
        words = 4
    nthreads = threads or (os.cpu_count() or 1)

    # contiguous runs of requested bins
    runs: List[Tuple[int, int]] = []
    for j in js:
        if runs and runs[-1][1] == j:
            runs[-1] = (runs[-1][0], j + 1)
        else:
            runs.append((j, j + 1))
    # split long runs for threads
    work: List[Tuple[int, int]] = []
    chunk = max(1, (len(js) + nthreads * 4 - 1) // (nthreads * 4))
    for (s, e) in runs:
        for t in range(s, e, chunk):
            work.append((t, min(e, t + chunk)))

    def run(se):
        s, e = se
        z = np.zeros((e - s, words), dtype=np.uint64)
        if small:
            L.or_correlate_i64(_ptr(A), _ptr(X), m, s, e, _ptr(z))
        else:
            L.or_correlate_i256(_ptr(A), _ptr(X), m, s, e, _ptr(z))
        return s, z

    if nthreads > 1 and len(work) > 1 and m * len(js) > (1 << 22):
        with ThreadPoolExecutor(nthreads) as ex:
            parts = list(ex.map(run, work))
    else:
        parts = [run(w) for w in work]
    val: Dict[int, int] = {}
    for s, z in parts:
        for off, v in enumerate(_from_words(z, 64 * words)):
            val[s + off] = v
    return [val[j] for j in js]


def hadamard(x: Sequence[int], y: Sequence[int]) -> List[int]:
    return [int(a) * int(b) for a, b in zip(x, y)]


def estimate_row(q: Query, sketches: Sequence[Sequence[int]], root: int = 0, threads: int = 0,
                 trace: Optional[list] = None) -> int:
    """Algorithm 3 for one median row.  sketches[k] is relation k's counter vector.
    root is the global id of the root attribute o (the paper picks any joined attribute).
    Every step is exact: Hadamard products and sums of Python integers, and
    correlations by the direct sum of Definition 3.1, so
    IFFT(conj(FFT(a)) o FFT(x)) is represented by its exact value a * x (star)."""
    m = len(sketches[0])
    visited = set()

    def combine(u: int) -> List[int]:
        k = q.rel_of[u]
        x = [int(v) for v in sketches[k]]
        visited.add(u)
        for u2 in q.omega(k):
            if u2 == u:
                continue
            visited.add(u2)
            a = [1] * m
            for v in q.gamma[u2]:
                a = hadamard(combine(v), a)
            x = correlate(a, x, threads)
            if trace is not None:
                trace.append(("corr", u2, list(x)))
        for v in q.gamma[u]:
            if v in visited:
                continue
            x = hadamard(combine(v), x)
        return x

    return sum(combine(root))


def brute_force_row(q: Query, sketches: Sequence[Sequence[int]]) -> int:
    """Eq. 5: X = sum over j in [m]^(#components) of prod_k c_k[G_k(j)], with
    G_k(j) = (sum_{u in Omega(R_k)} j_{Psi(u)}) mod m.  Exponential; tiny m only."""
    m = len(sketches[0])
    total = 0
    for j in itertools.product(range(m), repeat=q.n_comp):
        prod = 1
        for k in range(q.r):
            g = sum(j[q.comp_of[u]] for u in q.omega(k)) % m
            prod *= int(sketches[k][g])
            if prod == 0:
                break
        total += prod
    return total


def median_lower(values: Sequence[int]) -> int:
    """Lower median sorted[(l-1)//2] of the l row estimates (an integer for every l)."""
    s = sorted(int(v) for v in values)
    return s[(len(s) - 1) // 2]


def mid_mean(values: Sequence[int]) -> float:
    """Mean of the two middle values (the middle value when l is odd)."""
    s = sorted(int(v) for v in values)
    n = len(s)
    return float(s[n // 2]) if n % 2 else (s[n // 2 - 1] + s[n // 2]) / 2.0


@dataclasses.dataclass
class Estimate:
    rows: List[int]
    median: int
    mid_mean: float


def sketch_all(q: Query, coeffs: np.ndarray, relations, m: int, threads: int = 1) -> List[np.ndarray]:
    """int64 [d][m] sketch of every relation; relations[k] = (cols [a][n], weights or None)."""
    return [sketch_relation(q, coeffs, k, np.asarray(c), None if w is None else np.asarray(w), m, threads)
            for k, (c, w) in enumerate(relations)]


def estimate(q: Query, sketches: Sequence[np.ndarray], root: int = 0, threads: int = 0,
             rows: Optional[Sequence[int]] = None) -> Estimate:
    """Median over rows of the Algorithm 3 estimates; sketches[k] is int64 [d][m]."""
    d = sketches[0].shape[0]
    rr = list(range(d)) if rows is None else list(rows)
    vals = [estimate_row(q, [s[row].tolist() for s in sketches], root, threads) for row in rr]
    return Estimate(vals, median_lower(vals), mid_mean(vals))


# --------------------------------------------------------------------------
# sub-queries of one query (Section 3.4: plan enumeration)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SubQuery:
    """One sub-query S of a query Q, given by a subset of Q's joins.

    query      S in canonical numbering (canonical_query of its own relations/joins)
    relations  the Q relation behind each S relation, ascending
    keep       for each S relation, the attribute positions of its Q relation that S joins,
               ascending (the columns an S relation's batch is made of)
    coeffs     uint64 [d][2 * n_comp(S) + 4 * |E(S)|] in S's layout
    """
    query: Query
    relations: List[int]
    keep: List[List[int]]
    coeffs: np.ndarray


def subquery(num_join_attrs: Sequence[int], edges: Sequence[Tuple[int, int, int, int]], coeffs: np.ndarray,
             chosen: Sequence[int]) -> SubQuery:
    """The sub-query S of Q = (num_join_attrs, edges) made of the joins edges[i], i in chosen,
    with hash functions inherited from Q's coefficients (the reading taken for the sketch
    reuse of Section 3.4):
      - each component of S takes the bin function of the component of Q containing it;
      - a component of S with one join takes the sign function of the first join (lowest
        canonical index) of the component of Q containing it; a component of S with two or
        more joins takes, for each of its joins, the sign function Q gives that join.
    In Figure 3, the two-way sub-queries {0, 1} and {1, 3} then sketch relation R1 (its
    attribute 1) identically, which is the reuse the paper describes.  Because Q's relations
    form a tree, a connected S has at most one component inside any component of Q, so the
    functions S uses for different joins stay independent and Theorem 3.1 applies to S."""
    q = canonical_query(num_join_attrs, edges)
    picked = [tuple(int(v) for v in edges[i]) for i in sorted(set(int(i) for i in chosen))]
    if not picked:
        raise QueryError("INVALID", "a sub-query needs at least one join")
    rels = sorted({e[0] for e in picked} | {e[2] for e in picked})
    rel_new = {k: i for i, k in enumerate(rels)}
    keep = [sorted({e[1] for e in picked if e[0] == k} | {e[3] for e in picked if e[2] == k}) for k in rels]
    attr_new = {(k, a): j for k, ks in zip(rels, keep) for j, a in enumerate(ks)}
    sub_edges = [(rel_new[ra], attr_new[(ra, aa)], rel_new[rb], attr_new[(rb, ab)]) for (ra, aa, rb, ab) in picked]
    qs = canonical_query([len(ks) for ks in keep], sub_edges)
    # global attribute of S -> global attribute of Q
    to_q = [q.attr(rels[qs.rel_of[us]], keep[qs.rel_of[us]][us - qs.offsets[qs.rel_of[us]]]) for us in range(qs.w)]
    # first join of every component of Q
    first_join = {}
    for jq, (u, v) in enumerate(q.edges):
        first_join.setdefault(q.comp_of[u], jq)
    joins_in_comp = [0] * qs.n_comp
    for (us, vs) in qs.edges:
        joins_in_comp[qs.comp_of[us]] += 1
    d = coeffs.shape[0]
    out = np.zeros((d, 2 * qs.n_comp + 4 * len(qs.edges)), dtype=np.uint64)
    for c in range(qs.n_comp):
        us = next(u for u in range(qs.w) if qs.comp_of[u] == c)
        cq = q.comp_of[to_q[us]]
        out[:, 2 * c:2 * c + 2] = coeffs[:, 2 * cq:2 * cq + 2]
    for j, (us, vs) in enumerate(qs.edges):
        u, v = to_q[us], to_q[vs]
        if joins_in_comp[qs.comp_of[us]] == 1:
            jq = first_join[q.comp_of[u]]
        else:
            jq = q.edges.index((min(u, v), max(u, v)))
        out[:, 2 * qs.n_comp + 4 * j:2 * qs.n_comp + 4 * j + 4] = \
            coeffs[:, 2 * q.n_comp + 4 * jq:2 * q.n_comp + 4 * jq + 4]
    return SubQuery(qs, rels, keep, out)


def subquery_relations(sq: SubQuery, relations) -> list:
    """The batches of S's relations: each keeps the columns of its Q relation that S joins."""
    return [(np.asarray(relations[k][0])[ks], relations[k][1]) for k, ks in zip(sq.relations, sq.keep)]


# --------------------------------------------------------------------------
# exact join size (the expectation of Theorem 3.1)
# --------------------------------------------------------------------------

def exact_join_size(q: Query, relations) -> int:
    """sum over tuple combinations of prod_k F_k(i) * prod_{u,v in E} 1(i_u = i_v),
    computed by aggregating along the relation tree from relation 0: each child
    relation sends to its parent, per join key, the total weight of its matching
    sub-joins.  relations[k] = (cols int64 [a][n], weights or None)."""
    r = q.r
    # relation tree adjacency: (k, attr_in_k, child, attr_in_child)
    adj: List[List[Tuple[int, int, int]]] = [[] for _ in range(r)]
    for (u, v) in q.edges:
        ku, kv = q.rel_of[u], q.rel_of[v]
        adj[ku].append((u - q.offsets[ku], kv, v - q.offsets[kv]))
        adj[kv].append((v - q.offsets[kv], ku, u - q.offsets[ku]))

    def tuple_values(k: int, parent: int) -> List[int]:
        cols = np.asarray(relations[k][0])
        w = relations[k][1]
        n = cols.shape[1]
        vals = [1] * n if w is None else [int(t) for t in np.asarray(w).tolist()]
        for (a, child, ca) in adj[k]:
            if child == parent:
                continue
            msg = message(child, k, ca)
            keys = cols[a].tolist()
            vals = [v * msg.get(key, 0) for v, key in zip(vals, keys)]
        return vals

    def message(k: int, parent: int, attr: int) -> Dict[int, int]:
        vals = tuple_values(k, parent)
        out: Dict[int, int] = {}
        for key, v in zip(np.asarray(relations[k][0])[attr].tolist(), vals):
            if v:
                out[key] = out.get(key, 0) + v
        return out

    return sum(tuple_values(0, -1))


def exact_join_size_nested(q: Query, relations) -> int:
    """The same quantity by nested loops over every tuple combination (tiny inputs only)."""
    tuples = []
    for (cols, w) in relations:
        cols = np.asarray(cols)
        n = cols.shape[1]
        ws = [1] * n if w is None else [int(t) for t in np.asarray(w).tolist()]
        tuples.append([(cols[:, i].tolist(), ws[i]) for i in range(n)])
    total = 0
    for combo in itertools.product(*tuples):
        ok = True
        for (u, v) in q.edges:
            ku, kv = q.rel_of[u], q.rel_of[v]
            if combo[ku][0][u - q.offsets[ku]] != combo[kv][0][v - q.offsets[kv]]:
                ok = False
                break
        if ok:
            prod = 1
            for (_, wt) in combo:
                prod *= wt
            total += prod
    return total
