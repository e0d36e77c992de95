"""Seeded synthetic inputs for the convolved Count-sketch method.

This module only draws keys and weights; it holds none of the method's
arithmetic (no hashing, no sketching, no estimation).  Both the CUDA path and
the CPU oracle consume what it produces, which is the only thing they share.

The paper evaluates on the IMDB / STATS databases (Section 4.1, Table 3),
which are not available here; skewed synthetic columns stand in for them.
Skew follows a Zipf law, the distribution family the paper fits to every
column of those databases (Figure 5): rank k in [1, N] has probability
proportional to k^(-s) and is emitted as the key k - 1, so key 0 is the most
frequent value.  Sampling is by inverse CDF (a float64 cumulative table and a
binary search).

Every generator takes an explicit seed and is deterministic for a given
(seed, device, torch version).  Large workloads are drawn on the GPU with a
seeded torch generator; small ones on the CPU.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch


# --------------------------------------------------------------------------
# primitive draws
# --------------------------------------------------------------------------

def _gen(seed: int, device: str) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFF_FFFF_FFFF_FFFF)
    return g


def sub_seed(seed: int, *parts: int) -> int:
    """A reproducible child seed for (seed, part...) -- plain mixing, no hashing of keys."""
    s = int(seed) & 0xFFFF_FFFF_FFFF_FFFF
    for p in parts:
        s = (s * 6364136223846793005 + 1442695040888963407 + int(p) * 0x9E37_79B9) & 0xFFFF_FFFF_FFFF_FFFF
    return s & 0x7FFF_FFFF_FFFF_FFFF


_CDF_CACHE: dict = {}


def zipf_cdf(s: float, n: int, device: str) -> torch.Tensor:
    key = (float(s), int(n), str(device))
    c = _CDF_CACHE.get(key)
    if c is None:
        # built on the CPU: a float64 cumulative sum on the GPU is not bit-reproducible
        # across runs, which would move a few sampled keys across bucket boundaries
        k = torch.arange(1, n + 1, dtype=torch.float64)
        w = k.pow(-float(s))
        c = torch.cumsum(w, 0)
        c = (c / c[-1]).to(device)
        if len(_CDF_CACHE) > 16:
            _CDF_CACHE.clear()
        _CDF_CACHE[key] = c
    return c


def zipf_keys(n: int, s: float, domain: int, seed: int, device: str = "cpu") -> torch.Tensor:
    """n int64 keys in [0, domain), P(key = k-1) proportional to k^(-s)."""
    if n == 0:
        return torch.empty(0, dtype=torch.int64, device=device)
    cdf = zipf_cdf(s, domain, device)
    u = torch.rand(n, dtype=torch.float64, generator=_gen(seed, device), device=device)
    idx = torch.searchsorted(cdf, u, right=True)
    return idx.clamp_(max=domain - 1).to(torch.int64)


def uniform_keys(n: int, lo: int, hi: int, seed: int, device: str = "cpu") -> torch.Tensor:
    """n int64 keys uniform on [lo, hi)."""
    return torch.randint(lo, hi, (n,), dtype=torch.int64, generator=_gen(seed, device), device=device)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Relation:
    """One relation stream: cols is int64 [a][n] (attribute-major), weights int64 [n] or None (Delta = 1)."""
    cols: torch.Tensor
    weights: Optional[torch.Tensor] = None

    @property
    def n(self) -> int:
        return int(self.cols.shape[1])

    @property
    def arity(self) -> int:
        return int(self.cols.shape[0])


@dataclasses.dataclass
class Workload:
    """A join query over r relations plus their tuple streams.

    num_join_attrs[k] = |Omega(R_k)|; edges are (rel_a, attr_a, rel_b, attr_b)
    joins.  m is the sketch width, d the number of median rows, hash_seed the
    seed the hash functions are drawn from.
    """
    name: str
    num_join_attrs: List[int]
    edges: List[Tuple[int, int, int, int]]
    m: int
    d: int
    hash_seed: int
    relations: List[Relation]
    domains: List[List[int]]

    @property
    def r(self) -> int:
        return len(self.num_join_attrs)

    @property
    def total_tuples(self) -> int:
        return sum(rel.n for rel in self.relations)

    def to(self, device: str) -> "Workload":
        rels = [Relation(rel.cols.to(device), None if rel.weights is None else rel.weights.to(device))
                for rel in self.relations]
        return dataclasses.replace(self, relations=rels)


def chain3(n: int = 10_000, m: int = 256, d: int = 5, seed: int = 42, device: str = "cpu",
           domain: int = 1000, zipf_s: float = 1.0) -> Workload:
    """Chain join R1(A) |x| R2(A,B) |x| R3(B): A uniform on [0, domain), B Zipf(zipf_s) on
    [0, domain), n rows each, unit weights."""
    a1 = uniform_keys(n, 0, domain, sub_seed(seed, 0, 0), device)
    a2 = uniform_keys(n, 0, domain, sub_seed(seed, 1, 0), device)
    b2 = zipf_keys(n, zipf_s, domain, sub_seed(seed, 1, 1), device)
    b3 = zipf_keys(n, zipf_s, domain, sub_seed(seed, 2, 0), device)
    rels = [Relation(a1[None, :]), Relation(torch.stack([a2, b2])), Relation(b3[None, :])]
    return Workload("chain3", [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)], m, d, seed, rels,
                    [[domain], [domain, domain], [domain]])


def star(n_fact: int = 100_000_000, n_dim: int = 1_000_000, k: int = 5, domain: int = 1_000_000,
         zipf_s: float = 1.1, m: int = 1 << 16, d: int = 9, seed: int = 42,
         device: str = "cpu") -> Workload:
    """Star join F(K1..Kk) |x| D_1(K1) ... D_k(Kk): F's columns Zipf(zipf_s) over [0, domain),
    each D_i uniform over [0, domain)."""
    fcols = torch.empty((k, n_fact), dtype=torch.int64, device=device)
    for i in range(k):
        fcols[i] = zipf_keys(n_fact, zipf_s, domain, sub_seed(seed, 0, i), device)
    rels = [Relation(fcols)]
    for i in range(k):
        rels.append(Relation(uniform_keys(n_dim, 0, domain, sub_seed(seed, 1 + i, 0), device)[None, :]))
    edges = [(0, i, 1 + i, 0) for i in range(k)]
    return Workload("star", [k] + [1] * k, edges, m, d, seed, rels,
                    [[domain] * k] + [[domain]] * k)


def chain(r: int = 8, n: int = 10_000_000, domain: int = 1_000_000, zipf_s: float = 1.2,
          m: int = 1 << 20, d: int = 16, seed: int = 42, device: str = "cpu") -> Workload:
    """Chain R_0(A_0) |x| R_1(A_0, A_1) |x| ... |x| R_{r-1}(A_{r-2}); every column Zipf."""
    rels = []
    attrs = []
    for k in range(r):
        a = 1 if k in (0, r - 1) else 2
        attrs.append(a)
        cols = torch.stack([zipf_keys(n, zipf_s, domain, sub_seed(seed, k, c), device) for c in range(a)])
        rels.append(Relation(cols))
    edges = []
    for k in range(r - 1):
        attr_a = 0 if k == 0 else 1
        edges.append((k, attr_a, k + 1, 0))
    return Workload(f"chain{r}", attrs, edges, m, d, seed, rels, [[domain] * a for a in attrs])


def fig3_query() -> Tuple[List[int], List[Tuple[int, int, int, int]]]:
    """The join graph of Figure 3: R0(0), R1(1,2), R2(3), R3(4) with joins 0=1, 3=1, 4=2."""
    return [1, 2, 1, 1], [(0, 0, 1, 0), (2, 0, 1, 0), (3, 0, 1, 1)]


def random_relation(n: int, domains: Sequence[int], seed: int, device: str = "cpu",
                    zipf_s: Optional[float] = None, signed: bool = False) -> Relation:
    """A relation with len(domains) columns; uniform keys, or Zipf when zipf_s is given.
    signed=True draws weights in {-3..3} \\ {0}."""
    cols = []
    for c, dom in enumerate(domains):
        if zipf_s is None:
            cols.append(uniform_keys(n, 0, dom, sub_seed(seed, c), device))
        else:
            cols.append(zipf_keys(n, zipf_s, dom, sub_seed(seed, c), device))
    cols_t = torch.stack(cols) if cols else torch.empty((0, n), dtype=torch.int64, device=device)
    w = None
    if signed:
        g = _gen(sub_seed(seed, 999), device)
        mag = torch.randint(1, 4, (n,), generator=g, device=device, dtype=torch.int64)
        sgn = torch.randint(0, 2, (n,), generator=g, device=device, dtype=torch.int64) * 2 - 1
        w = mag * sgn
    return Relation(cols_t, w)


def with_deletions(rel: Relation, frac: float, seed: int) -> Relation:
    """Turnstile stream: append deletions (Delta = -1) of a `frac` sample of earlier-inserted
    rows, each placed after its insert (Section 2.1, general turnstile)."""
    n = rel.n
    k = int(round(n * frac))
    dev = rel.cols.device
    g = _gen(seed, str(dev) if dev.type == "cpu" else "cuda")
    idx = torch.randperm(n, generator=g, device=dev)[:k]
    cols = torch.cat([rel.cols, rel.cols[:, idx]], dim=1)
    w0 = rel.weights if rel.weights is not None else torch.ones(n, dtype=torch.int64, device=dev)
    w = torch.cat([w0, -w0[idx]])
    return Relation(cols.contiguous(), w)


def lognormal_sizes(count: int, median: float, sigma: float, lo: int, hi: int, seed: int) -> List[int]:
    rng = np.random.default_rng(seed)
    x = rng.lognormal(math.log(median), sigma, size=count)
    return [int(v) for v in np.clip(np.round(x), lo, hi)]


@dataclasses.dataclass
class BatchedSet:
    """One sketch set of the batched workload: a star query whose relation 0 carries the
    stream (a join columns) and whose relations 1..a are one-attribute partners, so every
    column is hashed."""
    num_join_attrs: List[int]
    edges: List[Tuple[int, int, int, int]]
    m: int
    d: int
    hash_seed: int
    relation: Relation
    domains: Optional[List[int]] = None   # relation 0's key domain per column: keys in [0, dom)


def batched(count: int = 256, median_rows: float = 1e5, sigma: float = 1.5, min_rows: int = 1000,
            max_rows: int = 10_000_000, d: int = 7, log2m: Tuple[int, int] = (10, 18), delete_frac: float = 0.1,
            seed: int = 42, device: str = "cpu") -> List[BatchedSet]:
    """count relations, rows lognormal(median_rows, sigma) clipped to [min_rows, max_rows],
    1-4 int64 join columns each with Zipf s ~ U[0.8, 1.4] over a domain log-uniform in
    [1e4, 1e7], width m = 2^U{log2m}, d rows, weights +1 with a delete_frac share of
    earlier-inserted rows deleted (-1) after their insert."""
    rng = np.random.default_rng(seed)
    sizes = lognormal_sizes(count, median_rows, sigma, min_rows, max_rows, seed + 1)
    out = []
    for i in range(count):
        a = int(rng.integers(1, 5))
        n = sizes[i]
        n_ins = max(1, int(round(n / (1 + delete_frac))))
        cols = []
        cols_dom = []
        for c in range(a):
            s_exp = float(rng.uniform(0.8, 1.4))
            dom = int(round(10 ** rng.uniform(4, 7)))
            cols_dom.append(dom)
            cols.append(zipf_keys(n_ins, s_exp, dom, sub_seed(seed, i, c), device))
        rel = with_deletions(Relation(torch.stack(cols)), delete_frac, sub_seed(seed, i, 77))
        m = 1 << int(rng.integers(log2m[0], log2m[1] + 1))
        out.append(BatchedSet([a] + [1] * a, [(0, k, 1 + k, 0) for k in range(a)], m, d,
                              sub_seed(seed, i, 5), rel, cols_dom))
    return out
