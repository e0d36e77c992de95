"""CPU pins of the arithmetic facts the exact GPU forms rely on, checked against the
oracle's exact Algorithm 3 (no GPU):

- the row estimate of any tree query is bounded by the product of the relations' l1
  norms (correlation, Hadamard product and sum are l1-submultiplicative), which fixes the
  number of CRT primes of the fused estimator;
- for queries whose components all join two attributes, X = (1/m) sum_nu prod_k C_k(+-nu),
  and bounding all factors but two by ||c_k||_1 and the remaining pair by Cauchy-Schwarz
  and Parseval gives ||c_a||_2 ||c_b||_2 prod_{k != a, b} ||c_k||_1 for every pair a != b;
- the reduction mod m by a precomputed reciprocal, r = v - hi64(v floor((2^64-1)/m)) m
  followed by at most two subtractions of m, is exact for every 64-bit v;
- 16-bit counters biased by 2^15, two per 32-bit word and updated by wrapping 32-bit adds
  of delta (low half) or delta * 2^16 (high half), never interfere while every partial
  sum stays within +-32767.
"""
import math
import random

import numpy as np

import oracle as O
from tests._helpers import random_tree_query


def _l1(v):
    return sum(abs(int(x)) for x in v)


def _l2(v):
    return math.isqrt(sum(int(x) * int(x) for x in v)) + 1   # an upper bound of sqrt(sum x^2)


def _random_sketches(rng, r, m, big):
    hi = (1 << 40) if big else 9
    return [[rng.randint(-hi, hi) if rng.random() < 0.7 else 0 for _ in range(m)] for _ in range(r)]


def test_l1_bound_for_every_tree_query():
    """|X_row| <= prod_k ||c_k||_1 for random tree queries, including components of three or
    more attributes, at small and large counter magnitudes and several widths."""
    rng = random.Random(11)
    for trial in range(120):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5), share_prob=0.5)
        q = O.canonical_query(attrs, edges)
        m = rng.choice([1, 2, 3, 5, 8, 16])
        sk = _random_sketches(rng, q.r, m, trial % 3 == 0)
        x = O.estimate_row(q, sk)
        bound = 1
        for v in sk:
            bound *= _l1(v)
        assert abs(x) <= bound, (attrs, edges, m)


def test_pairwise_l2_refinement_for_every_pair():
    """Queries whose components all join two attributes (chains, stars and their mixes):
    |X_row| <= ||c_a||_2 ||c_b||_2 prod_{k != a, b} ||c_k||_1 for every pair of relations."""
    rng = random.Random(12)
    checked = 0
    for trial in range(200):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5), share_prob=0.0)
        q = O.canonical_query(attrs, edges)
        m = rng.choice([1, 2, 4, 7, 16])
        sk = _random_sketches(rng, q.r, m, trial % 3 == 0)
        x = abs(O.estimate_row(q, sk))
        l1 = [_l1(v) for v in sk]
        l2 = [_l2(v) for v in sk]
        for a in range(q.r):
            for b in range(a + 1, q.r):
                bound = l2[a] * l2[b]
                for k in range(q.r):
                    if k not in (a, b):
                        bound *= l1[k]
                assert x <= bound, (attrs, edges, m, a, b)
                checked += 1
    assert checked > 300


def test_pairwise_bound_is_attained_by_identical_relations():
    """Two identical relations joined on one attribute: X = ||c||_2^2, so the l2 bound is
    tight (the fused estimator's prime count must cover exactly this)."""
    rng = random.Random(13)
    q = O.canonical_query([1, 1], [(0, 0, 1, 0)])
    for m in (1, 4, 32):
        c = [rng.randint(-1000, 1000) for _ in range(m)]
        assert O.estimate_row(q, [c, c]) == sum(v * v for v in c)


def _mod_by_reciprocal(v, m):
    mrec = ((1 << 64) - 1) // m
    q = (v * mrec) >> 64
    assert v // m - 2 <= q <= v // m
    r = v - q * m
    if r >= m:
        r -= m
    if r >= m:
        r -= m
    return r


def test_reciprocal_reduction_is_exact():
    rng = random.Random(14)
    ms = [2, 3, 7, 1000, 77777, 999_983, 1_000_000, (1 << 31) - 1, (1 << 30) + 3, 65535]
    edges = [0, 1, (1 << 61) - 2, (1 << 61) - 1, (1 << 62), (1 << 63), (1 << 64) - 1]
    for m in ms:
        for v in edges + [rng.randrange(1 << 64) for _ in range(2000)] + [k * m + j for k in (1, 2**40)
                                                                          for j in (-1, 0, 1) if k * m + j >= 0]:
            assert _mod_by_reciprocal(v, m) == v % m, (v, m)


def test_biased_16bit_pairs_do_not_interfere():
    """Random update streams on one word holding two counters: wrapping 32-bit adds of
    delta or delta << 16 on the biased word leave each half equal to 2^15 plus its own
    sum, as long as no partial sum leaves [-32767, 32767]."""
    rng = random.Random(15)
    for trial in range(300):
        word = 0x80008000
        sums = [0, 0]
        limit = rng.choice([7, 300, 32767])
        for _ in range(rng.randint(1, 4000)):
            half = rng.randint(0, 1)
            delta = rng.randint(-3, 3)
            if abs(sums[half] + delta) > limit:
                continue
            sums[half] += delta
            word = (word + ((delta << (16 * half)) & 0xFFFFFFFF)) & 0xFFFFFFFF
            assert (word & 0xFFFF) - 32768 == sums[0] and (word >> 16) - 32768 == sums[1]
