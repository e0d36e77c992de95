"""Pins of the oracle's estimator: Algorithm 3 against Eq. 5 by brute force, the
closed form printed for Figure 3's query, the Count-sketch inner product of
Section 2.4, exactness under injective (identity) hashing, Theorem 3.1's
expectation and variance bound, and the exact join size by nested loops."""
import json
import os
import random

import numpy as np
import pytest

import oracle as O
from tests._helpers import random_relations, random_tree_query

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_correlate_definition_cases():
    """Definition 3.1: a one-hot a = e_i shifts x: (e_i * x)_j = x_{(j+i) mod m}; the
    int64/int128 and the 256-bit paths agree; small cases match a float FFT (numpy)."""
    rng = random.Random(1)
    for m in [1, 2, 5, 8, 33]:
        x = [rng.randrange(-100, 100) for _ in range(m)]
        for i in range(m):
            e = [0] * m
            e[i] = 1
            assert O.correlate(e, x) == [x[(j + i) % m] for j in range(m)]
        a = [rng.randrange(-100, 100) for _ in range(m)]
        z = O.correlate(a, x)
        ref = np.real(np.fft.ifft(np.conj(np.fft.fft(a)) * np.fft.fft(x)))
        assert z == [int(round(v)) for v in ref]
        # force the 256-bit path by scaling one operand beyond int64
        big = [v * (1 << 70) for v in a]
        assert O.correlate(big, x) == [v * (1 << 70) for v in z]
        # sum identity: sum_j z_j = (sum a)(sum x)
        assert sum(z) == sum(a) * sum(x)
    assert O.correlate([3, 1, 4, 1], [1, 5, 9, 2], bins=[2, 0]) == [
        O.correlate([3, 1, 4, 1], [1, 5, 9, 2])[2], O.correlate([3, 1, 4, 1], [1, 5, 9, 2])[0]]


def test_fig3_closed_form_every_root():
    g = json.load(open(os.path.join(GOLD, "fig3.json")))
    q = O.canonical_query(g["num_join_attrs"], [tuple(e) for e in g["edges"]])
    comps = {}
    for u, c in enumerate(q.comp_of):
        comps.setdefault(c, []).append(u)
    assert sorted(comps.values()) == g["components"]
    assert q.omega(1) == g["omega_R1"] and q.gamma[1] == g["gamma_1"]
    rng = random.Random(2)
    for m in [1, 3, 4, 7]:
        c = [[rng.randrange(-9, 10) for _ in range(m)] for _ in range(4)]
        closed = sum(c[0][j0] * c[2][j0] * c[1][(j0 + j1) % m] * c[3][j1]
                     for j0 in range(m) for j1 in range(m))
        assert O.brute_force_row(q, c) == closed
        for root in range(q.w):
            assert O.estimate_row(q, c, root=root) == closed


def test_two_relations_is_count_sketch_inner_product():
    """With one join, Algorithm 3 reduces to the Count-sketch estimate <c0, c1> (Section 2.4)."""
    q = O.canonical_query([1, 1], [(0, 0, 1, 0)])
    rng = random.Random(3)
    for m in [1, 4, 16]:
        c0 = [rng.randrange(-50, 50) for _ in range(m)]
        c1 = [rng.randrange(-50, 50) for _ in range(m)]
        ip = sum(a * b for a, b in zip(c0, c1))
        assert O.estimate_row(q, [c0, c1]) == ip
        assert O.estimate_row(q, [c0, c1], root=1) == ip


def test_algorithm3_equals_eq5_on_random_tiny_queries():
    rng = random.Random(4)
    for trial in range(60):
        r = rng.randint(2, 5)
        attrs, edges = random_tree_query(rng, r)
        q = O.canonical_query(attrs, edges)
        m = rng.choice([1, 2, 3, 4, 5]) if q.n_comp >= 3 else rng.choice([2, 3, 5, 8])
        c = [[rng.randrange(-5, 6) for _ in range(m)] for _ in range(r)]
        bf = O.brute_force_row(q, c)
        for root in range(q.w):
            assert O.estimate_row(q, c, root=root) == bf, (attrs, edges, m, root)


def test_identity_hashing_gives_exact_join_size():
    """With injective test hashes (bin h_q(x) = x * R_q, sign +1, m >= product of domains)
    each sketch is the relation's histogram in mixed radix, and Eq. 5 counts exactly the
    matching tuple combinations: X equals the join size (Theorem 3.1 without noise)."""
    rng = random.Random(5)
    for trial in range(25):
        r = rng.randint(2, 4)
        attrs, edges = random_tree_query(rng, r)
        q = O.canonical_query(attrs, edges)
        dom = rng.choice([2, 3])
        m = dom ** q.n_comp
        if m > 81:
            continue
        rels = random_relations(rng, attrs, 6, dom)
        co = O.identity_coefficients(q, 2, [dom] * q.n_comp)
        sk = O.sketch_all(q, co, rels, m)
        truth = O.exact_join_size_nested(q, rels)
        assert O.exact_join_size(q, rels) == truth
        for row in range(2):
            assert O.estimate_row(q, [s[row].tolist() for s in sk]) == truth


def test_identity_hashing_chain3_shape():
    """The chain R1(A) - R2(A, B) - R3(B) with A, B on [0, 10): m = 100 identity hashing."""
    rng = random.Random(6)
    q = O.canonical_query([1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)])
    rels = random_relations(rng, [1, 2, 1], 200, 10, signed=False)
    co = O.identity_coefficients(q, 1, [10, 10])
    sk = O.sketch_all(q, co, rels, 100)
    assert O.estimate_row(q, [s[0].tolist() for s in sk]) == O.exact_join_size(q, rels)


def test_exact_join_size_nested_vs_aggregation():
    rng = random.Random(7)
    for trial in range(30):
        attrs, edges = random_tree_query(rng, rng.randint(2, 4))
        q = O.canonical_query(attrs, edges)
        rels = random_relations(rng, attrs, 5, 3)
        assert O.exact_join_size(q, rels) == O.exact_join_size_nested(q, rels)


def test_row_magnitude_bound():
    """For a tree query each tuple combination lands in at most one j of Eq. 5, so
    |X| <= prod_k sum_t |Delta_t| for every choice of hash functions."""
    rng = random.Random(8)
    for trial in range(30):
        attrs, edges = random_tree_query(rng, rng.randint(2, 4))
        q = O.canonical_query(attrs, edges)
        rels = random_relations(rng, attrs, 6, 5)
        m = rng.choice([2, 3, 4])
        co = O.draw_coefficients(trial, 3, q.n_comp, len(q.edges))
        sk = O.sketch_all(q, co, rels, m)
        bound = 1
        for (_, w) in rels:
            bound *= int(np.abs(w).sum())
        for row in range(3):
            assert abs(O.brute_force_row(q, [s[row].tolist() for s in sk])) <= bound


def test_median_lower():
    assert O.median_lower([5]) == 5
    assert O.median_lower([3, 1, 2]) == 2
    assert O.median_lower([4, 1, 3, 2]) == 2
    assert O.median_lower([10, -4, 7, 7, 0]) == 7
    assert O.mid_mean([4, 1, 3, 2]) == 2.5
    assert O.median_lower([-(1 << 200), 1 << 199, 5]) == 5


def test_query_validation():
    with pytest.raises(O.QueryError) as e:
        O.canonical_query([1, 1], [(0, 0, 0, 0)])
    assert e.value.code in ("SELF_EDGE", "INVALID")
    with pytest.raises(O.QueryError) as e:
        O.canonical_query([2, 2], [(0, 0, 1, 0), (0, 1, 1, 1)])
    assert e.value.code == "CYCLIC"
    with pytest.raises(O.QueryError) as e:
        O.canonical_query([1, 1, 1, 1], [(0, 0, 1, 0), (2, 0, 3, 0)])
    assert e.value.code == "DISCONNECTED"
    with pytest.raises(O.QueryError) as e:
        O.canonical_query([2, 1], [(0, 0, 1, 0)])
    assert e.value.code == "INVALID"
    with pytest.raises(O.QueryError) as e:
        O.canonical_query([2, 2], [(0, 1, 0, 0), (0, 0, 1, 0)])
    assert e.value.code == "SELF_EDGE"


@pytest.mark.parametrize("shape", ["chain", "star", "fig3"])
def test_unbiased_and_variance_bound(shape):
    """Theorem 3.1: E[X] is the join size and Var(X) <= (1/m) 3^(r-1) prod_k ||F_k||^2.
    Over 1000 independent hash draws (one row each) the sample mean is within 3
    standard errors of the exact join size and the sample variance stays below the
    bound (with 20% slack for sampling error of the variance)."""
    rng = random.Random({"chain": 11, "star": 12, "fig3": 13}[shape])
    if shape == "chain":
        attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    elif shape == "star":
        attrs, edges = [3, 1, 1, 1], [(0, 0, 1, 0), (0, 1, 2, 0), (0, 2, 3, 0)]
    else:
        attrs, edges = [1, 2, 1, 1], [(0, 0, 1, 0), (2, 0, 1, 0), (3, 0, 1, 1)]
    q = O.canonical_query(attrs, edges)
    rels = []
    for a in attrs:
        n = 30
        cols = np.array([[rng.choice([0, 0, 0, 1, 1, 2, 3, 4, 5]) for _ in range(n)] for _ in range(a)],
                        dtype=np.int64)
        rels.append((cols, None))
    truth = O.exact_join_size(q, rels)
    m = 8
    N = 1000
    co = O.draw_coefficients(20240229, N, q.n_comp, len(q.edges))
    sk = O.sketch_all(q, co, rels, m)
    xs = np.array([O.estimate_row(q, [s[i].tolist() for s in sk]) for i in range(N)], dtype=np.float64)
    mean, var = xs.mean(), xs.var(ddof=1)
    se = np.sqrt(var / N)
    assert abs(mean - truth) <= 3 * se, (mean, truth, se)
    norms = 1.0
    for (cols, _) in rels:
        _, counts = np.unique(cols.T, axis=0, return_counts=True)
        norms *= float((counts.astype(np.float64) ** 2).sum())
    bound = (1.0 / m) * 3 ** (q.r - 1) * norms
    assert var <= 1.2 * bound, (var, bound)


def test_correlation_evaluation_identity_mod_goldilocks():
    """The identity behind the GPU's evaluation certificate: for z = a star x (Definition 3.1)
    and an m-th root of unity w modulo q = 2^64 - 2^32 + 1, sum z_j w^j = A(1/w) X(w).  Checked
    on exact oracle correlations (operands beyond 2^64, negative values) at primitive roots
    w = (7^((q-1)/m))^r, r odd; changing one output by 1 breaks it."""
    q = (1 << 64) - (1 << 32) + 1
    rng = random.Random(2024)
    for m in [2, 8, 64, 256]:
        a = [rng.randrange(-(1 << 90), 1 << 90) for _ in range(m)]
        x = [rng.randrange(-(1 << 70), 1 << 70) for _ in range(m)]
        z = O.correlate(a, x)
        for _ in range(3):
            r = rng.randrange(m) | 1
            w = pow(pow(7, (q - 1) // m, q), r, q)
            assert pow(w, m, q) == 1 and (m == 1 or pow(w, m // 2, q) != 1)
            wi = pow(w, q - 2, q)
            lhs = sum(zj * pow(w, j, q) for j, zj in enumerate(z)) % q
            rhs = (sum(ai * pow(wi, i, q) for i, ai in enumerate(a)) * sum(xk * pow(w, k, q) for k, xk in enumerate(x))) % q
            assert lhs == rhs
            bad = list(z)
            bad[rng.randrange(m)] += 1
            assert sum(zj * pow(w, j, q) for j, zj in enumerate(bad)) % q != rhs
