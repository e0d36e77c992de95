"""Pins for the oracle's sub-queries (Section 3.4): the inherited hash functions, the
sketch reuse the paper describes for Figure 3, and Theorem 3.1 for sub-query estimates."""
import itertools
import random

import numpy as np
import pytest

import oracle as O
from tests._helpers import random_tree_query

FIG3_ATTRS, FIG3_EDGES = [1, 2, 1, 1], [(0, 0, 1, 0), (2, 0, 1, 0), (3, 0, 1, 1)]


def connected_subsets(attrs, edges):
    """Every non-empty subset of joins whose relations form one tree."""
    out = []
    for size in range(1, len(edges) + 1):
        for sub in itertools.combinations(range(len(edges)), size):
            rels = {edges[i][0] for i in sub} | {edges[i][2] for i in sub}
            parent = {k: k for k in rels}

            def find(x):
                while parent[x] != x:
                    x = parent[x]
                return x

            for i in sub:
                parent[find(edges[i][0])] = find(edges[i][2])
            if len({find(k) for k in rels}) == 1:
                out.append(list(sub))
    return out


def test_full_query_keeps_every_function():
    rng = random.Random(1)
    for _ in range(20):
        attrs, edges = random_tree_query(rng, rng.randint(2, 6), share_prob=0.5)
        q = O.canonical_query(attrs, edges)
        co = O.draw_coefficients(rng.randrange(1 << 60), 3, q.n_comp, len(q.edges))
        sq = O.subquery(attrs, edges, co, range(len(edges)))
        assert sq.relations == list(range(len(attrs)))
        assert sq.keep == [list(range(a)) for a in attrs]
        assert sq.query.edges == q.edges and sq.query.comp_of == q.comp_of
        assert np.array_equal(sq.coeffs, co)


def test_figure3_two_way_subqueries_share_the_sketch_of_attribute_1():
    """Section 3.4's example: deciding between joins {0, 1} and {1, 3} of Figure 3 reuses the
    sketch of attribute 1 (relation R1) for both."""
    q = O.canonical_query(FIG3_ATTRS, FIG3_EDGES)
    co = O.draw_coefficients(77, 5, q.n_comp, len(q.edges))
    rng = np.random.default_rng(0)
    r1 = rng.integers(0, 50, size=(2, 400)).astype(np.int64)
    w = rng.choice(np.array([-1, 1, 2], dtype=np.int64), size=400)
    s01 = O.subquery(FIG3_ATTRS, FIG3_EDGES, co, [0])     # R0.0 = R1.0
    s13 = O.subquery(FIG3_ATTRS, FIG3_EDGES, co, [1])     # R2.0 = R1.0
    assert s01.relations == [0, 1] and s13.relations == [1, 2]
    assert s01.keep[1] == [0] and s13.keep[0] == [0]
    a = O.sketch_relation(s01.query, s01.coeffs, 1, r1[[0]], w, 64)
    b = O.sketch_relation(s13.query, s13.coeffs, 0, r1[[0]], w, 64)
    assert np.array_equal(a, b)
    # ... but not with the full query, where R1's attribute 1 carries two independent signs
    full = O.sketch_relation(q, co, 1, r1, w, 64)
    three = O.subquery(FIG3_ATTRS, FIG3_EDGES, co, [0, 1])
    c = O.sketch_relation(three.query, three.coeffs, 1, r1[[0]], w, 64)
    assert not np.array_equal(a, c)
    assert not np.array_equal(full, a)


def _poly_bin(co_row, c, x, m):
    return O.poly([int(co_row[2 * c]), int(co_row[2 * c + 1])], O.field(x)) % m


def _poly_sign(co_row, n_comp, j, x):
    cs = [int(v) for v in co_row[2 * n_comp + 4 * j:2 * n_comp + 4 * j + 4]]
    return -1 if O.poly(cs, O.field(x)) & 1 else 1


def test_inherited_functions_evaluated_by_hand():
    """R1's sketch for sub-queries of Figure 3, rebuilt tuple by tuple from Q's coefficient
    table: bins from Q's component functions, signs from the functions the reading assigns
    (the component's first join for a one-join component, each join's own otherwise)."""
    q = O.canonical_query(FIG3_ATTRS, FIG3_EDGES)
    # Q's canonical joins: (0,1) #0, (1,3) #1, (2,4) #2; components {0,1,3} -> 0, {2,4} -> 1
    assert q.edges == [(0, 1), (1, 3), (2, 4)] and q.comp_of == [0, 0, 1, 0, 1]
    d, m = 4, 32
    co = O.draw_coefficients(99, d, q.n_comp, len(q.edges))
    rng = np.random.default_rng(1)
    cols = rng.integers(0, 1 << 40, size=(2, 60)).astype(np.int64)
    w = rng.integers(-3, 4, size=60).astype(np.int64)
    # sub-query, R1's kept columns, the Q join whose sign each kept attribute multiplies in
    cases = [([0], [0], [[0]]),               # {0,1}: attr 1 alone, one-join comp -> join #0
             ([1], [0], [[0]]),               # {1,3}: one-join comp -> first join #0
             ([0, 1], [0], [[0, 1]]),         # {0,1},{1,3}: two-join comp -> own joins
             ([2], [1], [[2]]),               # {2,4}
             ([1, 2], [0, 1], [[0], [2]]),    # {1,3},{2,4}: both one-join comps
             ([0, 1, 2], [0, 1], [[0, 1], [2]])]
    for chosen, keep, joins in cases:
        sq = O.subquery(FIG3_ATTRS, FIG3_EDGES, co, chosen)
        k1 = sq.relations.index(1)
        assert sq.keep[k1] == keep
        got = O.sketch_relation(sq.query, sq.coeffs, k1, cols[keep], w, m)
        for row in range(d):
            bins, signs = [], []
            for i in range(cols.shape[1]):
                b, s = 0, 1
                for t, a in enumerate(keep):
                    x = int(cols[a, i])
                    b += _poly_bin(co[row], q.comp_of[1 + a], x, m)
                    for j in joins[t]:
                        s *= _poly_sign(co[row], q.n_comp, j, x)
                bins.append(b % m)
                signs.append(s)
            assert got[row].tolist() == O.sketch_from_hashes(bins, signs, w.tolist(), m), (chosen, row)


@pytest.mark.parametrize("chosen", [[0], [1], [0, 1], [1, 2], [0, 2]])
def test_subquery_estimates_are_unbiased(chosen):
    """Theorem 3.1 for sub-queries estimated with inherited functions: over 800 independent
    draws of Q's functions (one row each), the mean sub-query estimate is within 3 standard
    errors of the sub-query's exact join size."""
    rng = random.Random(sum(chosen) * 7 + len(chosen))
    rels = []
    for a in FIG3_ATTRS:
        cols = np.array([[rng.choice([0, 0, 1, 1, 2, 3, 4]) for _ in range(25)] for _ in range(a)], dtype=np.int64)
        rels.append((cols, None))
    q = O.canonical_query(FIG3_ATTRS, FIG3_EDGES)
    N, m = 800, 8
    co = O.draw_coefficients(4242 + len(chosen), N, q.n_comp, len(q.edges))
    sq = O.subquery(FIG3_ATTRS, FIG3_EDGES, co, chosen)
    srels = O.subquery_relations(sq, rels)
    truth = O.exact_join_size(sq.query, srels)
    sk = O.sketch_all(sq.query, sq.coeffs, srels, m)
    xs = np.array([O.estimate_row(sq.query, [s[i].tolist() for s in sk]) for i in range(N)], dtype=np.float64)
    se = np.sqrt(xs.var(ddof=1) / N)
    assert truth > 0
    assert abs(xs.mean() - truth) <= 3 * se, (xs.mean(), truth, se)


def test_connected_subsets_of_figure3():
    subs = connected_subsets(FIG3_ATTRS, FIG3_EDGES)
    assert sorted(map(tuple, subs)) == [(0,), (0, 1), (0, 1, 2), (0, 2), (1,), (1, 2), (2,)]
    q = O.canonical_query(FIG3_ATTRS, FIG3_EDGES)
    co = O.draw_coefficients(5, 2, q.n_comp, len(q.edges))
    for sub in subs:
        sq = O.subquery(FIG3_ATTRS, FIG3_EDGES, co, sub)
        assert sq.query.r == len(sub) + 1
