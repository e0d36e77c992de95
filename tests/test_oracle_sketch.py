"""Pins of the oracle's sketch creation (Algorithm 2, Eqs. 2-4) against the
worked example of Figure 4, the tensor-sketch identity of Section 2.5 and the
linearity of Section 2.2."""
import json
import os
import random

import numpy as np

import oracle as O
from tests._helpers import random_relations, random_tree_query

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _conv(x, y):
    """Definition 2.2, circular convolution."""
    m = len(x)
    return [sum(x[i] * y[(j - i) % m] for i in range(m)) for j in range(m)]


def test_fig4_worked_example():
    g = json.load(open(os.path.join(GOLD, "fig4.json")))
    m = g["m"]
    sa = O.sketch_from_hashes([g["a"]["bin"]], [g["a"]["sign"]], [1], m)
    sb = O.sketch_from_hashes([g["b"]["bin"]], [g["b"]["sign"]], [1], m)
    assert sa == g["sketch_a"] and sb == g["sketch_b"]
    assert O.hadamard(sa, sb) == g["hadamard"]
    assert _conv(sa, sb) == g["convolution"]
    # the tuple (a, b): bin = sum of bins mod m (Eq. 3), sign = product (Eq. 2)
    tup = O.sketch_from_hashes([(g["a"]["bin"] + g["b"]["bin"]) % m], [g["a"]["sign"] * g["b"]["sign"]], [1], m)
    assert tup == g["convolution"]


def test_single_tuple_is_convolution_of_one_hot_sketches():
    """Section 2.5 / Section 3.2: sketching a multi-attribute tuple equals the circular
    convolution of the single-attribute one-hot sketches of its values."""
    rng = random.Random(5)
    for trial in range(20):
        attrs, edges = random_tree_query(rng, rng.randint(2, 4))
        q = O.canonical_query(attrs, edges)
        m = rng.choice([3, 7, 8, 16])
        co = O.draw_coefficients(100 + trial, 2, q.n_comp, len(q.edges))
        k = max(range(q.r), key=lambda t: q.num_join_attrs[t])
        keys = [rng.randrange(-1000, 1000) for _ in range(q.num_join_attrs[k])]
        cols = np.array([[x] for x in keys], dtype=np.int64)
        sk = O.sketch_relation(q, co, k, cols, None, m)
        for row in range(2):
            acc = [1] + [0] * (m - 1)  # identity of circular convolution
            for ai, u in enumerate(q.omega(k)):
                xf = O.field(keys[ai])
                b = co[row, 2 * q.comp_of[u]: 2 * q.comp_of[u] + 2]
                h = O.lib().or_bin(np.ascontiguousarray(b).ctypes.data, xf, m)
                s = 1
                for e in q.incident[u]:
                    sc = np.ascontiguousarray(co[row, 2 * q.n_comp + 4 * e: 2 * q.n_comp + 4 * e + 4])
                    s *= O.lib().or_sign(sc.ctypes.data, xf)
                one_hot = [0] * m
                one_hot[h] = s
                acc = _conv(acc, one_hot)
            assert sk[row].tolist() == acc


def test_linearity_deletion_and_order():
    """Section 2.2: sketches are linear -- sk(R u S) = sk(R) + sk(S), a deletion
    (Delta = -1) cancels its insert, and tuple order does not matter."""
    rng = random.Random(6)
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(9, 3, q.n_comp, len(q.edges))
    m = 32
    n = 500
    cols = np.array([[rng.randrange(50) for _ in range(n)] for _ in range(2)], dtype=np.int64)
    w = np.array([rng.choice([-3, -1, 1, 2, 5]) for _ in range(n)], dtype=np.int64)
    full = O.sketch_relation(q, co, 1, cols, w, m)
    a = O.sketch_relation(q, co, 1, cols[:, :200], w[:200], m)
    b = O.sketch_relation(q, co, 1, cols[:, 200:], w[200:], m)
    assert (full == a + b).all()
    perm = np.array(rng.sample(range(n), n))
    assert (O.sketch_relation(q, co, 1, cols[:, perm], w[perm], m) == full).all()
    both = O.sketch_relation(q, co, 1, np.concatenate([cols, cols], 1), np.concatenate([w, -w]), m)
    assert not both.any()
    unit = O.sketch_relation(q, co, 1, cols, None, m)
    ones = O.sketch_relation(q, co, 1, cols, np.ones(n, dtype=np.int64), m)
    assert (unit == ones).all()
    # threads split the stream; linearity makes the result identical
    assert (O.sketch_relation(q, co, 1, np.tile(cols, 20), np.tile(w, 20), m, threads=4)
            == O.sketch_relation(q, co, 1, np.tile(cols, 20), np.tile(w, 20), m)).all()


def test_sketch_matches_per_tuple_hashes():
    """Eq. 4 written out: c_j = sum over tuples with H(i) = j of F(i) S(i)."""
    rng = random.Random(8)
    q = O.canonical_query(*random_tree_query(rng, 4))
    co = O.draw_coefficients(3, 4, q.n_comp, len(q.edges))
    m = 13
    for k in range(q.r):
        (cols, w), = random_relations(rng, [q.num_join_attrs[k]], 40, 30)
        sk = O.sketch_relation(q, co, k, cols, w, m)
        for row in range(4):
            bins, signs = [], []
            for i in range(cols.shape[1]):
                b, s = O.tuple_hash(q, co, k, cols[:, i].tolist(), m)
                bins.append(b[row])
                signs.append(s[row])
            assert sk[row].tolist() == O.sketch_from_hashes(bins, signs, w.tolist(), m)


def test_int64_wraparound():
    q = O.canonical_query([1, 1], [(0, 0, 1, 0)])
    co = O.draw_coefficients(1, 1, q.n_comp, len(q.edges))
    big = np.array([(1 << 62), (1 << 62), (1 << 62)], dtype=np.int64)
    cols = np.array([[5, 5, 5]], dtype=np.int64)
    sk = O.sketch_relation(q, co, 0, cols, big, 4)
    b, sg = O.tuple_hash(q, co, 0, [5], 4)
    exp = (3 * (1 << 62) * int(sg[0]) + (1 << 63)) % (1 << 64) - (1 << 63)
    assert int(sk[0][b[0]]) == exp
