"""The fused estimator (SK_ESTIMATOR_FUSED): for queries whose components all join two
attributes and power-of-two widths, X = (1/m) sum_nu prod_k C_k(+-nu) modulo CRT primes;
for other query shapes and widths, Algorithm 3's schedule modulo the same primes.  Rows
must equal the oracle's exact Algorithm 3 rows."""
import random

import numpy as np
import pytest
import torch

import oracle as O
import paper_2402_15953_gb300 as pkg
import synth
from tests._helpers import random_relations, random_tree_query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_15953_gb300 import build
    build.build()
    O.build()


def _estimate(attrs, edges, m, d, seed, rels, estimator):
    s = pkg.SketchSet(attrs, edges, m, d, seed)
    s.set_estimator(estimator)
    for k, (cols, w) in enumerate(rels):
        s.update(k, torch.as_tensor(np.ascontiguousarray(cols)).cuda(),
                 None if w is None else torch.as_tensor(np.ascontiguousarray(w)).cuda())
    e = s.estimate()
    s.close()
    return e


def _oracle_rows(attrs, edges, m, d, seed, rels):
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
    return O.estimate(q, O.sketch_all(q, co, rels, m)).rows


@pytest.mark.parametrize("m", [2, 4, 64, 1024, 1 << 14, 1 << 17])
def test_pairwise_queries_exact(m):
    """Random tree queries where every attribute is joined once (components of two), keys
    over small and wide domains, signed weights."""
    rng = random.Random(500 + m)
    for trial in range(4 if m <= 1024 else 2):
        attrs, edges = random_tree_query(rng, rng.randint(2, 6), share_prob=0.0)
        rels = random_relations(rng, attrs, 2000 if m <= 1024 else 800, 1 << rng.choice([4, 12, 40]))
        d = rng.choice([1, 3, 7])
        seed = rng.randrange(1 << 60)
        e = _estimate(attrs, edges, m, d, seed, rels, "fused")
        assert e["limb_bits"] == 0 and 1 <= e["max_limbs"] <= 9       # the fused path ran
        assert e["rows"] == _oracle_rows(attrs, edges, m, d, seed, rels), (m, trial)


def test_many_primes_for_large_weights():
    """A five-relation chain with weights up to 2^30 in magnitude: the bound needs most of
    the nine primes."""
    rng = random.Random(9)
    attrs, edges = [1, 2, 2, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0), (2, 1, 3, 0), (3, 1, 4, 0)]
    rels = []
    for a in attrs:
        n = 300
        cols = np.array([[rng.randrange(50) for _ in range(n)] for _ in range(a)], dtype=np.int64)
        w = np.array([rng.choice([-1, 1]) * rng.randrange(1, 1 << 30) for _ in range(n)], dtype=np.int64)
        rels.append((cols, w))
    e = _estimate(attrs, edges, 256, 5, 77, rels, "fused")
    assert e["max_limbs"] >= 6
    assert e["rows"] == _oracle_rows(attrs, edges, 256, 5, 77, rels)
    assert max(abs(v) for v in e["rows"]) > (1 << 64)


def test_schedule_modulo_primes_for_other_shapes_and_widths():
    """Components of three attributes (Figure 3's {0, 1, 3}) and widths that are not powers
    of two run Algorithm 3's schedule modulo the CRT primes (no limbs)."""
    rng = random.Random(4)
    attrs, edges = synth.fig3_query()
    rels = random_relations(rng, attrs, 1500, 64)
    e = _estimate(attrs, edges, 128, 5, 3, rels, "fused")
    assert e["limb_bits"] == 0 and e["max_limbs"] >= 1
    assert e["rows"] == _oracle_rows(attrs, edges, 128, 5, 3, rels)
    w = synth.chain3()
    rels = [(r.cols.numpy(), None) for r in w.relations]
    e = _estimate(w.num_join_attrs, w.edges, 1000, 5, 42, rels, "fused")
    assert e["limb_bits"] == 0
    assert e["rows"] == _oracle_rows(w.num_join_attrs, w.edges, 1000, 5, 42, rels)


@pytest.mark.parametrize("m", [2, 3, 12, 64, 777, 1000, 1024, 3000, 1 << 13, 1 << 14])
def test_shared_attribute_queries_exact(m):
    """Random tree queries where a relation's attribute often joins several others (so
    components span three or more relations), signed weights, over small and wide key
    domains: the schedule modulo the primes gives the oracle's rows."""
    rng = random.Random(700 + m)
    for trial in range(4 if m <= 1024 else 2):
        attrs, edges = random_tree_query(rng, rng.randint(3, 6), share_prob=0.7)
        rels = random_relations(rng, attrs, 600 if m <= 1024 else 1500, 1 << rng.choice([3, 10, 40]))
        d = rng.choice([1, 2, 5])
        seed = rng.randrange(1 << 60)
        e = _estimate(attrs, edges, m, d, seed, rels, "fused")
        assert e["limb_bits"] == 0, (m, trial)
        assert e["rows"] == _oracle_rows(attrs, edges, m, d, seed, rels), (m, trial, attrs, edges)


def test_shared_attribute_query_large_weights():
    """Figure 3's query with weights up to 2^30 in magnitude: most of the nine primes."""
    rng = random.Random(19)
    attrs, edges = synth.fig3_query()
    rels = []
    for a in attrs:
        n = 200
        cols = np.array([[rng.randrange(30) for _ in range(n)] for _ in range(a)], dtype=np.int64)
        w = np.array([rng.choice([-1, 1]) * rng.randrange(1, 1 << 30) for _ in range(n)], dtype=np.int64)
        rels.append((cols, w))
    for m in (256, 300):
        e = _estimate(attrs, edges, m, 3, 8, rels, "fused")
        assert e["limb_bits"] == 0 and e["max_limbs"] >= 5
        assert e["rows"] == _oracle_rows(attrs, edges, m, 3, 8, rels)


def test_width_one_million_fused():
    """m = 10^6 (Section 4.4's width): R1 with one tuple makes each row one output of the
    circular correlation of R3's and R2's sketches, which the oracle computes directly."""
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    n = 300_000
    r2 = torch.stack([synth.zipf_keys(n, 1.2, 1 << 20, 3), synth.zipf_keys(n, 1.2, 1 << 20, 4)])
    r3 = synth.zipf_keys(n, 1.2, 1 << 20, 5)[None, :].contiguous()
    m, d = 1_000_000, 3
    s = pkg.SketchSet(attrs, edges, m, d, 91)
    s.set_estimator("fused")
    s.update(0, torch.tensor([[777]], dtype=torch.int64, device="cuda"))
    s.update(1, r2.cuda())
    s.update(2, r3.cuda())
    est = s.estimate()
    assert est["limb_bits"] == 0
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(91, d, q.n_comp, len(q.edges))
    c2 = O.sketch_relation(q, co, 1, r2.numpy(), None, m, threads=16)
    c3 = O.sketch_relation(q, co, 2, r3.numpy(), None, m, threads=16)
    bins, signs = O.tuple_hash(q, co, 0, [777], m)
    for row in range(d):
        z = O.correlate(c3[row].tolist(), c2[row].tolist(), threads=16, bins=[int(bins[row])])[0]
        assert est["rows"][row] == int(signs[row]) * z
    s.set_estimator("ntt")
    assert s.estimate()["rows"] == est["rows"]
    s.close()


def test_star_and_chain8_full_size_match_fft64():
    """The headline star (F 1e8 x 5, m = 2^16, d = 9) at 2e7 fact rows and the 8-relation
    chain (8 x 1e7 rows, m = 2^20, d = 16): fused rows equal the certified FP64 rows."""
    for wl in (synth.star(n_fact=20_000_000, device="cuda"), synth.chain(device="cuda")):
        s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed)
        for k, rel in enumerate(wl.relations):
            s.update(k, rel.cols)
        a = s.estimate()
        s.set_estimator("fused")
        b = s.estimate()
        c = s.estimate()
        assert b["limb_bits"] == 0
        assert a["rows"] == b["rows"] == c["rows"] and a["median"] == b["median"]
        s.close()
        del wl
        torch.cuda.empty_cache()


def test_family_with_fused_estimator():
    """Sub-query families estimate each sub-query with the fused arithmetic where it
    applies (every two-way or chain sub-query of a chain)."""
    from tests.test_oracle_subquery import connected_subsets
    rng = random.Random(12)
    attrs, edges = [1, 2, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0), (2, 1, 3, 0)]
    rels = random_relations(rng, attrs, 2000, 200)
    subs = connected_subsets(attrs, edges)
    fam = pkg.SketchFamily(attrs, edges, subs, 512, 5, 99)
    for k, (cols, w) in enumerate(rels):
        fam.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda())
    ref = fam.estimate()
    fam.set_estimator("fused")
    got = fam.estimate()
    assert [e["rows"] for e in got] == [e["rows"] for e in ref]
    assert all(e["limb_bits"] == 0 for e in got)
    fam.close()


def test_widest_width_two_relations():
    """m = 2^22 (the largest estimator width), two relations: each row is the Count-sketch
    inner product of the two oracle sketches (Section 2.4)."""
    rng = np.random.default_rng(22)
    n = 100_000
    a = rng.integers(0, 5000, size=(1, n)).astype(np.int64)
    b = rng.integers(0, 5000, size=(1, n)).astype(np.int64)
    wa = rng.choice(np.array([-2, 1, 3], dtype=np.int64), size=n)
    attrs, edges, m, d = [1, 1], [(0, 0, 1, 0)], 1 << 22, 2
    e = _estimate(attrs, edges, m, d, 5, [(a, wa), (b, None)], "fused")
    assert e["limb_bits"] == 0
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(5, d, q.n_comp, len(q.edges))
    sa = O.sketch_relation(q, co, 0, a, wa, m, threads=16)
    sb = O.sketch_relation(q, co, 1, b, None, m, threads=16)
    assert e["rows"] == [int(np.dot(sa[r], sb[r])) for r in range(d)]


def test_eight_relation_chain_d64():
    """An 8-relation chain with d = 64 rows (the largest d) at m = 64."""
    wl = synth.chain(r=8, n=3000, domain=300, m=64, d=64, seed=3)
    rels = [(r.cols.numpy(), None) for r in wl.relations]
    e = _estimate(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed, rels, "fused")
    assert e["limb_bits"] == 0 and len(e["rows"]) == 64
    assert e["rows"] == _oracle_rows(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed, rels)


@pytest.mark.parametrize("m", [64, 4096])
def test_bound_is_tight_for_identical_relations(m):
    """Two identical relations joined on one attribute: both sketches are the same vector c,
    so each row is ||c||_2^2, exactly the l2 bound that sets the number of primes (weights
    near 2^57, counters far from int64 wrap-around, several primes).  Through one estimate
    and through sk_estimate_many."""
    rng = np.random.default_rng(m)
    n = 1000
    cols = rng.integers(0, 300, size=(1, n)).astype(np.int64)
    w = (rng.integers(1 << 55, 1 << 57, size=n) * rng.choice(np.array([-1, 1]), size=n)).astype(np.int64)
    attrs, edges, d = [1, 1], [(0, 0, 1, 0)], 4
    sets = []
    for seed in (5, 6):
        s = pkg.SketchSet(attrs, edges, m, d, seed)
        s.set_estimator("fused")
        for k in range(2):
            s.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda())
        sets.append(s)
    many = pkg.estimate_many(sets)
    q = O.canonical_query(attrs, edges)
    for s, seed, e in zip(sets, (5, 6), many):
        one = s.estimate()
        co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
        c = O.sketch_relation(q, co, 0, cols, w, m)
        want = [sum(int(v) * int(v) for v in c[r]) for r in range(d)]
        assert one["limb_bits"] == 0 and one["max_limbs"] >= 4
        assert one["rows"] == want and e["rows"] == want
        s.close()


@pytest.mark.parametrize("r,m", [(3, 4096), (6, 4096), (2, 2048), (5, 1024), (7, 4096)])
def test_small_width_single_launch_smem_edges(r, m):
    """The single-launch form for widths up to 4096 keeps a set's r sketches of one row in
    shared memory (r m 4 bytes, at most 96 KB): exactly 48 KB of dynamic shared memory beside
    the kernel's static reduction array (r = 3, m = 4096), the largest (r = 6), smaller ones,
    and r = 7 at m = 4096 (112 KB: the general fused path).  Star queries with r - 1 joins,
    rows equal to the oracle's."""
    rng = random.Random(17 * r + m)
    attrs = [r - 1] + [1] * (r - 1)
    edges = [(0, k, k + 1, 0) for k in range(r - 1)]
    rels = random_relations(rng, attrs, 3000, 1 << 12)
    d = 7
    seed = rng.randrange(1 << 60)
    e = _estimate(attrs, edges, m, d, seed, rels, "fused")
    assert e["limb_bits"] == 0 and 1 <= e["max_limbs"] <= 9
    assert e["rows"] == _oracle_rows(attrs, edges, m, d, seed, rels)


def test_small_width_rows_take_their_own_prime_counts():
    """The single-launch form bounds each row by itself: at m = 2, relation 1 holds two keys
    of weight +2^50 and -2^50, so in rows where they share a bin with the same sign its vector
    is zero (estimate 0, one prime) and elsewhere the row needs several primes.  Every row
    equals the oracle's, over seeds that produce both kinds of rows."""
    zero_rows = wide_rows = 0
    for seed in (11, 12, 13, 14):
        rng = random.Random(seed)
        x, z = 5, 9
        r1 = (np.array([[x, z]], dtype=np.int64), np.array([1 << 50, -(1 << 50)], dtype=np.int64))
        keys = [x] + [rng.randrange(40) for _ in range(199)]
        r2 = (np.array([keys], dtype=np.int64),
              np.array([rng.choice([-1, 1]) * rng.randrange(1, 1 << 40) for _ in keys], dtype=np.int64))
        rels = [r1, r2]
        e = _estimate([1, 1], [(0, 0, 1, 0)], 2, 9, seed, rels, "fused")
        assert e["limb_bits"] == 0
        assert e["rows"] == _oracle_rows([1, 1], [(0, 0, 1, 0)], 2, 9, seed, rels), seed
        zero_rows += sum(1 for v in e["rows"] if v == 0)
        wide_rows += sum(1 for v in e["rows"] if abs(v) > (1 << 62))
    assert zero_rows > 0 and wide_rows > 0
