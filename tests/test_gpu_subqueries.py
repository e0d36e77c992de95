"""Sub-query families (Section 3.4) through the C ABI against the oracle: every sub-query's
sketches bit-exact and estimates exact, shared sketches exactly where the oracle's
sketches coincide, and the full query identical to a plain sketch set."""
import random

import numpy as np
import pytest
import torch

import oracle as O
import paper_2402_15953_gb300 as pkg
from tests._helpers import random_tree_query
from tests.test_oracle_subquery import FIG3_ATTRS, FIG3_EDGES, connected_subsets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_15953_gb300 import build
    build.build()
    O.build()


def _relations(rng, attrs, n_max, domain, signed=True):
    rels = []
    for a in attrs:
        n = rng.randint(200, n_max)
        cols = np.array([[rng.randrange(domain) for _ in range(n)] for _ in range(a)], dtype=np.int64)
        w = np.array([rng.choice([-2, -1, 1, 1, 3]) for _ in range(n)], dtype=np.int64) if signed else None
        rels.append((cols, w))
    return rels


def _check_family(attrs, edges, subs, rels, m, d, seed, estimator="fft64"):
    fam = pkg.SketchFamily(attrs, edges, subs, m, d, seed)
    fam.set_estimator(estimator)
    for k, (cols, w) in enumerate(rels):
        fam.update(k, torch.as_tensor(cols).cuda(), None if w is None else torch.as_tensor(w).cuda())
    fam.sync()
    ests = fam.estimate()
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
    by_view = {}
    for i, sub in enumerate(subs):
        sq = O.subquery(attrs, edges, co, sub)
        srels = O.subquery_relations(sq, rels)
        sk = O.sketch_all(sq.query, sq.coeffs, srels, m)
        for ks in range(sq.query.r):
            qrel, view = fam.view(i, ks)
            assert qrel == sq.relations[ks]
            got = fam.sketch(i, ks)
            assert np.array_equal(got, sk[ks]), (sub, ks)
            by_view.setdefault(view, []).append(sk[ks])
        ref = O.estimate(sq.query, sk)
        assert ests[i]["rows"] == ref.rows, sub
        assert ests[i]["median"] == ref.median
    # a shared sketch is one sketch; distinct views hold distinct sketches (random data)
    for view, sks in by_view.items():
        assert all(np.array_equal(s, sks[0]) for s in sks)
    firsts = [sks[0] for sks in by_view.values()]
    for a in range(len(firsts)):
        for b in range(a + 1, len(firsts)):
            assert not np.array_equal(firsts[a], firsts[b])
    assert fam.info()["views"] == len(by_view)
    return fam, ests


@pytest.mark.parametrize("m", [64, 1000])
def test_figure3_all_connected_subqueries(m):
    rng = random.Random(m)
    rels = _relations(rng, FIG3_ATTRS, 3000, 40)
    subs = connected_subsets(FIG3_ATTRS, FIG3_EDGES)
    fam, ests = _check_family(FIG3_ATTRS, FIG3_EDGES, subs, rels, m, 5, 2024)
    # the paper's reuse: {0,1} and {1,3} share relation R1's sketch
    i01, i13 = subs.index([0]), subs.index([1])
    assert fam.view(i01, 1) == fam.view(i13, 0)
    # the full query equals a plain sketch set with the same seed
    full = subs.index([0, 1, 2])
    s = pkg.SketchSet(FIG3_ATTRS, FIG3_EDGES, m, 5, 2024)
    for k, (cols, w) in enumerate(rels):
        s.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda())
    assert s.estimate()["rows"] == ests[full]["rows"]
    for k in range(4):
        assert np.array_equal(s.counters[k].cpu().numpy(), fam.sketch(full, k))
    s.close()
    fam.close()


def test_random_tree_queries_and_both_estimators():
    rng = random.Random(77)
    for trial in range(5):
        attrs, edges = random_tree_query(rng, rng.randint(3, 6), share_prob=0.5)
        subs = connected_subsets(attrs, edges)
        rng.shuffle(subs)
        subs = subs[:12]
        rels = _relations(rng, attrs, 2000, 1 << rng.choice([5, 12, 40]))
        m = rng.choice([32, 256, 4096, 777])
        fam, e1 = _check_family(attrs, edges, subs, rels, m, 3, rng.randrange(1 << 60))
        fam.set_estimator("ntt")
        e2 = fam.estimate()
        assert [e["rows"] for e in e1] == [e["rows"] for e in e2]
        fam.close()


def test_family_linearity_reset_and_domains():
    rng = random.Random(5)
    rels = _relations(rng, FIG3_ATTRS, 1000, 30)
    subs = connected_subsets(FIG3_ATTRS, FIG3_EDGES)
    fam = pkg.SketchFamily(FIG3_ATTRS, FIG3_EDGES, subs, 128, 3, 9)
    for rep in range(2):
        for k, (cols, w) in enumerate(rels):
            fam.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda(), domain=[30] * cols.shape[0])
    fam.sync()
    twice = fam.estimate()
    fam.reset()
    for k, (cols, w) in enumerate(rels):
        ww = torch.as_tensor(2 * w).cuda()
        fam.update(k, torch.as_tensor(cols).cuda(), ww)
    doubled = fam.estimate()
    assert [e["rows"] for e in twice] == [e["rows"] for e in doubled]
    bad = torch.tensor([[5, 31, 7]], dtype=torch.int64, device="cuda")
    fam.update(0, bad, domain=[30])
    with pytest.raises(pkg.SketchError):
        fam.sync()
    fam.close()


def test_invalid_subqueries():
    for subs in ([[]], [[0, 0]], [[5]], [[-1]]):
        with pytest.raises(pkg.SketchError):
            pkg.SketchFamily(FIG3_ATTRS, FIG3_EDGES, subs, 64, 3, 1)
    # joins 0 (R0-R1) and 2 (R3-R1) are connected through R1; a chain's end joins are not
    attrs, edges = [1, 2, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0), (2, 1, 3, 0)]
    with pytest.raises(pkg.SketchError):
        pkg.SketchFamily(attrs, edges, [[0, 2]], 64, 3, 1)
    fam = pkg.SketchFamily(attrs, edges, [[0, 1], [1, 2]], 64, 3, 1)
    assert fam.info()["subqueries"] == 2
    fam.close()


def test_six_attribute_relation_and_view_limit():
    """A star whose fact relation joins 6 attributes (the update kernel's runtime-arity
    path), d = 13, sub-queries of one to six joins; then a 7-dimension star asking for all
    127 sub-queries, which gives the fact relation more views than SK_MAX_VIEWS allows."""
    rng = random.Random(21)
    k = 6
    attrs, edges = [k] + [1] * k, [(0, t, 1 + t, 0) for t in range(k)]
    subs = [[0], [5], [1, 2], [0, 3, 5], [1, 2, 3, 4], list(range(k))]
    rels = _relations(rng, attrs, 3000, 25)
    fam, _ = _check_family(attrs, edges, subs, rels, 512, 13, 31337)
    fam.close()
    k = 7
    attrs, edges = [k] + [1] * k, [(0, t, 1 + t, 0) for t in range(k)]
    subs = [s for s in connected_subsets(attrs, edges)]
    assert len(subs) == 127
    with pytest.raises(pkg.SketchError):
        pkg.SketchFamily(attrs, edges, subs, 64, 3, 1)
    fam = pkg.SketchFamily(attrs, edges, subs[:64], 64, 3, 1)
    assert fam.info()["subqueries"] == 64
    fam.close()


@pytest.mark.parametrize("m,n,doms,bad", [(1 << 13, 200_003, [5000, 7000, 30_000, 300], False),
                                          (1 << 16, 1_048_607, [5000, 70_000, 100_000, 300], True)])
def test_star_family_partitioned_views(m, n, doms, bad):
    """A 4-dimension star's family with declared key domains and unit weights: the fact
    relation's 15 views (one per non-empty subset of its joins; every attribute in one join)
    go through one key table and the two-phase partitioned update per view (table build,
    validity pass, two launches per view).  Every sub-query's sketches bit-exact against the oracle (the
    estimator, unchanged, is checked on these sketches elsewhere); with keys outside their
    domain, those tuples are skipped and reported."""
    import itertools
    import synth
    k = 4
    attrs, edges = [k] + [1] * k, [(0, i, 1 + i, 0) for i in range(k)]
    subs = [list(c) for size in range(1, k + 1) for c in itertools.combinations(range(k), size)]
    fcols = np.stack([synth.zipf_keys(n, 1.1, doms[u], 60 + u).numpy() for u in range(k)])
    if bad:
        fcols[1, 7] = doms[1]
        fcols[3, n - 1] = -4
    rng = np.random.default_rng(3)
    rels = [(fcols, None)] + [(rng.integers(0, doms[u], size=(1, 20_000)).astype(np.int64), None) for u in range(k)]
    fam = pkg.SketchFamily(attrs, edges, subs, m, 9, 21)
    fam.set_estimator("fused")
    L0 = pkg.sk_launch_count()
    fam.update(0, torch.as_tensor(fcols).cuda(), domain=doms)
    assert pkg.sk_launch_count() - L0 == 2 + 2 * len(subs)
    for kk in range(1, k + 1):
        fam.update(kk, torch.as_tensor(rels[kk][0]).cuda(), domain=[doms[kk - 1]])
    if bad:
        with pytest.raises(pkg.SketchError):
            fam.sync()
    fam.sync()
    keep = np.all((fcols >= 0) & (fcols < np.array(doms)[:, None]), axis=0)
    rels[0] = (fcols[:, keep], None)
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(21, 9, q.n_comp, len(q.edges))
    for i, sub in enumerate(subs):
        sq = O.subquery(attrs, edges, co, sub)
        sk = O.sketch_all(sq.query, sq.coeffs, O.subquery_relations(sq, rels), m, threads=16)
        for ks in range(sq.query.r):
            assert np.array_equal(fam.sketch(i, ks), sk[ks]), (sub, ks)
    fam.close()
