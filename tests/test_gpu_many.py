"""sk_estimate_many: many sets in one call give exactly each set's own estimate (fused
sets grouped by width, the others concurrently on worker streams)."""
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


def _make(attrs, edges, m, d, seed, rels, estimator):
    s = pkg.SketchSet(attrs, edges, m, d, seed)
    s.set_estimator(estimator)
    for k, (cols, w) in enumerate(rels):
        s.update(k, torch.as_tensor(np.ascontiguousarray(cols)).cuda(),
                 None if w is None else torch.as_tensor(np.ascontiguousarray(w)).cuda())
    return s


def test_mixed_sets_equal_single_estimates():
    rng = random.Random(31)
    specs = []
    for i in range(18):
        pairwise = i % 3 != 2
        attrs, edges = random_tree_query(rng, rng.randint(2, 5), share_prob=0.0 if pairwise else 0.7)
        m = rng.choice([64, 1024, 1 << 14]) if i % 5 else rng.choice([777, 3000])
        est = ["fused", "fused", "fft64", "ntt"][i % 4]
        rels = random_relations(rng, attrs, 1500, 1 << rng.choice([6, 20]))
        specs.append((attrs, edges, m, rng.choice([1, 3, 5]), rng.randrange(1 << 60), rels, est))
    sets = [_make(*sp) for sp in specs]
    many = pkg.estimate_many(sets)
    for s, sp, e in zip(sets, specs, many):
        one = s.estimate()
        assert e["rows"] == one["rows"] and e["median"] == one["median"], sp[2:4] + (sp[6],)
    for sp, e in list(zip(specs, many))[:6]:
        attrs, edges, m, d, seed, rels, _ = sp
        q = O.canonical_query(attrs, edges)
        co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
        assert e["rows"] == O.estimate(q, O.sketch_all(q, co, rels, m)).rows
    for s in sets:
        s.close()


def test_group_of_star_sets():
    """40 star sets (one fused group per width) against their single estimates."""
    sets, rels_all = [], []
    for i in range(40):
        w = synth.star(n_fact=20_000, n_dim=2_000, k=3, domain=500, m=4096 if i % 2 else 1 << 16, d=7,
                       seed=100 + i)
        s = pkg.SketchSet(w.num_join_attrs, w.edges, w.m, w.d, w.hash_seed)
        s.set_estimator("fused")
        for k, rel in enumerate(w.relations):
            s.update(k, rel.cols.cuda())
        sets.append(s)
    many = pkg.estimate_many(sets)
    for s, e in zip(sets, many):
        assert e["limb_bits"] == 0 and e["rows"] == s.estimate()["rows"]
        s.set_estimator("fft64")
        assert e["rows"] == s.estimate()["rows"]
        s.close()


def test_errors_and_empty():
    assert pkg.estimate_many([]) == []
    s = _make([1, 1], [(0, 0, 1, 0)], 64, 3, 1,
              [(np.array([[1, 2, 3]], dtype=np.int64), None), (np.array([[2, 3]], dtype=np.int64), None)], "fused")
    with pytest.raises(pkg.SketchError):
        pkg.estimate_many([s, s])
    assert pkg.estimate_many([s])[0]["rows"] == s.estimate()["rows"]
    s.close()
