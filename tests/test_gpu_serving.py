"""The serving loop: requests that run mixed and overlapped on the device give, for
every estimate, exactly the result of running that set's requests one by one, and that
result is the CPU oracle's Algorithm 3 over the updates of the set submitted before it."""
import random

import numpy as np
import pytest
import torch

import oracle as O
import paper_2402_15953_gb300 as pkg
from paper_2402_15953_gb300.serve import SketchServer
from tests._helpers import random_relations, random_tree_query

pytestmark = pytest.mark.gpu


def _trace(seed, n_sets=6, n_req=90):
    rng = random.Random(seed)
    sets = []
    for i in range(n_sets):
        attrs, edges = random_tree_query(rng, rng.randint(2, 4))
        sets.append((attrs, edges, 1 << rng.randint(6, 12), rng.choice([1, 3, 5]), rng.randrange(1 << 60)))
    reqs = []
    for j in range(n_req):
        sid = rng.randrange(n_sets)
        attrs = sets[sid][0]
        if rng.random() < 0.2:
            reqs.append(("estimate", sid))
        else:
            rel = rng.randrange(len(attrs))
            (cols, w), = random_relations(rng, [attrs[rel]], 3000, 1 << 20)
            reqs.append(("update", sid, rel, torch.as_tensor(cols).pin_memory(), torch.as_tensor(w).pin_memory()))
    for sid in range(n_sets):
        reqs.append(("estimate", sid))
    return sets, reqs


def _oracle_expected(sets, reqs):
    """Per estimate request j: the oracle's rows and lower median (Algorithm 3, Section 3.3)
    for the sketches of exactly the updates of its set submitted before it.  The oracle
    sketches each update batch itself (Algorithm 2, Eq. 4) and the batches of one relation
    add up (Eq. 4 is a sum over tuples)."""
    qs, cos, acc = [], [], []
    for (attrs, edges, m, d, seed) in sets:
        q = O.canonical_query(attrs, edges)
        qs.append(q)
        cos.append(O.draw_coefficients(seed, d, q.n_comp, len(q.edges)))
        acc.append([np.zeros((d, m), dtype=np.int64) for _ in attrs])
    out = {}
    for j, r in enumerate(reqs):
        if r[0] == "update":
            _, sid, rel, cols, w = r
            acc[sid][rel] += O.sketch_relation(qs[sid], cos[sid], rel, cols.numpy(), w.numpy(), sets[sid][2])
        else:
            out[j] = O.estimate(qs[r[1]], acc[r[1]])
    return out


def _alone(sets, reqs):
    """Each set's requests run one by one on a fresh set."""
    out = {}
    live = [pkg.SketchSet(a, e, m, d, s) for (a, e, m, d, s) in sets]
    for j, r in enumerate(reqs):
        if r[0] == "update":
            _, sid, rel, cols, w = r
            live[sid].update(rel, cols.cuda(), w.cuda())
        else:
            out[j] = live[r[1]].estimate()
    for s in live:
        s.close()
    return out


def _mixed(sets, reqs, budget=32 << 30, slots=8, workers=4):
    srv = SketchServer(hbm_budget_bytes=budget, update_slots=slots, estimate_workers=workers)
    for i, (a, e, m, d, s) in enumerate(sets):
        assert srv.register_set(i, a, e, m, d, s)
    handles = {}
    for j, r in enumerate(reqs):
        if r[0] == "update":
            _, sid, rel, cols, w = r
            srv.submit_update(sid, rel, cols, w)
        else:
            handles[j] = srv.submit_estimate(r[1])
    srv.serve()
    srv.close()
    return {j: h.result for j, h in handles.items()}, handles


@pytest.mark.parametrize("seed", [1, 2])
def test_results_equal_alone_in_the_mix_and_the_oracle(seed):
    sets, reqs = _trace(seed)
    ref = _oracle_expected(sets, reqs)
    alone = _alone(sets, reqs)
    mixed, handles = _mixed(sets, reqs)
    assert set(alone) == set(mixed) == set(ref)
    for j in alone:
        assert handles[j].error is None, handles[j].error
        assert mixed[j]["rows"] == alone[j]["rows"] == ref[j].rows, j
        assert mixed[j]["median"] == alone[j]["median"] == ref[j].median


def test_tight_budget_queues_but_stays_exact():
    sets, reqs = _trace(3, n_sets=4, n_req=40)
    resident = sum(len(a) * d * m * 8 for (a, e, m, d, s) in sets)
    est = max((max(2, len(a)) + 1) * d * m * 32 + 2 * d * 4 * m * 16 + (m // 2) * 16 for (a, e, m, d, s) in sets)
    budget = resident + est + 4 * 3000 * 8 * 2 + 4096
    ref = _oracle_expected(sets, reqs)
    alone = _alone(sets, reqs)
    mixed, handles = _mixed(sets, reqs, budget=budget, slots=2, workers=1)
    for j in alone:
        assert handles[j].error is None, handles[j].error
        assert mixed[j]["rows"] == alone[j]["rows"] == ref[j].rows
        assert mixed[j]["median"] == ref[j].median


def test_register_beyond_budget_is_refused():
    srv = SketchServer(hbm_budget_bytes=1 << 20)
    assert srv.register_set(0, [1, 1], [(0, 0, 1, 0)], 1 << 12, 4, 1)      # 256 KB
    assert not srv.register_set(1, [1, 1], [(0, 0, 1, 0)], 1 << 16, 4, 1)  # 4 MB
    srv.close()


def test_native_server_edges():
    """Unknown sets and relations are refused at submission; an update that could never
    fit the budget finishes with SK_ERR_OVER_BUDGET instead of waiting; an empty update
    finishes at once; an estimate of an untouched set is all zero."""
    srv = SketchServer(hbm_budget_bytes=1 << 26)
    assert srv.register_set(0, [1, 1], [(0, 0, 1, 0)], 256, 3, 5)
    with pytest.raises(pkg.SketchError):
        srv.submit_estimate(7)
    with pytest.raises(pkg.SketchError):
        srv.submit_update(0, 5, torch.zeros((1, 3), dtype=torch.int64))
    empty = srv.submit_update(0, 0, torch.zeros((1, 0), dtype=torch.int64))
    big = srv.submit_update(0, 1, torch.zeros((1, 1 << 23), dtype=torch.int64))
    est = srv.submit_estimate(0)
    srv.serve()
    assert srv.pending() == 0
    assert empty.error is None and big.error == "SK_ERR_OVER_BUDGET"
    assert est.error is None and est.result["rows"] == [0, 0, 0]
    assert est.latency >= 0.0
    srv.close()


def test_hold_then_release_equals_alone():
    """Requests queued on a held server wait (nothing finishes); released at once they give
    the results of running each set's requests one by one."""
    import time
    sets, reqs = _trace(5, n_sets=4, n_req=40)
    alone = _alone(sets, reqs)
    srv = SketchServer()
    for i, (a, e, m, d, s) in enumerate(sets):
        assert srv.register_set(i, a, e, m, d, s)
    srv.hold(True)
    handles = {}
    for j, r in enumerate(reqs):
        if r[0] == "update":
            srv.submit_update(r[1], r[2], r[3], r[4])
        else:
            handles[j] = srv.submit_estimate(r[1])
    time.sleep(0.05)
    assert srv.pending() == len(reqs)
    srv.hold(False)
    srv.serve()
    ref = _oracle_expected(sets, reqs)
    for j in alone:
        assert handles[j].error is None and handles[j].result["rows"] == alone[j]["rows"] == ref[j].rows
        assert handles[j].result["median"] == ref[j].median
    st = srv.stats()
    n_upd = sum(1 for r in reqs if r[0] == "update")
    assert st["batched_updates"] == n_upd and st["batches"] < n_upd   # released at once: coalesced
    srv.close()


def test_coalesced_updates_with_declared_domains():
    """Updates that declare key domains (launched as their own calls inside a batch, key
    tables allowed) mixed with plain ones: every estimate equals the oracle's."""
    sets, reqs = _trace(7, n_sets=4, n_req=40)
    srv = SketchServer()
    for i, (a, e, m, d, s) in enumerate(sets):
        assert srv.register_set(i, a, e, m, d, s)
    srv.hold(True)
    handles = {}
    for j, r in enumerate(reqs):
        if r[0] == "update":
            dom = [1 << 20] * r[3].shape[0] if j % 2 else None
            srv.submit_update(r[1], r[2], r[3], r[4], domain=dom)
        else:
            handles[j] = srv.submit_estimate(r[1])
    srv.hold(False)
    srv.serve()
    ref = _oracle_expected(sets, reqs)
    for j, h in handles.items():
        assert h.error is None, h.error
        assert h.result["rows"] == ref[j].rows and h.result["median"] == ref[j].median
    srv.close()
