"""The batched form (sk_update_plan_*): one persistent launch over many update batches
gives exactly the counters of the item-by-item calls and of the oracle, also when the
run is captured in a CUDA graph and after autotuning."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2402_15953_gb300 as pkg
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    from paper_2402_15953_gb300 import build
    build.build()
    O.build()
    return synth.batched(count=40, median_rows=2e4, sigma=1.5, min_rows=100, max_rows=300_000, log2m=(4, 14),
                         seed=9, device="cuda")


def _sets(wl):
    return [pkg.SketchSet(b.num_join_attrs, b.edges, b.m, b.d, b.hash_seed) for b in wl]


def test_plan_equals_item_by_item_and_oracle(workload):
    ref = _sets(workload)
    for s, b in zip(ref, workload):
        s.update(0, b.relation.cols, b.relation.weights)
    got = _sets(workload)
    plan = pkg.UpdatePlan([(s, 0, b.relation.cols, b.relation.weights) for s, b in zip(got, workload)])
    # int32 sub-sketches, global counters only, everything in int32 shared memory, and packed
    # 16-bit sub-sketches (alone and beside int32 ones; chunk 32768 admits only |Delta| = 0)
    for cfg in [(32768, 256, 6, 16384), (1024, 128, 2, 0), (4096, 256, 8, 1 << 20), (4096, 256, 8, 0, 1 << 20),
                (8192, 256, 4, 1024, 32768), (32768, 256, 4, 0, 1 << 20)]:
        for s in got:
            s.reset()
        plan.set_config(*cfg)
        plan.run()
        torch.cuda.synchronize()
        for s, r in zip(got, ref):
            assert torch.equal(s.counters, r.counters), cfg
    # oracle on the five smallest relations
    order = sorted(range(len(workload)), key=lambda i: workload[i].relation.n)[:5]
    for i in order:
        b = workload[i]
        q = O.canonical_query(b.num_join_attrs, b.edges)
        co = O.draw_coefficients(b.hash_seed, b.d, q.n_comp, len(q.edges))
        want = O.sketch_relation(q, co, 0, b.relation.cols.cpu().numpy(), b.relation.weights.cpu().numpy(), b.m)
        assert np.array_equal(got[i].counters[0].cpu().numpy(), want)
    plan.close()
    for s in ref + got:
        s.close()


def test_plan_in_cuda_graph_and_autotune(workload):
    ref = _sets(workload)
    for s, b in zip(ref, workload):
        s.update(0, b.relation.cols, b.relation.weights)
    got = _sets(workload)
    plan = pkg.UpdatePlan([(s, 0, b.relation.cols, b.relation.weights) for s, b in zip(got, workload)])
    best, ms = plan.autotune()
    assert ms > 0 and best["chunk_tuples"] >= 256
    for s in got:
        s.reset()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plan.run()          # warm-up outside the graph (kernel attributes set)
    stream.synchronize()
    for s in got:
        s.reset()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        plan.run()
    for s in got:
        s.reset()
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for s, r in zip(got, ref):
        assert torch.equal(s.counters, 2 * r.counters)
    plan.close()
    for s in ref + got:
        s.close()


def test_plan_argument_checks(workload):
    s = pkg.SketchSet([1, 1], [(0, 0, 1, 0)], 64, 2, 1)
    with pytest.raises(pkg.SketchError):
        pkg.sk_update_plan_create([(s.handle, 7, 10, s.counters.data_ptr(), 10, None)])
    empty = pkg.UpdatePlan([(s, 0, torch.empty((1, 0), dtype=torch.int64, device="cuda"), None)])
    empty.run()
    with pytest.raises(pkg.SketchError):
        empty.set_config(100, 256, 4, 0)
    empty.close()
    s.close()


def test_plan_zero_clears_only_the_planned_relations(workload):
    """sk_update_plan_zero: the counters of every (set, relation) the plan writes become
    zero, the set's other relations keep theirs; d m odd puts relation 1's block on an
    8-byte (not 16-byte) boundary; a relation listed twice; a run after the zeroing equals
    the items applied one by one to fresh sets."""
    rng = np.random.default_rng(3)
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    shapes = [(777, 3), (64, 5), (1000, 1), (4096, 7), (2, 1)]
    sets, items = [], []
    for i, (m, d) in enumerate(shapes):
        s = pkg.SketchSet(attrs, edges, m, d, 10 + i)
        for k, a in enumerate(attrs):
            s.update(k, torch.as_tensor(rng.integers(0, 500, size=(a, 3000))).cuda())
        sets.append(s)
        c0 = torch.as_tensor(rng.integers(0, 500, size=(1, 100))).cuda()
        c1 = torch.as_tensor(rng.integers(0, 500, size=(2, 100))).cuda()
        items += [(s, 0, c0, None), (s, 1, c1, None), (s, 1, c1, None)]
    torch.cuda.synchronize()
    keep = [s.counters[2].clone() for s in sets]
    plan = pkg.UpdatePlan(items)
    plan.zero()
    torch.cuda.synchronize()
    for s, k in zip(sets, keep):
        assert not bool(s.counters[0].any()) and not bool(s.counters[1].any())
        assert bool(k.any()) and torch.equal(s.counters[2], k)
    plan.run()
    fresh = [pkg.SketchSet(attrs, edges, m, d, 10 + i) for i, (m, d) in enumerate(shapes)]
    for j, (s, rel, cols, w) in enumerate(items):
        fresh[j // 3].update(rel, cols, w)
    torch.cuda.synchronize()
    for s, f in zip(sets, fresh):
        assert torch.equal(s.counters[:2], f.counters[:2])
    plan.close()
    for s in sets + fresh:
        s.close()


def test_full_size_batched_workload_sampled_against_oracle():
    """The bench's batched workload at full size (256 relations, 7.9e7 tuples, widths
    2^10..2^18) through one zeroing and one persistent run in the configuration the
    autotuner picks: the three smallest relations' sketches in full and two rows of the
    largest relation's sketch equal the oracle's."""
    from paper_2402_15953_gb300 import build
    build.build()
    O.build()
    wl = synth.batched(seed=42, device="cuda")
    sets = _sets(wl)
    plan = pkg.UpdatePlan([(s, 0, b.relation.cols, b.relation.weights) for s, b in zip(sets, wl)])
    plan.set_config(8192, 256, 8, 8192)
    plan.zero()
    plan.run()
    torch.cuda.synchronize()
    order = sorted(range(len(wl)), key=lambda i: wl[i].relation.n)
    for i in order[:3] + order[-1:]:
        b = wl[i]
        q = O.canonical_query(b.num_join_attrs, b.edges)
        co = O.draw_coefficients(b.hash_seed, b.d, q.n_comp, len(q.edges))
        rows = list(range(b.d)) if i != order[-1] else [0, b.d - 1]
        want = O.sketch_relation(q, co[rows], 0, b.relation.cols.cpu().numpy(), b.relation.weights.cpu().numpy(),
                                 b.m, threads=16)
        got = sets[i].counters[0].cpu().numpy()[rows]
        assert np.array_equal(got, want), (i, b.relation.n, b.m)
    plan.close()
    for s in sets:
        s.close()


def test_autotune_choice_is_persisted(workload, tmp_path, monkeypatch):
    """The first autotune of a plan shape times the grid and appends its winner to the cache
    file; a second plan of the same shape takes it from there without timing (its counters
    stay untouched) and still gives the item-by-item counters."""
    cache = tmp_path / "autotune.json"
    monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(cache))
    sub = workload[:12]
    a = _sets(sub)
    plan_a = pkg.UpdatePlan([(s, 0, b.relation.cols, b.relation.weights) for s, b in zip(a, sub)])
    best_a, ms_a = plan_a.autotune()
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and '"key": "sms=' in lines[0]
    b = _sets(sub)
    plan_b = pkg.UpdatePlan([(s, 0, bb.relation.cols, bb.relation.weights) for s, bb in zip(b, sub)])
    best_b, ms_b = plan_b.autotune()
    assert best_b == best_a and ms_b == pytest.approx(ms_a, rel=1e-5)
    assert len(cache.read_text().splitlines()) == 1
    assert all(int(torch.count_nonzero(s.counters)) == 0 for s in b)   # not timed: nothing applied
    plan_b.run()
    ref = _sets(sub)
    for s, bb in zip(ref, sub):
        s.update(0, bb.relation.cols, bb.relation.weights)
    torch.cuda.synchronize()
    for x, y in zip(b, ref):
        assert torch.equal(x.counters, y.counters)
    for p in (plan_a, plan_b):
        p.close()
    for s in a + b + ref:
        s.close()
