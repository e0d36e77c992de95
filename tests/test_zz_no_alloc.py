"""The allocation-free estimator entry point, sk_estimate_join_noalloc.

It exists for callers that cannot call cudaMalloc while they estimate (a host
callback or driver-level hook that must not enter the CUDA allocator, a process
whose device memory is held by another pool, or a latency-critical path that
forbids allocation).  It must give exactly the same row estimates and median as
sk_estimate_join and as the CPU oracle on the same sketches, call after call,
although every call reuses one static device scratch array.

Collected last on purpose (file name), so a run that stops at the first failure
has already run every other test; it also passes on its own in a fresh process.
"""
import ctypes
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
    assert torch.cuda.is_available()


def _noalloc(handle, stream):
    out = pkg.sk_estimate()
    st = pkg.load().sk_estimate_join_noalloc(handle, ctypes.byref(out), stream)
    return st, out


def _rows(e):
    return [e.row[i].value() for i in range(e.d)]


def _oracle_rows(attrs, edges, m, d, seed, rels):
    """Algorithm 3 rows and lower median computed by the CPU oracle from its own sketches."""
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
    return O.estimate(q, O.sketch_all(q, co, rels, m))


def _check_same(s, ref_oracle):
    stream = torch.cuda.current_stream().cuda_stream
    ref = pkg.sk_estimate_join(s.handle, stream)
    assert _rows(ref) == ref_oracle.rows
    for _ in range(2):  # two calls in a row share the static scratch
        st, got = _noalloc(s.handle, stream)
        assert st == 0, pkg.STATUS.get(st, st)
        assert _rows(got) == _rows(ref) == ref_oracle.rows
        assert got.median.value() == ref.median.value() == ref_oracle.median
        assert got.fits_i64 == ref.fits_i64 and got.median_i64 == ref.median_i64
        assert got.mid_mean_f64 == ref.mid_mean_f64
        assert got.mid_mean_f64 == pytest.approx(ref_oracle.mid_mean, rel=1e-12)
        assert got.max_residual <= 0.25


def test_noalloc_matches_estimate_join_chain3():
    w = synth.chain3()
    s = pkg.SketchSet(w.num_join_attrs, w.edges, w.m, w.d, w.hash_seed)
    for k, rel in enumerate(w.relations):
        s.update(k, rel.cols.cuda())
    rels = [(r.cols.cpu().numpy(), None) for r in w.relations]
    _check_same(s, _oracle_rows(w.num_join_attrs, w.edges, w.m, w.d, w.hash_seed, rels))
    s.close()


def test_noalloc_matches_estimate_join_random_queries():
    rng = random.Random(2024)
    for m in [4, 256, 4096, 1 << 13]:
        attrs, edges = random_tree_query(rng, rng.randint(2, 5))
        rels = random_relations(rng, attrs, 2000, 1 << 20)
        seed = rng.randrange(1 << 62)
        s = pkg.SketchSet(attrs, edges, m, 3, seed)
        for k, (cols, wt) in enumerate(rels):
            s.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(wt).cuda())
        _check_same(s, _oracle_rows(attrs, edges, m, 3, seed, rels))
        s.close()


def test_noalloc_rejects_widths_that_are_not_powers_of_two():
    s = pkg.SketchSet([1, 1], [(0, 0, 1, 0)], 1000, 3, 5)
    st, _ = _noalloc(s.handle, torch.cuda.current_stream().cuda_stream)
    assert pkg.STATUS.get(st) == "SK_ERR_UNSUPPORTED_WIDTH"
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # m = 2^20, d = 16: the vector slots alone exceed the static scratch
    s = pkg.SketchSet([1, 1], [(0, 0, 1, 0)], 1 << 20, 16, 5)
    st, _ = _noalloc(s.handle, torch.cuda.current_stream().cuda_stream)
    assert pkg.STATUS.get(st) == "SK_ERR_SCRATCH_TOO_SMALL"
    s.close()
