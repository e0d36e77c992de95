"""GPU <-> oracle parity through the C ABI: sketches bit-exact, estimates exact.

Every test builds the same seeded inputs for both sides; the oracle draws its
own hash coefficients from the same seed (it never reads the library's)."""
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
    assert torch.cuda.is_available()


def _gpu_sketch(attrs, edges, m, d, seed, rels, domain=None):
    s = pkg.SketchSet(attrs, edges, m, d, seed)
    for k, (cols, w) in enumerate(rels):
        c = torch.as_tensor(np.ascontiguousarray(cols)).cuda()
        wt = None if w is None else torch.as_tensor(np.ascontiguousarray(w)).cuda()
        s.update(k, c, wt, domain=None if domain is None else domain[k])
    s.sync()
    torch.cuda.synchronize()
    return s


def _oracle(attrs, edges, m, d, seed, rels):
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
    return q, co, O.sketch_all(q, co, rels, m)


def test_coefficients_match_oracle_draw():
    attrs, edges = [1, 2, 1, 1], [(0, 0, 1, 0), (2, 0, 1, 0), (3, 0, 1, 1)]
    s = pkg.SketchSet(attrs, edges, 16, 3, 12345)
    q = O.canonical_query(attrs, edges)
    assert np.array_equal(np.array(s.coefficients(), dtype=np.uint64),
                          O.draw_coefficients(12345, 3, q.n_comp, len(q.edges)))
    s.close()


@pytest.mark.parametrize("m", [1, 5, 13, 64, 256, 1000, 4096, 1 << 16])
def test_update_bit_exact_random_queries(m):
    rng = random.Random(m)
    for trial in range(4):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5))
        rels = random_relations(rng, attrs, 3000, 1 << rng.choice([4, 10, 40]), signed=trial % 2 == 0)
        d = rng.choice([1, 3, 7])
        seed = rng.randrange(1 << 62)
        s = _gpu_sketch(attrs, edges, m, d, seed, rels)
        _, _, sk = _oracle(attrs, edges, m, d, seed, rels)
        got = s.counters.cpu().numpy()
        for k in range(len(attrs)):
            assert np.array_equal(got[k], sk[k]), (m, trial, k)
        s.close()


def test_update_extreme_keys_and_weights():
    """Keys at the field's edges (0, p - 1, p, 2^61, 2^63 - 1, negatives) and weights near
    the int64 limits, wrapping like two's complement."""
    p = O.P61
    keys = [0, 1, p - 1, p, p + 1, 1 << 61, (1 << 63) - 1, -1, -(1 << 63), -p, 123456789012345]
    cols = np.array([keys, keys[::-1]], dtype=np.int64)
    w = np.array([(1 << 62), -(1 << 62), (1 << 63) - 1, -(1 << 63), 1, -1, 7, 1 << 40, -(1 << 40), 3, 5],
                 dtype=np.int64)
    attrs, edges = [2, 1, 1], [(0, 0, 1, 0), (0, 1, 2, 0)]
    rels = [(cols, w), (cols[:1].copy(), w), (cols[1:].copy(), None)]
    for m in [7, 256, 1 << 20]:
        s = _gpu_sketch(attrs, edges, m, 5, 99, rels)
        _, _, sk = _oracle(attrs, edges, m, 5, 99, rels)
        got = s.counters.cpu().numpy()
        for k in range(3):
            assert np.array_equal(got[k], sk[k])
        s.close()


def test_large_batch_smem_and_global_paths():
    """The same stream through the shared-memory path (small d*m) and the global-atomic path
    (large d*m) matches the oracle."""
    w = synth.chain3(n=200_000, m=512, d=7, seed=3)
    rels = [(r.cols.numpy(), None) for r in w.relations]
    for m in [512, 1 << 15]:
        s = _gpu_sketch(w.num_join_attrs, w.edges, m, 7, 77, rels)
        _, _, sk = _oracle(w.num_join_attrs, w.edges, m, 7, 77, rels)
        got = s.counters.cpu().numpy()
        for k in range(3):
            assert np.array_equal(got[k], sk[k]), m
        s.close()


@pytest.mark.parametrize("a,d,m", [(1, 3, 1 << 14), (2, 9, 1 << 16), (3, 17, 1 << 12), (5, 9, 1 << 16),
                                    (4, 32, 1 << 13), (5, 5, 1 << 20)])
@pytest.mark.parametrize("cached", ["0", "1"])
def test_update_hot_key_cache_path(a, d, m, cached, monkeypatch):
    """Large Zipf batches (many repeated keys), some keys >= 2^32 and negative keys (the
    full-width arithmetic), signed weights; through the plain kernel and through the
    hot-key cached kernel (SK_UPDATE_CACHE=1)."""
    monkeypatch.setenv("SK_UPDATE_CACHE", cached)
    n = 300_000
    rng = np.random.default_rng(a * 100 + d)
    cols = np.stack([synth.zipf_keys(n, 1.1, 1 << 16, 1000 + c).numpy() for c in range(a)])
    wide = rng.random((a, n)) < 0.05
    cols = np.where(wide, cols * 1_000_003_117 + (1 << 40), cols)
    neg = rng.random((a, n)) < 0.02
    cols = np.where(neg, -cols - 1, cols).astype(np.int64)
    w = rng.choice(np.array([-2, -1, 1, 1, 3], dtype=np.int64), size=n)
    attrs = [a] + [1] * a
    edges = [(0, i, 1 + i, 0) for i in range(a)]
    rels = [(cols, w)] + [(np.zeros((1, 0), dtype=np.int64), None)] * a
    s = _gpu_sketch(attrs, edges, m, d, 4242, rels)
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(4242, d, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, cols, w, m, threads=16)
    assert np.array_equal(s.counters[0].cpu().numpy(), ref)
    s.close()


@pytest.mark.parametrize("agg", ["0", "1"])
def test_update_shared_memory_path_warp_aggregation(agg, monkeypatch):
    """Shared-memory sub-sketch path with and without warp-aggregated atomics
    (SK_WARP_AGG=1): Zipf keys so lanes of a warp often hit the same counter, a domain
    hint with violations (those tuples are skipped), signed weights.  Key tables are
    turned off so the declared domain does not route the batch around the hashing kernel."""
    monkeypatch.setenv("SK_WARP_AGG", agg)
    monkeypatch.setenv("SK_KEY_TABLE", "0")
    n = 100_003
    rng = np.random.default_rng(5)
    cols = np.stack([synth.zipf_keys(n, 1.3, 5000, 70 + c).numpy() for c in range(2)])
    cols[0, ::977] = 6000                       # outside the declared domain
    w = rng.choice(np.array([-1, 1, 2], dtype=np.int64), size=n)
    attrs, edges = [2, 1, 1], [(0, 0, 1, 0), (0, 1, 2, 0)]
    s = pkg.SketchSet(attrs, edges, 256, 5, 31)
    s.update(0, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda(), domain=[5000, 5000])
    with pytest.raises(pkg.SketchError):
        s.sync()
    keep = cols[0] < 5000
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(31, 5, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, cols[:, keep], w[keep], 256, threads=8)
    assert np.array_equal(s.counters[0].cpu().numpy(), ref)
    s.close()


@pytest.mark.parametrize("estimator", ["fft64", "ntt", "fused"])
def test_chain3_config_exact(estimator):
    """Chain R1(A) - R2(A,B) - R3(B), 10^4 rows each, m = 256, d = 5, seed 42: bit-exact
    sketches, exact row estimates and median in each arithmetic."""
    w = synth.chain3()
    rels = [(r.cols.numpy(), None) for r in w.relations]
    s = _gpu_sketch(w.num_join_attrs, w.edges, w.m, w.d, w.hash_seed, rels)
    q, co, sk = _oracle(w.num_join_attrs, w.edges, w.m, w.d, w.hash_seed, rels)
    got = s.counters.cpu().numpy()
    for k in range(3):
        assert np.array_equal(got[k], sk[k])
    s.set_estimator(estimator)
    est = s.estimate()
    ref = O.estimate(q, sk)
    assert est["rows"] == ref.rows
    assert est["median"] == ref.median and est["fits_i64"] and est["median_i64"] == ref.median
    assert est["max_residual"] <= 0.25
    assert est["mid_mean_f64"] == pytest.approx(ref.mid_mean, rel=1e-12)
    s.close()


@pytest.mark.parametrize("estimator", ["fft64", "fused"])
@pytest.mark.parametrize("m", [2, 4, 8, 64, 1024, 1 << 13, 1 << 14])
def test_estimate_exact_random_queries(m, estimator):
    rng = random.Random(1000 + m)
    trials = 6 if m <= 1024 else 2
    for trial in range(trials):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5))
        rels = random_relations(rng, attrs, 400 if m <= 1024 else 3000, 1 << rng.choice([3, 12, 30]))
        d = rng.choice([1, 2, 5])
        seed = rng.randrange(1 << 62)
        s = _gpu_sketch(attrs, edges, m, d, seed, rels)
        s.set_estimator(estimator)
        q, co, sk = _oracle(attrs, edges, m, d, seed, rels)
        est = s.estimate()
        ref = O.estimate(q, sk)
        assert est["rows"] == ref.rows, (m, trial, attrs, edges)
        assert est["median"] == ref.median
        s.close()


@pytest.mark.parametrize("estimator", ["fft64", "fused"])
@pytest.mark.parametrize("m", [3, 5, 12, 100, 1000, 10007])
def test_estimate_exact_non_power_of_two_width(m, estimator):
    """Widths that are not powers of two (the paper's experiments use m = 10^6): zero-padded
    transforms folded back mod m give the exact Algorithm 3 rows."""
    rng = random.Random(2000 + m)
    for trial in range(3 if m < 10000 else 1):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5))
        rels = random_relations(rng, attrs, 500 if m < 10000 else 4000, 1 << rng.choice([3, 12, 30]))
        d = rng.choice([1, 3])
        seed = rng.randrange(1 << 62)
        s = _gpu_sketch(attrs, edges, m, d, seed, rels)
        s.set_estimator(estimator)
        q, co, sk = _oracle(attrs, edges, m, d, seed, rels)
        assert np.array_equal(s.counters.cpu().numpy(), np.stack(sk))
        est = s.estimate()
        ref = O.estimate(q, sk)
        assert est["rows"] == ref.rows, (m, trial, attrs, edges)
        s.close()


@pytest.mark.parametrize("estimator", ["fft64", "fused"])
def test_width_one_million_correlation_through_a_one_tuple_relation(estimator):
    """m = 10^6 (Section 4.4's width): R1 with one tuple turns each row estimate into one output
    of the circular correlation of R3's and R2's sketches, computed directly by the oracle."""
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    n = 300_000
    r2 = torch.stack([synth.zipf_keys(n, 1.2, 1 << 20, 3), synth.zipf_keys(n, 1.2, 1 << 20, 4)])
    r3 = synth.zipf_keys(n, 1.2, 1 << 20, 5)[None, :].contiguous()
    m, d = 1_000_000, 3
    s = pkg.SketchSet(attrs, edges, m, d, 91)
    s.set_estimator(estimator)
    s.update(0, torch.tensor([[777]], dtype=torch.int64, device="cuda"))
    s.update(1, r2.cuda())
    s.update(2, r3.cuda())
    est = s.estimate()
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(91, d, q.n_comp, len(q.edges))
    c2 = O.sketch_relation(q, co, 1, r2.numpy(), None, m, threads=16)
    c3 = O.sketch_relation(q, co, 2, r3.numpy(), None, m, threads=16)
    bins, signs = O.tuple_hash(q, co, 0, [777], m)
    for row in range(d):
        z = O.correlate(c3[row].tolist(), c2[row].tolist(), threads=16, bins=[int(bins[row])])[0]
        assert est["rows"][row] == int(signs[row]) * z
    s.close()


@pytest.mark.parametrize("m", [2, 8, 12, 64, 1000, 1024, 1 << 13, 1 << 14])
def test_estimate_exact_ntt_backend(m):
    """The GF(2^64 - 2^32 + 1) transform backend gives the oracle's exact rows (power-of-two
    widths, single-pass and four-step transforms, and zero-padded other widths)."""
    rng = random.Random(3000 + m)
    for trial in range(4 if m <= 1024 else 2):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5))
        rels = random_relations(rng, attrs, 400 if m <= 1024 else 3000, 1 << rng.choice([3, 12, 30]))
        d = rng.choice([1, 2, 5])
        seed = rng.randrange(1 << 62)
        s = _gpu_sketch(attrs, edges, m, d, seed, rels)
        s.set_estimator("ntt")
        q, co, sk = _oracle(attrs, edges, m, d, seed, rels)
        est = s.estimate()
        ref = O.estimate(q, sk)
        assert est["rows"] == ref.rows, (m, trial, attrs, edges)
        assert est["max_residual"] == 0.0
        s.close()


def test_default_estimator_is_fused():
    s = pkg.SketchSet([1, 1], [(0, 0, 1, 0)], 64, 2, 1)
    s.update(0, torch.arange(50, dtype=torch.int64, device="cuda")[None, :])
    s.update(1, torch.arange(50, dtype=torch.int64, device="cuda")[None, :])
    e = s.estimate()
    assert e["limb_bits"] == 0 and e["max_limbs"] >= 1      # CRT primes, no limbs
    s.close()


def test_ntt_and_fft_backends_agree_on_the_star_and_chain8_shapes():
    for wl in (synth.star(n_fact=2_000_000, n_dim=200_000, m=1 << 16, d=3, device="cuda"),
               synth.chain(r=8, n=200_000, m=1 << 14, d=2, device="cuda")):
        s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed)
        for k, rel in enumerate(wl.relations):
            s.update(k, rel.cols)
        s.set_estimator("fft64")
        a = s.estimate()
        s.set_estimator("ntt")
        b = s.estimate()
        s.set_estimator("fused")
        c = s.estimate()
        assert a["rows"] == b["rows"] == c["rows"] and a["median"] == b["median"] == c["median"]
        s.close()
    assert pkg.load().sk_sketch_set_estimator(None, 1) == pkg.SK_ERR_INVALID_ARG


def test_identity_hashing_gives_exact_join_size_on_gpu():
    """With injective test hashes (bin x * R_q, sign +1) the GPU estimate is the exact join size."""
    rng = random.Random(7)
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    rels = random_relations(rng, attrs, 5000, 30, signed=True)
    m = 1024
    s = pkg.SketchSet(attrs, edges, m, 2, 1)
    q = O.canonical_query(attrs, edges)
    s.set_coefficients(O.identity_coefficients(q, 2, [30, 30]).tolist())
    for k, (cols, w) in enumerate(rels):
        s.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda())
    est = s.estimate()
    truth = O.exact_join_size(q, rels)
    assert est["rows"] == [truth, truth]
    s.close()


def test_merge_equals_single_pass():
    w = synth.chain3(n=5000, m=128, d=3, seed=5)
    rels = [(r.cols.numpy(), None) for r in w.relations]
    full = _gpu_sketch(w.num_join_attrs, w.edges, 128, 3, 8, rels)
    a = _gpu_sketch(w.num_join_attrs, w.edges, 128, 3, 8, [(c[:, :2000], None) for c, _ in rels])
    b = _gpu_sketch(w.num_join_attrs, w.edges, 128, 3, 8, [(c[:, 2000:], None) for c, _ in rels])
    a.merge(b)
    torch.cuda.synchronize()
    assert torch.equal(a.counters, full.counters)
    c = _gpu_sketch(w.num_join_attrs, w.edges, 128, 3, 9, rels)
    with pytest.raises(pkg.SketchError) as e:
        a.merge(c)
    assert e.value.name == "SK_ERR_MISMATCH"
    for x in (full, a, b, c):
        x.close()


def test_key_out_of_domain_is_reported_and_skipped():
    attrs, edges = [1, 1], [(0, 0, 1, 0)]
    cols = np.array([[1, 2, 3, 50, 4]], dtype=np.int64)
    s = pkg.SketchSet(attrs, edges, 16, 2, 3)
    s.update(0, torch.as_tensor(cols).cuda(), domain=[10])
    with pytest.raises(pkg.SketchError) as e:
        s.sync()
    assert e.value.name == "SK_ERR_KEY_OUT_OF_DOMAIN"
    s.sync()  # cleared
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(3, 2, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, np.array([[1, 2, 3, 4]], dtype=np.int64), None, 16)
    assert np.array_equal(s.counters[0].cpu().numpy(), ref)
    s.close()


def test_invalid_arguments():
    with pytest.raises(pkg.SketchError) as e:
        pkg.SketchSet([1, 1], [(0, 0, 0, 0)], 16, 2, 1)
    assert e.value.name == "SK_ERR_SELF_EDGE"
    with pytest.raises(pkg.SketchError) as e:
        pkg.SketchSet([2, 2], [(0, 0, 1, 0), (0, 1, 1, 1)], 16, 2, 1)
    assert e.value.name == "SK_ERR_CYCLIC_QUERY"
    s = pkg.SketchSet([1, 1], [(0, 0, 1, 0)], (1 << 21) + 1, 1, 1)
    with pytest.raises(pkg.SketchError) as e:
        s.estimate()
    assert e.value.name == "SK_ERR_UNSUPPORTED_WIDTH"
    s.close()
    s = pkg.SketchSet([1, 1], [(0, 0, 1, 0)], 1, 1, 1)
    with pytest.raises(pkg.SketchError) as e:
        s.estimate()
    assert e.value.name == "SK_ERR_UNSUPPORTED_WIDTH"
    with pytest.raises(pkg.SketchError):
        pkg.sk_sketch_update_batch(s.handle, 5, 10, s.counters.data_ptr(), 10, None, None, 0)
    s.close()


def test_empty_batch_and_empty_relation():
    attrs, edges = [1, 1], [(0, 0, 1, 0)]
    s = pkg.SketchSet(attrs, edges, 64, 3, 4)
    s.update(0, torch.empty((1, 0), dtype=torch.int64, device="cuda"))
    est = s.estimate()
    assert est["rows"] == [0, 0, 0] and est["median"] == 0
    s.close()
