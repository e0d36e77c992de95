"""The 8-relation chain R0(A0) - R1(A0,A1) - ... - R7(A6) (Zipf(1.2) keys): full
parity at a reduced size, and at the full size (10^7 rows per relation, m = 2^20,
d = 16) checks the oracle can make: sampled sketch rows, an m = 2^20 correlation
read through a one-tuple relation, and exact linearity of the estimate."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2402_15953_gb300 as pkg
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_15953_gb300 import build
    build.build()
    O.build()


def test_chain8_reduced_full_parity():
    wl = synth.chain(r=8, n=100_000, domain=100_000, m=1 << 12, d=3, seed=8, device="cuda")
    s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed)
    for k, rel in enumerate(wl.relations):
        s.update(k, rel.cols)
    est = s.estimate()
    q = O.canonical_query(wl.num_join_attrs, wl.edges)
    co = O.draw_coefficients(wl.hash_seed, wl.d, q.n_comp, len(q.edges))
    sk = O.sketch_all(q, co, [(r.cols.cpu().numpy(), None) for r in wl.relations], wl.m, threads=16)
    got = s.counters.cpu().numpy()
    for k in range(8):
        assert np.array_equal(got[k], sk[k]), k
    ref = O.estimate(q, sk, threads=16)
    assert est["rows"] == ref.rows
    assert est["median"] == ref.median
    assert abs(est["median"]) > (1 << 64)   # beyond int64: exercised the 256-bit path
    s.close()


@pytest.fixture(scope="module")
def chain8_full():
    wl = synth.chain(device="cuda")     # 8 x 1e7 rows, Zipf 1.2 over 1e6, m = 2^20, d = 16
    return wl


def test_chain8_full_sketch_rows(chain8_full):
    wl = chain8_full
    s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed)
    for k, rel in enumerate(wl.relations):
        s.update(k, rel.cols)
    torch.cuda.synchronize()
    q = O.canonical_query(wl.num_join_attrs, wl.edges)
    co = O.draw_coefficients(wl.hash_seed, wl.d, q.n_comp, len(q.edges))
    for k in (0, 3):
        ref = O.sketch_relation(q, co[[0, 11]], k, wl.relations[k].cols.cpu().numpy(), None, wl.m, threads=16)
        got = s.counters[k].cpu().numpy()
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[11], ref[1]), k
    s.close()


def test_chain8_full_estimate_linearity(chain8_full):
    """Doubling one relation's counters (its batch applied twice) doubles every row exactly."""
    wl = chain8_full
    s = pkg.SketchSet(wl.num_join_attrs, wl.edges, wl.m, wl.d, wl.hash_seed)
    for k, rel in enumerate(wl.relations):
        s.update(k, rel.cols)
    e1 = s.estimate()
    s.update(4, wl.relations[4].cols)
    e2 = s.estimate()
    assert e2["rows"] == [2 * v for v in e1["rows"]]
    assert e1["max_residual"] <= 0.25 and e2["max_residual"] <= 0.25
    assert max(abs(v) for v in e1["rows"]) > (1 << 100)
    s.close()


def test_chain8_full_fft_and_ntt_backends_agree(chain8_full):
    """At full size (estimates near 10^46, operands split into up to 10 limbs) the certified
    FP64 FFT, the exact GF(q) transform and the fused CRT form give the same 16 rows."""
    wl = chain8_full
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
    assert a["max_limbs"] >= 6 and a["max_residual"] <= 0.25
    s.close()


@pytest.mark.parametrize("backend", ["fft64", "ntt"])
def test_correlation_at_width_2_20_through_a_one_tuple_relation(chain8_full, backend):
    """R1(A) with one tuple, R2(A, B) and R3(B) with 1e7 rows each: the row estimate is
    s * (c3 star c2)[h], one output of an m = 2^20 correlation of two large sketches,
    which the oracle computes directly."""
    wl = chain8_full
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    r2 = wl.relations[3].cols            # two Zipf columns
    r3 = wl.relations[7].cols            # one column
    one = torch.tensor([[12345]], dtype=torch.int64, device="cuda")
    d, m = 4, 1 << 20
    s = pkg.SketchSet(attrs, edges, m, d, 77)
    s.set_estimator(backend)
    s.update(0, one)
    s.update(1, r2)
    s.update(2, r3)
    est = s.estimate()
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(77, d, q.n_comp, len(q.edges))
    c2 = O.sketch_relation(q, co, 1, r2.cpu().numpy(), None, m, threads=16)
    c3 = O.sketch_relation(q, co, 2, r3.cpu().numpy(), None, m, threads=16)
    bins, signs = O.tuple_hash(q, co, 0, [12345], m)
    for row in range(d):
        z = O.correlate(c3[row].tolist(), c2[row].tolist(), threads=16, bins=[int(bins[row])])[0]
        assert est["rows"][row] == int(signs[row]) * z, row
    s.close()
