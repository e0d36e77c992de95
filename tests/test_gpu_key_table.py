"""Key-table update path (declared key domains): bit-exact against the oracle.

With SK_KEY_TABLE=1 every update that declares domains goes through the per-domain-key
tables; with 0 it hashes per tuple.  Both must give the oracle's sketches, including
for tuples outside the declared domain (reported and skipped), widths that are and are
not powers of two, the shared-memory and global-atomic scatter, both record formats
(16-bit bins for m <= 2^16 and d <= 32, at the record-length boundaries d = 14 / 15;
32-bit otherwise), d not a multiple of the record vector, and relations with more
attributes than the fixed-arity kernels."""
import random

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


def _star(a):
    return [a] + [1] * a, [(0, i, 1 + i, 0) for i in range(a)]


def _run(attrs, edges, m, d, seed, cols, w, dom):
    s = pkg.SketchSet(attrs, edges, m, d, seed)
    s.update(0, torch.as_tensor(cols).cuda(), None if w is None else torch.as_tensor(w).cuda(), domain=dom)
    bad = bool(((cols < 0) | (cols >= np.array(dom)[:, None])).any())
    if bad:
        with pytest.raises(pkg.SketchError):
            s.sync()
    else:
        s.sync()
    got = s.counters[0].cpu().numpy()
    s.close()
    return got


MODES = {"direct": ("0", "1"), "table": ("1", "1"), "table-16B-loads": ("1", "0")}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("a,d,m", [(1, 1, 64), (2, 3, 1000), (3, 9, 1 << 16), (5, 9, 1 << 16), (5, 7, 77777),
                                    (4, 64, 1 << 12), (7, 5, 1 << 14), (2, 13, 256), (3, 14, 1 << 16),
                                    (2, 15, 4096), (3, 32, 2048), (6, 9, 65535), (2, 5, 1 << 18),
                                    (2, 9, 50000), (5, 11, 1 << 15), (3, 1, 2)])
def test_key_table_bit_exact(mode, a, d, m, monkeypatch):
    """mode: per-tuple hashing; key tables with 32-byte records read by one 256-bit load
    where they apply; key tables read in 16-byte loads only (SK_TAB_V8=0)."""
    monkeypatch.setenv("SK_KEY_TABLE", MODES[mode][0])
    monkeypatch.setenv("SK_TAB_V8", MODES[mode][1])
    rng = np.random.default_rng(a * 1000 + d)
    n = 200_003
    doms = [int(x) for x in rng.integers(50, 5000, size=a)]
    cols = np.stack([synth.zipf_keys(n, 1.1, doms[u], 17 + u).numpy() for u in range(a)])
    w = rng.choice(np.array([-3, -1, 1, 1, 2], dtype=np.int64), size=n)
    attrs, edges = _star(a)
    got = _run(attrs, edges, m, d, 99 + a, cols, w, doms)
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(99 + a, d, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, cols, w, m, threads=16)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", list(MODES))
def test_key_table_domain_violations_and_edges(mode, monkeypatch):
    """Keys -1, dom and beyond are skipped and reported; keys 0 and dom - 1 (the table's
    first and last records) count."""
    monkeypatch.setenv("SK_KEY_TABLE", MODES[mode][0])
    monkeypatch.setenv("SK_TAB_V8", MODES[mode][1])
    rng = np.random.default_rng(3)
    n = 50_000
    doms = [1000, 1 << 20]
    cols = np.stack([rng.integers(0, doms[0], n), rng.integers(0, doms[1], n)]).astype(np.int64)
    cols[0, :7] = [0, 999, -1, 1000, 5000, 0, 999]
    cols[1, :7] = [0, (1 << 20) - 1, 5, 6, 7, -(1 << 40), (1 << 20)]
    attrs, edges = _star(2)
    for m in (512, 1 << 17):
        got = _run(attrs, edges, m, 6, 5, cols, None, doms)
        keep = (cols[0] >= 0) & (cols[0] < doms[0]) & (cols[1] >= 0) & (cols[1] < doms[1])
        q = O.canonical_query(attrs, edges)
        co = O.draw_coefficients(5, 6, q.n_comp, len(q.edges))
        ref = O.sketch_relation(q, co, 0, cols[:, keep], None, m, threads=16)
        assert np.array_equal(got, ref), m


def test_key_table_shared_attribute_queries(monkeypatch):
    """Random tree queries where one attribute sits in several joins (its record carries
    the product of those signs) and components span three relations; every relation of
    the query is updated through the tables."""
    monkeypatch.setenv("SK_KEY_TABLE", "1")
    from tests._helpers import random_tree_query
    rng = random.Random(11)
    for trial in range(6):
        attrs, edges = random_tree_query(rng, rng.randint(2, 5), share_prob=0.6)
        m = rng.choice([256, 1000, 1 << 15])
        d = rng.choice([1, 4, 5, 11])
        seed = rng.randrange(1 << 60)
        s = pkg.SketchSet(attrs, edges, m, d, seed)
        rels = []
        for k, a in enumerate(attrs):
            n = rng.randint(1000, 30000)
            dom = [rng.randint(1, 3000) for _ in range(a)]
            cols = np.stack([np.array([rng.randrange(x) for _ in range(n)], dtype=np.int64) for x in dom])
            w = np.array([rng.choice([-1, 1, 2]) for _ in range(n)], dtype=np.int64)
            s.update(k, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda(), domain=dom)
            rels.append((cols, w))
        s.sync()
        got = s.counters.cpu().numpy()
        q = O.canonical_query(attrs, edges)
        co = O.draw_coefficients(seed, d, q.n_comp, len(q.edges))
        sk = O.sketch_all(q, co, rels, m)
        for k in range(len(attrs)):
            assert np.array_equal(got[k], sk[k]), (trial, k)
        s.close()


def test_key_table_auto_matches_direct_on_star_shape(monkeypatch):
    """The default choice (tables when the domains are small against the batch) and the
    per-tuple path give the same sketch on a 2e6-row (ragged last CTA), 5-column Zipf(1.1)
    fact table."""
    n, dom = 2_000_003, 100_000
    cols = torch.stack([synth.zipf_keys(n, 1.1, dom, 500 + u, device="cuda") for u in range(5)])
    attrs, edges = _star(5)
    out = []
    monkeypatch.delenv("SK_TAB_V8", raising=False)
    for mode in ("", "0"):
        monkeypatch.setenv("SK_KEY_TABLE", mode)
        s = pkg.SketchSet(attrs, edges, 1 << 16, 9, 42)
        s.update(0, cols, domain=[dom] * 5)
        s.sync()
        out.append(s.counters[0].cpu().numpy())
        s.close()
    assert np.array_equal(out[0], out[1])
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(42, 9, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co[[0, 8]], 0, cols.cpu().numpy(), None, 1 << 16, threads=16)
    assert np.array_equal(out[0][0], ref[0]) and np.array_equal(out[0][8], ref[1])


def test_key_table_from_page_locked_host_columns(monkeypatch):
    """Columns and weights in page-locked host memory passed straight to the C ABI (the
    kernels read them across the host link); the tables stay in device memory."""
    monkeypatch.setenv("SK_KEY_TABLE", "1")
    monkeypatch.delenv("SK_TAB_V8", raising=False)
    n, doms = 300_001, [4000, 700, 90000]
    cols = torch.stack([synth.zipf_keys(n, 1.2, x, 40 + u) for u, x in enumerate(doms)]).pin_memory()
    w = torch.randint(-2, 3, (n,), dtype=torch.int64, generator=torch.Generator().manual_seed(9)).pin_memory()
    attrs, edges = _star(3)
    ref = None
    for host in (True, False):
        s = pkg.SketchSet(attrs, edges, 1 << 15, 9, 8)
        c, ww = (cols, w) if host else (cols.cuda(), w.cuda())
        pkg.sk_sketch_update_batch(s.handle, 0, n, c.data_ptr(), int(c.stride(0)), ww.data_ptr(), doms,
                                   torch.cuda.current_stream().cuda_stream)
        s.sync()
        got = s.counters[0].cpu().numpy()
        s.close()
        if ref is None:
            q = O.canonical_query(attrs, edges)
            co = O.draw_coefficients(8, 9, q.n_comp, len(q.edges))
            ref = O.sketch_relation(q, co, 0, cols.numpy(), w.numpy(), 1 << 15, threads=16)
        assert np.array_equal(got, ref), host


@pytest.mark.parametrize("record", ["24", "32"])
@pytest.mark.parametrize("a,d,m,n,window", [(5, 9, 1 << 16, 1_200_007, 0), (5, 9, 1 << 16, 1_200_007, 262_144),
                                             (3, 14, 1 << 15, 600_001, 0), (2, 5, 1 << 14, 300_007, 65_536),
                                             (1, 13, 1 << 12, 100_003, 0), (4, 2, 1 << 16, 1_048_576, 262_144),
                                             (2, 7, 1 << 13, 200_003, 0), (3, 6, 1 << 15, 524_288, 0)])
def test_partitioned_update_bit_exact(a, d, m, n, window, record, monkeypatch):
    """Unit-weight batches with declared domains, power-of-two m <= 2^16 and sketches too
    large for one CTA's shared memory take the two-phase update (per-row bin planes, then
    shared-memory accumulation per (row, part)), with 24- and 32-byte key-table records for
    d <= 9; one window or several with a ragged last one; keys at the table's first and last
    records and outside the domain (skipped and reported).  The launch count shows which path
    ran: the table build plus two launches per window."""
    monkeypatch.setenv("SK_KEY_TABLE", "1")
    monkeypatch.setenv("SK_PART_RECORD", record)
    if window:
        monkeypatch.setenv("SK_PART_WINDOW", str(window))
    rng = np.random.default_rng(a * 7919 + d)
    doms = [int(x) for x in rng.integers(1000, 200_000, size=a)]
    cols = np.stack([synth.zipf_keys(n, 1.1, doms[u], 300 + u).numpy() for u in range(a)])
    cols[0, :5] = [0, doms[0] - 1, -1, doms[0], 3]
    cols[a - 1, n - 3:] = [doms[a - 1], 0, doms[a - 1] - 1]
    attrs, edges = _star(a)
    L0 = pkg.sk_launch_count()
    got = _run(attrs, edges, m, d, 1234 + a, cols, None, doms)
    launches = pkg.sk_launch_count() - L0
    per_window = window if window else n
    assert launches == 1 + 2 * ((n + per_window - 1) // per_window), launches
    keep = np.all((cols >= 0) & (cols < np.array(doms)[:, None]), axis=0)
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(1234 + a, d, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, cols[:, keep], None, m, threads=16)
    assert np.array_equal(got, ref)


def test_partitioned_update_edges(monkeypatch):
    """The two-phase update at its edges: one row (d = 1) at m = 2^16; a window whose every
    tuple has a key outside its domain (all reported and skipped: the tiles hold no items);
    window lengths that leave a ragged last tile (not a multiple of 32 or of 8); one part per
    row (m = 4096, d = 13: the smallest sketch that does not fit one CTA's shared memory);
    every tuple with the same keys, so that each row's items all fall in one part and every
    warp's region of that row fills from one end to the other."""
    monkeypatch.setenv("SK_KEY_TABLE", "1")
    rng = np.random.default_rng(77)
    cases = [(2, 1, 1 << 16, (1 << 20) + 3, 0, False), (3, 9, 1 << 16, (1 << 20) + 37, 262_144 + 256, True),
             (1, 13, 4096, 65_536 + 13, 0, False), (4, 9, 1 << 16, (1 << 20) + 29, 0, "same")]
    for a, d, m, n, window, bad_window in cases:
        if window:
            monkeypatch.setenv("SK_PART_WINDOW", str(window))
        else:
            monkeypatch.delenv("SK_PART_WINDOW", raising=False)
        doms = [int(x) for x in rng.integers(500, 50_000, size=a)]
        cols = np.stack([synth.zipf_keys(n, 1.2, doms[u], 900 + u).numpy() for u in range(a)])
        if bad_window == "same":   # one key per attribute for every tuple
            cols[:, :] = cols[:, :1]
        elif bad_window:   # every tuple of the second window out of domain
            cols[0, window:2 * window] = doms[0] + 5
        attrs, edges = _star(a)
        L0 = pkg.sk_launch_count()
        got = _run(attrs, edges, m, d, 4321 + d, cols, None, doms)
        launches = pkg.sk_launch_count() - L0
        per = window if window else n
        assert launches == 1 + 2 * ((n + per - 1) // per), (a, d, m, launches)
        keep = np.all((cols >= 0) & (cols < np.array(doms)[:, None]), axis=0)
        q = O.canonical_query(attrs, edges)
        co = O.draw_coefficients(4321 + d, d, q.n_comp, len(q.edges))
        ref = O.sketch_relation(q, co, 0, cols[:, keep], None, m, threads=16)
        assert np.array_equal(got, ref), (a, d, m)


@pytest.mark.parametrize("m,d", [(1 << 12, 13), (1 << 16, 3)])
def test_partitioned_update_heavy_bins(m, d, monkeypatch):
    """Two heavy bins per row: 3e6 tuples of which 45 % carry one key pair and 45 % another,
    so that every CTA's range adds about 9000 same-sign items to one shared counter of every
    row while the rest spread over the row.  Bit-exact against the oracle (counters past 10^6
    in magnitude), at one part per row (m = 2^12, d = 13: too large for one CTA's shared
    memory) and two (m = 2^16)."""
    monkeypatch.setenv("SK_KEY_TABLE", "1")
    n, a = 3_000_000, 2
    doms = [5000, 7000]
    cols = np.stack([synth.zipf_keys(n, 1.1, doms[u], 700 + u).numpy() for u in range(a)])
    rng = np.random.default_rng(5)
    pick = rng.random(n)
    cols[0, pick < 0.45], cols[1, pick < 0.45] = 0, 0
    heavy2 = (pick >= 0.45) & (pick < 0.9)
    cols[0, heavy2], cols[1, heavy2] = 17, 4242
    attrs, edges = _star(a)
    L0 = pkg.sk_launch_count()
    got = _run(attrs, edges, m, d, 99, cols, None, doms)
    assert pkg.sk_launch_count() - L0 == 3   # table build, phase 1, phase 2
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(99, d, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, cols, None, m, threads=16)
    assert np.abs(ref).max() > 1_000_000
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("a,d,m,n,window,force,same", [
    (2, 16, 1 << 20, 1_200_007, 0, False, False),      # the chain's inner relations: 2 attributes, d = 16
    (1, 9, 1 << 19, 600_001, 0, False, False),
    (2, 16, 1 << 20, 1_100_000, 300_000, False, False),  # several windows, ragged last one
    (3, 5, 1 << 17, 300_007, 0, True, False),
    (5, 13, 1 << 18, 200_003, 65_536, True, False),
    (1, 1, 1 << 24, 100_001, 0, True, False),          # 512 parts per row
    (2, 16, 1 << 20, 1_048_583, 0, False, True),       # every tuple the same keys: one part per row
    (4, 10, 1 << 21, 50_000, 0, True, False),          # d not a multiple of the record vector
])
def test_wide_partitioned_update_bit_exact(a, d, m, n, window, force, same, monkeypatch):
    """Unit-weight batches with declared domains into sketches wider than 2^16 bins (the
    chain of eight relations at m = 2^20, d = 16) take the wide partitioned update: items
    with per-chunk part counts, a scan, a scatter by part of 2^15 bins, shared-memory
    accumulation per (row, part).  By default only for sketches larger than 32 MiB with at
    least m tuples; SK_PART_UPDATE=2 forces it for the smaller cases.  Keys at the table's
    first and last records and outside the domain (skipped and reported); one window or
    several; all tuples alike (every row's items in one part).  The launch count shows which
    path ran: the table build plus seven launches per window."""
    monkeypatch.setenv("SK_KEY_TABLE", "1")
    if force:
        monkeypatch.setenv("SK_PART_UPDATE", "2")
    else:
        monkeypatch.delenv("SK_PART_UPDATE", raising=False)
    if window:
        monkeypatch.setenv("SK_PART_WINDOW", str(window))
    else:
        monkeypatch.delenv("SK_PART_WINDOW", raising=False)
    rng = np.random.default_rng(a * 131 + d + m % 977)
    doms = [int(x) for x in rng.integers(1000, 300_000, size=a)]
    cols = np.stack([synth.zipf_keys(n, 1.2, doms[u], 500 + u).numpy() for u in range(a)])
    if same:
        cols[:, :] = cols[:, :1]
    else:
        cols[0, :5] = [0, doms[0] - 1, -1, doms[0], 3]
        cols[a - 1, n - 3:] = [doms[a - 1], 0, doms[a - 1] - 1]
    attrs, edges = _star(a)
    L0 = pkg.sk_launch_count()
    got = _run(attrs, edges, m, d, 777 + a, cols, None, doms)
    launches = pkg.sk_launch_count() - L0
    per = window if window else n
    per = (per + 255) // 256 * 256
    assert launches == 1 + 7 * ((n + per - 1) // per), launches
    keep = np.all((cols >= 0) & (cols < np.array(doms)[:, None]), axis=0)
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(777 + a, d, q.n_comp, len(q.edges))
    ref = O.sketch_relation(q, co, 0, cols[:, keep], None, m, threads=16)
    assert np.array_equal(got, ref)
