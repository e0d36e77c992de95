"""Per-tuple updates whose int64 counters exceed the L2 share of one pass run the rows in
several passes over the batch (SK_ROW_PASS_MB sets the share): the counters stay
bit-exact with the oracle for every split, an uneven last pass included."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2402_15953_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_15953_gb300 import build
    build.build()
    O.build()


# (SK_ROW_PASS_MB, m, d): 1 MiB at 2^16 x 5 rows -> passes of 2, 2, 1 rows; 0 = one pass;
# 48 MiB at 2^20 x 8 rows (64 MiB) -> two passes of 4 rows; the default (unset) at 2^20 x 9
# rows (72 MiB) -> passes of 5 and 4 rows; 50021 x 3 rows at 1 MiB -> 2 and 1 rows
@pytest.mark.parametrize("mb,m,d", [("1", 1 << 16, 5), ("0", 1 << 16, 5), ("48", 1 << 20, 8), (None, 1 << 20, 9),
                                    ("1", 50021, 3)])
@pytest.mark.parametrize("wide", [False, True])
def test_row_passes_bit_exact(mb, m, d, wide, monkeypatch):
    if mb is None:
        monkeypatch.delenv("SK_ROW_PASS_MB", raising=False)
    else:
        monkeypatch.setenv("SK_ROW_PASS_MB", mb)
    rng = np.random.default_rng(m + d + int(wide))
    attrs, edges = [1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)]
    n = 20_000
    hi = 1 << 40 if wide else 5000
    cols = rng.integers(0, hi, size=(2, n)).astype(np.int64)
    w = rng.choice(np.array([-2, -1, 1, 3], dtype=np.int64), size=n)
    s = pkg.SketchSet(attrs, edges, m, d, 77)
    s.update(1, torch.as_tensor(cols).cuda(), torch.as_tensor(w).cuda())
    got = s.counters[1].cpu().numpy()
    s.close()
    q = O.canonical_query(attrs, edges)
    co = O.draw_coefficients(77, d, q.n_comp, len(q.edges))
    want = O.sketch_relation(q, co, 1, cols, w, m, threads=16)
    assert np.array_equal(got, want)
