"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, exports every
function include/sketch.h declares, and validates queries without touching a GPU."""
import os
import re

import pytest

import paper_2402_15953_gb300 as pkg
from paper_2402_15953_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pkg.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "sketch.h")).read()
    return sorted(set(re.findall(r"^(?:sk_status|const char\*|int64_t)\s+(sk_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert set(pkg.EXPORTS) <= set(names)


def test_status_strings(lib):
    for code, name in pkg.STATUS.items():
        assert pkg.sk_status_string(code) == name
    assert pkg.sk_status_string(12345) == "SK_ERR_UNKNOWN"


def test_sketch_bytes_and_query_validation(lib):
    q, keep = pkg.make_query([1, 2, 1], [(0, 0, 1, 0), (1, 1, 2, 0)])
    assert pkg.sk_sketch_bytes(q, 256, 5) == 3 * 5 * 256 * 8
    cases = [
        (([1, 1], [(0, 0, 0, 0)]), "SK_ERR_SELF_EDGE"),
        (([2, 2], [(0, 0, 1, 0), (0, 1, 1, 1)]), "SK_ERR_CYCLIC_QUERY"),
        (([1, 1, 1, 1], [(0, 0, 1, 0), (2, 0, 3, 0)]), "SK_ERR_DISCONNECTED_QUERY"),
        (([2, 1], [(0, 0, 1, 0)]), "SK_ERR_INVALID_ARG"),          # attribute without a join
        (([1], []), "SK_ERR_INVALID_ARG"),                          # one relation
        (([1, 1], [(0, 0, 1, 3)]), "SK_ERR_INVALID_ARG"),           # attribute out of range
        (([1, 1], [(0, 0, 1, 0), (1, 0, 0, 0)]), "SK_ERR_INVALID_ARG"),  # duplicate join
    ]
    for (attrs, edges), want in cases:
        q, keep = pkg.make_query(attrs, edges)
        with pytest.raises(pkg.SketchError) as e:
            pkg.sk_sketch_bytes(q, 16, 2)
        assert e.value.name == want, (attrs, edges)
    q, keep = pkg.make_query([1, 1], [(0, 0, 1, 0)])
    for m, d, want in [(0, 1, "SK_ERR_UNSUPPORTED_WIDTH"), ((1 << 30) + 1, 1, "SK_ERR_UNSUPPORTED_WIDTH"),
                       (16, 0, "SK_ERR_INVALID_ARG"), (16, 65, "SK_ERR_INVALID_ARG")]:
        with pytest.raises(pkg.SketchError) as e:
            pkg.sk_sketch_bytes(q, m, d)
        assert e.value.name == want


def test_fig3_query_is_accepted(lib):
    q, keep = pkg.make_query([1, 2, 1, 1], [(0, 0, 1, 0), (2, 0, 1, 0), (3, 0, 1, 1)])
    assert pkg.sk_sketch_bytes(q, 1 << 10, 3) == 4 * 3 * 1024 * 8


def test_null_handles_are_rejected(lib):
    assert lib.sk_sketch_destroy(None) == 0
    assert lib.sk_sync(None, None) == pkg.SK_ERR_INVALID_ARG
    assert lib.sk_sketch_merge(None, None, None) == pkg.SK_ERR_INVALID_ARG
    assert lib.sk_sketch_update_batch(None, 0, 0, None, 0, None, None, None) == pkg.SK_ERR_INVALID_ARG
