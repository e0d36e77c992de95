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


def test_batched_serving_and_many_argument_checks(lib):
    """Host-side argument checks of the batched, many-set and serving entry points (no
    GPU call is reached)."""
    import ctypes
    inv = pkg.SK_ERR_INVALID_ARG
    assert lib.sk_update_plan_zero(None, None) == inv
    assert lib.sk_update_plan_run(None, None) == inv
    assert lib.sk_estimate_many(None, -1, None, None) == inv
    assert lib.sk_estimate_many(None, 2, None, None) == inv
    assert lib.sk_estimate_many(None, 0, None, None) == 0
    nulls = (ctypes.c_void_p * 2)(None, None)
    out = (pkg.sk_estimate * 2)()
    assert lib.sk_estimate_many(nulls, 2, out, None) == inv
    h = ctypes.c_void_p()
    for budget, slots, workers in [(0, 1, 1), (1 << 20, 0, 1), (1 << 20, 1, 0), (1 << 20, 1, 65)]:
        assert lib.sk_server_create(budget, slots, workers, 0, ctypes.byref(h)) == inv
    assert lib.sk_server_create(1 << 20, 1, 1, 0, None) == inv
    rid, n = ctypes.c_int64(), ctypes.c_int64()
    fin = ctypes.c_int32()
    assert lib.sk_server_register_set(None, 0, None) == inv
    assert lib.sk_server_submit_update(None, 0, 0, 0, None, 0, None, None, ctypes.byref(rid)) == inv
    assert lib.sk_server_stats(None, None, None) == inv
    assert lib.sk_server_submit_estimate(None, 0, ctypes.byref(rid)) == inv
    assert lib.sk_server_result(None, 1, 0, ctypes.byref(fin), None, None, None, None) == inv
    assert lib.sk_server_hold(None, 1) == inv
    assert lib.sk_server_pending(None, ctypes.byref(n)) == inv
    assert lib.sk_server_drain(None) == inv
    assert lib.sk_server_destroy(None) == 0
    assert pkg.sk_status_string(-15) == "SK_ERR_OVER_BUDGET"
