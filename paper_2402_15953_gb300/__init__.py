"""GB300 (sm_103a) convolved Count sketches for multi-join cardinality estimation.

Heddes, Nunes, Givargis, Nicolau, "Convolution and Cross-Correlation of Count
Sketches Enables Fast Cardinality Estimation of Multi-Join Queries", PACMMOD
2024.  The computation lives in libsketch.so (C ABI, include/sketch.h; CUDA
kernels under csrc/); this module only marshals arguments to it with ctypes.
PyTorch is used for device memory and streams.

The C functions are exposed under their own names (sk_sketch_create,
sk_sketch_update_batch, sk_sketch_merge, sk_estimate_join, ...), each raising
SketchError on a non-zero status; SketchSet wraps a handle together with its
torch-owned counters, UpdatePlan a batched plan (sk_update_plan_*), SketchFamily
a sub-query family (sk_family_*), estimate_many the many-set estimate, and
serve.SketchServer the native serving loop (sk_server_*).
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsketch.so")

SK_MAX_ROWS = 64

STATUS = {
    0: "SK_OK", -1: "SK_ERR_INVALID_ARG", -2: "SK_ERR_CYCLIC_QUERY", -3: "SK_ERR_DISCONNECTED_QUERY",
    -4: "SK_ERR_SELF_EDGE", -5: "SK_ERR_UNSUPPORTED_WIDTH", -6: "SK_ERR_BUFFER_TOO_SMALL",
    -7: "SK_ERR_MISMATCH", -8: "SK_ERR_KEY_OUT_OF_DOMAIN", -9: "SK_ERR_TIMEOUT", -10: "SK_ERR_CUDA",
    -11: "SK_ERR_OVERFLOW", -12: "SK_ERR_INEXACT", -13: "SK_ERR_NO_MEMORY", -14: "SK_ERR_SCRATCH_TOO_SMALL",
          -15: "SK_ERR_OVER_BUDGET",
}
globals().update({name: code for code, name in STATUS.items()})


class SketchError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class sk_edge(ctypes.Structure):
    _fields_ = [("rel_a", ctypes.c_int32), ("attr_a", ctypes.c_int32),
                ("rel_b", ctypes.c_int32), ("attr_b", ctypes.c_int32)]


class sk_query(ctypes.Structure):
    _fields_ = [("num_relations", ctypes.c_int32), ("num_join_attrs", ctypes.POINTER(ctypes.c_int32)),
                ("num_edges", ctypes.c_int32), ("edges", ctypes.POINTER(sk_edge))]


class sk_i256(ctypes.Structure):
    _fields_ = [("limb", ctypes.c_uint64 * 4)]

    def value(self) -> int:
        v = 0
        for k in range(4):
            v |= int(self.limb[k]) << (64 * k)
        return v - (1 << 256) if v >> 255 else v


class sk_estimate(ctypes.Structure):
    _fields_ = [("median", sk_i256), ("median_i64", ctypes.c_int64), ("fits_i64", ctypes.c_int32),
                ("d", ctypes.c_int32), ("median_f64", ctypes.c_double), ("mid_mean_f64", ctypes.c_double),
                ("max_residual", ctypes.c_double), ("max_limbs", ctypes.c_int32), ("limb_bits", ctypes.c_int32),
                ("corr_steps", ctypes.c_int32), ("retries", ctypes.c_int32), ("row", sk_i256 * SK_MAX_ROWS)]


class sk_update_item(ctypes.Structure):
    _fields_ = [("set", ctypes.c_void_p), ("relation", ctypes.c_int32), ("n_rows", ctypes.c_int64),
                ("dev_cols", ctypes.c_void_p), ("col_stride", ctypes.c_int64), ("dev_weights", ctypes.c_void_p)]


class sk_update_plan_config(ctypes.Structure):
    _fields_ = [("chunk_tuples", ctypes.c_int32), ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("smem_max_counters", ctypes.c_int32), ("smem16_max_counters", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["sk_sketch_bytes", "sk_sketch_create", "sk_sketch_update_batch", "sk_sketch_merge",
           "sk_estimate_join", "sk_sync", "sk_sketch_destroy", "sk_status_string", "sk_sketch_info",
           "sk_get_coefficients", "sk_set_coefficients", "sk_sketch_reset", "sk_launch_count",
           "sk_estimate_join_noalloc", "sk_sketch_set_estimator", "sk_update_plan_create", "sk_update_plan_run", "sk_update_plan_zero", "sk_update_plan_get_config",
           "sk_server_create", "sk_server_register_set", "sk_server_submit_update", "sk_server_submit_estimate",
           "sk_server_result", "sk_server_hold", "sk_server_pending", "sk_server_drain", "sk_server_stats",
           "sk_server_destroy",
           "sk_update_plan_set_config", "sk_update_plan_autotune", "sk_update_plan_destroy",
           "sk_family_create", "sk_family_update_batch", "sk_family_estimate", "sk_family_set_estimator",
           "sk_family_info", "sk_family_view", "sk_family_copy_sketch", "sk_family_reset", "sk_family_sync",
           "sk_family_destroy", "sk_estimate_many"]

_lib = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Loads libsketch.so (build it with paper_2402_15953_gb300.build.build()).  There is
    no fallback: without the library nothing in this package runs."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libsketch.so not built ({p}); run python -m paper_2402_15953_gb300.build")
    L = ctypes.CDLL(p)
    vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    qp = ctypes.POINTER(sk_query)
    L.sk_sketch_bytes.argtypes = [qp, i64, i32, ctypes.POINTER(sz)]
    L.sk_sketch_create.argtypes = [qp, i64, i32, u64, vp, sz, vp, ctypes.POINTER(vp)]
    L.sk_sketch_update_batch.argtypes = [vp, i32, i64, vp, i64, vp, vp, vp]
    L.sk_sketch_merge.argtypes = [vp, vp, vp]
    L.sk_estimate_join.argtypes = [vp, ctypes.POINTER(sk_estimate), vp]
    L.sk_estimate_join_noalloc.argtypes = [vp, ctypes.POINTER(sk_estimate), vp]
    L.sk_sketch_set_estimator.argtypes = [vp, i32]
    L.sk_sync.argtypes = [vp, vp]
    L.sk_sketch_destroy.argtypes = [vp]
    L.sk_status_string.argtypes = [i32]
    L.sk_status_string.restype = ctypes.c_char_p
    L.sk_sketch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                 ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.sk_get_coefficients.argtypes = [vp, ctypes.POINTER(u64), sz]
    L.sk_set_coefficients.argtypes = [vp, ctypes.POINTER(u64), sz, vp]
    L.sk_sketch_reset.argtypes = [vp, vp]
    L.sk_update_plan_create.argtypes = [ctypes.POINTER(sk_update_item), i32, ctypes.POINTER(vp)]
    L.sk_update_plan_run.argtypes = [vp, vp]
    L.sk_update_plan_zero.argtypes = [vp, vp]
    L.sk_server_create.argtypes = [i64, i32, i32, i32, ctypes.POINTER(vp)]
    L.sk_server_register_set.argtypes = [vp, i32, vp]
    L.sk_server_submit_update.argtypes = [vp, i32, i32, i64, vp, i64, vp, vp, ctypes.POINTER(i64)]
    L.sk_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.sk_server_submit_estimate.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.sk_server_result.argtypes = [vp, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(sk_estimate),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.sk_server_hold.argtypes = [vp, i32]
    L.sk_server_pending.argtypes = [vp, ctypes.POINTER(i64)]
    L.sk_server_drain.argtypes = [vp]
    L.sk_server_destroy.argtypes = [vp]
    L.sk_update_plan_get_config.argtypes = [vp, ctypes.POINTER(sk_update_plan_config)]
    L.sk_update_plan_set_config.argtypes = [vp, ctypes.POINTER(sk_update_plan_config)]
    L.sk_update_plan_autotune.argtypes = [vp, vp, ctypes.POINTER(sk_update_plan_config), ctypes.POINTER(ctypes.c_double)]
    L.sk_update_plan_destroy.argtypes = [vp]
    L.sk_family_create.argtypes = [qp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), i64, i32, u64, vp,
                                   ctypes.POINTER(vp)]
    L.sk_family_update_batch.argtypes = [vp, i32, i64, vp, i64, vp, vp, vp]
    L.sk_family_estimate.argtypes = [vp, ctypes.POINTER(sk_estimate), vp]
    L.sk_family_set_estimator.argtypes = [vp, i32]
    L.sk_family_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(sz)]
    L.sk_family_view.argtypes = [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.sk_family_copy_sketch.argtypes = [vp, i32, i32, ctypes.POINTER(i64), vp]
    L.sk_family_reset.argtypes = [vp, vp]
    L.sk_family_sync.argtypes = [vp, vp]
    L.sk_family_destroy.argtypes = [vp]
    L.sk_estimate_many.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(sk_estimate), vp]
    L.sk_launch_count.argtypes = []
    L.sk_launch_count.restype = i64
    for name in EXPORTS:
        if name not in ("sk_status_string", "sk_launch_count"):
            getattr(L, name).restype = i32
    if path is None:
        _lib = L
    return L


def _check(st: int, where: str) -> None:
    if st != 0:
        raise SketchError(st, where)


def make_query(num_join_attrs: Sequence[int], edges: Sequence[Tuple[int, int, int, int]]):
    """Builds an sk_query; returns (query, keepalive) -- keep the second value alive while the
    query is in use."""
    attrs = (ctypes.c_int32 * len(num_join_attrs))(*[int(a) for a in num_join_attrs])
    earr = (sk_edge * max(1, len(edges)))(*[sk_edge(*[int(v) for v in e]) for e in edges])
    q = sk_query(len(num_join_attrs), attrs, len(edges), earr)
    return q, (attrs, earr)


# ---- the C ABI under its own names ----------------------------------------------------

def sk_sketch_bytes(query: sk_query, m: int, d: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().sk_sketch_bytes(ctypes.byref(query), m, d, ctypes.byref(out)), "sk_sketch_bytes")
    return out.value


def sk_sketch_create(query: sk_query, m: int, d: int, seed: int, dev_counters: int, nbytes: int,
                     stream: int) -> int:
    h = ctypes.c_void_p(0)
    _check(load().sk_sketch_create(ctypes.byref(query), m, d, seed & 0xFFFF_FFFF_FFFF_FFFF, dev_counters, nbytes,
                                   stream, ctypes.byref(h)), "sk_sketch_create")
    return h.value


def sk_sketch_update_batch(handle: int, relation: int, n_rows: int, dev_cols: int, col_stride: int,
                           dev_weights: Optional[int], domain_hint: Optional[Sequence[int]], stream: int) -> None:
    dom = None
    if domain_hint is not None:
        dom = (ctypes.c_int64 * len(domain_hint))(*[int(v) for v in domain_hint])
    _check(load().sk_sketch_update_batch(handle, relation, n_rows, dev_cols, col_stride, dev_weights or None,
                                         ctypes.cast(dom, ctypes.c_void_p) if dom is not None else None, stream),
           "sk_sketch_update_batch")


def sk_sketch_merge(dst: int, src: int, stream: int) -> None:
    _check(load().sk_sketch_merge(dst, src, stream), "sk_sketch_merge")


def sk_estimate_join(handle: int, stream: int) -> sk_estimate:
    out = sk_estimate()
    _check(load().sk_estimate_join(handle, ctypes.byref(out), stream), "sk_estimate_join")
    return out


def sk_sync(handle: int, stream: int) -> None:
    _check(load().sk_sync(handle, stream), "sk_sync")


def sk_sketch_destroy(handle: int) -> None:
    _check(load().sk_sketch_destroy(handle), "sk_sketch_destroy")


ESTIMATORS = {"fft64": 0, "ntt": 1, "fused": 2}


def sk_sketch_set_estimator(handle: int, estimator: str) -> None:
    """estimator: "fft64" (FP64 FFT, certified rounding), "ntt" (GF(2^64 - 2^32 + 1) transform) or
    "fused" (one product of spectra modulo CRT primes, for queries whose components all join two
    attributes; others as "ntt")."""
    _check(load().sk_sketch_set_estimator(handle, ESTIMATORS[estimator]), "sk_sketch_set_estimator")


def sk_sketch_reset(handle: int, stream: int) -> None:
    _check(load().sk_sketch_reset(handle, stream), "sk_sketch_reset")


def sk_launch_count() -> int:
    return int(load().sk_launch_count())


def sk_status_string(status: int) -> str:
    return load().sk_status_string(status).decode()


def sk_sketch_info(handle: int):
    r, m, d, c, e = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().sk_sketch_info(handle, ctypes.byref(r), ctypes.byref(m), ctypes.byref(d), ctypes.byref(c),
                                 ctypes.byref(e)), "sk_sketch_info")
    return r.value, m.value, d.value, c.value, e.value


def sk_get_coefficients(handle: int) -> List[List[int]]:
    _, _, d, c, e = sk_sketch_info(handle)
    row = 2 * c + 4 * e
    buf = (ctypes.c_uint64 * (d * row))()
    _check(load().sk_get_coefficients(handle, buf, d * row), "sk_get_coefficients")
    return [[int(buf[i * row + j]) for j in range(row)] for i in range(d)]


def sk_set_coefficients(handle: int, coeffs: Sequence[Sequence[int]], stream: int) -> None:
    flat = [int(v) for r in coeffs for v in r]
    buf = (ctypes.c_uint64 * len(flat))(*flat)
    _check(load().sk_set_coefficients(handle, buf, len(flat), stream), "sk_set_coefficients")


def sk_update_plan_create(items) -> int:
    """items: sequence of (set_handle, relation, n_rows, dev_cols, col_stride, dev_weights or None)."""
    arr = (sk_update_item * max(1, len(items)))(*[sk_update_item(h, r, n, c, st, w or None)
                                                   for (h, r, n, c, st, w) in items])
    out = ctypes.c_void_p(0)
    _check(load().sk_update_plan_create(arr, len(items), ctypes.byref(out)), "sk_update_plan_create")
    return out.value


def sk_update_plan_run(plan: int, stream: int) -> None:
    _check(load().sk_update_plan_run(plan, stream), "sk_update_plan_run")


def sk_update_plan_zero(plan: int, stream: int) -> None:
    _check(load().sk_update_plan_zero(plan, stream), "sk_update_plan_zero")


def sk_update_plan_get_config(plan: int) -> sk_update_plan_config:
    c = sk_update_plan_config()
    _check(load().sk_update_plan_get_config(plan, ctypes.byref(c)), "sk_update_plan_get_config")
    return c


def sk_update_plan_set_config(plan: int, chunk_tuples: int, threads: int, ctas_per_sm: int,
                              smem_max_counters: int, smem16_max_counters: int = 0) -> None:
    c = sk_update_plan_config(chunk_tuples, threads, ctas_per_sm, smem_max_counters, smem16_max_counters)
    _check(load().sk_update_plan_set_config(plan, ctypes.byref(c)), "sk_update_plan_set_config")


def sk_update_plan_autotune(plan: int, stream: int):
    c = sk_update_plan_config()
    ms = ctypes.c_double(0.0)
    _check(load().sk_update_plan_autotune(plan, stream, ctypes.byref(c), ctypes.byref(ms)), "sk_update_plan_autotune")
    return c.as_dict(), ms.value


def sk_update_plan_destroy(plan: int) -> None:
    _check(load().sk_update_plan_destroy(plan), "sk_update_plan_destroy")


# ---- convenience wrapper ---------------------------------------------------------------

class SketchSet:
    """The sketches of one join query: counters are a torch int64 tensor [r][d][m] on the
    current CUDA device; all work runs in libsketch.so on the current torch stream."""

    def __init__(self, num_join_attrs: Sequence[int], edges: Sequence[Tuple[int, int, int, int]], m: int,
                 d: int, seed: int, device=None, counters=None):
        import torch
        self._torch = torch
        self.num_join_attrs = list(num_join_attrs)
        self.edges = [tuple(e) for e in edges]
        self.m, self.d, self.seed = int(m), int(d), int(seed)
        self.query, self._keep = make_query(self.num_join_attrs, self.edges)
        nbytes = sk_sketch_bytes(self.query, self.m, self.d)
        r = len(self.num_join_attrs)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if counters is None:
            counters = torch.empty((r, self.d, self.m), dtype=torch.int64, device=dev)
        self.counters = counters
        self.handle = None
        self.handle = sk_sketch_create(self.query, self.m, self.d, self.seed, counters.data_ptr(), nbytes,
                                       self._stream())

    def _stream(self) -> int:
        return self._torch.cuda.current_stream(self.counters.device).cuda_stream

    def update(self, relation: int, cols, weights=None, domain: Optional[Sequence[int]] = None) -> None:
        """cols: int64 [a][n] CUDA tensor (attribute-major; the row stride is cols.stride(0));
        weights: int64 [n] or None (unit weights)."""
        t = self._torch
        assert cols.dtype == t.int64 and cols.is_cuda and cols.dim() == 2
        n = int(cols.shape[1])
        assert n == 0 or cols.stride(1) == 1
        wp = None
        if weights is not None:
            assert weights.dtype == t.int64 and weights.is_cuda and weights.is_contiguous()
            wp = weights.data_ptr()
        sk_sketch_update_batch(self.handle, relation, n, cols.data_ptr(), int(cols.stride(0)) if n else 0, wp,
                               domain, self._stream())

    def merge(self, other: "SketchSet") -> None:
        sk_sketch_merge(self.handle, other.handle, self._stream())

    def estimate(self) -> dict:
        e = sk_estimate_join(self.handle, self._stream())
        rows = [e.row[i].value() for i in range(e.d)]
        return {"median": e.median.value(), "rows": rows, "fits_i64": bool(e.fits_i64), "median_i64": e.median_i64,
                "median_f64": e.median_f64, "mid_mean_f64": e.mid_mean_f64, "max_residual": e.max_residual,
                "max_limbs": e.max_limbs, "limb_bits": e.limb_bits, "corr_steps": e.corr_steps,
                "retries": e.retries}

    def sync(self) -> None:
        sk_sync(self.handle, self._stream())

    def reset(self) -> None:
        sk_sketch_reset(self.handle, self._stream())

    def set_estimator(self, estimator: str) -> None:
        sk_sketch_set_estimator(self.handle, estimator)

    def coefficients(self) -> List[List[int]]:
        return sk_get_coefficients(self.handle)

    def set_coefficients(self, coeffs) -> None:
        sk_set_coefficients(self.handle, coeffs, self._stream())

    def close(self) -> None:
        if self.handle is not None:
            sk_sketch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UpdatePlan:
    """Many update batches applied by one persistent launch (sk_update_plan_*).  items are
    (SketchSet, relation, cols [a][n] int64 CUDA tensor, weights int64 [n] or None); the
    tensors are kept alive by the plan and may be refilled in place between runs."""

    def __init__(self, items):
        import torch
        self._torch = torch
        self._keep = []
        raw = []
        for (sset, rel, cols, w) in items:
            assert cols.dtype == torch.int64 and cols.is_cuda and cols.dim() == 2
            n = int(cols.shape[1])
            assert n == 0 or cols.stride(1) == 1
            if w is not None:
                assert w.dtype == torch.int64 and w.is_cuda and w.is_contiguous()
            self._keep.append((sset, cols, w))
            raw.append((sset.handle, rel, n, cols.data_ptr() if n else None, int(cols.stride(0)) if n else 0,
                        None if w is None else w.data_ptr()))
        self.handle = sk_update_plan_create(raw)

    def _stream(self) -> int:
        return self._torch.cuda.current_stream().cuda_stream

    def run(self) -> None:
        sk_update_plan_run(self.handle, self._stream())

    def zero(self) -> None:
        """Zeroes the counters of every (set, relation) the plan writes, in one launch."""
        sk_update_plan_zero(self.handle, self._stream())

    def config(self) -> dict:
        return sk_update_plan_get_config(self.handle).as_dict()

    def set_config(self, chunk_tuples: int, threads: int, ctas_per_sm: int, smem_max_counters: int,
                   smem16_max_counters: int = 0) -> None:
        sk_update_plan_set_config(self.handle, chunk_tuples, threads, ctas_per_sm, smem_max_counters,
                                  smem16_max_counters)

    def autotune(self):
        return sk_update_plan_autotune(self.handle, self._stream())

    def close(self) -> None:
        if self.handle is not None:
            sk_update_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- sub-query families (Section 3.4) ---------------------------------------------------

def sk_family_create(query: sk_query, subqueries: Sequence[Sequence[int]], m: int, d: int, seed: int,
                     stream: int) -> int:
    offs = [0]
    flat: List[int] = []
    for sub in subqueries:
        flat.extend(int(i) for i in sub)
        offs.append(len(flat))
    oa = (ctypes.c_int32 * len(offs))(*offs)
    ea = (ctypes.c_int32 * max(1, len(flat)))(*flat)
    h = ctypes.c_void_p(0)
    _check(load().sk_family_create(ctypes.byref(query), len(subqueries), oa, ea, m, d,
                                   seed & 0xFFFF_FFFF_FFFF_FFFF, stream, ctypes.byref(h)), "sk_family_create")
    return h.value


def sk_family_update_batch(handle: int, relation: int, n_rows: int, dev_cols: int, col_stride: int,
                           dev_weights: Optional[int], domain_hint: Optional[Sequence[int]], stream: int) -> None:
    dom = None
    if domain_hint is not None:
        dom = (ctypes.c_int64 * len(domain_hint))(*[int(v) for v in domain_hint])
    _check(load().sk_family_update_batch(handle, relation, n_rows, dev_cols, col_stride, dev_weights or None,
                                         ctypes.cast(dom, ctypes.c_void_p) if dom is not None else None, stream),
           "sk_family_update_batch")


def sk_family_info(handle: int) -> Tuple[int, int, int]:
    n, v, b = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_size_t(0)
    _check(load().sk_family_info(handle, ctypes.byref(n), ctypes.byref(v), ctypes.byref(b)), "sk_family_info")
    return n.value, v.value, b.value


def sk_family_estimate(handle: int, stream: int):
    n = sk_family_info(handle)[0]
    out = (sk_estimate * n)()
    _check(load().sk_family_estimate(handle, out, stream), "sk_family_estimate")
    return out


def sk_family_set_estimator(handle: int, estimator: str) -> None:
    _check(load().sk_family_set_estimator(handle, ESTIMATORS[estimator]), "sk_family_set_estimator")


def sk_family_view(handle: int, sub: int, rel_s: int) -> Tuple[int, int]:
    q, v = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().sk_family_view(handle, sub, rel_s, ctypes.byref(q), ctypes.byref(v)), "sk_family_view")
    return q.value, v.value


def sk_family_copy_sketch(handle: int, sub: int, rel_s: int, d: int, m: int, stream: int):
    import numpy as np
    out = np.zeros((d, m), dtype=np.int64)
    _check(load().sk_family_copy_sketch(handle, sub, rel_s, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        stream), "sk_family_copy_sketch")
    return out


def sk_family_reset(handle: int, stream: int) -> None:
    _check(load().sk_family_reset(handle, stream), "sk_family_reset")


def sk_family_sync(handle: int, stream: int) -> None:
    _check(load().sk_family_sync(handle, stream), "sk_family_sync")


def sk_family_destroy(handle: int) -> None:
    _check(load().sk_family_destroy(handle), "sk_family_destroy")


def _estimate_dict(e) -> dict:
    rows = [e.row[i].value() for i in range(e.d)]
    return {"median": e.median.value(), "rows": rows, "fits_i64": bool(e.fits_i64), "median_i64": e.median_i64,
            "median_f64": e.median_f64, "mid_mean_f64": e.mid_mean_f64, "max_residual": e.max_residual,
            "max_limbs": e.max_limbs, "limb_bits": e.limb_bits, "corr_steps": e.corr_steps, "retries": e.retries}


class SketchFamily:
    """The sketches of many sub-queries of one query (plan enumeration, Section 3.4): each
    sub-query is a list of indices into `edges`; relations are updated once, with Q's
    columns, and every sub-query is estimated by estimate()."""

    def __init__(self, num_join_attrs: Sequence[int], edges: Sequence[Tuple[int, int, int, int]],
                 subqueries: Sequence[Sequence[int]], m: int, d: int, seed: int):
        import torch
        self._torch = torch
        self.num_join_attrs = list(num_join_attrs)
        self.edges = [tuple(e) for e in edges]
        self.subqueries = [list(s) for s in subqueries]
        self.m, self.d, self.seed = int(m), int(d), int(seed)
        self.query, self._keep = make_query(self.num_join_attrs, self.edges)
        self.handle = None
        self.handle = sk_family_create(self.query, self.subqueries, self.m, self.d, self.seed, self._stream())

    def _stream(self) -> int:
        return self._torch.cuda.current_stream().cuda_stream

    def update(self, relation: int, cols, weights=None, domain: Optional[Sequence[int]] = None) -> None:
        t = self._torch
        assert cols.dtype == t.int64 and cols.is_cuda and cols.dim() == 2
        n = int(cols.shape[1])
        assert n == 0 or cols.stride(1) == 1
        wp = None
        if weights is not None:
            assert weights.dtype == t.int64 and weights.is_cuda and weights.is_contiguous()
            wp = weights.data_ptr()
        sk_family_update_batch(self.handle, relation, n, cols.data_ptr(), int(cols.stride(0)) if n else 0, wp,
                               domain, self._stream())

    def estimate(self) -> List[dict]:
        return [_estimate_dict(e) for e in sk_family_estimate(self.handle, self._stream())]

    def info(self) -> dict:
        n, v, b = sk_family_info(self.handle)
        return {"subqueries": n, "views": v, "counter_bytes": b}

    def view(self, sub: int, rel_s: int) -> Tuple[int, int]:
        return sk_family_view(self.handle, sub, rel_s)

    def sketch(self, sub: int, rel_s: int):
        return sk_family_copy_sketch(self.handle, sub, rel_s, self.d, self.m, self._stream())

    def set_estimator(self, estimator: str) -> None:
        sk_family_set_estimator(self.handle, estimator)

    def reset(self) -> None:
        sk_family_reset(self.handle, self._stream())

    def sync(self) -> None:
        sk_family_sync(self.handle, self._stream())

    def close(self) -> None:
        if self.handle is not None:
            sk_family_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- many sets in one call ---------------------------------------------------------------

def sk_estimate_many(handles: Sequence[int], stream: int):
    n = len(handles)
    hs = (ctypes.c_void_p * max(1, n))(*handles)
    out = (sk_estimate * max(1, n))()
    _check(load().sk_estimate_many(hs, n, out, stream), "sk_estimate_many")
    return [out[i] for i in range(n)]


def estimate_many(sets: Sequence["SketchSet"]) -> List[dict]:
    """The estimates of several SketchSets in one call (sk_estimate_many), on the current stream."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    return [_estimate_dict(e) for e in sk_estimate_many([s.handle for s in sets], stream)]
