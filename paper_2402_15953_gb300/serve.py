"""Continuous-batching request loop over live sketch sets resident on one GPU.

Requests
  - update(set_id, relation, cols, weights): Algorithm 2 for one batch of tuples
    (host int64 [a][n] columns, copied to the device by the server);
  - estimate(set_id): Algorithm 3 and the median over rows for that set.

The scheduling runs in libsketch.so (sk_server_*, native threads): every set keeps its
requests in arrival order, so an estimate sees exactly the updates of its set submitted
before it and results equal running the requests one by one; across sets, requests are
admitted as update slots, estimate workers and the HBM budget allow, and their work
overlaps on the device (updates staged on a copy stream and run on an update stream,
estimates on their workers' streams).  This module only marshals requests and results.
"""
from __future__ import annotations

import ctypes
import dataclasses
import threading
from typing import Dict, List, Optional

import torch

from . import STATUS, SketchError, SketchSet, _estimate_dict, load, sk_estimate


@dataclasses.dataclass
class Request:
    kind: str                      # "update" | "estimate"
    set_id: int
    arrival: float = 0.0           # seconds since the server started (native clock)
    relation: int = 0
    cols: Optional[torch.Tensor] = None     # host int64 [a][n] (page-locked for overlap)
    weights: Optional[torch.Tensor] = None  # host int64 [n] or None
    seq: int = 0                   # request id
    done: float = 0.0
    result: Optional[dict] = None
    error: Optional[str] = None
    event: threading.Event = dataclasses.field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _LiveSet:
    def __init__(self, sset: SketchSet):
        self.sset = sset


def _ck(status: int, what: str) -> None:
    if status != 0:
        raise SketchError(status, what)


class SketchServer:
    def __init__(self, hbm_budget_bytes: int = 32 << 30, update_slots: int = 8, estimate_workers: int = 4,
                 device=None, estimate_priority: bool = False):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._L = load()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _ck(self._L.sk_server_create(int(hbm_budget_bytes), int(update_slots), int(estimate_workers),
                                         1 if estimate_priority else 0, ctypes.byref(h)), "sk_server_create")
        self.handle = h.value
        self.sets: Dict[int, _LiveSet] = {}
        self.completed: List[Request] = []
        self._open: Dict[int, Request] = {}
        self._lock = threading.Lock()

    # ---- registration ---------------------------------------------------------------
    def register_set(self, set_id: int, num_join_attrs, edges, m: int, d: int, seed: int) -> bool:
        """Creates a resident sketch set; False (and nothing kept) when its counters do not
        fit in the remaining budget."""
        with torch.cuda.device(self.device):
            sset = SketchSet(num_join_attrs, edges, m, d, seed, device=self.device)
        torch.cuda.synchronize(self.device)
        st = self._L.sk_server_register_set(self.handle, int(set_id), sset.handle)
        if STATUS.get(st) == "SK_ERR_OVER_BUDGET":
            sset.close()
            return False
        _ck(st, "sk_server_register_set")
        self.sets[set_id] = _LiveSet(sset)
        return True

    # ---- submission -----------------------------------------------------------------
    def submit_update(self, set_id: int, relation: int, cols: torch.Tensor,
                      weights: Optional[torch.Tensor] = None, domain=None) -> Request:
        """Queues an update; domain: None or the relation's per-column exclusive key bounds
        (as SketchSet.update), copied at submission."""
        if cols.is_cuda:
            cols = cols.cpu()
        if cols.dtype != torch.int64 or cols.dim() != 2:
            raise ValueError("cols must be an int64 [a][n] tensor")
        if cols.shape[1] > 0 and cols.stride(1) != 1:
            cols = cols.contiguous()
        if weights is not None:
            if weights.is_cuda:
                weights = weights.cpu()
            weights = weights.contiguous()
        n = int(cols.shape[1])
        rid = ctypes.c_int64()
        req = Request("update", set_id, relation=relation, cols=cols, weights=weights)
        dom = None if domain is None else (ctypes.c_int64 * len(domain))(*[int(x) for x in domain])
        with self._lock:
            _ck(self._L.sk_server_submit_update(self.handle, int(set_id), int(relation), n,
                                                cols.data_ptr() if n else None, int(cols.stride(0)) if n else 0,
                                                None if weights is None else weights.data_ptr(),
                                                None if dom is None else ctypes.cast(dom, ctypes.c_void_p),
                                                ctypes.byref(rid)),
                "sk_server_submit_update")
            req.seq = rid.value
            self._open[req.seq] = req
        return req

    def submit_estimate(self, set_id: int) -> Request:
        rid = ctypes.c_int64()
        req = Request("estimate", set_id)
        with self._lock:
            _ck(self._L.sk_server_submit_estimate(self.handle, int(set_id), ctypes.byref(rid)),
                "sk_server_submit_estimate")
            req.seq = rid.value
            self._open[req.seq] = req
        return req

    # ---- results --------------------------------------------------------------------
    def _collect(self) -> None:
        fin, st = ctypes.c_int32(), ctypes.c_int32()
        est = sk_estimate()
        t_arr, t_done = ctypes.c_double(), ctypes.c_double()
        with self._lock:
            for rid in list(self._open):
                _ck(self._L.sk_server_result(self.handle, rid, 0, ctypes.byref(fin), ctypes.byref(st),
                                             ctypes.byref(est), ctypes.byref(t_arr), ctypes.byref(t_done)),
                    "sk_server_result")
                if not fin.value:
                    continue
                req = self._open.pop(rid)
                req.arrival, req.done = t_arr.value, t_done.value
                if st.value != 0:
                    req.error = STATUS.get(st.value, str(st.value))
                elif req.kind == "estimate":
                    req.result = _estimate_dict(est)
                self.completed.append(req)
                req.event.set()

    def hold(self, on: bool = True) -> None:
        """Pauses (on) or resumes admission; submitted requests queue while held."""
        _ck(self._L.sk_server_hold(self.handle, 1 if on else 0), "sk_server_hold")

    def stats(self) -> dict:
        """Update batches launched so far and the update requests they held."""
        b, u = ctypes.c_int64(), ctypes.c_int64()
        _ck(self._L.sk_server_stats(self.handle, ctypes.byref(b), ctypes.byref(u)), "sk_server_stats")
        return {"batches": int(b.value), "batched_updates": int(u.value)}

    def pending(self) -> int:
        n = ctypes.c_int64()
        _ck(self._L.sk_server_pending(self.handle, ctypes.byref(n)), "sk_server_pending")
        return int(n.value)

    def serve(self, until_idle: bool = True, poll_s: float = 0.0) -> None:
        """Waits (outside the interpreter lock) until every submitted request has finished,
        then fills in the results; with until_idle=False it only collects what has finished."""
        if until_idle:
            _ck(self._L.sk_server_drain(self.handle), "sk_server_drain")
        self._collect()

    def stop(self) -> None:
        pass

    def close(self) -> None:
        """Finishes every submitted request, collects the results and releases the server
        and its sets."""
        if self.handle:
            self.hold(False)
            self.serve(until_idle=True)
            self._L.sk_server_destroy(self.handle)
            self.handle = None
        for ls in self.sets.values():
            ls.sset.close()
        self.sets.clear()
