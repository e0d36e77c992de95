"""Continuous-batching request loop over live sketch sets resident on one GPU.

Requests
  - update(set_id, relation, cols, weights): Algorithm 2 for one batch of tuples
    (host int64 [a][n] columns, copied to the device by the server);
  - estimate(set_id): Algorithm 3 and the median over rows for that set.

Scheduling
  - Every set keeps its requests in arrival order.  An estimate of a set sees
    exactly the updates of that set that arrived before it; updates that arrive
    after it wait until the estimate has finished reading the counters.  Results
    are therefore identical to running the requests one by one (sketch updates are
    exact integer additions, order independent within a set's batch of updates).
  - Across sets nothing is serialised: the scheduler admits a request as soon as
    an update slot (a bounded number of in-flight update batches) or an estimate
    worker is free and its device memory fits the HBM budget, so newly arrived
    work joins the work already running on the device.
  - Updates are copied on a copy stream and run on an update stream; each
    estimate runs on its worker's own stream, after an event that marks the set's
    last admitted update.
  - Memory: the resident counters of every registered set, the staging buffer of
    every in-flight update and a per-estimate scratch allowance are charged
    against the budget; a request that does not fit waits.

All GPU work goes through the library's C ABI (SketchSet / sk_* calls).
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Deque, Dict, List, Optional

import torch

from . import SketchSet


@dataclasses.dataclass
class Request:
    kind: str                      # "update" | "estimate"
    set_id: int
    arrival: float                 # time.perf_counter() at submission
    relation: int = 0
    cols: Optional[torch.Tensor] = None     # host int64 [a][n] (pinned for overlap)
    weights: Optional[torch.Tensor] = None  # host int64 [n] or None
    seq: int = 0
    done: float = 0.0
    result: Optional[dict] = None
    error: Optional[str] = None
    event: threading.Event = dataclasses.field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _LiveSet:
    def __init__(self, sset: SketchSet, nbytes: int, est_bytes: int):
        self.sset = sset
        self.nbytes = nbytes
        self.est_bytes = est_bytes
        self.queue: Deque[Request] = collections.deque()
        self.estimating = False
        self.last_update: Optional[torch.cuda.Event] = None
        self.lock = threading.Lock()    # one estimate at a time per set (its scratch is per set)


class SketchServer:
    def __init__(self, hbm_budget_bytes: int = 32 << 30, update_slots: int = 8, estimate_workers: int = 4,
                 device=None, estimate_priority: bool = False):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.update_slots = int(update_slots)
        self.sets: Dict[int, _LiveSet] = {}
        self.lock = threading.Condition()
        self.copy_stream = torch.cuda.Stream(self.device)
        self.update_stream = torch.cuda.Stream(self.device)
        self.inflight_updates: List[tuple] = []
        self.est_free = int(estimate_workers)
        # estimate_priority schedules estimate kernels ahead of queued update work when SMs free
        # up; off by default: on the 64-set mix it raised the p99 at 90 % load (updates waited)
        pr = -1 if estimate_priority else 0
        self.est_streams = [torch.cuda.Stream(self.device, priority=pr) for _ in range(estimate_workers)]
        self.completed: List[Request] = []
        self._seq = 0
        self._stop = False
        self._threads: List[threading.Thread] = []

    # ---- registration ---------------------------------------------------------------
    def register_set(self, set_id: int, num_join_attrs, edges, m: int, d: int, seed: int) -> bool:
        """Creates a resident sketch set if its counters fit in the remaining budget."""
        r = len(num_join_attrs)
        nbytes = r * d * m * 8
        slots = max(2, r)
        est_bytes = (slots + 1) * d * m * 32 + 2 * d * 4 * m * 16 + (m // 2) * 16
        with self.lock:
            if self.used + nbytes > self.budget:
                return False
            self.used += nbytes
        with torch.cuda.device(self.device):
            sset = SketchSet(num_join_attrs, edges, m, d, seed, device=self.device)
        torch.cuda.synchronize(self.device)
        self.sets[set_id] = _LiveSet(sset, nbytes, est_bytes)
        return True

    # ---- submission -----------------------------------------------------------------
    def submit_update(self, set_id: int, relation: int, cols: torch.Tensor,
                      weights: Optional[torch.Tensor] = None) -> Request:
        req = Request("update", set_id, time.perf_counter(), relation, cols, weights)
        self._enqueue(req)
        return req

    def submit_estimate(self, set_id: int) -> Request:
        req = Request("estimate", set_id, time.perf_counter())
        self._enqueue(req)
        return req

    def _enqueue(self, req: Request) -> None:
        with self.lock:
            req.seq = self._seq
            self._seq += 1
            self.sets[req.set_id].queue.append(req)
            self.lock.notify_all()

    # ---- scheduling -----------------------------------------------------------------
    def _admit(self) -> bool:
        """One scheduling pass under self.lock; returns True if anything was admitted."""
        progressed = False
        # retire finished updates
        still = []
        for (ev, req, nbytes, bufs) in self.inflight_updates:
            if ev.query():
                self.used -= nbytes
                req.done = time.perf_counter()
                req.event.set()
                self.completed.append(req)
                progressed = True
            else:
                still.append((ev, req, nbytes, bufs))
        self.inflight_updates = still
        # admit in global arrival order across sets (head of each set's queue)
        heads = sorted((ls.queue[0].seq, sid) for sid, ls in self.sets.items() if ls.queue and not ls.estimating)
        for _, sid in heads:
            ls = self.sets[sid]
            while ls.queue and not ls.estimating:
                req = ls.queue[0]
                if req.kind == "update":
                    if len(self.inflight_updates) >= self.update_slots:
                        break
                    nbytes = req.cols.numel() * 8 + (0 if req.weights is None else req.weights.numel() * 8)
                    if self.used + nbytes > self.budget:
                        break
                    ls.queue.popleft()
                    self.used += nbytes
                    self._launch_update(ls, req, nbytes)
                    progressed = True
                else:
                    if self.est_free == 0 or self.used + ls.est_bytes > self.budget:
                        break
                    ls.queue.popleft()
                    self.used += ls.est_bytes
                    self.est_free -= 1
                    ls.estimating = True
                    t = threading.Thread(target=self._run_estimate, args=(ls, req), daemon=True)
                    self._threads.append(t)
                    t.start()
                    progressed = True
                    break
        return progressed

    def _launch_update(self, ls: _LiveSet, req: Request, nbytes: int) -> None:
        with torch.cuda.device(self.device):
            with torch.cuda.stream(self.copy_stream):
                dc = req.cols.to(self.device, non_blocking=True)
                dw = None if req.weights is None else req.weights.to(self.device, non_blocking=True)
                copied = torch.cuda.Event()
                copied.record(self.copy_stream)
            self.update_stream.wait_event(copied)
            with torch.cuda.stream(self.update_stream):
                ls.sset.update(req.relation, dc, dw)
                done = torch.cuda.Event()
                done.record(self.update_stream)
            dc.record_stream(self.update_stream)
            if dw is not None:
                dw.record_stream(self.update_stream)
        ls.last_update = done
        self.inflight_updates.append((done, req, nbytes, (dc, dw)))

    def _run_estimate(self, ls: _LiveSet, req: Request) -> None:
        with self.lock:
            stream = self.est_streams.pop()
        try:
            with torch.cuda.device(self.device), torch.cuda.stream(stream):
                if ls.last_update is not None:
                    stream.wait_event(ls.last_update)
                with ls.lock:
                    req.result = ls.sset.estimate()
        except Exception as e:  # reported on the request; the server keeps running
            req.error = repr(e)
        req.done = time.perf_counter()
        with self.lock:
            self.est_streams.append(stream)
            self.est_free += 1
            self.used -= ls.est_bytes
            ls.estimating = False
            self.completed.append(req)
            self.lock.notify_all()
        req.event.set()

    def pending(self) -> int:
        return sum(len(ls.queue) for ls in self.sets.values()) + len(self.inflight_updates) + \
            sum(1 for ls in self.sets.values() if ls.estimating)

    def serve(self, until_idle: bool = True, poll_s: float = 2e-5) -> None:
        """Runs the scheduler in the calling thread until no request is pending (or stop())."""
        while not self._stop:
            with self.lock:
                progressed = self._admit()
                idle = self.pending() == 0
                if idle and until_idle:
                    break
                if not progressed:
                    self.lock.wait(timeout=poll_s)

    def stop(self) -> None:
        with self.lock:
            self._stop = True
            self.lock.notify_all()

    def close(self) -> None:
        for t in self._threads:
            t.join()
        torch.cuda.synchronize(self.device)
        for ls in self.sets.values():
            ls.sset.close()
        self.sets.clear()
