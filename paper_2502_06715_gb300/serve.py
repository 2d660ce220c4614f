"""Continuous-batching join server over device-resident indexes.

Relations are indexed once and stay in HBM.  A request names a query, the
relation bound to each of its binary atoms and, optionally, the values its
unary atoms restrict variables to (a selection pushed into the query,
Sec. 2); a request without a selection joins the relations as they are.  The loop admits queued requests while a stream slot is free and
the request's device footprint (``join_footprint``) fits in what is left of
the HBM budget; admitted requests run concurrently, one CUDA stream each, so
their kernels overlap on the device; a finished request frees its slot and
budget at once and the next queued one is admitted.  Arrival, admission
and completion times are recorded per request.

``serve_serial`` runs the same requests one at a time (FIFO) for the
baseline and for the "alone" results.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import Index, Query, build_unary_index, join_footprint, run_join, run_join_async


@dataclass
class Request:
    rid: int
    query: Query            # binary atoms first, then unary atoms over `restrict`
    relations: tuple        # relation name per binary atom
    restrict: np.ndarray | None  # values the unary atoms allow; None: no unary atoms
    arrival: float = 0.0    # seconds from the start of the run


@dataclass
class Outcome:
    rid: int
    count: int
    arrival: float
    admitted: float
    done: float

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def _selection_values(values) -> np.ndarray:
    """A request's selection as the unary builder needs it: uint32 values,
    strictly ascending (sorted and de-duplicated on the host, because the
    builder trusts its input order and takes the last value as the largest)."""
    return np.unique(np.asarray(values, dtype=np.uint32))


def _unary_index(values: np.ndarray | None, device, stream) -> Index | None:
    """The request's selection as a unary index, built on `stream` without
    waiting for the GPU (None without a selection)."""
    if values is None:
        return None
    v = _selection_values(values)
    d = torch.from_numpy(v.view(np.int32)).to(device)
    return build_unary_index(d, int(v[-1]) if v.shape[0] else 0, stream=stream)


@dataclass
class Server:
    indexes: dict                      # relation name -> Index (attr order 0)
    budget_bytes: int = 120 << 30
    max_inflight: int = 8
    device: str = "cuda"
    options: dict = field(default_factory=dict)
    _fp: dict = field(default_factory=dict, repr=False)  # footprint cache

    def _indexes(self, req: Request, unary: Index | None) -> list:
        # every atom after the binary ones is a unary atom over the request's values
        extra = len(req.query.atoms) - len(req.relations)
        if extra and unary is None:
            raise ValueError("a request with unary atoms needs its selection")
        return [self.indexes[n] for n in req.relations] + [unary] * extra

    def footprint(self, req: Request) -> int:
        """Device bytes the request may take.  Cached per (query, relations,
        size class of the selection): the class's largest selection (the next
        power of two, values up to the next power of two) stands in for the
        request's own, so the cached figure bounds every request of the class."""
        if req.restrict is None:
            cn = cv = -1
        else:
            n = max(1, int(req.restrict.shape[0]))
            top = int(req.restrict.max()) if req.restrict.shape[0] else 0
            cn, cv = 1 << (n - 1).bit_length(), (1 << max(1, top.bit_length())) - 1
        key = (req.query.n_vars, tuple(req.query.atoms), req.query.order, tuple(req.relations), cn, cv)
        fp = self._fp.get(key)
        if fp is None:
            stand_in = None if req.restrict is None else Index.from_stats(cn, cn, 0, cv, 0)
            fp = join_footprint(req.query, self._indexes(req, stand_in), **self.options)
            self._fp[key] = fp
        return fp

    def run(self, requests: list, realtime: bool = True) -> list:
        """Serve requests arriving at req.arrival (seconds from now)."""
        streams = collections.deque(torch.cuda.Stream(device=self.device) for _ in range(self.max_inflight))
        order = sorted(requests, key=lambda r: r.arrival)
        queue: collections.deque = collections.deque()
        inflight = []
        out = []
        budget = self.budget_bytes
        nxt = 0
        t0 = time.perf_counter()
        while nxt < len(order) or queue or inflight:
            now = time.perf_counter() - t0
            while nxt < len(order) and (not realtime or order[nxt].arrival <= now):
                queue.append(order[nxt])
                nxt += 1
            # admit while a slot and the budget allow (head of line first)
            while queue and streams:
                req = queue[0]
                fp = self.footprint(req)
                if fp > budget and inflight:
                    break
                queue.popleft()
                s = streams.popleft()
                with torch.cuda.stream(s):
                    unary = _unary_index(req.restrict, self.device, s)
                    pend = run_join_async(req.query, self._indexes(req, unary), stream=s, **self.options)
                    ev = torch.cuda.Event()
                    ev.record(s)
                budget -= fp
                inflight.append((req, s, unary, pend, ev, fp, time.perf_counter() - t0))
            # retire finished requests
            still = []
            for item in inflight:
                req, s, unary, pend, ev, fp, t_adm = item
                if ev.query():
                    c = pend.count()
                    if unary is not None:
                        unary.free()
                    out.append(Outcome(req.rid, c, req.arrival, t_adm, time.perf_counter() - t0))
                    budget += fp
                    streams.append(s)
                else:
                    still.append(item)
            inflight = still
            if not queue and inflight and (nxt >= len(order) or order[nxt].arrival > time.perf_counter() - t0):
                time.sleep(0)
        return out


def serve_serial(server: Server, requests: list) -> list:
    """One request at a time, FIFO by arrival; returns per-request service
    outcomes with arrival 0 (service time = done - admitted)."""
    out = []
    s = torch.cuda.Stream(device=server.device)
    for req in sorted(requests, key=lambda r: r.rid):
        t = time.perf_counter()
        with torch.cuda.stream(s):
            unary = _unary_index(req.restrict, server.device, s)
            c = run_join(req.query, server._indexes(req, unary), stream=s, **server.options).count
            if unary is not None:
                unary.free()
        s.synchronize()
        out.append(Outcome(req.rid, c, 0.0, t, time.perf_counter()))
    return out


def fifo_latencies(service: list, arrivals: list) -> list:
    """Latencies of a single FIFO server with the measured service times
    (exact for serial execution)."""
    free_at = 0.0
    lat = []
    for a, sv in sorted(zip(arrivals, service)):
        start = max(a, free_at)
        free_at = start + sv
        lat.append(free_at - a)
    return lat
