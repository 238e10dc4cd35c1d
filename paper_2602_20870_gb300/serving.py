"""Continuous-batching server over resident FGFRFT plans.

Requests (one graph, one kind, one order and truncation order, 1..64 signals)
arrive over time.  A scheduler loop, run on the host:

  1. moves arrived requests into the pending queue;
  2. polls the batches in flight (CUDA events) and completes their requests;
  3. for every graph whose stream has room, admits pending requests of that
     graph in arrival order while the HBM budget and the column cap allow,
     groups them by (kind, L) and launches one library call per group on the
     graph's own CUDA stream (apply: one stacked launch with per-column orders;
     grad: Y and dY/dalpha in one pass; assemble: all orders fused);
  4. repeats, so requests that arrive while others run are admitted as soon as
     slots and memory free up and their work overlaps on the device.

Every column's arithmetic is independent of the other columns of its launch
(per-column orders, per-column scaling, one output tile per CTA), so a result is
the same alone and in a batch.  Waits are bounded: a batch whose event has not
completed by its deadline fails its requests with a timeout.

The plan memory of each graph stays resident for the server's lifetime (the
paper's cached powers, Sec. III-G); admission counts only per-request memory.
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fgfrft as FG


@dataclass
class Graph:
    """A resident graph: its plan and its own stream."""
    plan: FG.Plan
    stream: torch.cuda.Stream


@dataclass
class Result:
    rid: int
    kind: str
    Y: torch.Tensor | None          # (cols, N) complex64, or (1, N, N) for "assemble"
    D: torch.Tensor | None          # dY/dalpha for "grad"
    arrival: float
    done: float
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Pending:
    req: object
    fut: Future
    arrival: float
    nbytes: int
    x: np.ndarray | None = None  # the request's signals as complex64 (cols, N), set at submit


@dataclass
class _Batch:
    graph: int
    kind: str
    L: int
    items: list
    event: torch.cuda.Event
    outputs: dict
    nbytes: int
    deadline: float
    launched: float = 0.0
    slot: int = -1  # the graph's pinned staging slot this batch's signals went through


def ncols(req) -> int:
    """Signal columns of a request (1 for "assemble")."""
    if req.kind == "assemble":
        return 1
    return req.cols if getattr(req, "cols", 0) else req.X.shape[0]


def request_bytes(N: int, kind: str, cols: int) -> int:
    """Device bytes a request holds while in flight (inputs, outputs, scratch share)."""
    if kind == "assemble":
        return 8 * N * N + 4096
    per = 8 * N * cols
    return per * (3 if kind == "grad" else 2) + 64 * cols + 4096


class Server:
    def __init__(self, plans: list, hbm_budget_bytes: int, max_cols: int = 1024,
                 max_inflight_per_graph: int = 2, deadline_s: float = 30.0, path: str = "auto",
                 stream_factory=None):
        make_stream = stream_factory or torch.cuda.Stream
        self.graphs = [Graph(p, make_stream()) for p in plans]
        self.budget = int(hbm_budget_bytes)
        self.max_cols = max_cols
        self.max_inflight = max_inflight_per_graph
        self.deadline_s = deadline_s
        self.path = path
        self.pending: deque[_Pending] = deque()
        self.inflight: list[_Batch] = []
        self.reserved = 0
        self.lock = threading.Lock()
        self.t0 = time.perf_counter()
        self.launches = 0
        self.max_reserved = 0
        # per graph: max_inflight pinned host slots of max_cols signals each; a batch's
        # signals are gathered into a free slot and reach the device in one copy, and the
        # slot is free again once the batch's event has completed
        self.slots = [None] * len(self.graphs)
        self.slot_busy = [[False] * max_inflight_per_graph for _ in self.graphs]

    # ------------------------------------------------------------------ client side
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req, arrival: float | None = None) -> Future:
        """Queue a request (workloads.Request); returns a Future of Result."""
        g = self.graphs[req.graph]
        N = g.plan.N
        if req.L > g.plan.L_max:
            raise ValueError("L exceeds the graph's stored L_max")
        p = _Pending(req, Future(), self.now() if arrival is None else arrival,
                     request_bytes(N, req.kind, ncols(req)))
        if p.nbytes > self.budget:
            p.fut.set_exception(MemoryError("request larger than the HBM budget"))
            return p.fut
        if ncols(req) > self.max_cols:
            p.fut.set_exception(ValueError("request has more signals than a batch holds"))
            return p.fut
        if req.kind != "assemble":
            # converted once here, by the submitting thread, not on the scheduler's launch path
            p.x = np.ascontiguousarray(np.asarray(req.X).reshape(-1, N), dtype=np.complex64)
        with self.lock:
            self.pending.append(p)
        return p.fut

    # ------------------------------------------------------------------ scheduler
    def _poll(self):
        done = []
        now = self.now()
        for b in self.inflight:
            if b.event.query():
                done.append(b)
            elif now > b.deadline:
                for it in b.items:
                    it.fut.set_result(Result(it.req.rid, b.kind, None, None, it.arrival, now,
                                             error="FGFRFT_ERR_TIMEOUT"))
                done.append(b)
                b.items = []
        for b in done:
            self.inflight.remove(b)
            self.reserved -= b.nbytes
            if b.slot >= 0:
                self.slot_busy[b.graph][b.slot] = False
            t = self.now()
            for it, out in zip(b.items, b.outputs["per_item"]):
                it.fut.set_result(Result(it.req.rid, b.kind, out[0], out[1], it.arrival, t))
        return len(done)

    def _admit(self):
        """Admit pending requests into batches, graph by graph, in arrival order."""
        launched = 0
        with self.lock:
            pend = list(self.pending)
        if not pend:
            return 0
        inflight_per_graph = {}
        for b in self.inflight:
            inflight_per_graph[b.graph] = inflight_per_graph.get(b.graph, 0) + 1
        taken = set()
        groups: dict = {}
        for p in pend:
            g = p.req.graph
            key = (g, p.req.kind, p.req.L)
            if key not in groups and inflight_per_graph.get(g, 0) >= self.max_inflight:
                continue  # this graph's stream already has enough batches queued
            if self.reserved + p.nbytes > self.budget:
                break  # keep arrival order under memory pressure
            if key not in groups:
                inflight_per_graph[g] = inflight_per_graph.get(g, 0) + 1
            cur = groups.setdefault(key, [])
            cols = sum(ncols(q.req) for q in cur)
            add = ncols(p.req)
            if cur and cols + add > self.max_cols:
                continue
            cur.append(p)
            self.reserved += p.nbytes
            taken.add(id(p))
        for (g, kind, L), items in groups.items():
            self._launch(g, kind, L, items)
            launched += 1
        with self.lock:
            self.pending = deque(p for p in self.pending if id(p) not in taken)
        self.max_reserved = max(self.max_reserved, self.reserved)
        return launched

    def _stage(self, g: int, items: list):
        """Gather the items' signals into a free pinned slot of graph g: (slot, pinned rows)."""
        N = self.graphs[g].plan.N
        if self.slots[g] is None:
            self.slots[g] = [torch.empty((self.max_cols, N), dtype=torch.complex64, pin_memory=True)
                             for _ in range(self.max_inflight)]
        slot = self.slot_busy[g].index(False)  # admission keeps at most max_inflight batches per graph
        self.slot_busy[g][slot] = True
        buf = self.slots[g][slot]
        view = buf.numpy()
        off = 0
        for it in items:
            c = it.x.shape[0]
            view[off:off + c] = it.x
            off += c
        return slot, buf[:off]

    def _launch(self, g: int, kind: str, L: int, items: list):
        graph = self.graphs[g]
        plan, stream = graph.plan, graph.stream
        nbytes = sum(it.nbytes for it in items)
        per_item = []
        slot = -1
        with torch.cuda.stream(stream):
            if kind == "assemble":
                alphas = np.array([float(it.req.alpha[0]) for it in items])
                Q = plan.assemble(alphas, L, stream=stream)
                per_item = [(Q[i:i + 1], None) for i in range(len(items))]
            else:
                slot, host = self._stage(g, items)
                X = torch.empty(host.shape, dtype=torch.complex64, device=plan.device)
                X.copy_(host, non_blocking=True)
                alphas = np.concatenate([np.asarray(it.req.alpha, dtype=np.float64) for it in items])
                if kind == "apply":
                    path = self.path if self.path != "auto" else "stacked"
                    if path == "stacked" and not plan.storage & FG.STORE_SPLIT_F16:
                        path = "stacked_fp32"
                    Y = plan.apply(alphas, X, L, path=path, stream=stream)
                    D = None
                else:
                    path = "stacked" if plan.storage & FG.STORE_SPLIT_F16 else "stacked_fp32"
                    Y, D = plan.forward_dual(alphas, X, L, path=path, stream=stream)
                off = 0
                for it in items:
                    c = ncols(it.req)
                    per_item.append((Y[off:off + c], None if D is None else D[off:off + c]))
                    off += c
            ev = torch.cuda.Event()
            ev.record(stream)
        self.launches += 1
        self.inflight.append(_Batch(g, kind, L, items, ev, {"per_item": per_item}, nbytes,
                                    self.now() + self.deadline_s, self.now(), slot))

    def step(self) -> bool:
        """One scheduler tick; returns True if anything happened."""
        a = self._poll()
        b = self._admit()
        return bool(a or b)

    def drain(self, timeout_s: float = 600.0):
        t_end = time.perf_counter() + timeout_s
        while (self.pending or self.inflight) and time.perf_counter() < t_end:
            if not self.step():
                time.sleep(50e-6)
        if self.pending or self.inflight:
            raise TimeoutError("server did not drain")


def replay(server: Server, requests, time_scale: float = 1.0, timeout_s: float = 600.0):
    """Feed requests at their arrival times (seconds x time_scale) and run the scheduler
    until all complete.  Returns the list of Results in request order."""
    futs = []
    i = 0
    n = len(requests)
    t_start = server.now()
    t_end = time.perf_counter() + timeout_s
    while (i < n or server.pending or server.inflight) and time.perf_counter() < t_end:
        now = server.now() - t_start
        while i < n and requests[i].arrival_s * time_scale <= now:
            futs.append(server.submit(requests[i], arrival=t_start + requests[i].arrival_s * time_scale))
            i += 1
        if not server.step():
            time.sleep(20e-6)
    if i < n or server.pending or server.inflight:
        raise TimeoutError("replay did not finish")
    return [f.result() for f in futs]


def sequential(plans: list, requests, time_scale: float = 1.0, path: str = "plain"):
    """The plain baseline: one request at a time on one stream, FP32 paths
    (assembly + CUDA-core GEMM for apply, stacked FP32 for grad).  Requests queue in
    arrival order; latency includes the queueing."""
    out = []
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    for r in requests:
        arr = r.arrival_s * time_scale
        while time.perf_counter() - t0 < arr:
            pass
        plan = plans[r.graph]
        if r.kind == "assemble":
            Q = plan.assemble([float(r.alpha[0])], r.L)
            Y, D = Q, None
        else:
            X = torch.as_tensor(r.X, dtype=torch.complex64).pin_memory().to("cuda", non_blocking=True)
            if r.kind == "apply":
                Y = plan.apply(r.alpha, X, r.L, path=path if plan.storage & FG.STORE_C64 else "stacked_fp32")
                D = None
            else:
                Y, D = plan.forward_dual(r.alpha, X, r.L, path="stacked_fp32")
        stream.synchronize()
        done = time.perf_counter() - t0
        out.append(Result(r.rid, r.kind, Y, D, arr, done))
    return out


def latency_stats(results) -> dict:
    lat = np.array([r.latency for r in results if r.error is None])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "count": 0}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "count": int(lat.size),
            "errors": int(sum(1 for r in results if r.error is not None))}
