"""Host-side logic of the continuous-batching server (no GPU): admission by memory
budget in arrival order, batching by (graph, kind, L), per-graph in-flight limits,
and deadline handling with a fake event that never completes."""
import types

import numpy as np
import pytest

from paper_2602_20870_gb300 import serving as S
from paper_2602_20870_gb300 import workloads as W


class FakeEvent:
    def __init__(self, done=True):
        self.done = done

    def query(self):
        return self.done


def fake_server(sizes, budget, done=True, **kw):
    plans = [types.SimpleNamespace(N=n, L_max=64, storage=3) for n in sizes]
    srv = S.Server(plans, budget, stream_factory=lambda: None, **kw)
    srv.launched = []

    def launch(g, kind, L, items):
        srv.launched.append((g, kind, L, [it.req.rid for it in items]))
        per = [(None, None) for _ in items]
        srv.inflight.append(S._Batch(g, kind, L, items, FakeEvent(done), {"per_item": per},
                                     sum(it.nbytes for it in items), srv.now() + srv.deadline_s))
        srv.launches += 1

    srv._launch = launch
    return srv


def test_request_bytes():
    assert S.request_bytes(1024, "apply", 4) == 8 * 1024 * 4 * 2 + 64 * 4 + 4096
    assert S.request_bytes(1024, "grad", 4) == 8 * 1024 * 4 * 3 + 64 * 4 + 4096
    assert S.request_bytes(256, "assemble", 1) == 8 * 256 * 256 + 4096


def test_batches_group_by_graph_kind_and_L():
    reqs = W.serving_requests([64, 128], 40, rate_per_s=1e6, seed=3, Ls=(16, 32), max_cols=8)
    srv = fake_server([64, 128], 1 << 40)
    futs = [srv.submit(r) for r in reqs]
    srv.drain(timeout_s=10)
    assert all(f.done() for f in futs)
    seen = set()
    for g, kind, L, rids in srv.launched:
        for rid in rids:
            r = reqs[rid]
            assert (r.graph, r.kind, r.L) == (g, kind, L)
            seen.add(rid)
    assert seen == set(range(40))
    # one tick batches everything pending: far fewer launches than requests
    assert len(srv.launched) < 40


def test_admission_respects_budget_and_order():
    reqs = W.serving_requests([256], 30, rate_per_s=1e6, seed=4, Ls=(16,), max_cols=16)
    one = max(S.request_bytes(256, r.kind, 1 if r.kind == "assemble" else r.X.shape[0]) for r in reqs)
    budget = 2 * one
    srv = fake_server([256], budget, done=True, max_inflight_per_graph=8)
    for r in reqs:
        srv.submit(r)
    admitted = set()
    while srv.pending or srv.inflight:
        srv._admit()
        assert srv.reserved <= budget
        for b in list(srv.inflight):
            admitted.update(it.req.rid for it in b.items)
        # memory pressure never lets a later request overtake an earlier one
        assert admitted == set(range(len(admitted)))
        srv._poll()
    assert srv.max_reserved <= budget
    assert admitted == set(range(30))


def test_oversized_request_is_rejected():
    srv = fake_server([512], 1000)
    r = W.serving_requests([512], 1, rate_per_s=1.0, seed=1, max_cols=4)[0]
    f = srv.submit(r)
    with pytest.raises(MemoryError):
        f.result()


def test_deadline_fails_requests_of_a_stuck_batch():
    srv = fake_server([64], 1 << 40, done=False, deadline_s=0.0, max_inflight_per_graph=8)
    reqs = W.serving_requests([64], 5, rate_per_s=1e6, seed=2, max_cols=4)
    futs = [srv.submit(r) for r in reqs]
    srv._admit()
    srv._poll()
    res = [f.result(timeout=1) for f in futs]
    assert all(r.error == "FGFRFT_ERR_TIMEOUT" for r in res)
    assert not srv.inflight and srv.reserved == 0


def test_latency_stats():
    rs = [S.Result(i, "apply", None, None, 0.0, 0.001 * (i + 1)) for i in range(100)]
    st = S.latency_stats(rs)
    assert abs(st["p50_ms"] - 50.5) < 1e-6 and st["count"] == 100


def test_inflight_limit_per_graph_within_one_tick():
    reqs = W.serving_requests([64], 30, rate_per_s=1e6, seed=5, Ls=(8, 16, 32), max_cols=4)
    srv = fake_server([64], 1 << 40, done=False, max_inflight_per_graph=2)
    for r in reqs:
        srv.submit(r)
    srv._admit()
    assert len(srv.inflight) <= 2
