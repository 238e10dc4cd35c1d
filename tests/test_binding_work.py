"""Host logic of the binding's work buffer (no GPU): a call first runs with the cached
buffer and sizes it (fgfrft_work_bytes, a pass over the orders) only when there is none
or the call reports it too small; an argument error that is not about the size is
returned as it is, without a second call.  Each stream has its own buffer, so calls
on two streams never share scratch."""
import numpy as np
import torch

from paper_2602_20870_gb300 import fgfrft as FG


class FakeLib:
    def __init__(self, need):
        self.need = need
        self.sized = 0

    def fgfrft_work_bytes(self, h, op, alpha, count, L, flags):
        self.sized += 1
        return self.need


def make_plan(monkeypatch, need):
    lib = FakeLib(need)
    monkeypatch.setattr(FG, "_lib", lambda: lib)
    plan = FG.Plan.__new__(FG.Plan)
    plan._h, plan._works, plan.device = None, {}, torch.device("cpu")
    return plan, lib


def test_first_call_sizes_the_buffer(monkeypatch):
    plan, lib = make_plan(monkeypatch, 1000)
    seen = []
    rc = plan._with_work(FG.OP_APPLY, np.zeros(4), 4, 3, 0, lambda w: seen.append(w.numel()) or FG.OK)
    assert rc == FG.OK and seen == [1000] and lib.sized == 1


def test_cached_buffer_is_used_without_sizing(monkeypatch):
    plan, lib = make_plan(monkeypatch, 1000)
    plan._works[0] = torch.empty(4096, dtype=torch.uint8)
    seen = []
    rc = plan._with_work(FG.OP_APPLY, np.zeros(4), 4, 3, 0, lambda w: seen.append(w.numel()) or FG.OK)
    assert rc == FG.OK and seen == [4096] and lib.sized == 0


def test_too_small_buffer_grows_and_retries(monkeypatch):
    plan, lib = make_plan(monkeypatch, 8192)
    plan._works[0] = torch.empty(4096, dtype=torch.uint8)
    seen = []

    def call(w):
        seen.append(w.numel())
        return FG.OK if w.numel() >= 8192 else FG.ERR_INVALID_ARG

    assert plan._with_work(FG.OP_GRAD, np.zeros(4), 4, 3, 0, call) == FG.OK
    assert seen == [4096, 8192] and lib.sized == 2  # the retry's sizing and the buffer's


def test_other_argument_errors_are_not_retried(monkeypatch):
    plan, lib = make_plan(monkeypatch, 1000)
    plan._works[0] = torch.empty(4096, dtype=torch.uint8)
    seen = []
    rc = plan._with_work(FG.OP_APPLY, np.zeros(4), 4, 3, 0, lambda w: seen.append(1) or FG.ERR_INVALID_ARG)
    assert rc == FG.ERR_INVALID_ARG and seen == [1] and lib.sized == 1


def test_buffers_are_kept_per_stream(monkeypatch):
    plan, lib = make_plan(monkeypatch, 1000)
    # two streams, told apart by their handles (a fake stream object on the host)
    monkeypatch.setattr(plan, "_stream_of", lambda st: (st or 0, None))
    seen = {}
    plan._with_work(FG.OP_APPLY, np.zeros(4), 4, 3, 0, lambda w: seen.setdefault("a", w) is w and FG.OK, 11)
    plan._with_work(FG.OP_APPLY, np.zeros(4), 4, 3, 0, lambda w: seen.setdefault("b", w) is w and FG.OK, 22)
    assert seen["a"] is not seen["b"]
    assert set(plan._works) == {11, 22}
    # the first stream's buffer is used again without sizing
    n = lib.sized
    plan._with_work(FG.OP_APPLY, np.zeros(4), 4, 3, 0, lambda w: (w is seen["a"]) and FG.OK, 11)
    assert lib.sized == n
