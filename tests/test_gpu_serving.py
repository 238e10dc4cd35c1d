"""Continuous batching on the GPU: every request's result is the same alone and in
the mix (bitwise for the stacked tensor-core path, whose columns are computed
independently), and matches the FP64 oracle within the split-path bar."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2602_20870_gb300 import build, fgfrft as FG, serving as S
    build.build()
    sizes = [64, 128, 200]
    Fs = [W.rgg_gft(n, 100 + i) for i, n in enumerate(sizes)]
    plans = [FG.Plan(F, 16) for F in Fs]
    reqs = W.serving_requests(sizes, 48, rate_per_s=2000.0, seed=9, Ls=(8, 16), max_cols=12)
    return FG, S, sizes, Fs, plans, reqs


def _np(t):
    return t.detach().cpu().numpy()


def test_alone_equals_mixed_and_oracle(setup):
    FG, S, sizes, Fs, plans, reqs = setup
    # arrivals compressed so that requests meet in the queue and share launches
    srv = S.Server(plans, hbm_budget_bytes=1 << 30, max_cols=64, max_inflight_per_graph=2)
    mixed = S.replay(srv, reqs, time_scale=0.02, timeout_s=120)
    torch.cuda.synchronize()
    assert srv.launches < len(reqs)  # requests were batched
    alone = []
    for r in reqs:
        s1 = S.Server(plans, hbm_budget_bytes=1 << 30)
        f = s1.submit(r)
        s1.drain(timeout_s=60)
        alone.append(f.result())
    torch.cuda.synchronize()
    P = [O.projector(F) for F in Fs]
    bitwise = 0
    for r, a, m in zip(reqs, alone, mixed):
        assert a.error is None and m.error is None
        ya, ym = _np(a.Y), _np(m.Y)
        if np.array_equal(ya, ym):
            bitwise += 1
        assert np.linalg.norm(ya - ym) <= 1e-6 * np.linalg.norm(ya)
        if r.kind == "grad":
            assert np.linalg.norm(_np(a.D) - _np(m.D)) <= 1e-6 * np.linalg.norm(_np(a.D))
    assert bitwise == len(reqs)
    # oracle on a sample of each kind
    for kind in ("apply", "grad", "assemble"):
        for r, m in [(r, m) for r, m in zip(reqs, mixed) if r.kind == kind][:3]:
            F, Pr = Fs[r.graph], P[r.graph]
            if kind == "assemble":
                ref = O.fgfrft_power(F, float(r.alpha[0]), r.L, Pr)
                got = _np(m.Y)[0]
                assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
                continue
            ref = O.apply_power(F, r.alpha, r.L, r.X.T, Pr).T
            assert np.linalg.norm(_np(m.Y) - ref) / np.linalg.norm(ref) < 5e-5
            if kind == "grad":
                refd = O.dalpha_apply(F, r.alpha, r.L, r.X.T, Pr).T
                assert np.linalg.norm(_np(m.D) - refd) / np.linalg.norm(refd) < 5e-5


def test_small_budget_still_completes(setup):
    FG, S, sizes, Fs, plans, reqs = setup
    one = max(S.request_bytes(sizes[r.graph], r.kind, 1 if r.kind == "assemble" else r.X.shape[0]) for r in reqs)
    srv = S.Server(plans, hbm_budget_bytes=2 * one, max_cols=64)
    res = S.replay(srv, reqs[:20], time_scale=0.0, timeout_s=120)
    assert all(r.error is None for r in res)
    assert srv.max_reserved <= 2 * one
