"""The zero-allocation alpha-gradient entry point (fgfrft_grad_alpha_noalloc),
called through the C ABI, against the gradient the regular entry point
(fgfrft_grad) returns for the same G and dY/dalpha, on two calls in a row.
Self-contained, so it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest
import torch

from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def FG():
    from paper_2602_20870_gb300 import build, fgfrft
    build.build()
    return fgfrft


def _case(FG, F, L, B, seed):
    """(dY/dalpha, G, the regular entry point's gradient) for one plan and batch."""
    plan = FG.Plan(F, L)
    rng = np.random.default_rng(seed)
    N = F.shape[0]
    a = rng.uniform(-2, 2, size=B)
    X = torch.as_tensor(W.complex_normal((B, N), rng), dtype=torch.complex64).cuda()
    G = torch.as_tensor(W.complex_normal((B, N), rng), dtype=torch.complex64).cuda()
    _, D = plan.forward_dual(a, X, L, path="stacked_fp32")
    _, ga = plan.backward(a, G, D, L, need_x=False, path="stacked_fp32")
    torch.cuda.synchronize()
    return D, G, ga.cpu().numpy(), plan


def test_noalloc_matches_regular_gradient_on_two_calls(FG):
    # a small graph (one 1024-entry chunk per signal) and a 2500-node cyclic shift
    # (three chunks per signal), one call after the other through the same scratch
    D1, G1, ref1, p1 = _case(FG, W.tiny().F, 16, 37, 1)
    D2, G2, ref2, p2 = _case(FG, W.cyclic_shift(2500), 2, 5, 2)
    out1 = torch.full((37,), float("nan"), dtype=torch.float32, device="cuda")
    out2 = torch.full((5,), float("nan"), dtype=torch.float32, device="cuda")
    FG.grad_alpha_noalloc(G1, D1, out1)
    FG.grad_alpha_noalloc(G2, D2, out2)
    torch.cuda.synchronize()
    for out, ref in ((out1, ref1), (out2, ref2)):
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    # and again, in the other order, after the scratch holds the previous contents
    FG.grad_alpha_noalloc(G2, D2, out2)
    FG.grad_alpha_noalloc(G1, D1, out1)
    torch.cuda.synchronize()
    assert np.allclose(out1.cpu().numpy(), ref1, rtol=1e-5, atol=1e-5 * np.abs(ref1).max())
    assert np.allclose(out2.cpu().numpy(), ref2, rtol=1e-5, atol=1e-5 * np.abs(ref2).max())


def test_noalloc_rejects_sizes_beyond_its_scratch(FG):
    G = torch.zeros((2, 8), dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    lib = FG.load()
    import ctypes
    # B * ceil(N / 1024) above the fixed maximum: rejected before any launch
    rc = lib.fgfrft_grad_alpha_noalloc(ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                       FG.NOALLOC_MAX_PARTIALS + 1, 8, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == FG.ERR_UNSUPPORTED
