"""The zero-allocation alpha-gradient entry point (fgfrft_grad_alpha_noalloc),
called through the C ABI, against the FP64 oracle's gradient (Re sum conj(G) D per
signal, on the same G and dY/dalpha) and against the gradient the regular entry point
(fgfrft_grad) returns, on two calls in a row; and that a call leaves the device's free
memory unchanged.  Self-contained, so it passes alone in a fresh process and after the
other tests."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def FG():
    from paper_2602_20870_gb300 import build, fgfrft
    build.build()
    return fgfrft


def _oracle(G, D):
    """The oracle's gradient on the very float32 G and D the GPU reads (FP64 sums)."""
    g = G.cpu().numpy().astype(np.complex128).T
    d = D.cpu().numpy().astype(np.complex128).T
    return O.grad_alpha(g, d), np.sum(np.abs(g) * np.abs(d), axis=0)


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
    exact1, scale1 = _oracle(G1, D1)
    exact2, scale2 = _oracle(G2, D2)
    for out, ref, exact, scale in ((out1, ref1, exact1, scale1), (out2, ref2, exact2, scale2)):
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        # FP64 partial sums rounded once to float32: within float32 rounding of the exact sum
        assert np.all(np.abs(got - exact) <= 1e-6 * scale + 1e-7 * np.abs(exact))
        assert np.allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    # and again, in the other order, after the scratch holds the previous contents
    FG.grad_alpha_noalloc(G2, D2, out2)
    FG.grad_alpha_noalloc(G1, D1, out1)
    torch.cuda.synchronize()
    assert np.allclose(out1.cpu().numpy(), ref1, rtol=1e-5, atol=1e-5 * np.abs(ref1).max())
    assert np.allclose(out2.cpu().numpy(), ref2, rtol=1e-5, atol=1e-5 * np.abs(ref2).max())
    assert np.all(np.abs(out1.cpu().numpy() - exact1) <= 1e-6 * scale1 + 1e-7 * np.abs(exact1))


def test_noalloc_call_leaves_free_memory_unchanged(FG):
    """The entry point allocates nothing: the device's free memory (cudaMemGetInfo) is the
    same before and after a call (after one first call, which looks up the scratch
    address; torch's caching allocator is not involved in the call itself)."""
    rng = np.random.default_rng(9)
    G = torch.as_tensor(W.complex_normal((40, 300), rng), dtype=torch.complex64).cuda()
    D = torch.as_tensor(W.complex_normal((40, 300), rng), dtype=torch.complex64).cuda()
    out = torch.empty(40, dtype=torch.float32, device="cuda")
    FG.grad_alpha_noalloc(G, D, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    FG.grad_alpha_noalloc(G, D, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    exact, scale = _oracle(G, D)
    assert np.all(np.abs(out.cpu().numpy() - exact) <= 1e-6 * scale + 1e-7 * np.abs(exact))


def test_noalloc_rejects_sizes_beyond_its_scratch(FG):
    G = torch.zeros((2, 8), dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    lib = FG.load()
    import ctypes
    # B * ceil(N / 1024) above the fixed maximum: rejected before any launch
    rc = lib.fgfrft_grad_alpha_noalloc(ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                       FG.NOALLOC_MAX_PARTIALS + 1, 8, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == FG.ERR_UNSUPPORTED
