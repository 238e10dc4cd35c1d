"""CUDA-graph capture of the hot path (Def. 2 applied as Y = Q X): a call captured once and
replayed reads the signals at replay time and matches the FP64 oracle, on the assembled,
stacked and plain paths, for a real and a complex operator.  Between replays eager calls
with other orders run on the same plan, so a replay that read its host tables from
reusable staging slots, or a stale work buffer, would fail."""
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
    fgfrft.load()
    return fgfrft


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


OPERATORS = {
    "rgg256": lambda: W.rgg_gft(256, 3).astype(np.complex128),  # real F
    "haar130": lambda: W.random_unitary(130, 3),                 # complex F, ragged tiles
}


@pytest.mark.parametrize("op", list(OPERATORS))
@pytest.mark.parametrize("path", ["auto", "stacked", "plain"])
def test_apply_graph_replay(FG, op, path):
    F = OPERATORS[op]()
    N, L = F.shape[0], 12
    P = O.projector(F)
    plan = FG.Plan(F, L)
    B = 192
    a = np.repeat([0.3, -0.7, 1.45], 64)  # three groups of 64 columns
    Xd = torch.as_tensor(W.complex_normal((B, N), np.random.default_rng(5)), dtype=torch.complex64,
                         device="cuda")
    Y = torch.empty_like(Xd)
    plan.apply(a, Xd, L, out=Y, path=path)  # outside the capture: work buffer, streams, attributes
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.apply(a, Xd, L, out=Y, path=path)
    tol = 1e-5 if path == "plain" else 5e-5
    for seed in (11, 12):
        X1 = W.complex_normal((B, N), np.random.default_rng(seed))
        Xd.copy_(torch.as_tensor(X1, dtype=torch.complex64))
        other = plan.apply(np.full(B, 0.9), Xd, L, path=path)  # eager: other orders, same work buffer
        g.replay()
        torch.cuda.synchronize()
        ref = O.apply_power(F, a, L, X1.T, P).T
        assert rel(Y.cpu().numpy(), ref) < tol, (op, path, seed)
        ref_other = O.apply_power(F, np.full(B, 0.9), L, X1.T, P).T
        assert rel(other.cpu().numpy(), ref_other) < tol, (op, path, seed)


def test_assemble_and_grad_graph_replay(FG):
    """fgfrft_assemble and fgfrft_grad (forward with dY/dalpha, backward with the adjoint and
    the alpha-gradient, Props. 2-3) captured and replayed on new inputs."""
    F = W.rgg_gft(256, 3).astype(np.complex128)
    N, L = F.shape[0], 12
    P = O.projector(F)
    plan = FG.Plan(F, L)
    orders = [0.37, -1.2, 0.8]
    B = 128
    a = np.repeat([0.43, -0.9], 64)
    Xd = torch.zeros((B, N), dtype=torch.complex64, device="cuda")
    Gd = torch.zeros((B, N), dtype=torch.complex64, device="cuda")
    Q = plan.assemble(orders, L)
    Yf, Df = plan.forward_dual(a, Xd, L)
    gX, ga = plan.backward(a, Gd, Df, L)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        Q = plan.assemble(orders, L)
        Yf, Df = plan.forward_dual(a, Xd, L)
        gX, ga = plan.backward(a, Gd, Df, L)
    rng = np.random.default_rng(21)
    X1, G1 = W.complex_normal((B, N), rng), W.complex_normal((B, N), rng)
    Xd.copy_(torch.as_tensor(X1, dtype=torch.complex64))
    Gd.copy_(torch.as_tensor(G1, dtype=torch.complex64))
    plan.apply(np.full(B, -0.3), Xd, L)  # eager call in between (other orders)
    g.replay()
    torch.cuda.synchronize()
    for k, ak in enumerate(orders):
        assert rel(Q[k].cpu().numpy(), O.fgfrft_power(F, ak, L, P)) < 1e-5
    assert rel(Yf.cpu().numpy(), O.apply_power(F, a, L, X1.T, P).T) < 5e-5
    Dref = O.dalpha_apply(F, a, L, X1.T, P).T
    assert rel(Df.cpu().numpy(), Dref) < 5e-5
    assert rel(gX.cpu().numpy(), O.apply_power(F, -a, L, G1.T, P).T) < 5e-5
    g_ref = np.real(np.sum(np.conj(G1) * Df.cpu().numpy().astype(np.complex128), axis=1))
    assert np.allclose(ga.cpu().numpy(), g_ref, rtol=1e-4, atol=1e-3 * np.abs(g_ref).max())
