"""Parity at the full workload sizes, in the launch configurations bench.py times,
on sampled outputs the FP64 oracle computes one by one (its signal recursion needs
no stored powers)."""
import numpy as np
import pytest
import scipy.linalg
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_SPLIT = 5e-5


@pytest.fixture(scope="module")
def FG():
    from paper_2602_20870_gb300 import build, fgfrft
    build.build()
    return fgfrft


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_projector(F):
    """P_-1 from the oracle: the real eigenvalues certify r_-1 = 0 cheaply (then P = 0);
    otherwise the complex Schur route."""
    lam = scipy.linalg.eigvals(F.real if np.all(F.imag == 0) else F)
    if np.min(np.abs(lam + 1.0)) > 1e-6:
        return np.zeros(F.shape, dtype=np.complex128), 0
    sp = O.spectral(F)
    return O.projector(F, sp), sp.r_neg1


def test_image_graph_bench_configuration(FG):
    """The bench step: 64 orders x 256 signals through fgfrft_apply (fused assembly on the
    tensor cores + grouped tcgen05 GEMM); sampled groups against the oracle."""
    wl = W.image_graph()
    N, L = wl.N, wl.L
    plan = FG.Plan(wl.F, L)
    P, r = oracle_projector(wl.F)
    assert plan.r_neg1 == r
    X = torch.as_tensor(wl.X, dtype=torch.complex64).cuda()
    Y = plan.apply(wl.alpha, X, L).cpu().numpy()
    Yp = plan.apply(wl.alpha, X, L, path="plain").cpu().numpy()
    per = wl.meta["per_order"]
    cols = np.concatenate([g * per + np.arange(0, per, 37) for g in (0, 17, 42, 63)])
    ref = O.apply_power(wl.F, wl.alpha[cols], L, wl.X[cols].T, P).T
    assert rel(Y[cols], ref) < TOL_SPLIT
    assert rel(Yp[cols], ref) < TOL_FP32
    # fused assembly of all 64 orders (c64 output) against Algorithm 1 for two of them
    orders = wl.meta["orders"]
    Q = plan.assemble(orders, L)
    M = O.powers(wl.F, L, P)
    for g in (0, 63):
        Qr = O.fgfrft_power(wl.F, float(orders[g]), L, P, M)
        assert rel(Q[g].cpu().numpy(), Qr) < TOL_FP32


def test_point_cloud_dual_adjoint_and_fd(FG):
    """Point-cloud config: Y and dY/dalpha in one tensor-core pass, the adjoint, the
    alpha-gradient, and a central difference (h = 1e-3) of the FP32 path."""
    wl = W.point_cloud()
    N, L = wl.N, wl.L
    plan = FG.Plan(wl.F, L)
    P, r = oracle_projector(wl.F)
    assert plan.r_neg1 == r
    X = torch.as_tensor(wl.X, dtype=torch.complex64).cuda()
    rng = np.random.default_rng(3)
    G = W.complex_normal(wl.X.shape, rng)
    Gd = torch.as_tensor(G, dtype=torch.complex64).cuda()
    Y, D = plan.forward_dual(wl.alpha, X, L, path="stacked")
    gX, ga = plan.backward(wl.alpha, Gd, D, L, path="stacked")
    cols = np.arange(0, wl.B, 29)
    a = wl.alpha[cols]
    Yr = O.apply_power(wl.F, a, L, wl.X[cols].T, P).T
    Dr = O.dalpha_apply(wl.F, a, L, wl.X[cols].T, P).T
    assert rel(Y.cpu().numpy()[cols], Yr) < TOL_SPLIT
    assert rel(D.cpu().numpy()[cols], Dr) < TOL_SPLIT
    assert rel(gX.cpu().numpy()[cols], O.adjoint_apply(wl.F, a, L, G[cols].T, P).T) < TOL_SPLIT
    gr = O.grad_alpha(G[cols].T, Dr.T)
    assert np.allclose(ga.cpu().numpy()[cols], gr, rtol=TOL_SPLIT, atol=TOL_SPLIT * np.abs(gr).max())
    h = 1e-3
    Xs = X[cols]
    Yp = plan.apply(a + h, Xs, L, path="stacked_fp32").cpu().numpy()
    Ym = plan.apply(a - h, Xs, L, path="stacked_fp32").cpu().numpy()
    assert rel((Yp - Ym) / (2 * h), Dr) < 1e-3


@pytest.mark.slow
def test_precision_configuration(FG):
    """N = 4096, L = 64 (129 stored powers): per-column orders on the stacked tensor-core
    path and a shared order on the plain FP32 path, each against the oracle."""
    wl = W.precision()
    N, L = wl.N, wl.L
    P, r = oracle_projector(wl.F)
    plan = FG.Plan(wl.F, L)
    assert plan.r_neg1 == r
    X = torch.as_tensor(wl.X, dtype=torch.complex64).cuda()
    Y = plan.apply(wl.alpha, X, L, path="stacked").cpu().numpy()
    Ys = plan.apply([0.37], X, L, path="plain").cpu().numpy()
    cols = np.arange(0, wl.B, 97)
    ref = O.apply_power(wl.F, wl.alpha[cols], L, wl.X[cols].T, P).T
    assert rel(Y[cols], ref) < TOL_SPLIT
    refs = O.apply_power(wl.F, 0.37, L, wl.X[cols].T, P).T
    assert rel(Ys[cols], refs) < TOL_FP32
