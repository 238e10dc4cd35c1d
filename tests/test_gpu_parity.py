"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs.  Bars: relative Frobenius error <= 1e-5 for the
FP32 paths, <= 5e-5 for the split-precision tensor-core paths."""
import math

import numpy as np
import pytest
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
    fgfrft.load()
    assert torch.cuda.is_available()
    return fgfrft


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex64, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


class Case:
    def __init__(self, name, F, L_max):
        self.name, self.F, self.L_max = name, F, L_max
        self.sp = O.spectral(F)
        self.P = O.projector(F, self.sp)


def cases():
    yield Case("tiny", W.tiny().F, 16)
    yield Case("tiny-flip", W.tiny(flip_one=True).F, 16)
    yield Case("haar65", W.random_unitary(65, 3), 9)
    yield Case("dft64", W.dft_matrix(64), 6)
    yield Case("shift96", W.cyclic_shift(96), 7)


CASES = list(cases())


@pytest.fixture(scope="module")
def plans(FG):
    return {c.name: FG.Plan(c.F, c.L_max) for c in CASES}


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_precompute_projector_and_powers(FG, plans, case):
    plan = plans[case.name]
    assert plan.r_neg1 == case.sp.r_neg1
    # real F (the Laplacian GFTs, the cyclic shift) takes the real-operator tensor paths
    assert plan.real == bool(np.all(case.F.imag == 0))
    P = host(plan.block(case.L_max + 1))
    assert np.abs(P - case.P).max() < 2e-6
    M = O.powers(case.F, case.L_max, case.P)
    for l in sorted({-case.L_max, -1, 0, 1, case.L_max}):
        ref = M[l] if l >= 0 else M[-l].conj().T
        got = host(plan.block(l))
        assert np.abs(got - ref).max() < 2e-6, l
        planes = plan.block(l, FG.STORE_SPLIT_F16).double().cpu().numpy()
        rec = ((planes[0] + planes[1]) + 1j * (planes[2] + planes[3])) / 4096.0
        assert np.abs(rec - ref).max() < 1e-6, l


ORDERS = [0.37, -1.62, 0.5, 2.0, 0.0, -0.999, 1.25]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_assemble_single_and_fused(FG, plans, case):
    plan = plans[case.name]
    for L in sorted({case.L_max, max(0, case.L_max - 3)}):
        orders = [a for a in ORDERS if not (a == round(a) and abs(a) > L)]
        refs = [O.fgfrft_power(case.F, a, L, case.P) for a in orders]
        fused = host(FG.Plan.assemble(plan, orders, L))
        for a, Qr, Qf in zip(orders, refs, fused):
            Q1 = host(plan.assemble([a], L))[0]
            assert rel(Q1, Qr) < TOL_FP32, (a, L)
            assert rel(Qf, Qr) < TOL_FP32, (a, L)


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("path", ["plain", "stacked_fp32", "assembled", "stacked", "auto"])
def test_apply_matches_oracle(FG, plans, case, path):
    plan = plans[case.name]
    rng = np.random.default_rng(7)
    N = case.F.shape[0]
    B = 70  # ragged against the 64-column tiles
    # plain / assembled: 7 runs of 10 equal orders (one assembly per run); others: one order per column
    a = np.repeat(rng.uniform(-2, 2, size=7), 10) if path in ("plain", "assembled") else rng.uniform(-2, 2, size=B)
    X = W.complex_normal((B, N), rng)
    L = case.L_max
    Y = host(plan.apply(a, dev(X), L, path=path))
    ref = O.apply_power(case.F, a, L, X.T, case.P).T
    tol = TOL_FP32 if path in ("plain", "stacked_fp32") else TOL_SPLIT
    assert rel(Y, ref) < tol
    # adjoint symmetry (Prop. 2): adjoint apply equals apply at -alpha, and (Q^a)^H x
    Yh = host(plan.apply(a, dev(X), L, adjoint=True, path=path))
    Ym = host(plan.apply(-a, dev(X), L, path=path))
    assert np.array_equal(Yh, Ym)
    refh = O.adjoint_apply(case.F, a, L, X.T, case.P).T
    assert rel(Yh, refh) < tol


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c.name)
def test_dual_forward_gradient_and_fd(FG, plans, case):
    plan = plans[case.name]
    rng = np.random.default_rng(11)
    N = case.F.shape[0]
    B = 9
    L = case.L_max
    a = rng.uniform(-2, 2, size=B)
    X = W.complex_normal((B, N), rng)
    G = W.complex_normal((B, N), rng)
    for path in ["stacked_fp32", "stacked"]:
        tol = TOL_FP32 if path == "stacked_fp32" else TOL_SPLIT
        Y, D = plan.forward_dual(a, dev(X), L, path=path)
        Yr = O.apply_power(case.F, a, L, X.T, case.P).T
        Dr = O.dalpha_apply(case.F, a, L, X.T, case.P).T
        assert rel(host(Y), Yr) < tol
        assert rel(host(D), Dr) < tol
        gX, ga = plan.backward(a, dev(G), D, L, path=path)
        assert rel(host(gX), O.adjoint_apply(case.F, a, L, G.T, case.P).T) < tol
        gr = O.grad_alpha(G.T, Dr.T)
        assert np.allclose(ga.cpu().numpy(), gr, rtol=tol, atol=tol * np.abs(gr).max())
        # central difference of the GPU forward, h = 1e-3
        h = 1e-3
        fd = (host(plan.apply(a + h, dev(X), L, path=path)) - host(plan.apply(a - h, dev(X), L, path=path))) / (2 * h)
        assert rel(fd, host(D)) < 1e-3


def test_autograd_function(FG, plans):
    case = CASES[1]
    plan = plans[case.name]
    rng = np.random.default_rng(5)
    N, B, L = 64, 6, 16
    a0 = rng.uniform(-1.5, 1.5, size=B)
    X = W.complex_normal((B, N), rng)
    T = W.complex_normal((B, N), rng)
    alpha = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    Xt = dev(X).requires_grad_(True)
    Y = FG.fgfrft(alpha, Xt, plan, L, path="stacked_fp32")
    loss = (Y - dev(T)).abs().pow(2).sum()
    loss.backward()
    Yr = O.apply_power(case.F, a0, L, X.T, case.P).T
    Gr = 2 * (Yr - T)
    g_alpha = O.grad_alpha(Gr.T, O.dalpha_apply(case.F, a0, L, X.T, case.P))
    assert np.allclose(alpha.grad.numpy(), g_alpha, rtol=2e-4, atol=2e-4 * np.abs(g_alpha).max())
    gX = O.adjoint_apply(case.F, a0, L, Gr.T, case.P).T
    assert rel(host(Xt.grad), gX) < 1e-4


def test_minus_identity_exact(FG):
    N = 40
    plan = FG.Plan(-np.eye(N), 3)
    assert plan.r_neg1 == N
    for a in [0.3, -1.7]:
        Q = host(plan.assemble([a], 3))[0]
        assert np.abs(Q - np.exp(1j * math.pi * a) * np.eye(N)).max() < 1e-6


def test_dft_closed_form_large(FG):
    """Unitary DFT (F^4 = I): r_-1 = N/4 and Q_L from the four closed-form projectors."""
    N, L = 256, 8
    F = W.dft_matrix(N)
    plan = FG.Plan(F, L)
    assert plan.r_neg1 == N // 4
    a = 0.37
    Fk = [np.eye(N), F, F @ F, F @ F @ F]
    n = np.arange(-L, L + 1)
    c = O.coeffs(a, L)
    Q = np.zeros((N, N), complex)
    for lam, th in {1: 0.0, -1j: -math.pi / 2, -1: math.pi, 1j: math.pi / 2}.items():
        Pl = sum(lam ** (-k) * Fk[k] for k in range(4)) / 4
        Q += (np.exp(1j * math.pi * a) if lam == -1 else np.sum(c * np.exp(1j * n * th))) * Pl
    assert rel(host(plan.assemble([a], L))[0], Q) < TOL_FP32


def test_error_codes(FG, plans):
    plan = plans["tiny"]
    X = dev(np.ones((2, 64)))
    with pytest.raises(FG.FGFRFTError) as e:
        plan.apply([17.0, 0.5], X, 16)
    assert e.value.code == FG.ERR_UNSUPPORTED
    with pytest.raises(FG.FGFRFTError) as e:
        plan.apply([float("nan"), 0.5], X, 16)
    assert e.value.code == FG.ERR_INVALID_ARG
    with pytest.raises(FG.FGFRFTError) as e:
        plan.apply([0.5, 0.5], X, 17)
    assert e.value.code == FG.ERR_UNSUPPORTED
    with pytest.raises(FG.FGFRFTError) as e:
        FG.Plan(np.random.default_rng(0).standard_normal((16, 16)), 2)
    assert e.value.code == FG.ERR_NOT_UNITARY
    plan.status()


def test_integer_order_beyond_L_rejected_but_within_L_exact(FG, plans):
    case = CASES[0]
    plan = plans["tiny"]
    Q = host(plan.assemble([3.0, -2.0], 16))
    assert rel(Q[0], O.integer_power(case.F, 3)) < TOL_FP32
    assert rel(Q[1], O.integer_power(case.F, -2)) < TOL_FP32


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c.name)
def test_assembled_path_single_order(FG, plans, case):
    """One order shared by every column: the assembled path assembles once (split output of
    the streaming kernel) and runs the tensor-core GEMM."""
    plan = plans[case.name]
    rng = np.random.default_rng(17)
    N = case.F.shape[0]
    X = W.complex_normal((96, N), rng)
    for a in (0.37, -1.4):
        Y = host(plan.apply([a], dev(X), case.L_max, path="assembled"))
        ref = O.apply_power(case.F, a, case.L_max, X.T, case.P).T
        assert rel(Y, ref) < TOL_SPLIT
