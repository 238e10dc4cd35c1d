"""Degenerate and edge cases against the oracle: N = 1 (a single eigenvalue, -1 included),
odd tiny N, L = 0 and L = 1 (only M_0 = P_c, P and the first powers), one signal, and
orders at integers, half-integers and |alpha| = L."""
import math

import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PATHS = ["plain", "stacked_fp32", "assembled", "stacked"]
TOL = {"plain": 1e-5, "stacked_fp32": 1e-5, "assembled": 5e-5, "stacked": 5e-5}


@pytest.fixture(scope="module")
def FG():
    from paper_2602_20870_gb300 import build, fgfrft
    build.build()
    return fgfrft


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


@pytest.mark.parametrize("theta", [0.3, -2.0, math.pi])
def test_scalar_unitary(FG, theta):
    """N = 1: F = e^{j theta}; theta = pi makes P = 1 and Q = e^{j pi a} for every L."""
    F = np.array([[np.exp(1j * theta)]])
    if theta == math.pi:
        F = np.array([[-1.0 + 0j]])
    plan = FG.Plan(F, 3)
    assert plan.r_neg1 == (1 if theta == math.pi else 0)
    X = np.array([[0.7 - 0.2j], [1.5 + 0.5j]])
    for a in (0.37, -1.25, 2.0):
        ref = O.apply_power(F, a, 3, X.T).T
        for path in PATHS:
            Y = plan.apply([a], torch.as_tensor(X, dtype=torch.complex64, device="cuda"), 3, path=path)
            assert rel(Y.cpu().numpy(), ref) < TOL[path], (path, a)
        Q = plan.assemble([a, -a], 3).cpu().numpy()
        assert rel(Q[0], O.fgfrft_power(F, a, 3)) < 1e-5
        assert rel(Q[1], O.fgfrft_power(F, -a, 3)) < 1e-5


@pytest.mark.parametrize("L", [0, 1])
def test_small_L_all_paths(FG, L):
    F = W.tiny(flip_one=True).F  # real F without a -1 eigenvalue; then one with it, and a complex unitary
    for Fx in (F, W.tiny().F, W.random_unitary(33, 5)):
        plan = FG.Plan(Fx, max(L, 1))
        P = O.projector(Fx)
        rng = np.random.default_rng(L)
        X = W.complex_normal((70, Fx.shape[0]), rng)
        a = np.repeat([0.37, -0.6], 35)
        ref = O.apply_power(Fx, a, L, X.T, P).T
        Xd = torch.as_tensor(X, dtype=torch.complex64, device="cuda")
        for path in PATHS:
            Y = plan.apply(a, Xd, L, path=path).cpu().numpy()
            assert rel(Y, ref) < TOL[path], (path, L)
        Yd, D = plan.forward_dual(a, Xd, L, path="stacked")
        assert rel(D.cpu().numpy(), O.dalpha_apply(Fx, a, L, X.T, P).T) < 5e-5


def test_one_signal_and_special_orders(FG):
    F = W.tiny().F
    L = 6
    plan = FG.Plan(F, L)
    P = O.projector(F)
    x = W.complex_normal((1, 64), np.random.default_rng(2))
    xd = torch.as_tensor(x, dtype=torch.complex64, device="cuda")
    for a in (0.5, -0.5, 1.5, 6.0, -6.0, 3.0, 1e-9, -2.999999):
        ref = O.apply_power(F, a, L, x.T, P).T
        for path in PATHS:
            y = plan.apply([a], xd, L, path=path).cpu().numpy()
            assert rel(y, ref) < TOL[path], (path, a)


@pytest.mark.parametrize("which", ["haar", "real_flip", "real"])
def test_real_signals(FG, which):
    """Real signals take the real-B tensor-core products (the imaginary B planes are not
    loaded); one complex signal in the batch switches the launch back to complex B."""
    F = {"haar": W.random_unitary(65, 3), "real_flip": W.tiny(flip_one=True).F, "real": W.tiny().F}[which]
    N, L = F.shape[0], 7
    plan = FG.Plan(F, L)
    P = O.projector(F)
    rng = np.random.default_rng(11)
    Xr = rng.standard_normal((130, N)).astype(np.complex128)
    Xm = Xr.copy()
    Xm[77] += 1j * rng.standard_normal(N)
    a = np.repeat(rng.uniform(-2.0, 2.0, size=2), 65)
    for X in (Xr, Xm):
        ref = O.apply_power(F, a, L, X.T, P).T
        Xd = torch.as_tensor(X, dtype=torch.complex64, device="cuda")
        for path in PATHS:
            Y = plan.apply(a, Xd, L, path=path).cpu().numpy()
            assert rel(Y, ref) < TOL[path], (path, which)
        Yd, D = plan.forward_dual(a, Xd, L, path="stacked")
        assert rel(Yd.cpu().numpy(), ref) < 5e-5
        assert rel(D.cpu().numpy(), O.dalpha_apply(F, a, L, X.T, P).T) < 5e-5
    # a real operator (real F, no -1 eigenvalue) on real signals gives real outputs exactly
    if which == "real_flip":
        Xd = torch.as_tensor(Xr, dtype=torch.complex64, device="cuda")
        for path in ("assembled", "stacked"):
            a1 = np.full(130, 0.37)
            Y = plan.apply(a1, Xd, L, path=path)
            assert float(Y.imag.abs().max()) == 0.0, path
