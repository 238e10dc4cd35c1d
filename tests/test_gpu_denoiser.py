"""Parity of the spectral denoiser x_hat = Q^{-a} diag(h) Q^{a} y (Sec. V-B) and of its
gradients in the order a and the filter h, computed by torch autograd through the
library's custom backward, against an FP64 restatement built from the oracle alone
(apply_power at +-a, dalpha_apply, and the adjoint by order reversal, Prop. 2).

For the linear functional l = Re sum conj(Wt) x_hat, with Z = Q^a Y, U = diag(h) Z and
A = (Q^{-a})^H Wt = Q^{a} Wt:
    dl/dh_i = Re sum_j conj(A_ij) Z_ij
    dl/da   = Re <A, diag(h) dZ/da> - Re <Wt, (dQ/db)_{b=-a} U>,  dZ/da = (dQ/da) Y (Prop. 3).
Also the shared-order gradient of fgfrft_grad (FGFRFT_SHARED_ALPHA: the library sums the
per-column gradients) against the per-column gradients and the oracle."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 5e-5


@pytest.fixture(scope="module")
def mods():
    from paper_2602_20870_gb300 import build, fgfrft, learning
    build.build()
    return fgfrft, learning


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_denoiser(F, a, L, h, Y, Wt):
    """(x_hat, dl/da, dl/dh) in FP64 from the oracle; signals as columns."""
    P = O.projector(F)
    Z = O.apply_power(F, a, L, Y, P)
    U = h[:, None] * Z
    Xh = O.apply_power(F, -a, L, U, P)
    A = O.adjoint_apply(F, -a, L, Wt, P)  # (Q^{-a})^H Wt = Q^{a} Wt
    dl_dh = np.real(np.sum(np.conj(A) * Z, axis=1))
    dZ = O.dalpha_apply(F, a, L, Y, P)
    dXh_fixed_U = O.dalpha_apply(F, -a, L, U, P)  # d/db Q^{b} U at b = -a
    dl_da = np.real(np.sum(np.conj(A) * (h[:, None] * dZ))) - np.real(np.sum(np.conj(Wt) * dXh_fixed_U))
    return Xh, dl_da, dl_dh


@pytest.mark.parametrize("case", ["grid 16x16, 64 signals", "Haar 48, 20 signals"])
def test_denoiser_forward_and_gradients(mods, case):
    FG, LR = mods
    rng = np.random.default_rng(21)
    if case.startswith("grid"):
        F = W.gft_from_gso(W.laplacian(W.grid_adjacency(16, 16)))
        L, B = 12, 64  # 64 columns of one order: the assembled (dual) path
        Y = W.gaussian_random_field(16, 16, 2.0, B, rng) + 0.3 * rng.standard_normal((B, 256))
        Y = Y.astype(np.complex128)
    else:
        F = W.random_unitary(48, 31)
        L, B = 10, 20  # complex F, few columns: the stacked path
        Y = W.complex_normal((B, 48), rng)
    N = F.shape[0]
    plan = FG.Plan(F, L)
    model = LR.SpectralDenoiser(plan, L, alpha_init=0.63)
    h = rng.uniform(0.2, 1.5, size=N)
    with torch.no_grad():
        model.h.copy_(torch.as_tensor(h, dtype=torch.float32))
    h = model.h.detach().cpu().numpy().astype(np.float64)  # the float32 values the GPU uses
    Wt = W.complex_normal((B, N), rng)
    Yd = torch.as_tensor(Y, dtype=torch.complex64, device="cuda")
    Wd = torch.as_tensor(Wt, dtype=torch.complex64, device="cuda")
    xh = model(Yd)
    loss = (Wd.conj() * xh).real.sum()
    loss.backward()
    Xh_ref, da_ref, dh_ref = oracle_denoiser(F, 0.63, L, h, Yd.cpu().numpy().astype(np.complex128).T,
                                             Wd.cpu().numpy().astype(np.complex128).T)
    assert rel(xh.detach().cpu().numpy().T, Xh_ref) < TOL
    assert abs(float(model.alpha.grad) - da_ref) < TOL * max(1.0, abs(da_ref)) * 4, (float(model.alpha.grad), da_ref)
    assert rel(model.h.grad.cpu().numpy(), dh_ref) < TOL


def test_shared_order_gradient_is_summed_in_the_library(mods):
    FG, _ = mods
    F = W.tiny(flip_one=True).F
    L, B = 16, 90
    plan = FG.Plan(F, L)
    rng = np.random.default_rng(5)
    X = torch.as_tensor(W.complex_normal((B, 64), rng), dtype=torch.complex64, device="cuda")
    G = torch.as_tensor(W.complex_normal((B, 64), rng), dtype=torch.complex64, device="cuda")
    a = 0.81
    _, D = plan.forward_dual(np.full(B, a), X, L)
    _, g_cols = plan.backward(np.full(B, a), G, D, L, need_x=False)
    _, g_one = plan.backward(np.array([a]), G, D, L, need_x=False, shared=True)
    assert g_one.shape == (1,)
    s_cols = float(g_cols.double().sum())
    assert abs(float(g_one[0]) - s_cols) <= 1e-6 * max(1.0, abs(s_cols))
    P = O.projector(F)
    Dref = O.dalpha_apply(F, a, L, X.cpu().numpy().astype(np.complex128).T, P)
    ref = float(np.sum(O.grad_alpha(G.cpu().numpy().astype(np.complex128).T, Dref)))
    assert abs(float(g_one[0]) - ref) <= TOL * np.sum(np.abs(G.cpu().numpy()) * np.abs(Dref.T)), (float(g_one[0]), ref)
