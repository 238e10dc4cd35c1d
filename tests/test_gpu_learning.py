"""End-to-end training through the differentiable transform (Sec. V): order learning of a
K-layer cascade against the exact GFRFT, and the spectral denoiser Q^{-a} diag(h) Q^{a}."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2602_20870_gb300 import build, fgfrft, learning
    build.build()
    return fgfrft, learning


@pytest.mark.parametrize("K", [1, 2])
def test_order_learning_reaches_target_order(mods, K):
    FG, LR = mods
    N, L = 96, 10
    F = W.rgg_gft(N, 77)
    plan = FG.Plan(F, L)
    X = torch.eye(N, dtype=torch.complex64, device="cuda")
    # target Y = F^{1.5} X, one signal per row (the exact GFRFT, from the oracle)
    target = torch.as_tensor(O.exact_gfrft(F, 1.5).T.copy(), dtype=torch.complex64, device="cuda")
    out = LR.learn_orders(plan, X, target, K=K, L=L, alpha_init=0.1, lr=0.01, iters=200)
    assert out["loss"][-1] < 0.05 * out["loss"][0]
    assert abs(out["order_sum"][-1] - 1.5) < 0.03
    assert all(np.isfinite(out["loss"]))


def test_spectral_denoiser_improves_snr(mods):
    FG, LR = mods
    side = 16
    F = W.gft_from_gso(W.laplacian(W.grid_adjacency(side, side)))
    plan = FG.Plan(F, 12)
    rng = np.random.default_rng(8)
    clean = W.gaussian_random_field(side, side, 2.0, 64, rng)
    noisy = clean + 0.5 * rng.standard_normal(clean.shape)
    x = torch.as_tensor(clean, dtype=torch.complex64, device="cuda")
    y = torch.as_tensor(noisy, dtype=torch.complex64, device="cuda")
    model = LR.SpectralDenoiser(plan, 12, alpha_init=0.8)
    out = LR.train_denoiser(model, y, x, lr=0.02, iters=150)
    mse_in = float((y - x).abs().pow(2).mean())
    assert out["loss"][-1] < 0.6 * out["loss"][0]
    assert out["loss"][-1] < 0.5 * mse_in
