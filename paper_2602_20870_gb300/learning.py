"""Learning with the differentiable FGFRFT (Sec. V of the paper).

* Transform-order learning (Sec. V-A): a cascade of K layers
  Y_hat = Q^{alpha_K} ... Q^{alpha_1} X with one learnable order per layer,
  trained with Adam on the loss (1/N^2) ||Y_hat - Y||_F^2 against a target Y.
* Graph-signal denoising (Sec. V-B): x_hat = Q^{-alpha} diag(h) Q^{alpha} y with a
  learnable order alpha and a learnable diagonal filter h in the transformed domain,
  trained to minimise ||x_hat - x||^2.

Every transform and its gradient runs in the CUDA library through
``fgfrft.FGFRFTFunction`` (dY/dalpha from the same pass as Y, the signal adjoint
by order reversal); the optimiser and the loss are plain PyTorch.
"""
from __future__ import annotations

import time

import torch

from .fgfrft import Plan, fgfrft


def cascade(plan: Plan, alphas, X: torch.Tensor, L: int, path: str = "auto") -> torch.Tensor:
    """Q^{alpha_K} ... Q^{alpha_1} X (signals as rows of X)."""
    Y = X
    for a in alphas:
        Y = fgfrft(a, Y, plan, L, path)
    return Y


def learn_orders(plan: Plan, X: torch.Tensor, target: torch.Tensor, K: int, L: int,
                 alpha_init: float = 0.1, lr: float = 0.01, iters: int = 200, path: str = "auto") -> dict:
    """Adam on the orders of a K-layer cascade (Sec. V-A).  Returns the history of the loss
    and of the total order sum(alpha), the final orders and the wall time."""
    N = plan.N
    alphas = [torch.tensor([alpha_init], dtype=torch.float64, requires_grad=True) for _ in range(K)]
    opt = torch.optim.Adam(alphas, lr=lr)
    hist_loss, hist_sum = [], []
    t0 = time.perf_counter()
    for _ in range(iters):
        opt.zero_grad()
        Y = cascade(plan, alphas, X, L, path)
        loss = (Y - target).abs().pow(2).sum() / (N * N)
        loss.backward()
        opt.step()
        hist_loss.append(float(loss.detach()))
        hist_sum.append(float(sum(a.detach() for a in alphas)))
    torch.cuda.synchronize()
    return {"loss": hist_loss, "order_sum": hist_sum, "orders": [float(a.detach()) for a in alphas],
            "seconds": time.perf_counter() - t0}


class SpectralDenoiser(torch.nn.Module):
    """x_hat = Q^{-alpha} diag(h) Q^{alpha} y (Sec. V-B), alpha and real h learnable."""

    def __init__(self, plan: Plan, L: int, alpha_init: float = 0.5, path: str = "auto"):
        super().__init__()
        self.plan, self.L, self.path = plan, int(L), path
        self.alpha = torch.nn.Parameter(torch.tensor([alpha_init], dtype=torch.float64))
        self.h = torch.nn.Parameter(torch.ones(plan.N, dtype=torch.float32, device=plan.device))

    def forward(self, Y: torch.Tensor) -> torch.Tensor:
        Z = fgfrft(self.alpha, Y, self.plan, self.L, self.path)
        Z = Z * self.h.to(Z.dtype)
        return fgfrft(-self.alpha, Z, self.plan, self.L, self.path)


def train_denoiser(model: SpectralDenoiser, noisy: torch.Tensor, clean: torch.Tensor, lr: float = 0.01,
                   iters: int = 100) -> dict:
    """Adam on ||x_hat - x||^2 / numel; returns the loss history."""
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    hist = []
    for _ in range(iters):
        opt.zero_grad()
        loss = (model(noisy) - clean).abs().pow(2).mean()
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
    return {"loss": hist, "alpha": float(model.alpha.detach())}
