"""The pair assembly against the FP64 oracle.  For a real F without a -1 eigenvalue the
plan keeps one row of the 2 L_max powers M_l, l != 0, per entry pair (i, k) with
i/128 <= k/128; the fused multi-order assembly forms Q[i][k] from c_l and Q[k][i] from
c_{-l} (M_{-l} = M_l^T, Prop. 2; M_0 = I adds c_0 on the diagonal; Def. 1), and the grouped
GEMM reads the operator left of each row tile's diagonal block from its transposed store.
Cases span one, two and three 128-row blocks (diagonal blocks only; mirrors), L_max = 16 ... 64
(one to four 32-power chunks; at 64 the launch keeps one output staging buffer per epilogue
group), ragged order groups, more than 64 groups (two assembly passes), integer orders, L below
L_max, complex and real signals.  Bars: the split-precision bar on relative Frobenius error per group, and
the same on each column's maximum relative error (a wrong tile or a missed mirror shows up
in the columns it touches)."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_SPLIT = 5e-5


@pytest.fixture(scope="module")
def FG():
    from paper_2602_20870_gb300 import build, fgfrft
    build.build()
    fgfrft.load()
    return fgfrft


def real_gft_without_minus_one(n, seed):
    """A random-geometric-graph GFT with det F = +1 (a real orthogonal F has the eigenvalue -1
    with odd multiplicity iff det F = -1; negating one eigenvector flips the determinant)."""
    F = W.rgg_gft(n, seed)
    if np.linalg.det(F.real) < 0:
        F = F.copy()
        F[0] = -F[0]
    return F


CASES = [(128, 16, 11), (256, 32, 12), (384, 16, 13), (256, 48, 14), (256, 64, 15)]
IDS = [f"N{n}-Lmax{L}" for n, L, _ in CASES]


@pytest.fixture(scope="module")
def plans(FG):
    out = {}
    for (n, L_max, seed), name in zip(CASES, IDS):
        F = real_gft_without_minus_one(n, seed)
        plan = FG.Plan(F, L_max)
        out[name] = (F, plan)
    return out


def check_groups(Y, X, F, alpha, L, starts, counts):
    zero_P = np.zeros(F.shape, dtype=np.complex128)
    for s, c in zip(starts, counts):
        cols = np.arange(s, s + c)
        ref = O.apply_power(F, alpha[cols], L, X[cols].T, zero_P).T
        got = Y[cols]
        e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert e < TOL_SPLIT, (s, c, e)
        col = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
        assert col.max() < TOL_SPLIT, (s, c, float(col.max()))


@pytest.mark.parametrize("name", IDS)
def test_plan_builds_the_pair_stack(plans, name):
    F, plan = plans[name]
    assert plan.real and plan.r_neg1 == 0 and plan.pair


@pytest.mark.parametrize("name", IDS)
@pytest.mark.parametrize("L_off", [0, 5])
def test_pair_assembly_groups_match_oracle(FG, plans, name, L_off):
    F, plan = plans[name]
    n = F.shape[0]
    L = plan.L_max - L_off
    rng = np.random.default_rng(100 + n + L_off)
    counts = [1, 17, 64, 3, 40, 9]
    orders = rng.uniform(-2, 2, size=len(counts))
    orders[1], orders[3] = 0.0, -1.0  # integer orders: Q = F^a exactly (c_l = delta)
    alpha = np.repeat(orders, counts)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    X = W.complex_normal((alpha.size, n), rng)
    Xd = torch.as_tensor(X, dtype=torch.complex64, device="cuda")
    Y = plan.apply(alpha, Xd, L, path="assembled").cpu().numpy().astype(np.complex128)
    plan.status()
    check_groups(Y, X, F, alpha, L, starts, counts)
    # the adjoint at -alpha (Prop. 2) goes through the same assembly
    Yh = plan.apply(alpha, Xd, L, adjoint=True, path="assembled").cpu().numpy().astype(np.complex128)
    check_groups(Yh, X, F, -alpha, L, starts, counts)


def test_more_than_64_orders_two_passes(FG, plans):
    F, plan = plans["N256-Lmax32"]
    L = plan.L_max
    rng = np.random.default_rng(7)
    counts = [2] * 70 + [5]  # 71 order groups: two passes of the pair assembly
    alpha = np.repeat(rng.uniform(-2, 2, size=len(counts)), counts)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    X = W.complex_normal((alpha.size, 256), rng)
    Y = plan.apply(alpha, torch.as_tensor(X, dtype=torch.complex64, device="cuda"), L, path="assembled")
    Y = Y.cpu().numpy().astype(np.complex128)
    check_groups(Y, X, F, alpha, L, starts[::7], counts[::7])
    check_groups(Y, X, F, alpha, L, starts[64:], counts[64:])


def test_real_signals_and_outputs(FG, plans):
    F, plan = plans["N384-Lmax16"]
    L = plan.L_max
    rng = np.random.default_rng(9)
    counts = [30, 1, 33]
    alpha = np.repeat(rng.uniform(-2, 2, size=3), counts)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    Xr = rng.standard_normal((alpha.size, 384))
    Xt = torch.as_tensor(Xr, dtype=torch.float32, device="cuda")
    Y = torch.empty_like(Xt)
    plan.apply(alpha, Xt, L, out=Y, real_io=True, real_output=True)
    plan.status()
    check_groups(Y.cpu().numpy().astype(np.float64), Xr.astype(np.complex128), F, alpha, L, starts, counts)
