"""The offline projector onto the lambda = -1 eigenspace (Sec. III-B; Algorithm 1, "identify
I_-1 / form W") as fgfrft_precompute computes it in FP64 on the GPU: the projector before
rounding against the oracle's W W^H, the caller-supplied W route, the gap bracket
(fgfrft_plan_info's min_gap) against the oracle's eigenvalues, the residual ||F P + P||,
and the classification (neg1_tol and FGFRFT_ERR_AMBIGUOUS_SPECTRUM) on unitaries whose
eigenphases are prescribed, so every |lambda + 1| is known."""
import math

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def phases(n, seed, near=(), exact_neg1=0, margin=0.3):
    """n eigenphases: `exact_neg1` at pi, one at pi - d for each d in `near` (|lambda + 1| =
    2 sin(d/2)), the rest uniform in (-pi + margin, pi - margin)."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(-math.pi + margin, math.pi - margin, size=n)
    k = 0
    for _ in range(exact_neg1):
        th[k] = math.pi
        k += 1
    for d in near:
        th[k] = math.pi - d
        k += 1
    return th


def gap_of(d):
    return 2.0 * math.sin(d / 2.0)


BR = 1e-7  # slack of the gap bracket checks (FP64 resolution of 1 - g^2/4 for g >= 1e-4)


CASES = {
    "tiny graph (det -1)": lambda: W.tiny().F,
    "cyclic shift 64": lambda: W.cyclic_shift(64),
    "DFT 24": lambda: W.dft_matrix(24),
    "3 exact -1, margin 0.3": lambda: W.unitary_with_phases(phases(80, 1, exact_neg1=3), 11),
    "Haar 72": lambda: W.random_unitary(72, 5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_projector_gap_and_residual(FG, name):
    F = CASES[name]()
    sp = O.spectral(F)
    Pref = O.projector(F, sp)
    plan = FG.Plan(F, 4, keep_projector=True)
    assert plan.r_neg1 == sp.r_neg1
    P = plan.P64.cpu().numpy()
    if sp.r_neg1 == 0:
        assert np.abs(P).max() == 0.0
    else:
        # where the gap allows: FP64 rounding of S and of its powers moves P by ~u N / gap^2
        assert rel(P, Pref) < 1e-10, rel(P, Pref)
        assert plan.proj_residual < 1e-12 * math.sqrt(sp.r_neg1)
    lo, hi = plan.min_gap
    g = sp.min_gap
    # FP64 holds s = 1 - g^2/4 to u, so the bracket is exact up to ~u / g^2 relative
    assert lo <= g * (1 + BR) and g <= hi * (1 + BR), (lo, g, hi)
    assert hi <= 1.0101 * lo


def test_caller_supplied_W(FG):
    """W (orthonormal basis of the -1 eigenspace) from the oracle's Schur vectors: the plan's
    P is W W^H, its stored blocks equal the library's own route's to FP32 rounding, and the
    transform matches the oracle."""
    F = W.unitary_with_phases(phases(64, 2, exact_neg1=2), 12)
    sp = O.spectral(F)
    Wm = sp.Z[:, sp.neg1]
    L = 8
    own = FG.Plan(F, L, keep_projector=True)
    given = FG.Plan(F, L, W=Wm, keep_projector=True)
    assert given.r_neg1 == own.r_neg1 == 2 and given.squarings == 0
    assert rel(given.P64.cpu().numpy(), Wm @ Wm.conj().T) < 1e-14
    assert rel(given.P64.cpu().numpy(), own.P64.cpu().numpy()) < 1e-10
    for l in (-L, 0, 3, L + 1):
        a, b = own.block(l).cpu().numpy(), given.block(l).cpu().numpy()
        assert np.abs(a - b).max() < 2e-7
    lo, hi = given.min_gap
    assert lo <= sp.min_gap * (1 + BR) and sp.min_gap <= hi * (1 + BR)
    rng = np.random.default_rng(3)
    X = W.complex_normal((70, 64), rng)
    a = rng.uniform(-2, 2, size=70)
    Y = given.apply(a, torch.as_tensor(X, dtype=torch.complex64, device="cuda"), L).cpu().numpy()
    ref = O.apply_power(F, a, L, X.T, O.projector(F, sp)).T
    assert rel(Y, ref) < 5e-5


def test_adaptive_classification_refuses_the_uncertifiable_band(FG):
    """Adaptive (neg1_tol = 0): an eigenvalue 1e-7 from -1 squares into the -1 basin, but
    FP64 cannot certify it as -1 (the residual ||F P + P|| sees 1e-7 above the rounding
    level), and one 4e-7 from -1 stays in the complement closer than 1e-6: both refused.
    1e-11 is -1 to FP64 accuracy and 3e-4 is clearly not: both accepted, as the oracle
    (tolerance 1e-8) classifies them.  (With every other eigenvalue ~0.39 from -1, the widest
    gap first puts 3e-4 with the exact -1; its residual sends it back to the complement.)"""
    for d in (1e-7, 4e-7):
        F = W.unitary_with_phases(phases(64, 4, near=(d,), exact_neg1=1), 14)
        with pytest.raises(FG.FGFRFTError) as e:
            FG.Plan(F, 4)
        assert e.value.code == FG.ERR_AMBIGUOUS_SPECTRUM, d
    for d, r in ((1e-11, 2), (3e-4, 1)):
        F = W.unitary_with_phases(phases(64, 4, near=(d,), exact_neg1=1), 14)
        plan = FG.Plan(F, 4, keep_projector=True)
        sp = O.spectral(F)
        assert plan.r_neg1 == r == sp.r_neg1, d
        assert rel(plan.P64.cpu().numpy(), O.projector(F, sp)) < 1e-8
        if d == 3e-4:
            lo, hi = plan.min_gap
            assert lo <= gap_of(d) * (1 + BR) and gap_of(d) <= hi * (1 + BR)


def test_fixed_threshold_classification(FG):
    """neg1_tol = 1e-3: |lambda + 1| = 1e-4 counts as -1, 1e-2 does not, and 1.2e-3 (inside
    the guard band around the threshold) is refused; the counted eigenvalues agree with
    the oracle's classification at the same tolerance, and the residual reports the
    counted eigenvalue's distance from -1."""
    tol = 1e-3
    d_in, d_out = 1e-4, 1e-2
    F = W.unitary_with_phases(phases(64, 5, near=(d_in, d_out), exact_neg1=1), 15)
    plan = FG.Plan(F, 6, neg1_tol=tol, keep_projector=True)
    sp = O.spectral(F, tol=tol)
    assert plan.r_neg1 == sp.r_neg1 == 2
    assert rel(plan.P64.cpu().numpy(), O.projector(F, sp)) < 1e-8
    assert abs(plan.proj_residual - gap_of(d_in)) < 1e-3 * gap_of(d_in)
    lo, hi = plan.min_gap
    assert lo <= gap_of(d_out) * (1 + BR) and gap_of(d_out) <= hi * (1 + BR) and hi <= 1.0101 * lo
    # transforms from this plan follow Def. 1 with the oracle's P at the same tolerance
    rng = np.random.default_rng(6)
    X = W.complex_normal((20, 64), rng)
    a = rng.uniform(-2, 2, size=20)
    Y = plan.apply(a, torch.as_tensor(X, dtype=torch.complex64, device="cuda"), 6).cpu().numpy()
    ref = O.apply_power(F, a, 6, X.T, O.projector(F, sp)).T
    assert rel(Y, ref) < 5e-5
    # the same F without a threshold: 1e-4 is then a complement eigenvalue (far above the
    # rounding level, far below the spectrum's other gaps), so r = 1
    assert FG.Plan(F, 6).r_neg1 == 1
    F2 = W.unitary_with_phases(phases(64, 5, near=(1.2e-3,), exact_neg1=1), 15)
    with pytest.raises(FG.FGFRFTError) as e:
        FG.Plan(F2, 6, neg1_tol=tol)
    assert e.value.code == FG.ERR_AMBIGUOUS_SPECTRUM
