"""Half-stack storage (only M_0..M_L and P stored; M_{-l} = M_l^H read as transposed
tiles, Prop. 2): single-order assembly, the plain and assembled apply paths, against the
FP64 oracle, on real and complex operators, ragged sizes (several tile pairs and a
partial edge tile), L below L_max, and integer / negative orders."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def FG():
    from paper_2602_20870_gb300 import build, fgfrft
    build.build()
    fgfrft.load()
    return fgfrft


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def real_orthogonal(n, seed):
    Z = np.random.default_rng(seed).standard_normal((n, n))
    Qm, R = np.linalg.qr(Z)
    return (Qm * np.sign(np.diag(R))).astype(np.complex128)


OPERATORS = {
    "tiny": lambda: W.tiny().F,                        # real, one -1 eigenvalue
    "tiny-flip": lambda: W.tiny(flip_one=True).F,      # real, no -1 eigenvalue
    "haar65": lambda: W.random_unitary(65, 3),         # complex, one partial edge tile
    "dft64": lambda: W.dft_matrix(64),                 # complex, large -1 eigenspace
    "real200": lambda: real_orthogonal(200, 5),        # real, 4 x 4 tiles (10 pairs), ragged edge
}


@pytest.fixture(scope="module", params=list(OPERATORS))
def case(request, FG):
    F = OPERATORS[request.param]()
    L_max = 9
    plan = FG.Plan(F, L_max, storage=FG.STORE_HALF)
    full = FG.Plan(F, L_max, storage=FG.STORE_C64 | FG.STORE_SPLIT_F16)
    return request.param, F, O.projector(F), plan, full


@pytest.mark.parametrize("L", [9, 4, 0])
def test_assemble_half(case, L):
    name, F, P, plan, full = case
    # an integer order above L is unsupported (Def. 1 needs its power): keep the valid ones
    orders = [a for a in (0.37, -1.3, 2.0, 0.5) if not (a == round(a) and abs(a) > L)]
    Q = plan.assemble(orders, L).cpu().numpy()
    for a, Qa in zip(orders, Q):
        ref = O.fgfrft_power(F, a, L, P)
        assert rel(Qa, ref) < TOL, (name, L, a, rel(Qa, ref))


def test_half_matches_full_storage(case):
    name, F, P, plan, full = case
    Qh = plan.assemble([0.61], 9).cpu().numpy()[0]
    Qf = full.assemble([0.61], 9).cpu().numpy()[0]
    assert rel(Qh, Qf) < 2e-6, name


def test_apply_paths_half(case):
    name, F, P, plan, full = case
    N = F.shape[0]
    rng = np.random.default_rng(7)
    X = W.complex_normal((130, N), rng)
    a = np.repeat([0.37, -0.8], 65)  # two groups of 65 columns: the assembled path by default
    ref = O.apply_power(F, a, 9, X.T, P).T
    Xd = torch.as_tensor(X, dtype=torch.complex64, device="cuda")
    for path, tol in (("auto", 5e-5), ("assembled", 5e-5), ("plain", TOL)):
        Y = plan.apply(a, Xd, 9, path=path).cpu().numpy()
        assert rel(Y, ref) < tol, (name, path)
    Yadj = plan.apply(a, Xd, 9, adjoint=True, path="plain").cpu().numpy()
    assert rel(Yadj, O.apply_power(F, -a, 9, X.T, P).T) < TOL


def test_half_stack_blocks_and_unsupported_paths(FG):
    F = W.tiny().F
    plan = FG.Plan(F, 5, storage=FG.STORE_HALF)
    full = FG.Plan(F, 5, storage=FG.STORE_C64)
    for l in (0, 3, 6):  # 6 = L_max + 1 is P: the same FP32 rounding of the same FP64 block
        assert torch.equal(plan.block(l, FG.STORE_HALF), full.block(l, FG.STORE_C64))
    with pytest.raises(FG.FGFRFTError):
        plan.block(-2, FG.STORE_HALF)
    X = torch.zeros((4, 64), dtype=torch.complex64, device="cuda")
    for path in ("stacked", "stacked_fp32"):
        with pytest.raises(FG.FGFRFTError) as e:
            plan.apply([0.3] * 4, X, 5, path=path)
        assert e.value.code == FG.ERR_UNSUPPORTED


def test_half_image_graph_size(FG):
    """N = 1024, L = 32 (the image-graph operator): 16 x 16 tiles, 136 pairs; against the
    full-storage assembly (whose parity with the oracle is tested at this size elsewhere)
    and against the oracle's action on a few columns."""
    wl = W.image_graph(n_orders=2, per_order=2)
    plan = FG.Plan(wl.F, 32, storage=FG.STORE_HALF | FG.STORE_C64)
    a = [0.37, -1.61]
    Q = plan.assemble(a, 32)
    full = FG.Plan(wl.F, 32, storage=FG.STORE_C64)
    Qf = full.assemble(a, 32)
    assert rel(Q.cpu().numpy(), Qf.cpu().numpy()) < 2e-6
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 1024)).astype(np.complex128)
    P = O.projector(wl.F)
    for k, ak in enumerate(a):
        ref = O.apply_power(wl.F, ak, 32, X.T, P).T
        got = (Q[k].cpu().numpy().astype(np.complex128) @ X.T).T
        assert rel(got, ref) < TOL


@pytest.mark.parametrize("path", ["auto", "assembled", "plain"])
def test_dual_and_backward_assembled_paths(case, path):
    """dY/dalpha from the assembled dQ/dalpha = sum_l c_l' M_l + j pi e^{j pi a} P (Prop. 3),
    the adjoint Q^H G and the alpha-gradient, on a half-stack plan and on a full one."""
    name, F, P, plan, full = case
    N = F.shape[0]
    rng = np.random.default_rng(11)
    X = W.complex_normal((128, N), rng)
    G = W.complex_normal((128, N), rng)
    a = np.repeat([0.43, -1.2], 64)
    Yref = O.apply_power(F, a, 9, X.T, P).T
    Dref = O.dalpha_apply(F, a, 9, X.T, P).T
    GXref = O.apply_power(F, -a, 9, G.T, P).T
    Xd = torch.as_tensor(X, dtype=torch.complex64, device="cuda")
    Gd = torch.as_tensor(G, dtype=torch.complex64, device="cuda")
    tol = 1e-5 if path == "plain" else 5e-5
    for pl in (plan, full):
        Y, D = pl.forward_dual(a, Xd, 9, path=path)
        assert rel(Y.cpu().numpy(), Yref) < tol, (name, path)
        assert rel(D.cpu().numpy(), Dref) < tol, (name, path)
        gX, ga = pl.backward(a, Gd, D, 9, path=path)
        assert rel(gX.cpu().numpy(), GXref) < tol, (name, path)
        g_ref = np.real(np.sum(np.conj(G) * D.cpu().numpy().astype(np.complex128), axis=1))
        assert np.allclose(ga.cpu().numpy(), g_ref, rtol=1e-4, atol=1e-3 * np.abs(g_ref).max())
