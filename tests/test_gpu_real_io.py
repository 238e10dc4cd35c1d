"""Real float32 signals and outputs through fgfrft_apply (FGFRFT_REAL_SIGNALS /
FGFRFT_REAL_OUTPUT): identical results to the complex64 interface on the same values,
the conditions under which they are refused, and the host round trip."""
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


def test_real_signals_match_complex(FG):
    wl = W.tiny(flip_one=True)  # real F, no -1 eigenvalue: Q is real
    plan = FG.Plan(wl.F, 16)
    assert plan.real and plan.r_neg1 == 0
    rng = np.random.default_rng(4)
    Xr = rng.standard_normal((130, 64)).astype(np.float32)
    a = np.repeat([0.37, -1.1], 65)
    Xc = torch.as_tensor(Xr.astype(np.complex64), device="cuda")
    Xd = torch.as_tensor(Xr, device="cuda")
    for path in ("assembled", "stacked"):
        Yc = plan.apply(a, Xc, 16, path=path)
        Yr = plan.apply(a, Xd, 16, path=path, real_io=True)
        assert torch.equal(Yc, Yr), path
    Yc = plan.apply(a, Xc, 16, path="assembled")
    Yro = plan.apply(a, Xd, 16, path="assembled", real_io=True, real_output=True)
    assert Yro.dtype == torch.float32
    assert torch.equal(Yro, Yc.real.contiguous()) and float(Yc.imag.abs().max()) == 0.0
    ref = O.apply_power(wl.F, a, 16, Xr.T.astype(np.complex128)).T
    assert np.linalg.norm(Yro.cpu().numpy() - ref) / np.linalg.norm(ref) < 5e-5
    # host buffers: the end-to-end form of the same call
    Yh = plan.apply(a, torch.as_tensor(Xr), 16, real_io=True, real_output=True)
    torch.cuda.synchronize()
    assert torch.equal(Yh, Yro.cpu())


def test_real_io_refused(FG):
    plan_c = FG.Plan(W.tiny().F, 8)  # real F with a -1 eigenvalue: Q has an imaginary part
    X = torch.zeros((70, 64), dtype=torch.float32, device="cuda")
    a = np.full(70, 0.3)
    with pytest.raises(FG.FGFRFTError) as e:
        plan_c.apply(a, X, 8, real_io=True, real_output=True)
    assert e.value.code == FG.ERR_UNSUPPORTED
    for path in ("plain", "stacked_fp32"):
        with pytest.raises(FG.FGFRFTError) as e:
            plan_c.apply(a, X, 8, path=path, real_io=True)
        assert e.value.code == FG.ERR_UNSUPPORTED
    # real signals on a complex-valued operator are fine (complex output)
    Y = plan_c.apply(a, X + 1.0, 8, real_io=True)
    Yc = plan_c.apply(a, (X + 1.0).to(torch.complex64), 8)
    assert torch.equal(Y, Yc)
