"""Failure detection without a GPU fault: a device wait that nothing completes runs out
after its bounded limit, the plan's status word reports FGFRFT_ERR_TIMEOUT, the status is
cleared by reading it, and the context keeps working."""
import numpy as np
import pytest
import torch

from oracle import fgfrft_oracle as O
from paper_2602_20870_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_context_survives():
    from paper_2602_20870_gb300 import build, fgfrft as FG
    build.build()
    wl = W.tiny()
    plan = FG.Plan(wl.F, 16)
    plan.status()  # clean
    plan.check_wait_timeout()
    with pytest.raises(FG.FGFRFTError) as e:
        plan.status()
    assert e.value.code == FG.ERR_TIMEOUT
    plan.status()  # reading cleared it
    X = torch.as_tensor(wl.X, dtype=torch.complex64, device="cuda")
    Y = plan.apply(wl.alpha, X, 16).cpu().numpy()
    ref = O.apply_power(wl.F, wl.alpha, 16, wl.X.T).T
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 5e-5
