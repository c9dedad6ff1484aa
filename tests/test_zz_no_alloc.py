"""hyp_rhs_noalloc: the right-hand side for callers that may not allocate device memory while they
run (stream capture, real-time loops, hosts owning all device memory). Its scratch lives in a
static device array of the library; its result must match hyp_rhs on the same grid and state,
on two calls in a row. This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_util import gpu_state, oracle_case
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [I.bl_case(48, 32), I.sbli_case(64, 40, seed=1)],
                         ids=["bl_48x32", "sbli_64x40"])
def test_noalloc_matches_rhs_twice(table, cfg):
    import torch
    from paper_2210_05547_gb300 import abi as A
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    tol, _ = F.parity_tolerance(case, case.U0)
    U = torch.as_tensor(case.U0).cuda()
    R_ref = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R_ref)
    outs = []
    for _ in range(2):
        R = torch.full_like(U, float("nan"))
        A.rhs_noalloc(gas, st.grid, U, R)
        torch.cuda.synchronize()
        outs.append(R.cpu().numpy())
    ref = F.unpack(5, cfg["nx"], cfg["ny"], R_ref.cpu().numpy())
    for out in outs:
        got = F.unpack(5, cfg["nx"], cfg["ny"], out)
        for k in ref:
            assert np.abs(got[k] - ref[k]).max() <= tol[k], k
    assert np.array_equal(outs[0], outs[1])       # same inputs, same static scratch reset


def test_noalloc_rejects_large_grid():
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.bl_case(256, 64)
    gas, st = gpu_state(cfg)
    R = torch.empty_like(st.U)
    with pytest.raises(A.HypError, match="too large for hyp_rhs_noalloc"):
        A.rhs_noalloc(gas, st.grid, st.U, R)
