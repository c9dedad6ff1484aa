"""hyp_grid_temperature: the cell-centre temperatures of a grid's last closure (Sec. 2.2), against
the oracle's temperature inversion at the same primitives.

* FP64: within 1e-13 relative (the Newton iteration stops after a step below 1e-8 T, leaving an
  error of order (1e-8)^2 relative, plus the rounding of the energy sums), on the first right-hand
  side (cold start from the cached 1000 K) and on a second one at a perturbed state (the
  second-order predictor from the cached species state).
* HYP_MIXED: within 3e-9 relative. The mixed closure evaluates the electronic levels with
  x = theta / T >= 9 in binary32; such a level holds at most (g_l / g_0) x e^-x <= 6 * 9 e^-9 =
  6.7e-3 of R_s T (g_l / g_0 <= 6 in both gas tables; the next weak level of a species holds far
  less), and its binary32 Boltzmann factor errs by about (1.5 x + 3) 2^-24 relative (the rounding
  of 1/T and of theta / T scaled by x, expf within 2 ulp, a product): 1e-6 at x = 9. So e_s moves
  by <= ~7e-9 R_s T and T by that over c_v,s: >= 2.5 R_s for the molecule with the ratio 6, and
  the atoms at their ratio 2.5 have >= 1.5 R_s: <= ~2e-9 T. The binary32 heat capacity enters
  only through the last Newton step, below 1e-6 T: 1e-13.
"""
import numpy as np
import pytest

from gpu_util import gpu_state, oracle_case
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [I.sbli_case(256, 96, seed=3), I.bl_case(48, 32)]
IDS = ["sbli_256x96", "bl_48x32"]


def _temperature(A, gas, st, U_host, precision, ncells):
    import torch
    U = torch.as_tensor(np.asarray(U_host), dtype=torch.float64).cuda()
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R, precision=precision)
    T = torch.empty(ncells, dtype=torch.float64, device="cuda")
    A.grid_temperature(st.grid, T)
    torch.cuda.synchronize()
    return T.cpu().numpy()


def _oracle_T(case, U):
    _, parts = F.rhs(case, U, return_parts=True)
    return (parts["T"] * case.sc.T_ref).ravel()


@pytest.mark.parametrize("cfg", CASES, ids=IDS)
@pytest.mark.parametrize("precision,bound", [(0, 1e-13), (1, 3e-9)], ids=["fp64", "mixed"])
def test_grid_temperature_matches_oracle(table, cfg, precision, bound):
    from paper_2210_05547_gb300 import abi as A
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    U1 = case.U0
    U2 = case.U0 * (1.0 + 1e-5 * np.cos(np.arange(case.U0.size)))   # a nearby state
    for U in (U1, U2):
        g = _temperature(A, gas, st, U, precision, cfg["nx"] * cfg["ny"])
        o = _oracle_T(case, U)
        err = np.max(np.abs(g - o) / o)
        assert err < bound, (precision, err)
    assert A.grid_status(st.grid) == 0


def test_grid_temperature_arguments():
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.bl_case(48, 32)
    gas, st = gpu_state(cfg)
    n = cfg["nx"] * cfg["ny"]
    R = torch.empty_like(st.U)
    # a fresh grid has no closure to read until a right-hand side or stage has run
    _, fresh = gpu_state(cfg)
    with pytest.raises(A.HypError, match="no closure"):
        A.grid_temperature(fresh.grid, torch.empty(n, dtype=torch.float64, device="cuda"))
    A.rhs(gas, st.grid, st.U, R)
    with pytest.raises(A.HypError, match="one double per cell"):
        A.grid_temperature(st.grid, torch.empty(n - 1, dtype=torch.float64, device="cuda"))
    T = torch.empty(n, dtype=torch.float64, device="cuda")
    A.grid_temperature(st.grid, T)
    torch.cuda.synchronize()
    assert torch.isfinite(T).all() and (T > 0).all()
