"""GPU parity of the right-hand side and the RK3 stage through the C ABI (hyp_state_init,
hyp_rhs, hyp_rk_stage) against the oracle: small grids that span several blocks with ragged
tails, every gas kind, with and without walls and artificial diffusivity; the 10-step run of
the Mach 10 boundary layer (256 x 64); and the full 2048 x 256 shock/boundary-layer case.

Tolerance: 1e-12 normwise relative per conserved field per right-hand side (max |gpu - oracle|
over the field / max |oracle| over the field)."""
import numpy as np
import pytest

from gpu_util import field_errors, gpu_rhs, gpu_state, nstate, normwise, oracle_case
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _cases():
    bl_cpg = I.bl_case(48, 32, kind="cpg")
    bl_frozen = I.bl_case(48, 32, kind="frozen")
    sbli_cpg = I.sbli_case(96, 40, kind="cpg")
    return {
        "box_24x16": I.box_case(24, 16),
        "bl_64x40": I.bl_case(64, 40),
        "bl_ragged_77x29": I.bl_case(77, 29, seed=3),
        "bl_min_8x8": I.bl_case(8, 8),
        "bl_cpg_48x32": bl_cpg,
        "bl_frozen_48x32": bl_frozen,
        "sbli_100x37": I.sbli_case(100, 37, seed=1),
        "sbli_cpg_96x40": sbli_cpg,
        "sbli_frozen_64x33": I.sbli_case(64, 33, seed=2, kind="frozen"),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_state_init_parity(table, name):
    cfg = CASES[name]
    gas, st = gpu_state(cfg)
    import torch
    torch.cuda.synchronize()
    case = oracle_case(table, cfg)
    from paper_2210_05547_gb300 import abi as A
    Uref, sigma = A.grid_reference(st.grid, nstate(cfg))
    for k, v in field_errors(cfg, st.U.cpu().numpy(), case.U0).items():
        assert v < 1e-13, ("U0", k, v)
    for k, v in field_errors(cfg, Uref, case.U_ref).items():
        assert v < 1e-13, ("Uref", k, v)
    osig = F.pack(5, cfg["nx"], cfg["ny"], {
        n: case.sigma["xf" if n == "rhou" else "yf" if n == "rhov" else "c"]
        for n, _ in F.state_layout(5, cfg["nx"], cfg["ny"])})
    assert np.max(np.abs(sigma - osig)) < 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_parity(table, name):
    cfg = CASES[name]
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    g = gpu_rhs(gas, st, case.U0)
    o = F.rhs(case, case.U0)
    errs = field_errors(cfg, g, o)
    assert max(errs.values()) < TOL, errs
    fg = F.unpack(5, cfg["nx"], cfg["ny"], g)
    assert not fg["rhou"][:, [0, -1]].any() and not fg["rhov"][[0, -1], :].any()


def test_rk3_ten_steps_boundary_layer(table):
    """Mach 10 boundary layer, 256 x 64, 10 RK steps: the RHS agrees at every one of the 30 stages
    and the states stay together."""
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.bl_case()
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    U = case.U0.copy()
    dQ = np.zeros_like(U)
    assert max(field_errors(cfg, st.U.cpu().numpy(), U).values()) < 1e-13
    st.U.copy_(torch.as_tensor(U).cuda())
    worst = 0.0
    for step in range(10):
        for k in range(3):
            Rg = gpu_rhs(gas, st, st.U.cpu().numpy())
            U, dQ, Ro = F.rk_stage(case, U, dQ, k, cfg["dt"])
            worst = max(worst, max(field_errors(cfg, Rg, Ro).values()))
            A.rk_stage(st, k, cfg["dt"])
    torch.cuda.synchronize()
    assert worst < TOL, worst
    errs = field_errors(cfg, st.U.cpu().numpy(), U)
    assert max(errs.values()) < 1e-13, errs
    assert A.grid_status(st.grid) == 0


def test_full_size_sbli_rhs(table):
    """The timed workload (2048 x 256, artificial diffusivity on): one full RHS against the
    oracle, every entry."""
    cfg = I.sbli_case()
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    g = gpu_rhs(gas, st, case.U0)
    o = F.rhs(case, case.U0)
    errs = field_errors(cfg, g, o)
    assert max(errs.values()) < TOL, errs


def test_status_flag_and_errors(table):
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.bl_case(32, 16)
    gas, st = gpu_state(cfg)
    U = st.U.clone()
    U[5] = -abs(float(U[5]))            # one cell with negative density
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R)
    assert A.grid_status(st.grid, clear=True) & 4
    assert A.grid_status(st.grid) == 0
    with pytest.raises(A.HypError, match="alias"):
        A.rhs(gas, st.grid, U, U)
    with pytest.raises(A.HypError, match="stage"):
        A.rk_stage(st, 3, 1e-4)
