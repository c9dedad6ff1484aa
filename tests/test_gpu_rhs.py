"""GPU parity of the right-hand side and the RK3 stage through the C ABI (hyp_state_init,
hyp_rhs, hyp_rk_stage) against the oracle: small grids that span several blocks with ragged
tails, every gas kind, with and without walls and artificial diffusivity; the 10-step run of
the Mach 10 boundary layer (256 x 64); and the full 2048 x 256 shock/boundary-layer case.

Tolerance, per conserved field per RHS: max |gpu - oracle| <= 1e-12 max |oracle| plus 32 times the
measured FP64 floor, the largest change of the oracle's right-hand side when every entry of the
state moves by one ulp (gpu_util.ulp_spread). The floor matters only where the RHS is a small
difference of large fluxes (rho*v in a boundary layer, where dp/dy comes from a pressure that is
uniform to the 1e-4 seeded noise). Achieved errors, the measured floor and the analytic rounding
bound of oracle.flow are written per field to the file named by HYP_PARITY_LOG.

Multi-step runs check every stage's right-hand side at the GPU's own state against the oracle at
that state, and the final GPU state against the oracle's within 1e-13 of each field plus the
difference the checked right-hand sides carry through the RK update (gpu_util.StateBound)."""
import numpy as np
import pytest

from gpu_util import (assert_states, check_rhs, field_errors, follow_stages, gpu_rhs, gpu_state,
                      nstate, normwise, oracle_case)
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu



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
        "bl_tpg_48x32": I.bl_case(48, 32, seed=4, kind="tpg"),
        "sbli_tpg_96x40": I.sbli_case(96, 40, seed=5, kind="tpg"),
        "bl_sm_64x40": dict(I.bl_case(64, 40, seed=8), diffusion_model="stefan_maxwell"),
        "sbli_sm_96x40": dict(I.sbli_case(96, 40, seed=9), diffusion_model="stefan_maxwell"),
        "bl_lte_64x40": I.bl_case(64, 40, seed=10, kind="lte"),
        "sbli_lte_96x40": I.sbli_case(96, 40, seed=11, kind="lte"),
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
    assert np.max(np.abs(sigma - osig)) <= 1e-14 * cfg["sponge_sigma"]


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_parity(table, name):
    cfg = CASES[name]
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    g = gpu_rhs(gas, st, case.U0)
    bad, o = check_rhs(case, case.U0, g, label=name)
    assert not bad, bad
    fg = F.unpack(5, cfg["nx"], cfg["ny"], g)
    assert not fg["rhou"][:, [0, -1]].any() and not fg["rhov"][[0, -1], :].any()
    from paper_2210_05547_gb300 import abi as A
    assert A.grid_status(st.grid) == 0


def test_rk3_ten_steps_boundary_layer(table):
    """Mach 10 boundary layer, 256 x 64, 10 RK steps: the RHS agrees at every one of the 30 stages
    and the states stay together."""
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.bl_case()
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    assert max(field_errors(cfg, st.U.cpu().numpy(), case.U0).values()) < 1e-13
    st.U.copy_(torch.as_tensor(case.U0).cuda())
    failures, Ug, Uo, bound = follow_stages(table, cfg, st, gas, 10, "bl_256x64_rk3",
                                      stage_fn=lambda k: A.rk_stage(st, k, cfg["dt"]))
    assert not failures, failures[:3]
    assert_states(cfg, Ug, Uo, bound)
    assert A.grid_status(st.grid) == 0


def test_state_filter_parity(table):
    """Stage 2 with dt = 0 on a fresh state (dQ = 0) leaves U unchanged and then applies the
    low-pass filter of the case: equal to the oracle's filter to rounding, and not a no-op."""
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.sbli_case(160, 48, seed=2)
    cfg["noise_amp"] = 1e-2
    cfg["filter_sigma"] = 0.2
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    U0 = st.U.cpu().numpy()
    A.rk_stage(st, 2, 0.0)
    torch.cuda.synchronize()
    got = F.unpack(5, cfg["nx"], cfg["ny"], st.U.cpu().numpy())
    ref = F.unpack(5, cfg["nx"], cfg["ny"], F.filter_state(case, U0))
    before = F.unpack(5, cfg["nx"], cfg["ny"], U0)
    for k in ref:
        scale = np.abs(ref[k]).max()
        assert np.abs(got[k] - ref[k]).max() <= 2e-15 * scale, k
        assert np.abs(ref[k] - before[k]).max() > 1e-6 * scale, k


def test_rk3_steps_with_filter_sbli(table):
    """Shock / boundary-layer case with the state filter on: 3 RK steps, every stage's RHS checked,
    GPU state against the oracle's within 1e-13 plus the carried right-hand-side differences (the
    filter multiplies a state difference by at most (1 + sigma) per pass in the max norm)."""
    from paper_2210_05547_gb300 import abi as A
    cfg = I.sbli_case(128, 48, seed=1)
    assert cfg["filter_sigma"] > 0
    gas, st = gpu_state(cfg)
    failures, Ug, Uo, bound = follow_stages(table, cfg, st, gas, 3, "sbli_128x48_filter",
                                      stage_fn=lambda k: A.rk_stage(st, k, cfg["dt"]))
    assert not failures, failures[:3]
    assert_states(cfg, Ug, Uo, bound)
    assert A.grid_status(st.grid) == 0


@pytest.mark.parametrize("scheme", ["tvd3", "ck4"])
@pytest.mark.parametrize("cfg", [I.bl_case(64, 40, seed=6), I.sbli_case(96, 40, seed=7)],
                         ids=["bl_64x40", "sbli_96x40"])
def test_other_schemes_parity(table, scheme, cfg):
    """TVD RK3 and the 2N-storage RK4 (Sec. 3.1) through hyp_rk_stage_scheme: 2 steps, every
    stage's RHS checked, GPU state against the oracle's within 1e-13 plus the carried
    right-hand-side differences."""
    from paper_2210_05547_gb300 import abi as A
    gas, st = gpu_state(cfg)
    failures, Ug, Uo, bound = follow_stages(
        table, cfg, st, gas, 2, f"{cfg['name']}_{scheme}", scheme=scheme,
        stage_fn=lambda k: A.rk_stage_scheme(st, scheme, k, cfg["dt"]))
    assert not failures, failures[:3]
    assert_states(cfg, Ug, Uo, bound)
    assert A.grid_status(st.grid) == 0
    with pytest.raises(A.HypError, match="stage out of range"):
        A.rk_stage_scheme(st, scheme, F.RK_STAGES[scheme], cfg["dt"])


def test_full_size_sbli_rhs(table):
    """The timed workload (2048 x 256, artificial diffusivity on): one full RHS against the
    oracle, every entry."""
    cfg = I.sbli_case()
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    g = gpu_rhs(gas, st, case.U0)
    bad, o = check_rhs(case, case.U0, g, label="sbli_2048x256_initial")
    assert not bad, bad


def test_full_size_sbli_rhs_after_twenty_steps(table):
    """The timed workload after 20 GPU RK3 steps (the interaction developing, the closure starting
    its Newton iteration from the cached species state of the previous stage, as in every timed
    right-hand side): one GPU right-hand side at that state against the oracle at that state,
    every entry."""
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.sbli_case()
    gas, st = gpu_state(cfg)
    for _ in range(20):
        for k in range(3):
            A.rk_stage(st, k, cfg["dt"])
    torch.cuda.synchronize()
    assert A.grid_status(st.grid) == 0
    U = st.U.cpu().numpy()
    R = torch.empty_like(st.U)
    A.rhs(gas, st.grid, st.U, R)        # predictor warmed by the last stage
    torch.cuda.synchronize()
    case = oracle_case(table, cfg)
    bad, o = check_rhs(case, U, R.cpu().numpy(), label="sbli_2048x256_step20")
    assert not bad, bad


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
