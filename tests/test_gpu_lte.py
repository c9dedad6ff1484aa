"""GPU parity of the closure in local thermodynamic equilibrium (Sec. 2.2.2) through the C ABI:
hyp_lte_eval against the oracle's lte_eval over 300-15000 K and 1e-4-1 kg/m^3, its edge cases,
the binary32-transport variant, and LTE grids stepped in a batch (bit-identical to alone). The
right-hand-side parity of the LTE kind is in test_gpu_rhs.py.

Tolerances (FP64): T from converged Newton iterations agrees to the cancellation floor of the
mixture energy (formation energies against c_v T, as for the finite-rate closure); the
composition is the Newton-converged element-potential solution on both sides, so mass fractions
agree to a few ulps of 1; p, mu, k_frozen are smooth functions of those. The reactive
conductivity is a sum of terms of both signs (h_s - h changes sign across the species): it is held
to 1e-11 of the total conductivity."""
import numpy as np
import pytest

from gpu_util import gpu_state, oracle_case
from oracle import gas as G
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

Y_AIR = np.array([0.767, 0.233, 0.0, 0.0, 0.0])


@pytest.fixture(scope="module")
def A():
    from paper_2210_05547_gb300 import abi
    abi.lib()
    return abi


@pytest.fixture(scope="module")
def gas(A):
    return A.gas_model_load(I.bl_case(kind="lte"))


def _states(table, n, seed):
    T, rho, _ = I.thermo_states(n, seed=seed)
    bm = G.element_content(table, Y_AIR)
    _, e, _, _ = G.equilibrium_at(table, T, rho, bm)
    return T, rho, e, bm


def _run(A, gas, rho, e, precision=0):
    import torch
    n = rho.size
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()
    out = {k: torch.empty(n, dtype=torch.float64, device="cuda")
           for k in ("T", "p", "mu", "k", "k_reactive")}
    out["Y"] = torch.empty((5, n), dtype=torch.float64, device="cuda")
    out["status"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    A.lte_eval(gas, t(rho), t(e), precision=precision, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n", [1, 257, 4099])
def test_lte_eval_parity(A, gas, table, n):
    T, rho, e, bm = _states(table, n, seed=21)
    g = _run(A, gas, rho, e)
    o = G.lte_eval(table, rho, e, bm)
    assert not g["status"].any() and not o["status"].any()
    assert np.max(np.abs(g["T"] / o["T"] - 1.0)) < 1e-13
    assert np.max(np.abs(g["T"] / T - 1.0)) < 1e-13
    assert np.max(np.abs(g["Y"] - o["Y"])) < 1e-13
    for k in ("p", "mu"):
        assert np.max(np.abs(g[k] / o[k] - 1.0)) < 1e-12, k
    assert np.max(np.abs(g["k"] - o["k"]) / o["k"]) < 1e-11
    assert np.max(np.abs(g["k_reactive"] - o["k_reactive"]) / o["k"]) < 1e-11
    if n > 1000:
        # the states exercise the equilibrium: dissociation and a large reactive conductivity
        assert g["Y"][3].max() > 0.5 and np.max(g["k_reactive"] / g["k"]) > 0.5


def test_lte_eval_edges(A, gas, table):
    """Energies below e(50 K) and above e(1e5 K) clamp with the status bit; rho <= 0 is flagged."""
    bm = G.element_content(table, Y_AIR)
    rho = np.array([0.1, 0.1, 0.1, -1.0])
    _, e_lo, _, _ = G.equilibrium_at(table, np.array([50.0]), np.array([0.1]), bm)
    _, e_hi, _, _ = G.equilibrium_at(table, np.array([1e5]), np.array([0.1]), bm)
    _, e_mid, _, _ = G.equilibrium_at(table, np.array([3000.0]), np.array([0.1]), bm)
    e = np.array([e_lo[0] - 1e5, e_hi[0] * 1.5, e_mid[0], e_mid[0]])
    g = _run(A, gas, rho, e)
    assert g["status"][0] & 2 and g["T"][0] == 50.0
    assert g["status"][1] & 2 and g["T"][1] == 1e5
    assert g["status"][2] == 0 and abs(g["T"][2] / 3000.0 - 1.0) < 1e-13
    assert g["status"][3] & 4


def test_lte_eval_mixed(A, gas, table):
    """HYP_MIXED: binary32 viscosity, frozen conductivity and diffusion coefficients (the latter
    entering k_reactive); temperature, pressure and composition stay FP64."""
    T, rho, e, bm = _states(table, 4099, seed=22)
    g = _run(A, gas, rho, e, precision=1)
    o = G.lte_eval(table, rho, e, bm)
    assert np.max(np.abs(g["T"] / o["T"] - 1.0)) < 1e-13
    assert np.max(np.abs(g["Y"] - o["Y"])) < 1e-13
    err_mu = np.max(np.abs(g["mu"] / o["mu"] - 1.0))
    err_k = np.max(np.abs(g["k"] / o["k"] - 1.0))
    assert err_mu < 4e-6 and err_k < 1e-5, (err_mu, err_k)
    assert max(err_mu, err_k) > 1e-9                 # binary32 is really in the result


def test_lte_gas_rejects_the_other_closure(A, gas):
    import torch
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    Y = torch.ones((5, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(A.HypError, match="hyp_lte_eval"):
        A.thermo_eval(gas, x, x, Y, T=torch.empty_like(x))
    cneq = A.gas_model_load(I.bl_case())
    with pytest.raises(A.HypError, match="needs an LTE gas"):
        A.lte_eval(cneq, x, x, T=torch.empty_like(x))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_lte_members_identical_alone_and_in_a_batch(A, precision):
    import torch
    cfgs = [I.sbli_case(160, 48, seed=3, kind="lte"), I.bl_case(96, 40, seed=4, kind="lte")]
    states = [gpu_state(c) for c in cfgs]
    batch = A.Batch(precision, use_graph=True, tile=1024)
    for (_, st), c in zip(states, cfgs):
        batch.add(st, c["dt"])
    batch.step(3)
    torch.cuda.synchronize()
    for (_, st), c in zip(states, cfgs):
        _, ref = gpu_state(c)
        for _ in range(3):
            for k in range(3):
                A.rk_stage(ref, k, c["dt"], precision=precision)
        assert A.grid_status(ref.grid) == 0
        assert torch.equal(st.U, ref.U), c["name"]


def test_lte_steps_follow_the_oracle(A, table):
    """Three RK3 steps of the interaction in LTE: each stage's right-hand side checked at the GPU
    state, and the state within the carried bound."""
    from gpu_util import assert_states, follow_stages
    cfg = I.sbli_case(128, 48, seed=6, kind="lte")
    gas_, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    failures, Ug, Uo, bound = follow_stages(table, cfg, st, gas_, 3, "lte_sbli_128x48",
                                            U0=case.U0,
                                            stage_fn=lambda k: A.rk_stage(st, k, cfg["dt"]))
    assert not failures, failures[:3]
    assert_states(cfg, Ug, Uo, bound)
    assert A.grid_status(st.grid) == 0
