"""GPU parity on eleven-species air (ions and electrons; libhyp11.so) through the C ABI against
the oracle: the pointwise closure on charge-neutral seeded states, the state initialisation, the
right-hand side of a boundary layer and a shock interaction with ions and electrons present (their
ambipolar diffusion and the zero-current electron flux active), three RK3 steps, the mixed
precision closure, and batched members bit-identical to alone. Tolerances as for five species
(test_gpu_thermo.py, test_gpu_rhs.py)."""
import numpy as np
import pytest

from gpu_util import check_rhs, field_errors, gpu_rhs, gpu_state, normwise, oracle_case
from oracle import flow as F
from oracle import gas as G
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NS = 11


@pytest.fixture(scope="module")
def A():
    from paper_2210_05547_gb300 import abi
    abi.lib(NS)
    return abi


@pytest.fixture(scope="module")
def gas(A):
    return A.gas_model_load(I.with_species(I.bl_case()))


def _run(A, gas, rho, e, Y, precision=0):
    import torch
    n = rho.size
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()
    out = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in ("T", "p", "mu", "k")}
    out["wdot"] = torch.empty((NS, n), dtype=torch.float64, device="cuda")
    out["D"] = torch.empty((NS, n), dtype=torch.float64, device="cuda")
    out["status"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    A.thermo_eval(gas, t(rho), t(e), t(Y), precision=precision, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n", [1, 257, 20011])
def test_thermo_eval_parity(A, gas, table11, n):
    T, rho, Y = I.charged_states(n, table11.M(), table11.charge(), seed=7)
    e = G.mixture_energy(table11, T, Y)
    g = _run(A, gas, rho, e, Y)
    o = G.thermo_eval(table11, rho, e, Y)
    assert not g["status"].any()
    assert np.max(np.abs(g["T"] - o["T"]) / o["T"]) < 1e-13
    for k in ("p", "mu", "k"):
        assert np.max(np.abs(g[k] - o[k]) / np.abs(o[k])) < 1e-12, k
    heavy = table11.heavy()
    assert np.max(np.abs(g["D"][heavy] - o["D"][heavy]) / np.abs(o["D"][heavy])) < 1e-12
    assert not g["D"][table11.electron()].any()
    scale = np.max(np.abs(o["wdot"]), axis=0) + 1e-300
    assert np.max(np.abs(g["wdot"] - o["wdot"]) / scale) < 1e-10
    for s in range(NS):
        assert normwise(g["wdot"][s], o["wdot"][s]) < 1e-12, s


def test_thermo_eval_mixed(A, gas, table11):
    T, rho, Y = I.charged_states(4099, table11.M(), table11.charge(), seed=8)
    e = G.mixture_energy(table11, T, Y)
    g = _run(A, gas, rho, e, Y, precision=1)
    o = G.thermo_eval(table11, rho, e, Y)
    assert np.max(np.abs(g["T"] - o["T"]) / o["T"]) < 1e-13
    err = {k: float(np.max(np.abs(g[k] - o[k]) / np.abs(o[k]))) for k in ("mu", "k")}
    assert max(err.values()) < 4e-6 and max(err.values()) > 1e-9, err


def _ionised(case, table11, frac=0.3):
    """The case's initial state with a fraction of NO and O inside the layer turned into NO+ and
    O+ (and their electrons): a neutral state that exercises ion diffusion and the electron flux.
    At 30% the state is far from equilibrium and its recombination far too fast for the case's
    explicit time step, which is fine for single right-hand sides; stepped states use 1e-4."""
    cfg = case.cfg
    nx, ny = cfg["nx"], cfg["ny"]
    f = F.unpack(NS, nx, ny, case.U0)
    names = [s.name for s in table11.species]
    M = table11.M()
    i_no, i_o = names.index("NO"), names.index("O")
    i_nop, i_op, i_e = names.index("NO+"), names.index("O+"), table11.electron()
    f[f"rs{i_nop}"] = frac * f[f"rs{i_no}"]
    f[f"rs{i_op}"] = 0.5 * frac * f[f"rs{i_o}"]
    f[f"rs{i_no}"] = (1.0 - frac) * f[f"rs{i_no}"]
    f[f"rs{i_o}"] = (1.0 - 0.5 * frac) * f[f"rs{i_o}"]
    f[f"rs{i_e}"] = M[i_e] * (f[f"rs{i_nop}"] / M[i_nop] + f[f"rs{i_op}"] / M[i_op])
    return F.pack(NS, nx, ny, f)


CASES = {
    "bl_air11_64x40": I.with_species(I.bl_case(64, 40, seed=12)),
    "sbli_air11_96x40": I.with_species(I.sbli_case(96, 40, seed=13)),
    "bl_air11_ragged_77x29": I.with_species(I.bl_case(77, 29, seed=14)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_state_init_and_rhs_parity(A, table11, name):
    cfg = CASES[name]
    gas_, st = gpu_state(cfg)
    case = oracle_case(table11, cfg)
    for k, v in field_errors(cfg, st.U.cpu().numpy(), case.U0, ns=NS).items():
        assert v < 1e-13, ("U0", k, v)
    for U in (case.U0, _ionised(case, table11)):
        g = gpu_rhs(gas_, st, U)
        bad, o = check_rhs(case, U, g)
        assert not bad, bad
    # charge conservation of the GPU right-hand side at the neutral ionised state
    R = F.unpack(NS, cfg["nx"], cfg["ny"], g)
    q, M = table11.charge(), table11.M()
    rate = sum(q[s] * R[f"rs{s}"] / M[s] for s in range(1, NS))
    scale = max(np.abs(R[f"rs{s}"] / M[s]).max() for s in range(1, NS) if q[s] != 0)
    assert np.abs(rate).max() <= 1e-12 * scale


def test_rk3_steps_follow_the_oracle(A, table11):
    """Three RK3 steps of the interaction with ions and electrons: every stage's right-hand side
    checked at the GPU state, the final state within 1e-13 of the oracle's plus the carried
    right-hand-side differences."""
    from gpu_util import assert_states, follow_stages
    cfg = I.with_species(I.sbli_case(128, 48, seed=15))
    gas_, st = gpu_state(cfg)
    case = oracle_case(table11, cfg)
    failures, Ug, Uo, bound = follow_stages(
        table11, cfg, st, gas_, 3, "air11_sbli_128x48", U0=_ionised(case, table11, 1e-4),
        stage_fn=lambda k: A.rk_stage(st, k, cfg["dt"]))
    assert not failures, failures[:3]
    assert_states(cfg, Ug, Uo, bound, ns=NS)
    assert A.grid_status(st.grid) == 0


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_members_identical_alone_and_in_a_batch(A, precision):
    import torch
    cfgs = [I.with_species(I.sbli_case(160, 48, seed=16)), I.with_species(I.bl_case(96, 40, seed=17))]
    states = [gpu_state(c) for c in cfgs]
    batch = A.Batch(precision, use_graph=True, tile=1024, species=NS)
    for (_, st), c in zip(states, cfgs):
        batch.add(st, c["dt"])
    batch.step(3)
    torch.cuda.synchronize()
    for (_, st), c in zip(states, cfgs):
        _, ref = gpu_state(c)
        for _ in range(3):
            for k in range(3):
                A.rk_stage(ref, k, c["dt"], precision=precision)
        assert torch.equal(st.U, ref.U), c["name"]
