"""GPU parity of the pointwise closure (Sec. 2.2) through the C ABI: hyp_thermo_eval and
hyp_thermo_energy against the oracle on seeded states, edge cases, and the full 1e8-state sweep
with sampled parity and bit-reproducibility."""
import numpy as np
import pytest

from gpu_util import normwise
from oracle import gas as G
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# Tolerances (FP64): T from a converged Newton agrees to the cancellation floor of
# sum Y_s e_s (formation energies ~3e7 J/kg against c_v T); every other output is a smooth
# function of T, rho, Y evaluated with correctly rounded-ish FP64 libm calls on both sides.
TOL_T = 1e-13
TOL_PROP = 1e-12


@pytest.fixture(scope="module")
def A():
    from paper_2210_05547_gb300 import abi
    abi.lib()
    return abi


@pytest.fixture(scope="module")
def gas(A):
    return A.gas_model_load(I.bl_case())


def run_gpu(A, gas, rho, e, Y):
    import torch
    n = rho.size
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()
    out = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in ("T", "p", "mu", "k")}
    out["wdot"] = torch.empty((5, n), dtype=torch.float64, device="cuda")
    out["D"] = torch.empty((5, n), dtype=torch.float64, device="cuda")
    out["status"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    A.thermo_eval(gas, t(rho), t(e), t(Y), **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n", [1, 257, 20011])
def test_thermo_eval_parity(A, gas, table, n):
    T, rho, Y = I.thermo_states(n, seed=5)
    e = G.mixture_energy(table, T, Y)
    g = run_gpu(A, gas, rho, e, Y)
    o = G.thermo_eval(table, rho, e, Y)
    assert not g["status"].any()
    assert np.max(np.abs(g["T"] - o["T"]) / o["T"]) < TOL_T
    for k in ("p", "mu", "k"):
        assert np.max(np.abs(g[k] - o[k]) / np.abs(o[k])) < TOL_PROP, k
    assert np.max(np.abs(g["D"] - o["D"]) / np.abs(o["D"])) < TOL_PROP
    # production rates: per point relative to the largest |w_s| at that point, and normwise
    scale = np.max(np.abs(o["wdot"]), axis=0) + 1e-300
    assert np.max(np.abs(g["wdot"] - o["wdot"]) / scale) < 1e-10
    for s in range(5):
        assert normwise(g["wdot"][s], o["wdot"][s]) < TOL_PROP


def test_thermo_energy_parity(A, gas, table):
    import torch
    T, rho, Y = I.thermo_states(5003, seed=6)
    e = torch.empty(T.size, dtype=torch.float64, device="cuda")
    A.thermo_energy(gas, torch.as_tensor(T).cuda(), torch.as_tensor(Y).cuda(), e)
    ref = G.mixture_energy(table, T, Y)
    assert np.max(np.abs(e.cpu().numpy() - ref) / np.abs(ref).max()) < 1e-14


def test_edge_cases(A, gas, table):
    import torch
    # empty input is a no-op
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    A.thermo_eval(gas, z, z, z)
    # out-of-range energies clamp T and flag it; non-positive density is flagged
    Y = np.zeros((5, 3))
    Y[0] = 1.0
    e_lo = G.mixture_energy(table, np.array([G.T_MIN]), Y[:, :1])[0] - 1e5
    e_hi = G.mixture_energy(table, np.array([G.T_MAX]), Y[:, :1])[0] + 1e5
    e_ok = G.mixture_energy(table, np.array([900.0]), Y[:, :1])[0]
    g = run_gpu(A, gas, np.array([0.1, 0.1, -0.1]), np.array([e_lo, e_hi, e_ok]), Y)
    o = G.thermo_eval(table, np.array([0.1, 0.1, -0.1]), np.array([e_lo, e_hi, e_ok]), Y)
    assert g["T"][0] == G.T_MIN and g["T"][1] == G.T_MAX
    assert list(g["status"]) == list(o["status"]) == [2, 2, 4]
    assert abs(g["T"][2] / 900.0 - 1) < 1e-13


def test_full_sweep_1e8_sampled_and_reproducible(A, gas, table):
    """Thermochemistry-only sweep at full size (1e8 states): sampled outputs against the oracle,
    and two runs bitwise identical."""
    import torch
    n = 100_000_000
    rng = np.random.default_rng(7)
    T, rho, Y = I.thermo_states(n, seed=9)
    Td = torch.as_tensor(T).cuda()
    Yd = torch.as_tensor(Y).cuda()
    rhod = torch.as_tensor(rho).cuda()
    del T, rho
    ed = torch.empty(n, dtype=torch.float64, device="cuda")
    A.thermo_energy(gas, Td, Yd, ed)
    idx = np.sort(rng.choice(n, 2000, replace=False))
    Ts, Ys = Td[idx].cpu().numpy(), Y[:, idx]
    es = G.mixture_energy(table, Ts, Ys)            # oracle inputs for the sampled states
    ed[torch.as_tensor(idx).cuda()] = torch.as_tensor(es).cuda()
    outs = []
    for _ in range(2):
        Tg = torch.empty(n, dtype=torch.float64, device="cuda")
        wd = torch.empty((5, n), dtype=torch.float64, device="cuda")
        mu = torch.empty(n, dtype=torch.float64, device="cuda")
        A.thermo_eval(gas, rhod, ed, Yd, T=Tg, wdot=wd, mu=mu)
        outs.append((Tg, wd, mu))
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(outs[0], outs[1]))
    o = G.thermo_eval(table, rhod[idx].cpu().numpy(), es, Ys)
    Tg, wd, mu = (x.cpu().numpy() for x in outs[0])
    assert np.max(np.abs(Tg[idx] - o["T"]) / o["T"]) < TOL_T
    assert np.max(np.abs(mu[idx] - o["mu"]) / o["mu"]) < TOL_PROP
    wds = wd[:, idx]
    scale = np.max(np.abs(o["wdot"]), axis=0) + 1e-300
    assert np.max(np.abs(wds - o["wdot"]) / scale) < 1e-10
