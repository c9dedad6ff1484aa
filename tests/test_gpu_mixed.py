"""Mixed-precision path (HYP_MIXED) through the C ABI, against the FP64 oracle.

HYP_MIXED evaluates the transport and diffusion coefficients (Blottner, Eucken, Wilke,
Chapman-Enskog; Sec. 2.2.1, Eq. 19), the forward-rate exponentials (Eq. 13), the species heat
capacities and the weakly populated electronic levels of the species thermodynamics (Sec. 2.2.1),
the Gaussian filter of the artificial diffusivities (Sec. 3.3) and the interior rows of the
compact operators that feed only the diffusive fluxes in binary32, the other derivatives'
recurrences in binary32 on binary64 differences, the other interpolations in double-word
binary32, and the rest (Newton iteration for T, the vibrational factors and populated electronic
levels that set e_s, equilibrium constants, backward rates, divergences, fluxes, stage update) in
binary64. The stated error of each output and the
bound held here:

* conversion (hyp_round_f32): equal to the hardware round-to-nearest-even for every result in the
  normal binary32 range, widening back exact;
* thermo_eval: T and p as the FP64 path (the sweep of independent states keeps the binary64
  modal sums; the right-hand side's binary32 electronic levels and their temperature bound are in
  test_gpu_temperature.py); mu, k, D within 4e-6 relative per state. The binary32 result of
  exp(x) carries the rounding of its argument, |x| 2^-24, and the Blottner exponent reaches
  |x| ~ 25 (1.5e-6); the binary32 sums of Wilke's rule and Eq. (19) add a few 2^-24;
* thermo_eval wdot: within 1e-5 of max|wdot_s| per species (forward-rate exponent up to ~40 at
  the states that dominate max|wdot|: 2.4e-6, times the few reactions feeding a species);
* rhs on the shock / boundary-layer interaction: within 1e-6 of max|R| per conserved field;
* rhs on the flat-plate boundary layer: within 1e-6 of the largest flux term entering each field
  (the y-momentum balance of the near-parallel layer cancels its viscous terms to a right-hand
  side ~1e-4 of them, so a normwise bound there would measure that cancellation, not the
  arithmetic);
* 1000 RK3 steps of the 2048 x 256 interaction: wall heat flux and skin friction within 1e-4
  normwise of the FP64 path.
"""
import numpy as np
import pytest

from gpu_util import gpu_state, normwise, oracle_case
from oracle import flow as F
from oracle import gas as G
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F32_MIN_NORMAL = 2.0 ** -126


@pytest.fixture(scope="module")
def A():
    from paper_2210_05547_gb300 import abi
    abi.lib()
    return abi


def test_round_f32_matches_hardware(A):
    import torch
    rng = np.random.default_rng(11)
    n = 200_000
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-140, 131, n)
    x = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], n)
    # exact ties between neighbouring binary32 values, and their neighbours one ulp (binary64) away
    f = rng.uniform(-3e5, 3e5, 4000).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    ties = (f.astype(np.float64) + g.astype(np.float64)) / 2.0
    special = np.array([0.0, -0.0, 1e-300, -1e-300, F32_MIN_NORMAL, np.nextafter(F32_MIN_NORMAL, 0),
                        3.4028234663852886e38, 3.4028235677973366e38, 1e300, -1e300, np.inf, -np.inf])
    x = np.concatenate([x, ties, np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf), special])
    xd = torch.as_tensor(x).cuda()
    y = torch.empty(x.size, dtype=torch.float32, device="cuda")
    back = torch.empty(x.size, dtype=torch.float64, device="cuda")
    A.round_f32(xd, y, back)
    hw = xd.to(torch.float32).cpu().numpy()
    got = y.cpu().numpy()
    normal = np.abs(x) >= F32_MIN_NORMAL
    assert np.array_equal(got[normal].view(np.uint32), hw[normal].view(np.uint32))
    sub = ~normal
    assert np.all(got[sub] == 0.0) and np.array_equal(np.signbit(got[sub]), np.signbit(x[sub]))
    assert np.array_equal(back.cpu().numpy(), got.astype(np.float64))
    nan = torch.tensor([np.nan], dtype=torch.float64, device="cuda")
    yn = torch.empty(1, dtype=torch.float32, device="cuda")
    A.round_f32(nan, yn)
    assert np.isnan(yn.cpu().numpy()[0])


def _thermo(A, gas, rho, e, Y, precision):
    import torch
    n = rho.size
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()
    out = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in ("T", "p", "mu", "k")}
    out["wdot"] = torch.empty((5, n), dtype=torch.float64, device="cuda")
    out["D"] = torch.empty((5, n), dtype=torch.float64, device="cuda")
    out["status"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    A.thermo_eval(gas, t(rho), t(e), t(Y), precision=precision, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_thermo_eval_mixed_errors(A, table):
    gas = A.gas_model_load(I.bl_case())
    T, rho, Y = I.thermo_states(20011, seed=7)
    e = G.mixture_energy(table, T, Y)
    g = _thermo(A, gas, rho, e, Y, A.MIXED)
    o = G.thermo_eval(table, rho, e, Y)
    assert not g["status"].any()
    assert np.max(np.abs(g["T"] - o["T"]) / o["T"]) < 1e-13
    assert np.max(np.abs(g["p"] - o["p"]) / o["p"]) < 1e-12
    err = {k: float(np.max(np.abs(g[k] - o[k]) / np.abs(o[k]))) for k in ("mu", "k", "D")}
    for k, v in err.items():
        assert v < 4e-6, (k, v)
    for s in range(5):
        assert normwise(g["wdot"][s], o["wdot"][s]) < 1e-5, s
    # the binary32 parts really run: the errors are those of binary32, not of binary64
    assert max(err.values()) > 1e-9


def _rhs(A, gas, st, U_host, precision):
    import torch
    U = torch.as_tensor(np.asarray(U_host), dtype=torch.float64).cuda()
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R, precision=precision)
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("cfg", [I.sbli_case(256, 96, seed=3), I.sbli_case(384, 64, seed=4)],
                         ids=["sbli_256x96", "sbli_384x64"])
def test_rhs_mixed_sbli_within_1e6(A, table, cfg):
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    o = F.unpack(5, cfg["nx"], cfg["ny"], F.rhs(case, case.U0))
    g = F.unpack(5, cfg["nx"], cfg["ny"], _rhs(A, gas, st, case.U0, A.MIXED))
    err = {k: normwise(g[k], o[k]) for k in o}
    assert max(err.values()) <= 1e-6, err
    assert max(err.values()) > 1e-12             # binary32 arithmetic is in the result


def test_rhs_mixed_boundary_layer_against_flux_scale(A, table):
    cfg = I.bl_case(128, 64)
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    R, parts = F.rhs(case, case.U0, return_parts=True)
    o = F.unpack(5, cfg["nx"], cfg["ny"], R)
    g = F.unpack(5, cfg["nx"], cfg["ny"], _rhs(A, gas, st, case.U0, A.MIXED))
    for k in o:
        assert np.abs(g[k] - o[k]).max() <= 1e-6 * parts["gross"][k], k


def test_rhs_mixed_is_deterministic(A):
    """Two grids built from the same case give bit-identical mixed right-hand sides (a grid's
    first evaluation starts the temperature inversion from the same cached state; later ones
    start from the previous call's, which moves T within the Newton tolerance)."""
    cfg = I.sbli_case(512, 128, seed=5)
    outs = []
    for _ in range(2):
        gas, st = gpu_state(cfg)
        outs.append(_rhs(A, gas, st, st.U.cpu().numpy(), A.MIXED))
    assert np.array_equal(outs[0], outs[1])


def test_wall_fluxes_match_oracle(A, table):
    import torch
    cfg = I.sbli_case(192, 64, seed=6)
    gas, st = gpu_state(cfg)
    case = oracle_case(table, cfg)
    U = torch.as_tensor(case.U0).cuda()
    q = torch.empty(cfg["nx"], dtype=torch.float64, device="cuda")
    tw = torch.empty(cfg["nx"] + 1, dtype=torch.float64, device="cuda")
    A.wall_fluxes(gas, st.grid, U, q, tw)
    qo, to = F.wall_fluxes(case, case.U0)
    assert normwise(q.cpu().numpy(), qo) < 1e-12
    assert normwise(tw.cpu().numpy(), to) < 1e-12
    # mixed: q_w and tau_w carry the binary32 conductivity and viscosity, interpolated to the
    # wall faces and corners (the per-state 4e-6 of thermo_eval plus the interpolation's sums)
    A.wall_fluxes(gas, st.grid, U, q, tw, precision=A.MIXED)
    assert normwise(q.cpu().numpy(), qo) < 1e-5
    assert normwise(tw.cpu().numpy(), to) < 1e-5


def test_mixed_1000_steps_wall_quantities():
    """The 2048 x 256 interaction advanced 1000 RK3 steps in each precision from the same initial
    state: wall heat flux and skin friction C_f = 2 tau_w / Ma^2 agree within 1e-4 normwise."""
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.sbli_case(2048, 256, seed=0)
    out = {}
    for prec in (A.FP64, A.MIXED):
        gas, st = gpu_state(cfg)
        for _ in range(1000):
            for k in range(3):
                A.rk_stage(st, k, cfg["dt"], precision=prec)
        q = torch.empty(cfg["nx"], dtype=torch.float64, device="cuda")
        tw = torch.empty(cfg["nx"] + 1, dtype=torch.float64, device="cuda")
        A.wall_fluxes(gas, st.grid, st.U, q, tw, precision=prec)
        assert A.grid_status(st.grid) == 0
        assert torch.isfinite(st.U).all()
        out[prec] = (q.cpu().numpy(), 2.0 * tw.cpu().numpy() / cfg["mach"] ** 2)
    eq = normwise(out[A.MIXED][0], out[A.FP64][0])
    ecf = normwise(out[A.MIXED][1], out[A.FP64][1])
    assert eq < 1e-4 and ecf < 1e-4, (eq, ecf)
