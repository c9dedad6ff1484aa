"""GPU parity of three-dimensional grids (spanwise-periodic z, jet from a circular orifice) through
the C ABI (hyp_state_init, hyp_rhs, hyp_rk_stage with nz > 1) against oracle/flow3d.py: the
initial and reference states, the right-hand side of a jet in crossflow with artificial
diffusivity, of a boundary layer without the jet, of a calorically perfect gas, and three RK3
steps; the mixed-precision right-hand side. Tolerance as in two dimensions
(oracle.flow3d.parity_tolerance): 1e-12 of max|R| per
field plus the FP64 rounding floor of the flux divergences, the sponge term on noise-level
differences and the temperature conditioning of the Arrhenius sources."""
import numpy as np
import pytest

from oracle import flow3d as F3
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _n(cfg, ns=5):
    return sum(a * b * c for _, (a, b, c) in F3.state_layout(ns, cfg["nx"], cfg["ny"], cfg["nz"]))


def _zoom(cfg):
    """The jet case on a small box around the orifice (resolved by the few cells of a test)."""
    cfg.update(x0=50.0, x1=55.0, z0=0.0, z1=3.0, jet_x=52.5, jet_z=1.5, sponge_in=0.5,
               sponge_out=0.5)
    return cfg


def _cases():
    jet = _zoom(I.jet_case(40, 24, 12, seed=1))
    bl = dict(I.bl_case(36, 20, seed=2), nz=8, z0=0.0, z1=2.0, jet=0)
    cpg = dict(_zoom(I.jet_case(40, 24, 12, seed=3, kind="cpg")), artificial_diffusivity=0)
    frozen = _zoom(I.jet_case(41, 21, 13, seed=4, kind="frozen"))
    return {"jet_40x24x12": jet, "bl_36x20x8": bl, "jet_cpg_40x24x12": cpg,
            "jet_frozen_41x21x13": frozen}


CASES = _cases()


def _gpu(cfg, ns=5):
    import torch
    from paper_2210_05547_gb300 import abi as A
    gas = A.gas_model_load(cfg)
    n = A.state_size(gas, cfg)
    assert n == _n(cfg, ns)
    U = torch.empty(n, dtype=torch.float64, device="cuda")
    dQ = torch.empty_like(U)
    st = A.state_init(gas, cfg, U, dQ, I.state_noise(n, cfg["seed"]))
    return A, gas, st


def _errors(cfg, a, b, ns=5):
    fa = F3.unpack(ns, cfg["nx"], cfg["ny"], cfg["nz"], np.asarray(a))
    fb = F3.unpack(ns, cfg["nx"], cfg["ny"], cfg["nz"], np.asarray(b))
    return {k: float(np.abs(fa[k] - fb[k]).max() / max(np.abs(fb[k]).max(), 1e-300)) for k in fa}


def _check(case, U, g, label=None):
    """Three-dimensional parity with the measured floor of gpu_util (1e-12 max|o| plus 32 times the
    largest change of the oracle's right-hand side under one-ulp moves of every state entry); the
    analytic tolerance of oracle.flow3d is recorded beside it."""
    from gpu_util import parity_report, ulp_spread
    tol, o = F3.parity_tolerance(case, U)
    cfg, ns = case.cfg, case.tab.ns

    def unpack(v):
        return F3.unpack(ns, cfg["nx"], cfg["ny"], cfg["nz"], np.asarray(v))

    spread = ulp_spread(lambda V: F3.rhs(case, V), unpack, U, o)
    bad, _ = parity_report(label or cfg["name"], unpack(g), unpack(o), spread, tol)
    return bad


@pytest.mark.parametrize("name", list(CASES))
def test_state_init_and_rhs_parity(table, name):
    import torch
    cfg = CASES[name]
    A, gas, st = _gpu(cfg)
    case = F3.make_case(cfg, table, I.state_noise(_n(cfg), cfg["seed"]))
    torch.cuda.synchronize()
    for k, v in _errors(cfg, st.U.cpu().numpy(), case.U0).items():
        assert v < 1e-13, ("U0", k, v)
    Uref, sigma = A.grid_reference(st.grid, _n(cfg))
    for k, v in _errors(cfg, Uref, case.U_ref).items():
        assert v < 1e-13, ("Uref", k, v)
    # the right-hand side at the oracle's state (the two initial states differ by rounding,
    # which the Mach-number cancellation in e = E - |u|^2/2 would amplify)
    U = torch.as_tensor(case.U0).cuda()
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R)
    torch.cuda.synchronize()
    bad = _check(case, case.U0, R.cpu().numpy(), label=f"3d_{name}")
    assert not bad, bad
    assert A.grid_status(st.grid) == 0


@pytest.mark.parametrize("name", ["jet_40x24x12", "bl_36x20x8"])
def test_rhs_mixed_within_1e6_of_the_flux_scale(table, name):
    """HYP_MIXED on three-dimensional grids: binary32 transport, diffusion coefficients and
    forward-rate exponentials in the closure, binary32 rows in the line jobs that feed only the
    diffusive fluxes (periodic z lines included); within 1e-6 of the larger of max|R| and the
    largest flux term entering each field (the spanwise momentum of the layer without the jet is a
    noise-level balance of much larger terms)."""
    import torch
    cfg = CASES[name]
    A, gas, st = _gpu(cfg)
    case = F3.make_case(cfg, table, I.state_noise(_n(cfg), cfg["seed"]))
    U = torch.as_tensor(case.U0).cuda()
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R, precision=A.MIXED)
    torch.cuda.synchronize()
    o, parts = F3.rhs(case, case.U0, return_parts=True)
    fg = F3.unpack(5, cfg["nx"], cfg["ny"], cfg["nz"], R.cpu().numpy())
    fo = F3.unpack(5, cfg["nx"], cfg["ny"], cfg["nz"], o)
    err = {k: float(np.abs(fg[k] - fo[k]).max() / max(np.abs(fo[k]).max(), parts["gross"][k]))
           for k in fo}
    assert max(err.values()) <= 1e-6, err
    assert max(err.values()) > 1e-12, err          # binary32 arithmetic is in the result
    assert A.grid_status(st.grid) == 0


def test_rk3_steps_follow_the_oracle(table):
    """Three RK3 steps of the jet: every stage's right-hand side at the GPU state checked against
    the oracle at that state; the final state within 1e-13 of the oracle's plus the carried
    right-hand-side differences (two-register update, gpu_util.StateBound)."""
    import torch
    from gpu_util import StateBound
    cfg = CASES["jet_40x24x12"]
    A, gas, st = _gpu(cfg)
    case = F3.make_case(cfg, table, I.state_noise(_n(cfg), cfg["seed"]))
    U = case.U0.copy()
    dQ = np.zeros_like(U)
    st.U.copy_(torch.as_tensor(U).cuda())
    dims = (5, cfg["nx"], cfg["ny"], cfg["nz"])
    bound = StateBound([name for name, _ in F3.state_layout(*dims)])
    failures = []
    for step in range(3):
        for k in range(3):
            Ug = st.U.cpu().numpy()
            Rg = torch.empty_like(st.U)
            A.rhs(gas, st.grid, st.U, Rg)
            torch.cuda.synchronize()
            Rg = Rg.cpu().numpy()
            bad = _check(case, Ug, Rg, label=f"3d_jet_40x24x12/step{step}/stage{k}")
            if bad:
                failures.append((step, k, bad))
            U, dQ, Ro = F3.rk_stage(case, U, dQ, k, cfg["dt"])
            fg, fo = F3.unpack(*dims, Rg), F3.unpack(*dims, Ro)
            bound.stage(k, cfg["dt"], {n: float(np.abs(fg[n] - fo[n]).max()) for n in fo})
            A.rk_stage(st, k, cfg["dt"])
    torch.cuda.synchronize()
    assert not failures, failures[:3]
    fg = F3.unpack(*dims, st.U.cpu().numpy())
    fo = F3.unpack(*dims, U)
    for name in fo:
        err = np.abs(fg[name] - fo[name]).max()
        lim = 1e-13 * np.abs(fo[name]).max() + bound.u[name]
        assert err <= lim, (name, err, lim)
    assert A.grid_status(st.grid) == 0


def test_full_size_z_uniform_state_gives_the_2d_rhs(table):
    """The timed geometry (512 x 256 x 128, the bench's grid and launch configuration) without the
    jet: a state that does not depend on z gives in every z-plane the right-hand side of the
    two-dimensional oracle at 512 x 256, every entry within the two-dimensional parity tolerance,
    and R_w = 0. The property holds at any size (z-derivatives of z-uniform fields vanish, so do
    the z-fluxes with w = 0); the oracle's own three-dimensional right-hand side is out of reach
    at 16.8 M cells. Tolerance: 1e-12 of max|R| plus 32 times the measured floor of the
    two-dimensional oracle at that state."""
    import torch
    from oracle import flow as F
    cfg3 = dict(I.jet_case(512, 256, 128, seed=7), jet=0)
    cfg2 = {k: v for k, v in cfg3.items() if k not in ("nz", "z0", "z1")}
    nx, ny, nz = cfg3["nx"], cfg3["ny"], cfg3["nz"]
    n2 = sum(a * b for _, (a, b) in F.state_layout(5, nx, ny))
    case2 = F.make_case(cfg2, table, I.state_noise(n2, 5))
    tol, o = F.parity_tolerance(case2, case2.U0)
    R2 = F.unpack(5, nx, ny, o)
    f = F.unpack(5, nx, ny, case2.U0)
    f3 = {k: np.broadcast_to(v, (nz,) + v.shape) for k, v in f.items()}
    f3["rhow"] = np.zeros((nz, ny, nx))
    U3 = F3.pack(5, nx, ny, nz, f3)
    del f3
    A, gas, st = _gpu(cfg3)
    U = torch.as_tensor(U3).cuda()
    del U3
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R)
    torch.cuda.synchronize()
    assert A.grid_status(st.grid) == 0
    g = F3.unpack(5, nx, ny, nz, R.cpu().numpy())
    from gpu_util import parity_report, ulp_spread
    spread = ulp_spread(lambda V: F.rhs(case2, V), lambda v: F.unpack(5, nx, ny, np.asarray(v)),
                        case2.U0, o)
    bad, _ = parity_report("3d_z_uniform_512x256x128", {k: g[k] for k in R2},
                           {k: v2[None] for k, v2 in R2.items()}, spread, tol)
    assert not bad, bad
    assert np.abs(g["rhow"]).max() <= 1e-12 * np.abs(R2["rhou"]).max()


def test_eleven_species_jet_rhs_parity(table11):
    """Eleven-species air on the three-dimensional jet (libhyp11.so): the initial state, then the
    right-hand side with 30% of NO and O inside the layer turned into NO+ and O+ and their
    electrons, so that ambipolar ion diffusion and the zero-current electron flux act along all
    three directions."""
    import torch
    ns = 11
    cfg = I.with_species(_zoom(I.jet_case(40, 24, 12, seed=5)))
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    A, gas, st = _gpu(cfg, ns)
    case = F3.make_case(cfg, table11, I.state_noise(_n(cfg, ns), cfg["seed"]))
    torch.cuda.synchronize()
    for k, v in _errors(cfg, st.U.cpu().numpy(), case.U0, ns).items():
        assert v < 1e-13, ("U0", k, v)
    f = F3.unpack(ns, nx, ny, nz, case.U0)
    names = [sp.name for sp in table11.species]
    M = table11.M()
    i_no, i_o, i_nop, i_op = (names.index(x) for x in ("NO", "O", "NO+", "O+"))
    i_e = table11.electron()
    f[f"rs{i_nop}"] = 0.3 * f[f"rs{i_no}"]
    f[f"rs{i_op}"] = 0.15 * f[f"rs{i_o}"]
    f[f"rs{i_no}"] = 0.7 * f[f"rs{i_no}"]
    f[f"rs{i_o}"] = 0.85 * f[f"rs{i_o}"]
    f[f"rs{i_e}"] = M[i_e] * (f[f"rs{i_nop}"] / M[i_nop] + f[f"rs{i_op}"] / M[i_op])
    U = F3.pack(ns, nx, ny, nz, f)
    Ud = torch.as_tensor(U).cuda()
    R = torch.empty_like(Ud)
    A.rhs(gas, st.grid, Ud, R)
    torch.cuda.synchronize()
    bad = _check(case, U, R.cpu().numpy(), label="3d_air11_jet_40x24x12")
    assert not bad, bad
    assert np.abs(F3.unpack(ns, nx, ny, nz, R.cpu().numpy())[f"rs{i_e}"]).max() > 0.0
    assert A.grid_status(st.grid) == 0


def test_three_dimensional_grids_are_rejected_where_unsupported(table):
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = CASES["bl_36x20x8"]
    _, gas, st = _gpu(cfg)
    with pytest.raises(A.HypError, match="two-dimensional"):
        A.Batch().add(st, 1e-4)
    q = torch.empty(cfg["nx"], dtype=torch.float64, device="cuda")
    tw = torch.empty(cfg["nx"] + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(A.HypError, match="two-dimensional"):
        A.wall_fluxes(gas, st.grid, st.U, q, tw)
    with pytest.raises(A.HypError, match="two-register RK3"):
        A.rk_stage_scheme(st, "tvd3", 0, 1e-4)
