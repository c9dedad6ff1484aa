"""Helpers shared by the GPU parity tests (the CUDA path through the C ABI vs the oracle)."""
import json
import os

import numpy as np

from oracle import flow as F
from oracle import gas as G
from paper_2210_05547_gb300 import inputs as I

TINY = 1e-300


def normwise(g, o):
    """max |g - o| / max |o| (normwise relative error of one field)."""
    return float(np.abs(np.asarray(g) - np.asarray(o)).max() / max(np.abs(o).max(), TINY))


def field_errors(cfg, a, b, ns=5):
    fa = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(a))
    fb = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(b))
    return {k: normwise(fa[k], fb[k]) for k in fa}


def nstate(cfg, ns=5):
    return sum(a * b for _, (a, b) in F.state_layout(ns, cfg["nx"], cfg["ny"]))


def oracle_case(table, cfg):
    return F.make_case(cfg, table, I.state_noise(nstate(cfg, table.ns), cfg["seed"]))


def gpu_state(cfg):
    import torch
    from paper_2210_05547_gb300 import abi as A
    gas = A.gas_model_load(cfg)
    n = A.state_size(gas, cfg)
    U = torch.empty(n, dtype=torch.float64, device="cuda")
    dQ = torch.empty_like(U)
    st = A.state_init(gas, cfg, U, dQ, I.state_noise(n, cfg["seed"]))
    return gas, st


def gpu_rhs(gas, st, U_host):
    import torch
    from paper_2210_05547_gb300 import abi as A
    U = torch.as_tensor(np.asarray(U_host), dtype=torch.float64).cuda()
    R = torch.empty_like(U)
    A.rhs(gas, st.grid, U, R)
    torch.cuda.synchronize()
    return R.cpu().numpy()


# Measured FP64 floor of a right-hand side: the oracle evaluated again at states whose every entry
# is moved by one unit in the last place, up or down with seeded signs. The largest change per
# field over FLOOR_REPS such states is how far two correct FP64 evaluations sit apart from the
# rounding of their inputs alone; the parity criterion allows FLOOR_C times that on top of
# 1e-12 max|o|. The two codes also round differently inside (order of the compact solves, the
# Newton iteration's last step, fused updates) and each builds its own reference state, so they
# differ by more than one input rounding: over the 95 checks of the GPU suite the error reached
# 35 times the measured floor where the floor dominates the bound (an 8 x 8 grid's energy); the
# constant is fixed at 32 with every check inside 1e-12 max|o| + 32 x floor.
FLOOR_REPS = 2
FLOOR_C = 32.0
RTOL = 1.0e-12


def ulp_spread(rhs_fn, unpack_fn, U, o, reps=FLOOR_REPS, seed=0x51ab):
    """Per-field max |rhs(U') - o| over `reps` states U' one ulp away from U in every entry."""
    rng = np.random.default_rng(seed)
    U = np.asarray(U, dtype=np.float64)
    fo = unpack_fn(o)
    spread = {k: 0.0 for k in fo}
    for _ in range(reps):
        up = rng.integers(0, 2, U.size).astype(bool)
        Up = np.where(up, np.nextafter(U, np.inf), np.nextafter(U, -np.inf))
        fp = unpack_fn(rhs_fn(Up))
        for k in fo:
            spread[k] = max(spread[k], float(np.abs(fp[k] - fo[k]).max()))
    return spread


def log_parity(record):
    """Append one JSON line to the file named by HYP_PARITY_LOG (if set): the achieved normwise
    errors of a parity check beside its bounds."""
    path = os.environ.get("HYP_PARITY_LOG")
    if not path:
        return
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "a") as fh:
        fh.write(json.dumps(record) + "\n")


def parity_report(label, fg, fo, spread, tol_analytic=None):
    """Per field: achieved error, the measured floor criterion and (if given) the analytic
    tolerance of oracle.flow. Returns (bad, record)."""
    rec, bad = {"case": label, "rtol": RTOL, "floor_c": FLOOR_C, "fields": {}}, {}
    for k in fo:
        scale = max(float(np.abs(fo[k]).max()), TINY)
        err = float(np.abs(np.asarray(fg[k]) - fo[k]).max())
        bound = RTOL * scale + FLOOR_C * spread[k]
        row = {"err": err / scale, "floor": spread[k] / scale, "bound": bound / scale}
        if tol_analytic is not None:
            row["analytic_tol"] = float(tol_analytic[k]) / scale
        rec["fields"][k] = row
        if not err <= bound:
            bad[k] = (err, bound)
    log_parity(rec)
    return bad, rec


def check_rhs(case, U, g, label=None):
    """Parity of a computed RHS g with the oracle at state U: per field,
    max|g - o| <= 1e-12 max|o| + FLOOR_C x the measured one-ulp floor (ulp_spread). The analytic
    rounding-floor tolerance of oracle.flow is recorded beside it."""
    tol, o = F.parity_tolerance(case, U)
    cfg = case.cfg
    ns = case.tab.ns

    def unpack(v):
        return F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(v))

    spread = ulp_spread(lambda V: F.rhs(case, V), unpack, U, o)
    bad, _ = parity_report(label or cfg.get("name", "case"), unpack(g), unpack(o), spread, tol)
    return bad, o


class StateBound:
    """Per-field bound on |U_gpu - U_oracle| carried through the stages of a run in which every
    stage's right-hand side was checked (GPU at its state against the oracle at its own, within
    tol). Two-register schemes (RK3, RK4): dQ <- A_k dQ + dt R, U <- U + B_k dQ, so the dQ
    difference is at most |A_k| times the previous one plus dt tol and the state's grows by |B_k|
    times that. TVD RK3: U <- a_k U0 + b_k (U + dt R). The state filter of a step (x, then y
    pass, f - sigma D f with ||D||_inf = 1) multiplies the state's bound by (1 + sigma)^2."""

    def __init__(self, names, scheme="rk3"):
        self.scheme = scheme
        self.u = {k: 0.0 for k in names}
        self.w = {k: 0.0 for k in names}

    def stage(self, k, dt, tol):
        for n in self.u:
            if self.scheme == "tvd3":
                if k == 0:
                    self.w[n] = self.u[n]
                self.u[n] = F.TVD3_W[k] * self.w[n] + F.TVD3_S[k] * (self.u[n] + dt * tol[n])
            else:
                A, B = (F.RK_A, F.RK_B) if self.scheme == "rk3" else (F.CK4_A, F.CK4_B)
                self.w[n] = abs(A[k]) * self.w[n] + dt * tol[n]
                self.u[n] += abs(B[k]) * self.w[n]

    def filter(self, sigma):
        for n in self.u:
            self.u[n] *= (1.0 + sigma) ** 2


def field_diff(cfg, a, b, ns=5):
    """Per-field max |a - b| of two state-layout vectors."""
    fa = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(a))
    fb = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(b))
    return {k: float(np.abs(fa[k] - fb[k]).max()) for k in fa}


def follow_stages(table, cfg, st, gas, steps, label, scheme="rk3", stage_fn=None, U0=None):
    """Run `steps` steps of `scheme` on the GPU (stage_fn(k) advances the GPU state one stage) and
    in the oracle from the same state (U0, else the GPU's). Every stage: the GPU right-hand side at
    the GPU state is checked against the oracle at that same state (check_rhs), and its difference
    from the oracle's right-hand side at the oracle's state feeds the carried bound. Returns
    (failures, final GPU state, final oracle state, StateBound)."""
    import torch
    case = oracle_case(table, cfg)
    ns = table.ns
    if U0 is not None:
        st.U.copy_(torch.as_tensor(U0).cuda())
    U = st.U.cpu().numpy()
    W = np.zeros_like(U)
    bound = StateBound([n for n, _ in F.state_layout(ns, cfg["nx"], cfg["ny"])], scheme)
    failures = []
    for step in range(steps):
        for k in range(F.RK_STAGES[scheme]):
            Ug = st.U.cpu().numpy()
            Rg = gpu_rhs(gas, st, Ug)
            bad, _ = check_rhs(case, Ug, Rg, label=f"{label}/step{step}/stage{k}")
            if bad:
                failures.append((step, k, bad))
            U, W, Ro = F.rk_stage_scheme(case, U, W, k, cfg["dt"], scheme)
            bound.stage(k, cfg["dt"], field_diff(cfg, Rg, Ro, ns))
            stage_fn(k)
        if cfg.get("filter_sigma", 0.0) > 0.0:
            bound.filter(cfg["filter_sigma"])
    torch.cuda.synchronize()
    return failures, st.U.cpu().numpy(), U, bound


def assert_states(cfg, Ug, Uo, bound, ns=5):
    """GPU state within 1e-13 of each oracle field plus the carried bound."""
    fg = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(Ug))
    fo = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(Uo))
    for name in fo:
        err = np.abs(fg[name] - fo[name]).max()
        lim = 1e-13 * np.abs(fo[name]).max() + bound.u[name]
        assert err <= lim, (name, err, lim)
