"""Helpers shared by the GPU parity tests (the CUDA path through the C ABI vs the oracle)."""
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


def check_rhs(case, U, g):
    """Parity of a computed RHS g with the oracle at state U: per field,
    max|g - o| <= 1e-12 max|o| + rounding floor of the flux divergence (oracle.flow)."""
    tol, o = F.parity_tolerance(case, U)
    cfg = case.cfg
    ns = case.tab.ns
    fg = F.unpack(ns, cfg["nx"], cfg["ny"], np.asarray(g))
    fo = F.unpack(ns, cfg["nx"], cfg["ny"], o)
    bad = {k: (float(np.abs(fg[k] - fo[k]).max()), float(tol[k])) for k in fo
           if not np.abs(fg[k] - fo[k]).max() <= tol[k]}
    return bad, o
