"""Thin Python binding of the C ABI in ``include/hyp.h`` (argument marshalling only).

Every arithmetic step of ``rhs``, ``rk_stage``, ``thermo_eval`` and ``thermo_energy`` runs in the
CUDA library (``_lib/libhyp.so`` for five-species tables, ``_lib/libhyp11.so`` for eleven-species
tables; a gas handle and everything made from it stay with the library that loaded its table);
this module only checks tensors, converts case dictionaries into the C structs and forwards raw
pointers. If a library has not been built, every call that needs it raises. PyTorch supplies
device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_SPECIES = 11
GAS_KINDS = {"cneq": 0, "frozen": 1, "cpg": 2, "tpg": 3, "lte": 4}
STRETCH = {"uniform": 0, "tanh": 1, "cubic": 2}
FLOWS = {"bl": 0, "sbli": 1}
DIFFUSION_MODELS = {"ramshaw": 0, "stefan_maxwell": 1}
FP64 = 0
MIXED = 1
DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
TABLE_AIR5 = os.path.join(DATA, "air5.dat")
TABLE_AIR11 = os.path.join(DATA, "air11.dat")
SCALE_NAMES = ("rho_inf", "a_inf", "T_inf", "p_inf", "mu_inf", "k_inf", "cp_inf", "gamma_inf",
               "R_inf", "T_ref", "L_ref", "Re", "Pr")


class Freestream(ctypes.Structure):
    _fields_ = [("T_inf", ctypes.c_double), ("p_inf", ctypes.c_double),
                ("Y_inf", ctypes.c_double * MAX_SPECIES), ("mach", ctypes.c_double),
                ("reynolds", ctypes.c_double), ("prandtl_cpg", ctypes.c_double)]


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("y_stretch", ctypes.c_int32), ("y_param", ctypes.c_double),
                ("nz", ctypes.c_int32), ("z0", ctypes.c_double), ("z1", ctypes.c_double)]


class CaseDesc(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int32), ("wall", ctypes.c_int32), ("T_wall", ctypes.c_double),
                ("delta_coef", ctypes.c_double), ("minor_species", ctypes.c_double),
                ("shock_deflection_deg", ctypes.c_double), ("shock_x", ctypes.c_double),
                ("shock_width", ctypes.c_double), ("sponge_sigma", ctypes.c_double),
                ("sponge_in", ctypes.c_double), ("sponge_out", ctypes.c_double),
                ("sponge_top_cells", ctypes.c_int32), ("artificial_diffusivity", ctypes.c_int32),
                ("C_mu", ctypes.c_double), ("C_beta", ctypes.c_double),
                ("C_kappa", ctypes.c_double), ("C_D", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("noise", ctypes.POINTER(ctypes.c_double)),
                ("filter_sigma", ctypes.c_double), ("diffusion_model", ctypes.c_int32),
                ("jet", ctypes.c_int32), ("jet_x", ctypes.c_double), ("jet_z", ctypes.c_double),
                ("jet_radius", ctypes.c_double), ("jet_edge", ctypes.c_double),
                ("jet_J", ctypes.c_double), ("jet_T_ratio", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("fs", Freestream), ("grid", GridDesc), ("cas", CaseDesc), ("dt", ctypes.c_double),
                ("nsteps", ctypes.c_int32), ("keep_result", ctypes.c_int32)]


class RequestStats(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_finish", ctypes.c_double), ("done", ctypes.c_int32),
                ("status", ctypes.c_uint32), ("error", ctypes.c_int32),
                ("points", ctypes.c_int64), ("bytes", ctypes.c_int64)]


_LIBS = {}
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64

EXPORTS = {
    "hyp_gas_model_load": (_I, [ctypes.c_char_p, _I, ctypes.POINTER(Freestream), ctypes.POINTER(_P)]),
    "hyp_gas_scales": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "hyp_gas_free": (None, [_P]),
    "hyp_state_size": (_I, [_P, ctypes.POINTER(GridDesc), ctypes.POINTER(_I64)]),
    "hyp_state_init": (_I, [_P, ctypes.POINTER(GridDesc), ctypes.POINTER(CaseDesc), _P, _P, _P,
                            ctypes.POINTER(_P)]),
    "hyp_state_grid": (_P, [_P]),
    "hyp_grid_reference": (_I, [_P, _P, _P]),
    "hyp_grid_status": (_I, [_P, ctypes.POINTER(ctypes.c_uint32), _I]),
    "hyp_grid_temperature": (_I, [_P, ctypes.c_int64, _P, _P]),
    "hyp_state_free": (None, [_P]),
    "hyp_rhs": (_I, [_P, _P, _P, _P, _I, _P]),
    "hyp_rk_stage": (_I, [_P, _I, _D, _I, _P]),
    "hyp_rk_stage_scheme": (_I, [_P, _I, _I, _D, _I, _P]),
    "hyp_thermo_eval": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P]),
    "hyp_thermo_energy": (_I, [_P, _I64, _P, _P, _P, _P]),
    "hyp_lte_eval": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P]),
    "hyp_rhs_noalloc": (_I, [_P, _P, _P, _P, _P]),
    "hyp_wall_fluxes": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "hyp_round_f32": (_I, [_I64, _P, _P, _P, _P]),
    "hyp_fp64_fast": (_I, [_I, _I64, _P, _P, _P, _P]),
    "hyp_batch_create": (_I, [_I, ctypes.POINTER(_P)]),
    "hyp_batch_add": (_I, [_P, _P, _D]),
    "hyp_batch_remove": (_I, [_P, _P]),
    "hyp_batch_configure": (_I, [_P, _I, _I]),
    "hyp_batch_size": (_I, [_P, ctypes.POINTER(_I)]),
    "hyp_batch_tile": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hyp_batch_step": (_I, [_P, _I, _P]),
    "hyp_batch_free": (None, [_P]),
    "hyp_server_create": (_I, [ctypes.c_char_p, _I, _I, _I64, _I, ctypes.POINTER(_P)]),
    "hyp_server_submit": (_I, [_P, ctypes.POINTER(Request), ctypes.POINTER(_I64)]),
    "hyp_server_wait": (_I, [_P, _I64, _D]),
    "hyp_server_stats": (_I, [_P, _I64, ctypes.POINTER(RequestStats)]),
    "hyp_server_result": (_I, [_P, _I64, _P]),
    "hyp_server_counters": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_D),
                                 ctypes.POINTER(ctypes.c_int32)]),
    "hyp_server_free": (None, [_P]),
    "hyp_grid_profile": (_I, [_P, _I]),
    "hyp_grid_profile_read": (_I, [_P, _I, _P, _P]),
    "hyp_profile_count": (_I, []),
    "hyp_profile_name": (ctypes.c_char_p, [_I]),
    "hyp_last_error": (ctypes.c_char_p, []),
}


class HypError(RuntimeError):
    pass


def library_path(ns=5):
    return _build.VARIANTS[ns]


def lib(ns=5):
    """Load the CUDA library built for ns species (raises if it has not been built)."""
    if ns not in _LIBS:
        path = library_path(ns)
        if not os.path.exists(path):
            raise HypError(f"CUDA library not built ({path}); run python -m paper_2210_05547_gb300.build")
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIBS[ns] = L
    return _LIBS[ns]


def table_path(cfg):
    """The gas table file of a case dictionary (key "table", default five-species air)."""
    return os.path.join(DATA, cfg.get("table", "air5") + ".dat")


def table_species(path):
    """Number of SPECIES lines of a gas table: which library loads it."""
    with open(path) as fh:
        return sum(1 for line in fh if line.split("#", 1)[0].split()[:1] == ["SPECIES"])


def _check(rc, L=None):
    if rc != 0:
        L = L or lib()
        raise HypError(f"hyp error {rc}: {L.hyp_last_error().decode()}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, n=None, dtype=None):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise HypError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise HypError(f"expected dtype {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise HypError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------------------------
# structs from the case dictionaries of paper_2210_05547_gb300.inputs
# ---------------------------------------------------------------------------------------------

def freestream_struct(cfg):
    fs = Freestream()
    fs.T_inf, fs.p_inf = cfg["T_inf"], cfg["p_inf"]
    for i, y in enumerate(cfg["Y_inf"]):
        fs.Y_inf[i] = y
    fs.mach, fs.reynolds, fs.prandtl_cpg = cfg["mach"], cfg["reynolds"], cfg["prandtl_cpg"]
    return fs


def grid_struct(cfg):
    return GridDesc(cfg["nx"], cfg["ny"], cfg["x0"], cfg["x1"], cfg["y0"], cfg["y1"],
                    STRETCH[cfg["y_stretch"]], cfg["y_param"], int(cfg.get("nz", 1)),
                    float(cfg.get("z0", 0.0)), float(cfg.get("z1", 1.0)))


def case_struct(cfg, noise=None):
    c = CaseDesc()
    c.flow, c.wall, c.T_wall = FLOWS[cfg["flow"]], int(cfg["wall"]), cfg["T_wall"]
    c.delta_coef, c.minor_species = cfg["delta_coef"], cfg["minor_species"]
    c.shock_deflection_deg, c.shock_x = cfg["shock_deflection_deg"], cfg["shock_x"]
    c.shock_width = cfg["shock_width"] if cfg["shock_width"] > 0 else 1.0
    c.sponge_sigma, c.sponge_in, c.sponge_out = cfg["sponge_sigma"], cfg["sponge_in"], cfg["sponge_out"]
    c.sponge_top_cells = int(cfg["sponge_top_cells"])
    c.artificial_diffusivity = int(cfg["artificial_diffusivity"])
    c.C_mu, c.C_beta, c.C_kappa, c.C_D = cfg["C_mu"], cfg["C_beta"], cfg["C_kappa"], cfg["C_D"]
    c.noise_amp = cfg["noise_amp"]
    c.filter_sigma = cfg.get("filter_sigma", 0.0)
    c.diffusion_model = DIFFUSION_MODELS[cfg.get("diffusion_model", "ramshaw")]
    c.jet = int(cfg.get("jet", 0))
    if c.jet:
        c.jet_x, c.jet_z, c.jet_radius = cfg["jet_x"], cfg["jet_z"], cfg["jet_radius"]
        c.jet_edge, c.jet_J, c.jet_T_ratio = cfg["jet_edge"], cfg["jet_J"], cfg["jet_T_ratio"]
    if noise is not None:
        arr = np.ascontiguousarray(noise, dtype=np.float64)
        c.noise = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c._keep = arr
    return c


# ---------------------------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------------------------

class Gas:
    def __init__(self, handle, L, path):
        self.handle = handle
        self.L = L
        self.path = path
        ns = ctypes.c_int()
        buf = (ctypes.c_double * 13)()
        _check(L.hyp_gas_scales(handle, ctypes.byref(ns), buf), L)
        self.ns = ns.value
        self.scales = dict(zip(SCALE_NAMES, list(buf)))

    def __del__(self):
        if getattr(self, "handle", None):
            self.L.hyp_gas_free(self.handle)
            self.handle = None


class Grid:
    """A grid handle (owned by its state) and the library it belongs to; passes as the raw
    pointer in calls."""

    def __init__(self, ptr, L):
        self._as_parameter_ = ptr
        self.L = L


class State:
    def __init__(self, handle, U, dQ, gas):
        self.handle = handle
        self.U = U
        self.dQ = dQ
        self.gas = gas
        self.L = gas.L
        self.grid = Grid(gas.L.hyp_state_grid(handle), gas.L)

    def __del__(self):
        if getattr(self, "handle", None):
            self.L.hyp_state_free(self.handle)
            self.handle = None


def _grid_lib(grid):
    return grid.L if isinstance(grid, Grid) else lib()


def gas_model_load(cfg, kind=None, path=None):
    """hyp_gas_model_load: gas table + kind + freestream (from a case dictionary). The table is
    the case's (key "table") unless a path is given; its species count picks the library."""
    path = path or table_path(cfg)
    L = lib(table_species(path)) if os.path.exists(path) else lib()
    h = ctypes.c_void_p()
    fs = freestream_struct(cfg)
    k = GAS_KINDS[kind or cfg["kind"]]
    _check(L.hyp_gas_model_load(path.encode(), k, ctypes.byref(fs), ctypes.byref(h)), L)
    return Gas(h, L, path)


def state_size(gas, cfg):
    n = ctypes.c_int64()
    _check(gas.L.hyp_state_size(gas.handle, ctypes.byref(grid_struct(cfg)), ctypes.byref(n)), gas.L)
    return n.value


def state_init(gas, cfg, U, dQ, noise=None, stream=None):
    """hyp_state_init: builds the grid handle and writes the initial state into U (device)."""
    import torch
    n = state_size(gas, cfg)
    h = ctypes.c_void_p()
    desc = grid_struct(cfg)
    cas = case_struct(cfg, noise)
    _check(gas.L.hyp_state_init(gas.handle, ctypes.byref(desc), ctypes.byref(cas),
                                _dptr(U, n, torch.float64), _dptr(dQ, n, torch.float64),
                                _stream(stream), ctypes.byref(h)), gas.L)
    return State(h, U, dQ, gas)


def rhs(gas, grid, U, dUdt, precision=FP64, stream=None):
    """hyp_rhs: dU/dt of the state U (device tensors, same length)."""
    _check(gas.L.hyp_rhs(gas.handle, grid, _dptr(U), _dptr(dUdt, U.numel()), precision,
                         _stream(stream)), gas.L)


def rhs_noalloc(gas, grid, U, dUdt, stream=None):
    """hyp_rhs_noalloc: the right-hand side with its scratch in the library's static device array."""
    _check(gas.L.hyp_rhs_noalloc(gas.handle, grid, _dptr(U), _dptr(dUdt, U.numel()),
                                 _stream(stream)), gas.L)


def rk_stage(state, stage, dt, precision=FP64, stream=None):
    """hyp_rk_stage: one stage of the two-register RK3 on the state's registers."""
    _check(state.L.hyp_rk_stage(state.handle, stage, dt, precision, _stream(stream)), state.L)


RK_SCHEMES = {"rk3": 0, "tvd3": 1, "ck4": 2}
RK_STAGES = {"rk3": 3, "tvd3": 3, "ck4": 5}


def rk_stage_scheme(state, scheme, stage, dt, precision=FP64, stream=None):
    """hyp_rk_stage_scheme: one stage of "rk3", "tvd3" or "ck4" on the state's registers."""
    _check(state.L.hyp_rk_stage_scheme(state.handle, RK_SCHEMES[scheme], stage, dt, precision,
                                       _stream(stream)), state.L)


def wall_fluxes(gas, grid, U, q_w, tau_w, precision=FP64, stream=None):
    """hyp_wall_fluxes: wall heat flux q_w (nx) and wall shear tau_w (nx + 1) of state U."""
    import torch
    if tau_w.numel() != q_w.numel() + 1:
        raise HypError("tau_w needs one entry more than q_w (nx + 1 wall corners, nx wall faces)")
    _check(gas.L.hyp_wall_fluxes(gas.handle, grid, _dptr(U), _dptr(q_w, None, torch.float64),
                                 _dptr(tau_w, None, torch.float64), precision, _stream(stream)),
           gas.L)


def round_f32(x, y=None, back=None, stream=None):
    """hyp_round_f32: binary64 -> binary32 rounding (y) and the widening back (back), device."""
    import torch
    n = x.numel()
    _check(lib().hyp_round_f32(n, _dptr(x, n, torch.float64),
                               _dptr(y, n, torch.float32) if y is not None else None,
                               _dptr(back, n, torch.float64) if back is not None else None,
                               _stream(stream)))


def fp64_fast(fn, out, a=None, b=None, stream=None):
    """hyp_fp64_fast: fn 0 exp(a), 1 a / b, 2 1 / b, 3 log(a) as the FP64 closure computes them,
    device."""
    import torch
    n = out.numel()
    _check(lib().hyp_fp64_fast(fn, n, _dptr(a, n, torch.float64) if a is not None else None,
                               _dptr(b, n, torch.float64) if b is not None else None,
                               _dptr(out, n, torch.float64), _stream(stream)))


class Batch:
    """hyp_batch: many states stepped in shared launches (members keep their own dt). species:
    the species count of the members' gas tables (which library runs the batch)."""

    def __init__(self, precision=FP64, use_graph=False, tile=0, species=5):
        self.L = lib(species)
        h = ctypes.c_void_p()
        _check(self.L.hyp_batch_create(precision, ctypes.byref(h)), self.L)
        self.handle = h
        self.members = []
        if use_graph or tile:
            self.configure(use_graph, tile)

    def configure(self, use_graph=False, tile=0):
        _check(self.L.hyp_batch_configure(self.handle, int(bool(use_graph)), int(tile)), self.L)

    def add(self, state, dt):
        if state.L is not self.L:
            raise HypError("the state's gas table has another species count than the batch")
        _check(self.L.hyp_batch_add(self.handle, state.handle, float(dt)), self.L)
        self.members.append(state)

    def remove(self, state):
        _check(self.L.hyp_batch_remove(self.handle, state.handle), self.L)
        self.members.remove(state)

    def size(self):
        n = ctypes.c_int()
        _check(self.L.hyp_batch_size(self.handle, ctypes.byref(n)), self.L)
        return n.value

    def tile(self):
        t, tuned = ctypes.c_int(), ctypes.c_int()
        _check(self.L.hyp_batch_tile(self.handle, ctypes.byref(t), ctypes.byref(tuned)), self.L)
        return t.value, bool(tuned.value)

    def step(self, nsteps=1, stream=None):
        _check(self.L.hyp_batch_step(self.handle, int(nsteps), _stream(stream)), self.L)

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            self.L.hyp_batch_free(self.handle)
            self.handle = None


def state_len(cfg, ns=None):
    """Length of the state vector of a case (layout of include/hyp.h)."""
    from .inputs import TABLE_SPECIES
    ns = ns or TABLE_SPECIES[cfg.get("table", "air5")]
    nx, ny, nz = cfg["nx"], cfg["ny"], int(cfg.get("nz", 1))
    n = (ns + 1) * nx * ny + (nx + 1) * ny + nx * (ny + 1)
    return n * nz + nx * ny * nz if nz > 1 else n


class Server:
    """hyp_server: continuous batching of independent solves on the current GPU, all on the gas
    table at `path` (its species count picks the library)."""

    def __init__(self, precision=FP64, reserve_bytes=4 << 30, max_members=64, kind="cneq",
                 path=TABLE_AIR5):
        self.L = lib(table_species(path))
        self.path = os.path.abspath(path)
        h = ctypes.c_void_p()
        _check(self.L.hyp_server_create(path.encode(), GAS_KINDS[kind], precision,
                                         int(reserve_bytes), int(max_members), ctypes.byref(h)),
               self.L)
        self.handle = h

    def submit(self, cfg, nsteps, dt=None, noise=None, keep_result=False):
        if os.path.abspath(table_path(cfg)) != self.path:
            raise ValueError(f"request on {table_path(cfg)}, server on {self.path}")
        r = Request()
        r.fs = freestream_struct(cfg)
        r.grid = grid_struct(cfg)
        r.cas = case_struct(cfg, noise)
        r.dt = cfg["dt"] if dt is None else dt
        r.nsteps = int(nsteps)
        r.keep_result = int(bool(keep_result))
        i = ctypes.c_int64()
        _check(self.L.hyp_server_submit(self.handle, ctypes.byref(r), ctypes.byref(i)), self.L)
        return i.value

    def wait(self, rid=-1, timeout=3600.0):
        _check(self.L.hyp_server_wait(self.handle, int(rid), float(timeout)), self.L)

    def stats(self, rid):
        st = RequestStats()
        _check(self.L.hyp_server_stats(self.handle, int(rid), ctypes.byref(st)), self.L)
        return {k: getattr(st, k) for k, _ in RequestStats._fields_}

    def result(self, rid, cfg):
        out = np.empty(state_len(cfg))
        _check(self.L.hyp_server_result(self.handle, int(rid), out.ctypes.data_as(ctypes.c_void_p)),
               self.L)
        return out

    def counters(self):
        a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32()
        _check(self.L.hyp_server_counters(self.handle, ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(c), ctypes.byref(d)), self.L)
        return {"batch_steps": a.value, "member_steps": b.value, "busy_s": c.value,
                "max_members": d.value}

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.L.hyp_server_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def grid_reference(grid, n):
    L = _grid_lib(grid)
    Uref = np.empty(n)
    sigma = np.empty(n)
    _check(L.hyp_grid_reference(grid, Uref.ctypes.data_as(ctypes.c_void_p),
                                sigma.ctypes.data_as(ctypes.c_void_p)), L)
    return Uref, sigma


def grid_status(grid, clear=False):
    L = _grid_lib(grid)
    flags = ctypes.c_uint32()
    _check(L.hyp_grid_status(grid, ctypes.byref(flags), int(clear)), L)
    return flags.value


def grid_temperature(grid, T, stream=None):
    """hyp_grid_temperature: the cell-centre temperatures (K) of the grid's last closure into the
    device tensor T (nx*ny or nx*ny*nz doubles)."""
    import torch
    L = _grid_lib(grid)
    _check(L.hyp_grid_temperature(grid, T.numel(), _dptr(T, None, torch.float64),
                                  _stream(stream)), L)


def thermo_eval(gas, rho, e, Y, T=None, p=None, wdot=None, mu=None, k=None, D=None,
                status=None, precision=FP64, stream=None):
    """hyp_thermo_eval on device tensors (SI). Y and the per-species outputs are (ns, n)."""
    import torch
    n = rho.numel()
    ns = gas.ns
    _check(gas.L.hyp_thermo_eval(
        gas.handle, n, _dptr(rho, n, torch.float64), _dptr(e, n, torch.float64),
        _dptr(Y, ns * n, torch.float64), _dptr(T, n), _dptr(p, n), _dptr(wdot, ns * n),
        _dptr(mu, n), _dptr(k, n), _dptr(D, ns * n),
        _dptr(status, n, torch.uint8) if status is not None else None, precision,
        _stream(stream)), gas.L)


def lte_eval(gas, rho, e, T=None, p=None, Y=None, mu=None, k=None, k_reactive=None, status=None,
             precision=FP64, stream=None):
    """hyp_lte_eval on device tensors (SI) for an "lte" gas. Y (output) is (ns, n)."""
    import torch
    n = rho.numel()
    _check(gas.L.hyp_lte_eval(
        gas.handle, n, _dptr(rho, n, torch.float64), _dptr(e, n, torch.float64), _dptr(T, n),
        _dptr(p, n), _dptr(Y, gas.ns * n), _dptr(mu, n), _dptr(k, n), _dptr(k_reactive, n),
        _dptr(status, n, torch.uint8) if status is not None else None, precision,
        _stream(stream)), gas.L)


def thermo_energy(gas, T, Y, e, stream=None):
    import torch
    n = T.numel()
    _check(gas.L.hyp_thermo_energy(gas.handle, n, _dptr(T, n, torch.float64),
                                   _dptr(Y, gas.ns * n, torch.float64), _dptr(e, n, torch.float64),
                                   _stream(stream)), gas.L)


def grid_profile(grid, enable):
    """hyp_grid_profile: start (clears totals) or stop the per-launch event profile of a grid."""
    L = _grid_lib(grid)
    _check(L.hyp_grid_profile(grid, int(bool(enable))), L)


def grid_profile_read(grid):
    """hyp_grid_profile_read: {kernel name: (total ms, launches)} since the profile was started."""
    L = _grid_lib(grid)
    n = L.hyp_profile_count()
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(L.hyp_grid_profile_read(grid, n, ms.ctypes.data_as(ctypes.c_void_p),
                                   cnt.ctypes.data_as(ctypes.c_void_p)), L)
    out = {}
    for k in range(n):
        name = L.hyp_profile_name(k).decode()
        t, c = out.get(name, (0.0, 0))
        out[name] = (t + float(ms[k]), c + int(cnt[k]))
    return out
