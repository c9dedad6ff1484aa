"""The C-ABI library: builds for sm_103a, loads, exports every symbol declared in include/hyp.h,
and its host-side logic (table parsing, freestream scales of Eqs. 7 and 11, state size, argument
checks) agrees with the oracle. No GPU is needed for any of these."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT, TABLE
from oracle import flow as F
from paper_2210_05547_gb300 import inputs as I


@pytest.fixture(scope="module")
def A():
    from paper_2210_05547_gb300 import abi, build
    if not os.path.exists(build.LIB):
        build.build()
    abi.lib()
    return abi


@pytest.mark.parametrize("ns", [5, 11])
def test_exports_every_declared_symbol(A, ns):
    hdr = open(os.path.join(ROOT, "include", "hyp.h")).read()
    declared = set(re.findall(r"\b(hyp_[a-z0-9_]+)\s*\(", hdr))
    assert len(declared) >= 14
    L = A.lib(ns)
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(A.EXPORTS)


@pytest.mark.parametrize("maker,kind", [(I.bl_case, "cneq"), (I.sbli_case, "cneq"),
                                        (I.bl_case, "frozen"), (I.bl_case, "cpg"),
                                        (I.sbli_case, "tpg"), (I.sbli_case, "lte")])
def test_freestream_scales_match_oracle(A, table, maker, kind):
    cfg = maker(kind=kind)
    g = A.gas_model_load(cfg)
    sc = F.freestream_scales(table, kind, cfg)
    ref = dict(rho_inf=sc.rho, a_inf=sc.a, T_inf=sc.T, p_inf=sc.p, mu_inf=sc.mu, k_inf=sc.k,
               cp_inf=sc.cp, gamma_inf=sc.gamma, R_inf=sc.R, T_ref=sc.T_ref, L_ref=sc.L_ref,
               Re=sc.Re, Pr=sc.Pr)
    for k, v in ref.items():
        assert abs(g.scales[k] / v - 1.0) < 1e-14, k


@pytest.mark.parametrize("maker", [I.bl_case, I.sbli_case])
def test_freestream_scales_eleven_species(A, table11, maker):
    cfg = I.with_species(maker())
    g = A.gas_model_load(cfg)
    assert g.ns == 11 and g.L is A.lib(11)
    sc = F.freestream_scales(table11, "cneq", cfg)
    ref = dict(rho_inf=sc.rho, a_inf=sc.a, mu_inf=sc.mu, k_inf=sc.k, cp_inf=sc.cp, Pr=sc.Pr)
    for k, v in ref.items():
        assert abs(g.scales[k] / v - 1.0) < 1e-14, k
    assert A.state_size(g, cfg) == A.state_len(cfg)


def test_species_count_and_charge_rules(A):
    cfg = I.bl_case()
    rc = A.lib(5).hyp_gas_model_load(A.TABLE_AIR11.encode(), 0,
                                     ctypes.byref(A.freestream_struct(cfg)),
                                     ctypes.byref(ctypes.c_void_p()))
    assert rc == -3 and b"must list 5 species" in A.lib(5).hyp_last_error()
    with pytest.raises(A.HypError, match="LTE conserves N and O only"):
        A.gas_model_load(I.with_species(cfg), kind="lte")


def test_eckert_number_is_one(A):
    """Ec = a_inf^2 / (c_p,inf T_ref) = 1 by construction (Sec. 2.1, after Eq. 10)."""
    g = A.gas_model_load(I.bl_case())
    s = g.scales
    assert abs(s["a_inf"] ** 2 / (s["cp_inf"] * s["T_ref"]) - 1.0) < 1e-14


def test_state_size(A):
    cfg = I.bl_case(37, 13)
    g = A.gas_model_load(cfg)
    n = sum(a * b for _, (a, b) in F.state_layout(5, 37, 13))
    assert A.state_size(g, cfg) == n


def test_argument_errors(A):
    cfg = I.bl_case()
    rc = A.lib().hyp_gas_model_load(TABLE.encode(), 7, ctypes.byref(A.freestream_struct(cfg)),
                                    ctypes.byref(ctypes.c_void_p()))
    assert rc == -1 and b"kind" in A.lib().hyp_last_error()
    with pytest.raises(A.HypError, match="cannot open"):
        A.gas_model_load(cfg, path="/nonexistent/table.dat")
    g = A.gas_model_load(cfg)
    bad = I.bl_case(4, 64)
    with pytest.raises(A.HypError, match="at least 8"):
        A.state_size(g, bad)
    bad_fs = dict(cfg, Y_inf=(0.5, 0.2, 0.0, 0.0, 0.0))
    with pytest.raises(A.HypError, match="mass fractions"):
        A.gas_model_load(bad_fs)
    with pytest.raises(A.HypError, match="LTE needs both elements"):
        A.gas_model_load(dict(cfg, Y_inf=(1.0, 0.0, 0.0, 0.0, 0.0)), kind="lte")
