"""The C-ABI library loads and exports every symbol include/pintmg.h declares (no GPU calls)."""
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "pintmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_\w+|fgmres_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mg_setup", "mg_vcycle", "fgmres_solve", "mg_destroy", "mg_status_string"):
        assert n in names


def test_library_exports_declared_symbols():
    from paper_2405_04808_gb300 import build as B
    from paper_2405_04808_gb300 import pintmg as P
    if not os.path.exists(B.LIB_PATH):
        B.build()
    L = P.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(P.EXPORTED) == set(_declared())
    assert P.mg_status_string(P.MG_ERR_SINGULAR).startswith("singular")
    o = P.mg_default_options()
    assert (o.levels, o.nu_pre, o.nu_post, o.coarse_maxit) == (2, 1, 1, 50)
    assert abs(o.coarse_rtol - 1e-3) < 1e-18
    assert o.krylov_basis == P.KRYLOV_BASIS["fp64"] and o.device_loops == 1
    assert P.mg_status_string(P.MG_ERR_TIMEOUT).startswith("a bounded device-side wait")


def test_argument_errors_need_no_gpu():
    """Invalid sizes are rejected on the host before any CUDA call."""
    from paper_2405_04808_gb300 import pintmg as P
    from paper_2405_04808_gb300 import workloads as W
    prob = W.vdp(n=12, seed=1)
    with pytest.raises(P.PintmgError) as e:
        P.mg_setup(prob, levels=4)           # 12 is not divisible by 2^3
    assert e.value.code == P.MG_ERR_ARG
    prob.Ju_cur[3, 0, 0] = float("nan")
    with pytest.raises(P.PintmgError) as e:
        P.mg_setup(prob, levels=2)
    assert e.value.code == P.MG_ERR_NONFINITE
