"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/fcd.h declares, and rejects bad parameter sets before touching the GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2410_11129_gb300 import fcd
from paper_2410_11129_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fcd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(fcd_[a-z_0-9]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("fcd_create", "fcd_step", "fcd_solve_magnetic", "fcd_observables", "fcd_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = fcd.load()
    for n in declared_functions():
        assert hasattr(L, n), n
    assert set(declared_functions()) <= set(fcd._SIGS)


@pytest.mark.parametrize("bad", [
    dict(nx=7), dict(nx=2), dict(ny=1), dict(r1=9.0, r2=6.0), dict(mobility=0.0),
    dict(xi=-1.0), dict(precision=5), dict(mag_tol=0.0),
    dict(s13_over_s12=3.0),          # gamma_2 < 0: total spreading without eta
    dict(s13_over_s12=2.0, eta=0.01),  # gamma_2 = 0
    dict(s13_over_s12=5.0, eta=0.01),  # gradient energy not positive
    dict(eta=-0.01),
    dict(ferro="core", chi_ferro=0.0),
])
def test_invalid_parameters_rejected(bad):
    L = fcd.load()
    cfg = W.small()
    if "ferro" in bad:
        cfg = W.small(ferro=bad["ferro"], chi_ferro=bad["chi_ferro"])
        cfg["ferro_phase"] = 1
    else:
        cfg.update(bad)
    p = fcd.make_params(cfg)
    h = C.c_void_p()
    st = L.fcd_create(C.byref(p), C.byref(h))
    assert st == fcd.FCD_EINVAL
    assert not h.value
    assert L.fcd_last_error(None).decode().startswith("fcd_create:")


def test_null_arguments():
    L = fcd.load()
    assert L.fcd_create(None, None) == fcd.FCD_EINVAL
    assert L.fcd_step(None, 1) == fcd.FCD_EINVAL
    assert L.fcd_observables(None, None) == fcd.FCD_EINVAL


@pytest.mark.parametrize("bad,K", [
    ({}, 0),                # checkpoint interval
    (dict(Bo_m=0.0), 10),   # H0 ~ sqrt(Bo_m): no derivative at 0
    (dict(nx=7), 10),
])
def test_adjoint_create_rejects(bad, K):
    L = fcd.load()
    cfg = W.small()
    cfg.update(bad)
    p = fcd.make_params(cfg)
    h = C.c_void_p()
    assert L.fcd_create_adjoint(C.byref(p), K, C.byref(h)) == fcd.FCD_EINVAL
    assert not h.value
    assert L.fcd_last_error(None).decode().startswith("fcd_create_adjoint:")
    assert L.fcd_adjoint_gradient(None, 1.0, 0.0, None, None, None) == fcd.FCD_EINVAL
