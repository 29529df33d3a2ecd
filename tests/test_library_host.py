"""Host-side checks of the solver library that need no GPU: it builds and loads,
exports every entry point include/lbs.h declares, its quadrature (an algorithm
independent of the oracle's) agrees with the oracle's, and bad arguments are
rejected before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import quadrature as oq
from paper_1702_01335_gb300 import lbs as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbs_\w+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = L.load()
    names = declared_symbols()
    assert "lbs_create" in names and "lbs_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(L.EXPORTS) >= set(names) - {"lbs_last_error"} | set()


@pytest.mark.parametrize("Q", [1, 2, 4, 7, 16])
def test_full_range_rule_matches_oracle(Q):
    x, w = L.quadrature(0, Q)
    xo, wo = oq.full_range_rule(Q)
    assert np.allclose(x, xo, rtol=0, atol=1e-13)
    assert np.allclose(w, wo, rtol=1e-12, atol=0)


@pytest.mark.parametrize("Q", [1, 4, 7, 16, 32, 48, 64])
def test_half_range_rule_matches_oracle(Q):
    x, w = L.quadrature(1, Q)
    xo, wo = oq.half_range_rule(Q)
    assert np.allclose(x, xo, rtol=1e-12, atol=0)
    assert np.allclose(w, wo, rtol=1e-11, atol=0)


def test_bad_arguments_are_rejected():
    lib = L.load()
    h = C.c_void_p()
    bad = [
        L.Instance(Qx=0), L.Instance(Qz=65), L.Instance(N_eq=9), L.Instance(Nz=5),
        L.Instance(Kn=0.0), L.Instance(T_w=-1.0), L.Instance(Pr=0.0), L.Instance(A=1.0),
        L.Instance(cfl=0.0, dt=0.0), L.Instance(visc_law=1, visc_param=0.0),
        L.Instance(Qx=64, Qy=64, Qz=64),
    ]
    for inst in bad:
        d = (L._Desc * 1)(inst.desc())
        st = lib.lbs_batch_create(C.byref(h), d, 1, 0, None)
        assert st == 1, inst
        assert lib.lbs_last_error().decode()
    assert lib.lbs_quadrature(2, 4, None, None) == 1
    assert lib.lbs_step(None, 1) == 1
