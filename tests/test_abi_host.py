"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every symbol declared in include/pssd.h, and its host-only routines (the
Zolotarev coefficients, written independently of the oracle with Jacobi theta
series) agree with the oracle's Landen-transformation coefficients."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2203_08900_gb300 import build as b
    b.build()
    import paper_2203_08900_gb300 as P
    P.lib()
    return P


def test_exports_every_declared_symbol(P):
    hdr = open(os.path.join(ROOT, "include", "pssd.h")).read()
    declared = set(re.findall(r"\b(pssd_[a-z_0-9]+)\s*\(", hdr))
    assert {"pssd_zolo_coeffs", "pssd_sign", "pssd_split", "pssd_eig"} <= declared
    L = P.lib()
    for name in sorted(declared | set(P.EXPORTS)):
        assert hasattr(L, name), name


@pytest.mark.parametrize("ell,r", [(1e-16, 8), (1e-12, 7), (1e-8, 5), (1e-4, 4), (1e-2, 3), (0.3, 2),
                                   (0.7071, 3), (0.71, 2), (0.95, 1), (0.999999, 2), (1.0, 1)])
def test_library_coefficients_match_oracle(P, ell, r):
    c, a, ch, l1 = P.zolo_coeffs(ell, r)
    co, ao, cho, l1o = O.zolo_coeffs(ell, r)
    assert np.max(np.abs(c - co) / co) < 1e-12
    assert np.max(np.abs(a - ao) / ao) < 1e-10
    assert abs(ch - cho) < 1e-13 * cho
    assert abs(l1 - l1o) < 1e-13


def test_choose_r_matches_oracle(P):
    for kap in [1.5, 10, 1e2, 1e3, 1e4, 1e8, 1e12, 1e16]:
        assert P.choose_r(1 / kap) == O.choose_r(1 / kap)
        assert P.choose_r(1 / kap, 2.0 ** -24) == O.choose_r(1 / kap, 2.0 ** -24)


def test_argument_errors(P):
    L = P.lib()
    c = (ctypes.c_double * 4)(); a = (ctypes.c_double * 2)(); x = ctypes.c_double(); y = ctypes.c_double()
    assert L.pssd_zolo_coeffs(0.0, 2, c, a, ctypes.byref(x), ctypes.byref(y)) == -1
    assert L.pssd_zolo_coeffs(0.5, 0, c, a, ctypes.byref(x), ctypes.byref(y)) == -2
    assert L.pssd_zolo_coeffs(0.5, 2, None, a, ctypes.byref(x), ctypes.byref(y)) == -3
    assert L.pssd_choose_r(2.0, 1e-15, 8) == -1
    assert L.pssd_status_string(1).decode().startswith("Sigma")
    # null handle is rejected before any device work
    assert L.pssd_sign(None, 4, None, None, 4, None, 4, None, None) == -1
