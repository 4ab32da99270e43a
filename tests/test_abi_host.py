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


@pytest.mark.parametrize("tau", [1e-15, 1e-6])
def test_library_choose_r_is_minimal(P, tau):
    """The library's rule (reading R3 of Sec. 5.3) against the product form of
    Eq. (hatZ) evaluated here: two steps of degree r reach [1 - tau, 1] and
    two steps of degree r - 1 do not."""
    for kappa in [10, 1e2, 1e3, 1e4, 1e8, 1e12, 1e16]:
        ell = 1.0 / kappa
        r = P.choose_r(ell, tau)

        def ell2(rr):
            l1 = min(float(O.zolo_eval(ell, ell, rr)), 1.0)
            return min(float(O.zolo_eval(l1, l1, rr)), 1.0)

        assert 1.0 - ell2(r) <= tau
        if r > 1:
            assert 1.0 - ell2(r - 1) > tau


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


def test_option_ranges_are_argument_errors(P):
    """Options outside their ranges are rejected before any device work (the
    pointers below are never dereferenced): r outside [0, 64] (the
    coefficient routine's range), beta > alpha, an unknown precision or
    method, a non-Zolotarev method in mixed precision, a negative wait bound."""
    L = P.lib()
    h = ctypes.c_void_p()
    assert L.pssd_create(ctypes.byref(h), None) == 0
    fake = ctypes.c_void_p(0x1000)      # H
    out = ctypes.c_void_p(0x2000)       # outputs (distinct from H)
    info = P.Info()
    bad = [dict(r=65), dict(r=-1), dict(alpha=1.0, beta=2.0), dict(alpha=-1.0), dict(precision=3),
           dict(method=3), dict(precision=P.PSSD_MIXED, method=P.METHOD_DWH), dict(wait_cycles=-5)]
    for kw in bad:
        o = P._opts(**kw)
        assert L.pssd_sign(h, 4, None, fake, 4, out, 4, ctypes.byref(o), ctypes.byref(info)) == -8, kw
        assert L.pssd_eig(h, 4, None, fake, 4, out, 4, out, ctypes.byref(o), ctypes.byref(info)) == -9, kw
        assert L.pssd_split(h, 4, None, fake, 4, None, 4, out, 4, out, 2, out, 2, None, ctypes.byref(o),
                            ctypes.byref(info)) == -15, kw
    # a split whose precomputed S has too small a leading dimension, and missing blocks
    o = P._opts()
    assert L.pssd_split(h, 4, None, fake, 4, out, 3, out, 4, out, 2, out, 2, None, ctypes.byref(o),
                        ctypes.byref(info)) == -7
    assert L.pssd_split(h, 4, None, fake, 4, None, 4, out, 4, None, 2, out, 2, None, ctypes.byref(o),
                        ctypes.byref(info)) == -10
    assert L.pssd_destroy(h) == 0


def test_phase_launch_counters(P):
    """pssd_launch_count_phases: one counter per PSSD_PHASE_* index, named in the
    binding in header order; without a GPU nothing has been launched."""
    hdr = open(os.path.join(ROOT, "include", "pssd.h")).read()
    idx = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"#define PSSD_PHASE_([A-Z_]+) (\d+)", hdr)}
    count = idx.pop("count")
    assert P.lib().pssd_launch_count_phases(None, 0) == count == len(P.PHASES)
    assert sorted(idx.values()) == list(range(count))
    for name, i in idx.items():
        assert P.PHASES[i] == name
    got = P.launch_count_phases()
    assert list(got) == P.PHASES
    assert all(v >= 0 for v in got.values())
