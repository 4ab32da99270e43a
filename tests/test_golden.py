"""Values the paper prints, stored as cited text fixtures under tests/golden/,
checked against the oracle and against the library's host coefficient routine
(no GPU needed)."""
import os

import pytest

import oracle as O

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U = 2.0 ** -53


def _rounding(r):
    """First-order rounding bound of an FP64 l-update l_{k+1} = Chat l prod_j
    (l^2 + c_2j) / (l^2 + c_{2j-1}): Chat is a product of 2r factors, then r
    additions pairs, r quotients and r + 1 products, about 6r + 2 rounded
    operations, each contributing at most u relatively (l_2 <= 1)."""
    return (6 * r + 2) * U


def _fixture(name):
    vals = {}
    for line in open(os.path.join(HERE, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_two_zolotarev_steps_r8_oracle():
    """Sec. 5.3 (after Eq. hatZ): r = 8, l >= 1e-16 -> two steps reach [1 - 1e-15, 1]."""
    f = _fixture("zolotarev_two_steps_r8.txt")
    r = int(f["r"])
    for ell in (f["ell_min"], 1e-14, 1e-10, 1e-6, 1e-3, 0.5):
        _, _, _, l1 = O.zolo_coeffs(ell, r)
        _, _, _, l2 = O.zolo_coeffs(min(l1, 1.0), r)
        assert 1.0 - l2 <= f["width"] + _rounding(r)


def test_two_zolotarev_steps_r8_library():
    """The same printed claim through the C ABI's host routine pssd_zolo_coeffs."""
    try:
        import paper_2203_08900_gb300 as P
        P.lib()
    except Exception as e:          # the library is built by __graft_entry__.build()
        pytest.skip("libpssd.so not built: %s" % e)
    f = _fixture("zolotarev_two_steps_r8.txt")
    r = int(f["r"])
    for ell in (f["ell_min"], 1e-12, 1e-6, 0.5):
        _, _, _, l1 = P.zolo_coeffs(ell, r)
        _, _, _, l2 = P.zolo_coeffs(min(l1, 1.0), r)
        assert 1.0 - l2 <= f["width"] + _rounding(r)
