"""Pins of the oracle's scalar Zolotarev machinery (Sec. 5.3) against facts
that do not come from the oracle itself."""
import math

import numpy as np
import pytest

import oracle as O


# --- Jacobi elliptic functions: classical special values -------------------

def test_ellipk_special_values():
    # modulus 0: K = pi/2
    assert abs(O.ellipk_from_comp(1.0) - math.pi / 2) < 1e-15
    # lemniscatic case, modulus 1/sqrt2: K = Gamma(1/4)^2 / (4 sqrt(pi))
    ref = math.gamma(0.25) ** 2 / (4 * math.sqrt(math.pi))
    assert abs(O.ellipk_from_comp(1 / math.sqrt(2)) - ref) < 1e-14 * ref
    # modulus -> 1: K ~ ln(4/kc) + O(kc^2 ln kc)
    kc = 1e-12
    assert abs(O.ellipk_from_comp(kc) - math.log(4 / kc)) < 1e-9


def test_sncn_limits_and_identity():
    for u in [0.1, 0.7, 1.3]:
        s, c = O.sncn(u, 1.0)            # modulus 0: circular functions
        assert abs(s - math.sin(u)) < 1e-15 and abs(c - math.cos(u)) < 1e-15
        s, c = O.sncn(u, 1e-300 ** 0.5)  # modulus ~1: hyperbolic functions
        assert abs(s - math.tanh(u)) < 1e-14 and abs(c - 1 / math.cosh(u)) < 1e-14
    for kc in [0.3, 1e-4, 1e-10]:
        K = O.ellipk_from_comp(kc)
        for u in np.linspace(0.05, 0.95, 7) * K:
            s, c = O.sncn(u, kc)
            assert abs(s * s + c * c - 1) < 1e-14
        s, c = O.sncn(K, kc)             # sn(K) = 1, cn(K) = 0
        assert abs(s - 1) < 1e-12 and abs(c) < 1e-6


# --- scaled Zolotarev function ---------------------------------------------

CASES = [(0.5, 1), (1e-2, 3), (1e-4, 5), (1e-4, 8), (1e-8, 6), (0.9, 2)]


@pytest.mark.parametrize("ell,r", CASES)
def test_zhat_one_and_ell1(ell, r):
    c, a, chat, ell1 = O.zolo_coeffs(ell, r)
    assert abs(O.zolo_eval(1.0, ell, r) - 1.0) < 1e-14            # Zhat(1) = 1 (Eq. hatZ)
    assert abs(O.zolo_eval(ell, ell, r) - ell1) < 1e-13 * max(ell1, 1e-3)
    assert np.all(np.diff(c) > 0) and np.all(c > 0)              # reading R1 gives increasing c
    assert np.all(a > 0)                                           # residues of Zhat/x are positive


@pytest.mark.parametrize("ell,r", CASES)
def test_partial_fractions_equal_product_form(ell, r):
    x = np.r_[np.geomspace(ell, 1, 200), -np.geomspace(ell, 1, 50)]
    y1 = O.zolo_eval(x, ell, r)
    y2 = O.zolo_eval_partial_fractions(x, ell, r)
    assert np.max(np.abs(y1 - y2)) < 1e-12


def _extrema(f, lo, hi, m=200001):
    x = np.geomspace(lo, hi, m)
    y = f(x)
    d = np.sign(np.diff(y))
    idx = [0] + [i for i in range(1, len(d)) if d[i] != d[i - 1] and d[i] != 0 and d[i - 1] != 0] + [len(y) - 1]
    return x[idx], y[idx]


@pytest.mark.parametrize("ell,r", [(1e-2, 3), (1e-4, 5), (1e-3, 4), (0.2, 2)])
def test_equioscillation(ell, r):
    """Best rational approximation on [l,1] (Eq. Zolo and its defining
    min-max problem): Zhat oscillates between l_1 (r+1 minima, x=l included)
    and 1 (r+1 maxima, x=1 included): 2r+2 alternation points of the error of
    the optimal (unscaled) function."""
    c, a, chat, ell1 = O.zolo_coeffs(ell, r)
    f = lambda x: O.zolo_eval(x, ell, r)
    xs, ys = _extrema(f, ell, 1.0)
    assert len(xs) == 2 * r + 2
    mins = ys[0::2]; maxs = ys[1::2]
    assert np.max(np.abs(mins - ell1)) < 1e-7 * max(ell1, 1e-2)
    assert np.max(np.abs(maxs - 1.0)) < 1e-7
    # the optimally scaled function equioscillates around sign(x) = 1
    s = 2 / (1 + ell1)
    err = 1 - s * ys
    assert np.max(np.abs(np.abs(err) - abs(err[0]))) < 1e-6 * abs(err[0])


@pytest.mark.parametrize("ell,r", [(1e-2, 1), (1e-3, 2), (0.3, 1), (1e-5, 2)])
def test_composition_law(ell, r):
    """Zhat_{2r+1}(Zhat_{2r+1}(x; l); l_1) = Zhat_{(2r+1)^2}(x; l)."""
    _, _, _, ell1 = O.zolo_coeffs(ell, r)
    R = ((2 * r + 1) ** 2 - 1) // 2
    x = np.geomspace(ell, 1, 400)
    lhs = O.zolo_eval(O.zolo_eval(x, ell, r), ell1, r)
    rhs = O.zolo_eval(x, ell, R)
    assert np.max(np.abs(lhs - rhs)) < 1e-10


@pytest.mark.parametrize("ell", [0.9, 0.3, 1e-2, 1e-4, 1e-8])
def test_r1_is_dwh(ell):
    """r = 1 gives the dynamically weighted Halley function of
    Nakatsukasa, Bai & Gygi (2010), f(x) = x (a + b x^2) / (1 + c x^2) with
    gamma = (4(1-l^2)/l^4)^{1/3},
    a = sqrt(1+gamma) + 1/2 sqrt(8 - 4 gamma + 8 (2-l^2) / (l^2 sqrt(1+gamma))),
    b = (a-1)^2/4, c = a + b - 1."""
    g = (4 * (1 - ell ** 2) / ell ** 4) ** (1 / 3)
    a = math.sqrt(1 + g) + 0.5 * math.sqrt(8 - 4 * g + 8 * (2 - ell ** 2) / (ell ** 2 * math.sqrt(1 + g)))
    b = (a - 1) ** 2 / 4
    cc = a + b - 1
    x = np.geomspace(ell, 1, 300)
    dwh = x * (a + b * x * x) / (1 + cc * x * x)
    z = O.zolo_eval(x, ell, 1)
    # the closed form itself cancels catastrophically (8 - 4 gamma + ...) for tiny l
    tol = 1e-9 if ell >= 1e-6 else 1e-7
    assert np.max(np.abs(dwh - z) / z) < tol


def test_two_steps_r8_reach_one():
    """Sec. 5.3: with r = 8 and l >= 1e-16, two steps map [l,1] into
    [1 - 1e-15, 1]."""
    for ell in [1e-16, 1e-12, 1e-6, 0.1]:
        _, _, _, l1 = O.zolo_coeffs(ell, 8)
        _, _, _, l2 = O.zolo_coeffs(min(l1, 1.0), 8)
        assert 1 - l2 <= 1e-15 + 2e-16


def test_choose_r_rule():
    """Reading R3 (smallest r with 1 - l_2 <= tau); monotone in kappa and
    r <= 8 up to kappa = 1e16 by the previous test."""
    rs = [O.choose_r(1 / kap) for kap in [10, 1e2, 1e3, 1e4, 1e8, 1e12, 1e16]]
    assert rs == sorted(rs)
    assert rs[-1] <= 8
    assert O.choose_r(1e-4, tau=2.0 ** -24) <= O.choose_r(1e-4)


_KAPPAS = [10, 1e2, 1e3, 1e4, 1e8, 1e12, 1e16]
_TAUS = [1e-15, 1e-6]   # the FP64 steps and the FP32 steps of the mixed path


def _ell2_product_form(ell, r):
    """l_2 of two steps, evaluated with the product form of Eq. (hatZ) at the
    interval's end point (independent of the coefficient routine's own
    l-update): l_1 = Zhat(l; l), l_2 = Zhat(l_1; l_1)."""
    l1 = min(float(O.zolo_eval(ell, ell, r)), 1.0)
    return min(float(O.zolo_eval(l1, l1, r)), 1.0)


@pytest.mark.parametrize("tau", _TAUS)
@pytest.mark.parametrize("kappa", _KAPPAS)
def test_choose_r_is_minimal(kappa, tau):
    """Reading R3 of the choice of r (Sec. 5.3, "two steps suffice"): r is the
    SMALLEST degree for which two steps map [1/kappa, 1] into [1 - tau, 1].
    Pins both halves of the rule: the criterion holds at r and fails at r - 1,
    so an off-by-one or a wrong tau fails here."""
    ell = 1.0 / kappa
    r = O.choose_r(ell, tau)
    assert 1 <= r <= 8
    assert 1.0 - _ell2_product_form(ell, r) <= tau
    if r > 1:
        assert 1.0 - _ell2_product_form(ell, r - 1) > tau


def test_sc_comp_against_real_argument_landen():
    """Two independent routes to sc(u) agree to within the real-argument
    route's own error, which grows like u_fp64/cn (cos of an angle near pi/2)."""
    for kc in [0.5, 1e-2, 1e-6]:
        K = O.ellipk_from_comp(kc)
        for u in np.linspace(0.05, 0.7, 6) * K:
            s, c = O.sncn(u, kc)
            assert abs(O.sc_comp(u, kc) - s / c) < (1e-13 + 1e-14 / abs(c)) * abs(s / c)


def test_coefficients_high_precision():
    """c_i against 50-digit Jacobi elliptic functions (mpmath), including
    l = 1e-16 where cn is below 1e-15."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for ell, r in [(1e-16, 8), (1e-8, 5), (1e-4, 4), (0.3, 2), (0.95, 1)]:
        e = mp.mpf(ell); m = 1 - e * e
        Kp = mp.ellipk(m)
        c, _, _, _ = O.zolo_coeffs(ell, r)
        for i in range(1, 2 * r + 1):
            u = i * Kp / (2 * r + 1)
            ref = e * e * (mp.ellipfun("sn", u, m=m) / mp.ellipfun("cn", u, m=m)) ** 2
            assert abs(c[i - 1] - float(ref)) <= 1e-12 * float(ref)
