"""GPU-vs-oracle parity of the C-ABI library (plain FP64 path).

Tolerances (from the target accuracy of the method):
  |lambda - lambda_ref| <= 1e-10 ||H||_2,  ||S^2 - I||_F <= 1e-12 n (scaled by
  ||S||_2^2 for non-normal S), J-symmetry defect <= 1e-12 (same scaling),
  ||HV - VD||_F / ||H||_F <= 1e-11.
"""
import numpy as np
import pytest
import torch

import casida_inputs as G
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2203_08900_gb300 import build as b
    b.build()
    import paper_2203_08900_gb300 as P
    P.lib()
    return P


def _J(n):
    return np.r_[np.ones(n // 2), -np.ones(n // 2)]


def _dev(H):
    return torch.from_numpy(np.ascontiguousarray(H)).cuda()


CASES = [
    ("u1_10_k1", 1, ("uniform", 1.0, 10.0)),
    ("u1_10_k33", 33, ("uniform", 1.0, 10.0)),       # n = 66: ragged tail of a 64 tile
    ("u0.1_100_k64", 64, ("uniform", 0.1, 100.0)),   # n = 128: exactly two tiles
    ("log_k97", 97, ("loguniform", 1e-2, 1e2)),      # n = 194, kappa ~ 1e4
    ("u1_10_k160", 160, ("uniform", 1.0, 10.0)),     # n = 320: several tiles + tail
]


@pytest.mark.parametrize("name,k,dist", CASES)
def test_sign_matches_oracle(P, name, k, dist):
    H, _, _ = G.casida(k, dist, seed=100 + k)
    n = 2 * k
    alpha, beta = O.estimate_bounds(H)
    S, info = P.sign(_dev(H), alpha=alpha, beta=beta)
    S = S.cpu().numpy()
    Sd = O.sign_def(H)
    Sa, oinfo = O.sign_alg(H, alpha=alpha, beta=beta)
    s2 = max(1.0, np.linalg.norm(Sd, 2)) ** 2
    assert info["r_used"][0] == oinfo["r"][0]                    # same coefficients as the oracle
    assert info["restarts"] == oinfo["restarts"]
    assert np.linalg.norm(S - Sd) <= 1e-11 * np.linalg.norm(Sd) * max(1.0, np.linalg.norm(Sd, 2))
    assert np.linalg.norm(S - Sa) <= 1e-10 * np.linalg.norm(Sd) * max(1.0, np.linalg.norm(Sd, 2))
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-12 * n * s2
    JS = _J(n)[:, None] * S
    assert np.linalg.norm(JS - JS.T) <= 1e-12 * np.linalg.norm(S) * s2
    assert abs(np.trace(S)) <= 1e-10 * n


def test_sign_estimated_bounds_and_restart_path(P):
    """Default (estimated) alpha, beta; the log-uniform input exercises the
    stopping test's restart."""
    H, _, _ = G.casida(100, ("loguniform", 1e-2, 1e2), seed=7)
    S, info = P.sign(_dev(H))
    Sd = O.sign_def(H)
    assert info["alpha"] >= np.max(np.abs(np.linalg.eigvals(H))) * 0.999
    assert np.linalg.norm(S.cpu().numpy() - Sd) <= 1e-11 * np.linalg.norm(Sd) * np.linalg.norm(Sd, 2)
    assert info["passes"] >= 1 and info["steps"] == 2 * info["passes"]


def test_sign_general_signature(P):
    """Example-1 inputs: random Sigma, A = Sigma Q D Q^T."""
    A, sig = G.example1(90, 1e3, seed=3)
    S, info = P.sign(_dev(A), sigma=sig)
    Sd = O.sign_def(A, sig.astype(float))
    assert np.linalg.norm(S.cpu().numpy() - Sd) <= 1e-10 * np.linalg.norm(Sd) * np.linalg.norm(Sd, 2)
    assert info["p"] == int((sig > 0).sum())


def test_n2_closed_form(P):
    H = np.array([[3.0, 1.0], [-1.0, -3.0]])
    S, _ = P.sign(_dev(H))
    assert np.max(np.abs(S.cpu().numpy() - H / np.sqrt(8.0))) < 1e-14
    D, V, _ = P.eig(_dev(H))
    assert np.allclose(D.cpu().numpy(), [np.sqrt(8.0), -np.sqrt(8.0)], rtol=1e-14)


@pytest.mark.parametrize("k,dist", [(40, ("uniform", 0.1, 100.0)), (150, ("loguniform", 1e-2, 1e2))])
def test_split_matches_oracle(P, k, dist):
    H, _, _ = G.casida(k, dist, seed=200 + k)
    n = 2 * k
    J = _J(n)
    Q, A11, A22, p, info = P.split(_dev(H))
    Q = Q.cpu().numpy(); A11 = A11.cpu().numpy(); A22 = A22.cpu().numpy()
    assert p == k
    Qp, Qm = Q[:, :p], Q[:, p:]
    # (Sigma, Sigma_hat)-orthogonality (Thm. HRisLDL / DefDivConq)
    assert np.linalg.norm(Q.T @ (J[:, None] * Q) - np.diag(J)) <= 1e-12 * n * np.linalg.norm(Q, 2) ** 2
    # projector onto the positive invariant subspace agrees with the oracle's (I+S)/2
    Pp = Qp @ Qp.T * J[None, :]
    Pref = 0.5 * (np.eye(n) + O.sign_def(H))
    assert np.linalg.norm(Pp - Pref) <= 1e-10 * np.linalg.norm(Pref) * np.linalg.norm(Pref, 2)
    # blocks: SPD / SND, and Q^{-1} H Q = diag(A11, A22)
    assert np.min(np.linalg.eigvalsh(A11)) > 0 and np.max(np.linalg.eigvalsh(A22)) < 0
    lam, _ = O.eig_def(H)
    nrm = np.max(np.abs(lam))
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(A11)) - lam[:p])) <= 1e-10 * nrm
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(A22))[::-1] - lam[p:])) <= 1e-10 * nrm
    assert np.linalg.norm(A11 - Qp.T @ (J[:, None] * H) @ Qp) <= 1e-10 * np.linalg.norm(A11)
    be = np.linalg.norm(Qp.T @ (J[:, None] * H) @ Qm) / np.linalg.norm(H)
    assert be <= 1e-11
    # the library's backward error of the split of the symmetric K = L^T Sigma L ~ H
    assert 0 <= info["split_backerr"] <= 1e-12
    # the oracle's Alg. 7 split spans the same subspace
    oQp, oQm, oA11, oA22 = O.split_alg(H)
    assert np.allclose(np.sort(np.linalg.eigvalsh(oA11)), np.sort(np.linalg.eigvalsh(A11)), rtol=1e-9)


@pytest.mark.parametrize("k,dist,leaf", [(33, ("uniform", 1.0, 10.0), 64), (100, ("uniform", 0.1, 100.0), 16),
                                         (128, ("loguniform", 1e-2, 1e2), 32)])
def test_eig_matches_oracle(P, k, dist, leaf):
    H, _, _ = G.casida(k, dist, seed=300 + k)
    n = 2 * k
    J = _J(n)
    D, V, info = P.eig(_dev(H), leaf=leaf)
    D = D.cpu().numpy(); V = V.cpu().numpy()
    lam, Vref = O.eig_def(H)
    nrmH2 = np.max(np.abs(lam))
    assert np.max(np.abs(D - lam)) <= 1e-10 * nrmH2
    assert np.linalg.norm(H @ V - V * D) <= 1e-11 * np.linalg.norm(H)
    assert np.linalg.norm(V.T @ (J[:, None] * V) - np.diag(J)) <= 1e-12 * n * max(1.0, np.linalg.norm(V, 2)) ** 2
    # eigenvectors of well-separated eigenvalues agree with the definition's
    gaps = np.abs(np.diff(np.sort(lam)))
    if np.min(gaps) > 1e-6 * nrmH2:
        assert np.max(np.abs(V - Vref)) <= 1e-7 * np.max(np.abs(Vref))
    if k > leaf:
        assert info["levels"] >= 2


def test_same_q_exact_spectrum(P):
    """Q1 = Q2: lambda = +-sqrt(d1_i d2_i) exactly."""
    H, d1, d2 = G.casida(200, ("loguniform", 1e-2, 1e2), seed=9, same_q=True)
    om = np.sort(np.sqrt(d1 * d2))
    D, V, info = P.eig(_dev(H))
    D = D.cpu().numpy()
    assert np.max(np.abs(D - np.r_[om, -om])) <= 1e-10 * om[-1]


def test_b_zero(P):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((50, 50)); A = X @ X.T / 50 + np.eye(50)
    H = np.block([[A, np.zeros((50, 50))], [np.zeros((50, 50)), -A]])
    S, _ = P.sign(_dev(H))
    assert np.max(np.abs(S.cpu().numpy() - np.diag(_J(100)))) < 1e-12


def test_errors_are_status_codes(P):
    H, _, _ = G.casida(20, ("uniform", 1.0, 10.0), seed=1)
    bad = H.copy(); bad[0, 1] += 1.0                      # not pseudosymmetric
    with pytest.raises(P.PssdError) as e:
        P.sign(_dev(bad))
    assert e.value.status == 8
    nd = H.copy(); nd[:20, :20] -= 20 * np.eye(20); nd[20:, 20:] += 20 * np.eye(20)   # Sigma H indefinite
    with pytest.raises(P.PssdError) as e:
        P.sign(_dev(nd))
    assert e.value.status == 1
    nan = H.copy(); nan[3, 3] = np.nan
    with pytest.raises(P.PssdError) as e:
        P.sign(_dev(nan))
    assert e.value.status == 4
    # the context is still usable afterwards
    S, _ = P.sign(_dev(H))
    assert torch.isfinite(S).all()


def test_order_limit_is_an_argument_error(P):
    """n above PSSD_MAX_N is rejected by argument validation (-2) before any
    device work; the pointers are never dereferenced."""
    import ctypes
    h = P.Handle()
    H = torch.zeros(2, 2, dtype=torch.float64, device="cuda")
    S = torch.empty_like(H)
    o = P._opts()
    info = P.Info()
    st = P.lib().pssd_sign(h._h, P.MAX_N + 1, None, ctypes.c_void_p(H.data_ptr()), P.MAX_N + 1,
                           ctypes.c_void_p(S.data_ptr()), P.MAX_N + 1, ctypes.byref(o), ctypes.byref(info))
    assert st == -2


@pytest.mark.parametrize("precision", ["fp64", "emulated"])
def test_split_backerr_estimate_tracks_exact(P, precision):
    """Without PSSD_FLAG_RESIDUALS the split's backward error ||U_+^T K U_-||_F/||K||_F
    comes from a 16-column Gaussian probe; with it, from the full product.  A
    chi-square(16) norm ratio lies within [1/3, 3] except with probability < 1e-3."""
    prec = {"fp64": P.PSSD_FP64, "emulated": P.PSSD_FP64_EMULATED}[precision]
    H, _, _ = G.casida(150, ("loguniform", 1e-2, 1e2), seed=77)
    Hd = _dev(H)
    _, _, _, _, est = P.split(Hd, precision=prec)
    _, _, _, _, ex = P.split(Hd, precision=prec, flags=P.FLAG_RESIDUALS)
    assert 0 < ex["split_backerr"] <= 1e-12
    assert ex["split_backerr"] / 3 <= est["split_backerr"] <= 3 * ex["split_backerr"]


@pytest.mark.parametrize("case", ["casida_log", "casida_unif", "example1"])
def test_estimated_bounds_enclose_the_spectrum(P, case):
    """Reading R5: alpha >= lambda_max(M), beta <= lambda_min(M) (M = sym(Sigma H)), from the
    extreme Ritz values of 24 Lanczos steps with the safety factors 1.05 and 0.9, and the
    estimated condition number within 1.2x of the exact one (so the r rule sees the same kappa
    band); the structure-aware entry point: alpha >= sigma_max(C) = max|lambda(H)|,
    beta <= min|lambda(H)|."""
    sigma = None
    if case == "casida_log":
        H, _, _ = G.casida(300, ("loguniform", 1e-2, 1e2), seed=71)
    elif case == "casida_unif":
        H, _, _ = G.casida(300, ("uniform", 1.0, 10.0), seed=72)
    else:
        H, sigma = G.example1(500, 1e6, seed=73)
    n = H.shape[0]
    s = O.signature(n, sigma.astype(float) if sigma is not None else None)
    M = s[:, None] * H
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    _, info = P.sign(_dev(H), sigma=sigma)
    assert ev[-1] <= info["alpha"] and info["beta"] <= ev[0]
    assert (info["alpha"] / info["beta"]) <= 1.2 * (ev[-1] / ev[0])
    if case != "example1":
        k = n // 2
        _, ic = P.casida_sign(_dev(H[:k, :k]), _dev(H[:k, k:]))
        lam = np.abs(np.linalg.eigvals(H))
        assert lam.max() <= ic["alpha"] and ic["beta"] <= lam.min()
