"""Pins of the oracle's matrix-level functions (Alg. 8, Alg. 7, Alg. 3) against
closed forms, special cases, brute force and the paper's theorems."""
import math

import numpy as np
import pytest

import casida_inputs as G
import oracle as O


def _J(n):
    return np.r_[np.ones(n // 2), -np.ones(n // 2)]


# --- scalar kernels against definitions / independent routines --------------

def test_cholesky_lu_jacobi_kernels():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((23, 23))
    A = X @ X.T + 23 * np.eye(23)
    L = O.cholesky(A)
    assert np.allclose(np.tril(L), L) and np.linalg.norm(L @ L.T - A) < 1e-13 * np.linalg.norm(A)
    B = rng.standard_normal((23, 5))
    Y = O.lu_solve(X, B)
    assert np.linalg.norm(X @ Y - B) < 1e-12 * np.linalg.norm(B) * np.linalg.cond(X)
    w, V = O.jacobi_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), rtol=1e-13, atol=0)
    assert np.linalg.norm(A @ V - V * w) < 1e-12 * np.linalg.norm(A)
    with pytest.raises(O.NotDefinite):
        O.cholesky(A - 200 * np.eye(23))


def test_pivoted_lowrank_chol_on_projector():
    """Lemma QRisChol: the low-rank Cholesky factor of an orthogonal
    projector has orthonormal columns."""
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 7)))
    P = Q @ Q.T
    W, piv = O.pivoted_lowrank_chol(P, 7)
    assert np.linalg.norm(W @ W.T - P) < 1e-13
    assert np.linalg.norm(W.T @ W - np.eye(7)) < 1e-13
    assert len(set(piv.tolist())) == 7


# --- closed forms ------------------------------------------------------------

@pytest.mark.parametrize("a,b", [(3.0, 1.0), (2.0, -1.5), (10.0, 9.0), (1.0, 0.0)])
def test_n2_closed_form(a, b):
    """k = 1: H = [[a, b], [-b, -a]] has H^2 = (a^2 - b^2) I, so
    lambda = +-sqrt(a^2 - b^2) and sign(H) = H / sqrt(a^2 - b^2)."""
    H = np.array([[a, b], [-b, -a]])
    mu = math.sqrt(a * a - b * b)
    S_ref = H / mu
    S_alg, info = O.sign_alg(H)
    assert np.max(np.abs(S_alg - S_ref)) < 1e-14
    assert np.max(np.abs(O.sign_def(H) - S_ref)) < 1e-14
    lam, V = O.eig_def(H)
    assert np.allclose(lam, [mu, -mu], rtol=1e-15)
    lam2, V2 = O.eig_alg(H)
    assert np.allclose(lam2, [mu, -mu], rtol=1e-14)


def test_n4_brute_force():
    """k = 2: omega^2 are the eigenvalues of the 2x2 (A - B)(A + B), by the
    quadratic formula."""
    rng = np.random.default_rng(3)
    H, d1, d2 = G.casida(2, ("uniform", 1, 10), seed=3)
    A = H[:2, :2]; B = H[:2, 2:]
    T = (A - B) @ (A + B)
    tr = T[0, 0] + T[1, 1]; det = T[0, 0] * T[1, 1] - T[0, 1] * T[1, 0]
    disc = math.sqrt(tr * tr - 4 * det)
    om = np.sqrt(np.sort([(tr - disc) / 2, (tr + disc) / 2]))
    lam, _ = O.eig_def(H)
    assert np.allclose(lam, np.r_[om, -om], rtol=1e-13)
    lam2, _ = O.eig_alg(H)
    assert np.allclose(lam2, np.r_[om, -om], rtol=1e-12)


def test_b_zero_special_case():
    """B = 0: H = diag(A, -A), sign(H) = diag(I, -I), lambda = +-eig(A)."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((6, 6)); A = X @ X.T + np.eye(6)
    H = np.block([[A, np.zeros((6, 6))], [np.zeros((6, 6)), -A]])
    S, _ = O.sign_alg(H)
    assert np.max(np.abs(S - np.diag(_J(12)))) < 1e-13
    lam, _ = O.eig_alg(H)
    ev = np.sort(np.linalg.eigvalsh(A))
    assert np.allclose(lam, np.r_[ev, -ev], rtol=1e-12)


def test_same_q_exact_spectrum():
    """Q1 = Q2: P and R commute and lambda = +-sqrt(d1_i d2_i) exactly."""
    H, d1, d2 = G.casida(24, ("loguniform", 1e-2, 1e2), seed=5, same_q=True)
    om = np.sort(np.sqrt(d1 * d2))
    lam, _ = O.eig_def(H)
    assert np.max(np.abs(lam - np.r_[om, -om])) < 1e-12 * om[-1]
    lam2, _ = O.eig_alg(H)
    assert np.max(np.abs(lam2 - np.r_[om, -om])) < 1e-11 * om[-1]


def test_casida_closed_form_spectrum():
    """lambda^2 = eig((A - B)(A + B)) for the Casida form (library eigvals of
    a nonsymmetric product, an independent route)."""
    H, _, _ = G.casida(40, ("uniform", 0.1, 100), seed=6)
    k = 40
    A = H[:k, :k]; B = H[:k, k:]
    om = np.sort(np.sqrt(np.real(np.linalg.eigvals((A - B) @ (A + B)))))
    lam, _ = O.eig_def(H)
    assert np.max(np.abs(lam - np.r_[om, -om])) < 1e-11 * om[-1]


# --- theorems as invariants ---------------------------------------------------

@pytest.mark.parametrize("name,k,dist,r", [
    ("casida_u1_10_r8", 32, ("uniform", 1, 10), 8),
    ("casida_u0.1_100", 40, ("uniform", 0.1, 100), None),
    ("casida_log", 48, ("loguniform", 1e-2, 1e2), None),
])
def test_sign_invariants(name, k, dist, r):
    """S^2 = I, SH = HS, Sigma S symmetric positive definite, trace S = 2p-n,
    and the algorithm agrees with the definition.  S is not normal: a
    relative error e in S shows up as about e ||S||_2^2 in S^2 - I, so the
    literal iteration's defects are measured against ||S||_2^2."""
    H, _, _ = G.casida(k, dist, seed=7)
    n = 2 * k
    s = _J(n)
    S, info = O.sign_alg(H, r=r)
    Sd = O.sign_def(H)
    s2 = max(1.0, np.linalg.norm(Sd, 2)) ** 2
    assert np.linalg.norm(Sd @ Sd - np.eye(n)) <= 1e-12 * n * s2
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-12 * n * s2
    assert np.linalg.norm(S @ H - H @ S) <= 1e-11 * np.linalg.norm(H) * s2
    SS = s[:, None] * S
    assert np.linalg.norm(SS - SS.T) <= 1e-12 * np.linalg.norm(S) * s2
    assert np.min(np.linalg.eigvalsh(0.5 * (SS + SS.T))) > 0
    assert abs(np.trace(S)) < 1e-10
    assert np.linalg.norm(S - Sd) <= 1e-10 * np.linalg.norm(Sd)
    assert info["ell"][0] < info["ell"][1] <= info["ell"][2] <= 1.0


def test_general_signature_example1():
    """Ex. 1 inputs (random Sigma, A = Sigma Q D Q^T): algorithm vs definition
    and the split's backward error within the paper's band (Fig. BackErr_all
    shows averages at or below 1e-9 up to kappa = 1e16)."""
    for kappa in [1e2, 1e6]:
        A, sig = G.example1(30, kappa, seed=8)
        s = sig.astype(float)
        S, _ = O.sign_alg(A, s)
        Sd = O.sign_def(A, s)
        assert np.linalg.norm(S - Sd) <= 1e-9 * np.linalg.norm(Sd)
        Qp, Qm, A11, A22 = O.split_alg(A, s, S)
        p = int(np.sum(s > 0))
        assert Qp.shape == (30, p)
        assert O.split_backward_error(A, s, Qp, Qm) < 1e-9


def test_split_theorem_def_div_conq():
    """Thm. DefDivConq / Thm. HRisLDL: Q_+^T Sigma Q_+ = I_p,
    Q_-^T Sigma Q_- = -I, Q_+^T Sigma Q_- = 0, A11 SPD, A22 SND, and the
    eigenvalues of A11 (A22) are the positive (negative) eigenvalues of H."""
    H, _, _ = G.casida(32, ("uniform", 0.1, 100), seed=9)
    n = 64; s = _J(n)
    Qp, Qm, A11, A22 = O.split_alg(H)
    assert np.linalg.norm(Qp.T @ (s[:, None] * Qp) - np.eye(32)) < 1e-12
    assert np.linalg.norm(Qm.T @ (s[:, None] * Qm) + np.eye(32)) < 1e-12
    assert np.linalg.norm(Qp.T @ (s[:, None] * Qm)) < 1e-11
    assert np.min(np.linalg.eigvalsh(A11)) > 0 and np.max(np.linalg.eigvalsh(A22)) < 0
    lam, _ = O.eig_def(H)
    assert np.allclose(np.sort(np.linalg.eigvalsh(A11)), lam[:32], rtol=1e-11)
    assert np.allclose(np.sort(np.linalg.eigvalsh(A22))[::-1], lam[32:], rtol=1e-11)
    assert O.split_backward_error(H, None, Qp, Qm) < 1e-13


def test_eig_alg_residuals():
    """||HV - VD||_F / ||H||_F <= 1e-11, V^T Sigma V = diag(I,-I), and
    agreement with the definition layer, eigenvalue by eigenvalue."""
    H, _, _ = G.casida(32, ("uniform", 1, 10), seed=10)
    n = 64; s = _J(n)
    lam, V = O.eig_alg(H)
    assert np.linalg.norm(H @ V - V * lam) <= 1e-11 * np.linalg.norm(H)
    assert np.linalg.norm(V.T @ (s[:, None] * V) - np.diag(s)) <= 1e-12 * n
    lam_d, V_d = O.eig_def(H)
    assert np.max(np.abs(lam - lam_d)) <= 1e-10 * np.max(np.abs(lam_d))
    # eigenvectors (simple eigenvalues here) agree under the sign convention
    assert np.max(np.abs(V - V_d)) <= 1e-8 * np.max(np.abs(V_d))


def test_newton_sign_and_block_gradient():
    """Eq. NewtonSign agrees with the definition; the block-sign gradient
    agrees with central finite differences of <G, sign(H)>."""
    H, _, _ = G.casida(6, ("uniform", 1, 10), seed=11)
    n = 12
    assert np.linalg.norm(O.newton_sign(H) - O.sign_def(H)) < 1e-12
    rng = np.random.default_rng(12)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    grad = O.sign_vjp_block(H, Gm)
    k = 6
    for _ in range(3):
        dA = rng.standard_normal((k, k)); dA = dA + dA.T
        dB = rng.standard_normal((k, k)); dB = dB + dB.T
        dH = np.block([[dA, dB], [-dB, -dA]])
        h = 1e-6
        fd = (np.sum(Gm * O.sign_def(H + h * dH)) - np.sum(Gm * O.sign_def(H - h * dH))) / (2 * h)
        an = np.sum(grad * dH)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def test_stopping_test_and_restart_counts():
    """Alg. 8's stopping test: with exact bounds the iteration either stops
    after two steps or restarts; r = 8 on a kappa <= 10 input stops at once."""
    H, _, _ = G.casida(16, ("uniform", 1, 10), seed=13)
    S, info = O.sign_alg(H, r=8)
    assert info["restarts"] == 0
    assert info["stop"][0] <= O.U_FP64 ** (1 / 17)
