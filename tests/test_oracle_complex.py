"""Pins of the oracle's complex pseudo-Hermitian layer (the BSE forms, Eqs. BSE1
and BSE2) against what the mathematics fixes: the scalar complex Cholesky and
Jacobi against the library routines they restate, the closed-form spectrum of
the Q1 = Q2 BSE2 form, the +-lambda pairing of BSE1, the real case, the 2 x 2
closed form, the invariants of sign(H) (S^2 = I, SH = HS, Sigma S Hermitian),
and the real embedding [[Re, -Im], [Im, Re]] through the real oracle."""
import math

import numpy as np
import pytest

import casida_inputs as G
import oracle as O


def _sig(n):
    return np.r_[np.ones(n // 2), -np.ones(n // 2)]


def test_zcholesky_matches_library():
    rng = np.random.default_rng(1)
    for n in (1, 5, 17):
        Z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        M = Z @ Z.conj().T + n * np.eye(n)
        L = O.zcholesky(M)
        assert np.allclose(np.triu(L, 1), 0)
        assert np.all(np.diag(L).real > 0) and np.allclose(np.diag(L).imag, 0)
        assert np.linalg.norm(L @ L.conj().T - M) <= 1e-14 * np.linalg.norm(M)
        assert np.linalg.norm(L - np.linalg.cholesky(M)) <= 1e-13 * np.linalg.norm(L)
    with pytest.raises(O.NotDefinite):
        O.zcholesky(np.diag([1.0, -1.0]).astype(complex))


def test_zjacobi_matches_library():
    rng = np.random.default_rng(2)
    for n in (2, 7, 24):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = A + A.conj().T
        w, U = O.zjacobi_eigh(A)
        assert np.max(np.abs(w - np.linalg.eigvalsh(A))) <= 1e-13 * np.max(np.abs(w))
        assert np.linalg.norm(U.conj().T @ U - np.eye(n)) <= 1e-13 * n
        assert np.linalg.norm(A @ U - U * w) <= 1e-13 * np.linalg.norm(A)


def test_bse2_same_q_closed_form():
    """Q1 = Q2: lambda = +-sqrt(d1_i d2_i)."""
    H, d1, d2 = G.bse2(12, ("uniform", 0.5, 5.0), seed=3, same_q=True)
    lam, V = O.zeig_def(H)
    om = np.sort(np.sqrt(d1 * d2))
    assert np.max(np.abs(lam - np.r_[om, -om])) <= 1e-13 * om[-1]
    n = H.shape[0]
    s = _sig(n)
    assert np.linalg.norm(H @ V - V * lam) <= 1e-13 * np.linalg.norm(H)
    assert np.linalg.norm(V.conj().T @ (s[:, None] * V) - np.diag(np.sign(lam))) <= 1e-12 * n


def test_bse1_pairing():
    """[[A, B], [-conj B, -conj A]]: if [x; y] has eigenvalue lambda then [conj y; conj x]
    has -lambda, so the spectrum is symmetric and the eigenvectors pair up."""
    H = G.bse1(10, seed=4)
    k = 10
    lam, V = O.zeig_def(H)
    assert np.max(np.abs(lam[:k] + lam[k:])) <= 1e-12 * np.max(np.abs(lam))
    for j in range(k):
        x, y = V[:k, j], V[k:, j]
        w = np.r_[np.conj(y), np.conj(x)]
        assert np.linalg.norm(H @ w + lam[j] * w) <= 1e-12 * np.linalg.norm(H) * np.linalg.norm(w)


def test_real_input_reduces_to_real_oracle():
    H, _, _ = G.casida(9, ("uniform", 1.0, 10.0), seed=5)
    lz, Vz = O.zeig_def(H.astype(complex))
    lr, Vr = O.eig_def(H)
    assert np.max(np.abs(lz - lr)) <= 1e-13 * np.max(np.abs(lr))
    # eigenvectors equal up to a phase (both sides fix it on the largest entry)
    assert np.max(np.abs(Vz - Vr)) <= 1e-10 * np.max(np.abs(Vr))
    assert np.linalg.norm(O.zsign_def(H.astype(complex)) - O.sign_def(H)) <= 1e-12 * H.shape[0]


def test_two_by_two_closed_form():
    """k = 1 BSE2: H = [[a, b], [-b, -a]] (a, b real by Hermiticity), lambda = +-sqrt(a^2 - b^2)."""
    a, b = 3.0, 1.25
    H = np.array([[a, b], [-b, -a]], dtype=complex)
    lam, _ = O.zeig_def(H)
    r = math.sqrt(a * a - b * b)
    assert np.max(np.abs(lam - np.array([r, -r]))) <= 1e-15 * a
    S = O.zsign_def(H)
    assert np.linalg.norm(S - H / r) <= 1e-14


@pytest.mark.parametrize("form", ["bse1", "bse2"])
def test_sign_invariants_and_real_embedding(form):
    if form == "bse1":
        H = G.bse1(8, seed=6)
    else:
        H, _, _ = G.bse2(8, ("loguniform", 0.1, 10.0), seed=6)
    n = H.shape[0]
    s = _sig(n)
    S = O.zsign_def(H)
    I = np.eye(n)
    assert np.linalg.norm(S @ S - I) <= 1e-12 * n
    assert np.linalg.norm(S @ H - H @ S) <= 1e-12 * np.linalg.norm(H)
    SS = s[:, None] * S
    assert np.linalg.norm(SS - SS.conj().T) <= 1e-12 * n
    # real embedding R(Z) = [[Re Z, -Im Z], [Im Z, Re Z]] with signature [sigma; sigma]
    R = np.block([[H.real, -H.imag], [H.imag, H.real]])
    Sr = O.sign_def(R, np.r_[s, s])
    RS = np.block([[S.real, -S.imag], [S.imag, S.real]])
    assert np.linalg.norm(Sr - RS) <= 1e-11 * n
