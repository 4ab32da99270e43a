"""Pins of the oracle's general (non-definite) pseudosymmetric layer: the sign from
its definition (R14), the hyperbolic bases of Alg. 5 (Thm. HRisLDL) and the
divide-and-conquer of Alg. 3, against what the construction and the theorems
fix -- the spectrum and sign(A) built in (A = V C V^{-1} with V^T Sigma V =
Sigma), the 2 x 2 closed form, the projector identity P = Q Sigma_hat Q^T Sigma,
invariance of the bases, Thm. DefDivConq's signatures and the definite oracle
(Cholesky + Jacobi) on definite inputs."""
import numpy as np
import pytest

import casida_inputs as G
import oracle as O


def _sign_C(C):
    """sign of the constructed block-diagonal C: sign(lambda) on 1 x 1 entries, sign(mu) I
    on each [[mu, nu], [-nu, mu]] block (its eigenvalues mu +- i nu)."""
    d = np.sign(np.diag(C))
    return np.diag(d)


def _spectrum_C(C):
    n = C.shape[0]
    vals = []
    for i in range(n):
        j = np.flatnonzero((C[i] != 0.0) & (np.arange(n) != i))
        if j.size:
            vals.append(complex(C[i, i], abs(C[i, j[0]])) if i < j[0] else complex(C[i, i], -abs(C[i, j[0]])))
        else:
            vals.append(complex(C[i, i]))
    return np.array(sorted(vals, key=lambda z: (round(z.real, 12), z.imag)))


CASES = [(7, 1, 0), (12, 2, 1), (24, 5, 2), (24, 0, 3), (31, 7, 4)]


@pytest.mark.parametrize("n,pairs,seed", CASES)
def test_generator_structure(n, pairs, seed):
    A, s, C, V = G.general_pseudosym(n, seed=seed, n_pairs=pairs)
    sf = s.astype(float)
    SA = sf[:, None] * A
    assert np.linalg.norm(SA - SA.T) <= 1e-13 * np.linalg.norm(SA)
    assert np.linalg.norm(V.T @ (sf[:, None] * V) - np.diag(sf)) <= 1e-13 * n
    assert np.sum(np.abs(C - np.diag(np.diag(C))) > 0) == 2 * pairs


@pytest.mark.parametrize("n,pairs,seed", CASES)
def test_gsign_matches_construction(n, pairs, seed):
    """sign(A) = V sign(C) V^{-1}, V^{-1} = Sigma V^T Sigma, built in by the generator."""
    A, s, C, V = G.general_pseudosym(n, seed=seed, n_pairs=pairs)
    sf = s.astype(float)
    Vinv = (sf[:, None] * V.T) * sf[None, :]
    S_ref = V @ _sign_C(C) @ Vinv
    S = O.gsign_def(A)
    k = np.linalg.cond(V)
    assert np.linalg.norm(S - S_ref) <= 1e-12 * k * k * np.linalg.norm(S_ref)
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-12 * k * k * n
    assert np.linalg.norm(S @ A - A @ S) <= 1e-12 * k * k * np.linalg.norm(A)
    SS = sf[:, None] * S                       # Sigma S symmetric: S is pseudosymmetric too
    assert np.linalg.norm(SS - SS.T) <= 1e-12 * k * k * n


def test_gsign_two_by_two_closed_form():
    """A = [[a, b], [-b, -c]] (Sigma = diag(1, -1), Sigma A symmetric) with real eigenvalues
    l+ > 0 > l-: P_+ = (A - l- I)/(l+ - l-), so sign(A) = (2A - (l+ + l-) I)/(l+ - l-)."""
    a, b, c = 2.0, 0.75, 1.5
    A = np.array([[a, b], [-b, -c]])
    disc = np.sqrt((a + c) ** 2 - 4 * b * b)
    lp, lm = ((a - c) + disc) / 2, ((a - c) - disc) / 2
    S = O.gsign_def(A)
    assert np.linalg.norm(S - (2 * A - (lp + lm) * np.eye(2)) / (lp - lm)) <= 1e-15 * 4


def test_gsign_on_definite_input_is_the_definite_oracle():
    """On a definite input the definition layer of the general case (general eigensolver)
    and the definite oracle (Cholesky of Sigma A, Jacobi on L^T Sigma L) agree."""
    A, s, _, V = G.general_pseudosym(20, seed=11, definite=True)
    k = np.linalg.cond(V)
    assert np.linalg.norm(O.gsign_def(A) - O.sign_def(A, s)) <= 1e-12 * k * k * 20


def test_gsign_rejects_imaginary_axis():
    A = np.array([[0.0, 1.0], [-1.0, 0.0]])        # eigenvalues +-i, Sigma = I
    with pytest.raises(ValueError):
        O.gsign_def(A)


@pytest.mark.parametrize("n,pairs,seed", CASES)
def test_alg5_bases(n, pairs, seed):
    """Thm. HRisLDL through Alg. 5: Q_+- ^T Sigma Q_+- = Sigma_hat_+-, the projector identity
    P_+- = Q_+- Sigma_hat_+- Q_+-^T Sigma (= H R with H = Sigma R^T Sigma_hat), Q_+^T Sigma Q_- = 0,
    rank = trace, and invariance A Q_+ = Q_+ A11 with the spectrum of A11 the eigenvalues
    of positive real part."""
    A, s, C, V = G.general_pseudosym(n, seed=seed, n_pairs=pairs)
    sf = s.astype(float)
    k = np.linalg.cond(V)
    S = O.gsign_def(A)
    Qp, Qm, sp, sm = O.hyp_basis_ldl(S, s)
    lam = _spectrum_C(C)
    npos = int(np.sum(lam.real > 0))
    assert Qp.shape == (n, npos) and Qm.shape == (n, n - npos)
    tol = 1e-11 * k ** 4 * n
    for Q, sh, sgn in ((Qp, sp, 1.0), (Qm, sm, -1.0)):
        P = 0.5 * (np.eye(n) + sgn * S)
        assert np.linalg.norm(Q.T @ (sf[:, None] * Q) - np.diag(sh)) <= tol
        assert np.linalg.norm(Q @ np.diag(sh) @ Q.T * sf[None, :] - P) <= tol * np.linalg.norm(P)
        Qd = (sh[:, None] * Q.T) * sf[None, :]         # Q^dagger = Sigma_hat Q^T Sigma
        A11 = Qd @ A @ Q
        assert np.linalg.norm(A @ Q - Q @ A11) <= tol * np.linalg.norm(A)
        ev = np.sort_complex(np.linalg.eigvals(A11)) if Q.shape[1] else np.zeros(0)
        ref = np.sort_complex(lam[lam.real > 0] if sgn > 0 else lam[lam.real < 0])
        assert np.max(np.abs(ev - ref), initial=0.0) <= 1e-9 * k * k * np.max(np.abs(lam))
    assert np.linalg.norm(Qp.T @ (sf[:, None] * Qm)) <= tol


def test_alg5_definite_signatures():
    """Thm. DefDivConq: for a definite A the hyperbolic bases are Sigma-orthonormal with
    Sigma_hat_+ = I and Sigma_hat_- = -I, and the blocks are those of the definite split."""
    A, s, _, V = G.general_pseudosym(16, seed=5, definite=True)
    Qp, Qm, sp, sm = O.hyp_basis_ldl(O.gsign_def(A), s)
    assert np.all(sp == 1.0) and np.all(sm == -1.0)
    sf = s.astype(float)
    A11 = Qp.T @ (sf[:, None] * A) @ Qp            # Q_+^dagger A Q_+ with Sigma_hat_+ = I
    assert np.min(np.linalg.eigvalsh(0.5 * (A11 + A11.T))) > 0
    w_ref = np.sort(np.linalg.eigvals(A).real)
    assert np.max(np.abs(np.sort(np.linalg.eigvals(A11).real) - w_ref[w_ref > 0])) <= 1e-10 * np.max(np.abs(w_ref))


@pytest.mark.parametrize("n,pairs,seed", CASES + [(40, 10, 6), (16, 0, 7)])
def test_alg3_full(n, pairs, seed):
    """Alg. 3: V^{-1} A V = D block diagonal (blocks of order <= 2), V^T Sigma V = Sigma_hat,
    one 2 x 2 block per conjugate pair, and D's eigenvalues the constructed spectrum."""
    A, s, C, V0 = G.general_pseudosym(n, seed=seed, n_pairs=pairs)
    sf = s.astype(float)
    k = np.linalg.cond(V0)
    V, sh, D = O.geig_alg(A, s)
    assert set(np.unique(sh)) <= {-1.0, 1.0}
    Vinv = (sh[:, None] * V.T) * sf[None, :]
    kv = np.linalg.cond(V)
    assert np.linalg.norm(Vinv @ V - np.eye(n)) <= 1e-11 * kv * kv * n
    assert np.linalg.norm(Vinv @ A @ V - D) <= 1e-11 * kv * kv * np.linalg.norm(A)
    off = D.copy()
    i = 0
    blocks2 = 0
    while i < n:
        if i + 1 < n and D[i + 1, i] != 0.0:
            off[i:i + 2, i:i + 2] = 0.0
            blocks2 += 1
            i += 2
        else:
            off[i, i] = 0.0
            i += 1
    assert not np.any(off)
    assert blocks2 == pairs
    lam = O.block_eigenvalues(D)
    ref = _spectrum_C(C)
    assert np.max(np.abs(lam - ref)) <= 1e-9 * k * k * np.max(np.abs(ref))


def test_alg3_small_cases():
    # order 1: nothing to split
    V, sh, D = O.geig_alg(np.array([[-2.5]]), [-1])
    assert V.shape == (1, 1) and sh[0] == -1 and D[0, 0] == -2.5
    # order 2 with a conjugate pair: Alg. 3 stops at once
    A = np.array([[1.0, 2.0], [-2.0, 1.0]])        # Sigma = diag(1, -1): Sigma A symmetric
    V, sh, D = O.geig_alg(A, [1, -1])
    assert np.array_equal(V, np.eye(2)) and np.array_equal(D, A)
    lam = O.block_eigenvalues(D)
    assert np.allclose(lam, [1 - 2j, 1 + 2j], rtol=0, atol=1e-15)
    # order 2 with real eigenvalues: split into two 1 x 1 blocks
    A = np.array([[2.0, 0.75], [-0.75, -1.5]])
    V, sh, D = O.geig_alg(A, [1, -1])
    assert D[0, 1] == 0.0 and D[1, 0] == 0.0
    assert np.allclose(np.sort(np.diag(D)), np.sort(np.linalg.eigvals(A).real), rtol=0, atol=1e-14)


def test_alg3_on_definite_input_matches_definite_oracle():
    """On a definite input Alg. 3's eigenvalues are the definite oracle's and every
    eigenvalue's Sigma_hat entry is its sign (Thm. EVRealSigmaOrth)."""
    A, s, _, _ = G.general_pseudosym(18, seed=9, definite=True)
    V, sh, D = O.geig_alg(A, s)
    lam = np.diag(D)
    assert np.all(np.sign(lam) == sh)
    ref, _ = O.eig_def(A, s)
    assert np.max(np.abs(np.sort(lam) - np.sort(ref))) <= 1e-11 * np.max(np.abs(ref))
