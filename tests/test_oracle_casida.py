"""The oracle's block-level (k x k) eigendecomposition of the Casida form,
pinned against the n x n definition (a different reduction: K = L^T Sigma L
of Sigma H) and against closed forms: Q1 = Q2 gives the spectrum
+-sqrt(d1_i d2_i) exactly, B = 0 gives +-eig(A), k = 1 gives +-sqrt(a^2 - b^2)."""
import math

import numpy as np
import pytest

import casida_inputs as G
import oracle as O


def _blocks(H):
    k = H.shape[0] // 2
    return H[:k, :k].copy(), H[:k, k:].copy()


@pytest.mark.parametrize("k,dist", [(1, ("uniform", 1.0, 10.0)), (7, ("uniform", 0.1, 100.0)),
                                    (40, ("loguniform", 1e-2, 1e2))])
def test_block_reduction_matches_the_n_by_n_definition(k, dist):
    H, _, _ = G.casida(k, dist, seed=30 + k)
    A, B = _blocks(H)
    lam, V = O.casida_eig_def(A, B)
    lam2, V2 = O.eig_def(H)
    nrm = np.max(np.abs(lam2))
    assert np.max(np.abs(lam - lam2)) <= 1e-12 * nrm
    n = 2 * k
    J = np.r_[np.ones(k), -np.ones(k)]
    assert np.linalg.norm(H @ V - V * lam[None, :]) <= 1e-12 * np.linalg.norm(H) * np.linalg.norm(V)
    assert np.linalg.norm(V.T @ (J[:, None] * V) - np.diag(np.sign(lam))) <= 1e-12 * n * np.linalg.norm(V, 2) ** 2
    S = O.casida_sign_def(A, B)
    Sd = O.sign_def(H)
    assert np.linalg.norm(S - Sd) <= 1e-11 * np.linalg.norm(Sd) * np.linalg.norm(Sd, 2)


def test_same_q_closed_form():
    k = 30
    H, d1, d2 = G.casida(k, ("loguniform", 1e-2, 1e2), seed=5, same_q=True)
    A, B = _blocks(H)
    lam, _ = O.casida_eig_def(A, B)
    ref = np.sort(np.sqrt(d1 * d2))
    assert np.max(np.abs(lam[:k] - ref)) <= 1e-12 * ref[-1]
    assert np.max(np.abs(lam[k:] + ref)) <= 1e-12 * ref[-1]


def test_b_zero_and_k1():
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    d = rng.uniform(1, 5, 6)
    A = (Q * d) @ Q.T
    lam, _ = O.casida_eig_def(A, np.zeros((6, 6)))
    assert np.allclose(lam[:6], np.sort(d), rtol=1e-13)
    assert np.allclose(lam[6:], -np.sort(d), rtol=1e-13)
    a, b = 3.0, 1.25
    lam, V = O.casida_eig_def(np.array([[a]]), np.array([[b]]))
    assert abs(lam[0] - math.sqrt(a * a - b * b)) <= 1e-15 * a and abs(lam[1] + lam[0]) <= 1e-15 * a
