"""Structure-aware Casida entry points (pssd_casida_sign / _split / _eig): the
k x k polar-factor formulation against the oracle's k x k Jacobi reduction
(casida_eig_def, itself pinned to the n x n definition and closed forms), the
n x n library path, and the method's invariants, in FP64 and FP64-emulated
arithmetic.  Tolerances are those of the n x n parity tests."""
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


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _blocks(H):
    k = H.shape[0] // 2
    return H[:k, :k].copy(), H[:k, k:].copy()


CASES = [(1, ("uniform", 1.0, 10.0)), (33, ("uniform", 1.0, 10.0)), (64, ("uniform", 0.1, 100.0)),
         (97, ("loguniform", 1e-2, 1e2)), (160, ("uniform", 1.0, 10.0))]
PRECS = ["fp64", "fp64e"]


def _prec(P, name):
    return {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[name]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("k,dist", CASES)
def test_casida_sign_matches_oracle(P, k, dist, precision):
    H, _, _ = G.casida(k, dist, seed=700 + k)
    A, B = _blocks(H)
    n = 2 * k
    alpha, beta = O.estimate_bounds(H)
    S, info = P.casida_sign(_dev(A), _dev(B), precision=_prec(P, precision), alpha=alpha, beta=beta)
    S = S.cpu().numpy()
    Sd = O.casida_sign_def(A, B)
    nrm2 = max(1.0, np.linalg.norm(Sd, 2))
    assert np.linalg.norm(S - Sd) <= 1e-11 * np.linalg.norm(Sd) * nrm2
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-12 * n * nrm2 ** 2
    J = np.r_[np.ones(k), -np.ones(k)]
    JS = J[:, None] * S
    assert np.linalg.norm(JS - JS.T) <= 1e-12 * np.linalg.norm(S) * nrm2 ** 2
    # same degree as Alg. 8 on the n x n congruence form (same bounds, same rule)
    _, oinfo = O.sign_alg(H, alpha=alpha, beta=beta)
    assert info["r_used"][0] == oinfo["r"][0]
    assert 0 <= info["comm_resid"] <= 1e-11 * nrm2


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("k,dist", [(40, ("uniform", 0.1, 100.0)), (150, ("loguniform", 1e-2, 1e2))])
def test_casida_split_matches_oracle(P, k, dist, precision):
    H, _, _ = G.casida(k, dist, seed=800 + k)
    A, B = _blocks(H)
    n = 2 * k
    J = np.r_[np.ones(k), -np.ones(k)]
    Q, A11, A22, p, info = P.casida_split(_dev(A), _dev(B), precision=_prec(P, precision),
                                          flags=P.FLAG_RESIDUALS)
    Q = Q.cpu().numpy(); A11 = A11.cpu().numpy(); A22 = A22.cpu().numpy()
    assert p == k
    Qp, Qm = Q[:, :k], Q[:, k:]
    assert np.linalg.norm(Q.T @ (J[:, None] * Q) - np.diag(J)) <= 1e-12 * n * np.linalg.norm(Q, 2) ** 2
    Pp = Qp @ Qp.T * J[None, :]
    Pref = 0.5 * (np.eye(n) + O.casida_sign_def(A, B))
    assert np.linalg.norm(Pp - Pref) <= 1e-10 * np.linalg.norm(Pref) * np.linalg.norm(Pref, 2)
    lam, _ = O.casida_eig_def(A, B)
    nrm = np.max(np.abs(lam))
    assert np.min(np.linalg.eigvalsh(A11)) > 0
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(A11)) - lam[:k])) <= 1e-10 * nrm
    assert np.max(np.abs(A22 + A11)) == 0.0
    M = J[:, None] * H
    assert np.linalg.norm(A11 - Qp.T @ M @ Qp) <= 1e-10 * np.linalg.norm(A11)
    assert np.linalg.norm(Qp.T @ M @ Qm) / np.linalg.norm(H) <= 1e-11
    assert 0 <= info["split_backerr"] <= 1e-12
    assert 0 <= info["comm_resid"] <= 1e-11 * np.linalg.norm(Pref, 2)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("k,dist", [(20, ("uniform", 1.0, 10.0)), (100, ("uniform", 0.1, 100.0)),
                                    (200, ("loguniform", 1e-2, 1e2))])
def test_casida_eig_matches_oracle(P, k, dist, precision):
    H, _, _ = G.casida(k, dist, seed=900 + k)
    A, B = _blocks(H)
    n = 2 * k
    J = np.r_[np.ones(k), -np.ones(k)]
    D, V, info = P.casida_eig(_dev(A), _dev(B), precision=_prec(P, precision))
    D = D.cpu().numpy(); V = V.cpu().numpy()
    lam, Vd = O.casida_eig_def(A, B)
    nrmH2 = np.max(np.abs(lam))
    assert np.max(np.abs(D - lam)) <= 1e-10 * nrmH2
    assert np.array_equal(D[k:], -D[:k])                      # exact +- pairing by construction
    assert np.linalg.norm(H @ V - V * D[None, :]) <= 1e-11 * np.linalg.norm(H) * max(1.0, np.linalg.norm(V, 2))
    assert np.linalg.norm(V.T @ (J[:, None] * V) - np.diag(np.sign(D))) <= 1e-12 * n * np.linalg.norm(V, 2) ** 2
    # eigenvectors agree with the oracle's where the eigenvalue is well separated
    gaps = np.minimum(np.abs(np.diff(np.r_[-np.inf, lam[:k]])), np.abs(np.diff(np.r_[lam[:k], np.inf])))
    sep = np.where(gaps > 1e-3 * nrmH2)[0]
    assert np.linalg.norm(V[:, sep] - Vd[:, sep]) <= 1e-8 * np.linalg.norm(Vd[:, sep])
    assert info["levels"] >= 1


def test_casida_matches_n_by_n_path(P):
    """The structure-aware split and the n x n split give the same projector and
    blocks' spectra on the same H."""
    H, _, _ = G.casida(128, ("loguniform", 1e-2, 1e2), seed=4)
    A, B = _blocks(H)
    J = np.r_[np.ones(128), -np.ones(128)]
    Q1, A1, _, _, _ = P.casida_split(_dev(A), _dev(B))
    Q2, A2, _, _, _ = P.split(_dev(H))
    Q1 = Q1.cpu().numpy(); Q2 = Q2.cpu().numpy()
    P1 = Q1[:, :128] @ Q1[:, :128].T * J[None, :]
    P2 = Q2[:, :128] @ Q2[:, :128].T * J[None, :]
    assert np.linalg.norm(P1 - P2) <= 1e-10 * np.linalg.norm(P2) * np.linalg.norm(P2, 2)
    e1 = np.sort(np.linalg.eigvalsh(A1.cpu().numpy())); e2 = np.sort(np.linalg.eigvalsh(A2.cpu().numpy()))
    assert np.max(np.abs(e1 - e2)) <= 1e-10 * e2[-1]


def test_casida_status_codes(P):
    H, _, _ = G.casida(20, ("uniform", 1.0, 10.0), seed=1)
    A, B = _blocks(H)
    A2 = A.copy(); A2[0, 1] += 1e-3                      # A not symmetric
    with pytest.raises(P.PssdError) as e:
        P.casida_sign(_dev(A2), _dev(B))
    assert e.value.status == 8
    with pytest.raises(P.PssdError) as e:                # A - B indefinite: H not definite
        P.casida_sign(_dev(A), _dev(A + 2 * np.eye(20)))
    assert e.value.status == 1
    with pytest.raises(P.PssdError) as e:                # mixed precision is not offered here
        P.casida_sign(_dev(A), _dev(B), precision=P.PSSD_MIXED)
    assert e.value.status == -9
