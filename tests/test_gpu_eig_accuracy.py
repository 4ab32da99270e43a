"""Accuracy of the diagonalisation beyond parity with the oracle.

* The final refinement step (one Ogita-Aishima correction of the symmetric
  eigendecomposition) against Alg. 2's recursion alone.
* Repeated eigenvalues: the basis of a multiple eigenvalue's eigenspace is not
  unique, its spectral projector is (Eq. signDef's V Sigma_hat V^{-1} restricted
  to the eigenvalue), so the test compares projectors with the oracle's and
  checks the rest (residual, Sigma-orthogonality) directly.
* The batched entry point in the mixed precision (FP32 Zolotarev steps, FP64
  split and recursion, refinement against the FP64 K)."""
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


def _sym(w, seed):
    m = len(w)
    Q = G.haar(np.random.default_rng(seed), m)
    B = (Q * w[None, :]) @ Q.T
    return 0.5 * (B + B.T)


def _J(n, k):
    return np.r_[np.ones(k), -np.ones(n - k)]


@pytest.mark.parametrize("precision", ["fp64", "fp64e"])
def test_refinement_step(P, precision):
    """m = 1024, eigenvalues log-uniform in [1e-2, 1e2].  Alg. 2 alone leaves a
    residual set by the sign iterations (about 1e-13 relative here); one
    refinement step brings ||B W - W diag(w)||_F / ||B||_F to a few hundred
    units of rounding (<= 2e-14) and ||W^T W - I||_F to <= 2e-13."""
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    m = 1024
    w0 = np.exp(np.random.default_rng(21).uniform(np.log(1e-2), np.log(1e2), m))
    B = _sym(w0, 22)
    Bd = torch.from_numpy(B).cuda()
    I = torch.eye(m, dtype=torch.float64, device="cuda")
    out = {}
    for fl in (P.FLAG_NO_REFINE, 0):
        w, W, _ = P.test_sym_eig(Bd, precision=pr, flags=fl)
        res = float(torch.linalg.norm(Bd @ W - W * w[None, :]) / torch.linalg.norm(Bd))
        orth = float(torch.linalg.norm(W.T @ W - I))
        ev = float(np.max(np.abs(np.sort(w.cpu().numpy()) - np.sort(w0))) / w0.max())
        out[fl] = (res, orth, ev)
    print(f"\nrefinement {precision}: without {out[P.FLAG_NO_REFINE]}  with {out[0]}")
    assert out[P.FLAG_NO_REFINE][0] <= 1e-11
    assert out[0][0] <= 2e-14
    assert out[0][1] <= 2e-13
    assert out[0][2] <= 1e-14


def test_repeated_eigenvalues_symmetric(P):
    """Six distinct eigenvalues, five of multiplicity 100 (above the Jacobi leaf
    order, so the recursion meets blocks that equal sigma I to rounding) and one
    of multiplicity 60: eigenvalues exact to rounding, each eigenspace's
    orthogonal projector W_g W_g^T equal to the one from the definition."""
    vals = np.array([-3.0, -1.0, 0.5, 2.0, 7.0, 11.0])
    mult = np.array([100, 100, 100, 100, 100, 60])
    w0 = np.repeat(vals, mult)
    B = _sym(w0, 31)
    Bd = torch.from_numpy(B).cuda()
    m = len(w0)
    for pr in (P.PSSD_FP64, P.PSSD_FP64_EMULATED):
        w, W, _ = P.test_sym_eig(Bd, precision=pr)
        w = w.cpu().numpy(); W = W.cpu().numpy()
        assert np.max(np.abs(np.sort(w) - w0)) <= 1e-13 * 11.0
        assert np.linalg.norm(B @ W - W * w[None, :]) <= 1e-13 * np.linalg.norm(B)
        assert np.linalg.norm(W.T @ W - np.eye(m)) <= 1e-12
        Q = G.haar(np.random.default_rng(31), m)          # the eigenvectors B was built from
        for v in vals:
            g = np.abs(w - v) <= 1e-9
            assert g.sum() == mult[vals == v][0]
            Pg = W[:, g] @ W[:, g].T
            Qg = Q[:, w0 == v]
            assert np.linalg.norm(Pg - Qg @ Qg.T) <= 1e-11 * np.sqrt(g.sum())


def test_repeated_eigenvalues_pseudosymmetric(P):
    """Casida form with Q1 = Q2 and d1 d2 taking 8 values, each 25 times (k = 200):
    lambda = +-sqrt(d1 d2) with multiplicity 25; against the oracle's
    eigendecomposition through each eigenvalue's spectral projector
    V_g Sigma_hat_g V_g^T Sigma, which is unique."""
    k = 200
    rng = np.random.default_rng(41)
    om = np.repeat(np.array([0.3, 0.7, 1.1, 2.0, 3.5, 5.0, 8.0, 13.0]), 25)
    d1 = np.exp(rng.uniform(np.log(0.5), np.log(2.0), k)) * om
    d2 = om * om / d1
    A, Bm = G.casida_blocks(k, d1, d2, rng, same_q=True)
    H = np.block([[A, Bm], [-Bm, -A]])
    n = 2 * k
    J = _J(n, k)
    lam, Vref = O.eig_def(H)
    for pr in (P.PSSD_FP64, P.PSSD_FP64_EMULATED):
        D, V, info = P.eig(torch.from_numpy(H).cuda(), precision=pr)
        D = D.cpu().numpy(); V = V.cpu().numpy()
        assert np.max(np.abs(D - lam)) <= 1e-12 * om.max()
        assert np.linalg.norm(H @ V - V * D) <= 1e-12 * np.linalg.norm(H)
        assert np.linalg.norm(V.T @ (J[:, None] * V) - np.diag(np.sign(D))) <= 1e-12 * n * np.linalg.norm(V, 2) ** 2
        for v in np.unique(np.round(lam, 9)):
            g = np.abs(D - v) <= 1e-8 * om.max()
            gr = np.abs(lam - v) <= 1e-8 * om.max()
            assert g.sum() == gr.sum() == 25
            s = np.sign(v)
            Pg = s * (V[:, g] @ V[:, g].T) * J[None, :]
            Pr = s * (Vref[:, gr] @ Vref[:, gr].T) * J[None, :]
            assert np.linalg.norm(Pg - Pr) <= 1e-10 * np.linalg.norm(Pr)


def test_batched_mixed_precision(P):
    """pssd_eig_batched with FP32 Zolotarev steps: the split then runs on an FP32-accurate
    sign, the recursion and the refinement on the FP64 K, so eigenvalues and residual land
    near FP64 accuracy (bounds 1e-9 and 1e-10 relative); p and the eigenvalue signs exact."""
    ks = [40, 100, 7, 64, 130]
    Hn = [G.casida(k, ("uniform", 0.5, 50.0), seed=900 + i)[0] for i, k in enumerate(ks)]
    Hs = [torch.from_numpy(x).cuda() for x in Hn]
    Ds, Vs, infos = P.eig_batched(Hs, precision=P.PSSD_MIXED)
    for H, D, V, info, k in zip(Hn, Ds, Vs, infos, ks):
        lam, _ = O.eig_def(H)
        D = D.cpu().numpy(); V = V.cpu().numpy()
        err = np.max(np.abs(D - lam)) / np.max(np.abs(lam))
        res = np.linalg.norm(H @ V - V * D) / np.linalg.norm(H)
        print(f"\nbatched mixed k={k}: eig err {err:.2e} residual {res:.2e}")
        assert info["p"] == k
        assert np.array_equal(np.sign(D), np.sign(lam))
        assert err <= 1e-9
        assert res <= 1e-10
