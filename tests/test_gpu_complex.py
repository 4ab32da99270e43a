"""Complex pseudo-Hermitian matrices (the BSE forms, Eqs. BSE1 and BSE2) through
pssd_zsign / pssd_zeig, against the oracle's native complex definition layer
(scalar complex Cholesky and Jacobi): sign element by element, eigenvalues one by
one, eigenvectors (phase-fixed on both sides) where the eigenvalues are separated,
spectral projectors where they repeat, and the residuals the method fixes."""
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _sig(n):
    return np.r_[np.ones(n // 2), -np.ones(n // 2)]


CASES = [("bse1", 20, "fp64"), ("bse2", 30, "fp64"), ("bse1", 33, "fp64e"), ("bse2", 48, "fp64e")]


def _make(form, k, seed):
    if form == "bse1":
        return G.bse1(k, ("uniform", 1.0, 10.0), seed=seed)
    return G.bse2(k, ("loguniform", 0.1, 10.0), seed=seed)[0]


@pytest.mark.parametrize("form,k,precision", CASES)
def test_zsign_matches_oracle(P, form, k, precision):
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    H = _make(form, k, 700 + k)
    n = 2 * k
    S, info = P.zsign(_dev(H), precision=pr)
    S = S.cpu().numpy()
    Sref = O.zsign_def(H)
    nrm2 = np.linalg.norm(Sref, 2)
    assert np.linalg.norm(S - Sref) <= 1e-10 * np.linalg.norm(Sref) * nrm2
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-12 * n * nrm2 ** 2
    s = _sig(n)
    SS = s[:, None] * S
    assert np.linalg.norm(SS - SS.conj().T) <= 1e-12 * n * nrm2
    assert info["p"] == k


@pytest.mark.parametrize("form,k,precision", CASES)
def test_zeig_matches_oracle(P, form, k, precision):
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    H = _make(form, k, 800 + k)
    n = 2 * k
    D, V, info = P.zeig(_dev(H), precision=pr)
    D = D.cpu().numpy(); V = V.cpu().numpy()
    lam, Vref = O.zeig_def(H)
    nrm = np.max(np.abs(lam))
    assert np.max(np.abs(D - lam)) <= 1e-10 * nrm
    assert np.linalg.norm(H @ V - V * D) <= 1e-12 * np.linalg.norm(H)
    s = _sig(n)
    assert np.linalg.norm(V.conj().T @ (s[:, None] * V) - np.diag(np.sign(D))) <= 1e-12 * n * np.linalg.norm(V, 2) ** 2
    gaps = np.abs(np.diff(np.sort(lam)))
    if np.min(gaps) > 1e-6 * nrm:
        assert np.max(np.abs(V - Vref)) <= 1e-7 * np.max(np.abs(Vref))


@pytest.mark.parametrize("values,mult", [((0.4, 1.0, 2.5, 4.0, 7.0), 6), ((0.8, 3.0), 36)])
def test_zeig_repeated_eigenvalues(P, values, mult):
    """BSE2 with Q1 = Q2 and d1 d2 taking a few values, each `mult` times: lambda = +-omega
    with that multiplicity (groups of 2 mult real values; 72 > 64 takes the recursive
    symmetric eigensolver for the group's Gram matrix); each eigenvalue's spectral projector
    V_g sign(lambda) V_g^H Sigma against the oracle's (unique, unlike the basis)."""
    om = np.repeat(np.array(values), mult)
    k = len(om)
    rng = np.random.default_rng(9)
    d1 = np.exp(rng.uniform(np.log(0.5), np.log(2.0), k)) * om
    d2 = om * om / d1
    A, B = G.bse2_blocks(k, d1, d2, rng, same_q=True)
    H = np.block([[A, B], [-B, -A]])
    n = 2 * k
    s = _sig(n)
    lam, Vref = O.zeig_def(H)
    for pr in (P.PSSD_FP64, P.PSSD_FP64_EMULATED):
        D, V, _ = P.zeig(_dev(H), precision=pr)
        D = D.cpu().numpy(); V = V.cpu().numpy()
        assert np.max(np.abs(D - lam)) <= 1e-12 * om.max()
        assert np.linalg.norm(H @ V - V * D) <= 1e-12 * np.linalg.norm(H)
        assert np.linalg.norm(V.conj().T @ (s[:, None] * V) - np.diag(np.sign(D))) <= 1e-11 * n
        for v in np.unique(np.round(lam, 9)):
            g = np.abs(D - v) <= 1e-8 * om.max()
            gr = np.abs(lam - v) <= 1e-8 * om.max()
            assert g.sum() == gr.sum() == mult
            sg = np.sign(v)
            Pg = sg * (V[:, g] @ V[:, g].conj().T) * s[None, :]
            Pr = sg * (Vref[:, gr] @ Vref[:, gr].conj().T) * s[None, :]
            assert np.linalg.norm(Pg - Pr) <= 1e-10 * np.linalg.norm(Pr)


def test_complex_status_codes(P):
    H = G.bse1(6, seed=1)
    bad = H.copy(); bad[0, 1] += 1.0          # Sigma H no longer Hermitian
    with pytest.raises(P.PssdError) as e:
        P.zsign(_dev(bad))
    assert e.value.status == 8                 # PSSD_ERR_NOT_PSEUDOSYMMETRIC
    with pytest.raises(ValueError):
        P.zsign(_dev(H.real.copy()))           # float64, not complex128


def test_bse1_example3_size(P):
    """The size of the paper's Example 3 (complex BSE, n = 2560) on a synthetic BSE1
    input: residual and Sigma-orthogonality of the full diagonalisation, FP64-emulated."""
    import time
    k = 1280
    n = 2 * k
    H = G.bse1(k, ("uniform", 1.0, 10.0), seed=2560)
    Hd = _dev(H)
    torch.cuda.synchronize(); t0 = time.time()
    D, V, info = P.zeig(Hd, precision=P.PSSD_FP64_EMULATED)
    torch.cuda.synchronize(); t1 = time.time()
    R = Hd @ V - V * D[None, :].to(V.dtype)
    res = float(torch.linalg.norm(R) / torch.linalg.norm(Hd))
    s = torch.from_numpy(_sig(n)).cuda().to(V.dtype)
    orth = float(torch.linalg.norm(V.conj().T @ (s[:, None] * V) - torch.diag(torch.sign(D)).to(V.dtype)))
    pair = float(torch.max(torch.abs(D[:k] + D[k:])) / torch.max(torch.abs(D)))
    print(f"\nBSE1 n=2560 fp64e: {t1 - t0:.2f} s, ||HV-VD||/||H|| {res:.2e}, V^H Sigma V defect {orth:.2e}, "
          f"+-pairing {pair:.2e}, levels {info['levels']}")
    assert res <= 1e-11
    assert orth <= 1e-12 * n
    assert pair <= 1e-12
