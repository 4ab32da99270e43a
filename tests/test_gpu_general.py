"""sign(H) of a general (not necessarily definite) pseudosymmetric H through
pssd_gsign, against the oracle's definition layer (gsign_def: X sign(Re Lambda)
X^{-1}) and against the sign built into the input (A = V C V^{-1}, V^T Sigma V =
Sigma): element by element, the involution, the count of eigenvalues with
positive real part, the definite path on definite inputs, and the status codes.
The iteration inverts W^2 (W = Sigma X), so its error grows like cond(H)^2 u:
the bounds carry that factor."""
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


CASES = [(7, 1, 0, 1.0), (24, 5, 2, 1.0), (64, 10, 12, 1.0), (130, 20, 13, 1.0), (200, 0, 14, 1.0),
         (96, 12, 21, 2.0)]


@pytest.mark.parametrize("precision", ["fp64", "fp64e"])
@pytest.mark.parametrize("n,pairs,seed,spread", CASES)
def test_gsign_matches_oracle(P, precision, n, pairs, seed, spread):
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    A, sg, C, V = G.general_pseudosym(n, seed=seed, n_pairs=pairs, spread=spread)
    s = sg.astype(float)
    S, info = P.gsign(_dev(A), sigma=sg, precision=pr)
    S = S.cpu().numpy()
    S_def = O.gsign_def(A)
    S_con = V @ np.diag(np.sign(np.diag(C))) @ ((s[:, None] * V.T) * s[None, :])
    kap = np.linalg.cond(A)
    tol = 1e-14 * kap * kap
    assert np.linalg.norm(S - S_def) <= tol * np.linalg.norm(S_def)
    assert np.linalg.norm(S - S_con) <= tol * np.linalg.norm(S_con)
    nrm2 = np.linalg.norm(S_def, 2)
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-12 * n * nrm2 ** 2
    assert info["s2_resid"] <= 1e-12 * n * nrm2 ** 2
    SS = s[:, None] * S
    assert np.array_equal(SS, SS.T)                       # Sigma S = W, symmetric by construction
    lam = np.linalg.eigvals(C)
    assert info["p"] == int(np.sum(lam.real > 0))
    assert 1 <= info["iterations"] <= 20


def test_gsign_on_definite_input_is_the_definite_sign(P):
    """On a definite input the general Newton iteration and the Zolotarev path of
    pssd_sign (congruence form) give the same sign."""
    A, sg, _, _ = G.general_pseudosym(120, seed=31, definite=True)
    Hd = _dev(A)
    Sg, ig = P.gsign(Hd, sigma=sg)
    Sz, iz = P.sign(Hd, sigma=sg)
    kap = np.linalg.cond(A)
    assert float(torch.linalg.norm(Sg - Sz)) <= 1e-14 * kap * kap * float(torch.linalg.norm(Sz))
    assert ig["p"] == iz["p"]


def test_gsign_status_codes(P):
    A, sg, _, _ = G.general_pseudosym(16, seed=3, n_pairs=2)
    bad = A.copy(); bad[0, 1] += 1.0                      # Sigma H no longer symmetric
    with pytest.raises(P.PssdError) as e:
        P.gsign(_dev(bad), sigma=sg)
    assert e.value.status == 8
    with pytest.raises(P.PssdError) as e:
        P.gsign(_dev(A), sigma=sg, precision=P.PSSD_MIXED)
    assert e.value.status == -8
    # eigenvalues +-i: W_1 = 0 exactly, the iteration cannot go on
    H = np.array([[0.0, 1.0], [-1.0, 0.0]])
    with pytest.raises(P.PssdError) as e:
        P.gsign(_dev(H), sigma=np.array([1, -1], dtype=np.int8))
    assert e.value.status == 2


@pytest.mark.parametrize("precision", ["fp64", "fp64e"])
def test_gsign_n2048_timed(P, precision):
    """n = 2048 with 200 conjugate pairs: against the constructed sign, timed with CUDA
    events after a warm-up (reported)."""
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    n = 2048
    A, sg, C, V = G.general_pseudosym(n, seed=2048, n_pairs=200)
    s = sg.astype(float)
    Hd = _dev(A)
    P.gsign(Hd, sigma=sg, precision=pr)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    S, info = P.gsign(Hd, sigma=sg, precision=pr)
    e1.record()
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    S_con = V @ np.diag(np.sign(np.diag(C))) @ ((s[:, None] * V.T) * s[None, :])
    kap = np.linalg.cond(A)
    err = np.linalg.norm(S - S_con) / np.linalg.norm(S_con)
    print(f"\ngsign n=2048 {precision}: {e0.elapsed_time(e1):.1f} ms, {info['iterations']} Newton steps, "
          f"rel. error {err:.1e}, ||S^2-I||_F {info['s2_resid']:.1e}, cond(H) {kap:.1e}")
    assert err <= 1e-14 * kap * kap
    assert info["s2_resid"] <= 1e-12 * n * np.linalg.norm(S_con, 2) ** 2
    assert info["p"] == int(np.sum(np.linalg.eigvals(C).real > 0))


@pytest.mark.parametrize("precision", ["fp64", "fp64e"])
@pytest.mark.parametrize("n,pairs,seed,spread", CASES)
def test_gsplit_invariants(P, precision, n, pairs, seed, spread):
    """The division of Alg. 3 through pssd_gsplit.  The basis is not unique; what is:
    p, the inertia of Sigma_hat on each side (Sylvester's law; the oracle's Alg. 5 basis
    gives it), the projector Q_+ Sigma_hat_+ Q_+^T Sigma = (I + S)/2, the spectra of the
    blocks; and Q^T Sigma Q = Sigma_hat, Q^{-1} H Q = diag(A11, A22), Sigma_hat A11
    symmetric hold for any valid basis."""
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    A, sg, C, V = G.general_pseudosym(n, seed=seed, n_pairs=pairs, spread=spread)
    s = sg.astype(float)
    Qd, A11, A22, sh, p, info = P.gsplit(_dev(A), sigma=sg, precision=pr)
    Q, A11, A22 = Qd.cpu().numpy(), A11.cpu().numpy(), A22.cpu().numpy()
    shf = sh.astype(float)
    lam = np.linalg.eigvals(C)
    assert p == int(np.sum(lam.real > 0))
    assert set(np.unique(sh)) <= {-1, 1}
    S_def = O.gsign_def(A)
    _, _, sp_o, sm_o = O.hyp_basis_ldl(S_def, s)
    assert np.sum(shf[:p] > 0) == np.sum(sp_o > 0) and np.sum(shf[p:] > 0) == np.sum(sm_o > 0)
    kap, kq = np.linalg.cond(A), np.linalg.cond(Q)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ (s[:, None] * Q) - np.diag(shf)) <= 1e-13 * n * kq * kq
    Pp = 0.5 * (np.eye(n) + S_def)
    Qp = Q[:, :p]
    assert np.linalg.norm(Qp @ np.diag(shf[:p]) @ Qp.T * s[None, :] - Pp) <= 1e-14 * kap * kap * np.linalg.norm(Pp)
    B = ((shf[:, None] * Q.T) * s[None, :]) @ A @ Q
    assert np.linalg.norm(B[:p, :p] - A11) <= 1e-13 * kq * kq * nA
    assert np.linalg.norm(B[p:, p:] - A22) <= 1e-13 * kq * kq * nA
    assert np.linalg.norm(B[:p, p:]) <= 1e-14 * kap * kap * kq * kq * nA
    if 0 < p < n:
        assert info["split_backerr"] <= 1e-14 * kap * kap * kq * kq
    for Ab, sb in ((A11, shf[:p]), (A22, shf[p:])):
        if Ab.size:
            SA = sb[:, None] * Ab
            assert np.linalg.norm(SA - SA.T) <= 1e-13 * kq * kq * nA
    scale = np.max(np.abs(lam))
    if p:
        ev, ref = np.sort_complex(np.linalg.eigvals(A11)), np.sort_complex(lam[lam.real > 0])
        assert np.max(np.abs(ev - ref)) <= 1e-10 * kap * scale
    if n - p:
        ev, ref = np.sort_complex(np.linalg.eigvals(A22)), np.sort_complex(lam[lam.real < 0])
        assert np.max(np.abs(ev - ref)) <= 1e-10 * kap * scale


def test_gsplit_definite_signatures(P):
    """Thm. DefDivConq through the general division: on a definite input Sigma_hat_+ = I,
    Sigma_hat_- = -I, A11 symmetric positive definite, A22 symmetric negative definite."""
    A, sg, _, _ = G.general_pseudosym(100, seed=41, definite=True)
    Qd, A11, A22, sh, p, info = P.gsplit(_dev(A), sigma=sg)
    assert np.all(sh[:p] == 1) and np.all(sh[p:] == -1)
    A11, A22 = A11.cpu().numpy(), A22.cpu().numpy()
    assert np.linalg.norm(A11 - A11.T) <= 1e-12 * np.linalg.norm(A11)
    assert np.min(np.linalg.eigvalsh(0.5 * (A11 + A11.T))) > 0
    assert np.max(np.linalg.eigvalsh(0.5 * (A22 + A22.T))) < 0
