"""Boundary features of the C ABI: a precomputed S passed to pssd_split, the
commutator residual ||SH - HS||_F / ||H||_F reported beside ||S^2 - I||
(Lemma SignProj), and the bounded pipeline waits of the tensor-core kernels
(pssd_opts.wait_cycles)."""
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


def _dev(H):
    return torch.from_numpy(np.ascontiguousarray(H)).cuda()


def _J(n):
    return np.r_[np.ones(n // 2), -np.ones(n // 2)]


@pytest.mark.parametrize("precision", ["fp64", "fp64e"])
def test_split_with_precomputed_sign(P, precision):
    """pssd_split(S = sign(H) from pssd_sign) gives the same spectral projector
    and the same blocks' spectra as pssd_split computing S itself (the basis
    within each invariant subspace is not unique; the projector and the
    spectra are)."""
    prec = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    H, _, _ = G.casida(90, ("loguniform", 1e-2, 1e2), seed=91)
    n = H.shape[0]
    J = _J(n)
    Hd = _dev(H)
    S, _ = P.sign(Hd, precision=prec)
    Q1, A1, B1, p1, i1 = P.split(Hd, precision=prec, S=S)
    Q0, A0, B0, p0, i0 = P.split(Hd, precision=prec)
    assert p1 == p0 == n // 2
    Q1 = Q1.cpu().numpy(); Q0 = Q0.cpu().numpy()
    P1 = Q1[:, :p1] @ Q1[:, :p1].T * J[None, :]
    P0 = Q0[:, :p0] @ Q0[:, :p0].T * J[None, :]
    Pref = 0.5 * (np.eye(n) + O.sign_def(H))
    assert np.linalg.norm(P1 - P0) <= 1e-10 * np.linalg.norm(Pref) * np.linalg.norm(Pref, 2)
    lam, _ = O.eig_def(H)
    nrm = np.max(np.abs(lam))
    for A, ref in ((A1, lam[:p1]), (A0, lam[:p0])):
        assert np.max(np.abs(np.sort(np.linalg.eigvalsh(A.cpu().numpy())) - ref)) <= 1e-10 * nrm
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(B1.cpu().numpy()))[::-1] - lam[p1:])) <= 1e-10 * nrm
    # S enters in H's coordinates and is mapped to K's by L^T S L^{-T}, which multiplies its
    # rounding error by up to kappa(L) = kappa(M)^(1/2) (about 1e2 here): 10x the internal path's bound
    assert 0 <= i1["split_backerr"] <= 1e-11
    assert 0 <= i1["comm_resid"] <= 1e-11 * np.linalg.norm(Pref, 2)   # ~ ||S||_2 for the non-normal S


def test_split_with_an_approximate_sign_reports_its_defect(P):
    """A perturbed S is used as given: its defect shows up in the reported
    backward error and commutator instead of being silently corrected."""
    H, _, _ = G.casida(60, ("uniform", 1.0, 10.0), seed=61)
    Hd = _dev(H)
    S, _ = P.sign(Hd)
    g = torch.Generator(device="cuda"); g.manual_seed(3)
    E = torch.randn(S.shape, dtype=S.dtype, device=S.device, generator=g)
    Sp = S + 1e-6 * E / torch.linalg.norm(E) * torch.linalg.norm(S)
    _, _, _, _, info = P.split(Hd, S=Sp, flags=P.FLAG_RESIDUALS)
    assert info["split_backerr"] > 1e-9
    assert info["comm_resid"] > 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp64e", "mixed"])
def test_commutator_is_reported_and_estimate_tracks_exact(P, precision):
    prec = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED, "mixed": P.PSSD_MIXED}[precision]
    H, _, _ = G.casida(100, ("loguniform", 1e-2, 1e2), seed=101)
    n = H.shape[0]
    Hd = _dev(H)
    S, est = P.sign(Hd, precision=prec)
    _, ex = P.sign(Hd, precision=prec, flags=P.FLAG_RESIDUALS)
    Sn = S.cpu().numpy()
    direct = np.linalg.norm(Sn @ H - H @ Sn) / np.linalg.norm(H)
    assert ex["comm_resid"] > 0 and est["comm_resid"] > 0
    assert abs(ex["comm_resid"] - direct) <= 0.05 * direct + 1e-15
    # chi-square(16) ratio within [1/3, 3] except with probability < 1e-3
    assert ex["comm_resid"] / 3 <= est["comm_resid"] <= 3 * ex["comm_resid"]
    if precision != "mixed":
        assert ex["comm_resid"] <= 1e-11 * max(1.0, np.linalg.norm(Sn, 2))
    for fn in ("split", "eig"):
        out = getattr(P, fn)(Hd, precision=prec)
        assert out[-1]["comm_resid"] > 0


@pytest.mark.parametrize("precision", ["fp64e", "mixed"])
def test_tensor_core_wait_bound_returns_timeout(P, precision):
    """A one-poll bound on every pipeline wait of the tensor-core kernels makes
    the waits run out (the copies cannot land within one poll).  The kernels
    then stop, let their own copies and products in flight finish under the
    fixed drain bound, free their tensor memory and return; the call reports
    PSSD_ERR_TIMEOUT.  The same handle then solves the problem normally."""
    prec = {"fp64e": P.PSSD_FP64_EMULATED, "mixed": P.PSSD_MIXED}[precision]
    H, _, _ = G.casida(128, ("uniform", 1.0, 10.0), seed=129)    # n = 256: tensor-core products
    Hd = _dev(H)
    h = P.Handle()
    with pytest.raises(P.PssdError) as ei:
        P.sign(Hd, handle=h, precision=prec, wait_cycles=1)
    assert ei.value.status == 5
    S, info = P.sign(Hd, handle=h, precision=prec)
    Sd = O.sign_def(H)
    tol = 1e-10 if precision == "fp64e" else 1e-3
    assert np.linalg.norm(S.cpu().numpy() - Sd) <= tol * np.linalg.norm(Sd) * np.linalg.norm(Sd, 2)
    torch.cuda.synchronize()
