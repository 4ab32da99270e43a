"""Adjoint of the sign function and of the eigenvalues (pssd_sign_vjp, the
step-reversal pssd_sign_vjp_rev and the torch.autograd wrappers), checked against
the oracle's block-sign reference (Newton iteration on [[H^T, G], [0, H^T]]), the
closed form d(sum of positive eigenvalues)/dH = P_+^T, and central finite
differences (h = 1e-6) along structure-preserving perturbations
dH = [[dA, dB], [-dB, -dA]].  The step-reversal adjoint differentiates the
computed function of sym(Sigma H), so it is compared with the reference projected
onto pseudosymmetric matrices, X -> Sigma sym(Sigma X)."""
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


def _loss_grad_ref(H, Gm):
    """<G, S> + sum of positive eigenvalues: block-sign reference + P_+^T."""
    S = O.sign_def(H)
    return O.sign_vjp_block(H, Gm) + 0.5 * (np.eye(H.shape[0]) + S).T


@pytest.mark.parametrize("k,dist", [(16, ("uniform", 1.0, 10.0)), (48, ("loguniform", 1e-1, 1e1))])
def test_vjp_matches_block_sign_reference(P, k, dist):
    H, _, _ = G.casida(k, dist, seed=600 + k)
    n = 2 * k
    rng = np.random.default_rng(1)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    lamb = torch.zeros(n, dtype=torch.float64, device="cuda"); lamb[:k] = 1.0   # positives come first
    Hbar = P.sign_vjp(_dev(H), _dev(Gm), lambar=lamb).cpu().numpy()
    ref = _loss_grad_ref(H, Gm)
    assert np.linalg.norm(Hbar - ref) <= 1e-8 * np.linalg.norm(ref)


def test_autograd_and_finite_differences(P):
    H, _, _ = G.casida(32, ("uniform", 1.0, 10.0), seed=5)
    n = 64
    rng = np.random.default_rng(2)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    Ht = _dev(H).requires_grad_(True)
    Gt = _dev(Gm)
    S = P.SignFn.apply(Ht, None, "spectral")
    D = P.EigvalsFn.apply(Ht)
    loss = (Gt * S).sum() + D[D > 0].sum()
    loss.backward()
    grad = Ht.grad.cpu().numpy()
    ref = _loss_grad_ref(H, Gm)
    assert np.linalg.norm(grad - ref) <= 1e-8 * np.linalg.norm(ref)

    def f(Hn):
        Hd = _dev(Hn)
        Sx, _ = P.sign(Hd)
        Dx, _, _ = P.eig(Hd)
        return float((Gt * Sx).sum() + Dx[Dx > 0].sum())

    k = 32
    for _ in range(4):
        dA = rng.standard_normal((k, k)); dA = dA + dA.T
        dB = rng.standard_normal((k, k)); dB = dB + dB.T
        dH = np.block([[dA, dB], [-dB, -dA]])
        hh = 1e-6
        fd = (f(H + hh * dH) - f(H - hh * dH)) / (2 * hh)
        an = float(np.sum(grad * dH))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_gradient_n2048_finite_differences(P):
    """n = 2048, d ~ U[1,10]: loss <G,S> + sum of positive eigenvalues, G symmetric
    N(0,1); central differences along 16 structure-preserving directions."""
    k = 1024
    n = 2 * k
    H, _, _ = G.casida(k, ("uniform", 1.0, 10.0), seed=2048)
    rng = np.random.default_rng(3)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    Hd = _dev(H); Gt = _dev(Gm)
    lamb = torch.zeros(n, dtype=torch.float64, device="cuda"); lamb[:k] = 1.0
    grad = P.sign_vjp(Hd, Gt, lambar=lamb)

    def f(Hx):
        Sx, _ = P.sign(Hx)
        Dx, _, _ = P.eig(Hx)
        return float((Gt * Sx).sum() + Dx[Dx > 0].sum())

    errs = []
    for _ in range(16):
        dA = torch.from_numpy(rng.standard_normal((k, k))).cuda(); dA = dA + dA.T
        dB = torch.from_numpy(rng.standard_normal((k, k))).cuda(); dB = dB + dB.T
        dH = torch.cat([torch.cat([dA, dB], 1), torch.cat([-dB, -dA], 1)], 0)
        hh = 1e-6
        fd = (f(Hd + hh * dH) - f(Hd - hh * dH)) / (2 * hh)
        an = float((grad * dH).sum())
        errs.append(abs(fd - an) / max(1.0, abs(an)))
    assert max(errs) <= 1e-6, errs


def _proj(X, k):
    """Sigma sym(Sigma X), Sigma = diag(I_k, -I_k)."""
    sg = np.r_[np.ones(k), -np.ones(k)]
    Y = sg[:, None] * X
    return sg[:, None] * (0.5 * (Y + Y.T))


@pytest.mark.parametrize("k,dist,precision", [(16, ("uniform", 1.0, 10.0), "fp64"),
                                              (48, ("loguniform", 1e-1, 1e1), "fp64"),
                                              (48, ("loguniform", 1e-1, 1e1), "fp64e")])
def test_step_reversal_matches_projected_reference(P, k, dist, precision):
    """Reversing each Zolotarev step (stored inverses, and recomputed from per-step checkpoints)
    gives the projected block-sign reference; the Daleckii-Krein adjoint projected agrees."""
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED}[precision]
    H, _, _ = G.casida(k, dist, seed=600 + k)
    n = 2 * k
    rng = np.random.default_rng(1)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    ref = _proj(_loss_grad_ref(H, Gm), k)
    Hd, Gd = _dev(H), _dev(Gm)
    Hs = P.sign_vjp_rev(Hd, Gd, pos_weight=1.0, precision=pr).cpu().numpy()
    Hr = P.sign_vjp_rev(Hd, Gd, pos_weight=1.0, precision=pr, flags=P.FLAG_RECOMPUTE).cpu().numpy()
    assert np.linalg.norm(Hs - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(Hr - Hs) <= 1e-12 * np.linalg.norm(ref)
    lamb = torch.zeros(n, dtype=torch.float64, device="cuda"); lamb[:k] = 1.0
    dk = _proj(P.sign_vjp(Hd, Gd, lambar=lamb, precision=pr).cpu().numpy(), k)
    assert np.linalg.norm(dk - Hs) <= 1e-8 * np.linalg.norm(ref)
    # the two parts separately: no cotangent of S, and no eigenvalue term
    Hp = P.sign_vjp_rev(Hd, None, pos_weight=1.0, precision=pr).cpu().numpy()
    S = O.sign_def(H)
    assert np.linalg.norm(Hp - _proj(0.5 * (np.eye(n) + S).T, k)) <= 1e-10 * n
    H0 = P.sign_vjp_rev(Hd, Gd, precision=pr).cpu().numpy()
    assert np.linalg.norm(H0 - _proj(O.sign_vjp_block(H, Gm), k)) <= 1e-8 * np.linalg.norm(ref)


def test_step_reversal_autograd(P):
    """SignFn (default adjoint: steps) + EigvalsFn through torch.autograd."""
    k = 24
    H, _, _ = G.casida(k, ("uniform", 1.0, 10.0), seed=15)
    n = 2 * k
    rng = np.random.default_rng(4)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    Ht = _dev(H).requires_grad_(True)
    S = P.SignFn.apply(Ht)
    loss = (_dev(Gm) * S).sum()
    loss.backward()
    ref = _proj(O.sign_vjp_block(H, Gm), k)
    assert np.linalg.norm(Ht.grad.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_step_reversal_n2048_finite_differences(P):
    """n = 2048, d ~ U[1,10]: loss <G,S> + sum of positive eigenvalues (= tr(H P_+),
    P_+ = (I + S)/2), G symmetric N(0,1); the step-reversal gradient against central
    differences (h = 1e-6) along 16 structure-preserving directions, relative error <= 1e-6."""
    import time
    k = 1024
    n = 2 * k
    H, _, _ = G.casida(k, ("uniform", 1.0, 10.0), seed=2048)
    rng = np.random.default_rng(3)
    Gm = rng.standard_normal((n, n)); Gm = 0.5 * (Gm + Gm.T)
    Hd = _dev(H); Gt = _dev(Gm)
    P.sign_vjp_rev(Hd, Gt, pos_weight=1.0)
    torch.cuda.synchronize(); t0 = time.time()
    grad = P.sign_vjp_rev(Hd, Gt, pos_weight=1.0)
    torch.cuda.synchronize(); t1 = time.time()
    lamb = torch.zeros(n, dtype=torch.float64, device="cuda"); lamb[:k] = 1.0
    gdk = P.sign_vjp(Hd, Gt, lambar=lamb)
    torch.cuda.synchronize(); t2 = time.time()
    print(f"\nadjoint n=2048: step reversal {t1 - t0:.3f} s, Daleckii-Krein {t2 - t1:.3f} s")

    def f(Hx):
        Sx, _ = P.sign(Hx)
        return float((Gt * Sx).sum() + 0.5 * (torch.trace(Hx) + (Hx * Sx.T).sum()))

    errs = []
    for _ in range(16):
        dA = torch.from_numpy(rng.standard_normal((k, k))).cuda(); dA = dA + dA.T
        dB = torch.from_numpy(rng.standard_normal((k, k))).cuda(); dB = dB + dB.T
        dH = torch.cat([torch.cat([dA, dB], 1), torch.cat([-dB, -dA], 1)], 0)
        hh = 1e-6
        fd = (f(Hd + hh * dH) - f(Hd - hh * dH)) / (2 * hh)
        an = float((grad * dH).sum())
        errs.append(abs(fd - an) / max(1.0, abs(an)))
        assert abs(float((gdk * dH).sum()) - an) <= 1e-8 * max(1.0, abs(an))
    assert max(errs) <= 1e-6, errs
