"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- none of the method's arithmetic --
and is the one module that both the CPU oracle's tests and the CUDA path's
tests and benchmark use.

Casida / real BSE form (Sec. 5, Eq. Casida):
    P = Q1 diag(d1) Q1^T,  R = Q2 diag(d2) Q2^T   (Q1, Q2 Haar orthogonal k-by-k)
    A = (P + R)/2,  B = (P - R)/2,  H = [[A, B], [-B, -A]],  J = diag(I_k, -I_k)
so that M = J H = [[A, B], [B, A]] is orthogonally similar to diag(P, R) and
has the eigenvalues d1 and d2: M is symmetric positive definite whenever the
d's are positive, i.e. H is a definite pseudosymmetric matrix.  The
eigenvalues of H are +-sqrt(eig(P R)); with Q1 = Q2 they are exactly
+-sqrt(d1_i d2_i).

Example-1 form (Sec. 6.1): Sigma random +-1, A = Sigma Q D Q^T with D equally
spaced in [1, kappa] and Q orthogonal (QR of a uniform random matrix).

Haar matrices: QR of a standard Gaussian matrix with the columns multiplied by
sign(diag R) (Mezzadri's recipe).
"""
from __future__ import annotations

import numpy as np

# named workloads: (k, distribution of d1 and d2)
WORKLOADS = {
    "casida_n128_u1_10": (64, ("uniform", 1.0, 10.0)),
    "casida_n4096_u0.1_100": (2048, ("uniform", 0.1, 100.0)),
    "casida_n16384_log1e-2_1e2": (8192, ("loguniform", 1e-2, 1e2)),
    "casida_n2048_u1_10": (1024, ("uniform", 1.0, 10.0)),
}


def draw_d(rng, k, dist):
    kind, lo, hi = dist
    if kind == "uniform":
        return rng.uniform(lo, hi, k)
    if kind == "loguniform":
        return np.exp(rng.uniform(np.log(lo), np.log(hi), k))
    raise ValueError(kind)


def haar(rng, k):
    Z = rng.standard_normal((k, k))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def casida_blocks(k, d1, d2, rng, same_q=False):
    """Return (A, B) of the Casida form with spectra d1 (of A+B), d2 (of A-B)."""
    Q1 = haar(rng, k)
    Q2 = Q1 if same_q else haar(rng, k)
    P = (Q1 * d1[None, :]) @ Q1.T
    R = (Q2 * d2[None, :]) @ Q2.T
    P = 0.5 * (P + P.T)
    R = 0.5 * (R + R.T)
    return 0.5 * (P + R), 0.5 * (P - R)


def casida(k, dist=("uniform", 1.0, 10.0), seed=0, same_q=False):
    """H (2k-by-2k, float64, C order), and the d1, d2 used.  Signature is
    diag(I_k, -I_k)."""
    rng = np.random.default_rng(seed)
    d1 = draw_d(rng, k, dist)
    d2 = draw_d(rng, k, dist)
    A, B = casida_blocks(k, d1, d2, rng, same_q=same_q)
    H = np.block([[A, B], [-B, -A]])
    return np.ascontiguousarray(H), d1, d2


def workload(name, seed=0, same_q=False):
    k, dist = WORKLOADS[name]
    return casida(k, dist, seed=seed, same_q=same_q)


def casida_torch(k, dist, seed=0, device="cuda", same_q=False):
    """The same recipe drawn with torch on a device (used where numpy would
    take minutes, e.g. k = 8192).  Different random stream from ``casida``;
    same distribution."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    kind, lo, hi = dist
    u = torch.rand(2, k, generator=g, device=device, dtype=torch.float64)
    if kind == "uniform":
        d = lo + (hi - lo) * u
    else:
        d = torch.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)

    def haar_t():
        Z = torch.randn(k, k, generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(Z)
        return Q * torch.sign(torch.diagonal(R))[None, :]

    Q1 = haar_t()
    Q2 = Q1 if same_q else haar_t()
    P = (Q1 * d[0][None, :]) @ Q1.T
    R = (Q2 * d[1][None, :]) @ Q2.T
    P = 0.5 * (P + P.T)
    R = 0.5 * (R + R.T)
    A = 0.5 * (P + R)
    B = 0.5 * (P - R)
    H = torch.empty(2 * k, 2 * k, device=device, dtype=torch.float64)
    H[:k, :k] = A; H[:k, k:] = B; H[k:, :k] = -B; H[k:, k:] = -A
    return H, d[0], d[1]


def example1(n, kappa, seed=0):
    """Sec. 6.1 Example 1: Sigma random +-1, A = Sigma Q D Q^T, D equally
    spaced in [1, kappa].  Returns (A, sigma as +-1 int8 vector)."""
    rng = np.random.default_rng(seed)
    sigma = np.where(rng.uniform(size=n) < 0.5, 1, -1).astype(np.int8)
    Q, _ = np.linalg.qr(rng.uniform(size=(n, n)))
    D = np.linspace(1.0, kappa, n)
    M = (Q * D[None, :]) @ Q.T
    M = 0.5 * (M + M.T)
    A = sigma.astype(np.float64)[:, None] * M
    return np.ascontiguousarray(A), sigma


def batch_sizes(count=512, k_lo=16, k_hi=1024, seed=0):
    """k for each instance of a batch: log-uniform integers in [k_lo, k_hi]."""
    rng = np.random.default_rng(seed)
    return np.clip(np.round(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi), count))),
                   k_lo, k_hi).astype(int)


def haar_unitary(rng, k):
    """Haar unitary k-by-k: QR of a complex Gaussian with the columns multiplied by
    the phases of diag R."""
    Z = (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def bse2(k, dist=("uniform", 1.0, 10.0), seed=0, same_q=False):
    """Complex Eq. (BSE2) form: P = Q1 diag(d1) Q1^H, R = Q2 diag(d2) Q2^H (Q1, Q2 Haar
    unitary), A = (P + R)/2, B = (P - R)/2 (both Hermitian), H = [[A, B], [-B, -A]].
    M = Sigma H = [[A, B], [B, A]] is unitarily similar to diag(P, R): Hermitian positive
    definite for positive d; with Q1 = Q2 the eigenvalues are +-sqrt(d1_i d2_i).
    Returns (H complex128 C order, d1, d2)."""
    rng = np.random.default_rng(seed)
    d1 = draw_d(rng, k, dist)
    d2 = draw_d(rng, k, dist)
    Q1 = haar_unitary(rng, k)
    Q2 = Q1 if same_q else haar_unitary(rng, k)
    P = (Q1 * d1[None, :]) @ Q1.conj().T
    R = (Q2 * d2[None, :]) @ Q2.conj().T
    P = 0.5 * (P + P.conj().T)
    R = 0.5 * (R + R.conj().T)
    A = 0.5 * (P + R)
    B = 0.5 * (P - R)
    H = np.block([[A, B], [-B, -A]])
    return np.ascontiguousarray(H), d1, d2


def bse2_blocks(k, d1, d2, rng, same_q=True):
    """(A, B) of the Eq. (BSE2) form for given d1, d2 (Q1 = Q2 by default)."""
    Q1 = haar_unitary(rng, k)
    Q2 = Q1 if same_q else haar_unitary(rng, k)
    P = (Q1 * d1[None, :]) @ Q1.conj().T
    R = (Q2 * d2[None, :]) @ Q2.conj().T
    P = 0.5 * (P + P.conj().T)
    R = 0.5 * (R + R.conj().T)
    return 0.5 * (P + R), 0.5 * (P - R)


def bse1(k, dist=("uniform", 1.0, 10.0), coupling=0.5, seed=0):
    """Complex Eq. (BSE1) form H = [[A, B], [-conj(B), -conj(A)]]: A = Q diag(d) Q^H
    Hermitian (Q Haar unitary, d from dist), B complex symmetric (a symmetrised complex
    Gaussian) scaled to ||B||_2 = coupling * min(d).  Then Sigma H = [[A, B], [conj(B),
    conj(A)]] is Hermitian and, since ||B||_2 < lambda_min(A), positive definite.
    Returns H (complex128, C order)."""
    rng = np.random.default_rng(seed)
    d = draw_d(rng, k, dist)
    Q = haar_unitary(rng, k)
    A = (Q * d[None, :]) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    Z = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    B = 0.5 * (Z + Z.T)
    B *= coupling * d.min() / np.linalg.norm(B, 2)
    H = np.block([[A, B], [-B.conj(), -A.conj()]])
    return np.ascontiguousarray(H)


def general_pseudosym(n, seed=0, n_pairs=0, definite=False, spread=1.0):
    """A general (not necessarily definite) real pseudosymmetric matrix with a known
    spectrum (Sec. 3.3, Def. pseudosym): A = V C Sigma V^T Sigma with V = expm(Sigma W)
    (W skew-symmetric Gaussian scaled to ||W||_2 = spread), so that V^T Sigma V = Sigma and
    V^{-1} = Sigma V^T Sigma, and C block diagonal with C Sigma symmetric: real 1 x 1
    entries lambda_i, and `n_pairs` 2 x 2 blocks [[mu, nu], [-nu, mu]] on index pairs with
    opposite signs of Sigma (eigenvalues mu +- i nu).  Then Sigma A = (Sigma V)(C Sigma)
    (Sigma V)^T is symmetric.  definite=True takes no pairs and sign(lambda_i) = sigma_i,
    which makes Sigma A positive definite.
    Returns (A, sigma as +-1 int8 vector, C, V)."""
    from scipy.linalg import expm
    rng = np.random.default_rng(seed)
    p = n // 2
    sig = np.r_[np.ones(p), -np.ones(n - p)]
    rng.shuffle(sig)
    W = rng.standard_normal((n, n))
    W = W - W.T
    W *= spread / np.linalg.norm(W, 2)
    V = expm(sig[:, None] * W)
    C = np.zeros((n, n))
    pos, neg = list(np.flatnonzero(sig > 0)), list(np.flatnonzero(sig < 0))
    used = set()
    if not definite:
        for _ in range(min(n_pairs, len(pos), len(neg))):
            i, j = pos.pop(), neg.pop()
            mu, nu = rng.uniform(-3.0, 3.0), rng.uniform(0.3, 2.0)
            C[i, i] = C[j, j] = mu
            C[i, j], C[j, i] = nu, -nu
            used.update((i, j))
    for i in range(n):
        if i in used:
            continue
        lam = rng.uniform(0.2, 3.0)
        s = sig[i] if definite else (1.0 if rng.uniform() < 0.5 else -1.0)
        C[i, i] = s * lam
    A = V @ C @ (sig[:, None] * V.T) * sig[None, :]
    return np.ascontiguousarray(A), sig.astype(np.int8), C, V
