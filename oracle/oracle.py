"""Plain FP64 CPU oracle: the paper's algorithms written out step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The scalar loops live
in ``pssd_oracle.c``; this module strings them together in the paper's order
and notation.  The only library primitive used as a step is the dense matrix
product (``numpy.matmul``), except in the general (non-definite) layer at the
end, whose steps also call numpy's general eigensolver (the definition of
sign(A) for a complex spectrum) and scipy's Bunch-Kaufman LDL^T (the ``ldl``
of Alg. 5).

Two layers (both FP64):

* definition layer (``eig_def``, ``sign_def``): the exact result the method
  converges to.  The eigenvalues of the definite pencil ``M v = lambda Sigma v``
  (``M = Sigma H``) come from the Jacobi eigensolver applied to the symmetric
  ``K = L^T Sigma L`` with ``M = L L^T``; the eigenvectors are
  ``v = sqrt|lambda| L^{-T} u`` normalised to ``v^T Sigma v = +-1``
  (Thm. EVRealSigmaOrth and its proof by simultaneous diagonalisation), and
  ``sign(H) = V sign(Lambda) V^{-1}`` (Eq. signDef) with
  ``V^{-1} = Sigma_hat V^T Sigma``.
* algorithm layer (``sign_alg``, ``split_alg``, ``eig_alg``): Alg. 8 with the
  inverse-form step Eq. (ZoloIt2), then Alg. 7, then the symmetric definite
  subproblems by Jacobi (Thm. DefDivConq).
* general (non-definite) layer (``gsign_def``, ``hyp_basis_ldl``,
  ``geig_alg``): Alg. 3 with the hyperbolic bases of Alg. 5 (readings R12-R14
  in that section).

Readings of the paper where it is garbled or silent:
  R1  Eq. (Compcis): the argument is i*K'/(2r+1) with the integer index i.
  R2  Eq. (ZPartialFrac2): the product between the two products is a quotient.
  R3  r is the smallest value for which two steps map [l,1] into [1-tau,1].
  R4  Alg. 8 step "X1 <- C(X_k + ...)" uses X_0; Alg. 4's Q_- uses P_-.
  R5  bounds alpha, beta: alpha = lambda_max(Sigma A), beta = lambda_min(Sigma A)
      (valid since |lambda(A)| lies in [lambda_min(M), lambda_max(M)]).
  R6  restart of Alg. 8 (failed stopping test): A <- X_2 with the bounds
      alpha = 1, beta = l_2, which bound |lambda(X_2)| because Zhat o Zhat maps
      [l,1] monotonically into [l_2,1]; r by R3; at most ``max_restarts``
      restarts.
"""
from __future__ import annotations

import ctypes
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

U_FP64 = 2.0 ** -53

_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.or_cholesky.argtypes = [ctypes.c_int, dp, dp]
        lib.or_lu_solve.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
        lib.or_jacobi_eigh.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int]
        lib.or_pivoted_lowrank_chol.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ip]
        lib.or_ellipk_from_comp.argtypes = [ctypes.c_double]
        lib.or_ellipk_from_comp.restype = ctypes.c_double
        lib.or_sncn.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
        lib.or_sc_comp.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.or_sc_comp.restype = ctypes.c_double
        lib.or_zolo_coeffs.argtypes = [ctypes.c_double, ctypes.c_int, dp, dp, dp, dp]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class NotDefinite(ValueError):
    """Sigma*H is not positive definite (a Cholesky pivot was not positive)."""


# --------------------------------------------------------------------------
# scalar Zolotarev machinery  (Sec. 5.3)
# --------------------------------------------------------------------------

def ellipk_from_comp(kc: float) -> float:
    """K for the modulus whose complementary modulus is ``kc`` (AGM)."""
    return _L().or_ellipk_from_comp(float(kc))


def sncn(u: float, kc: float):
    """Jacobi sn(u), cn(u) by descending Landen/AGM; modulus sqrt(1-kc^2)."""
    s = ctypes.c_double(); c = ctypes.c_double()
    _L().or_sncn(float(u), float(kc), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sc_comp(u: float, kc: float) -> float:
    """sn(u)/cn(u) for the modulus sqrt(1-kc^2) (imaginary transformation +
    descending Landen on the small modulus kc)."""
    return _L().or_sc_comp(float(u), float(kc))


def zolo_coeffs(ell: float, r: int):
    """Coefficients of the scaled Zolotarev function (Eqs. Compcis, hatZ,
    ZPartialFrac2 and the l-update of Alg. 8; readings R1, R2).

    Returns ``(c, a, chat, ell_next)`` with ``c[i-1] = c_i`` (i = 1..2r),
    ``a[j-1] = a_j`` (j = 1..r).
    Pinned by: equioscillation, Zhat(1)=1, the partial-fraction identity,
    the composition law and the r=1 closed form (tests/test_oracle_zolo.py).
    """
    c = np.zeros(2 * r); a = np.zeros(r)
    ch = ctypes.c_double(); l1 = ctypes.c_double()
    st = _L().or_zolo_coeffs(float(ell), int(r), _p(c), _p(a), ctypes.byref(ch), ctypes.byref(l1))
    if st:
        raise ValueError("zolo_coeffs: invalid ell=%r r=%r" % (ell, r))
    return c, a, ch.value, l1.value


def zolo_eval(x, ell: float, r: int):
    """Scaled Zolotarev function, product form (Eq. hatZ):
    Zhat(x) = Chat x prod_j (x^2 + c_{2j}) / (x^2 + c_{2j-1})."""
    c, _, chat, _ = zolo_coeffs(ell, r)
    x = np.asarray(x, dtype=np.float64)
    y = chat * x
    for j in range(r):
        y = y * (x * x + c[2 * j + 1]) / (x * x + c[2 * j])
    return y


def zolo_eval_partial_fractions(x, ell: float, r: int):
    """Scaled Zolotarev function, partial-fraction form (Eq. ZPartialFrac):
    Zhat(x) = Chat x (1 + sum_j a_j / (x^2 + c_{2j-1}))."""
    c, a, chat, _ = zolo_coeffs(ell, r)
    x = np.asarray(x, dtype=np.float64)
    s = np.ones_like(x)
    for j in range(r):
        s = s + a[j] / (x * x + c[2 * j])
    return chat * x * s


def choose_r(ell: float, tau: float = 1e-15, r_max: int = 8) -> int:
    """Reading R3 of the choice of r (the paper defers to a table that is not
    reproduced): the smallest r <= r_max with 1 - l_2 <= tau, where
    l_1 = Zhat(l; l) and l_2 = Zhat(l_1; l_1)."""
    for r in range(1, r_max + 1):
        l1 = min(zolo_coeffs(ell, r)[3], 1.0)
        if 1.0 - l1 <= tau:
            return r
        l2 = zolo_coeffs(l1, r)[3]
        if 1.0 - l2 <= tau:
            return r
    return r_max


# --------------------------------------------------------------------------
# dense scalar-loop kernels
# --------------------------------------------------------------------------

def cholesky(A):
    """Lower Cholesky factor (scalar loops).  Raises NotDefinite."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros((n, n))
    st = _L().or_cholesky(n, _p(A), _p(L))
    if st:
        raise NotDefinite("non-positive pivot at index %d" % (st - 1))
    return L


def lu_solve(A, B):
    """Solve A X = B by Gaussian elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    B = np.array(B, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    m = 1 if B.ndim == 1 else B.shape[1]
    st = _L().or_lu_solve(n, _p(A), m, _p(B))
    if st:
        raise np.linalg.LinAlgError("singular at %d" % (st - 1))
    return B


def jacobi_eigh(A, max_sweeps: int = 60):
    """Symmetric eigendecomposition by cyclic Jacobi; eigenvalues ascending."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    A = 0.5 * (A + A.T)
    A = np.ascontiguousarray(A)
    w = np.zeros(n); V = np.zeros((n, n))
    sweeps = _L().or_jacobi_eigh(n, _p(A), _p(w), _p(V), int(max_sweeps))
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    idx = np.argsort(w, kind="stable")
    return w[idx], np.ascontiguousarray(V[:, idx])


def pivoted_lowrank_chol(A, rank: int):
    """A ~= W W^T, W n-by-rank, diagonal pivoting (largest first, ties lowest)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    W = np.zeros((n, rank)); piv = np.zeros(rank, dtype=np.int32)
    st = _L().or_pivoted_lowrank_chol(n, _p(A), int(rank), _p(W),
                                      piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if st:
        raise NotDefinite("pivoted low-rank Cholesky broke down at step %d" % (st - 1))
    return W, piv


# --------------------------------------------------------------------------
# signature helpers (Def. pseudosym)
# --------------------------------------------------------------------------

def signature(n: int, sigma=None):
    """Diagonal of Sigma as a float vector; None means diag(I_{n/2}, -I_{n/2})."""
    if sigma is None:
        if n % 2:
            raise ValueError("default signature needs even n")
        return np.r_[np.ones(n // 2), -np.ones(n // 2)]
    s = np.asarray(sigma, dtype=np.float64).ravel()
    if s.shape[0] != n or not np.all(np.abs(s) == 1.0):
        raise ValueError("sigma must hold n entries in {+1,-1}")
    return s


def pseudosymmetry_defect(H, sigma=None):
    """||Sigma H - (Sigma H)^T||_F / ||Sigma H||_F (Def. pseudosym)."""
    s = signature(H.shape[0], sigma)
    M = s[:, None] * H
    return np.linalg.norm(M - M.T) / np.linalg.norm(M)


# --------------------------------------------------------------------------
# definition layer
# --------------------------------------------------------------------------

def _sign_fix_columns(V):
    """Output convention: each column's largest-magnitude entry is positive
    (ties: lowest index)."""
    V = V.copy()
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return V


def _order(lam, V):
    """Output convention: positive eigenvalues ascending, then negative ones by
    ascending magnitude."""
    pos = np.where(lam > 0)[0]; neg = np.where(lam < 0)[0]
    pos = pos[np.argsort(lam[pos], kind="stable")]
    neg = neg[np.argsort(-lam[neg], kind="stable")]
    idx = np.r_[pos, neg]
    return lam[idx], V[:, idx]


def eig_def(H, sigma=None):
    """Definition-level eigendecomposition of a definite pseudosymmetric H.

    M = Sigma H = L L^T (scalar Cholesky), K = L^T Sigma L is symmetric and
    similar to H (L^T H L^{-T} = K), so lambda(H) = lambda(K) (Jacobi).
    Eigenvectors v = sqrt|lambda| L^{-T} u satisfy V^T Sigma V = Sigma_hat
    (Eq. VSigmaOrth, up to the column order of the output convention).
    Returns (lam, V) in the output convention.
    """
    n = H.shape[0]
    s = signature(n, sigma)
    M = s[:, None] * H
    M = 0.5 * (M + M.T)
    L = cholesky(M)
    K = L.T @ (s[:, None] * L)
    w, U = jacobi_eigh(K)
    Y = lu_solve(L.T, U)                     # L^{-T} U
    V = Y * np.sqrt(np.abs(w))[None, :]
    lam, V = _order(w, V)
    return lam, _sign_fix_columns(V)


def sign_def(H, sigma=None):
    """sign(H) = V sign(Lambda) V^{-1} (Eq. signDef) with
    V^{-1} = Sigma_hat V^T Sigma; since Sigma_hat = sign(Lambda) here
    (Thm. EVRealSigmaOrth), S = V V^T Sigma."""
    n = H.shape[0]
    s = signature(n, sigma)
    lam, V = eig_def(H, sigma)
    return (V @ V.T) * s[None, :]


def casida_eig_def(A, B):
    """Definition-level eigendecomposition of the Casida matrix
    H = [[A, B], [-B, -A]] (Eq. Casida) from its k x k blocks.

    With T = [[I, I], [I, -I]]/sqrt 2, T H T = [[0, R], [P, 0]] (P = A + B,
    R = A - B).  An eigenvector [x; y] for lambda satisfies R y = lambda x,
    P x = lambda y; with P = L L^T (scalar Cholesky) and x = L^{-T} z this is
    L^T R L z = lambda^2 z (the k x k reduction P^{1/2} R P^{1/2} up to
    similarity), y = L z / lambda.  Jacobi gives omega^2 and z; the
    eigenvalues are +-omega and v = T [L^{-T} z; +-L z/omega] sqrt(omega/2)
    has v^T Sigma v = +-1 (Eq. VSigmaOrth).
    Returns (lam, V) in the output convention."""
    A = np.asarray(A, dtype=np.float64); B = np.asarray(B, dtype=np.float64)
    k = A.shape[0]
    P = 0.5 * ((A + B) + (A + B).T)
    R = 0.5 * ((A - B) + (A - B).T)
    L = cholesky(P)
    W = L.T @ R @ L
    w2, Z = jacobi_eigh(0.5 * (W + W.T))
    if not w2[0] > 0:
        raise NotDefinite("A - B is not positive definite")
    om = np.sqrt(w2)
    X = lu_solve(L.T, Z)                       # L^{-T} z
    Y = (L @ Z) / om[None, :]                  # L z / omega
    c = np.sqrt(om / 2.0)[None, :]
    Vp = np.vstack([X + Y, X - Y]) / math.sqrt(2.0) * c     # T [X; Y]
    Vm = np.vstack([X - Y, X + Y]) / math.sqrt(2.0) * c     # T [X; -Y]
    lam = np.r_[om, -om]
    V = np.hstack([Vp, Vm])
    lam, V = _order(lam, V)
    return lam, _sign_fix_columns(V)


def casida_sign_def(A, B):
    """sign(H) of the Casida matrix from casida_eig_def: S = V V^T Sigma
    (as sign_def, Eq. signDef with V^{-1} = Sigma_hat V^T Sigma)."""
    k = A.shape[0]
    _, V = casida_eig_def(A, B)
    s = np.r_[np.ones(k), -np.ones(k)]
    return (V @ V.T) * s[None, :]


# --------------------------------------------------------------------------
# algorithm layer: Alg. 8 (hyperbolic Zolo-PD), Alg. 7, Alg. 3
# --------------------------------------------------------------------------

def estimate_bounds(A, sigma=None):
    """Alg. 8 first step, reading R5: alpha = lambda_max(Sigma A),
    beta = lambda_min(Sigma A), from the Jacobi eigensolver."""
    s = signature(A.shape[0], sigma)
    M = s[:, None] * A
    w, _ = jacobi_eigh(0.5 * (M + M.T))
    if not w[0] > 0:
        raise NotDefinite("Sigma*A is not positive definite")
    return float(w[-1]), float(w[0])


def zolo_step(X, sigma, c, a, chat, threads: int | None = None):
    """One step of Eq. (ZoloIt2) with M = Sigma:
    X_{k+1} = Chat (X + sum_j a_j X (X^T Sigma X + c_{2j-1} Sigma)^{-1} Sigma).

    The r shifted systems are mutually independent and are solved in
    parallel threads (Gaussian elimination with partial pivoting, which the
    paper's pivoted LDL^T / hyperbolic QR forms equal in exact arithmetic,
    Eqs. LDLZolo, HRZolo and Lemma HRnoInv)."""
    n = X.shape[0]
    s = signature(n, sigma)
    XtSX = X.T @ (s[:, None] * X)
    Sig = np.diag(s)
    r = len(a)

    def term(j):
        Z = XtSX + c[2 * j] * Sig
        Y = lu_solve(Z, Sig)                 # Z^{-1} Sigma
        return a[j] * (X @ Y)

    with ThreadPoolExecutor(max_workers=threads or r) as ex:
        terms = list(ex.map(term, range(r)))
    acc = X.copy()
    for t in terms:
        acc = acc + t
    return chat * acc


def sign_alg(H, sigma=None, r: int | None = None, alpha: float | None = None,
             beta: float | None = None, max_restarts: int = 2, tau: float = 1e-15):
    """Alg. 8 (hyperbolic Zolo-PD) for a definite pseudosymmetric H.

    Returns (S, info) where info holds the per-step iterates X1, X2 of the
    first pass, r per pass, the l values, the stopping quantity and the
    number of restarts.  A failed stopping test restarts from A <- X_2
    (reading R6); more than ``max_restarts`` restarts raises RuntimeError.
    """
    n = H.shape[0]
    s = signature(n, sigma)
    A = np.array(H, dtype=np.float64)
    info = {"r": [], "ell": [], "stop": [], "restarts": 0, "X1": None, "X2": None}
    ell_last = None
    for attempt in range(max_restarts + 1):
        if attempt > 0:
            al, be = 1.0, ell_last                       # reading R6
        elif alpha is not None and beta is not None:
            al, be = float(alpha), float(beta)
        else:
            al, be = estimate_bounds(A, s)
        X0 = A / al
        ell = min(be / al, 1.0)
        rr = r if (r is not None and attempt == 0) else choose_r(ell, tau)
        info["r"].append(rr); info["ell"].append(ell)
        c, a, chat, ell1 = zolo_coeffs(ell, rr)
        X1 = zolo_step(X0, s, c, a, chat)               # first iteration
        ell = min(ell1, 1.0)
        info["ell"].append(ell)
        c, a, chat, ell2 = zolo_coeffs(ell, rr)         # coefficient update
        X2 = zolo_step(X1, s, c, a, chat)               # second iteration
        info["ell"].append(min(ell2, 1.0))
        ell_last = min(ell2, 1.0)
        if attempt == 0:
            info["X1"], info["X2"] = X1, X2
        crit = np.linalg.norm(X2 - X1) / np.linalg.norm(X2)
        info["stop"].append(crit)
        if crit <= U_FP64 ** (1.0 / (2 * rr + 1)):
            info["S"] = X2
            return X2, info
        info["restarts"] += 1
        A = X2
    raise RuntimeError("Zolo-PD: stopping test failed after %d restarts" % max_restarts)


def dwh_sign_alg(H, sigma=None, alpha: float | None = None, beta: float | None = None, max_iter: int = 30):
    """The Sigma-DWH iteration Sec. 6 compares against: the Zolotarev step of
    Eq. (ZoloIt2) with degree r = 1 (the dynamically weighted Halley step;
    Sec. 5.3 identifies the two) repeated with the l-update of Alg. 8 after
    every step, until ||X_{k+1} - X_k||_F / ||X_{k+1}||_F <= u^{1/3} (the step
    converges cubically).  Bounds as in Alg. 8 (reading R5).
    Returns (S, info) with info["iterations"] and the l sequence."""
    n = H.shape[0]
    s = signature(n, sigma)
    A = np.array(H, dtype=np.float64)
    al, be = (float(alpha), float(beta)) if (alpha is not None and beta is not None) else estimate_bounds(A, s)
    X = A / al
    ell = min(be / al, 1.0)
    info = {"ell": [ell], "iterations": 0}
    for it in range(max_iter):
        c, a, chat, ell1 = zolo_coeffs(ell, 1)
        Xn = zolo_step(X, s, c, a, chat)
        crit = np.linalg.norm(Xn - X) / np.linalg.norm(Xn)
        X = Xn
        ell = min(ell1, 1.0)
        info["ell"].append(ell)
        info["iterations"] = it + 1
        if crit <= U_FP64 ** (1.0 / 3.0):
            return X, info
    raise RuntimeError("Sigma-DWH did not converge in %d steps" % max_iter)


def byers_xu_scalings(a: float, b: float, count: int):
    """The suboptimal scaling factors of Byers and Xu for Newton's iteration
    (the comparison method of Sec. 6) for a spectrum whose magnitudes lie in
    [b, a]: z_0 = 1/sqrt(ab), z_1 = sqrt(2 sqrt(ab)/(a+b)),
    z_{k+1} = 1/sqrt((z_k + 1/z_k)/2)."""
    z = [1.0 / math.sqrt(a * b)]
    if count > 1:
        z.append(math.sqrt(2.0 * math.sqrt(a * b) / (a + b)))
    while len(z) < count:
        z.append(1.0 / math.sqrt(0.5 * (z[-1] + 1.0 / z[-1])))
    return z[:count]


def newton_sign_scaled(H, sigma=None, alpha: float | None = None, beta: float | None = None, max_iter: int = 60):
    """Scaled Newton iteration for sign(H) (Eq. NewtonSign with the scaling of
    Byers and Xu, the comparison method of Sec. 6):
    X_{k+1} = (z_k X_k + (z_k X_k)^{-1}) / 2, X_0 = H/alpha, spectral bounds
    a = 1, b = beta/alpha; the inverse by Gaussian elimination with partial
    pivoting.  Stops when ||X_{k+1} - X_k||_F / ||X_{k+1}||_F <= u^{1/2}
    (quadratic convergence), never after the first step.
    Returns (S, info) with info["iterations"]."""
    n = H.shape[0]
    s = signature(n, sigma)
    A = np.array(H, dtype=np.float64)
    al, be = (float(alpha), float(beta)) if (alpha is not None and beta is not None) else estimate_bounds(A, s)
    X = A / al
    zs = byers_xu_scalings(1.0, min(be / al, 1.0), max_iter)
    I = np.eye(n)
    for it in range(max_iter):
        z = zs[it]
        Xn = 0.5 * (z * X + lu_solve(z * X, I))
        crit = np.linalg.norm(Xn - X) / np.linalg.norm(Xn)
        X = Xn
        if it > 0 and crit <= math.sqrt(U_FP64):
            return X, {"iterations": it + 1}
    raise RuntimeError("scaled Newton did not converge in %d steps" % max_iter)


def split_alg(H, sigma=None, S=None):
    """Alg. 7 (robust (Sigma, Sigma_hat)-orthogonal basis via pivoted,
    truncated LDL^T) and the projections of Thm. DefDivConq.

    P_+ = (I+S)/2 and P_- = (I-S)/2 (Lemma SignProj); Sigma P_+ and
    -Sigma P_- are positive semidefinite of ranks p and n-p
    (Thm. EVRealSigmaOrth); their pivoted low-rank Cholesky factors W_+-
    give Q_+- = Sigma W_+-, with Q_+^T Sigma Q_+ = I_p and
    Q_-^T Sigma Q_- = -I_{n-p} (Thm. HRisLDL).  Then
    A11 = Q_+^T M Q_+ (SPD) and A22 = -Q_-^T M Q_- (SND), M = Sigma H.
    Returns (Qp, Qm, A11, A22).
    """
    n = H.shape[0]
    s = signature(n, sigma)
    if S is None:
        S, _ = sign_alg(H, s)
    p = int(np.sum(s > 0))
    I = np.eye(n)
    Pp = 0.5 * (I + S)
    Pm = 0.5 * (I - S)
    SPp = s[:, None] * Pp
    SPm = -(s[:, None] * Pm)
    Wp, _ = pivoted_lowrank_chol(0.5 * (SPp + SPp.T), p)
    Wm, _ = pivoted_lowrank_chol(0.5 * (SPm + SPm.T), n - p)
    Qp = s[:, None] * Wp
    Qm = s[:, None] * Wm
    M = s[:, None] * H
    A11 = Qp.T @ M @ Qp
    A22 = -(Qm.T @ M @ Qm)
    return Qp, Qm, A11, A22


def split_backward_error(H, sigma, Qp, Qm):
    """The paper's backward error ||Q_+^T Sigma A Q_-||_F / ||A||_F (Ex. 1)."""
    s = signature(H.shape[0], sigma)
    return np.linalg.norm(Qp.T @ (s[:, None] * H) @ Qm) / np.linalg.norm(H)


def eig_alg(H, sigma=None, S=None):
    """Alg. 3 for a definite H: one structure-preserving split (Alg. 8 +
    Alg. 7), after which A11 is SPD and A22 SND (Thm. DefDivConq), so the
    recursion ends in two symmetric eigenproblems solved by Jacobi.
    V = [Q_+ V_1, Q_- V_2] satisfies V^T Sigma V = diag(I_p, -I_{n-p}).
    Returns (lam, V) in the output convention."""
    Qp, Qm, A11, A22 = split_alg(H, sigma, S)
    w1, U1 = jacobi_eigh(A11)
    w2, U2 = jacobi_eigh(A22)
    lam = np.r_[w1, w2]
    V = np.hstack([Qp @ U1, Qm @ U2])
    lam, V = _order(lam, V)
    return lam, _sign_fix_columns(V)


# --------------------------------------------------------------------------
# reference gradient: Newton sign iteration (Eq. NewtonSign)
# --------------------------------------------------------------------------

def newton_sign(X, tol: float = 1e-14, max_iter: int = 100):
    """Unscaled Newton iteration X <- (X + X^{-1})/2 (Eq. NewtonSign), the
    inverse by Gaussian elimination.  Stops when the relative change is
    below ``tol`` (plus one more step)."""
    X = np.array(X, dtype=np.float64)
    n = X.shape[0]
    I = np.eye(n)
    for it in range(max_iter):
        Xn = 0.5 * (X + lu_solve(X, I))
        d = np.linalg.norm(Xn - X) / np.linalg.norm(Xn)
        X = Xn
        if d <= tol:
            X = 0.5 * (X + lu_solve(X, I))
            return X
    raise RuntimeError("Newton sign iteration did not converge")


def sign_vjp_block(H, G, tol: float = 1e-14):
    """Reference cotangent of <G, sign(H)> with respect to H: the (1,2) block
    of sign([[H^T, G], [0, H^T]]) (Frechet derivative of the sign function
    applied to G, transposed into a gradient), computed by Newton because the
    block matrix is not diagonalisable."""
    n = H.shape[0]
    B = np.zeros((2 * n, 2 * n))
    B[:n, :n] = H.T; B[n:, n:] = H.T; B[:n, n:] = G
    SB = newton_sign(B, tol=tol)
    return SB[:n, n:]


# --------------------------------------------------------------------------
# complex pseudo-Hermitian matrices (the BSE forms, Eqs. BSE1 and BSE2): the
# definition layer in complex arithmetic, scalar loops (small n only)
# --------------------------------------------------------------------------

def zcholesky(M):
    """M = L L^H for a Hermitian positive definite M (scalar loops, row by row);
    L lower triangular with a real positive diagonal."""
    M = np.array(M, dtype=np.complex128)
    n = M.shape[0]
    L = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        for j in range(i + 1):
            acc = M[i, j]
            for k in range(j):
                acc -= L[i, k] * np.conj(L[j, k])
            if i == j:
                d = acc.real
                if not d > 0:
                    raise NotDefinite("pivot %d is not positive" % i)
                L[i, i] = math.sqrt(d)
            else:
                L[i, j] = acc / L[j, j]
    return L


def zupper_solve(U, B):
    """X with U X = B for an upper triangular U (back substitution over rows)."""
    U = np.asarray(U, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128)
    n = U.shape[0]
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def zjacobi_eigh(A, max_sweeps: int = 60):
    """Hermitian eigendecomposition by cyclic Jacobi: for each pair (p, q) with
    a_pq = |a_pq| e^{i phi}, the unitary W = diag(1, e^{-i phi}) J (J the real
    rotation that diagonalises [[a_pp, |a_pq|], [|a_pq|, a_qq]]) is applied as
    A <- W^H A W on rows and columns p, q.  Eigenvalues ascending."""
    A = np.array(A, dtype=np.complex128)
    A = 0.5 * (A + A.conj().T)
    n = A.shape[0]
    U = np.eye(n, dtype=np.complex128)
    for sweep in range(max_sweeps):
        off = np.sum(np.abs(A - np.diag(np.diag(A))) ** 2)
        # the off-diagonal norm cannot fall below rounding, about u sqrt(n) ||A||_F
        if off <= (4.0 * n * U_FP64) ** 2 * np.sum(np.abs(A) ** 2):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                b = A[p, q]
                ab = abs(b)
                if ab == 0.0:
                    continue
                ph = b / ab                                   # e^{i phi}
                tau = (A[q, q].real - A[p, p].real) / (2.0 * ab)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                # W = [[c, s], [-s conj(ph), c conj(ph)]] on columns p, q
                cp = A[:, p].copy(); cq = A[:, q].copy()
                A[:, p] = c * cp - s * np.conj(ph) * cq
                A[:, q] = s * cp + c * np.conj(ph) * cq
                rp = A[p, :].copy(); rq = A[q, :].copy()
                A[p, :] = c * rp - s * ph * rq
                A[q, :] = s * rp + c * ph * rq
                up = U[:, p].copy(); uq = U[:, q].copy()
                U[:, p] = c * up - s * np.conj(ph) * uq
                U[:, q] = s * up + c * np.conj(ph) * uq
    else:
        raise RuntimeError("complex Jacobi did not converge")
    w = np.diag(A).real.copy()
    idx = np.argsort(w, kind="stable")
    return w[idx], np.ascontiguousarray(U[:, idx])


def _phase_fix_columns(V):
    """Each column multiplied by conj(v_max)/|v_max|, v_max its entry of largest
    modulus (first on ties): that entry becomes real and positive."""
    V = np.array(V, dtype=np.complex128)
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        a = abs(V[i, j])
        if a > 0:
            V[:, j] *= np.conj(V[i, j]) / a
    return V


def zeig_def(H, sigma=None):
    """Definition-level eigendecomposition of a definite complex pseudo-Hermitian H
    (Sigma H Hermitian positive definite): M = Sigma H = L L^H (scalar Cholesky),
    K = L^H Sigma L is Hermitian and similar to H (L^H H L^{-H} = K), so
    lambda(H) = lambda(K) (complex Jacobi), and v = sqrt|lambda| L^{-H} u has
    v^H Sigma v = sign(lambda) (Eq. VSigmaOrth, the complex case of Thm.
    EVRealSigmaOrth).  Returns (lam, V) in the output convention, phases fixed."""
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    s = signature(n, sigma)
    M = s[:, None] * H
    M = 0.5 * (M + M.conj().T)
    L = zcholesky(M)
    K = L.conj().T @ (s[:, None] * L)
    w, U = zjacobi_eigh(K)
    Y = zupper_solve(L.conj().T, U)                 # L^{-H} U
    V = Y * np.sqrt(np.abs(w))[None, :]
    lam, V = _order(w, V)
    return lam, _phase_fix_columns(V)


def zsign_def(H, sigma=None):
    """sign(H) = V sign(Lambda) V^{-1} with V^{-1} = Sigma_hat V^H Sigma, i.e.
    S = V V^H Sigma (Eq. signDef, complex case)."""
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    s = signature(n, sigma)
    _, V = zeig_def(H, sigma)
    return (V @ V.conj().T) * s[None, :]


# --------------------------------------------------------------------------
# general (non-definite) pseudosymmetric case  (Sec. 3.3 Alg. 3, Sec. 4 Alg. 5)
#
# Library steps in this layer: numpy's general eigensolver (the definition of
# sign(A) for a spectrum that may be complex) and scipy's Bunch-Kaufman LDL^T
# (the `ldl` that Alg. 5 calls).  Readings:
#   R12 Alg. 5 writes D^{1/2}; D has negative entries, so R = (L V |D|^{1/2})^T
#       with Sigma_hat = sign(D), which keeps R^T Sigma_hat R = L D L^T; its last
#       steps write Sigma_hat (and diag(Sigma_+, Sigma_-)) where the sizes call
#       for Sigma_hat_+ and Sigma_hat_-: Q_+- = Sigma R_+-^T Sigma_hat_+-.
#   R13 Alg. 3 "find shift" (no rule given): the widest gap between consecutive
#       distinct real parts of the eigenvalues among the splits that leave between
#       a quarter and three quarters of them on each side (any split if none does);
#       the shift is the gap's midpoint, so a conjugate pair is never separated.
#   R14 The paper's sign iterations (Eqs. LDLZolo, HRZolo) are analysed for the
#       definite case (Lemma RationalIter); for a general pseudosymmetric A the
#       oracle takes the definition sign(A) = X sign(Re Lambda) X^{-1}.
# --------------------------------------------------------------------------

def gsign_def(A):
    """sign(A) for a real A with no eigenvalue on the imaginary axis, from its
    definition: A = X Lambda X^{-1}, sign(A) = X sign(Re Lambda) X^{-1} (the
    definition behind Eq. signDef, for a spectrum that may be complex).  The result of
    a real A is real; the imaginary rounding residue is dropped."""
    A = np.asarray(A, dtype=np.float64)
    lam, X = np.linalg.eig(A)
    scale = max(1.0, float(np.max(np.abs(lam)))) if lam.size else 1.0
    if np.any(np.abs(lam.real) <= 1e-13 * scale):
        raise ValueError("an eigenvalue lies on the imaginary axis: sign(A) is undefined")
    S = np.linalg.solve(X.T, (X * np.sign(lam.real)[None, :]).T).T     # X sign(Re Lambda) X^{-1}
    return np.ascontiguousarray(S.real)


def _diagonalise_blocks(D):
    """D (block diagonal, 1 x 1 and 2 x 2 symmetric blocks, as Bunch-Kaufman leaves it)
    = Vd diag(w) Vd^T with Vd orthogonal and block diagonal (Alg. 5, "diagonalize D")."""
    n = D.shape[0]
    w, Vd = np.zeros(n), np.zeros((n, n))
    i = 0
    while i < n:
        if i + 1 < n and D[i + 1, i] != 0.0:
            wb, vb = np.linalg.eigh(D[i:i + 2, i:i + 2])
            w[i:i + 2], Vd[i:i + 2, i:i + 2] = wb, vb
            i += 2
        else:
            w[i], Vd[i, i] = D[i, i], 1.0
            i += 1
    return w, Vd


def hyp_basis_ldl(S, sigma=None):
    """Alg. 5: from S = sign(A) of a pseudosymmetric A, bases Q_+ and Q_- of the invariant
    subspaces of the eigenvalues with positive and negative real part such that
    Q_+-^T Sigma Q_+- = Sigma_hat_+- (Thm. HRisLDL): P = (I +- S)/2, r = trace(P),
    Sigma P = L D L^T (Bunch-Kaufman), D diagonalised block by block, the r nonzero values
    kept, R = (L Vd_r |D_r|^{1/2})^T, Sigma_hat = sign(D_r), Q = Sigma R^T Sigma_hat
    (readings R12).  Returns (Q_+, Q_-, sigma_hat_+, sigma_hat_-)."""
    from scipy.linalg import ldl
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    s = signature(n, sigma)
    out = []
    for sgn in (1.0, -1.0):
        P = 0.5 * (np.eye(n) + sgn * S)
        r = int(round(float(np.trace(P))))
        if r <= 0:
            out.append((np.zeros((n, 0)), np.zeros(0)))
            continue
        L, D, _ = ldl(s[:, None] * P, lower=True)        # Sigma P = L D L^T (lower triangle read)
        w, Vd = _diagonalise_blocks(D)
        keep = np.sort(np.argsort(-np.abs(w), kind="stable")[:r])
        R = ((L @ Vd[:, keep]) * np.sqrt(np.abs(w[keep]))[None, :]).T     # r x n
        sh = np.sign(w[keep])
        out.append((s[:, None] * R.T * sh[None, :], sh))                # Q = Sigma R^T Sigma_hat
    (Qp, sp), (Qm, sm) = out
    return Qp, Qm, sp, sm


def _general_shift(lam):
    """Reading R13: the midpoint of the widest gap between consecutive distinct real parts
    among the balanced splits (a quarter to three quarters on each side), else among all."""
    re = np.sort(np.asarray(lam).real)
    n = re.size
    tol = 1e-12 * max(1.0, float(np.max(np.abs(re))))
    gaps = [(re[i + 1] - re[i], i + 1, 0.5 * (re[i] + re[i + 1])) for i in range(n - 1) if re[i + 1] - re[i] > tol]
    if not gaps:
        return None
    balanced = [g for g in gaps if n / 4.0 <= g[1] <= 3.0 * n / 4.0]
    return max(balanced or gaps)[2]


def geig_alg(A, sigma=None):
    """Alg. 3 (pseudosymmetric spectral divide-and-conquer) with sign(A - shift I) from its
    definition (R14), the bases of Alg. 5 and the shift of R13.  Stops at 1 x 1 blocks and
    at 2 x 2 blocks holding a complex conjugate pair.  Returns (V, sigma_hat, D):
    V^T Sigma V = Sigma_hat, V^{-1} = Sigma_hat V^T Sigma, and V^{-1} A V = D block
    diagonal with blocks of order 1 (real eigenvalues) and 2 (conjugate pairs); the
    off-diagonal blocks each split leaves are dropped (they are its backward error)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    s = signature(n, sigma)
    if n == 1:
        return np.eye(1), s.copy(), A.copy()
    lam = np.linalg.eigvals(A)
    if n == 2 and abs(lam[0].imag) > 0.0:
        return np.eye(2), s.copy(), A.copy()
    shift = _general_shift(lam)
    if shift is None:
        raise ValueError("all eigenvalues share one real part: Alg. 3 finds no shift")
    S = gsign_def(A - shift * np.eye(n))
    Qp, Qm, sp, sm = hyp_basis_ldl(S, s)
    V0 = np.hstack([Qp, Qm])
    s0 = np.r_[sp, sm]
    B = ((s0[:, None] * V0.T) * s[None, :]) @ A @ V0            # V0^dagger A V0, V0^dagger = Sigma_0 V0^T Sigma
    r = Qp.shape[1]
    V1, s1, D1 = geig_alg(B[:r, :r], sp) if r else (np.zeros((0, 0)), np.zeros(0), np.zeros((0, 0)))
    V2, s2, D2 = geig_alg(B[r:, r:], sm) if n - r else (np.zeros((0, 0)), np.zeros(0), np.zeros((0, 0)))
    Z = np.zeros((r, n - r))
    V = V0 @ np.block([[V1, Z], [Z.T, V2]])
    D = np.block([[D1, Z], [Z.T, D2]])
    return V, np.r_[s1, s2], D


def block_eigenvalues(D):
    """The eigenvalues of a block-diagonal D with 1 x 1 and 2 x 2 blocks (as geig_alg
    returns it): the 1 x 1 entries and, per 2 x 2 block, the roots of its characteristic
    polynomial x^2 - tr x + det, sorted by real part, then imaginary part."""
    n = D.shape[0]
    vals, i = [], 0
    while i < n:
        if i + 1 < n and (D[i + 1, i] != 0.0 or D[i, i + 1] != 0.0):
            tr, det = D[i, i] + D[i + 1, i + 1], D[i, i] * D[i + 1, i + 1] - D[i, i + 1] * D[i + 1, i]
            disc = complex(tr * tr - 4.0 * det)
            root = disc ** 0.5
            vals += [(tr - root) / 2.0, (tr + root) / 2.0]
            i += 2
        else:
            vals.append(complex(D[i, i]))
            i += 1
    return np.array(sorted(vals, key=lambda z: (round(z.real, 12), z.imag)))
