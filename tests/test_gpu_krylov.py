"""The Krylov loops behind the bounds of Alg. 8 (largest eigenvalues of M and of
L^{-T} L^{-1}), the shift search of Alg. 2 (Lanczos quadrature nodes) and the
screening of a shift (power iteration on R^{-T} R^{-1}): the one-launch cluster
kernel against the step-by-step launches and against the three-term recurrence
and the power iteration written out in numpy from the same starting vector, on
sizes that leave the cluster's CTAs ragged or empty."""
import numpy as np
import pytest
import torch

import casida_inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2203_08900_gb300 import build as b
    b.build()
    import paper_2203_08900_gb300 as P
    P.lib()
    return P


def _sym(m, seed):
    rng = np.random.default_rng(seed)
    Q = G.haar(rng, m)
    w = np.sort(rng.uniform(-1.0, 3.0, m))
    return 0.5 * ((Q * w) @ Q.T + ((Q * w) @ Q.T).T)


def _lower(m, seed):
    """L^{-1} of an SPD matrix's Cholesky factor (what the screening and the bounds apply)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((m, m))
    L = np.linalg.cholesky(Z @ Z.T / m + 0.5 * np.eye(m))
    Li = np.linalg.inv(L)
    Li[np.triu_indices(m, 1)] = 7.0      # never read: the operator takes the lower triangle
    return Li


def _op(A, op):
    if op == 0:
        return A
    L = np.tril(A)
    return L.T @ L


def _lanczos_np(Aop, v0, steps):
    """alpha_j = v_j^T A v_j, w = A v_j - alpha_j v_j - beta_{j-1} v_{j-1}, beta_j = ||w||."""
    v = v0 / np.linalg.norm(v0)
    vp = np.zeros_like(v)
    al, be = np.zeros(steps), np.zeros(steps)
    b = 0.0
    for j in range(steps):
        w = Aop @ v
        al[j] = v @ w
        w = w - al[j] * v - b * vp
        be[j] = np.linalg.norm(w)
        vp, v, b = v, (w / be[j] if be[j] > 0 else 0 * w), be[j]
    return al, be


def _ritz(al, be):
    s = len(al)
    T = np.diag(al) + np.diag(be[:s - 1], 1) + np.diag(be[:s - 1], -1)
    return np.linalg.eigvalsh(T)


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("m", [1, 9, 64, 200, 777, 1024])
def test_lanczos_fused_matches(P, op, m):
    A = _sym(m, 100 + m) if op == 0 else _lower(m, 200 + m)
    Ad = torch.from_numpy(A).cuda()
    steps = min(m, 24)
    outs = {}
    for fused in (False, True):
        out, v0 = P.test_krylov(Ad, op=op, steps=steps, seed=0x1a2c05 + m, fused=fused)
        outs[fused] = out.cpu().numpy()
    v0 = v0.cpu().numpy()
    Aop = _op(A, op)
    nrm = np.linalg.norm(Aop, 2)
    al_np, be_np = _lanczos_np(Aop, v0, steps)
    for fused, out in outs.items():
        al, be = out[:steps], out[steps + 1:2 * steps + 1]
        k = min(steps, 6)              # before the recurrence's rounding is amplified
        assert np.max(np.abs(al[:k] - al_np[:k])) <= 1e-12 * nrm, fused
        kb = min(k, steps - 1)         # the last beta of a full-length run is rounding noise
        assert np.max(np.abs(be[:kb] - be_np[:kb]), initial=0.0) <= 1e-12 * nrm, fused
        th, th_np = _ritz(al, be), _ritz(al_np, be_np)
        assert abs(th[-1] - th_np[-1]) <= 1e-10 * nrm and abs(th[0] - th_np[0]) <= 1e-10 * nrm, fused
        ev = np.linalg.eigvalsh(Aop)
        assert th[-1] <= ev[-1] + 1e-12 * nrm and th[0] >= ev[0] - 1e-12 * nrm   # Cauchy interlacing
    s = min(steps, 6)
    assert np.max(np.abs(outs[True][:s] - outs[False][:s])) <= 1e-12 * nrm


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("m", [9, 130, 1000])
def test_power_fused_matches(P, op, m):
    A = _sym(m, 300 + m) if op == 0 else _lower(m, 400 + m)
    if op == 0:
        A = A @ A.T                   # SPD, as the bounds apply it
    Ad = torch.from_numpy(A).cuda()
    iters = 20
    res = {}
    for fused in (False, True):
        out, v0 = P.test_krylov(Ad, op=op, power=iters, fused=fused)
        res[fused] = float(out.cpu()[0])
    v = v0.cpu().numpy()
    Aop = _op(A, op)
    v = v / np.linalg.norm(v)
    for _ in range(iters):
        w = Aop @ v
        v = w / np.linalg.norm(w)
    rq = v @ (Aop @ v)
    for fused, r in res.items():
        assert abs(r - rq) <= 1e-12 * abs(rq), (fused, r, rq)
        assert r <= np.linalg.eigvalsh(Aop)[-1] * (1 + 1e-12)


def test_fused_size_limit(P):
    """The cluster kernel keeps whole vectors in shared memory: order 1025 is refused
    with the argument status, the step-by-step loop takes it."""
    m = 1025
    Ad = torch.from_numpy(_sym(m, 5)).cuda()
    with pytest.raises(P.PssdError) as e:
        P.test_krylov(Ad, steps=4, fused=True)
    assert e.value.status == -3
    out, _ = P.test_krylov(Ad, steps=4, fused=False)
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("m", [256, 1024])
def test_fused_is_one_launch_and_timed(P, m):
    """The fused loop is one launch (the step-by-step loop: four per Lanczos step plus two
    to start); both are timed with CUDA events after a warm-up and reported (each call also
    holds the hook's host synchronisation)."""
    Ad = torch.from_numpy(_sym(m, 600 + m)).cuda()
    h = P._handle(None)
    times, launches = {}, {}
    for fused in (True, False):
        P.test_krylov(Ad, steps=24, fused=fused, want_v0=False)
        torch.cuda.synchronize()
        l0 = h.launch_count()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            P.test_krylov(Ad, steps=24, fused=fused, want_v0=False)
        e1.record()
        torch.cuda.synchronize()
        launches[fused] = (h.launch_count() - l0) / 10
        times[fused] = e0.elapsed_time(e1) / 10
    print(f"\nLanczos 24 steps m={m}: fused {times[True] * 1e3:.0f} us ({launches[True]:.0f} launch), "
          f"step by step {times[False] * 1e3:.0f} us ({launches[False]:.0f} launches)")
    assert launches[True] == 1
    assert launches[False] == 2 + 4 * 24
