"""Batched diagonalisation (pssd_eig_batched): many independent Hamiltonians of
uneven orders in one call, each checked against the oracle and against the
single-instance entry point."""
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


def test_batched_matches_single_and_oracle(P):
    ks = [1, 3, 16, 17, 40, 64, 65, 100, 8, 33, 128, 2]
    Hn = [G.casida(k, ("uniform", 0.5, 50.0), seed=700 + i)[0] for i, k in enumerate(ks)]
    Hs = [torch.from_numpy(x).cuda() for x in Hn]
    Ds, Vs, infos = P.eig_batched(Hs)
    for H, Hd, D, V in zip(Hn, Hs, Ds, Vs):
        lam, _ = O.eig_def(H)
        D = D.cpu().numpy(); V = V.cpu().numpy()
        assert np.max(np.abs(D - lam)) <= 1e-10 * np.max(np.abs(lam))
        assert np.linalg.norm(H @ V - V * D) <= 1e-11 * np.linalg.norm(H)
        D1, V1, _ = P.eig(Hd)
        assert np.max(np.abs(D1.cpu().numpy() - D)) <= 1e-12 * np.max(np.abs(lam))


def test_batched_general_signatures_and_precision(P):
    mats = [G.example1(n, 1e2, seed=800 + n) for n in (10, 37, 90)]
    Hs = [torch.from_numpy(a).cuda() for a, _ in mats]
    sig = [s for _, s in mats]
    Ds, Vs, infos = P.eig_batched(Hs, sigmas=sig, precision=P.PSSD_FP64_EMULATED)
    for (A, s), D in zip(mats, Ds):
        lam, _ = O.eig_def(A, s.astype(float))
        assert np.max(np.abs(D.cpu().numpy() - lam)) <= 1e-9 * np.max(np.abs(lam))
    assert [i["p"] for i in infos] == [int((s > 0).sum()) for s in sig]


def test_batched_error_is_reported(P):
    good = G.casida(10, ("uniform", 1.0, 10.0), seed=1)[0]
    bad = good.copy(); bad[0, 1] += 1.0
    with pytest.raises(P.PssdError) as e:
        P.eig_batched([torch.from_numpy(good).cuda(), torch.from_numpy(bad).cuda()])
    assert e.value.status == 8
