"""Caller-owned workspace (pssd_workspace_bytes / pssd_set_workspace /
pssd_workspace_peak): the bound covers the measured peak of every driver and
precision mode, a buffer of exactly the peak gives the same results as the
library-managed workspace without any allocation by the library, and a buffer
that is too small is reported as PSSD_ERR_ALLOC with the handle still usable."""
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


def _H(k, seed):
    H, _, _ = G.casida(k, ("loguniform", 1e-2, 1e2), seed=seed)
    return torch.from_numpy(H).cuda()


@pytest.mark.parametrize("k", [128, 512])
@pytest.mark.parametrize("prec", ["fp64", "fp64e", "mixed"])
def test_bound_covers_peak(P, k, prec):
    pr = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED, "mixed": P.PSSD_MIXED}[prec]
    H = _H(k, 40 + k)
    n = 2 * k
    h = P.Handle()
    P.sign(H, handle=h, precision=pr)
    P.split(H, handle=h, precision=pr)
    P.eig(H, handle=h, precision=pr)
    peak = h.workspace_peak()
    bound = h.workspace_bytes(n, precision=pr)
    print(f"\n{prec} n={n}: peak {peak / (8 * n * n):.2f} n^2 doubles, bound {bound / (8 * n * n):.2f}")
    assert 0 < peak <= bound
    h.close()


def test_bound_covers_r8(P):
    H = _H(256, 7)
    h = P.Handle()
    P.eig(H, handle=h, r=8)
    assert h.workspace_peak() <= h.workspace_bytes(512, r=8)
    h.close()


def test_caller_workspace_same_results_no_allocation(P):
    H = _H(300, 3)
    h = P.Handle()
    Q0, A0, B0, p0, _ = P.split(H, handle=h, precision=P.PSSD_FP64_EMULATED)
    D0, V0, _ = P.eig(H, handle=h)
    peak = h.workspace_peak()
    # load the comparison kernels now: lazily loaded device code takes device memory too
    assert torch.allclose(Q0, Q0, rtol=0, atol=1e-13 * float(Q0.abs().max()))
    assert torch.allclose(D0, D0, rtol=0, atol=1e-13 * float(D0.abs().max()))
    buf = torch.empty(peak + 256, dtype=torch.uint8, device="cuda")   # room for the 256-byte alignment
    h.set_workspace(buf)
    torch.cuda.synchronize()
    free0, res0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(2):
        Q1, A1, B1, p1, _ = P.split(H, handle=h, precision=P.PSSD_FP64_EMULATED)
        D1, V1, _ = P.eig(H, handle=h)
        assert p1 == p0
        assert torch.allclose(Q1, Q0, rtol=0, atol=1e-13 * float(Q0.abs().max()))
        assert torch.allclose(A1, A0, rtol=0, atol=1e-13 * float(A0.abs().max()))
        assert torch.allclose(D1, D0, rtol=0, atol=1e-13 * float(D0.abs().max()))
    assert h.workspace_peak() <= buf.numel()
    # device memory taken meanwhile, minus what torch's caching allocator reserved for the
    # outputs and the comparisons: the library's own allocations (none expected)
    torch.cuda.synchronize()
    free1, res1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    assert (free0 - free1) - (res1 - res0) <= 8 * 2 ** 20
    h.close()


def test_too_small_workspace_is_an_error_and_recoverable(P):
    H = _H(200, 5)
    h = P.Handle()
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    h.set_workspace(buf)
    with pytest.raises(P.PssdError) as e:
        P.split(H, handle=h)
    assert e.value.status == 7
    h.set_workspace(None)
    Q, A11, A22, p, info = P.split(H, handle=h)
    assert p == 200 and torch.isfinite(Q).all()
    h.close()
