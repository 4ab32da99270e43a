"""The allocation-free sign entry point (pssd_sign_noalloc).

Some callers cannot let a library call cudaMalloc: applications whose device
memory is owned by their own pool or caching allocator, and latency-critical
loops that cannot take the synchronisation an allocation can cause.  This entry
point must compute what pssd_sign computes while taking every temporary from the
library's fixed device scratch array.  Checked through the C ABI against
pssd_sign on two calls in a row (the shared scratch keeps the previous call's
contents, which must not leak into the next result), in each precision mode,
together with the absence of device allocations, the order limit and a call
whose temporaries cannot fit (a large explicit r), which must stop cleanly.

This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

import casida_inputs as G

pytestmark = pytest.mark.gpu

NOALLOC_TOO_LARGE = 9


@pytest.fixture(scope="module")
def P():
    from paper_2203_08900_gb300 import build as b
    b.build()
    import paper_2203_08900_gb300 as P
    P.lib()
    return P


def _call(P, h, H, S, **kw):
    L = P.lib()
    n = H.shape[0]
    info = P.Info()
    o = P._opts(**kw)
    st = L.pssd_sign_noalloc(h._h, n, None, ctypes.c_void_p(H.data_ptr()), H.stride(0),
                             ctypes.c_void_p(S.data_ptr()), S.stride(0), ctypes.byref(o), ctypes.byref(info))
    return st, info


# relative tolerance of the comparison with pssd_sign: the same computation on
# the same kernels, so the results agree to rounding (FP32 rounding order is the
# same too, so the mixed path agrees as closely)
TOL = {"fp64": 1e-13, "fp64e": 1e-13, "mixed": 1e-13}


@pytest.mark.parametrize("precision", ["fp64", "fp64e", "mixed"])
def test_noalloc_matches_pssd_sign_two_calls(P, precision):
    prec = {"fp64": P.PSSD_FP64, "fp64e": P.PSSD_FP64_EMULATED, "mixed": P.PSSD_MIXED}[precision]
    h = P.Handle()
    inputs = [G.casida(50, ("uniform", 1.0, 10.0), seed=1)[0],            # n = 100
              G.casida(64, ("loguniform", 1e-2, 1e2), seed=2)[0]]         # n = 128 (the limit)
    Hs = [torch.from_numpy(x).cuda() for x in inputs]
    outs = [torch.empty_like(x) for x in Hs]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    a0 = P.device_alloc_count()
    for H, S in zip(Hs, outs):                       # two calls in a row on the shared scratch
        st, info = _call(P, h, H, S, precision=prec)
        assert st == 0, P.lib().pssd_status_string(st).decode() + " " + P.lib().pssd_last_cuda_error(h._h).decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert P.device_alloc_count() == a0              # the library made no device allocation
    # no workspace allocation (pssd_sign's first call takes >= 1 GiB); the 8 MiB scratch array
    # itself may be mapped in by the first call when the module loads lazily
    assert free0 - free1 < (64 << 20)
    for H, S in zip(Hs, outs):
        S_ref, _ = P.sign(H, precision=prec)
        n = H.shape[0]
        err = torch.linalg.norm(S - S_ref).item() / torch.linalg.norm(S_ref).item()
        assert err <= TOL[precision], err
        I = torch.eye(n, dtype=torch.float64, device=H.device)
        s2 = max(1.0, torch.linalg.matrix_norm(S_ref, 2).item()) ** 2
        assert torch.linalg.norm(S @ S - I).item() <= 1e-12 * n * s2


def test_noalloc_rejects_large_n(P):
    h = P.Handle()
    H = torch.from_numpy(G.casida(65, ("uniform", 1.0, 10.0), seed=3)[0]).cuda()   # n = 130 > 128
    S = torch.empty_like(H)
    st, _ = _call(P, h, H, S)
    assert st == NOALLOC_TOO_LARGE
    assert "scratch" in P.lib().pssd_status_string(st).decode()


def test_noalloc_overflow_stops_without_allocating(P):
    """r = 64 at n = 128 needs 2 x 64 n^2 doubles (16 MiB) for the shifted
    factors alone: the call stops when a temporary would overflow the 8 MiB
    array, returns the size status and allocates nothing; the next call on the
    same handle works."""
    h = P.Handle()
    H = torch.from_numpy(G.casida(64, ("uniform", 1.0, 10.0), seed=4)[0]).cuda()
    S = torch.empty_like(H)
    a0 = P.device_alloc_count()
    st, _ = _call(P, h, H, S, r=64)
    torch.cuda.synchronize()
    assert st == NOALLOC_TOO_LARGE
    assert P.device_alloc_count() == a0              # stopped instead of allocating
    st, _ = _call(P, h, H, S)
    assert st == 0
