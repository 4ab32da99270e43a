"""Parity of the FP64-accurate GEMM engines -- integer slices on the BF16
tensor cores (engine 2), float pairs on the FP32 pipe (engine 1) and native
DFMA (engine 0) -- against an FP64 reference, including operands whose rows
span 2^60 in magnitude (the per-row/column power-of-two scaling)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2203_08900_gb300 import build as b
    b.build()
    import paper_2203_08900_gb300 as P
    P.lib()
    return P


def _ops(A, B, ta, tb, triA, triB, ks):
    opA = A.transpose(-1, -2) if ta else A
    opB = B.transpose(-1, -2) if tb else B
    if triA == 1: opA = torch.tril(opA)
    if triA == 2: opA = torch.triu(opA)
    if triB == 1: opB = torch.tril(opB)
    if triB == 2: opB = torch.triu(opB)
    if ks is not None:
        opA = opA * ks[None, :]
    return opA, opB


CASES = [
    # m, n, k, ta, tb, triA, triB, lowerC, beta, kscale, batch, wide
    (128, 64, 256, 0, 0, 0, 0, 0, 0.0, False, 1, False),
    (200, 130, 77, 0, 0, 0, 0, 0, 0.0, False, 1, False),
    (384, 320, 1000, 1, 1, 0, 0, 0, 0.5, False, 1, False),
    (256, 256, 256, 1, 0, 2, 1, 1, 0.0, False, 2, False),
    (300, 64, 300, 0, 1, 0, 2, 0, 0.0, False, 1, False),
    (260, 260, 260, 1, 0, 2, 1, 1, 0.0, True, 1, False),
    (129, 257, 33, 0, 0, 1, 0, 0, -1.0, False, 3, False),
    (192, 192, 600, 0, 0, 0, 0, 0, 0.0, False, 1, True),
]


@pytest.mark.parametrize("engine", [2, 1, 0])
@pytest.mark.parametrize("m,n,k,ta,tb,triA,triB,lowerC,beta,ks,batch,wide", CASES)
def test_f64_gemm(P, engine, m, n, k, ta, tb, triA, triB, lowerC, beta, ks, batch, wide):
    g = torch.Generator(device="cuda"); g.manual_seed(m * 11 + n * 5 + k + engine)
    A = torch.randn(batch, k if ta else m, m if ta else k, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(batch, n if tb else k, k if tb else n, device="cuda", dtype=torch.float64, generator=g)
    if wide:   # rows of op(A) and columns of op(B) scaled by 2^[-30, 30]
        ra = torch.exp2(torch.randint(-30, 31, (m,), device="cuda", generator=g).double())
        cb = torch.exp2(torch.randint(-30, 31, (n,), device="cuda", generator=g).double())
        A = A * ra[None, :, None]
        B = B * cb[None, None, :]
    Cin = torch.randn(batch, m, n, device="cuda", dtype=torch.float64, generator=g)
    kscale = (torch.randint(0, 2, (k,), device="cuda", generator=g).double() * 2 - 1) if ks else None
    alpha = 0.75
    C = P.test_gemm_f64(A, B, engine=engine, ta=ta, tb=tb, triA=triA, triB=triB, lowerC=lowerC, alpha=alpha,
                        beta=beta, Cin=Cin, kscale=kscale)
    opA, opB = _ops(A, B, ta, tb, triA, triB, kscale)
    Cref = alpha * (opA @ opB) + (beta * Cin if beta != 0.0 else 0.0)
    # error bound per entry: 2^-46 (k) max_p|opA_ip| max_p|opB_pj|  (+ the Cin term's rounding)
    ra = opA.abs().amax(dim=-1, keepdim=True)
    cb = opB.abs().amax(dim=-2, keepdim=True)
    bound = 2.0 ** -46 * k * abs(alpha) * ra * cb + 1e-15 * abs(beta) * Cin.abs() + 1e-300
    err = (C - Cref).abs()
    if lowerC:
        err = torch.tril(err)
    assert torch.all(err <= bound), float((err / bound).max())
