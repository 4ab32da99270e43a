"""Parity of the tcgen05 tensor-core FP32 GEMM (3xTF32, TMA + TMEM) and of the
FP32 SIMT GEMM against an FP64 reference of the same operation, over tile
edges, ragged k, transposes, triangular operands, lower-only output, inner
scaling and batches."""
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


def _ref(A, B, ta, tb, triA, triB, lowerC, alpha, beta, Cin, ks):
    A = A.double(); B = B.double()
    opA = A.transpose(-1, -2) if ta else A
    opB = B.transpose(-1, -2) if tb else B
    if triA == 1: opA = torch.tril(opA)
    if triA == 2: opA = torch.triu(opA)
    if triB == 1: opB = torch.tril(opB)
    if triB == 2: opB = torch.triu(opB)
    if ks is not None:
        opA = opA * ks.double()[None, :]
    C = alpha * (opA @ opB)
    if beta != 0.0:
        C = C + beta * Cin.double()
    return C, opA.abs() @ opB.abs()


CASES = [
    # m, n, k, ta, tb, triA, triB, lowerC, beta, kscale, batch
    (128, 128, 128, 0, 0, 0, 0, 0, 0.0, False, 1),
    (200, 130, 77, 0, 0, 0, 0, 0, 0.0, False, 1),
    (384, 384, 300, 1, 1, 0, 0, 0, 0.5, False, 1),
    (256, 256, 256, 1, 0, 2, 1, 1, 0.0, False, 2),     # R^{-T} R^{-1}-type product, lower output
    (300, 64, 300, 0, 1, 0, 2, 0, 0.0, False, 1),      # X L^{-T}-type product
    (260, 260, 260, 1, 0, 2, 1, 1, 0.0, True, 1),      # L^T Sigma L
    (129, 257, 33, 0, 0, 1, 0, 0, -1.0, False, 3),
]


@pytest.mark.parametrize("use_tc", [True, False])
@pytest.mark.parametrize("m,n,k,ta,tb,triA,triB,lowerC,beta,ks,batch", CASES)
def test_f32_gemm(P, use_tc, m, n, k, ta, tb, triA, triB, lowerC, beta, ks, batch):
    g = torch.Generator(device="cuda"); g.manual_seed(m * 7 + n * 3 + k)
    A = torch.randn(batch, k if ta else m, m if ta else k, device="cuda", generator=g)
    B = torch.randn(batch, n if tb else k, k if tb else n, device="cuda", generator=g)
    Cin = torch.randn(batch, m, n, device="cuda", generator=g)
    kscale = (torch.randint(0, 2, (k,), device="cuda", generator=g).float() * 2 - 1) if ks else None
    alpha = 0.75
    C = P.test_gemm_f32(A, B, use_tc=use_tc, ta=ta, tb=tb, triA=triA, triB=triB, lowerC=lowerC, alpha=alpha,
                        beta=beta, Cin=Cin, kscale=kscale)
    Cref, mag = _ref(A, B, ta, tb, triA, triB, lowerC, alpha, beta, Cin, kscale)
    if lowerC:
        mask = torch.tril(torch.ones(m, n, dtype=torch.bool, device="cuda"))
        C = torch.where(mask, C.double(), torch.zeros((), dtype=torch.float64, device="cuda"))
        Cref = torch.where(mask, Cref, torch.zeros((), dtype=torch.float64, device="cuda"))
    err = (C.double() - Cref).abs()
    bound = 1e-5 * (abs(alpha) * mag + abs(beta) * Cin.double().abs()) + 1e-30
    assert torch.all(err <= bound + 1e-6 * mag.max()), float((err / bound).max())
