"""Parity of the float-float GEMM (ff_gemm, through the C ABI) with the CPU
oracle: every element bit-identical to the oracle's in-order Add22
accumulation of Mul22 terms, for shapes that span several 64 x 64 tiles and
16-deep slices with ragged tails, all four transpose combinations, padded
leading dimensions, an empty inner dimension, special values, the adjoints of
the autograd function, writes confined to C, and sampled rows of a
4096 x 4096 x 4096 product.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import _lib

DEV = "cuda"


def same_bits(got, want):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    assert got.shape == want.shape
    nan = np.isnan(got) & np.isnan(want)
    eq = (got.view(np.uint32) == want.view(np.uint32)) | nan
    if not eq.all():
        bad = np.argwhere(~eq)[:5]
        raise AssertionError(f"{(~eq).sum()} mismatches, first at {bad.tolist()}")


def operands(m, n, k, seed, transa=False, transb=False):
    g = inputs.gemm(m, n, k, seed)
    A = g.A.permute(1, 0, 2).contiguous() if transa else g.A
    B = g.B.permute(1, 0, 2).contiguous() if transb else g.B
    return A, B


SHAPES = [(1, 1, 1), (64, 64, 16), (130, 67, 50), (1, 200, 33), (77, 1, 300), (65, 129, 17), (200, 190, 64)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_gemm_bitexact(m, n, k):
    A, B = operands(m, n, k, inputs.seed_for(6, m % 16))
    C = ff.gemm(A.to(DEV), B.to(DEV)).cpu().numpy()
    same_bits(C, oracle.gemm(A.numpy(), B.numpy()))


@pytest.mark.parametrize("transa,transb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(130, 67, 50), (65, 129, 17), (3, 70, 129)])
def test_gemm_transposes_bitexact(m, n, k, transa, transb):
    A, B = operands(m, n, k, inputs.seed_for(6, 20 + transa + 2 * transb), bool(transa), bool(transb))
    C = ff.gemm(A.to(DEV), B.to(DEV), transa=bool(transa), transb=bool(transb)).cpu().numpy()
    same_bits(C, oracle.gemm(A.numpy(), B.numpy(), transa=bool(transa), transb=bool(transb)))


@pytest.mark.parametrize("transa,transb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_many_ragged_tiles_bitexact(transa, transb):
    """1285 x 1097 (ragged in both directions): 21 x 18 = 378 tiles, more
    than one wave of resident blocks, every element equal to the oracle's
    in-order loop."""
    m, n, k = 1285, 1097, 24
    A, B = operands(m, n, k, inputs.seed_for(6, 50 + transa + 2 * transb), bool(transa), bool(transb))
    C = ff.gemm(A.to(DEV), B.to(DEV), transa=bool(transa), transb=bool(transb)).cpu().numpy()
    same_bits(C, oracle.gemm(A.numpy(), B.numpy(), transa=bool(transa), transb=bool(transb)))


def test_gemm_padded_leading_dimensions_and_guards():
    """lda, ldb, ldc larger than the rows; nothing outside C's m x n block
    (the padding columns and the rows around it) is written."""
    m, n, k = 70, 45, 37
    pa, pb, pc = 3, 5, 7
    g = inputs.gemm(m, n, k, inputs.seed_for(6, 30))
    Ap = torch.zeros((m, k + pa, 2)); Ap[:, :k] = g.A
    Bp = torch.zeros((k, n + pb, 2)); Bp[:, :n] = g.B
    sentinel = np.array([0x7FC0DEAD], np.uint32).view(np.float32)[0]
    guard = 8
    Cbuf = torch.full((m * (n + pc) + 2 * guard, 2), float(sentinel), device=DEV)
    Ad, Bd = Ap.to(DEV), Bp.to(DEV)
    Cview = Cbuf[guard:]
    _lib.call("ff_gemm", 0, 0, m, n, k, Ad.data_ptr(), k + pa, Bd.data_ptr(), n + pb, Cview.data_ptr(), n + pc,
              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    buf = Cbuf.cpu().numpy()
    body = buf[guard:guard + m * (n + pc)].reshape(m, n + pc, 2)
    same_bits(body[:, :n], oracle.gemm(g.A.numpy(), g.B.numpy()))
    s = np.uint32(0x7FC0DEAD)
    assert (body[:, n:].view(np.uint32) == s).all()
    assert (buf[:guard].view(np.uint32) == s).all() and (buf[guard + m * (n + pc):].view(np.uint32) == s).all()


def test_gemm_empty_inner_dimension_writes_zeros():
    A = torch.zeros((5, 0, 2), device=DEV)
    B = torch.zeros((0, 9, 2), device=DEV)
    C = ff.gemm(A, B, out=torch.full((5, 9, 2), 7.0, device=DEV)).cpu().numpy()
    same_bits(C, np.zeros((5, 9, 2), np.float32))
    assert ff.gemm(torch.zeros((0, 4, 2), device=DEV), torch.zeros((4, 3, 2), device=DEV)).shape == (0, 3, 2)


def test_gemm_special_values_follow_the_oracle():
    m, n, k = 20, 19, 40
    A, B = operands(m, n, k, inputs.seed_for(6, 31))
    A = A.clone(); B = B.clone()
    A[0, 3, 0] = float("inf"); A[1, 5] = float("nan"); A[2, 7] = -0.0
    B[4, 2, 0] = float("-inf"); B[9, 0, 0] = 0.0; B[9, 0, 1] = 0.0
    A[3, 1, 0] = 1e-40; B[1, 3, 0] = 3e-39     # subnormal operands and products
    C = ff.gemm(A.to(DEV), B.to(DEV)).cpu().numpy()
    same_bits(C, oracle.gemm(A.numpy(), B.numpy()))


def test_gemm_autograd_adjoints_bitexact():
    m, n, k = 70, 33, 90
    g = inputs.gemm(m, n, k, inputs.seed_for(6, 32))
    A = g.A.to(DEV).requires_grad_(True)
    B = g.B.to(DEV).requires_grad_(True)
    C = ff.ffgemm(A, B)
    same_bits(C.detach().cpu().numpy(), oracle.gemm(g.A.numpy(), g.B.numpy()))
    C.backward(g.dC.to(DEV))
    same_bits(A.grad.cpu().numpy(), oracle.gemm(g.dC.numpy(), g.B.numpy(), transb=True))
    same_bits(B.grad.cpu().numpy(), oracle.gemm(g.A.numpy(), g.dC.numpy(), transa=True))
    # against the float64 gradient dC B^T of the exact values (normwise)
    f64 = lambda t: t[..., 0].double() + t[..., 1].double()
    dA64 = f64(g.dC) @ f64(g.B).T
    got = f64(A.grad.cpu())
    scale = f64(g.dC).abs() @ f64(g.B).abs().T
    assert ((got - dA64).abs() <= n * 2.0 ** -44 * scale + 1e-300).all()


def test_gemm_full_size_sampled_rows():
    """4096 x 4096 x 4096: eight sampled rows of C recomputed by the oracle
    (same in-order accumulation) are bit-identical, and sampled elements are
    within k 2^-44 sum|a b| of the exact value."""
    m = n = k = 4096
    g = inputs.gemm(m, n, k, inputs.seed_for(6, 40), device=DEV)
    C = ff.gemm(g.A, g.B)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(m, 8, replace=False))
    rows[0] = 0; rows[-1] = m - 1
    Bh = g.B.cpu().numpy()
    Ah = g.A[torch.as_tensor(rows, device=DEV)].cpu().numpy()
    want = oracle.gemm(Ah, Bh)
    got = C[torch.as_tensor(rows, device=DEV)].cpu().numpy()
    same_bits(got, want)
    for r in range(len(rows)):
        for j in rng.choice(n, 4, replace=False):
            _, _, Aabs, E = oracle.exact_dot(Ah[r], np.ascontiguousarray(Bh[:, j]), got[r, j])
            assert abs(E) <= k * 2.0 ** -44 * Aabs
