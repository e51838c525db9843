"""The torch wrappers refuse outputs and instances whose size, dtype,
contiguity or device would let a kernel write outside them: a ValueError,
raised before anything is launched."""
import pytest
import torch

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import batch

DEV = "cuda"


def test_outputs_of_the_wrong_shape_are_refused():
    a = torch.randn(100, 2, device=DEV)
    b = torch.randn(100, 2, device=DEV)
    with pytest.raises(ValueError):
        ff.add(a, b, out=torch.empty(99, 2, device=DEV))
    with pytest.raises(ValueError):
        ff.axpy((1.0, 0.0), a, b, out=torch.empty(50, 2, device=DEV))
    with pytest.raises(ValueError):
        ff.dot(a, b, out=torch.empty(1, device=DEV))
    with pytest.raises(ValueError):
        ff.sum(a, out=torch.empty(2, dtype=torch.float64, device=DEV))
    with pytest.raises(ValueError):
        ff.dot_backward(torch.tensor([1.0, 0.0], device=DEV), a, b, dx=torch.empty(10, 2, device=DEV))
    A = torch.randn(8, 6, 2, device=DEV)
    with pytest.raises(ValueError):
        ff.gemv(A, torch.randn(3, 6, 2, device=DEV), out=torch.empty(3, 7, 2, device=DEV))
    with pytest.raises(ValueError):
        ff.gemm(A, torch.randn(6, 5, 2, device=DEV), out=torch.empty(8, 4, 2, device=DEV))
    with pytest.raises(ValueError):
        ff.gemm(A, torch.randn(6, 5, 2, device=DEV), out=torch.empty(5, 8, 2, device=DEV).transpose(0, 1))
    with pytest.raises(ValueError):
        ff.f64_add(a.double(), b.double(), out=torch.empty(100, 2, device=DEV))
    with pytest.raises(ValueError):
        ff.dot(a.cpu(), b)


def test_batched_instances_of_the_wrong_size_are_refused():
    x = torch.randn(1000, 2, device=DEV)
    y = torch.randn(1000, 2, device=DEV)
    with pytest.raises(ValueError):
        batch.make_instances([(batch.AXPY, x, y, torch.empty(999, 2, device=DEV), (1.0, 0.0))])
    with pytest.raises(ValueError):
        batch.make_instances([(batch.DOT, x, y[:500], torch.empty(2, device=DEV), None)])
    with pytest.raises(ValueError):
        batch.make_instances([(batch.GEMV, x.view(10, 100, 2), y[:99], torch.empty(10, 2, device=DEV), None)])
    with pytest.raises(ValueError):
        batch.make_instances([(batch.DOT_GRAD, x, y, torch.empty_like(x), torch.empty_like(x), torch.empty(3, device=DEV))])
    # the valid forms still build
    batch.make_instances([(batch.DOT, x, y, torch.empty(2, device=DEV), None),
                          (batch.GEMV, x.view(10, 100, 2), y[:100], torch.empty(10, 2, device=DEV), None)])
