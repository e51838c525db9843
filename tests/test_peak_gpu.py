"""The FMA throughput probe computes what it claims: with a = b = 1 every
chain advances by exactly one per round, so each thread's sum of its eight
chains (started at 0..7) is 28 + 8 iters, in binary32 and binary64."""
import pytest
import torch

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_cs_0603115_gb300 as ff


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("iters", [0, 1, 3, 5, 1000])
def test_fma_probe_counts_every_round(f64, iters):
    out = ff.fma_peak(f64, iters, blocks=3, threads=64)
    torch.cuda.synchronize()
    assert out.numel() == 192
    assert bool((out == 28 + 8 * iters).all())
