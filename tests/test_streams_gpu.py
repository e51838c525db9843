"""Calls on several CUDA streams at once: the torch wrappers give every
stream its own cached workspace, so concurrent reductions on different
streams return exactly what they return alone."""
import pytest
import torch

from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_cs_0603115_gb300 as ff


def test_concurrent_reductions_on_separate_streams():
    n = 1 << 22
    data = [inputs.ill_dot(n, 1e6, inputs.seed_for(2, 40 + i), device="cuda") for i in range(4)]
    want = [(ff.dot(g.x, g.y).clone(), ff.sum(g.x).clone(), ff.dot2(g.x[:, 0].contiguous(), g.y[:, 0].contiguous()).clone())
            for g in data]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in data]
    for _ in range(3):
        got = []
        for g, s in zip(data, streams):
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                x32, y32 = g.x[:, 0].contiguous(), g.y[:, 0].contiguous()
                got.append((ff.dot(g.x, g.y), ff.sum(g.x), ff.dot2(x32, y32)))
        torch.cuda.synchronize()
        for w, r in zip(want, got):
            for a, b in zip(w, r):
                assert torch.equal(a.view(torch.int32), b.view(torch.int32))
