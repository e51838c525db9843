"""Calls on several CUDA streams at once: the torch wrappers give every
stream its own cached workspace, so concurrent reductions on different
streams return exactly what they return alone; and reductions replayed
from a CUDA graph, which reuse one workspace without a memset."""
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


def test_reductions_replayed_from_a_cuda_graph():
    """A reduction workspace is zeroed once and every reduction leaves its
    arrival ticket zero again, so a CUDA graph of reductions, captured after
    the stream's workspace exists (no memset is captured with them), gives
    the eager bits on every replay.  The outputs are overwritten with NaN
    between replays, so each replay must write them again."""
    n = (1 << 22) + 5
    g = inputs.ill_dot(n, 1e6, inputs.seed_for(2, 48), device="cuda")
    x32, y32 = g.x[:, 0].contiguous(), g.y[:, 0].contiguous()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        calls = [lambda: ff.dot(g.x, g.y), lambda: ff.sum(g.x), lambda: ff.dot2(x32, y32), lambda: ff.sum2(x32)]
        want = [c().clone() for c in calls]
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        got = [c() for c in calls]
    for _ in range(5):
        for o in got:
            o.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        for w, r in zip(want, got):
            assert torch.equal(w.view(torch.int32), r.view(torch.int32))
    del graph
