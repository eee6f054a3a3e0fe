"""Batched execution of independent plans (p3_batch_*): every plan's result
equals the same plan run alone, bit for bit (the same kernels run, only on
other streams), with plain calls and replayed from a captured CUDA graph."""
import numpy as np
import pytest

from paper_1905_02803_gb300 import inputs

pytestmark = pytest.mark.gpu

GRIDS = [((512, 256, 6), "f32", "zyx"), ((48, 60, 35), "f32", "zyx"), ((96, 80, 72), "f32", "xyz"),
         ((30, 14, 9), "f64", "zyx"), ((64, 64, 64), "f32", "xyz"), ((2, 3, 5), "f64", "xyz"),
         ((384, 360, 12), "f32", "zyx")]


def _setup():
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    plans, xs = [], []
    for k, ((nx, ny, nz), prec, layout) in enumerate(GRIDS):
        p = Plan(nx, ny, nz, precision=prec, layout=layout)
        plans.append(p)
        xs.append(torch.from_numpy(inputs.uniform_field((nz, ny, nx), 40 + k)).to("cuda", p.real_dtype))
    return plans, xs


@pytest.mark.parametrize("nstreams", [1, 3, 16])
def test_batch_matches_single_plans(nstreams):
    import torch
    from paper_1905_02803_gb300.p3dfft import Batch
    plans, xs = _setup()
    ref_X = [p.forward(x) for p, x in zip(plans, xs)]
    ref_y = [p.backward(X) for p, X in zip(plans, ref_X)]
    torch.cuda.synchronize()
    b = Batch(plans, nstreams=nstreams)
    Xs = b.forward(xs)
    ys = b.backward(Xs)
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(Xs[i], ref_X[i]), i
        assert torch.equal(ys[i], ref_y[i]), i


def test_batch_in_cuda_graph():
    import torch
    from paper_1905_02803_gb300.p3dfft import Batch
    plans, xs = _setup()
    ref_X = [p.forward(x) for p, x in zip(plans, xs)]
    ref_y = [p.backward(X) for p, X in zip(plans, ref_X)]
    b = Batch(plans, nstreams=4)
    Xs = [p.empty_complex() for p in plans]
    ys = [p.empty_real() for p in plans]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        b.forward(xs, Xs)
        b.backward(Xs, ys)
        torch.cuda.synchronize()
        for X in Xs:
            X.zero_()
        for y in ys:
            y.zero_()
        with torch.cuda.graph(g, stream=s):
            b.forward(xs, Xs)
            b.backward(Xs, ys)
    torch.cuda.synchronize()
    for X in Xs:
        X.zero_()
    g.replay()
    torch.cuda.synchronize()
    for i in range(len(plans)):
        assert torch.equal(Xs[i], ref_X[i]), i
        assert torch.equal(ys[i], ref_y[i]), i
