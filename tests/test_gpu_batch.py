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


# Persistent mode: one launch per call over every stage of every plan
# (FP32 plans, the generic stage kernel for every stage)
P_GRIDS = [((512, 256, 6), ("fft", "fft", "fft"), "zyx"), ((48, 60, 35), ("fft", "fft", "fft"), "zyx"),
           ((96, 80, 72), ("fft", "fft", "fft"), "xyz"), ((64, 64, 64), ("fft", "fft", "fft"), "xyz"),
           ((384, 360, 12), ("fft", "fft", "fft"), "zyx"), ((22, 13, 97), ("fft", "fft", "fft"), "zyx"),
           ((15, 9, 7), ("fft", "fft", "fft"), "xyz"), ((40, 12, 33), ("fft", "fft", "cheb"), "zyx"),
           ((36, 10, 31), ("fft", "fft", "sine"), "zyx"), ((20, 6, 5), ("fft", "empty", "empty"), "zyx"),
           ((1, 1, 1), ("fft", "fft", "fft"), "zyx")]


def _setup_persistent():
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    plans, xs, Gs = [], [], []
    for k, ((nx, ny, nz), tt, layout) in enumerate(P_GRIDS):
        p = Plan(nx, ny, nz, precision="f32", ttypes=tt, layout=layout)
        plans.append(p)
        xs.append(torch.from_numpy(inputs.uniform_field((nz, ny, nx), 60 + k)).to("cuda", torch.float32))
        n = 2 * p.H * ny * nz
        g = torch.from_numpy(inputs.normal(70 + k, 1, n).astype(np.float32)).cuda()
        Gs.append(torch.view_as_complex(g.view(*p.complex_shape, 2)))
    return plans, xs, Gs


def _rel(a, b):
    import torch
    a = a.to(torch.complex128) if a.is_complex() else a.double()
    b = b.to(torch.complex128) if b.is_complex() else b.double()
    n = b.abs().norm().item()
    return (a - b).abs().norm().item() / (n if n > 0 else 1.0)


def test_persistent_batch_matches_plans_and_oracle():
    import torch
    import oracle as O
    from paper_1905_02803_gb300 import p3dfft as P
    from paper_1905_02803_gb300.p3dfft import Batch
    from _gpu_helpers import TT
    plans, xs, Gs = _setup_persistent()
    b = Batch(plans, nstreams=0)
    assert b.launches(0) == 1 and b.launches(1) == 1
    Xs = b.forward(xs)
    ys = b.backward(Gs)
    torch.cuda.synchronize()
    assert P.p3_batch_wait_status(b.handle) == P.P3_OK
    for i, (p, x, G) in enumerate(zip(plans, xs, Gs)):
        assert _rel(Xs[i], p.forward(x)) <= 1e-6, i
        assert _rel(ys[i], p.backward(G)) <= 1e-6, i
        tt = tuple(TT[t] for t in p.ttypes)
        ref = O.forward(x.double().cpu().numpy(), tt)
        ref = O.to_zyx(ref) if p.layout == "zyx" else ref
        got = Xs[i].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) <= 2e-6 * max(np.linalg.norm(ref), 1e-30), i
        Gin = G.cpu().numpy().astype(np.complex128)
        refb = O.backward(O.from_zyx(Gin) if p.layout == "zyx" else Gin, p.nx, tt)
        assert np.linalg.norm(ys[i].double().cpu().numpy() - refb) <= 2e-6 * np.linalg.norm(refb), i


def test_persistent_batch_in_cuda_graph_and_repeated():
    """Replays of a captured persistent call, and plain repeated calls, give
    the same bits (a tile's arithmetic does not depend on which CTA takes
    its ticket)."""
    import torch
    from paper_1905_02803_gb300.p3dfft import Batch
    plans, xs, Gs = _setup_persistent()
    b = Batch(plans, nstreams=0)
    ref_X = [X.clone() for X in b.forward(xs)]
    ref_y = [y.clone() for y in b.backward(Gs)]
    Xs = [p.empty_complex() for p in plans]
    ys = [p.empty_real() for p in plans]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        b.forward(xs, Xs)
        b.backward(Gs, ys)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            b.forward(xs, Xs)
            b.backward(Gs, ys)
    torch.cuda.synchronize()
    for _ in range(2):
        for X in Xs:
            X.zero_()
        for y in ys:
            y.zero_()
        g.replay()
        torch.cuda.synchronize()
        for i in range(len(plans)):
            assert torch.equal(Xs[i], ref_X[i]), i
            assert torch.equal(ys[i], ref_y[i]), i


def test_persistent_batch_wait_gives_up_and_reports():
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    from paper_1905_02803_gb300.p3dfft import Batch
    plans, xs, Gs = _setup_persistent()
    b = Batch(plans, nstreams=0)
    P.p3_batch_set_wait_limits(b.handle, 500, 1)
    b.forward(xs)
    torch.cuda.synchronize()
    assert P.p3_batch_wait_status(b.handle) == P.P3_ERR_TIMEOUT
    assert P.p3_batch_wait_status(b.handle) == P.P3_OK
    P.p3_batch_set_wait_limits(b.handle, 1 << 23, 0)
    Xs = b.forward(xs)
    torch.cuda.synchronize()
    assert P.p3_batch_wait_status(b.handle) == P.P3_OK
    for p, x, X in zip(plans, xs, Xs):
        assert _rel(X, p.forward(x)) <= 1e-6


def test_persistent_batch_rejects_fp64_and_stream_mode_counts_launches():
    from paper_1905_02803_gb300 import p3dfft as P
    from paper_1905_02803_gb300.p3dfft import Batch, Plan
    p32 = Plan(16, 8, 4, precision="f32")
    p64 = Plan(16, 8, 4, precision="f64")
    st, h = P.p3_batch_create([p32.handle, p64.handle], 0, check=False)
    assert st == P.P3_ERR_UNSUPPORTED and h is None
    b = Batch([p32, p64], nstreams=2)
    assert b.launches(0) == p32.launches(0) + p64.launches(0)
    assert P.p3_batch_wait_status(b.handle) == P.P3_OK
