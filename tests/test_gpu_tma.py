"""TMA-staged forward Z stage (ZYX store): the input tile arrives by tensor
copies instead of per-thread loads; the arithmetic is the column kernel's, so
the result equals the plan with P3_FLAG_NO_TMA bit for bit, and the oracle
within the FP32 tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, TT, rel_l2

pytestmark = pytest.mark.gpu

CASES = [((64, 32, 1024), ("fft", "fft", "fft")), ((32, 24, 256), ("fft", "fft", "fft")),
         ((48, 20, 512), ("fft", "fft", "fft")), ((16, 8, 2048), ("fft", "fft", "fft")),
         ((40, 12, 257), ("fft", "fft", "cheb")), ((36, 10, 511), ("fft", "fft", "sine")),
         ((1024, 256, 1024), ("fft", "fft", "fft")), ((30, 7, 1025), ("fft", "empty", "cheb"))]


@pytest.mark.parametrize("shape,tt", CASES)
def test_tma_zyx_store_matches(shape, tt):
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    pt = P.Plan(nx, ny, nz, precision="f32", ttypes=tt, layout="zyx")
    pn = P.Plan(nx, ny, nz, precision="f32", ttypes=tt, layout="zyx", flags=P.P3_FLAG_NO_TMA)
    assert "zyx_store_tma" in pt.describe() and "zyx_store_tma" not in pn.describe(), pt.describe()
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), nz)).to("cuda", torch.float32)
    Xt, Xn = pt.forward(x), pn.forward(x)
    torch.cuda.synchronize()
    assert torch.equal(Xt, Xn)
    assert P.p3_plan_wait_status(pt.handle) == P.P3_OK
    if nx * ny * nz <= 1 << 22:
        ref = O.to_zyx(O.forward(x.double().cpu().numpy(), tuple(TT[t] for t in tt)))
        assert rel_l2(Xt.cpu().numpy(), ref) <= TOL["f32"]


@pytest.mark.parametrize("shape", [(1024, 1024, 64), (512, 256, 1024), (512, 512, 256), (1024, 256, 512)])
def test_bulk_zyx_load_matches(shape):
    """Inverse Z stage of a plane-fused ZYX plan (transposed planes): its
    input lines lie one after another, so the row-style kernel takes the
    tile with one bulk copy; bit-identical to P3_FLAG_NO_TMA."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    pt = P.Plan(nx, ny, nz, precision="f32", layout="zyx")
    pn = P.Plan(nx, ny, nz, precision="f32", layout="zyx", flags=P.P3_FLAG_NO_TMA)
    d = pt.describe()
    if nz >= 256:
        assert "pow2_zrow_bulk" in d, d
    assert "pow2_zrow_bulk" not in pn.describe()
    G = torch.from_numpy(np.asarray(inputs.normal(5, 1, 2 * (nx // 2 + 1) * ny * nz), dtype=np.float32)).cuda()
    X = torch.view_as_complex(G.view(nx // 2 + 1, ny, nz, 2))
    yt, yn = pt.backward(X), pn.backward(X)
    torch.cuda.synchronize()
    assert torch.equal(yt, yn)
    assert P.p3_plan_wait_status(pt.handle) == P.P3_OK


def test_tma_copy_wait_gives_up_and_reports():
    """The forward Z stage's wait for its tensor copies: with the test knob
    the barrier needs one arrival more than the copies make, so every wait
    runs out; the plan reports a copy wait (and no other kind), the launch
    finishes, and with the default limits the next call is exact again."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 64, 32, 1024
    pt = P.Plan(nx, ny, nz, precision="f32", layout="zyx", flags=P.P3_FLAG_NO_FUSE)
    pn = P.Plan(nx, ny, nz, precision="f32", layout="zyx", flags=P.P3_FLAG_NO_FUSE | P.P3_FLAG_NO_TMA)
    assert "zyx_store_tma" in pt.describe(), pt.describe()
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 11)).to("cuda", torch.float32)
    P.p3_plan_set_wait_limits(pt.handle, 2000, 1)
    pt.forward(x)
    torch.cuda.synchronize()
    assert P.p3_plan_wait_flags(pt.handle) == P.P3_WAIT_COPY
    assert P.p3_plan_wait_status(pt.handle) == P.P3_OK  # the mark was cleared
    P.p3_plan_set_wait_limits(pt.handle, 1 << 23, 0)
    Xt, Xn = pt.forward(x), pn.forward(x)
    torch.cuda.synchronize()
    assert P.p3_plan_wait_status(pt.handle) == P.P3_OK
    assert torch.equal(Xt, Xn)


def test_bulk_copy_wait_gives_up_and_reports():
    """The inverse Z stage's wait for its bulk-copied tile, the same way (the
    plan's plane-fused launch gives up too under the knob)."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 512, 256, 256
    pt = P.Plan(nx, ny, nz, precision="f32", layout="zyx")
    pn = P.Plan(nx, ny, nz, precision="f32", layout="zyx", flags=P.P3_FLAG_NO_TMA)
    assert "pow2_zrow_bulk" in pt.describe(), pt.describe()
    G = torch.from_numpy(np.asarray(inputs.normal(6, 1, 2 * (nx // 2 + 1) * ny * nz), dtype=np.float32)).cuda()
    X = torch.view_as_complex(G.view(nx // 2 + 1, ny, nz, 2))
    P.p3_plan_set_wait_limits(pt.handle, 2000, 1)
    pt.backward(X)
    torch.cuda.synchronize()
    assert P.p3_plan_wait_flags(pt.handle) & P.P3_WAIT_COPY
    P.p3_plan_set_wait_limits(pt.handle, 1 << 23, 0)
    yt, yn = pt.backward(X), pn.backward(X)
    torch.cuda.synchronize()
    assert P.p3_plan_wait_flags(pt.handle) == 0
    assert torch.equal(yt, yn)
