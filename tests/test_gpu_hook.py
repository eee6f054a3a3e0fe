"""User Z hook in place of the empty third-dimension transform (Sect. 3.1:
the empty transform lets the user substitute a transform of their own).

The hook here is a plain complex FFT along Z (torch.fft on the strided view
the library hands over), so the whole transform must then equal the oracle's
3D FFT; a failing hook must stop the call with P3_ERR_HOOK."""
import numpy as np
import pytest

import oracle as O
from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, random_complex, rel_l2

pytestmark = pytest.mark.gpu


def _fft_hook(calls):
    import torch

    def fn(lines, direction):
        calls.append((direction, tuple(lines.shape), tuple(lines.stride())))
        if direction == 0:
            lines.copy_(torch.fft.fft(lines, dim=1))
        else:
            lines.copy_(torch.fft.ifft(lines, dim=1, norm="forward"))  # unnormalised, + sign
    return fn


@pytest.mark.parametrize("shape", [(20, 12, 16), (33, 5, 9), (64, 16, 1)])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_z_hook_reproduces_the_fft(shape, layout, prec):
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    nx, ny, nz = shape
    H = nx // 2 + 1
    plan = Plan(nx, ny, nz, precision=prec, ttypes=("fft", "fft", "empty"), layout=layout)
    calls = []
    plan.set_z_hook(_fft_hook(calls))
    assert "z_hook" in plan.describe()
    f = inputs.uniform_field((nz, ny, nx), nx + nz)
    x = torch.from_numpy(f).to("cuda", plan.real_dtype)
    X = plan.forward(x)
    ref = O.forward(x.double().cpu().numpy())
    ref = O.to_zyx(ref) if layout == "zyx" else ref
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), ref) < TOL[prec]

    G = random_complex((nz, ny, H), 5)
    Gd = torch.from_numpy(O.to_zyx(G) if layout == "zyx" else G).to("cuda", plan.complex_dtype)
    G0 = Gd.clone()
    g = plan.backward(Gd)
    Gin = Gd.cpu().numpy().astype(np.complex128)
    refb = O.backward(O.from_zyx(Gin) if layout == "zyx" else Gin, nx)
    torch.cuda.synchronize()
    assert rel_l2(g.cpu().numpy(), refb) < TOL[prec]
    assert torch.equal(Gd, G0)  # the hook ran on a copy

    fwd_stride = (nz, 1) if layout == "zyx" else (1, H * ny)
    assert calls == [(0, (H * ny, nz), fwd_stride), (1, (H * ny, nz), (1, H * ny))]
    assert plan.launches(1) == 3


def test_z_hook_in_place_padded():
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan, P3_FLAG_PADDED_REAL
    nx, ny, nz = 32, 10, 12
    plan = Plan(nx, ny, nz, precision="f64", ttypes=("fft", "fft", "empty"), layout="xyz",
                flags=P3_FLAG_PADDED_REAL)
    plan.set_z_hook(_fft_hook([]))
    f = inputs.uniform_field((nz, ny, nx), 2)
    buf = torch.zeros(plan.real_shape, dtype=torch.float64, device="cuda")
    buf[..., :nx] = torch.from_numpy(f).cuda()
    X = plan.complex_view(buf)
    plan.forward(buf, out=X)
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), O.forward(f)) < TOL["f64"]
    plan.backward(X, out=buf)
    torch.cuda.synchronize()
    assert rel_l2(buf[..., :nx].cpu().numpy() / (nx * ny * nz), f) < 1e-14


def test_z_hook_error_and_clear():
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 16, 8, 6
    plan = P.Plan(nx, ny, nz, precision="f64", ttypes=("fft", "fft", "empty"), layout="xyz")

    def bad(lines, direction):
        raise ValueError("hook failure")

    plan.set_z_hook(bad)
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 1)).cuda()
    with pytest.raises(P.P3Error) as ei:
        plan.forward(x)
    assert ei.value.status == P.P3_ERR_HOOK and isinstance(ei.value.__cause__, ValueError)
    torch.cuda.synchronize()
    plan.set_z_hook(None)
    assert plan.launches(1) == 2
    X = plan.forward(x)
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), O.forward(x.cpu().numpy(), (O.FFT, O.FFT, O.EMPTY))) < TOL["f64"]


def test_z_hook_needs_an_empty_third_dimension():
    from paper_1905_02803_gb300 import p3dfft as P
    plan = P.Plan(16, 8, 8, precision="f32", ttypes=("fft", "fft", "fft"))
    cb = P.Z_HOOK(lambda *a: 0)
    assert P.p3_plan_set_z_hook(plan.handle, cb, check=False) == P.P3_ERR_INVALID
