"""Plane-fused X + Y launches (one persistent kernel per direction that works
z-plane by z-plane through L2) against the FP64 oracle and against the same
plan with the stages launched separately (P3_FLAG_NO_FUSE): both run the
same tile arithmetic, so their outputs must agree bit for bit.  Also the
bounded-wait error path: a wait that cannot be satisfied gives up, the
launch finishes and p3_plan_wait_status() reports P3_ERR_TIMEOUT."""
import numpy as np
import pytest

import oracle as O
from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, check_case, random_complex

pytestmark = pytest.mark.gpu

FUSED = [(512, 256, 16), (1024, 1024, 4), (2048, 512, 6), (512, 1024, 9), (1024, 256, 1), (2048, 1024, 3),
         (512, 2048, 3), (2048, 2048, 2)]


@pytest.mark.parametrize("shape", FUSED)
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_fused_parity(shape, layout):
    nx, ny, nz = shape
    ef, eb, plan = check_case(nx, ny, nz, "f32", layout=layout, seed=nx + ny + nz)
    d = plan.describe()
    assert "xy_fused" in d, d
    # the inverse fuses when its Y stage runs in place, i.e. after a Z stage
    # (XYZ with Nz = 1 has none: its Y stage reads the input)
    assert ("yx_fused_inv" in d) == (layout == "zyx" or nz > 1), d
    assert ef <= TOL["f32"] and eb <= TOL["f32"], (ef, eb)


@pytest.mark.parametrize("shape", FUSED[:4])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_fused_equals_separate_stages(shape, layout):
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    pf = P.Plan(nx, ny, nz, precision="f32", layout=layout)
    ps = P.Plan(nx, ny, nz, precision="f32", layout=layout, flags=P.P3_FLAG_NO_FUSE)
    assert "plane_fused" in pf.describe() and "plane_fused" not in ps.describe()
    assert pf.launches(0) == ps.launches(0) - 1 and pf.launches(1) == ps.launches(1) - 1
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 7)).to("cuda", torch.float32)
    Xf, Xs = pf.forward(x), ps.forward(x)
    G = random_complex(pf.complex_shape, 8)
    Gd = torch.from_numpy(G).to("cuda", torch.complex64)
    yf, ys = pf.backward(Gd), ps.backward(Gd)
    torch.cuda.synchronize()
    assert torch.equal(Xf, Xs)
    assert torch.equal(yf, ys)
    assert P.p3_plan_wait_status(pf.handle) == P.P3_OK


def test_fused_wait_gives_up_and_reports():
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 512, 256, 8
    plan = P.Plan(nx, ny, nz, precision="f32", layout="zyx")
    assert "plane_fused" in plan.describe()
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 3)).to("cuda", torch.float32)
    # every wait needs one more finished producer tile than exists: a count
    # nothing reaches, so each wait gives up after a few polls
    P.p3_plan_set_wait_limits(plan.handle, 2000, 1)
    plan.forward(x)
    torch.cuda.synchronize()
    assert P.p3_plan_wait_status(plan.handle) == P.P3_ERR_TIMEOUT
    assert P.p3_plan_wait_status(plan.handle) == P.P3_OK  # the mark was cleared
    # the context is still usable and the default limits give the right result
    P.p3_plan_set_wait_limits(plan.handle, 1 << 23, 0)
    X = plan.forward(x)
    torch.cuda.synchronize()
    assert P.p3_plan_wait_status(plan.handle) == P.P3_OK
    ref = O.to_zyx(O.forward(x.double().cpu().numpy()))
    err = np.linalg.norm(X.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= TOL["f32"]


def test_fused_workspace_includes_counters():
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 512, 256, 16
    pf = P.Plan(nx, ny, nz, precision="f32", layout="xyz")
    ps = P.Plan(nx, ny, nz, precision="f32", layout="xyz", flags=P.P3_FLAG_NO_FUSE)
    assert pf.ws_bytes >= ps.ws_bytes + 4 * (nz + 1)
    # the padded in-place layout keeps its no-workspace promise: not fused
    pp = P.Plan(nx, ny, nz, precision="f32", layout="xyz", flags=P.P3_FLAG_PADDED_REAL)
    assert pp.ws_bytes == 0 and "plane_fused" not in pp.describe()


@pytest.mark.parametrize("lag", [1, 2, 5, 1000])
def test_fused_lag_keeps_results(lag):
    """The queue order (how far consumers trail producers) changes nothing
    in the arithmetic: bit-identical to the separate stages at any lag."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 512, 256, 12
    pf = P.Plan(nx, ny, nz, precision="f32", layout="zyx")
    ps = P.Plan(nx, ny, nz, precision="f32", layout="zyx", flags=P.P3_FLAG_NO_FUSE)
    P.p3_plan_set_fused_lag(pf.handle, lag)
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 9)).to("cuda", torch.float32)
    Xf, Xs = pf.forward(x), ps.forward(x)
    yf, ys = pf.backward(Xf), ps.backward(Xs)
    torch.cuda.synchronize()
    assert torch.equal(Xf, Xs) and torch.equal(yf, ys)
    assert P.p3_plan_wait_status(pf.handle) == P.P3_OK


@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_tuned_plan_keeps_results(layout):
    """P3_FLAG_TUNE times the fused launch at a few lags and the separate
    stages, keeps the fastest per direction (the same arithmetic), and picks
    the radix order of the generic 24-point Z stage (the same transform,
    rounded in another order): the result agrees with the separate-stage
    plan's to rounding."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = 512, 256, 24
    pt = P.Plan(nx, ny, nz, precision="f32", layout=layout, flags=P.P3_FLAG_TUNE)
    ps = P.Plan(nx, ny, nz, precision="f32", layout=layout, flags=P.P3_FLAG_NO_FUSE)
    d = pt.describe()
    assert "fwd tuned:" in d and "bwd tuned:" in d and "separate=" in d, d
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 21)).to("cuda", torch.float32)
    Xt, Xs = pt.forward(x), ps.forward(x)
    yt, ys = pt.backward(Xt), ps.backward(Xs)
    torch.cuda.synchronize()
    for a, b in ((Xt, Xs), (yt, ys)):
        a, b = a.to(torch.complex128), b.to(torch.complex128)
        assert ((a - b).abs().norm() / b.abs().norm()).item() <= 5e-7
    assert P.p3_plan_wait_status(pt.handle) == P.P3_OK


@pytest.mark.parametrize("shape,prec,layout", [((384, 360, 48), "f32", "zyx"), ((150, 98, 63), "f32", "xyz"),
                                               ((60, 45, 42), "f64", "zyx")])
def test_tuned_generic_stages_keep_results(shape, prec, layout):
    """P3_FLAG_TUNE on lengths of the generic kernel: radix order and tile
    height are chosen by timing; the result still matches the oracle."""
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    ef, eb, plan = check_case(nx, ny, nz, prec, layout=layout, seed=3, flags=P.P3_FLAG_TUNE)
    assert "tuned:" in plan.describe(), plan.describe()
    assert ef <= TOL[prec] and eb <= TOL[prec], (ef, eb)
