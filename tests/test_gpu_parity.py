"""GPU path (through the C ABI) vs the FP64 CPU oracle, element by element.

Tolerances: relative L2 <= 1e-13 for FP64 and <= 2e-6 for FP32.  Sizes span
several CTA tiles with ragged tails, odd X lengths (no Nyquist bin), mixed
radices 2/3/5/7, Bluestein lengths, degenerate extents of 1 and 2, the
Chebyshev, sine and empty third-dimension transforms, and both Z-pencil
layouts.
"""
import numpy as np
import pytest

from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, check_case, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_config1_32cubed_fp64_plane_wave(layout):
    """32^3 FP64: U[-1,1) field plus sin(2 pi 3 x/32), and the plane wave alone."""
    total, rnd, wave = inputs.config1_field(32, seed=0)
    for field, name in ((total, "32cube_f64 U[-1,1)+sin"), (wave, "32cube_f64 sin"), (rnd, "32cube_f64 U[-1,1)")):
        ef, eb, _ = check_case(32, 32, 32, "f64", layout=layout, field=field, label=name)
        assert ef <= TOL["f64"] and eb <= TOL["f64"], (ef, eb)


def test_plane_wave_single_bin_on_gpu():
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    plan = Plan(32, 32, 32, precision="f64", layout="xyz")
    x = torch.from_numpy(inputs.plane_wave_sin((32, 32, 32), 3)).cuda()
    X = plan.forward(x).cpu().numpy()
    N = 32 ** 3
    assert abs(X[0, 0, 3] - (-0.5j * N)) < 1e-9
    X[0, 0, 3] = 0
    assert np.abs(X).max() < 1e-10


SHAPES = [
    (64, 48, 40), (30, 20, 12), (7, 9, 15), (1, 1, 1), (2, 3, 5), (1, 7, 4), (9, 1, 1), (4, 1, 6),
    (96, 7, 5), (49, 75, 343 // 7), (210, 6, 10), (16, 256, 8), (8, 8, 1024), (2048, 2, 2),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_fft3_parity(shape, prec, layout):
    nx, ny, nz = shape
    ef, eb, _ = check_case(nx, ny, nz, prec, layout=layout, seed=nx + ny + nz)
    assert ef <= TOL[prec] and eb <= TOL[prec], (ef, eb)


@pytest.mark.parametrize("shape", [(11, 13, 97), (22, 26, 14), (34, 17, 19), (12, 1, 23)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bluestein_lengths(shape, prec):
    nx, ny, nz = shape
    for layout in ("zyx", "xyz"):
        ef, eb, plan = check_case(nx, ny, nz, prec, layout=layout, seed=3)
        assert "bluestein" in plan.describe()
        assert ef <= TOL[prec] and eb <= TOL[prec], (layout, ef, eb)


# FP32 generic stages factor lengths with a factor 3, 5 or 7 into the fewest
# passes over the native radices and the composite register butterflies 6,
# 9, 10, 12, 14 and 15; FP64 stages keep the native radices.  Each composite
# appears in one of these plans (Y and Z lengths; X half-lengths of even Nx).
COMPOSITE_CASES = [
    ((12, 54, 100), {"6", "9", "10"}),     # X 6; Y 54 = 9 x 6; Z 100 = 10 x 10
    ((30, 14, 135), {"15", "14", "9"}),    # X 15; Y 14; Z 135 = 15 x 9
    ((24, 96, 225), {"12", "8", "15"}),    # X 12; Y 96 = 12 x 8; Z 225 = 15 x 15
]


@pytest.mark.parametrize("shape,radices", COMPOSITE_CASES)
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_composite_radices(shape, radices, layout):
    nx, ny, nz = shape
    ef, eb, plan = check_case(nx, ny, nz, "f32", layout=layout, seed=nx + nz)
    used = set()
    for line in plan.describe().splitlines():
        for w in line.split():
            if w.startswith("radices="):
                used.update(w[len("radices="):].split("x"))
    assert radices <= used, (radices, used)
    assert ef <= TOL["f32"] and eb <= TOL["f32"], (ef, eb)
    # the same grid in FP64 keeps the native radices 2, 3, 4, 5, 7, 8, 16
    ef64, eb64, plan64 = check_case(nx, ny, nz, "f64", layout=layout, seed=nx + nz)
    for line in plan64.describe().splitlines():
        for w in line.split():
            if w.startswith("radices="):
                assert set(w[len("radices="):].split("x")) <= {"2", "3", "4", "5", "7", "8", "16"}, line
    assert ef64 <= TOL["f64"] and eb64 <= TOL["f64"], (ef64, eb64)


@pytest.mark.parametrize("ttypes", [("fft", "fft", "cheb"), ("fft", "empty", "cheb"), ("fft", "empty", "empty"),
                                    ("fft", "fft", "empty"), ("fft", "empty", "fft"), ("fft", "fft", "sine"),
                                    ("fft", "empty", "sine")])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_transform_types(ttypes, layout, prec):
    for shape in ((20, 12, 17), (9, 5, 2), (16, 6, 33), (6, 4, 12)):
        nx, ny, nz = shape
        ef, eb, _ = check_case(nx, ny, nz, prec, ttypes=ttypes, layout=layout, seed=nz)
        assert ef <= TOL[prec] and eb <= TOL[prec], (shape, ef, eb)


def test_config4_channel_480x360x257_fp64():
    """Uneven channel-flow grid: FFT in X and Y, Chebyshev (DCT-I) in Z."""
    nx, ny, nz = 480, 360, 257
    f = inputs.channel_field(nx, ny, nz, seed=0)
    ef, eb, _ = check_case(nx, ny, nz, "f64", ttypes=("fft", "fft", "cheb"), layout="zyx", field=f,
                           label="channel_480x360x257_f64")
    assert ef <= TOL["f64"] and eb <= TOL["f64"], (ef, eb)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_turbulence_field_128(prec):
    f = inputs.turbulence_field((96, 128, 128), seed=2)
    ef, eb, _ = check_case(128, 128, 96, prec, field=f)
    assert ef <= TOL[prec] and eb <= TOL[prec], (ef, eb)


def test_round_trip_and_inputs_untouched():
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    for layout in ("zyx", "xyz"):
        plan = Plan(40, 30, 20, precision="f64", layout=layout)
        x = torch.from_numpy(inputs.uniform_field((20, 30, 40), 5)).cuda()
        x0 = x.clone()
        X = plan.forward(x)
        X0 = X.clone()
        y = plan.backward(X)
        torch.cuda.synchronize()
        assert torch.equal(x, x0) and torch.equal(X, X0)
        assert rel_l2(y.cpu().numpy() / plan.scale, x0.cpu().numpy()) < 1e-14


def test_error_paths_on_device():
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    plan = P.Plan(16, 8, 8, precision="f32", layout="zyx")
    x = plan.empty_real().normal_()
    X = plan.empty_complex()
    ws = plan.workspace()
    h = plan.handle
    s = None
    assert P.p3_ftran_r2c(h, x.data_ptr(), X.data_ptr(), None, s, check=False) == P.P3_ERR_WORKSPACE
    assert P.p3_ftran_r2c(h, x.data_ptr(), x.data_ptr(), ws.data_ptr(), s, check=False) == P.P3_ERR_UNSUPPORTED
    assert P.p3_ftran_r2c(h, x.data_ptr() + 4, X.data_ptr(), ws.data_ptr(), s, check=False) == P.P3_ERR_INVALID
    assert P.p3_ftran_r2c(h, x.data_ptr(), X.data_ptr(), x.data_ptr(), s, check=False) == P.P3_ERR_INVALID
    assert P.p3_ftran_r2c(h, x.data_ptr(), X.data_ptr(), ws.data_ptr(), s, check=False) == P.P3_OK
    assert P.p3_plan_get_dims(h) == ((16, 8, 8), (8, 8, 9))
    assert plan.ws_bytes == 9 * 8 * 8 * 8
    torch.cuda.synchronize()


POW2_SHAPES = [(128, 64, 256), (256, 128, 64), (1024, 4, 6), (4096, 2, 3), (8192, 1, 2), (6, 4096, 2),
               (10, 3, 2048), (130, 64, 64), (64, 2, 4096)]


@pytest.mark.parametrize("shape", POW2_SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_pow2_kernels_parity(shape, prec, layout):
    nx, ny, nz = shape
    ef, eb, plan = check_case(nx, ny, nz, prec, layout=layout, seed=7)
    assert "pow2_" in plan.describe()
    assert ef <= TOL[prec] and eb <= TOL[prec], (ef, eb)


@pytest.mark.parametrize("nz", [65, 129, 257, 1025])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_pow2_chebyshev(nz, layout):
    for prec in ("f64", "f32"):
        ef, eb, plan = check_case(12, 6, nz, prec, ttypes=("fft", "fft", "cheb"), layout=layout, seed=nz)
        assert "pow2_col" in plan.describe()
        assert ef <= TOL[prec] and eb <= TOL[prec], (prec, ef, eb)


@pytest.mark.parametrize("shape", [(16, 1024, 6), (6, 4, 1024), (130, 1024, 3), (8, 1024, 1024)])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
def test_tc_split_parity(shape, layout):
    """FP32 1024-point Y / Z stages on the tensor cores (TF32 head/tail split,
    three products): within 5e-6 of the FP64 oracle."""
    from _gpu_helpers import TOL_TC
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    ef, eb, plan = check_case(nx, ny, nz, "f32", layout=layout, seed=11, flags=P.P3_FLAG_TC_SPLIT)
    assert "tc_split_col" in plan.describe()
    assert ef <= TOL_TC and eb <= TOL_TC, (ef, eb)


@pytest.mark.parametrize("nz", [1, 3, 9, 31, 63, 127, 511, 1023, 2047, 100])
@pytest.mark.parametrize("layout", ["zyx", "xyz"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sine_third_dimension(nz, layout, prec):
    """DST-I in Z: odd extension to 2(Nz+1) points; Nz = 2^k - 1 runs the
    power-of-two column kernels (sine variant), others the generic kernel
    (Nz = 100: 202 = 2 * 101 is a Bluestein length)."""
    nx, ny = (24, 6) if nz >= 1023 else (34, 10)
    ef, eb, plan = check_case(nx, ny, nz, prec, ttypes=("fft", "fft", "sine"), layout=layout, seed=nz)
    assert ef <= TOL[prec] and eb <= TOL[prec], (ef, eb)
    assert "dst1" in plan.describe()
    if nz in (63, 127, 511, 1023, 2047):
        assert "pow2_col" in plan.describe()
    assert plan.scale == nx * ny * 2 * (nz + 1)


def test_sine_mode_delta_on_gpu():
    """f = sin(pi m (z+1)/(Nz+1)): the forward is Nx Ny (Nz+1) at
    (kx, ky, kz) = (0, 0, m-1) and zero elsewhere."""
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    nx, ny, nz, m = 8, 4, 255, 5
    plan = Plan(nx, ny, nz, precision="f64", ttypes=("fft", "fft", "sine"), layout="xyz")
    zz = np.arange(nz)
    f = np.broadcast_to(np.sin(np.pi * m * (zz + 1) / (nz + 1))[:, None, None], (nz, ny, nx)).copy()
    X = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy()
    expect = np.zeros_like(X)
    expect[m - 1, 0, 0] = nx * ny * (nz + 1)
    assert np.abs(X - expect).max() < 1e-9 * nx * ny * (nz + 1)


@pytest.mark.parametrize("shape", [(16, 8, 2048), (24, 6, 1024), (40, 4, 512)])
def test_row_style_zyx_load_lengths(shape):
    """ZYX-load (inverse Z) stage of the row-style kernel at 512 .. 2048
    points (2048: 8-line tiles of 512 threads), forward and inverse."""
    nx, ny, nz = shape
    ef, eb, plan = check_case(nx, ny, nz, "f32", layout="zyx", seed=nz)
    assert "pow2_col_zyx_load" in plan.describe() or "pow2_zrow_bulk" in plan.describe()
    assert ef <= TOL["f32"] and eb <= TOL["f32"], (ef, eb)
