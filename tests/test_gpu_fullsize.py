"""Full-size parity: the benchmark configurations in the launch
configuration bench.py times, compared with the FP64 oracle element by
element (Sect. 3.2 defines the output; Table 1 the layouts).

* 512^3 FP32 and FP64 (and FP32 in the XYZ layout): config 2's input, a
  dense Gaussian random field -- a seeded half-spectrum with power |k|^-5/3
  on every bin and uniform phases, taken to real space by the oracle's c2r,
  scaled to unit RMS -- plus 16 random plane waves.  The whole forward output
  is compared with the whole oracle forward (relative L2 over all elements);
  the inverse of an independent dense complex input, likewise.
* 1024^3 FP32, ZYX (the benchmark workload and plan), and its tensor-core
  split form: a dense i.i.d. U[-1, 1) input, so that every output line holds
  energy; the whole output is compared with the whole oracle output, and
  every line is also measured against its own norm.
* 2048^3 FP32, ZYX: the oracle computes whole output planes only.  Forward:
  one kx plane in every 4-line Y tile of the plane-fused launch (the tile
  position rotating, kx = H - 1 for the ragged last tile), every line of each
  plane -- so every Z tile of those planes, and element offsets beyond 2^31
  for kx > 512.  Inverse: 24 whole z planes, including planes beyond 2^31
  elements.  Each line / row against its own norm; global Parseval and round
  trip besides.

Set P3_PARITY_LOG to a file path to append one JSON line per check (the
measured errors quoted in the benchmark report).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, TOL_TC, check_case, log_parity as _log, rel_l2

pytestmark = pytest.mark.gpu


def grf_field(shape, seed):
    """Config 2's input: a dense random-phase field with power |k|^-5/3 per
    bin (the oracle's c2r takes the seeded half-spectrum to real space),
    scaled to unit RMS, plus 16 random plane waves."""
    nz, ny, nx = shape
    f = O.backward(inputs.power_law_half_spectrum(shape, seed), nx)
    f /= math.sqrt(float(np.mean(f * f)))
    return f + inputs.plane_waves(shape, seed)


def _dense_complex(plan, seed):
    """Independent dense complex input in the plan's layout: re, im i.i.d.
    U[-1, 1) (two streams of the counter-based generator), on the device."""
    import torch
    shp = plan.complex_shape
    npdt = np.float32 if plan.precision == "f32" else np.float64
    re = inputs.uniform_field_device(shp, seed, stream=1, device=plan.device, dtype=npdt)
    im = inputs.uniform_field_device(shp, seed, stream=2, device=plan.device, dtype=npdt)
    G = torch.complex(re, im)
    del re, im
    return G


def _per_line(got, ref, axis=-1):
    """Per-line (last axis) squared error and squared reference norm."""
    d = got.astype(np.complex128 if np.iscomplexobj(got) else np.float64) - ref
    return (np.abs(d) ** 2).sum(axis=axis), (np.abs(ref) ** 2).sum(axis=axis)


# ---------------------------------------------------------------------------
# 512^3: whole arrays, config 2's Gaussian random field
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,layout", [("f32", "zyx"), ("f64", "zyx"), ("f32", "xyz")])
def test_512cubed_grf_whole_array(prec, layout):
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    n = 512
    plan = Plan(n, n, n, precision=prec, layout=layout)
    f = grf_field((n, n, n), seed=2)
    x = torch.from_numpy(f).to("cuda", plan.real_dtype)
    del f
    X = plan.forward(x)
    xin = x.double().cpu().numpy()  # the exact values the GPU saw
    ref = O.forward(xin)
    if layout == "zyx":
        ref = O.to_zyx(ref)
    got = X.cpu().numpy()
    err = rel_l2(got, ref)
    _log(check="forward", grid=[n, n, n], precision=prec, layout=layout, input="grf k^-5/3 + 16 waves",
         compared="whole array", rel_l2=err)
    assert err <= TOL[prec], err
    del ref, got
    y = plan.backward(X)
    rt = rel_l2(y.double().cpu().numpy() / plan.scale, xin)
    assert rt <= TOL[prec], ("round trip", rt)
    del X, y
    torch.cuda.empty_cache()
    G = _dense_complex(plan, seed=12)
    g = plan.backward(G)
    Gh = G.cpu().numpy().astype(np.complex128)
    refb = O.backward(O.from_zyx(Gh) if layout == "zyx" else Gh, n)
    gh = g.cpu().numpy()
    errb = rel_l2(gh, refb)
    e2, r2 = _per_line(gh, refb)
    worst = float(np.sqrt(e2 / r2).max())
    _log(check="inverse", grid=[n, n, n], precision=prec, layout=layout, input="dense i.i.d. complex",
         compared="whole array", rel_l2=errb, worst_row_rel=worst)
    assert errb <= TOL[prec], errb
    assert worst <= TOL[prec], worst


# ---------------------------------------------------------------------------
# 1024^3: whole arrays, the benchmark's plan
# ---------------------------------------------------------------------------

def _whole_1024(flags, tol, seed, label):
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    n = 1024
    H = n // 2 + 1
    plan = Plan(n, n, n, precision="f32", layout="zyx", flags=flags)
    x = inputs.uniform_field_device((n, n, n), seed, device=plan.device, dtype=np.float32)
    X = plan.forward(x)
    torch.cuda.synchronize()
    ref = O.forward(x.cpu().numpy())  # [z][y][kx], FP64
    num = den = 0.0
    worst = 0.0
    for k0 in range(0, H, 32):
        k1 = min(H, k0 + 32)
        got = X[k0:k1].cpu().numpy()                 # [kx][ky][kz]
        r = ref[:, :, k0:k1].transpose(2, 1, 0)      # same order
        e2, r2 = _per_line(got, r)
        num += float(e2.sum())
        den += float(r2.sum())
        worst = max(worst, float(np.sqrt(e2 / r2).max()))
    err = math.sqrt(num / den)
    _log(check="forward", grid=[n, n, n], precision="f32", layout="zyx", plan=label, input="dense i.i.d. U[-1,1)",
         compared="whole array", rel_l2=err, worst_line_rel=worst)
    assert err <= tol, err
    assert worst <= tol, worst
    del ref
    # round trip on the device (FP64 reductions, chunked)
    y = plan.backward(X)
    rt_num = rt_den = 0.0
    for z0 in range(0, n, 64):
        xd = x[z0:z0 + 64].double()
        rt_num += (torch.linalg.vector_norm(y[z0:z0 + 64].double() / plan.scale - xd) ** 2).item()
        rt_den += (torch.linalg.vector_norm(xd) ** 2).item()
    assert math.sqrt(rt_num / rt_den) <= tol
    del x, X, y
    torch.cuda.empty_cache()
    # inverse of an independent dense complex input
    G = _dense_complex(plan, seed + 100)
    g = plan.backward(G)
    torch.cuda.synchronize()
    Gx = np.empty((n, n, H), dtype=np.complex128)    # XYZ order for the oracle
    for k0 in range(0, H, 32):
        Gx[:, :, k0:k0 + 32] = G[k0:k0 + 32].cpu().numpy().transpose(2, 1, 0)
    refb = O.backward(Gx, n)
    del Gx
    num = den = 0.0
    worst = 0.0
    for z0 in range(0, n, 64):
        e2, r2 = _per_line(g[z0:z0 + 64].cpu().numpy(), refb[z0:z0 + 64])
        num += float(e2.sum())
        den += float(r2.sum())
        worst = max(worst, float(np.sqrt(e2 / r2).max()))
    errb = math.sqrt(num / den)
    _log(check="inverse", grid=[n, n, n], precision="f32", layout="zyx", plan=label, input="dense i.i.d. complex",
         compared="whole array", rel_l2=errb, worst_row_rel=worst)
    assert errb <= tol, errb
    assert worst <= tol, worst
    del G, g
    plan._ws = None
    torch.cuda.empty_cache()


def test_1024cubed_fp32_zyx_bench_workload_whole_array():
    _whole_1024(0, TOL["f32"], seed=21, label="plain")


def test_1024cubed_fp32_zyx_tc_split_whole_array():
    from paper_1905_02803_gb300 import p3dfft as P
    _whole_1024(P.P3_FLAG_TC_SPLIT, TOL_TC, seed=22, label="tc_split")


def test_1024cubed_tc_split_against_gpu_fp64_path():
    """The tensor-core split form against the GPU's own FP64 path on the same
    input (config 3's second reference), besides the oracle above."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    from paper_1905_02803_gb300.p3dfft import Plan
    n = 1024
    x = inputs.uniform_field_device((n, n, n), 23, device=torch.device("cuda"), dtype=np.float32)
    p64 = Plan(n, n, n, precision="f64", layout="zyx")
    X64 = p64.forward(x.double())
    del p64
    torch.cuda.empty_cache()
    ptc = Plan(n, n, n, precision="f32", layout="zyx", flags=P.P3_FLAG_TC_SPLIT)
    Xtc = ptc.forward(x)
    num = den = 0.0
    for k0 in range(0, n // 2 + 1, 64):
        d = Xtc[k0:k0 + 64].to(torch.complex128) - X64[k0:k0 + 64]
        num += (torch.linalg.vector_norm(d) ** 2).item()
        den += (torch.linalg.vector_norm(X64[k0:k0 + 64]) ** 2).item()
    err = math.sqrt(num / den)
    _log(check="forward vs GPU FP64 path", grid=[n, n, n], precision="f32", layout="zyx", plan="tc_split",
         input="dense i.i.d. U[-1,1)", compared="whole array", rel_l2=err)
    assert err <= TOL_TC, err
    del x, X64, Xtc
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# 2048^3: whole sampled planes
# ---------------------------------------------------------------------------

def test_2048cubed_fp32_zyx_sampled_planes():
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan
    n = 2048
    H = n // 2 + 1
    plan = Plan(n, n, n, precision="f32", layout="zyx")
    x = inputs.uniform_field_device((n, n, n), 24, device=plan.device, dtype=np.float32)
    X = plan.forward(x)
    torch.cuda.synchronize()
    # one kx per 4-line Y tile, rotating the position in the tile; the last
    # (ragged) tile holds only kx = H - 1
    kxs = sorted({min(H - 1, 4 * g + (g % 4)) for g in range((H + 3) // 4)})
    assert kxs[0] == 0 and kxs[-1] == H - 1 and max(kxs) * n * n > 2 ** 31
    chunks = ((z0, x[z0:z0 + 16].cpu().numpy()) for z0 in range(0, n, 16))
    planes = O.forward_kx_planes(chunks, n, n, n, kxs)  # [k][ky][kz]
    num = den = 0.0
    worst = 0.0
    for i, kx in enumerate(kxs):
        e2, r2 = _per_line(X[kx].cpu().numpy(), planes[i])
        num += float(e2.sum())
        den += float(r2.sum())
        worst = max(worst, float(np.sqrt(e2 / r2).max()))
    err = math.sqrt(num / den)
    _log(check="forward", grid=[n, n, n], precision="f32", layout="zyx", plan="plain", input="dense i.i.d. U[-1,1)",
         compared="%d whole kx planes (every line of each)" % len(kxs), rel_l2=err, worst_line_rel=worst)
    assert err <= TOL["f32"], err
    assert worst <= TOL["f32"], worst
    del planes
    # Parseval (half spectrum weights) and round trip, FP64 reductions on the device
    w = torch.full((H,), 2.0, dtype=torch.float64, device=x.device)
    w[0] = w[-1] = 1.0
    e_in = sum((x[a:a + 16].double() ** 2).sum().item() for a in range(0, n, 16))
    e_out = sum((w[a:a + 16].view(-1, 1, 1) * X[a:a + 16].abs().double() ** 2).sum().item()
                for a in range(0, H, 16)) / float(n) ** 3
    assert abs(e_in - e_out) <= 4 * TOL["f32"] * e_in, ("Parseval", e_in, e_out)
    y = plan.backward(X)
    num = den = 0.0
    for z0 in range(0, n, 16):
        xd = x[z0:z0 + 16].double()
        num += (torch.linalg.vector_norm(y[z0:z0 + 16].double() / plan.scale - xd) ** 2).item()
        den += (torch.linalg.vector_norm(xd) ** 2).item()
    assert math.sqrt(num / den) <= TOL["f32"]
    del x, X, y
    plan._ws = None
    torch.cuda.empty_cache()
    # inverse: whole z planes of an independent dense complex input
    G = _dense_complex(plan, 25)
    g = plan.backward(G)
    torch.cuda.synchronize()
    zs = [0, 1, 2, 7, 8, 15, 255, 256, 511, 512, 513, 700, 1023, 1024, 1025, 1200, 1535, 1536, 1800, 2000,
          2040, 2045, 2046, 2047]
    assert max(zs) * n * n > 2 ** 31
    chunks = ((k0, G[k0:k0 + 8].cpu().numpy()) for k0 in range(0, H, 8))
    refz = O.backward_z_planes(chunks, n, n, n, zs)
    num = den = 0.0
    worst = 0.0
    for j, z in enumerate(zs):
        e2, r2 = _per_line(g[z].cpu().numpy(), refz[j])
        num += float(e2.sum())
        den += float(r2.sum())
        worst = max(worst, float(np.sqrt(e2 / r2).max()))
    errb = math.sqrt(num / den)
    _log(check="inverse", grid=[n, n, n], precision="f32", layout="zyx", plan="plain", input="dense i.i.d. complex",
         compared="%d whole z planes (every row of each)" % len(zs), rel_l2=errb, worst_row_rel=worst)
    assert errb <= TOL["f32"], errb
    assert worst <= TOL["f32"], worst
    del G, g
    torch.cuda.empty_cache()


def test_512x512x255_sine_whole_array():
    """FFT, FFT, sine (DST-I) third dimension, ZYX: whole arrays."""
    f = grf_field((255, 512, 512), seed=6)
    ef, eb, _ = check_case(512, 512, 255, "f32", ttypes=("fft", "fft", "sine"), layout="zyx", field=f,
                           label="sine_512x512x255_f32")
    assert ef <= TOL["f32"] and eb <= TOL["f32"], (ef, eb)


def test_512cubed_in_place_whole_array():
    """Padded real rows, in == out both ways (XYZ): the whole forward output
    and the whole inverse output against the oracle."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    n = 512
    plan = P.Plan(n, n, n, precision="f32", layout="xyz", flags=P.P3_FLAG_PADDED_REAL)
    f = grf_field((n, n, n), seed=7)
    buf = torch.zeros(plan.real_shape, dtype=torch.float32, device="cuda")
    buf[..., :n].copy_(torch.from_numpy(f))
    xin = buf[..., :n].double().cpu().numpy()
    X = plan.complex_view(buf)
    plan.forward(buf, X)
    ref = O.forward(xin)
    err = rel_l2(X.cpu().numpy(), ref)
    del ref
    plan.backward(X, buf)
    rt = rel_l2(buf[..., :n].double().cpu().numpy() / plan.scale, xin)
    _log(check="forward+round trip", config="inplace_512cube_f32_xyz", grid=[n, n, n], precision="f32",
         layout="xyz", compared="whole array", rel_l2_forward=err, round_trip=rt)
    assert err <= TOL["f32"] and rt <= TOL["f32"], (err, rt)
