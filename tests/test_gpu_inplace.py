"""In-place transforms with padded real rows (Sect. 3.1: in-place and
out-of-place transforms), compared with the FP64 oracle.

With P3_FLAG_PADDED_REAL a real array is [Nz][Ny][2H]; its first Nx values
per row are the data, the rest is padding the library may overwrite.  The
complex array [Nz][Ny][H] occupies the same bytes, so forward and inverse
can run with in == out."""
import numpy as np
import pytest

import oracle as O
from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, TT, random_complex, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    (64, 48, 40, "f32", ("fft", "fft", "fft")),        # pow2 rows, generic columns
    (256, 64, 128, "f32", ("fft", "fft", "fft")),      # pow2 row and column kernels
    (1024, 32, 16, "f32", ("fft", "fft", "cheb")),
    (30, 12, 10, "f64", ("fft", "fft", "fft")),        # mixed-radix rows
    (27, 9, 17, "f64", ("fft", "fft", "cheb")),        # odd Nx: rows in pairs, odd row count
    (45, 7, 10, "f32", ("fft", "fft", "fft")),         # odd Nx: rows in pairs, even row count
    (128, 20, 24, "f64", ("fft", "empty", "fft")),
    (64, 16, 8, "f64", ("fft", "empty", "empty")),
    (2, 3, 2, "f64", ("fft", "fft", "fft")),
]


def _plan(nx, ny, nz, prec, tt):
    from paper_1905_02803_gb300.p3dfft import Plan, P3_FLAG_PADDED_REAL
    return Plan(nx, ny, nz, precision=prec, ttypes=tt, layout="xyz", flags=P3_FLAG_PADDED_REAL)


def _padded(plan, f, fill):
    import torch
    nz, ny, nx = f.shape
    x = torch.full(plan.real_shape, fill, dtype=plan.real_dtype, device="cuda")
    x[..., :nx] = torch.from_numpy(f).to(device="cuda", dtype=plan.real_dtype)
    return x


@pytest.mark.parametrize("nx,ny,nz,prec,tt", CASES)
def test_inplace_round_trip(nx, ny, nz, prec, tt):
    import torch
    plan = _plan(nx, ny, nz, prec, tt)
    assert plan.ws_bytes == 0
    f = inputs.uniform_field((nz, ny, nx), 11)
    x = _padded(plan, f, 1e30)  # padding must not leak into the result
    xin = x[..., :nx].double().cpu().numpy()
    X = plan.complex_view(x)
    assert X.data_ptr() == x.data_ptr()
    plan.forward(x, out=X)
    ref = O.forward(xin, tuple(TT[t] for t in tt))
    torch.cuda.synchronize()
    assert rel_l2(X.cpu().numpy(), ref) < TOL[prec]

    # inverse in place of a fresh (non-Hermitian) spectrum
    G = random_complex((nz, ny, plan.H), 12)
    X.copy_(torch.from_numpy(G).to(device="cuda", dtype=plan.complex_dtype))
    Gin = X.cpu().numpy().astype(np.complex128)
    y = plan.real_view(X)
    plan.backward(X, out=y)
    refb = O.backward(Gin, nx, tuple(TT[t] for t in tt))
    torch.cuda.synchronize()
    assert rel_l2(y[..., :nx].cpu().numpy(), refb) < TOL[prec]


@pytest.mark.parametrize("nx,ny,nz,prec,tt", CASES[:5])
def test_padded_out_of_place_keeps_input(nx, ny, nz, prec, tt):
    import torch
    plan = _plan(nx, ny, nz, prec, tt)
    f = inputs.uniform_field((nz, ny, nx), 13)
    x = _padded(plan, f, -7.0)
    x0 = x.clone()
    X = plan.forward(x)
    torch.cuda.synchronize()
    assert torch.equal(x, x0)
    ref = O.forward(x[..., :nx].double().cpu().numpy(), tuple(TT[t] for t in tt))
    assert rel_l2(X.cpu().numpy(), ref) < TOL[prec]

    G = random_complex((nz, ny, plan.H), 14)
    Gd = torch.from_numpy(G).to(device="cuda", dtype=plan.complex_dtype)
    G0 = Gd.clone()
    y = plan.backward(Gd)
    torch.cuda.synchronize()
    assert torch.equal(Gd, G0)  # the inverse works in its output, not its input
    refb = O.backward(Gd.cpu().numpy().astype(np.complex128), nx, tuple(TT[t] for t in tt))
    assert rel_l2(y[..., :nx].cpu().numpy(), refb) < TOL[prec]


def test_padded_partial_overlap_rejected():
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    plan = _plan(32, 8, 8, "f32", ("fft", "fft", "fft"))
    buf = torch.zeros(2 * plan.H * 8 * 8 * 2, dtype=torch.float32, device="cuda")
    st = P.p3_ftran_r2c(plan.handle, buf.data_ptr(), buf.data_ptr() + 64, None,
                        torch.cuda.current_stream().cuda_stream, check=False)
    assert st == P.P3_ERR_INVALID


def test_padded_zyx_unsupported():
    from paper_1905_02803_gb300 import p3dfft as P
    st, h = P.p3_plan_create(16, 8, 8, P.P3_F32, (P.P3_FFT,) * 3, P.P3_LAYOUT_ZYX, P.P3_FLAG_PADDED_REAL,
                             check=False)
    assert st == P.P3_ERR_UNSUPPORTED and h is None
