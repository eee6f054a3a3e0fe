"""Guard bands: every input, output and workspace buffer of a call sits
between bands of canary bytes in one device arena, and after the call every
band must still hold its canary bit for bit (an out-of-bounds write of any
stage kernel, ragged tile, queue counter or bulk copy lands in a band), the
input must be untouched (out of place), and the result must equal the one
the same plan gives in ordinary buffers.  This stands in for a memory checker
on the GPU.  Cases: ragged and odd grids, Bluestein lengths, Chebyshev and
sine third dimensions, both layouts, FP32 and FP64, the plane-fused launch,
the TMA / bulk-copy Z stages, in place, and the allocation-free entry point
(whose workspace is inside the library, so only its input and output have
bands)."""
import numpy as np
import pytest

from paper_1905_02803_gb300 import inputs

pytestmark = pytest.mark.gpu

BAND = 4096  # canary bytes before and after every buffer


def _round(n, a=256):
    return (n + a - 1) // a * a


class Arena:
    """One uint8 device tensor: band, buffer 0, band, buffer 1, ..., band,
    every buffer 256-byte aligned; the bands and any free space hold seeded
    canary bytes."""

    def __init__(self, sizes, seed):
        import torch
        self.sizes = list(sizes)
        self.offs = []
        pos = BAND
        for n in self.sizes:
            self.offs.append(pos)
            pos += _round(max(n, 1)) + BAND
        self.total = pos
        canary = inputs.u64(seed, 90, 0, (self.total + 7) // 8).view(np.uint8)[:self.total]
        self.canary = torch.from_numpy(canary.copy()).cuda()
        self.buf = self.canary.clone()

    def ptr(self, i):
        return self.buf.data_ptr() + self.offs[i]

    def view(self, i, dtype, shape):
        import torch
        n = self.sizes[i]
        return self.buf[self.offs[i]:self.offs[i] + n].view(dtype).view(shape) if n else torch.empty(0)

    def bands_intact(self, skip=()):
        """True when every byte outside buffers (other than those in `skip`,
        whose whole extent may change) equals the canary."""
        import torch
        mask = torch.ones(self.total, dtype=torch.bool, device=self.buf.device)
        for i, (o, n) in enumerate(zip(self.offs, self.sizes)):
            if i in skip:
                mask[o:o + n] = False
        return bool(torch.equal(self.buf[mask], self.canary[mask]))


CASES = [
    # (nx, ny, nz), precision, ttypes, layout, flags name
    ((24, 20, 18), "f64", ("fft", "fft", "fft"), "zyx", ""),
    ((15, 9, 7), "f32", ("fft", "fft", "fft"), "xyz", ""),
    ((22, 13, 97), "f32", ("fft", "fft", "fft"), "zyx", ""),
    ((26, 11, 19), "f64", ("fft", "fft", "fft"), "xyz", ""),
    ((40, 12, 257), "f32", ("fft", "fft", "cheb"), "zyx", ""),
    ((30, 7, 33), "f64", ("fft", "fft", "cheb"), "xyz", ""),
    ((36, 10, 511), "f32", ("fft", "fft", "sine"), "zyx", ""),
    ((20, 6, 5), "f32", ("fft", "empty", "empty"), "zyx", ""),
    ((512, 256, 8), "f32", ("fft", "fft", "fft"), "zyx", ""),
    ((1024, 1024, 3), "f32", ("fft", "fft", "fft"), "zyx", ""),
    ((64, 32, 1024), "f32", ("fft", "fft", "fft"), "zyx", "NO_FUSE"),
    ((512, 256, 256), "f32", ("fft", "fft", "fft"), "zyx", ""),
    ((130, 66, 34), "f64", ("fft", "fft", "fft"), "xyz", ""),
    ((256, 64, 64), "f32", ("fft", "fft", "fft"), "xyz", ""),
]


def _flags(P, name):
    return {"": 0, "NO_FUSE": P.P3_FLAG_NO_FUSE}[name]


@pytest.mark.parametrize("shape,prec,tt,layout,flag", CASES)
def test_guard_bands_out_of_place(shape, prec, tt, layout, flag):
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    plan = P.Plan(nx, ny, nz, precision=prec, ttypes=tt, layout=layout, flags=_flags(P, flag))
    rdt, cdt = plan.real_dtype, plan.complex_dtype
    rbytes = nx * ny * nz * (4 if prec == "f32" else 8)
    cbytes = plan.H * ny * nz * (8 if prec == "f32" else 16)
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 7)).to("cuda", rdt)
    G = torch.from_numpy(np.asarray(inputs.normal(8, 1, 2 * plan.H * ny * nz))).to("cuda", rdt)
    G = torch.view_as_complex(G.view(*plan.complex_shape, 2)).contiguous()
    ref_f = plan.forward(x)
    ref_b = plan.backward(G)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for direction in (0, 1):
        nin, nout = (rbytes, cbytes) if direction == 0 else (cbytes, rbytes)
        ar = Arena([nin, nout, plan.ws_bytes], seed=31 + direction)
        src = x if direction == 0 else G
        ar.view(0, rdt if direction == 0 else cdt, src.shape).copy_(src)
        ar.canary[ar.offs[0]:ar.offs[0] + nin].copy_(ar.buf[ar.offs[0]:ar.offs[0] + nin])  # input must stay
        fn = P.p3_ftran_r2c if direction == 0 else P.p3_btran_c2r
        fn(plan.handle, ar.ptr(0), ar.ptr(1), ar.ptr(2) if plan.ws_bytes else None, stream)
        torch.cuda.synchronize()
        assert P.p3_plan_wait_status(plan.handle) == P.P3_OK
        assert ar.bands_intact(skip=(1, 2)), ("a band or the input changed", direction)
        got = ar.view(1, cdt if direction == 0 else rdt, ref_f.shape if direction == 0 else ref_b.shape)
        assert torch.equal(got, ref_f if direction == 0 else ref_b), direction


@pytest.mark.parametrize("shape,prec", [((48, 20, 16), "f32"), ((34, 9, 12), "f64"), ((512, 128, 32), "f32")])
def test_guard_bands_in_place(shape, prec):
    """Padded real rows, in == out both ways: one buffer between two bands."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    plan = P.Plan(nx, ny, nz, precision=prec, layout="xyz", flags=P.P3_FLAG_PADDED_REAL)
    assert plan.ws_bytes == 0
    rdt, cdt = plan.real_dtype, plan.complex_dtype
    nbytes = plan.H * ny * nz * (8 if prec == "f32" else 16)
    x = torch.zeros(plan.real_shape, dtype=rdt, device="cuda")
    x[..., :nx].copy_(torch.from_numpy(inputs.uniform_field((nz, ny, nx), 9)))
    ref_f = plan.forward(x.clone())
    ref_b = plan.backward(ref_f.clone())
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    ar = Arena([nbytes], seed=41)
    ar.view(0, rdt, plan.real_shape).copy_(x)
    P.p3_ftran_r2c(plan.handle, ar.ptr(0), ar.ptr(0), None, stream)
    torch.cuda.synchronize()
    assert ar.bands_intact(skip=(0,))
    assert torch.equal(ar.view(0, cdt, plan.complex_shape), ref_f)
    P.p3_btran_c2r(plan.handle, ar.ptr(0), ar.ptr(0), None, stream)
    torch.cuda.synchronize()
    assert ar.bands_intact(skip=(0,))
    assert torch.equal(ar.view(0, rdt, plan.real_shape)[..., :nx], ref_b[..., :nx])


@pytest.mark.parametrize("shape", [(256, 128, 96), (512, 256, 64)])
def test_guard_bands_noalloc(shape):
    """The allocation-free forward: bands around its input and output."""
    import torch
    from paper_1905_02803_gb300 import p3dfft as P
    nx, ny, nz = shape
    plan = P.Plan(nx, ny, nz, precision="f32", layout="zyx")
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), 12)).to("cuda", torch.float32)
    ref = plan.forward(x)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    ar = Arena([x.numel() * 4, plan.H * ny * nz * 8], seed=51)
    ar.view(0, torch.float32, x.shape).copy_(x)
    ar.canary[ar.offs[0]:ar.offs[0] + x.numel() * 4].copy_(ar.buf[ar.offs[0]:ar.offs[0] + x.numel() * 4])
    P.p3_ftran_r2c_noalloc(plan.handle, ar.ptr(0), ar.ptr(1), stream)
    torch.cuda.synchronize()
    assert ar.bands_intact(skip=(1,))
    assert torch.equal(ar.view(1, torch.complex64, plan.complex_shape), ref)
