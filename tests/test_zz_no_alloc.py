"""The allocation-free forward transform gives the same result as p3_ftran_r2c.

p3_ftran_r2c_noalloc is for callers that must not allocate device memory when
they run a transform: programs that give out all device memory from their own
pre-sized pool and forbid libraries to call cudaMalloc, or latency-bound loops
that cannot pay for a cudaMalloc/cudaFree (which can synchronise the device).
Its workspace is a fixed array inside the library.  This file is collected
last so that a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_1905_02803_gb300 import inputs

from _gpu_helpers import TOL, rel_l2

pytestmark = pytest.mark.gpu


# (512, 256, 64) FP32 runs the plane-fused X+Y launch: its queue counters
# (cleared by the call itself) and its transposed [x][y] planes, which the Z
# stage reads, both live in the built-in array
@pytest.mark.parametrize("shape,prec", [((64, 48, 40), "f32"), ((128, 96, 64), "f64"), ((30, 20, 12), "f32"),
                                        ((256, 128, 96), "f32"), ((512, 256, 64), "f32")])
def test_noalloc_matches_workspace_entry_point(shape, prec):
    import torch
    from paper_1905_02803_gb300 import p3dfft as P

    nx, ny, nz = shape
    plan = P.Plan(nx, ny, nz, precision=prec, layout="zyx")
    assert 0 < plan.ws_bytes <= P.P3_NOALLOC_SCRATCH_BYTES
    if shape == (512, 256, 64):
        d = plan.describe()
        assert "plane_fused" in d, d
    x = torch.from_numpy(inputs.uniform_field((nz, ny, nx), seed=nx)).to("cuda", plan.real_dtype)
    ref = plan.forward(x).cpu().numpy()  # caller-supplied workspace
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the built-in array
        out = torch.full(plan.complex_shape, float("nan"), dtype=plan.complex_dtype, device="cuda")
        P.p3_ftran_r2c_noalloc(plan.handle, x.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL[prec]


def test_noalloc_rejects_plans_beyond_the_array():
    from paper_1905_02803_gb300 import p3dfft as P

    plan = P.Plan(512, 512, 128, precision="f32", layout="zyx")  # 134 MB workspace
    assert plan.ws_bytes > P.P3_NOALLOC_SCRATCH_BYTES
    x = plan.empty_real()
    X = plan.empty_complex()
    st = P.p3_ftran_r2c_noalloc(plan.handle, x.data_ptr(), X.data_ptr(), None, check=False)
    assert st == P.P3_ERR_UNSUPPORTED
