"""The roofline arithmetic of bench.py (CPU): the stage model's algorithmic
bytes (each stage reads and writes its whole array once; a plane-fused X+Y
launch moves the real and the complex array once each), pinned to the
figures the benchmark configurations are quoted with, and the parsing of a
plan's launch groups."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def pair_bytes(nx, ny, nz, e):
    return sum(bench.stage_model_bytes(nx, ny, nz, e))


@pytest.mark.parametrize("dims,e,expect,rel", [
    ((1024, 1024, 1024), 4, 51.62e9, 1e-3),   # 1024^3 FP32: 51.62 GB per fwd+inv pair
    ((512, 512, 512), 4, 6.463e9, 1e-3),      # 512^3 FP32: 6.463 GB
    ((2048, 2048, 2048), 4, 412.7e9, 1e-3),   # 2048^3 FP32: 412.7 GB
    ((480, 360, 257), 8, 4.278e9, 1e-3),      # channel grid FP64: 4.278 GB
    ((32, 32, 32), 8, 3.31e6, 2e-3),          # 32^3 FP64: 3.31 MB
])
def test_stage_model_pair_bytes(dims, e, expect, rel):
    assert abs(pair_bytes(*dims, e) - expect) <= rel * expect


def test_stage_model_terms():
    nx, ny, nz, e = 10, 6, 4, 8
    H = nx // 2 + 1
    real, cplx = e * nx * ny * nz, 2 * e * H * ny * nz
    assert bench.stage_model_bytes(nx, ny, nz, e) == [real + cplx, 2 * cplx, 2 * cplx, 2 * cplx, 2 * cplx,
                                                      real + cplx]
    # odd Nx: H = (Nx - 1)/2 + 1
    assert bench.stage_model_bytes(7, 1, 1, 4)[1] == 2 * 2 * 4 * 4


def test_launch_bytes_fused_and_separate():
    nx = ny = nz = 1024
    sb = bench.stage_model_bytes(nx, ny, nz, 4)
    fused = bench.launch_bytes("xy_fused", nx, ny, nz, 4)
    assert fused == sb[0] == bench.launch_bytes("yx_fused_inv", nx, ny, nz, 4)
    assert bench.launch_bytes("x_r2c", nx, ny, nz, 4) == sb[0]
    assert bench.launch_bytes("y_c2c", nx, ny, nz, 4) == sb[1]
    assert bench.launch_bytes("z_c2c_zyx", nx, ny, nz, 4) == sb[2]
    # the executed launches of the fused 1024^3 pair: 34.41 GB, 5.142 ms at 6692.5 GB/s
    pair = 2 * fused + 2 * sb[2]
    assert abs(pair - 34.41e9) <= 1e-3 * 34.41e9
    assert abs(pair / 6692.5e9 * 1e3 - 5.142) <= 2e-3


def test_plan_groups_parses_describe():
    class FakePlan:
        def describe(self):
            return ("fwd groups=xy_fused,z_c2c_zyx\n"
                    "fwd xy_fused kernel=plane_fused x_nfft=512 lag=10\n"
                    "bwd groups=z_c2c_zyx_inv,yx_fused_inv\n"
                    "bwd z_c2c_zyx_inv kernel=pow2_zrow_bulk nfft=1024\n")

    g = bench.plan_groups(FakePlan())
    assert g == {0: ["xy_fused", "z_c2c_zyx"], 1: ["z_c2c_zyx_inv", "yx_fused_inv"]}


def test_peaks_reads_measured_file_or_falls_back():
    peak, kind = bench.peaks()
    assert kind in ("measured", "fallback")
    assert peak > 1000.0


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the contract's keys; on a small grid it samples every
    line, so the estimate is the oracle's actual time."""
    import json
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "32",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "first 1 of the lines" in cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["grid"] == [32, 32, 32]
