"""Benchmark: forward + inverse 3D FFT (r2c then c2r) on a 1024^3 FP32 grid.

One step = one p3_ftran_r2c plus one p3_btran_c2r over the whole grid (all
stages of the hot path: X r2c, Y c2c, Z c2c with the fused ZYX re-orientation,
and the inverse stages), inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores instead (each
step a bounded sample of the same workload's lines, scaled to the full grid).
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the transform has no cross-GPU exchange on one device); value is the job's
ms per transform pair, max over ranks divided by N.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+inv 3D FFT ms & HBM-roofline % at 1024³ FP32; TC-split vs plain at ≤5e-6"
NX = NY = NZ = 1024
LAYOUT = "zyx"
PREC = "f32"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp64_peak_tflops(n=4096, reps=5):
    """Measured FP64 arithmetic peak of this GPU: cuBLAS DGEMM (torch.matmul
    on float64 n x n matrices, 2 n^3 flop), best of `reps`, CUDA events.  The
    FP64 transforms are compared with it (their FP64 operations per launch
    come from ncu, profiles/fp64_ops.json)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = torch.empty(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def fp64_ops_record(config):
    """FP64 work of one forward + inverse pair of a report configuration
    (ncu counters, profiles/fp64_ops.json): (flop, FP64-pipe instructions),
    a DFMA counting 2 flop and each of DFMA, DADD, DMUL one instruction.
    None when absent or when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "fp64_ops.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    ent = rec.get("configs", {}).get(config)
    if ent is None:
        return None
    # a configuration may name the sources of its own kernels
    srcs = ent.get("kernel_sources", rec.get("kernel_sources", []))
    want = ent.get("kernel_source_sha256_16", rec.get("kernel_source_sha256_16"))
    h = hashlib.sha256()
    for rel in srcs:
        try:
            h.update(open(os.path.join(ROOT, rel), "rb").read())
        except OSError:
            return None
    if not srcs or want != h.hexdigest()[:16]:
        return None
    return float(ent["fp64_flop_per_pair"]), float(ent["fp64_inst_per_pair"])


def stage_model_bytes(nx, ny, nz, e):
    """Algorithmic bytes of each stage launch (each stage reads and writes its
    whole array once): X stages e*N + 2e*H*Ny*Nz, Y and Z stages 2 * 2e*H*Ny*Nz."""
    H = nx // 2 + 1
    real = e * nx * ny * nz
    cplx = 2 * e * H * ny * nz
    return [real + cplx, 2 * cplx, 2 * cplx, 2 * cplx, 2 * cplx, real + cplx]


def launch_bytes(group, nx, ny, nz, e):
    """Algorithmic bytes of one launch of a plan group: a separate stage as
    in stage_model_bytes; the plane-fused X+Y launch reads (or writes) the
    real array once and writes (or reads) the complex array once."""
    sb = stage_model_bytes(nx, ny, nz, e)
    if "fused" in group:
        return sb[0]
    return {"x": sb[0], "y": sb[1], "z": sb[2]}[group[0]]


def plan_groups(plan):
    """The launch groups of each direction, from the plan description."""
    groups = {0: [], 1: []}
    for line in plan.describe().strip().splitlines():
        head = line.split()
        if len(head) > 1 and head[1].startswith("groups="):
            groups[0 if head[0] == "fwd" else 1] = head[1][len("groups="):].split(",")
    return groups


def workload_name():
    return "%dx%dx%d real %s, r2c forward + c2r inverse, FFT in x/y/z, %s complex layout" % (
        NX, NY, NZ, PREC.upper(), LAYOUT.upper())


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: the system temporary directory unless P3_BENCH_CLOCKS_DIR
        # names another (the JSON line carries their summary either way)
        out_dir = os.environ.get("P3_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                rows.append(parts)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(rows), "reasons": reasons}


def cpu_oracle_sample(frac, nthreads=0):
    """Time the FP64 oracle's stage functions on the first `frac` of the lines
    of every stage of the grid's pair (full-size strides; buffers are
    allocated lazily and only sampled lines are touched), scaled to all lines.
    Returns (estimated ms per fwd+inv pair, threads, description)."""
    import numpy as np

    import oracle as O
    from paper_1905_02803_gb300 import inputs

    nx, ny, nz = NX, NY, NZ
    H = nx // 2 + 1
    nthreads = nthreads or O.nthreads_default()
    # at least 2^24 points' worth of lines per stage (the whole grid below
    # that), so that starting the oracle's threads stays a small part of
    # each timed call; 1024^3 samples 1/64 of its lines or more
    frac = sample_fraction(frac)
    rows = ny * nz
    ylines = H * nz
    zlines = H * ny
    kr = max(1, int(rows * frac))
    ky = max(1, int(ylines * frac))
    kz = max(1, int(zlines * frac))
    f = np.zeros(rows * nx)
    f[:kr * nx] = inputs.uniform(0, 70, kr * nx)
    F = np.zeros(rows * H, dtype=np.complex128)
    out = np.zeros(rows * nx)
    total = 0.0
    # X r2c and c2r on the first kr rows
    t = time.perf_counter()
    O.x_r2c_rows(nx, f, F, 0, kr, nthreads)
    total += (time.perf_counter() - t) * rows / kr
    t = time.perf_counter()
    O.x_c2r_rows(nx, F, out, 0, kr, nthreads)
    total += (time.perf_counter() - t) * rows / kr
    # Y lines: base (L/H)*ny*H + L%H, stride H (first ky lines touch a few planes)
    for sign in (-1, 1):
        t = time.perf_counter()
        O.c2c_lines(ny, H, ny * H, 1, H, F, 0, ky, sign, nthreads)
        total += (time.perf_counter() - t) * ylines / ky
    # Z lines: base L, stride ny*H over the full volume (touch the lines first)
    Z = np.zeros(H * ny * nz, dtype=np.complex128)
    view = Z.reshape(nz, ny * H)
    view[:, :kz] = 1.0
    for sign in (-1, 1):
        t = time.perf_counter()
        O.c2c_lines(nz, H * ny, 0, 1, ny * H, Z, 0, kz, sign, nthreads)
        total += (time.perf_counter() - t) * zlines / kz
    desc = ("FP64 oracle stage functions on the first %.4g of the lines of each of the 6 stages of the %dx%dx%d "
            "pair (%d X rows, %d Y lines, %d Z lines per direction), scaled by line count" % (
                frac, nx, ny, nz, kr, ky, kz))
    return total * 1e3, nthreads, desc


def sample_fraction(frac):
    """The fraction of each stage's lines cpu_oracle_sample actually times."""
    return min(1.0, max(frac, float(1 << 24) / (NX * NY * NZ)))


def traffic_record(kernel_name):
    """dram bytes per launch of a kernel from the committed ncu summary, or
    None when the kernel source has changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    h = hashlib.sha256()
    for rel in rec.get("kernel_sources", []):
        try:
            h.update(open(os.path.join(ROOT, rel), "rb").read())
        except OSError:
            return None
    if not rec.get("kernel_sources") or rec.get("kernel_source_sha256_16") != h.hexdigest()[:16]:
        return None
    ent = rec.get("stages", {}).get(kernel_name)
    return None if ent is None else float(ent)


def reduce_over_ranks(values, world, device=None):
    """Max over ranks of per-rank timings (the job is as slow as its slowest
    replica); identity on one rank."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_value(ms_max, world):
    """Whole-job ms per transform pair: N replicas each finish one pair per
    step, so the job delivers N pairs per max-over-ranks step time."""
    return ms_max / max(1, world)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    frac = 1.0 / 64
    for _ in range(args.warmup):
        cpu_oracle_sample(frac)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ms, cores, desc = cpu_oracle_sample(frac)
        vals.append(ms)
    wall = time.perf_counter() - t0
    v = statistics.mean(vals)
    sampled = sample_fraction(frac)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "grid": [NX, NY, NZ], "precision": PREC, "layout": LAYOUT},
        "estimated": True, "sample_fraction": sampled,
        "timed_ms_per_step": round(wall * 1e3 / max(1, args.steps), 1),
        "estimate_note": ("each step times the oracle on %.4g of the lines of every stage and scales by the line "
                          "count: value and ms_per_step are the extrapolated full-pair time, timed_ms_per_step "
                          "the host time a step took" % sampled),
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle", "sample": desc,
                         "estimated": True, "sample_fraction": sampled},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host_wall_s": wall,
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core split-precision comparison")
    ap.add_argument("--no-fuse", action="store_true", help="launch the X and Y stages separately (P3_FLAG_NO_FUSE)")
    ap.add_argument("--report", action="store_true",
                    help="measure every benchmark configuration (one JSON line each) instead of the 1024^3 line")
    ap.add_argument("--report-only", default="",
                    help="with --report: only these comma-separated configs (names in REPORT_CONFIGS, or batch64)")
    ap.add_argument("--grid", default="1024",
                    help="grid edge N, or NX,NY,NZ (1024 is the benchmark workload; others are for profiling)")
    ap.add_argument("--cpu-report", action="store_true",
                    help="time the FP64 CPU oracle's full forward + inverse pair at the small configurations, "
                         "on all host threads and on one (no GPU use)")
    args = ap.parse_args()
    global NX, NY, NZ
    g = [int(v) for v in str(args.grid).split(",")]
    NX, NY, NZ = (g * 3)[:3] if len(g) == 1 else g
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.cpu_report:
        run_cpu_report()
        return
    if args.report:
        run_report(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1905_02803_gb300 import inputs
    from paper_1905_02803_gb300 import p3dfft as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world, device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    plan = P.Plan(NX, NY, NZ, precision=PREC, layout=LAYOUT, flags=P.P3_FLAG_NO_FUSE if args.no_fuse else 0)
    x = inputs.turbulence_field((NZ, NY, NX), seed=local, dtype=np.float32, device=dev)
    X = plan.empty_complex()
    y = plan.empty_real()
    ws = plan.workspace()
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.forward(x, X, ws, stream)
        plan.backward(X, y, ws, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # per-stage events: 8 per step (4 per direction), created by a first record
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(args.steps)]
    for row in evs:
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(args.steps):
            P.p3_plan_set_stage_events(plan.handle, [e.cuda_event for e in evs[k]])
            step()
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        P.p3_plan_set_stage_events(plan.handle, None)
        elapsed = t0.elapsed_time(t1)

        # end to end through the public API: pinned host in -> device -> host out
        xh = torch.empty(plan.real_shape, dtype=plan.real_dtype, pin_memory=True)
        xh.copy_(x)
        yh = torch.empty(plan.real_shape, dtype=plan.real_dtype, pin_memory=True)
        e2e_steps = max(3, min(args.steps, 10))
        xd = plan.empty_real()
        for _ in range(2):
            xd.copy_(xh, non_blocking=True)
            plan.forward(xd, X, ws, stream)
            plan.backward(X, y, ws, stream)
            yh.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            xd.copy_(xh, non_blocking=True)
            plan.forward(xd, X, ws, stream)
            plan.backward(X, y, ws, stream)
            yh.copy_(y, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_serial_ms = e0.elapsed_time(e1) / e2e_steps

        # the same loop double-buffered on three streams: the host-to-device
        # copy of step k+1 and the device-to-host copy of step k-1 run while
        # step k transforms
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        xds = [xd, plan.empty_real()]
        yds = [y, plan.empty_real()]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_c = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def pipelined(nsteps, t_start=None, t_end=None):
            if t_start is not None:
                t_start.record(stream)
            s_in.wait_stream(stream)
            s_out.wait_stream(stream)
            for k in range(nsteps):
                i = k % 2
                s_in.wait_event(ev_c[i])  # step k-2 no longer reads xds[i]
                with torch.cuda.stream(s_in):
                    xds[i].copy_(xh, non_blocking=True)
                ev_in[i].record(s_in)
                stream.wait_event(ev_in[i])
                stream.wait_event(ev_out[i])  # step k-2's result has left yds[i]
                plan.forward(xds[i], X, ws, stream)
                plan.backward(X, yds[i], ws, stream)
                ev_c[i].record(stream)
                s_out.wait_event(ev_c[i])
                with torch.cuda.stream(s_out):
                    yh.copy_(yds[i], non_blocking=True)
                ev_out[i].record(s_out)
            stream.wait_stream(s_out)
            stream.wait_stream(s_in)
            if t_end is not None:
                t_end.record(stream)

        pipelined(2)
        torch.cuda.synchronize()
        barrier()
        pipelined(e2e_steps, e0, e1)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = e0.elapsed_time(e1) / e2e_steps

    ms, e2e_ms, e2e_serial_ms = reduce_over_ranks([elapsed / args.steps, e2e_ms, e2e_serial_ms], world, device=dev)

    # per-group durations over the timed region (a group is one stage, or the
    # X and Y stages run slab by slab through L2)
    desc = plan.describe().strip().splitlines()
    groups = plan_groups(plan)
    e_bytes = 4 if PREC == "f32" else 8
    sb = stage_model_bytes(NX, NY, NZ, e_bytes)
    names, gbytes, dur = [], [], []
    for d in (0, 1):
        for gi in range(3):
            if gi < len(groups[d]):
                g = groups[d][gi]
                names.append(("fwd " if d == 0 else "bwd ") + g)
                gbytes.append(launch_bytes(g, NX, NY, NZ, e_bytes))
                dur.append(sum(row[4 * d + gi].elapsed_time(row[4 * d + gi + 1]) for row in evs) / args.steps)
    peak, peak_kind = peaks()
    stages = []
    for nm, d, b in zip(names, dur, gbytes):
        gbs = b / (d * 1e-3) / 1e9
        ent = {"kernel": nm, "ms": round(d, 4), "bytes": b, "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
               "share": round(d / sum(dur), 4)}
        if "fused" in nm:
            ent["note"] = ("X and Y stages in one persistent launch, z-plane by z-plane through L2: the real "
                           "array and the complex array each cross HBM once")
        stages.append(ent)
    dom = max(range(len(names)), key=lambda i: dur[i])
    dom_gbs = gbytes[dom] / (dur[dom] * 1e-3) / 1e9
    traffic = traffic_record(names[dom].split(" ", 1)[1])
    # roofline of the executed launches (fused X+Y where the plan fuses them)
    # and of the unfused six-stage model, for comparison
    pair_bytes = sum(gbytes)
    roof_ms = pair_bytes / (peak * 1e9) * 1e3
    roof_ms_unfused = sum(sb) / (peak * 1e9) * 1e3

    # tensor-core split-precision form of the same workload (the metric's
    # "TC-split vs plain"): time it and compare its output with the plain one
    tc = None
    if not args.no_tc and PREC == "f32":
        ptc = P.Plan(NX, NY, NZ, precision=PREC, layout=LAYOUT, flags=P.P3_FLAG_TC_SPLIT)
        if "tc_split_col" in ptc.describe():
            Xtc = ptc.empty_complex()
            ytc = ptc.empty_real()
            wtc = ptc.workspace()
            for _ in range(3):
                ptc.forward(x, Xtc, wtc, stream)
                ptc.backward(Xtc, ytc, wtc, stream)
            torch.cuda.synchronize()
            t0.record(stream)
            for _ in range(args.steps):
                ptc.forward(x, Xtc, wtc, stream)
                ptc.backward(Xtc, ytc, wtc, stream)
            t1.record(stream)
            torch.cuda.synchronize()
            ms_tc = t0.elapsed_time(t1) / args.steps
            num = den = 0.0
            for a0 in range(0, X.shape[0], 64):
                d = (Xtc[a0:a0 + 64] - X[a0:a0 + 64]).to(torch.complex128)
                num += (torch.linalg.vector_norm(d) ** 2).item()
                den += (torch.linalg.vector_norm(X[a0:a0 + 64].to(torch.complex128)) ** 2).item()
            tc = {"ms": round(ms_tc, 4), "plain_ms": round(ms, 4), "speedup_vs_plain": round(ms / ms_tc, 4),
                  "rel_l2_vs_plain": math.sqrt(num / den),
                  "what": "FP32 1024-point Y/Z stages as tensor-core products (mma.sync TF32, each operand split "
                          "into a TF32 head and tail, 3 products accumulated in FP32); X stages as plain",
                  "oracle_check": "tests/test_gpu_fullsize.py: within 5e-6 of the FP64 oracle at 1024^3"}
            del Xtc, ytc, wtc, ptc
            torch.cuda.empty_cache()

    # round-trip sanity (torch reduction on the device, test-style check only)
    num = den = 0.0
    for z0 in range(0, NZ, 64):  # chunked FP64 reductions (the 2048^3 arrays are 34 GB)
        xd = x[z0:z0 + 64].double()
        num += (torch.linalg.vector_norm(y[z0:z0 + 64].double() / plan.scale - xd) ** 2).item()
        den += (torch.linalg.vector_norm(xd) ** 2).item()
    rt = math.sqrt(num / den)

    out = {
        "metric": METRIC, "value": job_value(ms, world), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(), "grid": [NX, NY, NZ], "precision": PREC, "layout": LAYOUT,
                   "input": "turbulence_field(seed=rank): k^-5/3 random-phase modes + 16 plane waves, unit RMS",
                   "l2": "no flush: every array (4.3 GB) is larger than L2 (129 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "hbm_roofline_frac": round(roof_ms / ms, 4),
        "roofline_ms": round(roof_ms, 4),
        "roofline_ms_unfused_stage_model": round(roof_ms_unfused, 4),
        "gflops": round(2 * 5 * NX * NY * NZ * math.log2(NX * NY * NZ) / (ms * 1e-3) / 1e9, 1),
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": round(dom_gbs, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(dom_gbs / peak, 4),
                     "traffic": traffic, "algorithmic_bytes": gbytes[dom]},
        "stages": stages,
        "e2e": {"value": job_value(e2e_ms, world), "unit": "ms", "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
                "d2h_bytes_per_step": int(yh.numel() * yh.element_size()),
                "mode": "pinned host -> device -> pinned host every step, double-buffered on three streams "
                        "(copies of neighbouring steps overlap the transforms)",
                "serial_value": job_value(e2e_serial_ms, world)},
        "gpu_launches": int(sum(plan.launches(d) for d in (0, 1)) * args.steps),
        "round_trip_rel_l2": rt,
        "tc_split": tc,
        "clocks": clk.summary(),
        "plan": desc,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cms, cores, desc = cpu_oracle_sample(1.0 / 8)
        out["cpu_baseline"] = {"value": cms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": desc,
                               "estimated": True, "sample_fraction": sample_fraction(1.0 / 8)}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()



# ---------------------------------------------------------------------------
# --report: every benchmark configuration, one JSON line each (not the
# default single-line benchmark output; used to fill profiles/configs_report.md)
# ---------------------------------------------------------------------------
REPORT_CONFIGS = [
    # name, (nx, ny, nz), precision, ttypes, layout, input
    ("32cube_f64", (32, 32, 32), "f64", ("fft", "fft", "fft"), "zyx", "config1"),
    ("512cube_f32", (512, 512, 512), "f32", ("fft", "fft", "fft"), "zyx", "turbulence"),
    ("512cube_f64", (512, 512, 512), "f64", ("fft", "fft", "fft"), "zyx", "turbulence"),
    ("1024cube_f32", (1024, 1024, 1024), "f32", ("fft", "fft", "fft"), "zyx", "turbulence"),
    ("2048cube_f32", (2048, 2048, 2048), "f32", ("fft", "fft", "fft"), "zyx", "turbulence"),
    ("channel_480x360x257_f64", (480, 360, 257), "f64", ("fft", "fft", "cheb"), "zyx", "channel"),
    ("sine_512x512x255_f32", (512, 512, 255), "f32", ("fft", "fft", "sine"), "zyx", "turbulence"),
    ("inplace_512cube_f32_xyz", (512, 512, 512), "f32", ("fft", "fft", "fft"), "xyz", "turbulence", "inplace"),
    # the generic mixed-radix kernel: an even 7-smooth grid, and odd X rows in pairs
    ("smooth_384cube_f32", (384, 384, 384), "f32", ("fft", "fft", "fft"), "zyx", "turbulence"),
    ("odd_375x360x343_f32", (375, 360, 343), "f32", ("fft", "fft", "fft"), "zyx", "turbulence"),
]


def _report_one(name, dims, prec, ttypes, layout, kind, mode="", *, steps, warmup):
    import numpy as np
    import torch

    from paper_1905_02803_gb300 import inputs
    from paper_1905_02803_gb300 import p3dfft as P

    nx, ny, nz = dims
    inplace = mode == "inplace"
    plan = P.Plan(nx, ny, nz, precision=prec, ttypes=ttypes, layout=layout,
                  flags=P.P3_FLAG_PADDED_REAL if inplace else 0)
    npdt = np.float32 if prec == "f32" else np.float64
    if kind == "config1":
        x = torch.from_numpy(inputs.config1_field(nx, 0)[0]).to("cuda", plan.real_dtype)
    elif kind == "channel":
        x = inputs.channel_field(nx, ny, nz, seed=0, dtype=npdt, device=plan.device)
    else:
        x = inputs.turbulence_field((nz, ny, nx), seed=0, dtype=npdt, device=plan.device)
    if inplace:
        # one padded buffer [nz][ny][2H]: forward and inverse both run with
        # in == out; it is refilled from x outside each timed pair
        buf = torch.zeros(plan.real_shape, dtype=plan.real_dtype, device=plan.device)
        X = plan.complex_view(buf)
        ws = None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(warmup + steps):
            buf[..., :nx].copy_(x)
            if i >= warmup:
                ev[i - warmup][0].record()
            plan.forward(buf, X)
            plan.backward(X, buf)
            if i >= warmup:
                ev[i - warmup][1].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        y = buf[..., :nx]
    else:
        X = plan.empty_complex()
        y = plan.empty_real()
        ws = plan.workspace()
        for _ in range(warmup):
            plan.forward(x, X, ws)
            plan.backward(X, y, ws)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(steps):
            plan.forward(x, X, ws)
            plan.backward(X, y, ws)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
    e = 4 if prec == "f32" else 8
    g = plan_groups(plan)
    pair_bytes = sum(launch_bytes(n, nx, ny, nz, e) for d in (0, 1) for n in g[d])
    peak, _ = peaks()
    roof_ms = pair_bytes / (peak * 1e9) * 1e3
    N = nx * ny * nz
    gflops = 2 * 5 * N * math.log2(N) / (ms * 1e-3) / 1e9
    num = den = 0.0
    for z0 in range(0, nz, 64):  # chunked FP64 reductions (2048^3 arrays are 34 GB)
        xd = x[z0:z0 + 64].double()
        num += (torch.linalg.vector_norm(y[z0:z0 + 64].double() / plan.scale - xd) ** 2).item()
        den += (torch.linalg.vector_norm(xd) ** 2).item()
    rt = math.sqrt(num / den)
    out = {"config": name, "grid": list(dims), "precision": prec, "ttypes": list(ttypes), "layout": layout,
           "in_place": inplace,
           "ms": round(ms, 4), "gflops": round(gflops, 1), "stage_model_bytes": pair_bytes,
           "hbm_roofline_ms": round(roof_ms, 4), "hbm_roofline_frac": round(roof_ms / ms, 4)}
    if prec == "f64":
        # the FP64 transforms are bound by the FP64 pipe: their roofline is
        # max(HBM time, FP64-pipe instructions / measured FP64 issue rate),
        # the rate being the DGEMM peak over 2 flop per DFMA (a DADD or DMUL
        # takes the pipe for the same slot as a DFMA)
        ops = fp64_ops_record(name)
        pk = fp64_peak_tflops()
        out["fp64_peak_tflops"] = round(pk, 3)
        out["fp64_peak_kind"] = "measured (cuBLAS DGEMM, torch.matmul float64 4096^3, best of 5)"
        if ops is not None:
            flop, inst = ops
            alu_ms = inst / (pk * 1e12 / 2.0) * 1e3
            out["fp64_flop_per_pair"] = flop
            out["fp64_inst_per_pair"] = inst
            out["fp64_flop_frac"] = round(flop / (pk * 1e12) * 1e3 / ms, 4)
            out["fp64_alu_ms"] = round(alu_ms, 4)
            out["fp64_alu_frac"] = round(alu_ms / ms, 4)
            out["roofline_bound"] = "fp64" if alu_ms > roof_ms else "hbm"
            out["roofline_frac"] = round(max(alu_ms, roof_ms) / ms, 4)
        else:
            out["fp64_alu_frac"] = None
    out.update({"round_trip_rel_l2": rt,
                "parity": "oracle comparison in tests/test_gpu_fullsize.py and tests/test_gpu_parity.py "
                          "(P3_PARITY_LOG records the measured errors)"})
    return out


def _report_batch(steps, warmup, nstreams=16):
    """64 independent FP32 transforms of 7-smooth sizes: 64 plans one after
    another on one stream, and the same plans as one p3_batch over nstreams
    internal streams; each plain and replayed from a captured CUDA graph."""
    import numpy as np
    import torch

    from paper_1905_02803_gb300 import inputs
    from paper_1905_02803_gb300 import p3dfft as P

    dims = inputs.batch_dims(0)
    plans, xs, Xs, ys = [], [], [], []
    for k, (nx, ny, nz) in enumerate(dims):
        p = P.Plan(nx, ny, nz, precision="f32", layout="zyx")
        plans.append(p)
        xs.append(torch.from_numpy(inputs.gaussian_field((nz, ny, nx), seed=k).astype(np.float32)).cuda())
        Xs.append(p.empty_complex())
        ys.append(p.empty_real())
        p.workspace()
    batch = P.Batch(plans, nstreams=nstreams)

    def serial():
        for p, x, X, y in zip(plans, xs, Xs, ys):
            p.forward(x, X)
            p.backward(X, y)

    def batched():
        batch.forward(xs, Xs)
        batch.backward(Xs, ys)

    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        t0.record()
        for _ in range(steps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    def graphed(fn):
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                fn()
        torch.cuda.synchronize()
        return timed(g.replay)

    pbatch = P.Batch(plans, nstreams=0)
    # the same grids with P3_FLAG_TUNE (radix order and tile height of every
    # generic stage chosen by timing at plan creation)
    tplans = [P.Plan(nx, ny, nz, precision="f32", layout="zyx", flags=P.P3_FLAG_TUNE) for nx, ny, nz in dims]
    for tp in tplans:
        tp.workspace()
    tbatch = P.Batch(tplans, nstreams=nstreams)

    def tuned():
        tbatch.forward(xs, Xs)
        tbatch.backward(Xs, ys)

    def persistent():
        pbatch.forward(xs, Xs)
        pbatch.backward(Xs, ys)

    ms = timed(serial)
    ms_graph = graphed(serial)
    ms_batch = timed(batched)
    ms_batch_graph = graphed(batched)
    ms_pers = timed(persistent)
    ms_pers_graph = graphed(persistent)
    ms_tuned_graph = graphed(tuned)
    pair_bytes = sum(sum(stage_model_bytes(nx, ny, nz, 4)) for nx, ny, nz in dims)
    peak, _ = peaks()
    roof_ms = pair_bytes / (peak * 1e9) * 1e3
    best = min(ms, ms_graph, ms_batch, ms_batch_graph, ms_pers, ms_pers_graph, ms_tuned_graph)
    launches = sum(p.launches(0) + p.launches(1) for p in plans)
    pers_launches = pbatch.launches(0) + pbatch.launches(1)
    kinds = sorted({l.split()[2] for p in plans for l in p.describe().splitlines() if "kernel=" in l})
    return {"config": "batch64_smooth7_f32", "grids": len(dims), "ms": round(best, 4),
            "ms_serial": round(ms, 4), "ms_serial_cuda_graph": round(ms_graph, 4),
            "ms_batch_streams": round(ms_batch, 4), "ms_batch_streams_cuda_graph": round(ms_batch_graph, 4),
            "ms_persistent": round(ms_pers, 4), "ms_persistent_cuda_graph": round(ms_pers_graph, 4),
            "persistent_launches_per_step": pers_launches,
            "ms_batch_streams_cuda_graph_tuned_plans": round(ms_tuned_graph, 4),
            "batch_streams": nstreams, "stage_model_bytes": pair_bytes, "hbm_roofline_ms": round(roof_ms, 4),
            "hbm_roofline_frac": round(roof_ms / best, 4), "launches_per_step": launches, "kernels": kinds}


CPU_REPORT_CONFIGS = [
    # name, (nx, ny, nz), oracle transform types, single-thread run too
    ("32cube_f64", (32, 32, 32), (0, 0, 0), True),
    ("256cube_f64", (256, 256, 256), (0, 0, 0), True),
    ("512cube_f64", (512, 512, 512), (0, 0, 0), False),
    ("channel_480x360x257_f64", (480, 360, 257), (0, 0, 1), False),
]


def run_cpu_report():
    """The CPU baseline at the small configurations: the FP64 oracle's whole
    forward + inverse pair (not a line sample), best of three (one at 512^3
    and for the channel grid), on every host thread and, where it stays short,
    on one.  One JSON line per configuration and thread count."""
    import oracle as O
    from paper_1905_02803_gb300 import inputs

    for name, (nx, ny, nz), tt, single in CPU_REPORT_CONFIGS:
        f = inputs.uniform_field((nz, ny, nx), 1)
        reps = 3 if nx * ny * nz <= 256 ** 3 else 1
        for nthreads in ([0, 1] if single else [0]):
            best = None
            for _ in range(reps):
                t = time.perf_counter()
                F = O.forward(f, tt, nthreads=nthreads)
                O.backward(F, nx, tt, nthreads=nthreads)
                dt = time.perf_counter() - t
                best = dt if best is None else min(best, dt)
            print(json.dumps({"config": name, "grid": [nx, ny, nz], "kind": "oracle", "cpu_ms": round(best * 1e3, 3),
                              "threads": nthreads or O.nthreads_default(), "reps": reps}), flush=True)


def run_report(args):
    import torch
    torch.cuda.set_device(0)
    only = set(filter(None, args.report_only.split(",")))
    for c in REPORT_CONFIGS:
        if only and c[0] not in only:
            continue
        steps = 3 if c[1][0] >= 2048 else 20
        r = _report_one(*c, steps=steps, warmup=3)
        print(json.dumps(r), flush=True)
        torch.cuda.empty_cache()
    if not only or "batch64" in only:
        print(json.dumps(_report_batch(10, 2)), flush=True)


if __name__ == "__main__":
    main()
