"""Shared helpers for the GPU parity tests (GPU path vs the FP64 oracle)."""
import json
import os

import numpy as np

import oracle as O
from paper_1905_02803_gb300 import inputs

TOL = {"f32": 2e-6, "f64": 1e-13}
TOL_TC = 5e-6  # tensor-core split-precision stages (FP32 data)
TT = {"fft": O.FFT, "cheb": O.CHEB, "empty": O.EMPTY, "sine": O.SINE}


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) or np.iscomplexobj(ref) else np.float64)
    ref = np.asarray(ref)
    n = np.linalg.norm(ref.ravel())
    d = np.linalg.norm((got - ref).ravel())
    return d / n if n > 0 else d


def log_parity(**kw):
    """Append one JSON line to the file P3_PARITY_LOG names (if set): the
    measured errors that the benchmark report quotes."""
    path = os.environ.get("P3_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(kw) + "\n")


def random_complex(shape, seed):
    n = int(np.prod(shape))
    return (inputs.normal(seed, 60, n) + 1j * inputs.normal(seed, 62, n)).reshape(shape)


def check_case(nx, ny, nz, prec="f64", ttypes=("fft", "fft", "fft"), layout="zyx", field=None, seed=0,
               check_inverse=True, flags=0, label=None):
    """Forward of a real field and inverse of a random (non-Hermitian) complex
    array, each compared element by element with the oracle; returns errors."""
    import torch
    from paper_1905_02803_gb300.p3dfft import Plan

    plan = Plan(nx, ny, nz, precision=prec, ttypes=ttypes, layout=layout, flags=flags)
    if field is None:
        field = inputs.uniform_field((nz, ny, nx), seed)
    x = torch.from_numpy(np.ascontiguousarray(field)).to(device="cuda", dtype=plan.real_dtype)
    X = plan.forward(x)
    xin = x.double().cpu().numpy()  # the exact values the GPU saw
    tt = tuple(TT[t] for t in ttypes)
    ref = O.forward(xin, tt)
    if layout == "zyx":
        ref = O.to_zyx(ref)
    torch.cuda.synchronize()
    err_f = rel_l2(X.cpu().numpy(), ref)
    err_b = None
    if check_inverse:
        G = random_complex((nz, ny, nx // 2 + 1), seed + 1)
        Gd = torch.from_numpy(O.to_zyx(G) if layout == "zyx" else G).to(device="cuda", dtype=plan.complex_dtype)
        g = plan.backward(Gd)
        Gin = Gd.cpu().numpy().astype(np.complex128)
        Gin = O.from_zyx(Gin) if layout == "zyx" else Gin
        refb = O.backward(Gin, nx, tt)
        torch.cuda.synchronize()
        err_b = rel_l2(g.cpu().numpy(), refb)
    if label:
        log_parity(check="forward+inverse", config=label, grid=[nx, ny, nz], precision=prec, ttypes=list(ttypes),
                   layout=layout, compared="whole array", rel_l2_forward=err_f, rel_l2_inverse=err_b)
    return err_f, err_b, plan
