"""ctypes binding of the FP64 CPU oracle (oracle/p3_oracle.c).

TEST INFRASTRUCTURE ONLY: the product path never imports this module.

Conventions (P3DFFT paper, Sect. 3.2 and Table 1, with one process holding
the whole grid):
  real arrays     numpy float64  [Nz][Ny][Nx]          (X fastest)
  complex arrays  numpy complex128 [Nz][Ny][H], H = Nx//2 + 1  (XYZ storage)
  ZYX storage     [H][Ny][Nz] (the STRIDE1 Z-pencil of Table 1), produced here
                  only by the trivial permutation to_zyx().
Transform types per dimension: FFT, CHEB (DCT-I, third dimension only), EMPTY,
SINE (DST-I, third dimension only).
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

FFT, CHEB, EMPTY, SINE = 0, 1, 2, 3

_lib = None


def nthreads_default() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    L, I, P = ctypes.c_long, ctypes.c_int, ctypes.c_void_p
    lib.p3o_fft1d.argtypes = [L, P, P, I]
    lib.p3o_dct1.argtypes = [L, P, P]
    lib.p3o_x_r2c_rows.argtypes = [L, P, P, L, L, I]
    lib.p3o_x_c2r_rows.argtypes = [L, P, P, L, L, I]
    lib.p3o_c2c_lines.argtypes = [L, L, L, L, L, P, L, L, I, I]
    lib.p3o_dct1_lines.argtypes = [L, L, L, L, L, P, L, L, I]
    lib.p3o_dst1.argtypes = [L, P, P]
    lib.p3o_dst1_lines.argtypes = [L, L, L, L, L, P, L, L, I]
    lib.p3o_forward.argtypes = [L, L, L, I, I, P, P, I]
    lib.p3o_phase_sum_yz.argtypes = [L, L, L, P, I, L, L, L, P, P, I, P, I]
    lib.p3o_backward.argtypes = [L, L, L, I, I, P, P, I]
    for name in ("p3o_fft1d", "p3o_dct1", "p3o_x_r2c_rows", "p3o_x_c2r_rows",
                 "p3o_c2c_lines", "p3o_dct1_lines", "p3o_forward", "p3o_backward", "p3o_phase_sum_yz", "p3o_dst1", "p3o_dst1_lines"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def half(nx: int) -> int:
    """H = floor(Nx/2) + 1 complex bins per X line (Sect. 3.2)."""
    return nx // 2 + 1


def scale(nx: int, ny: int, nz: int, ttypes=(FFT, FFT, FFT)) -> float:
    """Round-trip factor of the unnormalised pair (Sect. 4.1 'apart from a
    scale factor'): the product over dimensions of n for FFT, 2(n-1) for
    Chebyshev (DCT-I applied twice), 2(n+1) for the sine transform (DST-I
    applied twice) and 1 for the empty transform."""
    s = float(nx)
    for n, t in ((ny, ttypes[1]), (nz, ttypes[2])):
        s *= {FFT: float(n), CHEB: 2.0 * (n - 1), EMPTY: 1.0, SINE: 2.0 * (n + 1)}[t]
    return s


def fft1d(x, sign: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(_load().p3o_fft1d(x.size, _ptr(x), _ptr(out), sign), "fft1d")
    return out


def dct1(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(_load().p3o_dct1(x.size, _ptr(x), _ptr(out)), "dct1")
    return out


def dst1(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(_load().p3o_dst1(x.size, _ptr(x), _ptr(out)), "dst1")
    return out


def forward(f, ttypes=(FFT, FFT, FFT), nthreads: int = 0) -> np.ndarray:
    """3D forward transform of a real [Nz][Ny][Nx] array -> [Nz][Ny][H]."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    F = np.empty((nz, ny, half(nx)), dtype=np.complex128)
    rc = _load().p3o_forward(nx, ny, nz, ttypes[1], ttypes[2], _ptr(f), _ptr(F),
                             nthreads or nthreads_default())
    _check(rc, "forward")
    return F


def backward(F, nx: int, ttypes=(FFT, FFT, FFT), nthreads: int = 0) -> np.ndarray:
    """3D inverse transform of a complex [Nz][Ny][H] array -> real [Nz][Ny][Nx]."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    nz, ny, H = F.shape
    if H != half(nx):
        raise ValueError("complex array has %d bins per X line, expected %d" % (H, half(nx)))
    f = np.empty((nz, ny, nx), dtype=np.float64)
    rc = _load().p3o_backward(nx, ny, nz, ttypes[1], ttypes[2], _ptr(F), _ptr(f),
                              nthreads or nthreads_default())
    _check(rc, "backward")
    return f


def to_zyx(F) -> np.ndarray:
    """XYZ [Nz][Ny][H] -> ZYX [H][Ny][Nz] (Table 1, STRIDE1 Z-pencil)."""
    return np.ascontiguousarray(np.transpose(F, (2, 1, 0)))


def from_zyx(G) -> np.ndarray:
    """ZYX [H][Ny][Nz] -> XYZ [Nz][Ny][H]."""
    return np.ascontiguousarray(np.transpose(G, (2, 1, 0)))


# --- stage-level entry points (used for line-sampled checks and timing) ---

def x_r2c_rows(nx, f_flat, F_flat, r0, r1, nthreads=0):
    _check(_load().p3o_x_r2c_rows(nx, _ptr(f_flat), _ptr(F_flat), r0, r1,
                                  nthreads or nthreads_default()), "x_r2c_rows")


def x_c2r_rows(nx, F_flat, f_flat, r0, r1, nthreads=0):
    _check(_load().p3o_x_c2r_rows(nx, _ptr(F_flat), _ptr(f_flat), r0, r1,
                                  nthreads or nthreads_default()), "x_c2r_rows")


def c2c_lines(n, per, gstride, lstride, es, data, l0, l1, sign, nthreads=0):
    _check(_load().p3o_c2c_lines(n, per, gstride, lstride, es, _ptr(data), l0, l1,
                                 sign, nthreads or nthreads_default()), "c2c_lines")


def dst1_lines(n, per, gstride, lstride, es, data, l0, l1, nthreads=0):
    _check(_load().p3o_dst1_lines(n, per, gstride, lstride, es, _ptr(data), l0, l1,
                                  nthreads or nthreads_default()), "dst1_lines")


def dct1_lines(n, per, gstride, lstride, es, data, l0, l1, nthreads=0):
    _check(_load().p3o_dct1_lines(n, per, gstride, lstride, es, _ptr(data), l0, l1,
                                  nthreads or nthreads_default()), "dct1_lines")


# --- sampled outputs of the definition on full-size grids ---

_TYPES = {np.dtype(np.float32): 0, np.dtype(np.float64): 1, np.dtype(np.complex64): 2,
          np.dtype(np.complex128): 3}


class PhaseSum:
    """Accumulates g[k][x] = sum_{z,y} A[z][y][x] exp(sign 2 pi i (a_k y/ny + b_k z/nz))
    over z-chunks of an [nz][ny][nx] array fed in order (so a full-size array
    never has to be on the host at once)."""

    def __init__(self, nx, ny, nz, a, b, sign, nthreads=0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.a = np.ascontiguousarray(a, dtype=np.int64)
        self.b = np.ascontiguousarray(b, dtype=np.int64)
        self.sign = sign
        self.g = np.zeros((len(self.a), nx), dtype=np.complex128)
        self.nthreads = nthreads or nthreads_default()

    def add(self, chunk, z0):
        chunk = np.ascontiguousarray(chunk)
        z1 = z0 + chunk.shape[0]
        rc = _load().p3o_phase_sum_yz(self.nx, self.ny, self.nz, _ptr(chunk), _TYPES[chunk.dtype], z0, z1,
                                      len(self.a), _ptr(self.a), _ptr(self.b), self.sign, _ptr(self.g),
                                      self.nthreads)
        _check(rc, "phase_sum_yz")


def forward_lines(g, nx):
    """Finish sampled forward lines: F[kx] = DFT_x(g)[kx], kx < H."""
    return np.stack([fft1d(row, -1)[:half(nx)] for row in g])


def backward_rows(g, nx):
    """Finish sampled inverse rows: the weighted c2r of each accumulated line."""
    H = half(nx)
    G = np.ascontiguousarray(g[:, :H], dtype=np.complex128)
    out = np.zeros((G.shape[0], nx))
    x_c2r_rows(nx, G.reshape(-1), out.reshape(-1), 0, G.shape[0])
    return out


# --- whole sampled planes of the output on full-size grids -----------------

def forward_kx_planes(chunks, nx, ny, nz, kxs, nthreads=0):
    """Forward output planes F[kx][ky][kz] (ZYX order: one [Ny][Nz] plane per
    requested kx) of a real [Nz][Ny][Nx] field fed as (z0, block) z-chunks in
    order.  The stages are the definition's three passes (Sect. 2): the X
    real-to-complex transform of every row (oracle rows), keeping bins kxs;
    then the Y and Z complex transforms of those planes (oracle lines)."""
    kxs = np.asarray(kxs, dtype=np.int64)
    H = half(nx)
    if np.any(kxs < 0) or np.any(kxs >= H):
        raise ValueError("kx outside the half spectrum")
    nk = len(kxs)
    G = np.empty((nk, nz, ny), dtype=np.complex128)  # [k][z][y]
    zdone = 0
    for z0, block in chunks:
        block = np.ascontiguousarray(block, dtype=np.float64)
        zc = block.shape[0]
        if z0 != zdone or block.shape[1:] != (ny, nx):
            raise ValueError("chunks must cover z in order with [zc][Ny][Nx] blocks")
        F = np.empty(zc * ny * H, dtype=np.complex128)
        x_r2c_rows(nx, block.reshape(-1), F, 0, zc * ny, nthreads)
        G[:, z0:z0 + zc, :] = F.reshape(zc, ny, H)[:, :, kxs].transpose(2, 0, 1)
        zdone += zc
    if zdone != nz:
        raise ValueError("chunks cover %d of %d planes" % (zdone, nz))
    flat = G.reshape(-1)
    if ny > 1:  # Y lines: line L = k * nz + z at L * ny, unit stride
        c2c_lines(ny, nk * nz, 0, ny, 1, flat, 0, nk * nz, -1, nthreads)
    if nz > 1:  # Z lines: line L = k * ny + y at k * nz * ny + y, stride ny
        c2c_lines(nz, ny, nz * ny, 1, ny, flat, 0, nk * ny, -1, nthreads)
    return np.ascontiguousarray(G.transpose(0, 2, 1))  # [k][ky][kz]


def inverse_z_table(nz, zs, sign=+1):
    """T[kz][j] = exp(sign 2 pi i kz zs[j] / Nz), the product kz * z reduced
    mod Nz exactly in integers before the FP64 cos / sin."""
    kz = np.arange(nz, dtype=np.int64)
    t = np.mod(np.outer(kz, np.asarray(zs, dtype=np.int64)), nz).astype(np.float64)
    ang = 2.0 * math.pi * t / nz
    return np.cos(ang) + sign * 1j * np.sin(ang)


def backward_z_planes(chunks, nx, ny, nz, zs, nthreads=0):
    """Inverse output planes f[z][y][x] for the requested z of a complex ZYX
    input [H][Ny][Nz] fed as (kx0, block) kx-chunks in order.  The inverse Z
    transform is the definition sum sum_kz F[kx][ky][kz] exp(+2 pi i kz z/Nz)
    evaluated at those z only (a matrix product with exact-index roots of
    unity); the inverse Y transform (oracle lines) and the weighted c2r of
    every row (oracle rows, Sect. 3.2 reading of the redundant bins) finish
    each plane."""
    zs = np.asarray(zs, dtype=np.int64)
    H = half(nx)
    nzs = len(zs)
    T = inverse_z_table(nz, zs)
    Q = np.empty((nzs, ny, H), dtype=np.complex128)  # [j][y][kx]
    kdone = 0
    for k0, block in chunks:
        block = np.ascontiguousarray(block, dtype=np.complex128)
        kc = block.shape[0]
        if k0 != kdone or block.shape[1:] != (ny, nz):
            raise ValueError("chunks must cover kx in order with [kc][Ny][Nz] blocks")
        A = block.reshape(kc * ny, nz) @ T  # [(k, y)][j]
        Q[:, :, k0:k0 + kc] = A.reshape(kc, ny, nzs).transpose(2, 1, 0)
        kdone += kc
    if kdone != H:
        raise ValueError("chunks cover %d of %d kx planes" % (kdone, H))
    flat = Q.reshape(-1)
    if ny > 1:  # Y lines: line L = j * H + kx at j * ny * H + kx, stride H
        c2c_lines(ny, H, ny * H, 1, H, flat, 0, nzs * H, +1, nthreads)
    out = np.empty(nzs * ny * nx, dtype=np.float64)
    x_c2r_rows(nx, flat, out, 0, nzs * ny, nthreads)
    return out.reshape(nzs, ny, nx)
