"""Seeded synthetic inputs shaped like the P3DFFT paper's workloads.

This module holds no transform arithmetic: it draws numbers and evaluates
closed-form fields (plane waves, Chebyshev polynomials on Gauss-Lobatto
points) in real space.  Both the CUDA path and the CPU oracle take their
inputs from here, so the two sides always see the same array.

Random numbers come from a counter-based generator: value i of stream s under
seed S is splitmix64 applied to the state (key(S, s) + (i + 1) * 0x9E3779B97F4A7C15),
where key(S, s) = splitmix64(S * 2^20 + s).  Uniform doubles take the top
53 bits; normals use Box-Muller on two uniform streams.  Every array is a pure
function of (seed, stream, index), so any sub-block can be regenerated alone.

Fields (all real, C row-major [Nz][Ny][Nx]):
  uniform_field      i.i.d. U[lo, hi)
  plane_wave_sin     sin(2 pi k x / Nx)
  turbulence_field   random-phase sum of Fourier modes whose shell energy
                     falls as k^(-5/3), plus 16 random plane waves, scaled to
                     unit RMS (stands in for the paper's turbulence fields)
  channel_field      sum of 64 Fourier(x, y) x T_n(z) modes on Gauss-Lobatto
                     points z_j = cos(pi j / (Nz-1)), n <= Nz-1 (always with
                     n = 0 and n = Nz-1), plus 1e-3 uniform noise
  gaussian_field     i.i.d. N(0, 1)
  uniform_field_device  uniform_field evaluated by torch on a device (or the
                     host), bit-identical to the numpy form, in z-chunks
  power_law_half_spectrum  seeded half-spectrum [Nz][Ny][Nx/2+1] with power
                     |k|^slope per bin (k on signed wavenumbers), uniform
                     phases, zero mean (a random-phase Gaussian random field
                     once transformed to real space, which this module does
                     not do)
  plane_waves        16 random-amplitude plane waves
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(int(seed) * (1 << 20) + int(stream)) & ((1 << 64) - 1)], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(s + _GAMMA)[0]


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Raw 64-bit outputs start .. start+count-1 of one stream."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed, stream) + idx * _GAMMA)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """U[0, 1) doubles."""
    return (u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """N(0, 1) doubles by Box-Muller from streams (stream, stream + 1)."""
    u1 = uniform(seed, stream, count, start)
    u2 = uniform(seed, stream + 1, count, start)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def randint(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi] (inclusive), by multiply-shift on 53-bit uniforms."""
    u = uniform(seed, stream, count)
    return lo + np.minimum(np.floor(u * (hi - lo + 1)).astype(np.int64), hi - lo)


# ---------------------------------------------------------------------------
# Real-space building blocks
# ---------------------------------------------------------------------------

def _phase_table(n: int, k: np.ndarray) -> np.ndarray:
    """exp(2 pi i k x / n) for x < n, rows per k, with (k x) reduced mod n exactly."""
    x = np.arange(n, dtype=np.int64)
    t = np.mod(np.outer(np.asarray(k, dtype=np.int64), x), n).astype(np.float64)
    return np.exp(2j * math.pi * t / n)


def _cheb_table(nz: int, orders: np.ndarray) -> np.ndarray:
    """T_n(z_j) = cos(pi n j / M) on Gauss-Lobatto points, M = nz - 1, exact index."""
    M = nz - 1
    j = np.arange(nz, dtype=np.int64)
    t = np.mod(np.outer(np.asarray(orders, dtype=np.int64), j), 2 * M).astype(np.float64)
    return np.cos(math.pi * t / M)


def gauss_lobatto(nz: int) -> np.ndarray:
    """z_j = cos(pi j / (nz - 1)), j = 0..nz-1 (descending from +1 to -1)."""
    return np.cos(math.pi * np.arange(nz) / (nz - 1))


def _rank_sum(cz: np.ndarray, cy: np.ndarray, cx: np.ndarray, device=None,
              dtype=np.float64):
    """Re sum_m cz[m, z] cy[m, y] cx[m, x] as a real [Nz][Ny][Nx] array.

    Evaluated as a (Nz*Ny x M) by (M x Nx) product, either with numpy in FP64
    on the host (device None) or with torch on a CUDA device in the output
    precision, in z-chunks."""
    M, nz = cz.shape
    ny, nx = cy.shape[1], cx.shape[1]
    if device is None:
        out = np.empty((nz, ny, nx), dtype=dtype)
        zc = max(1, min(nz, (1 << 24) // max(1, ny * M)))
        for z0 in range(0, nz, zc):
            z1 = min(nz, z0 + zc)
            A = (cz[:, z0:z1, None] * cy[:, None, :]).reshape(M, -1).T  # [(z,y), m]
            block = A.real @ cx.real - A.imag @ cx.imag
            out[z0:z1] = block.reshape(z1 - z0, ny, nx)
        return out
    import torch
    tdt = {np.float32: torch.float32, np.float64: torch.float64}[np.dtype(dtype).type]
    # evaluated in the output precision (full-precision FP32 products, no TF32)
    torch.backends.cuda.matmul.allow_tf32 = False
    out = torch.empty((nz, ny, nx), dtype=tdt, device=device)
    czr = torch.from_numpy(np.ascontiguousarray(cz.real)).to(device=device, dtype=tdt)
    czi = torch.from_numpy(np.ascontiguousarray(cz.imag)).to(device=device, dtype=tdt)
    cyr = torch.from_numpy(np.ascontiguousarray(cy.real)).to(device=device, dtype=tdt)
    cyi = torch.from_numpy(np.ascontiguousarray(cy.imag)).to(device=device, dtype=tdt)
    cxr = torch.from_numpy(np.ascontiguousarray(cx.real)).to(device=device, dtype=tdt)
    cxi = torch.from_numpy(np.ascontiguousarray(cx.imag)).to(device=device, dtype=tdt)
    zc = max(1, min(nz, (1 << 26) // max(1, ny * M)))
    for z0 in range(0, nz, zc):
        z1 = min(nz, z0 + zc)
        ar = czr[:, z0:z1, None] * cyr[:, None, :] - czi[:, z0:z1, None] * cyi[:, None, :]
        ai = czr[:, z0:z1, None] * cyi[:, None, :] + czi[:, z0:z1, None] * cyr[:, None, :]
        ar = ar.reshape(M, -1).T
        ai = ai.reshape(M, -1).T
        block = ar @ cxr - ai @ cxi
        out[z0:z1] = block.reshape(z1 - z0, ny, nx).to(tdt)
    return out


# ---------------------------------------------------------------------------
# Fields
# ---------------------------------------------------------------------------

def uniform_field(shape, seed: int = 0, lo: float = -1.0, hi: float = 1.0,
                  stream: int = 1) -> np.ndarray:
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform(seed, stream, n)).reshape(shape)


def gaussian_field(shape, seed: int = 0, stream: int = 3) -> np.ndarray:
    n = int(np.prod(shape))
    return normal(seed, stream, n).reshape(shape)


def plane_wave_sin(shape, kx: int) -> np.ndarray:
    """sin(2 pi kx x / Nx), constant in y and z."""
    nz, ny, nx = shape
    t = np.mod(kx * np.arange(nx, dtype=np.int64), nx).astype(np.float64)
    row = np.sin(2.0 * math.pi * t / nx)
    return np.broadcast_to(row, shape).copy()


def cosine_mode(shape, kx: int, ky: int, kz: int, phase: float = 0.0) -> np.ndarray:
    """cos(2 pi (kx x/Nx + ky y/Ny + kz z/Nz) + phase)."""
    nz, ny, nx = shape
    ex = _phase_table(nx, np.array([kx]))
    ey = _phase_table(ny, np.array([ky]))
    ez = _phase_table(nz, np.array([kz])) * np.exp(1j * phase)
    return _rank_sum(ez, ey, ex)


def config1_field(n: int = 32, seed: int = 0):
    """U[-1, 1) field plus the unit plane wave sin(2 pi 3 x / n); returns
    (sum, random part, plane-wave part)."""
    shape = (n, n, n)
    r = uniform_field(shape, seed)
    w = plane_wave_sin(shape, 3)
    return r + w, r, w


def _wave_params(shape, seed: int, n_waves: int):
    """Plane waves: A ~ U[0,1), integer k in [-N/4, N/4] per axis (x, y, z
    columns), phase ~ U[0, 2 pi)."""
    nz, ny, nx = shape
    wa = uniform(seed, 20, n_waves)
    wk = np.stack([randint(seed, 21 + i, n_waves, -(s // 4), s // 4)
                   for i, s in enumerate((nx, ny, nz))], axis=1)
    wphi = 2.0 * math.pi * uniform(seed, 24, n_waves)
    return wa, wk, wphi


def _turbulence_modes(shape, seed: int, n_modes: int, n_waves: int):
    nz, ny, nx = shape
    kmax = max(1.0, min(nx, ny, nz) / 2.0)
    # spectrum modes: |k| log-uniform in [1, kmax], isotropic direction,
    # amplitude k^(-1/3) so that the energy per unit k falls as k^(-5/3)
    u = uniform(seed, 10, n_modes)
    mag = np.exp(u * math.log(kmax))
    d = normal(seed, 11, 3 * n_modes).reshape(n_modes, 3)
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-300)
    k = np.rint(d * mag[:, None]).astype(np.int64)
    k[np.all(k == 0, axis=1), 0] = 1
    kn = np.linalg.norm(k.astype(np.float64), axis=1)
    amp = kn ** (-1.0 / 3.0)
    phi = 2.0 * math.pi * uniform(seed, 13, n_modes)
    wa, wk, wphi = _wave_params(shape, seed, n_waves)
    K = np.concatenate([k, wk], axis=0)
    A = np.concatenate([amp, wa])
    P = np.concatenate([phi, wphi])
    return K, A, P


def turbulence_field(shape, seed: int = 0, n_modes: int = 240, n_waves: int = 16,
                     dtype=np.float64, device=None):
    """Random-phase modal field with a k^(-5/3) shell spectrum plus n_waves
    random plane waves, normalised to unit RMS (analytically: each cosine
    mode with a distinct +-k carries mean square A^2/2).

    device=None returns a numpy array; a torch device returns a torch tensor
    evaluated there with the same formula."""
    nz, ny, nx = shape
    K, A, P = _turbulence_modes(shape, seed, n_modes, n_waves)
    # merge duplicate and +-k pairs: cos(k.x + p) with k -> -k is cos(-k.x - p)
    coef = {}
    for (kx, ky, kz), a, p in zip(K.tolist(), A.tolist(), P.tolist()):
        key = (kx % nx, ky % ny, kz % nz)
        neg = ((-kx) % nx, (-ky) % ny, (-kz) % nz)
        c = a * complex(math.cos(p), math.sin(p))
        if neg in coef and neg != key:
            coef[neg] = coef[neg] + c.conjugate()
        else:
            coef[key] = coef.get(key, 0.0) + c
    keys = sorted(coef)
    ks = np.array(keys, dtype=np.int64).reshape(-1, 3)
    cs = np.array([coef[k] for k in keys], dtype=np.complex128)
    # mean square of Re(c e^{i k.x}) is |c|^2/2 unless k is its own negative
    self_neg = np.all(np.mod(-ks, [nx, ny, nz]) == ks, axis=1)
    ms = np.where(self_neg, np.real(cs) ** 2, np.abs(cs) ** 2 / 2.0).sum()
    cs = cs / math.sqrt(ms)
    ex = _phase_table(nx, ks[:, 0])
    ey = _phase_table(ny, ks[:, 1])
    ez = _phase_table(nz, ks[:, 2]) * cs[:, None]
    return _rank_sum(ez, ey, ex, device=device, dtype=dtype)


def channel_field(nx: int, ny: int, nz: int, seed: int = 0, n_modes: int = 64,
                  noise: float = 1e-3, dtype=np.float64, device=None):
    """sum_m a_m cos(2 pi (kx_m x/Nx + ky_m y/Ny) + phi_m) T_{n_m}(z_j)
    + noise * U[-1, 1).  a_m ~ U[-1, 1), kx_m < Nx/2, ky_m < Ny/2,
    n_m in [0, Nz-1] with n_0 = 0 and n_1 = Nz-1."""
    M = nz - 1
    a = -1.0 + 2.0 * uniform(seed, 30, n_modes)
    kx = randint(seed, 31, n_modes, 0, max(0, nx // 2 - 1))
    ky = randint(seed, 32, n_modes, 0, max(0, ny // 2 - 1))
    order = randint(seed, 33, n_modes, 0, M)
    order[0] = 0
    if n_modes > 1:
        order[1] = M
    phi = 2.0 * math.pi * uniform(seed, 34, n_modes)
    ex = _phase_table(nx, kx)
    ey = _phase_table(ny, ky) * (a * np.exp(1j * phi))[:, None]
    ez = _cheb_table(nz, order).astype(np.complex128)
    field = _rank_sum(ez, ey, ex, device=device, dtype=dtype)
    nvals = nx * ny * nz
    eps = noise * (-1.0 + 2.0 * uniform(seed, 35, nvals)).reshape(nz, ny, nx)
    if device is None:
        return (field + eps).astype(dtype)
    import torch
    return field + torch.from_numpy(eps).to(device=device, dtype=field.dtype)


def prime_factors(n: int):
    out, p = [], 2
    while p * p <= n:
        while n % p == 0:
            out.append(p)
            n //= p
        p += 1
    if n > 1:
        out.append(n)
    return out


def smooth7_sizes(lo: int = 48, hi: int = 384):
    """All 2/3/5/7-smooth integers in [lo, hi]."""
    return [n for n in range(lo, hi + 1) if all(p <= 7 for p in prime_factors(n))]


def batch_dims(seed: int = 0, count: int = 64, lo: int = 48, hi: int = 384):
    """count grids, each dimension drawn independently from the 7-smooth sizes."""
    sizes = np.array(smooth7_sizes(lo, hi), dtype=np.int64)
    idx = randint(seed, 40, 3 * count, 0, len(sizes) - 1).reshape(count, 3)
    return [tuple(int(sizes[i]) for i in row) for row in idx]


# ---------------------------------------------------------------------------
# The counter-based generator on a torch device (large grids)
# ---------------------------------------------------------------------------

def _i64(v: int) -> int:
    """A 64-bit pattern as the signed value torch's int64 holds."""
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(z, s: int):
    """Logical right shift of int64 bit patterns (torch's >> is arithmetic)."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix_torch(z):
    z = (z ^ _srl(z, 30)) * _i64(int(_M1))
    z = (z ^ _srl(z, 27)) * _i64(int(_M2))
    return z ^ _srl(z, 31)


def uniform_torch(seed: int, stream: int, start: int, count: int, device=None):
    """U[0, 1) doubles start .. start+count-1 of one stream, as a torch FP64
    tensor on `device`: the numpy generator's values, computed with
    wrap-around int64 arithmetic."""
    import torch
    key = _i64(int(_key(seed, stream)))
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = _mix_torch(idx * _i64(int(_GAMMA)) + key)
    return _srl(z, 11).to(torch.float64) * (2.0 ** -53)


def uniform_field_device(shape, seed: int = 0, lo: float = -1.0, hi: float = 1.0, stream: int = 1,
                         device=None, dtype=np.float32, zchunk: int = 0):
    """uniform_field(shape, seed, lo, hi, stream) as a torch tensor of `dtype`
    on `device`, generated there z-plane chunk by chunk (the same values the
    numpy form gives, rounded once to dtype)."""
    import torch
    tdt = {np.float32: torch.float32, np.float64: torch.float64}[np.dtype(dtype).type]
    nz, ny, nx = shape
    plane = ny * nx
    out = torch.empty(shape, dtype=tdt, device=device)
    zc = zchunk or max(1, (1 << 27) // max(1, plane))
    for z0 in range(0, nz, zc):
        z1 = min(nz, z0 + zc)
        u = uniform_torch(seed, stream, z0 * plane, (z1 - z0) * plane, device=device)
        out[z0:z1] = (lo + (hi - lo) * u).view(z1 - z0, ny, nx).to(tdt)
        del u
    return out


# ---------------------------------------------------------------------------
# Spectral-space draws (the caller takes them to real space)
# ---------------------------------------------------------------------------

def power_law_half_spectrum(shape, seed: int = 0, slope: float = -5.0 / 3.0) -> np.ndarray:
    """Half-spectrum S[kz][ky][kx], kx < Nx/2 + 1, with |S|^2 = |k|^slope
    (|k| the length of the signed wavenumber vector (kx, ky', kz'), ky' and
    kz' folded into [-N/2, N/2)), uniform random phases from the seed, and
    S = 0 at k = 0.  Every bin is non-zero: a dense spectrum."""
    nz, ny, nx = shape
    H = nx // 2 + 1
    ky = np.fft.fftfreq(ny) * ny
    kz = np.fft.fftfreq(nz) * nz
    kx = np.arange(H, dtype=np.float64)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (slope / 4.0), 0.0)
    phi = 2.0 * math.pi * uniform(seed, 50, nz * ny * H).reshape(nz, ny, H)
    return amp * np.exp(1j * phi)


def plane_waves(shape, seed: int = 0, n_waves: int = 16, dtype=np.float64, device=None):
    """sum_i A_i cos(2 pi (k_i . x) / N + phi_i), A_i ~ U[0, 1), integer k_i
    in [-N/4, N/4]^3 per axis, phi_i ~ U[0, 2 pi)."""
    nz, ny, nx = shape
    wa, wk, wphi = _wave_params(shape, seed, n_waves)
    ex = _phase_table(nx, wk[:, 0])
    ey = _phase_table(ny, wk[:, 1])
    ez = _phase_table(nz, wk[:, 2]) * (wa * np.exp(1j * wphi))[:, None]
    return _rank_sum(ez, ey, ex, device=device, dtype=dtype)
