"""Pins of the FP64 CPU oracle to facts fixed by the mathematics (CPU only).

The paper prints no worked example, so each oracle function is pinned to
something other than itself: brute-force O(N^2) sums of the definitions on
tiny grids, closed-form plane-wave and Chebyshev-polynomial deltas, Parseval,
Hermitian symmetry, linearity and the round trip.  A dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of
these (test_planted_mistakes checks that on purpose-built broken copies).
"""
import math
import os
import subprocess
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1905_02803_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return d / n if n > 0 else d


def brute_dft(x, sign=-1):
    """Direct O(n^2) DFT with the exponent index (j k mod n) reduced exactly."""
    n = len(x)
    jk = np.mod(np.outer(np.arange(n), np.arange(n)), n)
    return np.exp(sign * 2j * math.pi * jk / n) @ np.asarray(x, dtype=complex)


def brute_forward_3d(f, ttz="fft"):
    """F[kz,ky,kx] = sum over all points of f * phase, one full phase matrix."""
    nz, ny, nx = f.shape
    H = nx // 2 + 1
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(H), indexing="ij")
    # phase (k . r) reduced with a common denominator to stay exact
    den = nx * ny * nz
    num = (np.outer(kx.ravel(), x.ravel()) * (ny * nz)
           + np.outer(ky.ravel(), y.ravel()) * (nx * nz))
    if ttz == "fft":
        num = num + np.outer(kz.ravel(), z.ravel()) * (nx * ny)
        P = np.exp(-2j * math.pi * np.mod(num, den) / den)
        return (P @ f.ravel()).reshape(nz, ny, H)
    P = np.exp(-2j * math.pi * np.mod(num, den) / den)
    if ttz == "sine":
        # DST-I in z: weight 2 sin(pi (z+1)(kz+1) / (nz+1))
        S = 2 * np.sin(math.pi * np.mod(np.outer(kz.ravel() + 1, z.ravel() + 1), 2 * (nz + 1)) / (nz + 1))
        return ((P * S) @ f.ravel()).reshape(nz, ny, H)
    # Chebyshev in z: weight c_j cos(pi j n / M) with c_0 = c_M = 1, else 2
    M = nz - 1
    w = np.where((z.ravel() == 0) | (z.ravel() == M), 1.0, 2.0)
    C = w[None, :] * np.cos(math.pi * np.mod(np.outer(kz.ravel(), z.ravel()), 2 * M) / M)
    return ((P * C) @ f.ravel()).reshape(nz, ny, H)


def brute_backward_3d(F, nx):
    """f[z,y,x] = Re sum_{kx<H} w_kx sum_{ky,kz} F exp(+2 pi i k . r)."""
    nz, ny, H = F.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(H), indexing="ij")
    den = nx * ny * nz
    num = (np.outer(x.ravel(), kx.ravel()) * (ny * nz)
           + np.outer(y.ravel(), ky.ravel()) * (nx * nz)
           + np.outer(z.ravel(), kz.ravel()) * (nx * ny))
    P = np.exp(2j * math.pi * np.mod(num, den) / den)
    w = np.full(H, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[nx // 2] = 1.0
    Fw = (F * w[None, None, :]).ravel()
    return np.real(P @ Fw).reshape(nz, ny, nx)


def rand_real(shape, seed):
    return inputs.uniform_field(shape, seed)


def rand_cplx(shape, seed):
    n = int(np.prod(shape))
    return (inputs.normal(seed, 50, n) + 1j * inputs.normal(seed, 52, n)).reshape(shape)


# --------------------------------------------------------------------------
# 1D FFT (the building block, Sect. 3.3 "each of the three FFTs")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", list(range(1, 34)) + [49, 64, 97, 100, 121, 128, 210, 243, 343, 512])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_brute_force(n, sign):
    x = rand_cplx((n,), n)
    assert rel_l2(O.fft1d(x, sign), brute_dft(x, sign)) < 1e-13


def test_fft1d_delta_and_constant():
    n = 60
    e = np.zeros(n, complex)
    e[7] = 1.0
    X = O.fft1d(e)
    k = np.arange(n)
    assert np.allclose(X, np.exp(-2j * math.pi * 7 * k / n), atol=1e-14)
    assert np.allclose(O.fft1d(np.ones(n)), n * (k == 0), atol=1e-12)


# --------------------------------------------------------------------------
# 3D forward / backward definitions (Sect. 2, Sect. 3.2, Table 1)
# --------------------------------------------------------------------------

SHAPES = [(8, 8, 8), (12, 12, 12), (15, 9, 7), (4, 5, 6), (1, 1, 1), (2, 3, 2),
          (1, 1, 9), (3, 1, 1), (5, 4, 1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_brute_force(shape):
    f = rand_real(shape, 1)
    assert rel_l2(O.forward(f), brute_forward_3d(f)) < 1e-13


@pytest.mark.parametrize("shape", [(8, 8, 8), (15, 9, 7), (4, 5, 6), (2, 3, 2), (1, 1, 9), (3, 2, 1)])
def test_backward_matches_brute_force_non_hermitian(shape):
    nz, ny, nx = shape
    F = rand_cplx((nz, ny, nx // 2 + 1), 2)
    assert rel_l2(O.backward(F, nx), brute_backward_3d(F, nx)) < 1e-13


@pytest.mark.parametrize("shape", [(9, 5, 6), (17, 4, 3), (2, 3, 4), (3, 2, 5)])
def test_forward_chebyshev_matches_brute_force(shape):
    f = rand_real(shape, 3)
    got = O.forward(f, (O.FFT, O.FFT, O.CHEB))
    assert rel_l2(got, brute_forward_3d(f, "cheb")) < 1e-13


@pytest.mark.parametrize("shape", [(9, 5, 6), (1, 4, 3), (2, 3, 4), (7, 2, 5)])
def test_forward_sine_matches_brute_force(shape):
    f = rand_real(shape, 3)
    got = O.forward(f, (O.FFT, O.FFT, O.SINE))
    assert rel_l2(got, brute_forward_3d(f, "sine")) < 1e-13


def test_empty_transforms_are_identity_in_their_dimension():
    f = rand_real((6, 5, 8), 4)
    x_only = O.forward(f, (O.FFT, O.EMPTY, O.EMPTY))
    rows = np.stack([np.fft.fft(r)[:5] for r in f.reshape(-1, 8)]).reshape(6, 5, 5)
    assert rel_l2(x_only, rows) < 1e-13
    xy = O.forward(f, (O.FFT, O.FFT, O.EMPTY))
    full = O.forward(f)
    # the remaining Z FFT applied by brute force along axis 0 closes the gap
    zdft = np.exp(-2j * math.pi * np.mod(np.outer(np.arange(6), np.arange(6)), 6) / 6)
    assert rel_l2(np.einsum("kz,zyx->kyx", zdft, xy), full) < 1e-13


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_plane_wave_32_cubed_single_bin():
    """sin(2 pi 3 x / 32): the only nonzero bin is F[kx=3] = -i N/2."""
    shape = (32, 32, 32)
    F = O.forward(inputs.plane_wave_sin(shape, 3))
    N = 32 ** 3
    assert abs(F[0, 0, 3] - (-1j * N / 2)) < 1e-9
    G = F.copy()
    G[0, 0, 3] = 0
    assert np.abs(G).max() < 1e-10


@pytest.mark.parametrize("shape,k", [((6, 10, 12), (1, 3, 2)), ((6, 10, 12), (0, 4, 5)),
                                     ((6, 10, 12), (6, 0, 0)), ((7, 9, 5), (2, 4, 3)),
                                     ((8, 4, 10), (5, 1, 7)), ((5, 5, 5), (0, 0, 0))])
def test_cosine_mode_deltas(shape, k):
    """cos(2 pi k . r / n) puts N/2 at +k and at -k (both kept only where
    kx is 0 or the Nyquist bin, since kx < H is stored)."""
    nz, ny, nx = shape
    kx, ky, kz = k
    f = inputs.cosine_mode(shape, kx, ky, kz)
    F = O.forward(f)
    N = nx * ny * nz
    expect = np.zeros_like(F)
    H = nx // 2 + 1
    for sx, sy, sz in ((kx, ky, kz), (-kx, -ky, -kz)):
        bx, by, bz = sx % nx, sy % ny, sz % nz
        if bx < H:
            expect[bz, by, bx] += N / 2
    assert np.abs(F - expect).max() < 1e-9


@pytest.mark.parametrize("nz,m", [(17, 0), (17, 1), (17, 5), (17, 16), (2, 0), (2, 1),
                                  (257, 0), (257, 37), (257, 256), (3, 1)])
def test_chebyshev_polynomial_deltas(nz, m):
    """T_m(z_j) on Gauss-Lobatto points: DCT-I gives M delta_nm for 0<m<M and
    2M delta_nm at the end points (per unit of Nx Ny)."""
    nx, ny = 4, 3
    M = nz - 1
    tz = np.cos(math.pi * np.mod(m * np.arange(nz), 2 * M) / M)
    # T_m(z_j) evaluated from z_j by the Chebyshev recurrence, independent of the table
    zj = inputs.gauss_lobatto(nz)
    t0, t1 = np.ones(nz), zj.copy()
    tm = t0 if m == 0 else t1
    for _ in range(2, m + 1):
        t0, t1 = t1, 2 * zj * t1 - t0
        tm = t1
    assert np.allclose(tm, tz, atol=1e-9)
    f = np.broadcast_to(tm[:, None, None], (nz, ny, nx)).copy()
    F = O.forward(f, (O.FFT, O.FFT, O.CHEB))
    expect = np.zeros_like(F)
    expect[m, 0, 0] = nx * ny * (2 * M if m in (0, M) else M)
    assert np.abs(F - expect).max() < 1e-9 * max(1, nx * ny * M)


def test_dct1_definition_small():
    x = rand_cplx((9,), 5)
    M = 8
    n = np.arange(9)
    ref = np.array([x[0] + (-1) ** q * x[M] + 2 * sum(x[j] * math.cos(math.pi * j * q / M)
                                                      for j in range(1, M)) for q in n])
    assert rel_l2(O.dct1(x), ref) < 1e-14


def test_dct1_self_inverse():
    for npts in (2, 3, 9, 33, 257):
        x = rand_cplx((npts,), npts)
        assert rel_l2(O.dct1(O.dct1(x)), 2 * (npts - 1) * x) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 63, 100])
def test_dst1_sine_mode_is_a_delta(n):
    """sin(pi m (j+1)/(n+1)) is the m-th discrete sine mode: its DST-I is
    (n+1) at k = m-1 and 0 elsewhere (orthogonality of the sine basis)."""
    j = np.arange(n)
    for m in sorted({1, (n + 1) // 2, n}):
        x = np.sin(math.pi * m * (j + 1) / (n + 1)).astype(complex)
        expect = np.zeros(n, complex)
        expect[m - 1] = n + 1
        assert np.abs(O.dst1(x) - expect).max() < 1e-12 * (n + 1)


def test_dst1_self_inverse():
    for npts in (1, 2, 5, 31, 255):
        x = rand_cplx((npts,), npts + 3)
        assert rel_l2(O.dst1(O.dst1(x)), 2 * (npts + 1) * x) < 1e-13


def test_dst1_odd_extension_identity():
    """The DST-I of x equals i times bins 1..n of the DFT of the odd
    extension [0, x, 0, -reversed(x)] of length 2(n+1)."""
    for n in (1, 6, 15, 40):
        x = rand_cplx((n,), n + 40)
        z = np.concatenate([[0], x, [0], -x[::-1]])
        assert rel_l2(O.dst1(x), 1j * brute_dft(z)[1:n + 1]) < 1e-13


def test_round_trip_sine():
    f = rand_real((11, 6, 8), 21)
    tt = (O.FFT, O.FFT, O.SINE)
    g = O.backward(O.forward(f, tt), 8, tt)
    assert rel_l2(g, O.scale(8, 6, 11, tt) * f) < 1e-13
    assert O.scale(8, 6, 11, tt) == 8 * 6 * 24


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(8, 6, 10), (5, 7, 9), (16, 16, 16)])
def test_parseval(shape):
    nz, ny, nx = shape
    f = rand_real(shape, 6)
    F = O.forward(f)
    w = np.full(nx // 2 + 1, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    lhs = np.sum(f ** 2)
    rhs = np.sum(w[None, None, :] * np.abs(F) ** 2) / (nx * ny * nz)
    assert abs(lhs - rhs) < 1e-12 * lhs


@pytest.mark.parametrize("shape", [(8, 6, 10), (5, 7, 9), (4, 4, 4)])
def test_hermitian_symmetry(shape):
    nz, ny, nx = shape
    F = O.forward(rand_real(shape, 7))
    planes = [0] + ([nx // 2] if nx % 2 == 0 else [])
    for px in planes:
        P = F[:, :, px]
        Q = np.conj(P[(-np.arange(nz)) % nz][:, (-np.arange(ny)) % ny])
        assert np.abs(P - Q).max() < 1e-12 * np.abs(F).max()
    assert abs(F[0, 0, 0].imag) < 1e-12


def test_linearity():
    shape = (6, 8, 10)
    f, g = rand_real(shape, 8), rand_real(shape, 9)
    a, b = 0.7, -2.5
    for tt in ((O.FFT, O.FFT, O.FFT), (O.FFT, O.FFT, O.CHEB), (O.FFT, O.EMPTY, O.CHEB), (O.FFT, O.FFT, O.SINE)):
        lhs = O.forward(a * f + b * g, tt)
        rhs = a * O.forward(f, tt) + b * O.forward(g, tt)
        assert rel_l2(lhs, rhs) < 1e-14


@pytest.mark.parametrize("tt", [(0, 0, 0), (0, 0, 1), (0, 2, 0), (0, 2, 2), (0, 0, 2), (0, 2, 1)])
@pytest.mark.parametrize("shape", [(8, 6, 10), (9, 5, 7), (2, 1, 1)])
def test_round_trip(tt, shape):
    nz, ny, nx = shape
    f = rand_real(shape, 10)
    back = O.backward(O.forward(f, tt), nx, tt)
    assert rel_l2(back, O.scale(nx, ny, nz, tt) * f) < 1e-14


def test_c2r_ignores_imaginary_dc_and_nyquist():
    """Reading C13: per X line the inverse takes Re of the DC and Nyquist terms."""
    nx = 10
    F = rand_cplx((1, 1, 6), 11)
    base = O.backward(F, nx)
    G = F.copy()
    G[0, 0, 0] += 5j
    G[0, 0, 5] -= 3j
    assert np.abs(O.backward(G, nx) - base).max() < 1e-12


def test_zyx_is_a_permutation():
    F = rand_cplx((3, 4, 5), 12)
    G = O.to_zyx(F)
    assert G.shape == (5, 4, 3)
    assert G[2, 1, 0] == F[0, 1, 2]
    assert np.array_equal(O.from_zyx(G), F)


def test_stage_entry_points_compose_to_forward():
    nz, ny, nx = 5, 6, 8
    H = nx // 2 + 1
    f = rand_real((nz, ny, nx), 13)
    F = np.zeros((nz, ny, H), complex)
    O.x_r2c_rows(nx, f.ravel(), F.reshape(-1), 0, ny * nz)
    O.c2c_lines(ny, H, ny * H, 1, H, F.reshape(-1), 0, H * nz, -1)
    O.c2c_lines(nz, H * ny, 0, 1, ny * H, F.reshape(-1), 0, H * ny, -1)
    assert rel_l2(F, O.forward(f)) < 1e-15


# --------------------------------------------------------------------------
# Optional cross-checks with library routines (never a dependency)
# --------------------------------------------------------------------------

def test_matches_numpy_rfftn():
    f = rand_real((12, 10, 14), 14)
    assert rel_l2(O.forward(f), np.fft.rfftn(f)) < 1e-14


def test_dct1_matches_scipy():
    sfft = pytest.importorskip("scipy.fft")
    x = rand_real((33,), 15)
    assert rel_l2(O.dct1(x).real, sfft.dct(x, type=1)) < 1e-14


def test_dst1_matches_scipy():
    sfft = pytest.importorskip("scipy.fft")
    for n in (1, 2, 17, 64):
        x = rand_real((n,), 15 + n)
        assert rel_l2(O.dst1(x).real, sfft.dst(x, type=1)) < 1e-14


# --------------------------------------------------------------------------
# The pins have teeth: plausible mistakes planted in copies of the oracle fail
# --------------------------------------------------------------------------

MUTANTS = {
    # wrong sign on the roots of unity
    "sign": ("r[t] = (double)cosl(a) + (double)sign * (double)sinl(a) * I;",
             "r[t] = (double)cosl(a) - (double)sign * (double)sinl(a) * I;"),
    # Nyquist weight of the c2r sum set to 2 like the interior bins
    "nyq_weight": ("if (nx % 2 == 0 && q == nx / 2) w = 1.0;", "if (0) w = 1.0;"),
    # DST-I sample index off by one (sin(pi j (k+1)/(n+1)) instead of (j+1))
    "dst_index": ("acc += 2.0 * k->sinv[((j + 1) * (q + 1)) % P] * line[j];",
                  "acc += 2.0 * k->sinv[(j * (q + 1)) % P] * line[j];"),
    # DCT-I end point dropped
    "dct_end": ("cplx acc = line[0] + ((q % 2) ? -line[M] : line[M]);", "cplx acc = line[0];"),
    # recombination index off: transposed operand
    "transpose": ("acc += roots[t * step] * tmp[r * m + k];", "acc += roots[t * step] * tmp[k * p + r < n ? k * p + r : r * m + k];"),
}


def _build_mutant(tmp_path, name):
    src = open(os.path.join(os.path.dirname(O.__file__), "p3_oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src, name
    path = tmp_path / ("mut_%s.c" % name)
    path.write_text(src.replace(old, new))
    so = tmp_path / ("libmut_%s.so" % name)
    subprocess.run(["gcc", "-std=c11", "-O1", "-fPIC", "-shared", "-pthread", "-o",
                    str(so), str(path), "-lm"], check=True)
    return ctypes.CDLL(str(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    L, I, P = ctypes.c_long, ctypes.c_int, ctypes.c_void_p
    lib.p3o_forward.argtypes = [L, L, L, I, I, P, P, I]
    lib.p3o_backward.argtypes = [L, L, L, I, I, P, P, I]
    failures = 0
    for shape, tz in (((8, 6, 10), O.FFT), ((9, 5, 6), O.CHEB), ((7, 5, 6), O.SINE)):
        nz, ny, nx = shape
        f = rand_real(shape, 16)
        F = np.zeros((nz, ny, nx // 2 + 1), complex)
        lib.p3o_forward(nx, ny, nz, O.FFT, tz, f.ctypes.data, F.ctypes.data, 1)
        if rel_l2(F, brute_forward_3d(f, {O.FFT: "fft", O.CHEB: "cheb", O.SINE: "sine"}[tz])) > 1e-12:
            failures += 1
        G = rand_cplx(F.shape, 17)
        g = np.zeros(shape)
        lib.p3o_backward(nx, ny, nz, O.FFT, O.FFT, G.ctypes.data, g.ctypes.data, 1)
        if rel_l2(g, brute_backward_3d(G, nx)) > 1e-12:
            failures += 1
    assert failures > 0, "mutant %s passed every pin" % name


def test_sampled_lines_match_brute_force():
    """PhaseSum + forward_lines / backward_rows (used for full-size parity)
    against the brute-force 3D sums, with chunked accumulation over z."""
    nz, ny, nx = 7, 6, 10
    f = rand_real((nz, ny, nx), 21)
    ref = brute_forward_3d(f)
    pairs = [(0, 0), (5, 6), (2, 3)]
    ps = O.PhaseSum(nx, ny, nz, [p[0] for p in pairs], [p[1] for p in pairs], -1)
    for z0 in range(0, nz, 3):
        ps.add(f[z0:z0 + 3], z0)
    lines = O.forward_lines(ps.g, nx)
    for i, (ky, kz) in enumerate(pairs):
        assert rel_l2(lines[i], ref[kz, ky, :]) < 1e-13
    F = rand_cplx((nz, ny, nx // 2 + 1), 22)
    refb = brute_backward_3d(F, nx)
    pts = [(0, 0), (4, 6), (5, 1)]
    ps = O.PhaseSum(nx // 2 + 1, ny, nz, [p[0] for p in pts], [p[1] for p in pts], +1)
    ps.add(F, 0)
    rows = O.backward_rows(ps.g, nx)
    for i, (y, z) in enumerate(pts):
        assert rel_l2(rows[i], refb[z, y, :]) < 1e-13


@pytest.mark.parametrize("shape", [(7, 6, 10), (5, 9, 15), (8, 1, 6), (1, 4, 4)])
def test_sampled_planes_match_brute_force(shape):
    """forward_kx_planes / backward_z_planes (the whole sampled planes of the
    full-size checks) against the brute-force 3D sums, the chunks fed in
    uneven pieces; the inverse on a non-Hermitian input."""
    nz, ny, nx = shape
    H = nx // 2 + 1
    f = rand_real(shape, 31)
    ref = brute_forward_3d(f)  # [kz][ky][kx]
    kxs = sorted({0, H - 1, H // 2})
    chunks = [(z0, f[z0:z0 + 2]) for z0 in range(0, nz, 2)]
    planes = O.forward_kx_planes(chunks, nx, ny, nz, kxs)  # [k][ky][kz]
    for i, kx in enumerate(kxs):
        assert rel_l2(planes[i], ref[:, :, kx].T) < 1e-13
    F = rand_cplx((nz, ny, H), 32)
    refb = brute_backward_3d(F, nx)
    zs = sorted({0, nz - 1, nz // 2})
    Z = O.to_zyx(F)
    chunks = [(k0, Z[k0:k0 + 3]) for k0 in range(0, H, 3)]
    rows = O.backward_z_planes(chunks, nx, ny, nz, zs)
    for j, z in enumerate(zs):
        assert rel_l2(rows[j], refb[z]) < 1e-13


def test_inverse_z_table_closed_form():
    T = O.inverse_z_table(4, [0, 1, 3])
    assert np.allclose(T[:, 0], 1.0, atol=0, rtol=0)
    assert np.allclose(T[:, 1], [1, 1j, -1, -1j], atol=1e-16)
    assert np.allclose(T[:, 2], [1, -1j, -1, 1j], atol=1e-16)


def test_sampled_plane_checks_catch_a_wrong_sign(monkeypatch):
    """A planted mistake (the inverse Z table with the forward sign) must make
    the sampled inverse planes disagree with the brute-force sums."""
    nz, ny, nx = 6, 5, 8
    H = nx // 2 + 1
    F = rand_cplx((nz, ny, H), 33)
    refb = brute_backward_3d(F, nx)
    good = O.inverse_z_table
    monkeypatch.setattr(O.oracle, "inverse_z_table", lambda n, zs, sign=+1: good(n, zs, -sign))
    rows = O.backward_z_planes([(0, O.to_zyx(F))], nx, ny, nz, [1, 2])
    assert rel_l2(rows[0], refb[1]) > 1e-3 and rel_l2(rows[1], refb[2]) > 1e-3
