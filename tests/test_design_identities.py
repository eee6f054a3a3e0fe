"""CPU pins of the identities the generic kernel's newer paths rest on, checked
in FP64 against the oracle's own row transforms (no GPU):

* odd X rows two per complex FFT: with z = f1 + i f2 and Z = DFT(z),
  F1[k] = (Z[k] + conj Z[N-k]) / 2 and F2[k] = -i (Z[k] - conj Z[N-k]) / 2;
  inverse: Z[k] = X1[k] + i X2[k], Z[N-k] = conj X1[k] + i conj X2[k]
  (1 <= k < H, N odd), Im X1[0] and Im X2[0] dropped; then Re and Im of the
  inverse DFT are the weighted-real C2R (Sect. 3.2) of X1 and X2, for any
  complex X1, X2 (Hermitian or not);
* the composite register butterflies: a DFT of R = R1 R2 points as R2 DFTs
  of size R1 over inputs n2, n2 + R2, ..., the twiddles exp(-2 pi i n2 k1 / R),
  and R1 DFTs of size R2, output k = k1 + R1 k2.
The same formulas written in the kernels are covered on the GPU by the parity
tests; these pin the algebra itself."""
import numpy as np

import oracle


def rows_r2c(f):
    """The oracle's X-stage R2C of each row of f (rows x nx)."""
    rows, nx = f.shape
    H = nx // 2 + 1
    F = np.zeros(rows * H, dtype=np.complex128)
    oracle.x_r2c_rows(nx, np.ascontiguousarray(f, dtype=np.float64).ravel(), F, 0, rows)
    return F.reshape(rows, H)


def rows_c2r(F, nx):
    rows = F.shape[0]
    f = np.zeros(rows * nx, dtype=np.float64)
    oracle.x_c2r_rows(nx, np.ascontiguousarray(F, dtype=np.complex128).ravel(), f, 0, rows)
    return f.reshape(rows, nx)


def test_two_real_rows_per_complex_fft_forward():
    rng = np.random.default_rng(11)
    for N in (1, 3, 5, 7, 15, 49, 75, 125, 375):
        f = rng.uniform(-1, 1, size=(2, N))
        H = N // 2 + 1
        Z = oracle.fft1d(f[0] + 1j * f[1], -1)
        k = np.arange(H)
        Zm = Z[(N - k) % N]
        F1 = (Z[k] + np.conj(Zm)) / 2
        F2 = -1j * (Z[k] - np.conj(Zm)) / 2
        ref = rows_r2c(f)
        assert np.abs(F1 - ref[0]).max() <= 1e-13 * max(1.0, np.abs(ref[0]).max()), N
        assert np.abs(F2 - ref[1]).max() <= 1e-13 * max(1.0, np.abs(ref[1]).max()), N


def test_two_half_spectra_per_complex_fft_inverse_any_input():
    rng = np.random.default_rng(12)
    for N in (1, 3, 5, 9, 21, 63, 105, 243):
        H = N // 2 + 1
        # arbitrary complex half spectra (not the spectrum of any real row)
        X = rng.uniform(-1, 1, size=(2, H)) + 1j * rng.uniform(-1, 1, size=(2, H))
        Z = np.zeros(N, dtype=np.complex128)
        Z[0] = X[0, 0].real + 1j * X[1, 0].real
        for k in range(1, H):
            Z[k] = X[0, k] + 1j * X[1, k]
            Z[N - k] = np.conj(X[0, k]) + 1j * np.conj(X[1, k])
        z = oracle.fft1d(Z, +1)
        ref = rows_c2r(X, N)
        assert np.abs(z.real - ref[0]).max() <= 1e-12 * max(1.0, np.abs(ref[0]).max()), N
        assert np.abs(z.imag - ref[1]).max() <= 1e-12 * max(1.0, np.abs(ref[1]).max()), N


def test_composite_butterfly_index_map():
    rng = np.random.default_rng(13)
    for R1, R2 in ((2, 3), (3, 3), (2, 5), (4, 3), (2, 7), (3, 5), (2, 9), (4, 5), (3, 7), (8, 3), (5, 5), (3, 9),
                   (4, 7)):
        R = R1 * R2
        x = rng.uniform(-1, 1, R) + 1j * rng.uniform(-1, 1, R)
        y = np.zeros((R2, R1), dtype=np.complex128)
        for n2 in range(R2):
            a = oracle.fft1d(x[n2::R2], -1)  # inputs n2, n2 + R2, ... (n = R2 n1 + n2)
            y[n2] = a * np.exp(-2j * np.pi * n2 * np.arange(R1) / R)
        out = np.zeros(R, dtype=np.complex128)
        for k1 in range(R1):
            b = oracle.fft1d(y[:, k1], -1)
            out[k1 + R1 * np.arange(R2)] = b
        ref = oracle.fft1d(x, -1)
        assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max(), (R1, R2)
