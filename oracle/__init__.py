"""FP64 CPU oracle for the P3DFFT 3D r2c / c2r transforms (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    FFT, CHEB, EMPTY, SINE, forward, backward, fft1d, dct1, dst1, to_zyx, from_zyx,
    x_r2c_rows, x_c2r_rows, c2c_lines, dct1_lines, dst1_lines, scale, half, nthreads_default,
    PhaseSum, forward_lines, backward_rows, forward_kx_planes, backward_z_planes, inverse_z_table,
)
