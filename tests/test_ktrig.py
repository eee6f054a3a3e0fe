"""Host logic: the compile-time cos / sin of 2 pi m / n behind the composite
register butterflies' internal twiddles (p3::ktrig2pi in p3_dft.cuh: octant
reduction, then Taylor series of sin and cos on [0, pi/4]), checked on a host
build against the C library's long-double cosl / sinl for every m < n <= 4096,
and the exact quarter-turn values.  No GPU needed (nvcc compiles the header
for the host)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_02803_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include "p3_dft.cuh"
int main()
{
    const long double two_pi = 6.283185307179586476925286766559005768L;
    double worst = 0.0;
    int wm = 0, wn = 0, exact_bad = 0;
    for (int n = 1; n <= 4096; ++n)
        for (int m = 0; m < n; ++m) {
            const p3::KTrigVal v = p3::ktrig2pi(m, n);
            const long double a = two_pi * (long double)m / (long double)n;
            const double e = fmax(fabs((double)((long double)v.c - cosl(a))), fabs((double)((long double)v.s - sinl(a))));
            if (e > worst) { worst = e; wm = m; wn = n; }
            // quarter turns are exact
            if (4 * m % n == 0) {
                const int q = 4 * m / n;
                const double c = q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0, s = q == 1 ? 1.0 : q == 3 ? -1.0 : 0.0;
                if (fabs(v.c - c) > 1e-300 || fabs(v.s - s) > 1e-300) ++exact_bad;
            }
        }
    // the table a butterfly of 24 points uses, evaluated at compile time
    constexpr p3::KTrigTab<24> t = p3::ktrig_tab<24>();
    static_assert(t.c[0] == 1.0 && t.s[0] == 0.0, "first entry");
    printf("%.3e %d %d %d %.17g %.17g\n", worst, wm, wn, exact_bad, t.c[1], t.s[1]);
    return 0;
}
"""


@pytest.fixture(scope="module")
def result(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("ktrig")
    src = d / "ktrig.cu"
    src.write_text(HARNESS)
    exe = d / "ktrig"
    r = subprocess.run([nvcc, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    if r.returncode != 0:
        pytest.fail("harness build failed:\n" + r.stderr)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return out


def test_within_double_rounding_of_long_double(result):
    worst = float(result[0])
    # a few units in the last place of values of magnitude <= 1
    assert worst < 1e-15, result


def test_quarter_turns_exact(result):
    assert int(result[3]) == 0, result


def test_table_values(result):
    import math
    # within a few units in the last place of the library's double values
    assert abs(float(result[4]) - math.cos(2 * math.pi / 24)) < 5e-16
    assert abs(float(result[5]) - math.sin(2 * math.pi / 24)) < 5e-16
