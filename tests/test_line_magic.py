"""Host logic: the multiply-high division behind every stage kernel's line
addressing (p3::line_magic, and the per-pass t / Ns constants built the same
way), checked exactly against integer division on a host build of the
internal header, no GPU needed.

The construction (Granlund and Montgomery, "Division by invariant integers
using multiplication", 1994, Sect. 4, with 31-bit numerators) claims
floor(L / d) = (L * m) >> s for 0 <= L < 2^31 with l = ceil(log2 d),
m = floor(2^(31+l) / d) + 1 and s = 31 + l; the test checks it on the
divisors and numerators where an off-by-one would show: powers of two and
their neighbours, the largest 31-bit values, and seeded random ones."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_02803_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include "p3_internal.h"
int main(int argc, char** argv)
{
    // stdin: lines "d nlines L"; prints one line per case: the quotient the
    // kernels compute (or -1 when line_magic leaves pm = 0) and L / d
    long long d, nl, L;
    while (scanf("%lld %lld %lld", &d, &nl, &L) == 3) {
        p3::LineMap m = p3::LineMap{d, 0, 1, 0};
        p3::line_magic(m, nl);
        long long q = -1;
        if (m.pm) q = (long long)(unsigned)(((unsigned long long)(unsigned)L * m.pm) >> m.ps);
        printf("%lld %lld\n", q, L / d);
    }
    return 0;
}
"""


def cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda.h")):
            return os.path.join(cand, "include")
    return None


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("magic")
    src = d / "magic.cpp"
    src.write_text(HARNESS)
    exe = d / "magic"
    r = subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("harness build failed:\n" + r.stderr)
    return str(exe)


def cases():
    rnd = random.Random(20261203)
    top = (1 << 31) - 1
    divs = set(range(1, 300))
    for k in range(1, 31):
        divs.update({(1 << k) - 1, 1 << k, (1 << k) + 1})
    divs.update({top, top - 1, 3 * (1 << 29), 1025 * 2048, 513 * 1024, 193 * 384})
    divs.update(rnd.randrange(1, top) for _ in range(300))
    out = []
    for d in sorted(divs):
        nums = {0, 1, d - 1, d, d + 1, 2 * d - 1, top, top - 1, top - d}
        nums.update(rnd.randrange(0, top + 1) for _ in range(8))
        for L in nums:
            if 0 <= L <= top:
                out.append((d, top + 1, L))
    return out


def test_multiply_high_division_is_exact(harness):
    cs = cases()
    inp = "".join("%d %d %d\n" % c for c in cs)
    r = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True)
    lines = r.stdout.split("\n")
    bad = []
    for (d, nl, L), line in zip(cs, lines):
        q, ref = (int(v) for v in line.split())
        if q != ref:
            bad.append((d, L, q, ref))
    assert len(lines) >= len(cs)
    assert not bad, bad[:10]


def test_falls_back_past_31_bits(harness):
    # per or nlines beyond 31 bits: pm = 0, the kernels divide plainly
    inp = "%d %d %d\n%d %d %d\n" % ((1 << 31), 10, 5, 7, (1 << 31) + 1, 5)
    r = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True)
    q = [int(line.split()[0]) for line in r.stdout.strip().split("\n")]
    assert q == [-1, -1]
