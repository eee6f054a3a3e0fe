"""Host logic of the generic kernel's line plans (no GPU): p3_plan_factor.

FP32 lines whose length has a factor 3, 5 or 7 take the fewest passes over
the native radices and the composite register butterflies up to 15, ties
going to the most even radices; FP64 lines and powers of two keep the native
sequence.  Checked against an independent brute-force search over multisets
of radices."""
import functools

import pytest

from paper_1905_02803_gb300 import p3dfft as P

NATIVE = {2, 3, 4, 5, 7, 8, 16}
COMPOSITE = {6, 9, 10, 12, 14, 15}


def smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


@functools.lru_cache(maxsize=None)
def fewest(n, allowed):
    """(passes, largest smallest radix) over all radix multisets with product n."""
    if n == 1:
        return 0, 1 << 30
    best = None
    for r in allowed:
        if n % r:
            continue
        p, m = fewest(n // r, allowed)
        cand = (p + 1, min(m, r))
        if best is None or cand[0] < best[0] or (cand[0] == best[0] and cand[1] > best[1]):
            best = cand
    return best


@pytest.fixture(scope="module")
def lib():
    try:
        P.load()
    except OSError as e:  # pragma: no cover - the build step makes it
        pytest.skip("library not built: %s" % e)
    return P


def test_fp32_fewest_passes_for_every_smooth_length(lib):
    allowed = tuple(sorted(NATIVE | COMPOSITE))
    for n in range(2, 4097):
        if not smooth(n):
            assert lib.p3_plan_factor(n, "f32") is None, n
            continue
        rad = lib.p3_plan_factor(n, "f32")
        prod = 1
        for r in rad:
            prod *= r
        assert prod == n, (n, rad)
        assert rad == sorted(rad, reverse=True), (n, rad)
        if n & (n - 1) == 0:
            # powers of two: the native sequence, 16s first
            assert rad == lib.p3_plan_factor(n, "f64"), (n, rad)
            continue
        assert set(rad) <= NATIVE | COMPOSITE, (n, rad)
        passes, minr = fewest(n, allowed)
        assert len(rad) == passes and min(rad) == minr, (n, rad, passes, minr)


def test_fp64_native_radices(lib):
    for n in range(2, 4097):
        rad = lib.p3_plan_factor(n, "f64")
        if not smooth(n):
            assert rad is None, n
            continue
        prod = 1
        for r in rad:
            prod *= r
        assert prod == n and set(rad) <= NATIVE, (n, rad)
        # at most one of 8 / 4 / 2 after the 16s, the odd primes last
        two = [r for r in rad if r in (2, 4, 8)]
        assert len(two) <= 1, (n, rad)
        odd = [r for r in rad if r in (3, 5, 7)]
        assert rad[len(rad) - len(odd):] == odd and odd == sorted(odd), (n, rad)


def test_examples(lib):
    assert lib.p3_plan_factor(384, "f32") == [8, 8, 6]
    assert lib.p3_plan_factor(384, "f64") == [16, 8, 3]
    assert lib.p3_plan_factor(375, "f32") == [15, 5, 5]
    assert lib.p3_plan_factor(324, "f32") == [9, 6, 6]
    assert lib.p3_plan_factor(1024, "f32") == [16, 16, 4]
    assert lib.p3_plan_factor(97, "f32") is None  # Bluestein


def test_invalid_arguments(lib):
    import ctypes
    buf = (ctypes.c_int * 4)()
    cnt = ctypes.c_int()
    L = lib.load()
    assert L.p3_plan_factor(1, lib.P3_F32, buf, 4, ctypes.byref(cnt)) == lib.P3_ERR_INVALID
    assert L.p3_plan_factor(12, 7, buf, 4, ctypes.byref(cnt)) == lib.P3_ERR_INVALID
    assert L.p3_plan_factor(12, lib.P3_F32, None, 4, ctypes.byref(cnt)) == lib.P3_ERR_INVALID
    assert L.p3_plan_factor(4096, lib.P3_F64, buf, 2, ctypes.byref(cnt)) == lib.P3_ERR_UNSUPPORTED  # 3 passes > cap
