"""The GPU inner products' 192-bit merge and final rounding (csrc/xacc.cuh),
compiled for the host, against exact rational arithmetic: every merged
partial equals the floor-aligned sum of its operands, and the final rounding
is the correctly rounded (nearest, ties to even) double of the exact value,
subnormals and overflow included."""
import ctypes
import math
import os
import random
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def xh(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("xh") / "libxh.so")
    subprocess.check_call([cxx, "-O1", "-shared", "-fPIC", "-std=c++17",
                           "-I" + os.path.join(ROOT, "paper_2108_10591_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "xacc_host_check.cpp"), "-o", out])
    L = ctypes.CDLL(out)
    U = ctypes.c_ulonglong
    L.xh_round.argtypes = [ctypes.c_int, U, U, U]
    L.xh_round.restype = ctypes.c_double
    L.xh_merge.argtypes = [ctypes.c_int, ctypes.POINTER(U), ctypes.c_int, ctypes.POINTER(U),
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(U)]
    return L


def words(v):
    v &= (1 << 192) - 1
    return (v >> 128) & M64, (v >> 64) & M64, v & M64


def signed(w2, w1, w0):
    v = (w2 << 128) | (w1 << 64) | w0
    return v - (1 << 192) if v >> 191 else v


def exact_double(v, e):
    """Correctly rounded double of v * 2^e (Python's int/int division rounds correctly)."""
    if v == 0:
        return 0.0
    q = Fraction(v) * Fraction(2) ** e
    try:
        return q.numerator / q.denominator
    except OverflowError:
        return math.copysign(math.inf, v)


def rnd(xh, v, e):
    return xh.xh_round(e, *words(v))


def test_round_random(xh):
    rng = random.Random(1)
    for _ in range(20000):
        bits = rng.randint(1, 187)
        v = rng.getrandbits(bits) * rng.choice((1, -1))
        e = rng.randint(-1300, 900)
        got, want = rnd(xh, v, e), exact_double(v, e)
        assert got == want or (math.isnan(got) and math.isnan(want)), (v, e, got, want)
        assert math.copysign(1.0, got) == math.copysign(1.0, want) or v == 0


def test_round_ties_to_even(xh):
    rng = random.Random(2)
    for _ in range(2000):
        m = rng.getrandbits(52) | (1 << 52)          # 53-bit significand
        for tail, extra in ((1, 1), (1, 7)):         # exactly half an ulp, then just above half
            v = ((m << extra) | (tail << (extra - 1))) * rng.choice((1, -1))
            e = rng.randint(-1000, 900)
            assert rnd(xh, v, e) == exact_double(v, e)
    # ties at the subnormal boundary
    for k in range(1, 60):
        v = (1 << k) + (1 << (k - 1))
        e = -1074 - k
        assert rnd(xh, v, e) == exact_double(v, e)


def test_round_special(xh):
    assert xh.xh_round(xh.xh_empty(), 0, 0, 0) == 0.0
    assert math.isnan(xh.xh_round(xh.xh_nan(), 0, 0, 0))
    assert rnd(xh, 1, -1074) == 5e-324 and rnd(xh, 1, -1076) == 0.0
    assert rnd(xh, 3, -1076) == 5e-324                      # 0.75 of the smallest subnormal
    assert rnd(xh, (1 << 53) - 1, 971) == float.fromhex("0x1.fffffffffffffp+1023")
    assert rnd(xh, 1, 1024) == math.inf and rnd(xh, -1, 1024) == -math.inf


def test_merge_is_floor_aligned_sum(xh):
    rng = random.Random(3)
    U3 = ctypes.c_ulonglong * 3
    for _ in range(20000):
        va = rng.getrandbits(rng.randint(1, 186)) * rng.choice((1, -1))
        vb = rng.getrandbits(rng.randint(1, 186)) * rng.choice((1, -1))
        ea = rng.randint(-400, 400)
        eb = ea + rng.randint(-200, 200)
        out_e = ctypes.c_int()
        out_w = U3()
        xh.xh_merge(ea, U3(*words(va)), eb, U3(*words(vb)), ctypes.byref(out_e), out_w)
        E = max(ea, eb)
        s = (va >> (E - ea)) + (vb >> (E - eb))   # arithmetic shifts: floor alignment
        if (s >> 188) not in (0, -1):              # renormalised by 8 bits
            s >>= 8
            E += 8
        assert out_e.value == E and signed(*out_w) == s, (va, ea, vb, eb)
        # aligned operands lose nothing: the merge is then the exact sum
        if (va % (1 << (E - ea)) == 0 or ea == E) and (vb % (1 << (E - eb)) == 0 or eb == E):
            assert Fraction(signed(*out_w)) * Fraction(2) ** out_e.value == \
                Fraction(va) * Fraction(2) ** ea + Fraction(vb) * Fraction(2) ** eb


def test_merge_empty_and_nan(xh):
    U3 = ctypes.c_ulonglong * 3
    out_e, out_w = ctypes.c_int(), U3()
    xh.xh_merge(xh.xh_empty(), U3(0, 0, 0), 5, U3(*words(-7)), ctypes.byref(out_e), out_w)
    assert out_e.value == 5 and signed(*out_w) == -7
    xh.xh_merge(5, U3(*words(-7)), xh.xh_empty(), U3(0, 0, 0), ctypes.byref(out_e), out_w)
    assert out_e.value == 5 and signed(*out_w) == -7
    xh.xh_merge(xh.xh_nan(), U3(0, 0, 0), 5, U3(*words(3)), ctypes.byref(out_e), out_w)
    assert out_e.value == xh.xh_nan()
