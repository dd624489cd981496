"""CPU checks of the integer fixed-point arithmetic that the EO_DD kernels run
(paper_1806_01036_gb300/csrc/fx.cuh, compiled here for the host through a
small shim) against exact rational arithmetic."""
import ctypes as C
import os
import shutil
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHIM = os.path.join(ROOT, "tests", "fxshim", "fx_shim.cu")
CSRC = os.path.join(ROOT, "paper_1806_01036_gb300", "csrc")


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("fx") / "libfxshim.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), SHIM, "-o", out], check=True, capture_output=True)
    L = C.CDLL(out)
    d, i, p, ll = C.c_double, C.c_int, C.c_void_p, C.c_longlong
    L.fxs_align_exp.argtypes = [d]
    L.fxs_align_exp.restype = i
    L.fxs_to_limbs.argtypes = [d, i, p]
    L.fxs_to_limbs_dd.argtypes = [d, d, i, p]
    L.fxs_dot.argtypes = [i, p, p, i, i, p, p]
    L.fxs_dot_rescaled.argtypes = [i, i, p, p, i, i, i, p, p]
    L.fxs_w_to_dd.argtypes = [ll, ll, i, p, p]
    L.fxs_w_to_double.argtypes = [ll, ll, i]
    L.fxs_w_to_double.restype = d
    L.fxs_sub_round.argtypes = [d, ll, ll, i]
    L.fxs_sub_round.restype = d
    L.fxs_w_to_double_fast.argtypes = [ll, ll, i, p]
    L.fxs_w_to_double_fast.restype = d
    L.fxs_sub_round_fast.argtypes = [d, ll, ll, i, p]
    L.fxs_sub_round_fast.restype = d
    L.fxs_acc256.argtypes = [i, p, p, p, p, p]
    L.fxs_scale_offset.restype = i
    return L


def limbs(fx, x, A):
    out = (C.c_int * 4)()
    fx.fxs_to_limbs(x, A, out)
    return list(out)


def value_of(L, A):
    X = sum(F(L[a]) * 2 ** (26 * (3 - a)) for a in range(4))
    return X * F(2) ** (A - 1126)


def split_w(w):
    w &= (1 << 128) - 1
    lo, hi = w & ((1 << 64) - 1), w >> 64
    to_s = lambda v: v - (1 << 64) if v >= 1 << 63 else v
    return to_s(lo), to_s(hi)


def rn(q):
    """Nearest double to the rational q (Python's float() rounds correctly)."""
    return float(q)


def test_alignment_exponent(fx):
    assert fx.fxs_align_exp(0.0) == 0
    assert fx.fxs_align_exp(1.0) == 1023
    assert fx.fxs_align_exp(-3.0) == 1024
    assert fx.fxs_align_exp(5e-324) == 1
    assert fx.fxs_align_exp(float("inf")) == 2047


def test_limbs_represent_values_exactly_within_51_binades(fx):
    g = np.random.default_rng(1)
    for _ in range(500):
        x = float(np.ldexp(g.standard_normal(), int(g.integers(-200, 200))))
        A = fx.fxs_align_exp(x) + int(g.integers(0, 52))
        L = limbs(fx, x, A)
        assert all(abs(v) < 2 ** 26 for v in L)
        assert value_of(L, A) == F(x)


def test_limbs_truncate_toward_zero_below_the_grid(fx):
    g = np.random.default_rng(2)
    for _ in range(500):
        x = float(np.ldexp(g.standard_normal(), int(g.integers(-200, 200))))
        A = fx.fxs_align_exp(x) + int(g.integers(52, 140))
        v = value_of(limbs(fx, x, A), A)
        unit = F(2) ** (A - 1126)
        assert abs(v) <= abs(F(x)) and abs(F(x) - v) < unit
        assert v == 0 or (v > 0) == (x > 0)


def test_limbs_of_double_double(fx):
    g = np.random.default_rng(3)
    for _ in range(300):
        h = float(g.standard_normal())
        l = float(np.ldexp(g.standard_normal(), -60))
        h, l = h + l, (F(h) + F(l)) - F(h + l)  # a normalized pair
        l = float(l)
        A = fx.fxs_align_exp(h) + 1
        out = (C.c_int * 4)()
        fx.fxs_to_limbs_dd(h, l, A, out)
        v = value_of(list(out), A)
        exact = F(h) + F(l)
        assert abs(v - exact) <= 2 * F(2) ** (A - 1126)


@pytest.mark.parametrize("n", [1, 7, 100, 384])
def test_dot_matches_exact_sum(fx, n):
    g = np.random.default_rng(10 + n)
    x = g.standard_normal(n)
    y = np.ldexp(g.standard_normal(n), -7)
    Ax = max(fx.fxs_align_exp(float(v)) for v in x)
    Ay = max(fx.fxs_align_exp(float(v)) for v in y)
    hi, lo = C.c_double(), C.c_double()
    fx.fxs_dot(n, x.ctypes.data, y.ctypes.data, Ax, Ay, C.byref(hi), C.byref(lo))
    exact = sum((F(float(a)) * F(float(b)) for a, b in zip(x, y)), F(0))
    bound = n * 8 * F(2) ** -104 * F(float(np.max(np.abs(x)))) * F(float(np.max(np.abs(y)))) * 4
    assert abs(F(hi.value) + F(lo.value) - exact) <= bound + F(2) ** -104 * abs(exact)
    assert hi.value == rn(exact) or abs(F(hi.value) - exact) <= F(2) ** -52 * abs(exact)


@pytest.mark.parametrize("grow", [1, 3, 30])
def test_dot_with_growing_alignment(fx, grow):
    # as in the Gram kernel: later rows raise a column's alignment exponent and the
    # accumulator is divided by 2^grow; the result keeps the full accuracy
    g = np.random.default_rng(40 + grow)
    n, n0 = 300, 120
    x = g.standard_normal(n)
    y = g.standard_normal(n)
    y[n0:] *= 2.0 ** grow
    Ax = max(fx.fxs_align_exp(float(v)) for v in x)
    Ay0 = max(fx.fxs_align_exp(float(v)) for v in y[:n0])
    Ay1 = max(fx.fxs_align_exp(float(v)) for v in y)
    hi, lo = C.c_double(), C.c_double()
    fx.fxs_dot_rescaled(n, n0, x.ctypes.data, y.ctypes.data, Ax, Ay0, Ay1, C.byref(hi), C.byref(lo))
    exact = sum((F(float(a)) * F(float(b)) for a, b in zip(x, y)), F(0))
    bound = n * 32 * F(2) ** -104 * F(float(np.max(np.abs(x)))) * F(float(np.max(np.abs(y))))
    assert abs(F(hi.value) + F(lo.value) - exact) <= bound


def test_w_to_dd_rounds_to_nearest(fx):
    g = np.random.default_rng(4)
    for _ in range(2000):
        bits = int(g.integers(1, 127))
        w = int(g.integers(0, 2 ** 62)) << max(0, bits - 62)
        w |= int(g.integers(0, 2 ** 62))
        w %= 1 << bits
        if g.random() < 0.5:
            w = -w
        S = int(g.integers(-1200, 800))
        lo_, hi_ = split_w(w)
        h, l = C.c_double(), C.c_double()
        fx.fxs_w_to_dd(lo_, hi_, S, C.byref(h), C.byref(l))
        exact = F(w) * F(2) ** S
        if exact == 0:
            assert h.value == 0 and l.value == 0
            continue
        assert h.value == rn(exact)
        assert l.value == rn(exact - F(h.value))


def test_w_to_double_ties_to_even(fx):
    # 2^53 + 1 and 2^53 + 3 sit exactly halfway between doubles
    for w, want in (((1 << 53) + 1, float(1 << 53)), ((1 << 53) + 3, float((1 << 53) + 4)),
                    (-((1 << 54) + 2), -float(1 << 54)), ((1 << 100) + (1 << 47), float(1 << 100))):
        lo_, hi_ = split_w(w)
        assert fx.fxs_w_to_double(lo_, hi_, 0) == want


def test_w_to_double_rounds_to_nearest(fx):
    """Random 128-bit integers (and halfway cases) against exact rational
    rounding, across the normal range and its edges (subnormal, overflow)."""
    g = np.random.default_rng(7)
    cases = []
    for _ in range(4000):
        bits = int(g.integers(1, 127))
        w = (int(g.integers(0, 2 ** 62)) << 64 | int(g.integers(0, 2 ** 62)) << 2) % (1 << bits)
        if g.random() < 0.25 and bits > 60:  # a tie: the bit right below the 53rd set, nothing below it
            top = bits - 53
            w = (w >> top << top) | (1 << (top - 1))
        if g.random() < 0.5:
            w = -w
        S = int(g.integers(-1200, 900)) if g.random() < 0.2 else int(g.integers(-300, 100))
        cases.append((w, S))
    cases += [(1, -1074), (3, -1075), ((1 << 53) - 1, 971), ((1 << 53) + 1, 971), (-(1 << 120) - 1, -30)]
    for w, S in cases:
        lo_, hi_ = split_w(w)
        got = fx.fxs_w_to_double(lo_, hi_, S)
        exact = F(w) * F(2) ** S
        try:
            want = rn(exact)
        except OverflowError:  # beyond the largest double: infinity, as IEEE rounding gives
            want = float("inf") if exact > 0 else float("-inf")
        assert got == want, (w, S)


def test_sub_round_is_correctly_rounded(fx):
    g = np.random.default_rng(5)
    for _ in range(3000):
        y = float(np.ldexp(g.standard_normal(), int(g.integers(-60, 60))))
        mode = g.integers(0, 3)
        S = int(g.integers(-250, -40))
        if mode == 0:  # cancellation: w 2^S close to y
            w = int(F(y) / F(2) ** S) + int(g.integers(-1000, 1000))
        elif mode == 1:
            w = int(g.integers(-2 ** 62, 2 ** 62))
        else:
            w = int(g.integers(-2 ** 40, 2 ** 40)) << int(g.integers(0, 80))
        if not -(1 << 126) < w < (1 << 126):
            continue
        lo_, hi_ = split_w(w)
        got = fx.fxs_sub_round(y, lo_, hi_, S)
        exact = F(y) - F(w) * F(2) ** S
        # the grid of the result is 2^S, or coarser when y dominates by more than 2^72
        unit = max(F(2) ** S, F(2) ** (int(np.frexp(abs(y))[1]) - 53 - 72))
        if unit == F(2) ** S or exact == 0:
            assert got == rn(exact), (y, w, S)
        else:  # w truncated to the coarser grid first: absolute error below two grid units
            assert abs(F(got) - exact) <= abs(exact) * F(2) ** -53 + 2 * unit


def _bits(x):
    return np.float64(x).view(np.uint64).item()


def test_fast_roundings_match_the_general_ones_bitwise(fx):
    """w_to_double_fast / sub_round_fast (the row kernels' branch-free
    epilogue forms): wherever they report ok, the same bits as w_to_double /
    sub_round; ok on every normal-range case of the kernels' kind (y normal,
    the product grid at or below y's, a normal result)."""
    g = np.random.default_rng(17)
    ok = C.c_int(0)
    n_ok = n_typ = 0
    for _ in range(6000):
        bits = int(g.integers(0, 127))
        w = (int(g.integers(0, 2 ** 62)) << 64 | int(g.integers(0, 2 ** 62)) << 2 | int(g.integers(0, 4)))
        w %= (1 << bits) if bits else 1
        if g.random() < 0.2 and bits > 60:  # a tie
            top = bits - 53
            w = (w >> top << top) | (1 << (top - 1))
        if g.random() < 0.5:
            w = -w
        S = int(g.integers(-1300, 1000)) if g.random() < 0.15 else int(g.integers(-300, 100))
        lo_, hi_ = split_w(w)
        got = fx.fxs_w_to_double_fast(lo_, hi_, S, C.byref(ok))
        if ok.value:
            n_ok += 1
            assert _bits(got) == _bits(fx.fxs_w_to_double(lo_, hi_, S)), (w, S)
        exact = abs(F(w)) * F(2) ** S
        if w == 0 or F(2) ** -1022 <= exact < F(2) ** 1023:
            n_typ += 1
            assert ok.value, (w, S)
    assert n_ok >= n_typ > 4000
    n_typ = 0
    for _ in range(8000):
        y = float(np.ldexp(g.standard_normal(), int(g.integers(-80, 80))))
        mode = int(g.integers(0, 4))
        S = int(g.integers(-300, -30))
        if mode == 0:  # cancellation: w 2^S close to y
            w = int(F(y) / F(2) ** S) + int(g.integers(-10 ** 6, 10 ** 6))
        elif mode == 1:  # y dominating by 0 .. 120 binades (the coarsened grid beyond 72)
            e = int(np.frexp(abs(y))[1]) - S - int(g.integers(0, 120))
            w = int(g.integers(-2 ** 60, 2 ** 60)) << max(e - 60, 0) if e > 0 else int(g.integers(-4, 4))
        elif mode == 2:
            w = int(g.integers(-2 ** 62, 2 ** 62)) << int(g.integers(0, 60))
        else:
            w = 0
        if not -(1 << 126) < w < (1 << 126):
            continue
        lo_, hi_ = split_w(w)
        got = fx.fxs_sub_round_fast(y, lo_, hi_, S, C.byref(ok))
        want = fx.fxs_sub_round(y, lo_, hi_, S)
        ey = int(np.frexp(abs(y))[1]) - 53
        if ok.value:
            assert _bits(got) == _bits(want), (y, w, S)
        if ey >= S and (want == 0.0 or 2.0 ** -1022 <= abs(want) < 2.0 ** 1023):
            n_typ += 1
            assert ok.value, (y, w, S)
    assert n_typ > 3000
    # the rare cases fall back: subnormal y, y below the grid, a result past the range
    assert not (fx.fxs_sub_round_fast(5e-324, *split_w(1), -1074, C.byref(ok)), ok.value)[1]
    assert not (fx.fxs_sub_round_fast(1.0, *split_w(3), -40, C.byref(ok)), ok.value)[1]
    assert not (fx.fxs_w_to_double_fast(*split_w(1), -1080, C.byref(ok)), ok.value)[1]
    assert not (fx.fxs_w_to_double_fast(*split_w(1 << 100), 950, C.byref(ok)), ok.value)[1]


def test_acc256_sums_exactly(fx):
    g = np.random.default_rng(6)
    for m in (1, 5, 40):
        ws = [int(g.integers(-2 ** 62, 2 ** 62)) << 63 for _ in range(m)]
        lo = np.array([split_w(w)[0] for w in ws], dtype=np.int64)
        hi = np.array([split_w(w)[1] for w in ws], dtype=np.int64)
        wl, wh, ex = C.c_longlong(), C.c_longlong(), C.c_int()
        fx.fxs_acc256(m, lo.ctypes.data, hi.ctypes.data, C.byref(wl), C.byref(wh), C.byref(ex))
        total = sum(ws)
        got = (wl.value & ((1 << 64) - 1)) | (wh.value << 64)
        if ex.value == 0:
            assert got == total
        else:
            assert got == (total >> ex.value) or got == -((-total) >> ex.value)
