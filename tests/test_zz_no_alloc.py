"""eo_gram_dd_noalloc: the compensated Gram product for callers that cannot
allocate device memory when they need it (their GPU memory is owned by
another allocator, or they must not pay for cudaMalloc/cudaFree on a
latency-critical path).  It uses only a fixed scratch array inside the
library.  It is checked here through the C-ABI against the binary128 oracle
directly, twice in a row (the second call reuses the scratch the first left
behind), with the EO_DD tolerance of the other Gram tests; its argument
checks (block width, row limit) are checked without a GPU.

This file is named to be collected last: a stop at its first failure leaves
every other test already run.  It also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

U2 = 2.0 ** -104


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(a).T)).cuda().t()


def _host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def _tol(x, y, ref):
    """EO_DD bound: |G - G*| <= 2^-104 |G*| + n 2^-101 max|x_i| max|y_j|."""
    n = x.shape[0]
    return U2 * np.abs(ref) + n * 2.0 ** -101 * np.outer(np.max(np.abs(x), axis=0), np.max(np.abs(y), axis=0))


def _noalloc(eo, X, Y=None, want_lo=True, n=None):
    """Call eo_gram_dd_noalloc through the C-ABI with torch-owned buffers."""
    import torch
    rows, kx = X.shape
    n = rows if n is None else n
    ky = kx if Y is None else Y.shape[1]
    hi = torch.full((ky, kx), np.nan, dtype=torch.float64, device="cuda").t()
    lo = torch.full((ky, kx), np.nan, dtype=torch.float64, device="cuda").t()
    st = eo.lib().eo_gram_dd_noalloc(n, kx, X.data_ptr(), max(1, X.stride(1)), ky,
                                     None if Y is None else Y.data_ptr(),
                                     max(1, X.stride(1) if Y is None else Y.stride(1)), hi.data_ptr(),
                                     lo.data_ptr() if want_lo else None, kx,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, hi, lo


@pytest.mark.gpu
def test_noalloc_gram_matches_oracle_on_two_calls(eo):
    # 400,003 rows x 16: every one of the 152 row chunks of the array is used
    cases = [(synth.gaussian(400_003, 16, 901), None),
             (synth.conditioned(70_001, 5, 1e6, 902), synth.gaussian(70_001, 11, 903))]
    for x, y in cases:
        yy = x if y is None else y
        rh, rl = oracle.gram(x, y)
        X = _dev(x)
        Y = None if y is None else _dev(y)
        for _ in range(2):  # two calls in a row on the shared array
            st, hi, lo = _noalloc(eo, X, Y)
            assert st == eo.OK
            err = np.abs((_host(hi) - rh) + (_host(lo) - rl))
            assert np.all(err <= _tol(x, yy, rh)), float(np.max(err / _tol(x, yy, rh)))


@pytest.mark.gpu
def test_noalloc_gram_without_low_part_and_empty(eo):
    x = synth.conditioned(50_000, 7, 1e4, 905)
    X = _dev(x)
    st, hi, lo = _noalloc(eo, X)
    st2, hi2, lo2 = _noalloc(eo, X, want_lo=False)
    assert st == st2 == eo.OK
    assert np.array_equal(_host(hi2), _host(hi))  # the high part does not depend on the low part's output
    assert np.all(np.isnan(_host(lo2)))  # G_lo == NULL: nothing written there
    st, hi, lo = _noalloc(eo, X, n=0)  # no rows: G = 0
    assert st == eo.OK and not np.any(_host(hi)) and not np.any(_host(lo))


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    """Block widths above EO_NOALLOC_KMAX, or more rows than the array's 152
    row chunks of 2^22 rows, are rejected before any CUDA call (so this runs
    without a GPU; the pointers are never read)."""
    from paper_1806_01036_gb300 import build
    L = C.CDLL(build.build())
    f = L.eo_gram_dd_noalloc
    f.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p,
                  C.c_void_p, C.c_int, C.c_void_p]
    f.restype = C.c_int
    fake = C.c_void_p(4096)  # never dereferenced: every case fails the size checks
    nmax = 152 << 22
    assert f(1000, 17, fake, 1000, 17, None, 1000, fake, fake, 17, None) == 1            # kx = 17 (symmetric)
    assert f(1000, 5, fake, 1000, 17, fake, 1000, fake, fake, 5, None) == 1               # ky = 17
    assert f(nmax + 1, 4, fake, nmax + 1, 4, None, nmax + 1, fake, fake, 4, None) == 1    # rows beyond the limit
    assert f(-1, 4, fake, 1, 4, None, 1, fake, fake, 4, None) == 1                         # negative rows
    assert f(100, 4, fake, 99, 4, None, 99, fake, fake, 4, None) == 1                      # ld < n
    import paper_1806_01036_gb300 as eo
    assert eo.NOALLOC_KMAX == 16 and eo.NOALLOC_NMAX == nmax
