"""eo_gram_dd_noalloc: the compensated Gram product for callers that cannot
allocate device memory when they need it (their GPU memory is owned by
another allocator, or they must not pay for cudaMalloc/cudaFree on a
latency-critical path).  It uses only a fixed scratch array inside the
library, so it is checked here through the C-ABI against eo_gram(EO_DD) on
the same inputs, twice in a row, with the tolerance of the other Gram tests.

This file is named to be collected last: a stop at its first failure leaves
every other test already run.  It also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U2 = 2.0 ** -104


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(a).T)).cuda().t()


def _host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def _tol(x, y, ref):
    n = x.shape[0]
    return U2 * np.abs(ref) + n * 2.0 ** -101 * np.outer(np.max(np.abs(x), axis=0), np.max(np.abs(y), axis=0))


def _noalloc(eo, X, Y=None):
    """Call eo_gram_dd_noalloc through the C-ABI with torch-owned buffers."""
    import torch
    n, kx = X.shape
    ky = kx if Y is None else Y.shape[1]
    hi = torch.full((ky, kx), np.nan, dtype=torch.float64, device="cuda").t()
    lo = torch.full((ky, kx), np.nan, dtype=torch.float64, device="cuda").t()
    st = eo.lib().eo_gram_dd_noalloc(n, kx, X.data_ptr(), X.stride(1), ky, None if Y is None else Y.data_ptr(),
                                     X.stride(1) if Y is None else Y.stride(1), hi.data_ptr(), lo.data_ptr(), kx,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, hi, lo


def test_noalloc_gram_matches_gram_on_two_calls(eo):
    import torch
    ctx = eo.Context(0)
    try:
        cases = [(synth.gaussian(200_003, 16, 901), None),
                 (synth.conditioned(70_001, 5, 1e6, 902), synth.gaussian(70_001, 11, 903))]
        for x, y in cases:  # two calls in a row: the second reuses the scratch the first left behind
            X = _dev(x)
            Y = None if y is None else _dev(y)
            st, hi, lo = _noalloc(eo, X, Y)
            assert st == eo.OK
            rh, rl = eo.gram(ctx, X, Y, prec=eo.DD)
            torch.cuda.synchronize()
            ref = _host(rh) + _host(rl)
            got_err = np.abs((_host(hi) - _host(rh)) + (_host(lo) - _host(rl)))
            yy = x if y is None else y
            assert np.all(got_err <= _tol(x, yy, ref))
    finally:
        ctx.close()


def test_noalloc_gram_rejects_sizes_beyond_its_scratch(eo):
    import torch
    X = _dev(synth.gaussian(1000, 17, 904))
    st, _, _ = _noalloc(eo, X)
    assert st == eo.EINVAL
    assert eo.NOALLOC_KMAX == 16
