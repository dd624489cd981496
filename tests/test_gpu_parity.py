"""GPU parity: the CUDA library (through its C-ABI binding) against the
binary128 oracle on the same seeded inputs.

Tolerances (u = 2^-53, u2 = 2^-104; |A| is the entry-wise absolute value):
  * Gram, EO_DD (exact fixed point): every summed group is aligned to an
      exponent at or above its largest; the integer-limb engine keeps the ten
      leading limb products of 104-bit integers (each product off by less than
      2^-101 max|x_i| max|y_j|), the tensor-core engine the 120 leading pairs
      of 15 balanced 7-bit digits with its alignment exponent up to two
      binades above the column's largest (each product off by less than
      22.2 * 2^-101 max|x_i| max|y_j| < 2^-96.5 max|x_i| max|y_j|); the sums
      are exact otherwise:
      |G - G*| <= u2 |G*| + n 2^-96 max|x_i| max|y_j|.
      This bound is normwise in the columns (max|x_i| max|y_j|), not
      componentwise like the Dot2 bound gamma_n^2 |x_i|^T |y_j|: a column
      whose entries span many binades is exact only down to its largest
      entry's grid, so an entry formed from its small members is judged
      against that column's largest value (test_gram_dd_componentwise_ratio
      reports how far the result is from the componentwise bound).
  * Gram, EO_DD_EFT (TwoProd + TwoSum on the FP64 pipe):
      |G - G*| <= u2 |G*| + (n + 64) 2^-105 (|X|^T |Y|): each thread's Dot2
      chain and the fixed reduction tree add a few u^2 per partial sum, so a
      bound linear in n holds (tighter than Dot2's gamma_n^2).
  * Gram, FP64/F32:   |G - G*| <= gamma_n |X|^T |Y|, gamma_n = n u / (1 - n u)
      (the textbook dot-product bound; F32 products are exact in FP64).
  * CholQR/SVQB, DD:  both sides factor a Gram matrix that is accurate to
      eps_M = (n + 64) 2^-104 relative; a perturbation of relative size eps of
      M moves R (and Q) by at most ~kappa^2 eps, so
      |Q - Q*| <= 4 u + 8 kappa^2 (eps_M + k u2) and the same, times ||R||, for R.
      The orthogonality gate of the method itself (||Q^T Q - I||_2 <= 1e-14 up
      to kappa(X) = 1e8 in one DD pass) is checked with the oracle's
      binary128 measure.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
U2 = 2.0 ** -104


def torch_mod():
    import torch
    return torch


def dev(a, dtype=None):
    """numpy column-major -> CUDA tensor with the same column-major layout."""
    torch = torch_mod()
    a = np.asfortranarray(a if dtype is None else a.astype(dtype))
    t = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    return t.t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def dd_err(hi, lo, ref_hi, ref_lo):
    """|(hi + lo) - (ref_hi + ref_lo)| entry-wise, evaluated without cancellation loss."""
    return np.abs((hi - ref_hi) + (lo - ref_lo))


def gamma(n):
    return n * U / (1 - n * U)


# ------------------------------------------------------------------ Gram

def dd_gram_tol(x, y, ref, engine):
    n = x.shape[0]
    if engine == 1:  # EO_DD, exact fixed point
        return U2 * np.abs(ref) + n * 2.0 ** -96 * np.outer(np.max(np.abs(x), axis=0), np.max(np.abs(y), axis=0))
    return U2 * np.abs(ref) + (n + 64) * 2.0 ** -105 * (np.abs(x).T @ np.abs(y))


@pytest.mark.parametrize("engine", [1, 3])
@pytest.mark.parametrize("n,kx,ky", [(1, 1, 1), (33, 3, 3), (1000, 8, 8), (4099, 13, 5), (100_003, 16, 16),
                                     (20_000, 64, 64), (20_001, 64, 16), (70_001, 2, 7)])
def test_gram_dd_matches_oracle(eo, ctx, engine, n, kx, ky):
    x = synth.gaussian(n, kx, 100 + kx)
    y = x if kx == ky and n % 2 else synth.gaussian(n, ky, 200 + ky)
    sym = y is x
    gh, gl = eo.gram(ctx, dev(x), None if sym else dev(y), prec=engine)
    rh, rl = oracle.gram(x, None if sym else y)
    err = dd_err(host(gh), host(gl), rh, rl)
    tol = dd_gram_tol(x, y, rh, engine)
    assert np.all(err <= tol), float(np.max(err / tol))
    # the high part is the FP64 rounding of the exact sum (up to the last bit)
    assert np.all(np.abs(host(gh) - rh) <= 2 * U * np.abs(rh) + tol)
    if sym:
        assert np.array_equal(host(gh), host(gh).T)


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("n,k", [(777, 5), (50_000, 16)])
def test_gram_fp64_and_f32_within_textbook_bound(eo, ctx, prec, n, k):
    x = synth.conditioned(n, k, 1e3, 300 + k)
    if prec == eo.F32:
        x32 = x.astype(np.float32)
        gh, gl = eo.gram(ctx, dev(x32), prec=prec)
        rh, rl = oracle.gram_f32(x32)
        ax = np.abs(x32.astype(np.float64))
    else:
        gh, gl = eo.gram(ctx, dev(x), prec=prec)
        rh, rl = oracle.gram(x)
        ax = np.abs(x)
    err = np.abs(host(gh) - (rh + rl))
    assert np.all(err <= gamma(n) * (ax.T @ ax) + U * np.abs(rh))
    assert not np.any(host(gl))


@pytest.mark.parametrize("n,kx,ky,sym", [(50_000, 16, 16, True), (20_001, 32, 32, True), (30_000, 64, 16, False),
                                         (7_777, 5, 19, False), (4_097, 64, 64, True), (1, 16, 16, True)])
def test_gram_f32_on_the_digit_engine(eo, ctx, monkeypatch, n, kx, ky, sym):
    """EO_F32 with 16 or more columns on one side: the FP32 products summed
    exactly by the tensor-core engine (values widened to FP64 exactly, by
    integer arithmetic), the sum rounded once -- within u |G*| plus the
    engine's own n 2^-96 max|x_i| max|y_j| of the binary128 value, i.e. at
    least as accurate as FP64 accumulation; the low parts are zero.  Edge
    values (subnormal, zero, negative zero, powers of two) go through the
    widening's conversion path.  The FP64-pipe sums (EO_F32_GRAM_ENGINE=fp64)
    agree within the textbook bound."""
    g = synth.rng(310 + kx)
    x = g.standard_normal((n, kx)).astype(np.float32)
    y = x if sym else g.standard_normal((n, ky)).astype(np.float32)
    if n > 8:
        x[3, 0] = np.float32(1e-40)  # subnormal
        x[4, 0] = np.float32(-0.0)
        x[5, min(1, kx - 1)] = np.float32(2.0 ** -20)
    dx = dev(x)
    dy = None if sym else dev(y)
    gh, gl = eo.gram(ctx, dx, dy, prec=eo.F32)
    rh, rl = oracle.gram_f32(x, None if sym else y)
    yy = x if sym else y
    ax, ay = np.abs(x.astype(np.float64)), np.abs(yy.astype(np.float64))
    err = np.abs(host(gh) - (rh + rl))
    bound = U * np.abs(rh) + n * 2.0 ** -96 * np.outer(ax.max(axis=0), ay.max(axis=0))
    assert np.all(err <= bound), float(np.max(err / bound))
    assert not np.any(host(gl))
    monkeypatch.setenv("EO_F32_GRAM_ENGINE", "fp64")
    ph, _ = eo.gram(ctx, dx, dy, prec=eo.F32)
    assert np.all(np.abs(host(ph) - (rh + rl)) <= gamma(n) * (ax.T @ ay) + U * np.abs(rh))


def test_cholqr_f32_wide_block(eo, ctx):
    n, k = 40_000, 24  # the Gram of the CholQR passes on the digit engine
    x = synth.conditioned(n, k, 1e2, 81).astype(np.float32)
    d = dev(x)
    rh, _, info = eo.cholqr(ctx, d, prec=eo.F32)
    assert int(info.item()) == 0
    q = host(d).astype(np.float64)
    assert oracle.orth_err(q)[0] <= 1e-5  # FP32 storage of Q
    q_o, (rh_o, _), _ = oracle.cholqr(x.astype(np.float64))
    np.testing.assert_allclose(host(rh), rh_o, rtol=0, atol=1e-12 * np.max(np.abs(rh_o)))


@pytest.mark.parametrize("engine", ["int", "umma"])
@pytest.mark.parametrize("n,kx,ky,sym", [(1, 1, 1, True), (33, 3, 3, True), (1000, 8, 8, False), (4099, 13, 5, False),
                                         (100_003, 16, 16, True), (20_000, 64, 64, True), (20_001, 64, 16, False),
                                         (70_001, 2, 7, False), (50_000, 40, 24, False), (30_017, 33, 33, True),
                                         (131, 17, 9, False), (9_000, 64, 12, False), (5_003, 48, 16, False),
                                         (9_000, 24, 24, True), (20_001, 48, 48, True)])
def test_gram_dd_both_engines(eo, ctx, monkeypatch, engine, n, kx, ky, sym):
    """The integer-limb and the tcgen05 digit engines of EO_DD against the
    oracle.  A symmetric product with more than 16 columns runs on the tensor
    cores as column strips of 16 (a partial last strip at k = 24, 33; odd n:
    operands copied by the converter threads); it is exactly symmetric."""
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", engine)
    x = synth.gaussian(n, kx, 400 + kx)
    y = x if sym else synth.gaussian(n, ky, 500 + ky)
    gh, gl = eo.gram(ctx, dev(x), None if sym else dev(y), prec=eo.DD)
    rh, rl = oracle.gram(x, None if sym else y)
    err = dd_err(host(gh), host(gl), rh, rl)
    tol = dd_gram_tol(x, y, rh, 1)
    assert np.all(err <= tol), float(np.max(err / tol))
    if sym:
        assert np.array_equal(host(gh), host(gh).T) and np.array_equal(host(gl), host(gl).T)


@pytest.mark.parametrize("engine", ["int", "umma"])
def test_gram_dd_engines_rescale_and_range(eo, ctx, monkeypatch, engine):
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", engine)
    n = 200_000
    x = synth.gaussian(n, 16, 18) * np.logspace(-30, 3, n)[:, None]
    y = synth.gaussian(n, 8, 19) * np.logspace(3, -30, n)[:, None]
    g = synth.rng(23)
    z = np.asfortranarray(np.ldexp(g.standard_normal((n, 16)), g.integers(-80, 20, size=(n, 16))))
    for a, b in ((x, None), (x, y), (z, None)):
        gh, gl = eo.gram(ctx, dev(a), None if b is None else dev(b), prec=eo.DD)
        rh, rl = oracle.gram(a, b)
        bb = a if b is None else b
        assert np.all(dd_err(host(gh), host(gl), rh, rl) <= dd_gram_tol(a, bb, rh, 1))


@pytest.mark.parametrize("engine", ["int", "umma"])
@pytest.mark.parametrize("kx,ky,sym", [(64, 16, False), (16, 16, True), (64, 40, False), (20, 8, False)])
def test_gram_dd_engines_largest_digits(eo, ctx, monkeypatch, engine, kx, ky, sym):
    """Every mantissa bit set and one exponent per column: all leading digits
    take their largest value, so every per-diagonal sum reaches its bound."""
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", engine)
    n = 70_001
    top = 2.0 - 2.0 ** -52
    g = synth.rng(31)
    x = np.asfortranarray(np.full((n, kx), top) * np.ldexp(1.0, g.integers(-3, 4, size=kx))[None, :])
    y = x if sym else np.asfortranarray(np.full((n, ky), -top) * np.ldexp(1.0, g.integers(-3, 4, size=ky))[None, :])
    y[::7, :] *= -1.0
    gh, gl = eo.gram(ctx, dev(x), None if sym else dev(y), prec=eo.DD)
    rh, rl = oracle.gram(x, None if sym else y)
    assert np.all(dd_err(host(gh), host(gl), rh, rl) <= dd_gram_tol(x, y, rh, 1))


@pytest.mark.parametrize("engine", ["int", "umma"])
def test_gram_dd_engines_odd_leading_dimension(eo, ctx, monkeypatch, engine):
    """Leading dimensions and base addresses that are only 8-byte aligned."""
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", engine)
    torch = torch_mod()
    n, kx, ky = 3001, 24, 16
    x = synth.gaussian(n, kx, 41)
    y = synth.gaussian(n, ky, 42)
    ts = []
    for a, ld in ((x, 3003), (y, 3005)):
        buf = synth.with_ld(a, ld + 1, fill=np.nan)
        t = torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().reshape(-1)
        # a view starting one element into the buffer, leading dimension ld (odd)
        v = t[1:1 + ld * a.shape[1]].reshape(a.shape[1], ld).t()[:n, :]
        v.copy_(torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t())
        assert v.stride(1) == ld and v.data_ptr() % 16 == 8
        ts.append(v)
    gh, gl = eo.gram(ctx, ts[0], ts[1], prec=eo.DD)
    rh, rl = oracle.gram(x, y)
    assert np.all(dd_err(host(gh), host(gl), rh, rl) <= dd_gram_tol(x, y, rh, 1))


def test_gram_dd_integer_inputs_are_exact(eo, ctx):
    # small integers sit exactly on the fixed-point grid: every product and sum is exact
    g = synth.rng(17)
    n, k = 50_001, 6
    xi = g.integers(-1000, 1001, size=(n, k))
    x = np.asfortranarray(xi.astype(np.float64))
    gh, gl = eo.gram(ctx, dev(x), prec=eo.DD)
    ref = xi.T @ xi  # exact in int64 (|sum| < 2^53)
    assert np.array_equal(host(gh), ref.astype(np.float64)) and not np.any(host(gl))


def _straddling_integers(g, n, k):
    """Integers sign * m * 2^j (m odd below 128, some zeros): in the first
    half of the rows j in [14, 25), so whole warps lie within 20 binades of
    their column's largest value; in the second half j in [0, 25), so most
    warps do not.  Products and sums stay exact in binary128."""
    m = 2 * g.integers(0, 64, size=(n, k)) + 1
    j = np.where(np.arange(n)[:, None] < n // 2, g.integers(14, 25, size=(n, k)), g.integers(0, 25, size=(n, k)))
    x = np.ldexp(m.astype(np.float64), j) * np.where(g.random((n, k)) < 0.5, -1.0, 1.0)
    x[g.random((n, k)) < 0.002] = 0.0
    return np.asfortranarray(x)


@pytest.mark.parametrize("n,kx,ky,sym", [(40_000, 64, 16, False), (40_000, 16, 16, True), (20_001, 24, 8, False),
                                         (30_000, 40, 40, True)])
def test_gram_dd_near_path_boundary_is_exact(eo, ctx, n, kx, ky, sym):
    """Integer values straddling the 20-binade window of the tensor-core
    Gram's near path (both paths in one product, panels of each kind): no
    digit pair is dropped for them, so G_hi + G_lo is the exact sum rounded
    to a double-double, bit for bit the oracle's (binary128 is exact here)."""
    g = synth.rng(83 + kx)
    x = _straddling_integers(g, n, kx)
    y = x if sym else _straddling_integers(g, n, ky)
    gh, gl = eo.gram(ctx, dev(x), None if sym else dev(y), prec=eo.DD)
    rh, rl = oracle.gram(x, None if sym else y)
    assert np.array_equal(host(gh), rh) and np.array_equal(host(gl), rl)


def test_gram_dd_growing_exponents_rescale(eo, ctx):
    # the first rows are tiny, later rows large: the running alignment exponent of
    # every column grows many times and the accumulators are shifted each time
    n, k = 300_000, 5
    x = synth.gaussian(n, k, 18)
    x *= np.logspace(-30, 3, n)[:, None]
    y = synth.gaussian(n, 3, 19) * np.logspace(3, -30, n)[:, None]
    for a, b in ((x, None), (x, y)):
        gh, gl = eo.gram(ctx, dev(a), None if b is None else dev(b), prec=eo.DD)
        rh, rl = oracle.gram(a, b)
        bb = a if b is None else b
        assert np.all(dd_err(host(gh), host(gl), rh, rl) <= dd_gram_tol(a, bb, rh, 1))


def test_gram_dd_wide_range_within_columns(eo, ctx):
    g = synth.rng(23)
    n, k = 40_000, 4
    x = np.asfortranarray(np.ldexp(g.standard_normal((n, k)), g.integers(-80, 20, size=(n, k))))
    gh, gl = eo.gram(ctx, dev(x), prec=eo.DD)
    rh, rl = oracle.gram(x)
    assert np.all(dd_err(host(gh), host(gl), rh, rl) <= dd_gram_tol(x, x, rh, 1))


@pytest.mark.parametrize("engine", ["int", "umma"])
def test_gram_dd_componentwise_ratio(eo, ctx, monkeypatch, engine, capsys):
    """How far EO_DD is from the componentwise Dot2 bound on columns whose
    entries span 100 binades: the ratio err / (u2 |G*| + gamma_n^2 |x_i|^T |x_j|)
    is reported; the normwise bound must hold, and so must twice the
    componentwise bound wherever that is above the normwise bound's grid
    term (there the normwise bound is at most twice the componentwise one)."""
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", engine)
    g = synth.rng(23)
    n, k = 40_000, 16
    x = np.asfortranarray(np.ldexp(g.standard_normal((n, k)), g.integers(-80, 20, size=(n, k))))
    gh, gl = eo.gram(ctx, dev(x), prec=eo.DD)
    rh, rl = oracle.gram(x)
    err = dd_err(host(gh), host(gl), rh, rl)
    comp = U2 * np.abs(rh) + gamma(n) ** 2 * (np.abs(x).T @ np.abs(x))
    ratio = float(np.max(err / comp))
    with capsys.disabled():
        print(f"\n[componentwise] engine={engine} max err / (u2|G| + gamma_n^2 |x_i|^T|x_j|) = {ratio:.3g}")
    assert np.all(err <= dd_gram_tol(x, x, rh, 1))
    grid = n * 2.0 ** -96 * np.outer(np.max(np.abs(x), axis=0), np.max(np.abs(x), axis=0))
    big = comp >= grid
    assert np.all(err[big] <= 2 * comp[big])


def test_gram_dd_nonfinite_input_gives_nan(eo, ctx):
    x = synth.gaussian(1000, 3, 20)
    x[500, 1] = np.inf
    gh, gl = eo.gram(ctx, dev(x), prec=eo.DD)
    assert np.isnan(host(gh)[1, 1]) and np.isnan(host(gh)[0, 1])


@pytest.mark.parametrize("n,k,ld", [(1001, 4, 1040), (5003, 40, 5010)])
def test_gram_ld_padding_is_not_read(eo, ctx, n, k, ld):
    """NaN in the padding rows between columns (ld > n) must not reach G; k =
    40 runs on the tensor cores as column strips, each at its own offset."""
    x = synth.gaussian(n, k, 5)
    buf = synth.with_ld(x, ld, fill=np.nan)
    torch = torch_mod()
    t = torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().t()[:n, :]
    assert t.stride(1) == ld
    gh, gl = eo.gram(ctx, t, prec=eo.DD)
    rh, rl = oracle.gram(x)
    assert np.all(np.isfinite(host(gh)))
    assert np.all(dd_err(host(gh), host(gl), rh, rl) <= U2 * np.abs(rh) + (n + 64) * 2.0 ** -105 * (np.abs(x).T @ np.abs(x)))


@pytest.mark.parametrize("k", [3, 12, 40])
def test_gram_empty_rows_give_zero(eo, ctx, k):
    """No rows: G = 0 for every engine (k = 3 integer limbs, 12 the tensor
    cores, 40 the tensor cores as column strips)."""
    torch = torch_mod()
    x = torch.zeros((0, k), dtype=torch.float64, device="cuda")
    x = x.t().contiguous().t()
    hi = torch.full((k, k), 7.0, dtype=torch.float64, device="cuda").t()
    lo = torch.full((k, k), 7.0, dtype=torch.float64, device="cuda").t()
    gh, gl = eo.gram(ctx, x, prec=eo.DD, out=(hi, lo))
    assert not torch.any(gh) and not torch.any(gl)


def test_gram_is_deterministic(eo, ctx):
    x = synth.gaussian(300_001, 8, 9)
    d = dev(x)
    a = eo.gram(ctx, d, prec=eo.DD)
    b = eo.gram(ctx, d, prec=eo.DD)
    assert np.array_equal(host(a[0]), host(b[0])) and np.array_equal(host(a[1]), host(b[1]))


# ------------------------------------------------------------ projection

@pytest.mark.parametrize("engine", [1, 3])
@pytest.mark.parametrize("n,kv,k", [(1, 1, 1), (5000, 10, 4), (20_003, 64, 16), (30_000, 40, 2)])
def test_project_dd_matches_oracle(eo, ctx, engine, n, kv, k):
    v = synth.orthonormal_basis(n, kv, 31) if n >= kv else synth.gaussian(n, kv, 31)
    y = synth.conditioned(n, k, 1e6, 32) if n >= k else synth.gaussian(n, k, 32)
    yt_d, (ch, cl), (mh, ml) = eo.project(ctx, dev(v), dev(y), prec=engine)
    yt_o, (ch_o, cl_o), _ = oracle.project(v, y)
    bound_c = dd_gram_tol(v, y, ch_o, engine)
    assert np.all(dd_err(host(ch), host(cl), ch_o, cl_o) <= bound_c)
    yt = host(yt_d)
    # y - V C summed exactly (EO_DD: per-row alignment of V, per-column of C) and rounded once
    row_max = np.max(np.abs(v), axis=1)[:, None] * np.max(np.abs(ch_o), axis=0)[None, :]
    tol_y = (2 * U * np.abs(yt_o) + 2.0 ** -100 * (np.abs(y) + np.abs(v) @ np.abs(ch_o))
             + kv * 2.0 ** -99 * row_max + np.abs(v) @ bound_c)
    assert np.all(np.abs(yt - yt_o) <= tol_y)
    # M is the Gram matrix of the rounded result the kernel wrote
    m_o = oracle.gram(yt)
    assert np.all(dd_err(host(mh), host(ml), *m_o) <= dd_gram_tol(yt, yt, m_o[0], engine))


@pytest.mark.parametrize("engine", [1, 0])
def test_project_apply_equals_project(eo, ctx, engine):
    n, kv, k = 33_333, 24, 6
    v = synth.orthonormal_basis(n, kv, 51)
    y = synth.conditioned(n, k, 1e4, 52)
    V, Y = dev(v), dev(y)
    yt1, c1, m1 = eo.project(ctx, V, Y, prec=engine)
    c = eo.gram(ctx, V, Y, prec=engine)
    yt2, m2 = eo.project_apply(ctx, V, Y, c, prec=engine)
    assert np.array_equal(host(c1[0]), host(c[0])) and np.array_equal(host(c1[1]), host(c[1]))
    assert np.array_equal(host(yt1), host(yt2))
    assert np.array_equal(host(m1[0]), host(m2[0])) and np.array_equal(host(m1[1]), host(m2[1]))


@pytest.mark.parametrize("engine", ["int", "umma"])
@pytest.mark.parametrize("n,kv,k", [(3001, 8, 5), (40_000, 16, 16), (20_011, 40, 16), (5000, 64, 7),
                                    (3000, 24, 40), (2049, 64, 64)])
def test_project_apply_integer_inputs_are_exact(eo, ctx, monkeypatch, engine, n, kv, k):
    """Integer V, C and Y: Y - V C is exact in FP64, so both row engines
    (integer limbs, tensor-core digits) must return it bit for bit."""
    monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
    torch = torch_mod()
    g = synth.rng(61)
    vi = g.integers(-1000, 1001, size=(n, kv))
    ci = g.integers(-1000, 1001, size=(kv, k))
    yi = g.integers(-2 ** 40, 2 ** 40, size=(n, k))
    c_hi = dev(ci.astype(np.float64))
    c_lo = torch.zeros_like(c_hi)
    out, _ = eo.project_apply(ctx, dev(vi.astype(np.float64)), dev(yi.astype(np.float64)), (c_hi, c_lo),
                              prec=eo.DD, want_m=False)
    exact = yi - vi @ ci  # |.| < 2^53: exact in int64 and in FP64
    assert np.array_equal(host(out), exact.astype(np.float64))


@pytest.mark.parametrize("n,kv", [(20_000, 64), (9_001, 32)])
def test_project_apply_near_path_boundary_is_exact(eo, ctx, n, kv):
    """Rows of V whose integer values straddle the 20-binade window of the
    row kernels' near path (kv > 16), in the first half of the rows within
    it, in the second half mostly not: Y - V C is exact in FP64 and must
    come back bit for bit."""
    torch = torch_mod()
    g = synth.rng(91 + kv)
    m = 2 * g.integers(0, 64, size=(n, kv)) + 1
    j = np.where(np.arange(n)[:, None] < n // 2, g.integers(7, 13, size=(n, kv)), g.integers(0, 18, size=(n, kv)))
    vi = (m << j) * np.where(g.random((n, kv)) < 0.5, -1, 1)
    vi[g.random((n, kv)) < 0.002] = 0
    ci = g.integers(-1000, 1001, size=(kv, 16))
    yi = g.integers(-2 ** 40, 2 ** 40, size=(n, 16))
    c_hi = dev(ci.astype(np.float64))
    out, _ = eo.project_apply(ctx, dev(vi.astype(np.float64)), dev(yi.astype(np.float64)),
                              (c_hi, torch.zeros_like(c_hi)), prec=eo.DD, want_m=False)
    exact = yi - vi @ ci  # |.| < 2^53: exact in int64 and in FP64
    assert np.array_equal(host(out), exact.astype(np.float64))


@pytest.mark.parametrize("n,kv,k", [(77_777, 64, 16), (10_001, 12, 16), (30_000, 33, 3)])
def test_project_apply_row_engines_agree(eo, ctx, monkeypatch, n, kv, k):
    """The tensor-core and integer row engines against the oracle on the same C."""
    v = synth.orthonormal_basis(n, kv, 71)
    y = synth.conditioned(n, k, 1e8, 72)
    V, Y = dev(v), dev(y)
    c = eo.gram(ctx, V, Y, prec=eo.DD)
    outs = {}
    for engine in ("int", "umma"):
        monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
        outs[engine] = host(eo.project_apply(ctx, V, Y, c, prec=eo.DD, want_m=False)[0])
    ch, cl = host(c[0]), host(c[1])
    ref = oracle.project_apply(v, y, ch, cl)
    row_max = np.max(np.abs(v), axis=1)[:, None] * np.max(np.abs(ch), axis=0)[None, :]
    tol = 2 * U * np.abs(ref) + kv * 2.0 ** -99 * row_max
    for engine, out in outs.items():
        assert np.all(np.abs(out - ref) <= tol), engine


@pytest.mark.parametrize("engine", ["int", "umma"])
@pytest.mark.parametrize("kv", [12, 16, 32, 64])
def test_project_apply_row_engines_largest_digits(eo, ctx, monkeypatch, engine, kv):
    """Every mantissa bit set, one exponent per row of V and per column of C
    (C's low part filling the next 53 bits), all of one sign: the leading
    digits of both operands take their largest values, so the digit-diagonal
    sums of the tensor-core row engine come as close to their bound as FP64
    data allows, at every tile width (kin <= 16, 32, 64)."""
    monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
    n, k = 20_011, 16
    top = 2.0 - 2.0 ** -52
    g = synth.rng(37 + kv)
    v = np.asfortranarray(np.full((n, kv), top) * np.ldexp(1.0, g.integers(-8, 9, size=n))[:, None])
    ch = np.asfortranarray(np.full((kv, k), top) * np.ldexp(1.0, g.integers(-8, 9, size=k))[None, :])
    cl = np.asfortranarray(ch * 2.0 ** -53)
    y = synth.gaussian(n, k, 38 + kv)
    out, _ = eo.project_apply(ctx, dev(v), dev(y), (dev(ch), dev(cl)), prec=eo.DD, want_m=False)
    ref = oracle.project_apply(v, y, ch, cl)
    row_max = np.max(np.abs(v), axis=1)[:, None] * np.max(np.abs(ch) + np.abs(cl), axis=0)[None, :]
    assert np.all(np.abs(host(out) - ref) <= 2 * U * np.abs(ref) + kv * 2.0 ** -99 * row_max)


def _random_dd(g, rows, cols):
    hi = np.asfortranarray(g.standard_normal((rows, cols)))
    lo = np.asfortranarray(hi * 2.0 ** -55 * g.uniform(-1, 1, (rows, cols)))
    return hi, lo


@pytest.mark.parametrize("engine", ["int", "umma"])
@pytest.mark.parametrize("n,kv,k", [(1, 64, 16), (127, 16, 1), (129, 17, 7), (255, 32, 16), (1000, 33, 2),
                                    (4097, 48, 16), (2049, 1, 16), (3333, 64, 5), (1000, 64, 33), (5000, 16, 64),
                                    (257, 8, 17), (4099, 32, 32), (600, 20, 24), (3001, 4, 20), (1025, 3, 32)])
def test_project_apply_shapes_against_oracle(eo, ctx, monkeypatch, engine, n, kv, k):
    """Row tails, every tile width of the tensor-core row engine (kv <= 16, 32,
    64), one and two blocks of 16 output columns (k <= 32 with kv <= 32: the
    inputs converted once), the integer limbs' register kernel with one to
    eight output groups per row (kv <= 8; 20 outputs leave three of eight
    groups idle) and odd output counts, with a genuine double-double C."""
    monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
    torch = torch_mod()
    g = synth.rng(90 + kv + k)
    v = synth.gaussian(n, kv, 91 + kv)
    y = synth.gaussian(n, k, 92 + k) * 1e-3
    ch, cl = _random_dd(g, kv, k)
    out, _ = eo.project_apply(ctx, dev(v), dev(y), (dev(ch), dev(cl)), prec=eo.DD, want_m=False)
    ref = oracle.project_apply(v, y, ch, cl)
    row_max = np.max(np.abs(v), axis=1)[:, None] * np.max(np.abs(ch) + np.abs(cl), axis=0)[None, :]
    assert np.all(np.abs(host(out) - ref) <= 2 * U * np.abs(ref) + kv * 2.0 ** -99 * row_max)


@pytest.mark.parametrize("engine", ["int", "umma"])
def test_project_apply_nonfinite_and_padding(eo, ctx, monkeypatch, engine):
    """NaN in a row of V poisons that row only; NaN in C poisons its column;
    padding rows of V and Y (leading dimension > n, filled with NaN) are not read."""
    monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
    torch = torch_mod()
    n, kv, k, ld = 1500, 24, 6, 1531
    g = synth.rng(95)
    v = synth.gaussian(n, kv, 96)
    y = synth.gaussian(n, k, 97)
    ch, cl = _random_dd(g, kv, k)

    def padded(a):
        buf = synth.with_ld(a, ld, fill=np.nan)
        return torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().t()[: a.shape[0], :]

    out, _ = eo.project_apply(ctx, padded(v), padded(y), (dev(ch), dev(cl)), prec=eo.DD, want_m=False)
    assert np.all(np.isfinite(host(out)))
    ref = oracle.project_apply(v, y, ch, cl)
    row_max = np.max(np.abs(v), axis=1)[:, None] * np.max(np.abs(ch) + np.abs(cl), axis=0)[None, :]
    assert np.all(np.abs(host(out) - ref) <= 2 * U * np.abs(ref) + kv * 2.0 ** -99 * row_max)
    v2 = v.copy()
    v2[700, 3] = np.nan
    ch2 = ch.copy()
    ch2[5, 4] = np.inf
    o2 = host(eo.project_apply(ctx, dev(v2), dev(y), (dev(ch2), dev(cl)), prec=eo.DD, want_m=False)[0])
    assert np.all(np.isnan(o2[700, :])) and np.all(np.isnan(o2[:, 4]))
    rest = np.ones_like(o2, dtype=bool)
    rest[700, :] = False
    rest[:, 4] = False
    assert np.all(np.isfinite(o2[rest]))


@pytest.mark.parametrize("n,k", [(60_000, 16), (30_001, 33), (20_000, 64), (9_000, 17)])
def test_cholqr_update_engines_agree(eo, ctx, monkeypatch, n, k):
    """One DD CholQR pass with either row engine for Q = X R^-1 (17 <= k <= 32:
    the tensor cores in one pass over two 16-column output blocks; k > 32: in
    groups of 16 output columns through a scratch copy)."""
    x = synth.conditioned(n, k, 1e6, 81)
    qs = {}
    for engine in ("int", "umma"):
        monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
        d = dev(x)
        eo.cholqr(ctx, d, passes=1, prec=eo.DD)
        qs[engine] = host(d)
    q_o, _, _ = oracle.cholqr(x, passes=1)
    tol = cholqr_tol(n, k, 1e6)
    for engine, q in qs.items():
        assert np.max(np.abs(q - q_o)) <= tol, engine
        assert oracle.orth_err(q)[0] <= 1e-14, engine


def test_project_in_place_and_fp64(eo, ctx):
    n, kv, k = 12_345, 12, 3
    v = synth.orthonormal_basis(n, kv, 41)
    y = synth.gaussian(n, k, 42)
    d = dev(y)
    yt_d, _, (mh, _) = eo.project(ctx, dev(v), d, Yout=d, prec=eo.FP64)
    assert yt_d.data_ptr() == d.data_ptr()
    yt_o, (ch_o, _), _ = oracle.project(v, y)
    yt = host(yt_d)
    c_bound = gamma(n) * (np.abs(v).T @ np.abs(y))
    tol = gamma(kv + 2) * (np.abs(y) + np.abs(v) @ (np.abs(ch_o) + c_bound)) + np.abs(v) @ c_bound
    assert np.all(np.abs(yt - yt_o) <= tol)
    assert oracle.cross_err(v, yt) < 1e-13 * np.linalg.norm(y, 2)


# --------------------------------------------------------------- CholQR

def cholqr_tol(n, k, kappa):
    eps_m = (n + 64) * U2
    return 4 * U + 8 * kappa ** 2 * (eps_m + k * U2)


@pytest.mark.parametrize("engine", [1, 3])
@pytest.mark.parametrize("n,k,kappa", [(20_000, 8, 1e2), (20_000, 8, 1e6), (20_001, 16, 1e8), (5_000, 4, 1e8),
                                       (4_097, 1, 1.0), (3000, 33, 1e4)])
def test_cholqr_dd_one_pass(eo, ctx, engine, n, k, kappa):
    x = synth.conditioned(n, k, kappa, 500 + k)
    d = dev(x)
    rh, rl, info = eo.cholqr(ctx, d, passes=1, prec=engine)
    assert int(info.item()) == 0
    q = host(d)
    q_o, (rh_o, rl_o), info_o = oracle.cholqr(x, passes=1)
    assert info_o == 0
    tol = cholqr_tol(n, k, kappa)
    assert np.max(np.abs(q - q_o)) <= tol
    r = host(rh) + host(rl)
    assert np.max(np.abs(r - (rh_o + rl_o))) <= tol * np.max(np.abs(rh_o))
    assert np.all(np.tril(host(rh), -1) == 0) and np.all(np.diag(host(rh)) > 0)
    # the method's own accuracy claim: one DD pass is orthogonal to 1e-14 up to kappa = 1e8
    assert oracle.orth_err(q)[0] <= 1e-14
    assert oracle.fact_err(x, q, host(rh), host(rl)) <= 1e-15 * np.sqrt(k) + 8 * U


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_cholqr_fp64_loses_orthogonality_like_kappa_squared(eo, ctx, kappa):
    n, k = 20_000, 8
    x = synth.conditioned(n, k, kappa, 600)
    dp, dd_ = dev(x), dev(x)
    _, _, info_p = eo.cholqr(ctx, dp, prec=eo.FP64)
    _, _, info_d = eo.cholqr(ctx, dd_, prec=eo.DD)
    assert int(info_p.item()) == 0 and int(info_d.item()) == 0
    e_plain = oracle.orth_err(host(dp))[0]
    e_dd = oracle.orth_err(host(dd_))[0]
    assert e_plain <= 10 * n * kappa ** 2 * U  # kappa^2 u law with the Gram's gamma_n
    assert e_dd <= 1e-14
    if kappa >= 1e6:
        assert e_plain >= 1e3 * e_dd  # DD wins by orders of magnitude once kappa^2 u dominates


def test_cholqr_fp64_parity_well_conditioned(eo, ctx):
    n, k, kappa = 20_000, 6, 10.0
    x = synth.conditioned(n, k, kappa, 601)
    d = dev(x)
    rh, _, info = eo.cholqr(ctx, d, prec=eo.FP64)
    q_o, (rh_o, _), _ = oracle.cholqr(x)
    tol = 8 * kappa ** 2 * (gamma(n) + gamma(k + 1))
    assert np.max(np.abs(host(d) - q_o)) <= tol
    assert np.max(np.abs(host(rh) - rh_o)) <= tol * np.max(np.abs(rh_o))


@pytest.mark.parametrize("kappa", [1e10, 1e12])
def test_cholqr_dd_two_passes_and_auto(eo, ctx, kappa):
    n, k = 20_000, 8
    x = synth.conditioned(n, k, kappa, 700)
    d2, da = dev(x), dev(x)
    rh, rl, info = eo.cholqr(ctx, d2, passes=2, prec=eo.DD)
    assert int(info.item()) == 0
    q = host(d2)
    assert oracle.orth_err(q)[0] <= 1e-14
    assert oracle.fact_err(x, q, host(rh), host(rl)) <= 1e-14
    eo.cholqr(ctx, da, passes=0, prec=eo.DD)  # automatic: a second pass runs here
    assert np.array_equal(host(da), q)


def test_cholqr_auto_single_pass_when_well_conditioned(eo, ctx):
    x = synth.conditioned(10_000, 8, 1e3, 701)
    d1, da = dev(x), dev(x)
    eo.cholqr(ctx, d1, passes=1, prec=eo.DD)
    eo.cholqr(ctx, da, passes=0, prec=eo.DD)
    assert np.array_equal(host(d1), host(da))


def test_cholqr_special_inputs(eo, ctx):
    # orthonormal input: R = I, Q = X
    u = synth.orthonormal_basis(9000, 6, 3)
    du = oracle.orth_err(u)[0]  # the FP64 basis itself is orthonormal only to ~u
    d = dev(u)
    rh, rl, _ = eo.cholqr(ctx, d, prec=eo.DD)
    assert np.max(np.abs(host(rh) + host(rl) - np.eye(6))) <= du + 4 * U
    assert np.max(np.abs(host(d) - u)) <= du + 4 * U
    # orthogonal, unnormalized columns: R diagonal
    s = np.array([1.0, 1e3, 1e-3, 7.0, 0.5, 2.0])
    d = dev(np.asfortranarray(u * s))
    rh, _, _ = eo.cholqr(ctx, d, prec=eo.DD)
    np.testing.assert_allclose(np.diag(host(rh)), s, rtol=1e-14)


def test_cholqr_breakdown_and_nan(eo, ctx):
    x = synth.gaussian(1000, 3, 4)
    x[:, 1] = 0.0  # the second pivot is exactly zero
    d = dev(x)
    _, _, info = eo.cholqr(ctx, d, prec=eo.DD)
    assert int(info.item()) == 2
    assert np.array_equal(host(d), x)  # X is left as it was
    y = synth.gaussian(1000, 3, 5)
    y[10, 2] = np.nan
    d = dev(y)
    _, _, info = eo.cholqr(ctx, d, prec=eo.DD)
    assert int(info.item()) == -1


def test_cholqr_with_gram_from_project(eo, ctx):
    n, kv, k = 40_000, 16, 4
    v = synth.orthonormal_basis(n, kv, 71)
    y = synth.conditioned(n, k, 1e5, 72)
    yt, _, m = eo.project(ctx, dev(v), dev(y), prec=eo.DD)
    a = yt.clone().t().contiguous().t()
    eo.cholqr(ctx, yt, prec=eo.DD, M=m)
    eo.cholqr(ctx, a, prec=eo.DD)
    assert np.max(np.abs(host(yt) - host(a))) <= cholqr_tol(n, k, 1e5)
    q = host(yt)
    assert oracle.orth_err(q)[0] <= 1e-14
    # Y~ is stored in FP64: its u-sized component along V is scaled by ||Z|| ~ kappa
    assert oracle.cross_err(v, q) <= 10 * 1e5 * U * np.sqrt(k)


def test_cholqr_f32(eo, ctx):
    n, k = 30_000, 8
    x = synth.conditioned(n, k, 1e2, 80).astype(np.float32)
    d = dev(x)
    rh, _, info = eo.cholqr(ctx, d, prec=eo.F32)
    assert int(info.item()) == 0
    q = host(d).astype(np.float64)
    assert oracle.orth_err(q)[0] <= 1e-5  # FP32 storage of Q: u32 = 6e-8 per entry
    q_o, (rh_o, _), _ = oracle.cholqr(x.astype(np.float64))
    np.testing.assert_allclose(host(rh), rh_o, rtol=0, atol=1e-12 * np.max(np.abs(rh_o)))


# ----------------------------------------------------------------- SVQB

@pytest.mark.parametrize("n,k,kappa", [(20_000, 8, 1e2), (20_000, 8, 1e6), (10_001, 16, 1e7), (777, 3, 1.0)])
def test_svqb_dd_matches_oracle(eo, ctx, n, k, kappa):
    x = synth.conditioned(n, k, kappa, 800 + k)
    d = dev(x)
    zh, zl, rank = eo.svqb(ctx, d, prec=eo.DD)
    assert int(rank.item()) == k
    q_o, (zh_o, zl_o), _ = oracle.svqb(x)
    tol = cholqr_tol(n, k, kappa)
    assert np.max(np.abs(host(d) - q_o)) <= tol
    z = host(zh) + host(zl)
    assert np.max(np.abs(z - (zh_o + zl_o))) <= tol * np.max(np.abs(zh_o))
    assert np.array_equal(host(zh), host(zh).T)
    assert oracle.orth_err(host(d))[0] <= 1e-14


def svqb2_tol(n, k, kappa):
    """|Q - Q*| after two SVQB passes: the first pass's difference Q1 - Q1* =
    Q1* E (E k-by-k, within cholqr_tol) survives the second pass only as
    Q1* skew(E) (the symmetric part is what the second pass removes), plus
    the second pass's own rounding."""
    return 4 * cholqr_tol(n, k, kappa) + 8 * U


@pytest.mark.parametrize("n,k,kappa", [(20_000, 8, 1e8), (20_001, 16, 1e10), (9_000, 32, 1e9), (3_000, 4, 1e12)])
def test_svqb_dd_two_passes_match_oracle(eo, ctx, n, k, kappa):
    x = synth.conditioned(n, k, kappa, 830 + k)
    d, da = dev(x), dev(x)
    zh, zl, rank = eo.svqb(ctx, d, passes=2, prec=eo.DD)
    assert int(rank.item()) == k
    q_o, (zh_o, zl_o), rank_o = oracle.svqb(x, passes=2)
    assert rank_o == k
    tol = svqb2_tol(n, k, kappa)
    q = host(d)
    assert np.max(np.abs(q - q_o)) <= tol
    z = host(zh) + host(zl)
    assert np.max(np.abs(z - (zh_o + zl_o))) <= tol * np.max(np.abs(zh_o))
    assert oracle.orth_err(q)[0] <= 1e-14
    # the automatic pass count takes the second pass here (lambda_max / lambda_min > 1e14)
    eo.svqb(ctx, da, passes=0, prec=eo.DD)
    assert np.array_equal(host(da), q)


# ------------------------------------------------- pivoted, partial CholQR

@pytest.mark.parametrize("n,k,kappa,passes", [(20_000, 8, 1e4, 1), (20_001, 16, 1e8, 2), (5_000, 5, 1.0, 1),
                                              (9_000, 32, 1e6, 2)])
def test_cholqr_piv_matches_oracle(eo, ctx, n, k, kappa, passes):
    x = synth.conditioned(n, k, kappa, 840 + k)
    d = dev(x)
    rh, rl, perm, rank, info = eo.cholqr_piv(ctx, d, passes=passes, prec=eo.DD)
    q_o, perm_o, rank_o, (rh_o, rl_o), info_o = oracle.cholqr_piv(x, tol=k * U2, passes=passes)
    assert int(info.item()) == 0 == info_o
    assert int(rank.item()) == rank_o == k
    assert list(perm.cpu().numpy()) == list(perm_o)
    tol = (4 if passes == 2 else 1) * cholqr_tol(n, k, kappa)
    q = host(d)
    assert np.max(np.abs(q - q_o)) <= tol
    r = host(rh) + host(rl)
    assert np.max(np.abs(r - (rh_o + rl_o))) <= tol * np.max(np.abs(rh_o))
    assert oracle.orth_err(q)[0] <= 1e-14
    assert oracle.fact_err(np.asfortranarray(x[:, perm_o]), q, host(rh), host(rl)) <= 1e-14


def test_cholqr_piv_ties_rank_and_special_inputs(eo, ctx):
    # orthogonal columns with equal norms: exact ties, broken by the lowest index as in the oracle
    u = synth.hadamard_basis(4096, 5, 841)
    s = np.array([0.5, 8.0, 2.0, 8.0, 0.25])
    d = dev(np.asfortranarray(u * s))
    rh, rl, perm, rank, info = eo.cholqr_piv(ctx, d, prec=eo.DD)
    assert list(perm.cpu().numpy()) == [1, 3, 2, 0, 4] and int(rank.item()) == 5
    assert np.array_equal(host(rh), np.diag(s[[1, 3, 2, 0, 4]])) and np.array_equal(host(d), u[:, [1, 3, 2, 0, 4]])
    # rank deficiency: the dependent columns are cut and their columns of Q are zero
    g = synth.rng(842)
    a, b = g.standard_normal((30_000, 1)), g.standard_normal((30_000, 1))
    x = np.asfortranarray(np.hstack([a, b, a + b, 3.0 * b, g.standard_normal((30_000, 1))]))
    d = dev(x)
    _, _, perm, rank, info = eo.cholqr_piv(ctx, d, prec=eo.DD, tol=1e-20)
    q_o, perm_o, rank_o, _, _ = oracle.cholqr_piv(x, tol=1e-20)
    assert int(rank.item()) == rank_o == 3 and list(perm.cpu().numpy()) == list(perm_o)
    q = host(d)
    assert not np.any(q[:, 3:])
    assert np.max(np.abs(q - q_o)) <= cholqr_tol(30_000, 3, 10.0)
    # NaN: info -1, X unchanged; the automatic pass count matches passes = 2 at kappa = 1e9
    y = synth.gaussian(1000, 3, 843)
    y[5, 1] = np.nan
    d = dev(y)
    _, _, _, rank, info = eo.cholqr_piv(ctx, d, prec=eo.DD)
    assert int(info.item()) == -1 and int(rank.item()) == -1
    assert np.array_equal(host(d), y, equal_nan=True)
    x = synth.conditioned(8000, 6, 1e9, 844)
    d2, da = dev(x), dev(x)
    eo.cholqr_piv(ctx, d2, passes=2, prec=eo.DD)
    eo.cholqr_piv(ctx, da, passes=0, prec=eo.DD)
    assert np.array_equal(host(d2), host(da))


def test_cholqr_piv_fp64(eo, ctx):
    n, k = 20_000, 6
    x = synth.conditioned(n, k, 10.0, 845)
    d = dev(x)
    rh, _, perm, rank, info = eo.cholqr_piv(ctx, d, prec=eo.FP64)
    q_o, perm_o, rank_o, (rh_o, _), _ = oracle.cholqr_piv(x, tol=k * U)
    assert list(perm.cpu().numpy()) == list(perm_o) and int(rank.item()) == rank_o == k
    tol = 8 * 100 * (gamma(n) + gamma(k + 1))
    assert np.max(np.abs(host(d) - q_o)) <= tol


def test_svqb_rank_deficient(eo, ctx):
    x = synth.gaussian(5000, 4, 90)
    x[:, 2] = 0.0
    d = dev(x)
    _, _, rank = eo.svqb(ctx, d, prec=eo.DD)
    assert int(rank.item()) == 3
    q = host(d)
    # Q spans the range of X: Q^T Q is the orthogonal projector onto it
    p = q.T @ q
    assert np.max(np.abs(p @ p - p)) < 1e-13
    assert abs(np.trace(p) - 3.0) < 1e-13


def test_svqb_orthonormal_input_is_fixed(eo, ctx):
    u = synth.orthonormal_basis(4000, 5, 91)
    du = oracle.orth_err(u)[0]
    d = dev(u)
    zh, zl, _ = eo.svqb(ctx, d, prec=eo.DD)
    assert np.max(np.abs(host(zh) + host(zl) - np.eye(5))) <= du + 4 * U
    assert np.max(np.abs(host(d) - u)) <= du + 8 * U


# ------------------------------------------- rotated SVQB (Z = D U Lambda^{-1/2})

def _rot_separated(x):
    """True when D M D has well-separated eigenvalues and every eigenvector a
    clear largest entry, so that the order and signs are fixed far above the
    rounding of either side."""
    m = x.T @ x
    d = 1 / np.sqrt(np.diag(m))
    lam, u = np.linalg.eigh(d[:, None] * m * d[None, :])
    au = np.sort(np.abs(u), axis=0)
    return np.min(np.diff(lam) / lam[1:]) > 1e-3 and np.min((au[-1] - au[-2]) / au[-1]) > 1e-4


@pytest.mark.parametrize("n,k,kappa", [(20_000, 8, 1e2), (10_001, 16, 1e5), (4_097, 40, 1e3), (9_000, 64, 1e4),
                                       (20_000, 8, 1e7)])
def test_svqb_rotated_dd_matches_oracle(eo, ctx, n, k, kappa):
    x = synth.conditioned(n, k, kappa, 900 + k)
    assert _rot_separated(x)
    d = dev(x)
    zh, zl, rank = eo.svqb_rotated(ctx, d, prec=eo.DD)
    assert int(rank.item()) == k
    q_o, (zh_o, zl_o), rank_o = oracle.svqb_rotated(x)
    assert rank_o == k
    tol = cholqr_tol(n, k, kappa)
    q = host(d)
    assert np.max(np.abs(q - q_o)) <= tol
    z = host(zh) + host(zl)
    assert np.max(np.abs(z - (zh_o + zl_o))) <= tol * np.max(np.abs(zh_o))
    assert oracle.orth_err(q)[0] <= 1e-14


def test_svqb_rotated_given_m_and_fp64(eo, ctx):
    n, k = 20_000, 12
    x = synth.conditioned(n, k, 1e3, 950)
    assert _rot_separated(x)
    mh, ml = oracle.gram(x)
    q_o, (zh_o, zl_o), _ = oracle.svqb_rotated(x, m=(mh, ml))
    d = dev(x)
    zh, zl, rank = eo.svqb_rotated(ctx, d, prec=eo.DD, M=(dev(mh), dev(ml)))
    assert int(rank.item()) == k
    assert np.max(np.abs(host(d) - q_o)) <= cholqr_tol(n, k, 1e3)
    # FP64: Gram, Jacobi and update in FP64 (M to n u |X|^2, the eigenvectors to u / relgap)
    d = dev(x)
    zh, _, rank = eo.svqb_rotated(ctx, d, prec=eo.FP64)
    assert int(rank.item()) == k
    assert np.max(np.abs(host(d) - q_o)) <= 1e-9
    assert oracle.orth_err(host(d))[0] <= 1e-9


def test_svqb_rotated_degenerate_and_special_inputs(eo, ctx):
    # exactly orthogonal columns (Hadamard, power-of-two scales): D M D = I with
    # no rotation, ties kept in index order, so Z = D and Q the unit columns exactly
    h = synth.hadamard_basis(4096, 4, 951)
    s = np.array([2.0, 0.25, 8.0, 1.0])
    x = np.asfortranarray(h * s)
    q_o, (zh_o, zl_o), _ = oracle.svqb_rotated(x)
    d = dev(x)
    zh, zl, rank = eo.svqb_rotated(ctx, d, prec=eo.DD)
    assert int(rank.item()) == 4
    assert np.array_equal(host(zh), zh_o) and np.array_equal(host(zl), zl_o)
    assert np.array_equal(host(d), h) and np.array_equal(q_o, h)
    # a zero column: eigenvalue 0 first in the order, its column of Z and Q zero
    x0 = x.copy(order="F")
    x0[:, 2] = 0.0
    d = dev(x0)
    zh, zl, rank = eo.svqb_rotated(ctx, d, prec=eo.DD)
    q_o, _, rank_o = oracle.svqb_rotated(x0)
    assert int(rank.item()) == rank_o == 3
    assert np.array_equal(host(d), q_o) and not np.any(host(zh)[:, 0])
    # a dependent column: its eigenvalue (at the rounding level) is cut
    g = synth.rng(952)
    a, b = g.standard_normal((30_000, 1)), g.standard_normal((30_000, 1))
    x = np.asfortranarray(np.hstack([a, b, a - 2.0 * b, g.standard_normal((30_000, 2))]))
    d = dev(x)
    _, _, rank = eo.svqb_rotated(ctx, d, prec=eo.DD, tol=1e-20)
    assert int(rank.item()) == 4
    q = host(d)
    assert not np.any(q[:, 0]) and oracle.orth_err(np.asfortranarray(q[:, 1:]))[0] <= 1e-14
    # nearly orthonormal input: D M D = I + O(u), order and vectors set by
    # rounding, so only what is unique is compared: the span and Z^T M Z = I
    x = synth.conditioned(777, 3, 1.0, 953)
    d = dev(x)
    zh, zl, rank = eo.svqb_rotated(ctx, d, prec=eo.DD)
    q = host(d)
    assert int(rank.item()) == 3 and oracle.orth_err(q)[0] <= 1e-14
    assert np.max(np.abs(q @ q.T - x @ x.T)) <= 1e-14
    # NaN: rank -1 and X left as it was
    y = synth.gaussian(1000, 3, 954)
    y[7, 2] = np.nan
    d = dev(y)
    _, _, rank = eo.svqb_rotated(ctx, d, prec=eo.DD)
    assert int(rank.item()) == -1
    assert np.array_equal(host(d), y, equal_nan=True)


# ------------------------------------------------------------ arguments

def test_invalid_arguments_are_rejected(eo, ctx):
    torch = torch_mod()
    x = dev(synth.gaussian(100, 3, 1))
    L = eo.lib()
    h = ctx.h
    g = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    assert L.eo_gram(h, 100, 0, x.data_ptr(), 100, 0, None, 100, g.data_ptr(), None, 3, 1) == eo.EINVAL
    assert L.eo_gram(h, 100, 65, x.data_ptr(), 100, 65, None, 100, g.data_ptr(), None, 65, 1) == eo.EINVAL
    assert L.eo_gram(h, 100, 3, x.data_ptr(), 99, 3, None, 99, g.data_ptr(), None, 3, 1) == eo.EINVAL
    assert L.eo_gram(h, 100, 3, None, 100, 3, None, 100, g.data_ptr(), None, 3, 1) == eo.EINVAL
    assert L.eo_gram(h, 100, 3, x.data_ptr(), 100, 3, None, 100, g.data_ptr(), None, 3, 7) == eo.EINVAL
    assert b"precision" in L.eo_last_error(h)
    assert L.eo_cholqr(h, 100, 3, x.data_ptr(), 100, None, None, 3, None, None, 3, 3, 1, None) == eo.EINVAL
    assert L.eo_project(h, 100, 3, x.data_ptr(), 100, 3, x.data_ptr(), 100, x.data_ptr(), 100, None, None, 3,
                        None, None, 3, eo.F32) == eo.EUNSUPPORTED


@pytest.mark.parametrize("k", [24, 32, 64])
def test_svqb_update_engines_agree(eo, ctx, monkeypatch, k):
    """SVQB's full Z with k > 16 (24 and 32: one tensor-core pass over two output
    blocks; 64: groups of 16 output columns) vs integer limbs, both against the oracle."""
    n, kappa = 12_000, 1e4
    x = synth.conditioned(n, k, kappa, 83 + k)
    qs = {}
    for engine in ("int", "umma"):
        monkeypatch.setenv("EO_DD_ROW_ENGINE", engine)
        d = dev(x)
        eo.svqb(ctx, d, passes=1, prec=eo.DD)
        qs[engine] = host(d)
    q_o, _, _ = oracle.svqb(x, passes=1)
    tol = cholqr_tol(n, k, kappa)
    for engine, q in qs.items():
        assert np.max(np.abs(q - q_o)) <= tol, engine
        assert oracle.orth_err(q)[0] <= 1e-14, engine


@pytest.mark.parametrize("n,kx,ky", [(5001, 16, None), (4097, 32, None), (2049, 64, 64), (3001, 64, 8),
                                     (70_001, 16, 16), (999, 20, None)])
def test_gram_umma_direct_loads_against_oracle(eo, ctx, monkeypatch, n, kx, ky):
    """Packed blocks with odd n (leading dimension n): not addressable by TMA,
    so the tensor-core engine's converters copy their own items."""
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", "umma")
    x = synth.gaussian(n, kx, 300 + kx)
    y = None if ky is None else synth.gaussian(n, ky, 400 + ky)
    gh, gl = eo.gram(ctx, dev(x), None if y is None else dev(y), prec=eo.DD)
    rh, rl = oracle.gram(x, y)
    assert np.all(dd_err(host(gh), host(gl), rh, rl) <= dd_gram_tol(x, x if y is None else y, rh, 1))


@pytest.mark.parametrize("kx,ky", [(16, None), (64, 16), (32, None)])
def test_gram_umma_direct_equals_tma(eo, ctx, monkeypatch, kx, ky):
    """The same values with an even (TMA) and an odd (direct copies) leading
    dimension: the same panels, chunks and digits, so bitwise the same result."""
    monkeypatch.setenv("EO_DD_GRAM_ENGINE", "umma")
    torch = torch_mod()
    n = 40_000
    x = synth.conditioned(n, kx, 1e6, 500 + kx)
    y = None if ky is None else synth.gaussian(n, ky, 501)

    def odd(a):
        buf = synth.with_ld(a, n + 1, fill=np.nan)
        return torch.from_numpy(np.ascontiguousarray(buf.T)).cuda().t()[:n, :]

    g1 = eo.gram(ctx, dev(x), None if y is None else dev(y), prec=eo.DD)
    xo = odd(x)
    assert xo.stride(1) == n + 1
    g2 = eo.gram(ctx, xo, None if y is None else odd(y), prec=eo.DD)
    assert np.array_equal(host(g1[0]), host(g2[0])) and np.array_equal(host(g1[1]), host(g2[1]))
