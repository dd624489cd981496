"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test checks the binary128 oracle against exact rational arithmetic
(``fractions.Fraction``), a closed form, an invariant of the factorization,
or a library routine on a case where that routine is accurate enough, so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
import synth

U64 = 2.0 ** -53


def fr(a):
    return [[F(float(a[i, j])) for j in range(a.shape[1])] for i in range(a.shape[0])]


def dd_fr(hi, lo, i, j):
    return F(float(hi[i, j])) + F(float(lo[i, j]))


def exact_gram(x, y):
    xs, ys = fr(x), fr(y)
    n = x.shape[0]
    return [[sum((xs[r][i] * ys[r][j] for r in range(n)), F(0)) for j in range(y.shape[1])]
            for i in range(x.shape[1])]


def abs_gram(x, y):
    return np.abs(x).T @ np.abs(y)


def wide_range(g, n, k):
    """Entries with random signs and exponents spread over 2^-30 .. 2^30."""
    m = g.standard_normal((n, k))
    e = g.integers(-30, 30, size=(n, k))
    return np.asfortranarray(np.ldexp(m, e))


# ------------------------------------------------------------------ Gram

@pytest.mark.parametrize("n,kx,ky", [(1, 1, 1), (7, 2, 3), (33, 3, 2), (64, 4, 4)])
def test_gram_matches_exact_rational_sum(n, kx, ky):
    g = synth.rng(11 + n)
    x = wide_range(g, n, kx)
    y = wide_range(g, n, ky)
    hi, lo = oracle.gram(x, y)
    ex = exact_gram(x, y)
    bound = abs_gram(x, y)
    for i in range(kx):
        for j in range(ky):
            err = abs(dd_fr(hi, lo, i, j) - ex[i][j])
            # n roundings in binary128 plus the split into hi + lo
            tol = F((n + 1) * 2.0 ** -112) * F(float(bound[i, j])) + F(2.0 ** -105) * abs(ex[i][j])
            assert err <= tol, (i, j, float(err), float(tol))
            assert hi[i, j] == float(ex[i][j]) or abs(F(float(hi[i, j])) - ex[i][j]) <= F(U64) * abs(ex[i][j]) * 1.0001


def test_gram_symmetric_default_and_transpose():
    g = synth.rng(5)
    x = wide_range(g, 40, 3)
    y = wide_range(g, 40, 5)
    hxy, _ = oracle.gram(x, y)
    hyx, _ = oracle.gram(y, x)
    assert np.array_equal(hxy, hyx.T)
    hs, ls = oracle.gram(x)
    hx, lx = oracle.gram(x, x)
    assert np.array_equal(hs, hx) and np.array_equal(ls, lx)
    assert np.array_equal(hs, hs.T)


def test_gram_f32_matches_exact():
    g = synth.rng(3)
    x = g.standard_normal((50, 3)).astype(np.float32)
    hi, lo = oracle.gram_f32(x)
    ex = exact_gram(x.astype(np.float64), x.astype(np.float64))
    for i in range(3):
        for j in range(3):
            # FP32 products are exact in 48 bits, so the binary128 sum of 50 of them is exact
            assert dd_fr(hi, lo, i, j) == ex[i][j]


def test_gram_cancellation_is_resolved():
    # x = [1, 2^-100, -1], y = [1, 1, 1]: every partial sum is exact in binary128
    # (1 + 2^-100 needs 101 bits), FP64 would return 0
    x = np.array([[1.0], [2.0 ** -100], [-1.0]])
    y = np.ones((3, 1))
    hi, lo = oracle.gram(x, y)
    assert hi[0, 0] == 2.0 ** -100 and lo[0, 0] == 0.0


# ------------------------------------------------------------ projection

def test_project_matches_exact_rational():
    g = synth.rng(21)
    n, kv, k = 24, 3, 2
    v = g.standard_normal((n, kv))
    y = g.standard_normal((n, k))
    yt, (chi, clo), (mhi, mlo) = oracle.project(v, y)
    vs, ys = fr(v), fr(y)
    c = [[sum((vs[r][i] * ys[r][j] for r in range(n)), F(0)) for j in range(k)] for i in range(kv)]
    for i in range(kv):
        for j in range(k):
            assert abs(dd_fr(chi, clo, i, j) - c[i][j]) <= F(2.0 ** -104) * (abs(c[i][j]) + 1)
    for r in range(n):
        for j in range(k):
            ex = ys[r][j] - sum((vs[r][i] * c[i][j] for i in range(kv)), F(0))
            # rounded once; the binary128 C perturbs the exact value far below one FP64 ulp
            assert abs(F(float(yt[r, j])) - ex) <= F(0.5 * U64 * 2) * abs(ex) * F(1.000001) + F(2.0 ** -200)
    ex_m = exact_gram(yt, yt)
    for i in range(k):
        for j in range(k):
            assert abs(dd_fr(mhi, mlo, i, j) - ex_m[i][j]) <= F(2.0 ** -104) * (abs(ex_m[i][j]) + 1)


def test_project_apply_matches_exact_rational():
    g = synth.rng(22)
    n, kv, k = 17, 4, 3
    v = wide_range(g, n, kv)
    y = wide_range(g, n, k)
    chi = g.standard_normal((kv, k))
    clo = chi * 2.0 ** -60 * g.standard_normal((kv, k))  # a genuine low part
    yt = oracle.project_apply(v, y, chi, clo)
    vs, ys = fr(v), fr(y)
    for r in range(n):
        for j in range(k):
            ex = ys[r][j] - sum((vs[r][i] * dd_fr(chi, clo, i, j) for i in range(kv)), F(0))
            # round-to-nearest of the exact value (float(Fraction) rounds correctly); binary128
            # sums of four products move it by far less than the FP64 half-ulp
            assert abs(F(float(yt[r, j])) - ex) <= abs(F(float(ex)) - ex) + F(2.0 ** -100) * (
                abs(ys[r][j]) + sum((abs(vs[r][i] * dd_fr(chi, clo, i, j)) for i in range(kv)), F(0)))


def test_project_apply_integer_inputs_and_consistency():
    g = synth.rng(23)
    n, kv, k = 300, 6, 4
    vi = g.integers(-1000, 1001, size=(n, kv))
    ci = g.integers(-1000, 1001, size=(kv, k))
    yi = g.integers(-2 ** 40, 2 ** 40, size=(n, k))
    yt = oracle.project_apply(vi.astype(np.float64), yi.astype(np.float64), ci.astype(np.float64))
    assert np.array_equal(yt, (yi - vi @ ci).astype(np.float64))
    # with the C that eoq_project computes, the result is eoq_project's own Y~
    v = synth.orthonormal_basis(500, 5, 24)
    y = synth.conditioned(500, 3, 1e4, 25)
    yt_p, (chi, clo), _ = oracle.project(v, y)
    yt_a = oracle.project_apply(v, y, chi, clo)
    assert np.max(np.abs(yt_a - yt_p)) <= 2 * U64 * np.max(np.abs(y))


def test_project_special_cases():
    v = synth.orthonormal_basis(200, 4, 7)
    a = synth.rng(8).standard_normal((4, 2))
    # Y in span(V): the projection leaves a residual at the FP64 rounding level of Y
    y_in = np.asfortranarray(v @ a)
    yt, (chi, _), _ = oracle.project(v, y_in)
    assert np.max(np.abs(yt)) < 1e-14 * np.max(np.abs(y_in))
    np.testing.assert_allclose(chi, a, rtol=0, atol=1e-14)
    # Y orthogonal to V (built from the complement): Y~ = Y and C ~ 0
    full = synth.orthonormal_basis(200, 6, 7)
    y_perp = np.asfortranarray(full[:, 4:6] * 3.0)
    yt2, (c2, _), _ = oracle.project(full[:, :4], y_perp)
    assert np.max(np.abs(c2)) < 1e-14
    np.testing.assert_allclose(yt2, y_perp, rtol=0, atol=1e-14)


# -------------------------------------------------------------- Cholesky

def spd(k, kappa, seed):
    x = synth.conditioned(4 * k + 8, k, kappa, seed)
    return oracle.gram(x)


def test_cholesky_diagonal_closed_form():
    d = np.array([4.0, 2.0, 9.0, 1e-8])
    m = np.diag(d)
    r_hi, r_lo, info = oracle.cholesky(m)
    assert info == 0
    for i in range(4):
        assert r_hi[i, i] == np.sqrt(d[i])  # IEEE sqrt is correctly rounded; so is hi
        assert abs((F(float(r_hi[i, i])) + F(float(r_lo[i, i]))) ** 2 - F(float(d[i]))) <= F(2.0 ** -104) * F(float(d[i]))
    assert np.count_nonzero(r_hi - np.diag(np.diag(r_hi))) == 0


@pytest.mark.parametrize("k,kappa", [(2, 10.0), (5, 1e3), (8, 1e6)])
def test_cholesky_reconstructs_m(k, kappa):
    m_hi, m_lo = spd(k, kappa, 40 + k)
    r_hi, r_lo, info = oracle.cholesky(m_hi, m_lo)
    assert info == 0
    assert np.all(np.diag(r_hi) > 0)
    assert np.all(np.tril(r_hi, -1) == 0)
    for i in range(k):
        for j in range(i, k):
            rtr = sum(((F(float(r_hi[l, i])) + F(float(r_lo[l, i]))) * (F(float(r_hi[l, j])) + F(float(r_lo[l, j])))
                       for l in range(k)), F(0))
            mij = dd_fr(m_hi, m_lo, i, j)
            scale = F(float(np.sqrt(m_hi[i, i] * m_hi[j, j])))
            assert abs(rtr - mij) <= F(2.0 ** -100) * scale


def test_cholesky_agrees_with_lapack_when_well_conditioned():
    m_hi, m_lo = spd(6, 1e2, 77)
    r_hi, _, info = oracle.cholesky(m_hi, m_lo)
    assert info == 0
    lap = np.linalg.cholesky(m_hi + m_lo).T
    np.testing.assert_allclose(r_hi, lap, rtol=1e-12, atol=1e-13 * np.max(np.abs(lap)))


def test_cholesky_breakdown_reports_column():
    assert oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))[2] == 2
    assert oracle.cholesky(np.array([[0.0, 0.0], [0.0, 1.0]]))[2] == 1
    assert oracle.cholesky(np.array([[-1.0]]))[2] == 1
    # exactly singular rank-one matrix x x^T with x = [1, 2, 3]: pivot 2 is exactly zero
    x = np.array([1.0, 2.0, 3.0])
    assert oracle.cholesky(np.outer(x, x))[2] == 2


def test_triinv_is_inverse():
    m_hi, m_lo = spd(6, 1e4, 91)
    r_hi, r_lo, _ = oracle.cholesky(m_hi, m_lo)
    z_hi, z_lo = oracle.triinv(r_hi, r_lo)
    assert np.all(np.tril(z_hi, -1) == 0)
    k = 6
    for i in range(k):
        for j in range(k):
            s = sum(((F(float(r_hi[i, l])) + F(float(r_lo[i, l]))) * (F(float(z_hi[l, j])) + F(float(z_lo[l, j])))
                     for l in range(k)), F(0))
            assert abs(s - (1 if i == j else 0)) <= F(2.0 ** -98) * F(1e4)
    np.testing.assert_allclose(z_hi, np.linalg.inv(r_hi + r_lo), rtol=1e-10, atol=1e-12 * np.max(np.abs(z_hi)))


# ---------------------------------------------------------------- Jacobi

def test_jacobi_2x2_closed_form():
    import mpmath as mp
    mp.mp.prec = 200
    a, b, c = 2.0, 0.75, -1.25
    (lh, ll), u = oracle.jacobi(np.array([[a, b], [b, c]]))
    lam = sorted(mp.mpf(h) + mp.mpf(l) for h, l in zip(lh, ll))
    mid = (mp.mpf(a) + c) / 2
    rad = mp.sqrt(((mp.mpf(a) - c) / 2) ** 2 + mp.mpf(b) ** 2)
    assert abs(lam[0] - (mid - rad)) < mp.mpf(2) ** -104
    assert abs(lam[1] - (mid + rad)) < mp.mpf(2) ** -104


@pytest.mark.parametrize("k,kappa", [(3, 10.0), (8, 1e6), (16, 1e12)])
def test_jacobi_invariants(k, kappa):
    m_hi, m_lo = spd(k, kappa, 300 + k)
    (lh, ll), u = oracle.jacobi(m_hi, m_lo)
    # eigenvectors orthonormal to FP64 rounding (U is returned rounded to FP64)
    assert np.max(np.abs(u.T @ u - np.eye(k))) < 10 * k * U64
    # eigenvalues equal the squared singular values built into the generator
    lam = np.sort(lh + ll)[::-1]
    sig = synth.logspace_sigma(k, kappa)
    ref = sig ** 2
    assert np.max(np.abs(lam - ref) / ref) < 1e3 * U64 * kappa  # FP64 input X perturbs sigma_min by ~u*kappa
    # library check where the library is accurate
    np.testing.assert_allclose(np.sort(lh), np.linalg.eigvalsh(m_hi + m_lo), rtol=0,
                               atol=50 * k * U64 * np.max(lh))


def test_jacobi_diagonal_is_fixed_point():
    d = np.array([3.0, 1.0, 2.0])
    (lh, ll), u = oracle.jacobi(np.diag(d))
    assert np.array_equal(lh, d) and np.array_equal(u, np.eye(3))


# ------------------------------------------------------------- SVQB's Z

@pytest.mark.parametrize("k,kappa", [(2, 1.0), (6, 1e3), (8, 1e8)])
def test_svqb_z_is_inverse_square_root(k, kappa):
    import mpmath as mp
    mp.mp.prec = 240
    m_hi, m_lo = spd(k, kappa, 500 + k)
    z_hi, z_lo, rank = oracle.svqb_z(m_hi, m_lo)
    assert rank == k
    assert np.array_equal(z_hi, z_hi.T)
    Z = mp.matrix(k, k)
    M = mp.matrix(k, k)
    for i in range(k):
        for j in range(k):
            Z[i, j] = mp.mpf(z_hi[i, j]) + mp.mpf(z_lo[i, j])
            M[i, j] = mp.mpf(m_hi[i, j]) + mp.mpf(m_lo[i, j])
    E = Z.T * M * Z - mp.eye(k)
    # binary128 eigen-solve of M with condition kappa^2: error ~ k * kappa^2 * 2^-113
    assert max(abs(E[i, j]) for i in range(k) for j in range(k)) < mp.mpf(2) ** -108 * k * max(kappa, 1e4) ** 2


def test_svqb_z_identity_and_library():
    z_hi, z_lo, rank = oracle.svqb_z(np.eye(4))
    assert rank == 4 and np.array_equal(z_hi, np.eye(4)) and not np.any(z_lo)
    import scipy.linalg as sl
    m_hi, m_lo = spd(5, 30.0, 61)
    z_hi, _, _ = oracle.svqb_z(m_hi, m_lo)
    ref = np.linalg.inv(np.real(sl.sqrtm(m_hi + m_lo)))
    np.testing.assert_allclose(z_hi, ref, rtol=1e-11, atol=1e-12 * np.max(np.abs(ref)))


def test_svqb_z_rank_cut():
    z_hi, _, rank = oracle.svqb_z(np.diag([1.0, 1e-20, 4.0]), tol=1e-10)
    assert rank == 2
    np.testing.assert_array_equal(z_hi, np.diag([1.0, 0.0, 0.5]))


# ------------------------------------------------------- CholQR / SVQB

@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e12])
def test_cholqr_invariants(kappa):
    n, k = 300, 6
    x = synth.conditioned(n, k, kappa, 900)
    q, (r_hi, r_lo), info = oracle.cholqr(x, passes=1)
    assert info == 0
    two, fro, mx = oracle.orth_err(q)
    # binary128 CholQR loses orthogonality like kappa^2 * u_128 (u_128 = 2^-113);
    # on top of that Q is rounded once to FP64
    assert two < 4 * k * U64 + kappa ** 2 * 2.0 ** -111
    if kappa >= 1e12:
        assert two > kappa ** 2 * 2.0 ** -120  # the kappa^2 law of the quad arithmetic is visible
    assert oracle.fact_err(x, q, r_hi, r_lo) < 4 * U64 * np.sqrt(k)
    assert np.all(np.diag(r_hi) > 0) and np.all(np.tril(r_hi, -1) == 0)
    sv = np.linalg.svd(r_hi + r_lo, compute_uv=False)
    sig = synth.logspace_sigma(k, kappa)
    assert np.max(np.abs(sv - sig)) < 1e2 * U64 * np.sqrt(n)


def test_cholqr_k1_is_normalization():
    g = synth.rng(1)
    x = g.standard_normal((37, 1))
    q, (r_hi, r_lo), info = oracle.cholqr(x)
    ss = sum((F(float(v)) ** 2 for v in x[:, 0]), F(0))
    r = F(float(r_hi[0, 0])) + F(float(r_lo[0, 0]))
    assert abs(r * r - ss) <= F(2.0 ** -104) * ss
    for i in range(37):
        ex = F(float(x[i, 0])) / r
        assert abs(F(float(q[i, 0])) - ex) <= F(U64) * abs(ex) * F(1.0000001)


def test_cholqr_orthonormal_and_orthogonal_inputs():
    u = synth.orthonormal_basis(100, 5, 3)
    q, (r_hi, _), info = oracle.cholqr(u)
    assert info == 0
    np.testing.assert_allclose(r_hi, np.eye(5), rtol=0, atol=1e-15)
    np.testing.assert_allclose(q, u, rtol=0, atol=4 * U64)
    s = np.array([1.0, 1e3, 1e-3, 7.0, 0.5])
    q2, (r2, _), _ = oracle.cholqr(np.asfortranarray(u * s))
    np.testing.assert_allclose(np.diag(r2), s, rtol=1e-14)
    off = r2 - np.diag(np.diag(r2))
    assert np.max(np.abs(off)) < 1e-14 * np.max(s)


def test_cholqr_two_passes_and_given_gram():
    x = synth.conditioned(200, 4, 1e6, 17)
    q1, (r1h, r1l), _ = oracle.cholqr(x, passes=1)
    q2, (r2h, r2l), _ = oracle.cholqr(x, passes=2)
    assert oracle.fact_err(x, q2, r2h, r2l) < 8 * U64
    assert oracle.orth_err(q2)[0] < 8 * U64
    m = oracle.gram(x)
    q3, (r3h, _), _ = oracle.cholqr(x, passes=1, m=m)
    assert np.array_equal(q3, q1) and np.array_equal(r3h, r1h)


def test_cholqr_breakdown_leaves_x():
    x = np.asfortranarray(np.ones((10, 2)))  # exactly rank one
    q, _, info = oracle.cholqr(x)
    assert info == 2
    assert np.array_equal(q, x)


@pytest.mark.parametrize("kappa", [1.0, 1e6, 1e10])
def test_svqb_invariants(kappa):
    x = synth.conditioned(250, 5, kappa, 4242)
    q, (z_hi, z_lo), rank = oracle.svqb(x)
    assert rank == 5
    assert oracle.orth_err(q)[0] < 20 * U64 + kappa ** 2 * 2.0 ** -111  # same kappa^2 u_128 law
    assert np.array_equal(z_hi, z_hi.T)
    # X Z = Q (the update is the only step after Z)
    np.testing.assert_allclose(x @ (z_hi + z_lo), q, rtol=0, atol=1e-12 * kappa * np.max(np.abs(q)))


def test_svqb_orthogonal_columns_give_diagonal_z():
    u = synth.orthonormal_basis(80, 3, 9)
    s = np.array([2.0, 0.25, 8.0])
    q, (z_hi, _), rank = oracle.svqb(np.asfortranarray(u * s))
    np.testing.assert_allclose(z_hi, np.diag(1 / s), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(q, u, rtol=0, atol=8 * U64)


# --------------------------------------------------------------- measures

def test_orth_err_closed_forms():
    q = np.array([[1.0], [2.0 ** -20]])  # Q^T Q - I = 2^-40
    two, fro, mx = oracle.orth_err(q)
    assert two == 2.0 ** -40 and fro == 2.0 ** -40 and mx == 2.0 ** -40
    d1, d2 = 2.0 ** -10, -(2.0 ** -12)
    q2 = np.diag([1 + d1, 1 + d2])
    e1, e2 = 2 * d1 + d1 * d1, 2 * d2 + d2 * d2
    two, fro, mx = oracle.orth_err(q2)
    assert two == max(abs(e1), abs(e2))
    assert abs(fro - np.hypot(e1, e2)) <= U64 * fro
    # a rotation-like off-diagonal perturbation: E = [[0, e],[e, 0]] has 2-norm |e|
    c = 2.0 ** -15
    q3 = np.array([[1.0, c], [0.0, 1.0]])  # Q^T Q = [[1, c], [c, 1 + c^2]]
    two, fro, mx = oracle.orth_err(q3)
    lam = abs(c * c / 2) + np.sqrt((c * c / 2) ** 2 + c * c)
    assert abs(two - lam) <= 4 * U64 * lam


def test_cross_err_and_fact_err_closed_forms():
    w = np.zeros((4, 1)); w[0, 0] = 1.0
    q = np.array([[0.25, -3.0], [1.0, 0.0], [0.0, 4.0], [0.0, 0.0]])
    assert oracle.cross_err(w, q) == np.hypot(0.25, 3.0)
    x = np.array([[3.0], [4.0]])
    qq = np.array([[0.375], [0.5]])  # exact binary fractions: Q R = X for R = 8
    assert oracle.fact_err(x, qq, np.array([[8.0]])) == 0.0
    # R = 8.5: X - Q R = [-0.1875, -0.25], norm 0.3125 = ||X|| / 16
    assert oracle.fact_err(x, qq, np.array([[8.5]])) == 0.0625


def test_hadamard_basis_is_exactly_orthonormal():
    w = synth.hadamard_basis(64, 10, 3)
    g = w.T @ w  # every product is +-1/64 and every partial sum is exact in FP64
    assert np.array_equal(g, np.eye(10))
    assert set(np.unique(np.abs(w))) == {0.125}
    hi, lo = oracle.gram(w)
    assert np.array_equal(hi, np.eye(10)) and not np.any(lo)


# ------------------------------------------------------ B-inner products
# With B = diag(d) and every d a power of four, sqrt(d) is a power of two, so
# scaling by it commutes with every rounding: the B-orthogonalization of X
# (given P = B X) must equal D^{-1/2} times the Euclidean one of sqrt(D) X,
# bit for bit, with the same R (or Z).  B = I must reproduce the Euclidean
# functions exactly.  These tie the B-variants to the independently pinned
# Euclidean oracle (and would fail for a transposed X^T P, a missing update
# of P, or a wrong symmetrization).

def pow4_diag(n, seed):
    g = np.random.default_rng(seed)
    return 4.0 ** g.integers(-3, 4, n).astype(np.float64)


@pytest.mark.parametrize("passes", [1, 2])
def test_cholqr_b_identity_is_cholqr(passes):
    x = synth.conditioned(500, 6, 1e5, 61)
    q, bq, (rh, rl), info = oracle.cholqr_b(x, x, passes=passes)
    q2, (rh2, rl2), info2 = oracle.cholqr(x, passes=passes)
    assert info == info2 == 0
    assert np.array_equal(q, q2) and np.array_equal(bq, q2)
    assert np.array_equal(rh, rh2) and np.array_equal(rl, rl2)


@pytest.mark.parametrize("passes", [1, 2])
def test_cholqr_b_diagonal_is_scaled_cholqr(passes):
    n, k = 700, 5
    x = synth.conditioned(n, k, 1e6, 62)
    d = pow4_diag(n, 63)
    s = np.sqrt(d)
    q, bq, (rh, rl), info = oracle.cholqr_b(x, d[:, None] * x, passes=passes)
    qs, (rhs, rls), infos = oracle.cholqr(s[:, None] * x, passes=passes)
    assert info == infos == 0
    assert np.array_equal(rh, rhs) and np.array_equal(rl, rls)
    assert np.array_equal(q, qs / s[:, None])
    assert np.array_equal(bq, d[:, None] * q)
    assert oracle.orth_err_diag(q, d)[0] <= 1e-14


def test_svqb_b_diagonal_is_scaled_svqb():
    n, k = 600, 4
    x = synth.conditioned(n, k, 1e4, 64)
    d = pow4_diag(n, 65)
    s = np.sqrt(d)
    q, bq, (zh, zl), rank = oracle.svqb_b(x, d[:, None] * x, passes=2)
    qs, (zhs, zls), ranks = oracle.svqb(s[:, None] * x, passes=2)
    assert rank == ranks == k
    assert np.array_equal(zh, zhs) and np.array_equal(zl, zls)
    assert np.array_equal(q, qs / s[:, None])


def test_project_b_diagonal_is_scaled_project():
    n, kv, k = 512, 6, 3
    d = pow4_diag(n, 66)
    s = np.sqrt(d)
    wt = synth.orthonormal_basis(n, kv, 67)      # Euclidean-orthonormal
    w, bw = wt / s[:, None], wt * s[:, None]     # B-orthonormal W and B W, exactly
    x = synth.gaussian(n, k, 68)
    xt, pt, (ch, cl), (mh, ml) = oracle.project_b(w, bw, x, d[:, None] * x)
    yt, (ch2, cl2), (mh2, ml2) = oracle.project(wt, s[:, None] * x)
    assert np.array_equal(ch, ch2) and np.array_equal(cl, cl2)
    assert np.array_equal(xt, yt / s[:, None]) and np.array_equal(pt, yt * s[:, None])
    assert np.array_equal(mh, mh2) and np.array_equal(ml, ml2)


def test_gram_b_takes_the_symmetric_part():
    # P not equal to B X for any symmetric B: M must be (X^T P + P^T X) / 2
    g = np.random.default_rng(69)
    x = g.standard_normal((40, 3))
    p = g.standard_normal((40, 3))
    xt, pt, (ch, cl), (mh, ml) = oracle.project_b(np.zeros((40, 1)), np.zeros((40, 1)), x, p)
    assert np.array_equal(xt, x) and np.array_equal(pt, p) and not ch.any()
    ex = exact_gram(x, p)
    for i in range(3):
        for j in range(3):
            assert dd_fr(mh, ml, i, j) == pytest.approx((ex[i][j] + ex[j][i]) / 2, rel=2.0 ** -104, abs=0)


def test_orth_err_diag_with_unit_weights_is_orth_err():
    q = synth.conditioned(300, 4, 10.0, 70)
    assert oracle.orth_err_diag(q, np.ones(300)) == oracle.orth_err(q)


# ------------------------------------------- two-pass SVQB transform
# In exact arithmetic the first pass gives X1 = X M0^{-1/2} with X1^T X1 = I,
# the second Z2 = I, so the accumulated transform is Z_tot = M0^{-1/2} and
# Q = X Z_tot is the orthogonal polar factor of X.  The rounding of X1 to
# FP64 makes Z2 = I + O(u), which leaves Z_tot within O(kappa u) of M0^{-1/2};
# the accumulated product order (Z1 Z2, not Z2 Z1 or a transpose) shows in
# X Z_tot = Q, whose error would then grow to the size of the commutator
# [Z2, Z1] ~ kappa u.  Everything below is computed in mpmath.

def _mp_mat(a, lo=None):
    import mpmath as mp
    m = mp.matrix(a.shape[0], a.shape[1])
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            m[i, j] = mp.mpf(float(a[i, j])) + (mp.mpf(float(lo[i, j])) if lo is not None else 0)
    return m


def _mp_maxabs(m):
    return max(abs(m[i, j]) for i in range(m.rows) for j in range(m.cols))


@pytest.mark.parametrize("k,kappa", [(3, 1e4), (4, 1e8), (6, 1e6)])
def test_svqb_two_pass_transform_mpmath(k, kappa):
    import mpmath as mp
    mp.mp.prec = 320
    n = 40
    x = synth.conditioned(n, k, kappa, 1300 + k)
    q, (zh, zl), rank = oracle.svqb(x, passes=2)
    assert rank == k
    X, Q, Z = _mp_mat(x), _mp_mat(q), _mp_mat(zh, zl)
    M0 = X.T * X
    # X Z_tot reproduces the returned Q to the rounding of the two updates
    assert _mp_maxabs(X * Z - Q) < 1e-14
    # Z_tot^T M0 Z_tot = I up to the FP64 rounding of the intermediate X1
    assert _mp_maxabs(Z.T * M0 * Z - mp.eye(k)) < 1e-14
    # Z_tot = M0^{-1/2} within kappa u, and Q is the polar factor U V^T of X
    lam, U = mp.eigsy(M0)
    Minv = U * mp.diag([1 / mp.sqrt(lam[i]) for i in range(k)]) * U.T
    assert _mp_maxabs(Z - Minv) <= 100 * kappa * U64 * _mp_maxabs(Minv)
    Us, S, Vt = mp.svd_r(X)
    polar = Us * Vt
    assert _mp_maxabs(Q - polar) <= 100 * kappa * U64


def test_svqb_two_pass_one_pass_on_orthonormal_columns():
    # orthogonal columns with power-of-two norms: both passes are exact, Z_tot = diag(1/s)
    u = synth.hadamard_basis(64, 4, 5)
    s = np.array([2.0, 0.25, 8.0, 1.0])
    q, (zh, zl), rank = oracle.svqb(np.asfortranarray(u * s), passes=2)
    assert rank == 4
    assert np.array_equal(zh, np.diag(1 / s)) and not np.any(zl)
    assert np.array_equal(q, u)


# ------------------------------------------- iterated two-phase algorithm

def test_orthogonalize_exact_case_takes_one_update():
    # W and X from disjoint columns of an exact Hadamard basis, X scaled by
    # powers of two: C = 0 exactly, M = S^2, SVQB gives Z = S^{-1} exactly,
    # and the second iteration finds C = 0, M = I: one update, exact result.
    full = synth.hadamard_basis(256, 9, 1401)
    w, u = full[:, :6], np.asfortranarray(full[:, 6:])
    s = np.array([4.0, 0.5, 2.0])
    q, iters, rank = oracle.orthogonalize(w, u * s, eps=1e-12, max_iter=5)
    assert iters == 1 and rank == 3
    assert np.array_equal(q, u)
    q0, iters0, _ = oracle.orthogonalize(w, u, eps=1e-12, max_iter=5)
    assert iters0 == 0 and np.array_equal(q0, u)


def test_orthogonalize_reports_no_convergence():
    w = synth.hadamard_basis(256, 8, 1402)
    x = synth.near_span(w, 2, 1e6, seed=1403)
    _, iters, _ = oracle.orthogonalize(w, x, eps=0.0, max_iter=3)
    assert iters == -3


@pytest.mark.parametrize("k,kxw", [(1, 1e12), (3, 1e12), (4, 1e6)])
def test_orthogonalize_invariants_and_span(k, kxw):
    """On exit both measures are below eps (the stopping rule), and the result
    spans the projection of X onto the complement of W:
    ||(I - Q Q^T)(I - W W^T) X|| / ||(I - W W^T) X|| small, checked in
    mpmath from the inputs alone."""
    import mpmath as mp
    mp.mp.prec = 260
    n, kv = 256, 8
    w = synth.hadamard_basis(n, kv, 1404 + k)
    x = synth.near_span(w, k, kxw, seed=1405 + k, kappa=1e3)
    q, iters, rank = oracle.orthogonalize(w, x, eps=1e-10, max_iter=8)
    assert iters >= 1 and rank == k
    # the stopping measures (Frobenius bounds the 2-norm), from the oracle's own measures
    assert oracle.cross_err(w, q) <= 1e-10
    assert oracle.orth_err(q)[1] <= 1e-10
    W, X, Q = _mp_mat(w), _mp_mat(x), _mp_mat(q)
    P = X - W * (W.T * X)
    R = P - Q * (Q.T * P)
    assert mp.mnorm(R, "f") <= 1e-12 * mp.mnorm(P, "f")


# ------------------------------------------- the paper's CPU arithmetic

def test_fp64_gram_plain_is_the_row_ordered_sum():
    g = synth.rng(1501)
    x = wide_range(g, 57, 3)
    y = wide_range(g, 57, 2)
    hi, lo = oracle.fp64_gram(x, y, mode=oracle.FP64)
    assert not np.any(lo)
    for i in range(3):
        for j in range(2):
            s = 0.0
            for r in range(57):
                s = s + float(x[r, i]) * float(y[r, j])
            assert hi[i, j] == s


@pytest.mark.parametrize("n", [10, 200, 3000])
def test_fp64_gram_within_textbook_bounds(n):
    g = synth.rng(1502 + n)
    x = wide_range(g, n, 2)
    y = wide_range(g, n, 2)
    ex = exact_gram(x, y)
    bound = abs_gram(x, y)
    gam = F(n) * F(U64) / (1 - F(n) * F(U64))
    ph, _ = oracle.fp64_gram(x, y, mode=oracle.FP64)
    dh, dl = oracle.fp64_gram(x, y, mode=oracle.DD)
    for i in range(2):
        for j in range(2):
            # plain: |s - x^T y| <= gamma_n |x|^T |y|
            assert abs(F(float(ph[i, j])) - ex[i][j]) <= gam * F(float(bound[i, j]))
            # Dot2 kept as a double-word: error <= gamma_n^2 |x|^T |y| (no final rounding)
            assert abs(dd_fr(dh, dl, i, j) - ex[i][j]) <= gam * gam * F(float(bound[i, j])) + F(2.0 ** -1074)


def test_fp64_gram_dot2_resolves_cancellation():
    # x^T y = 2^-80 with terms of size 1: plain FP64 returns 0, Dot2 the exact value
    x = np.array([[1.0], [2.0 ** -80], [-1.0], [3.0], [-3.0]])
    y = np.ones((5, 1))
    ph, _ = oracle.fp64_gram(x, y, mode=oracle.FP64)
    dh, dl = oracle.fp64_gram(x, y, mode=oracle.DD)
    assert ph[0, 0] == 0.0
    assert dh[0, 0] + dl[0, 0] == 2.0 ** -80


def test_fp64_cholqr_k1_dd_square_root():
    # k = 1: R = ||x|| in double-double, Q = x / R rounded once
    g = synth.rng(1503)
    x = g.standard_normal((41, 1))
    q, (rh, rl), info = oracle.fp64_cholqr(x, mode=oracle.DD)
    assert info == 0
    ss = sum((F(float(v)) ** 2 for v in x[:, 0]), F(0))
    r = F(float(rh[0, 0])) + F(float(rl[0, 0]))
    assert abs(r * r - ss) <= F(2.0 ** -100) * ss
    for i in range(41):
        ex = F(float(x[i, 0])) / r
        assert abs(F(float(q[i, 0])) - ex) <= F(U64) * abs(ex) * F(1.0000001)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6, 1e7])
def test_fp64_cholqr_orthogonality_laws(kappa):
    """Sec. 4.2: FP64 CholQR loses orthogonality like kappa^2 u, the DD form
    like kappa^2 u^2 (stays at the rounding floor of the stored Q up to
    kappa ~ 1e8); the binary128 oracle measures both."""
    n, k = 2000, 6
    x = synth.conditioned(n, k, kappa, 1504)
    qp, _, ip = oracle.fp64_cholqr(x, mode=oracle.FP64)
    qd, (rh, rl), idd = oracle.fp64_cholqr(x, mode=oracle.DD)
    assert ip == 0 and idd == 0
    ep = oracle.orth_err(qp)[0]
    ed = oracle.orth_err(qd)[0]
    assert ep <= 10 * k * kappa ** 2 * U64 + 20 * U64
    if kappa >= 1e4:
        assert ep >= 1e-3 * kappa ** 2 * U64  # the law is visible
    assert ed <= 1e-14
    if kappa >= 1e6:
        assert ep >= 1e3 * ed
    # the DD factorization agrees with the binary128 oracle's
    qo, (roh, rol), _ = oracle.cholqr(x)
    assert np.max(np.abs(qd - qo)) <= 4 * U64 + 8 * kappa ** 2 * (n + 64) * 2.0 ** -104
    assert oracle.fact_err(x, qd, rh, rl) <= 8 * U64


def test_fp64_cholqr_breakdown_and_two_passes():
    x = synth.gaussian(300, 3, 1505)
    x[:, 1] = 0.0
    q, _, info = oracle.fp64_cholqr(x, mode=oracle.DD)
    assert info == 2 and np.array_equal(q, x)
    # plain FP64 CholQR2 repairs the kappa^2 u loss at kappa = 1e6
    y = synth.conditioned(1000, 5, 1e6, 1506)
    q2, (rh, rl), info = oracle.fp64_cholqr(y, passes=2, mode=oracle.FP64)
    assert info == 0 and oracle.orth_err(q2)[0] <= 1e-14


@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_project_against_binary128(mode):
    n, kv, k = 3000, 8, 3
    v = synth.orthonormal_basis(n, kv, 1507)
    y = synth.conditioned(n, k, 1e3, 1508)
    yt, (ch, cl), (mh, ml) = oracle.fp64_project(v, y, mode=mode)
    yo, (cho, clo), _ = oracle.project(v, y)
    cref = np.abs(v).T @ np.abs(y)
    if mode == oracle.FP64:
        assert np.all(np.abs(ch - cho) <= (n * U64 / (1 - n * U64)) * cref)
        tol = (kv + 2) * U64 * (np.abs(y) + np.abs(v) @ np.abs(cho)) + np.abs(v) @ (n * U64 * cref)
        assert np.all(np.abs(yt - yo) <= tol)
    else:
        assert np.all(np.abs((ch - cho) + (cl - clo)) <= (n * U64) ** 2 * cref + 2.0 ** -1000)
        tol = 2 * U64 * np.abs(yo) + 2.0 ** -100 * (np.abs(y) + np.abs(v) @ np.abs(cho))
        assert np.all(np.abs(yt - yo) <= tol)
    mo = oracle.gram(yt)
    assert np.all(np.abs((mh - mo[0]) + (ml - mo[1])) <= (n * U64) ** (1 + mode) * (np.abs(yt).T @ np.abs(yt)))


# ------------------------------------------- pivoted, partial CholQR

def test_cholqr_piv_orthogonal_columns_closed_form():
    # orthogonal columns with power-of-two norms: the pivots are the columns
    # in decreasing norm (ties: lowest index), R = diag(sorted norms) and Q the
    # normalized columns, all exact
    u = synth.hadamard_basis(64, 5, 1601)
    s = np.array([0.5, 8.0, 2.0, 8.0, 0.25])
    q, perm, rank, (rh, rl), info = oracle.cholqr_piv(np.asfortranarray(u * s))
    assert info == 0 and rank == 5
    assert list(perm) == [1, 3, 2, 0, 4]
    assert np.array_equal(rh, np.diag(s[perm])) and not np.any(rl)
    assert np.array_equal(q, u[:, perm])


def test_cholqr_piv_rank_deficient():
    g = synth.rng(1602)
    a, b = g.standard_normal((200, 1)), g.standard_normal((200, 1))
    x = np.asfortranarray(np.hstack([a, b, a + b, 3.0 * b]))  # rank 2
    q, perm, rank, (rh, rl), info = oracle.cholqr_piv(x, tol=1e-20)
    assert info == 0 and rank == 2
    assert not np.any(q[:, 2:])
    assert oracle.orth_err(q[:, :2])[0] < 1e-15
    # the kept columns span X: (I - Q Q^T) X = 0 to rounding
    assert np.max(np.abs(x - q[:, :2] @ (q[:, :2].T @ x))) < 1e-13 * np.max(np.abs(x))
    # the first pivot is the largest column (3b here or a + b)
    norms = np.sum(x * x, axis=0)
    assert perm[0] == int(np.argmax(norms))


@pytest.mark.parametrize("kappa", [1e2, 1e8])
def test_cholqr_piv_invariants(kappa):
    n, k = 400, 7
    x = synth.conditioned(n, k, kappa, 1603)
    for passes in (1, 2):
        q, perm, rank, (rh, rl), info = oracle.cholqr_piv(x, passes=passes)
        assert info == 0 and rank == k and sorted(perm) == list(range(k))
        r = rh + rl
        # the pivoted diagonal does not increase
        d = np.diag(rh)
        assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))
        assert np.all(np.tril(rh, -1) == 0)
        assert oracle.orth_err(q)[0] < 20 * U64 + kappa ** 2 * 2.0 ** -111
        assert oracle.fact_err(np.asfortranarray(x[:, perm]), q, rh, rl) < 8 * U64 * np.sqrt(k)


def test_cholqr_piv_drops_negligible_column():
    u = synth.orthonormal_basis(300, 4, 1604)
    x = np.asfortranarray(u * np.array([1.0, 1e-20, 2.0, 0.5]))
    q, perm, rank, _, info = oracle.cholqr_piv(x, tol=1e-30)
    assert rank == 3 and perm[3] == 1 and not np.any(q[:, 3])
    q2, _, rank2, _, _ = oracle.cholqr_piv(x, tol=1e-50)
    assert rank2 == 4  # below the cut it is kept


# ------------------------------------------------- rotated SVQB (Z = D U Lambda^{-1/2})

def _rot_parts(m, z):
    """V = D^{-1} Z (its columns u_j lambda_j^{-1/2}) and S = D M D, in mpmath."""
    import mpmath as mp
    mp.mp.prec = 120
    k = m.shape[0]
    M = mp.matrix([[mp.mpf(float(m[i, j])) for j in range(k)] for i in range(k)])
    d = [1 / mp.sqrt(M[i, i]) for i in range(k)]
    S = mp.matrix(k, k)
    for i in range(k):
        for j in range(k):
            S[i, j] = d[i] * M[i, j] * d[j]
    return M, d, S


def test_svqb_rotated_invariants_in_mpmath():
    """Z^T M Z = I; the columns of V = D^{-1} Z are eigenvectors of D M D
    with eigenvalue 1 / |v_j|^2, ascending; each one's largest entry is
    positive."""
    import mpmath as mp
    x = synth.conditioned(2000, 5, 1e3, 707)
    m = x.T @ x
    _, (zh, zl), rank = oracle.svqb_rotated(x, m=(m, None))
    assert rank == 5
    M, d, S = _rot_parts(m, zh)
    k = 5
    Z = mp.matrix([[mp.mpf(float(zh[i, j])) + mp.mpf(float(zl[i, j])) for j in range(k)] for i in range(k)])
    G = Z.T * M * Z
    assert max(abs(G[i, j] - (1 if i == j else 0)) for i in range(k) for j in range(k)) < 1e-28
    lams = []
    for j in range(k):
        v = mp.matrix([Z[i, j] / d[i] for i in range(k)])
        lam = 1 / sum(v[i] ** 2 for i in range(k))
        r = S * v - lam * v
        assert max(abs(r[i]) for i in range(k)) < 1e-28 * max(abs(v[i]) for i in range(k))
        big = max(range(k), key=lambda i: abs(v[i]))
        assert v[big] > 0
        lams.append(lam)
    assert all(lams[j] <= lams[j + 1] for j in range(k - 1))


def test_svqb_rotated_matches_numpy_eigh_on_a_separated_spectrum():
    """A well-conditioned case with distinct eigenvalues: Z equals
    D U Lambda^{-1/2} built from numpy's eigh (ascending; signs fixed by the
    largest entry) to FP64 accuracy."""
    g = synth.rng(708)
    x = np.asfortranarray(g.standard_normal((400, 6)) * np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.7]))
    q, (zh, zl), rank = oracle.svqb_rotated(x)
    m = x.T @ x
    d = 1 / np.sqrt(np.diag(m))
    lam, u = np.linalg.eigh(d[:, None] * m * d[None, :])
    assert np.min(np.diff(lam)) > 1e-3
    for a in range(6):
        u[:, a] *= np.sign(u[np.argmax(np.abs(u[:, a])), a])
    z = d[:, None] * u / np.sqrt(lam)[None, :]
    assert rank == 6 and np.max(np.abs((zh + zl) - z)) <= 1e-12 * np.max(np.abs(z))
    assert np.max(np.abs(q - x @ z)) <= 1e-12 * np.max(np.abs(q))


def test_svqb_rotated_orthogonal_columns_and_rank():
    """Orthogonal columns: D M D = I, no rotation, the eigenpairs keep their
    index order, so Z = D and Q = the normalized columns, exactly; a zero
    column gives eigenvalue 0, a zero first column of Z and rank k - 1."""
    h = synth.hadamard_basis(256, 4, 709)  # exactly orthonormal columns
    scale = np.array([2.0, 0.25, 8.0, 1.0])
    x = np.asfortranarray(h * scale)
    q, (zh, zl), rank = oracle.svqb_rotated(x)
    assert rank == 4
    assert np.array_equal(zh, np.diag(1 / scale)) and not np.any(zl)
    assert np.array_equal(q, h)
    x0 = x.copy(order="F")
    x0[:, 2] = 0.0
    q0, (zh0, zl0), rank0 = oracle.svqb_rotated(x0)
    assert rank0 == 3
    assert not np.any(zh0[:, 0]) and not np.any(q0[:, 0])
    assert oracle.orth_err(q0[:, 1:])[0] < 1e-15


@pytest.mark.parametrize("a", [0.5, -0.25, 0.9])
def test_svqb_rotated_2x2_closed_form(a):
    """M = D^-1 [[1, a], [a, 1]] D^-1 with D = diag(1/2, 4): D M D has
    eigenvalues 1 - a and 1 + a with eigenvectors (1, -1)/sqrt 2 and
    (1, 1)/sqrt 2, so |Z| = |D U Lambda^-1/2| is known in closed form, the
    columns follow the eigenvalues in ascending order, the column of
    (1, -1) has entries of opposite sign and the column of (1, 1) two
    positive ones (its largest entry is positive).  (Which entry of (1, -1)
    is positive is a tie that rounding decides.)"""
    import mpmath as mp
    mp.mp.prec = 120
    d = np.array([0.5, 4.0])
    m = np.asfortranarray(np.array([[1.0, a], [a, 1.0]]) / d[:, None] / d[None, :])  # exact: powers of two
    x = np.asfortranarray(np.linalg.cholesky(m).T)  # any X: M is passed explicitly
    _, (zh, zl), rank = oracle.svqb_rotated(x, m=(m, None))
    assert rank == 2
    lam = sorted([1 - mp.mpf(a), 1 + mp.mpf(a)])
    for j in range(2):
        want = [mp.mpf(d[i]) / mp.sqrt(2) / mp.sqrt(lam[j]) for i in range(2)]
        got = [mp.mpf(float(zh[i, j])) + mp.mpf(float(zl[i, j])) for i in range(2)]
        assert max(abs(abs(got[i]) - want[i]) for i in range(2)) < mp.mpf(2) ** -100 * max(want)
    j_anti = 0 if a > 0 else 1  # the eigenvalue 1 - a of (1, -1) is the smaller when a > 0
    assert zh[0, j_anti] * zh[1, j_anti] < 0
    assert zh[0, 1 - j_anti] > 0 and zh[1, 1 - j_anti] > 0
