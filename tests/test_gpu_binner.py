"""B-inner products (eo_cholqr_b, eo_svqb_b, eo_project_b) against the
binary128 oracle's B-variants, with B = diag(d) so that B-orthonormality can
be measured with the true B in binary128.

Tolerances as for the Euclidean calls (tests/test_gpu_parity.py): both sides
factor a Gram matrix accurate to (n + 64) 2^-104 relative (the symmetric part
of X^T (B X) in the compensated mode), and a relative perturbation eps of M
moves Q by at most ~kappa_B^2 eps, kappa_B the condition number of X in the
B-norm.

B-orthonormality with the true B cannot beat the representation of B X: P
arrives rounded to FP64, and its relative rounding error enters M directly
(a second pass orthonormalizes in the metric P implies, not in B's).  So the
gate is the oracle's own ||Q^T B Q - I|| on the same P (times 2, plus 1e-14):
the library must do as well as exact arithmetic on the inputs it is given.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
U2 = 2.0 ** -104


def dev(a):
    import torch
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def weights(n, seed, spread=1e3):
    g = np.random.default_rng(seed)
    return np.exp(g.uniform(0.0, np.log(spread), n))


def dd_tol(n, k, kappa):
    return 4 * U + 8 * kappa ** 2 * ((n + 64) * U2 + k * U2)


@pytest.mark.parametrize("n,k,kappa,passes", [(20_000, 8, 1e4, 1), (30_001, 16, 1e7, 2), (4_000, 4, 1e2, 1),
                                              (10_000, 32, 1e5, 2)])
def test_cholqr_b_matches_oracle(eo, ctx, n, k, kappa, passes):
    x = synth.conditioned(n, k, kappa, 900 + k)
    d = weights(n, 901 + k)
    p = d[:, None] * x
    dx, dp = dev(x), dev(p)
    rh, rl, info = eo.cholqr_b(ctx, dx, dp, passes=passes, prec=eo.DD)
    q_o, bq_o, (rh_o, rl_o), info_o = oracle.cholqr_b(x, p, passes=passes)
    assert int(info.item()) == info_o == 0
    kap_b = kappa * np.sqrt(d.max() / d.min())  # bound on the B-norm condition number
    tol = dd_tol(n, k, min(kap_b, kappa * 40))
    q = host(dx)
    assert np.max(np.abs(q - q_o)) <= tol * np.max(np.abs(q_o))
    assert np.max(np.abs(host(dp) - bq_o)) <= tol * np.max(np.abs(bq_o))
    assert oracle.orth_err_diag(q, d)[0] <= 2 * oracle.orth_err_diag(q_o, d)[0] + 1e-14
    r = host(rh) + host(rl)
    assert np.max(np.abs(r - (rh_o + rl_o))) <= tol * np.max(np.abs(rh_o))


def test_svqb_b_matches_oracle(eo, ctx):
    n, k, kappa = 25_000, 8, 1e5
    x = synth.conditioned(n, k, kappa, 910)
    d = weights(n, 911)
    p = d[:, None] * x
    dx, dp = dev(x), dev(p)
    zh, zl, rank = eo.svqb_b(ctx, dx, dp, passes=1, prec=eo.DD)
    q_o, bq_o, (zh_o, zl_o), rank_o = oracle.svqb_b(x, p, passes=1)
    assert int(rank.item()) == rank_o == k
    tol = dd_tol(n, k, kappa * 40)
    assert np.max(np.abs(host(dx) - q_o)) <= tol * np.max(np.abs(q_o))
    assert np.max(np.abs(host(zh) + host(zl) - (zh_o + zl_o))) <= tol * np.max(np.abs(zh_o))
    assert np.array_equal(host(zh), host(zh).T)
    assert oracle.orth_err_diag(host(dx), d)[0] <= 2 * oracle.orth_err_diag(q_o, d)[0] + 1e-14


def test_project_b_matches_oracle(eo, ctx):
    n, kv, k = 40_000, 16, 4
    d = weights(n, 920)
    s = np.sqrt(d)
    wt = synth.orthonormal_basis(n, kv, 921)
    w, bw = wt / s[:, None], wt * s[:, None]  # B-orthonormal to FP64 rounding
    x = synth.conditioned(n, k, 1e3, 922)
    p = d[:, None] * x
    dy, dby = dev(x), dev(p)
    (ch, cl), (mh, ml) = eo.project_b(ctx, dev(w), dev(bw), dy, dby, prec=eo.DD)
    xt_o, pt_o, (ch_o, cl_o), (mh_o, ml_o) = oracle.project_b(w, bw, x, p)
    c_err = np.abs((host(ch) - ch_o) + (host(cl) - cl_o))
    assert np.max(c_err) <= 2 * n * 2.0 ** -96 * np.max(np.abs(bw)) * np.max(np.abs(x))
    assert np.max(np.abs(host(dy) - xt_o)) <= 2 * U * np.max(np.abs(xt_o))
    assert np.max(np.abs(host(dby) - pt_o)) <= 2 * U * np.max(np.abs(pt_o))
    # M against the oracle's symmetric Gram of the GPU's own rounded Y~ and BY~
    # (a projection on an empty basis is exactly that Gram)
    yg, pg = host(dy), host(dby)
    _, _, _, (mh_g, ml_g) = oracle.project_b(np.zeros((n, 1)), np.zeros((n, 1)), yg, pg)
    m_err = np.abs((host(mh) - mh_g) + (host(ml) - ml_g))
    assert np.max(m_err) <= U2 * np.max(np.abs(mh_g)) + 4 * n * 2.0 ** -96 * np.max(np.abs(yg)) * np.max(np.abs(pg))
    assert np.array_equal(host(mh), host(mh).T)


def test_b_identity_matches_euclidean(eo, ctx):
    # B = I: BX is a copy of X and the result is the Euclidean CholQR (within its bound)
    n, k, kappa = 20_000, 8, 1e6
    x = synth.conditioned(n, k, kappa, 930)
    dx, dp = dev(x), dev(x.copy())
    eo.cholqr_b(ctx, dx, dp, passes=1, prec=eo.DD)
    q_o, _, _ = oracle.cholqr(x, passes=1)
    assert np.max(np.abs(host(dx) - q_o)) <= dd_tol(n, k, kappa)
    assert np.array_equal(host(dx), host(dp)) or np.max(np.abs(host(dx) - host(dp))) <= 4 * U


def test_b_fp64_mode(eo, ctx):
    n, k = 10_000, 6
    x = synth.conditioned(n, k, 1e3, 940)
    d = weights(n, 941, 10.0)
    dx, dp = dev(x), dev(d[:, None] * x)
    eo.cholqr_b(ctx, dx, dp, passes=2, prec=eo.FP64)
    q_o, _, _, _ = oracle.cholqr_b(x, d[:, None] * x, passes=2)
    assert oracle.orth_err_diag(host(dx), d)[0] <= 2 * oracle.orth_err_diag(q_o, d)[0] + 1e-13


def test_b_rejects_aliasing(eo, ctx):
    x = dev(synth.gaussian(100, 3, 950))
    with pytest.raises(eo.EoError):
        eo.cholqr_b(ctx, x, x)
