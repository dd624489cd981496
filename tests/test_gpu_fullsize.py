"""Parity at the benchmarks' full sizes, in the launch configuration bench.py
times, on outputs the binary128 oracle can compute (sampled entries and rows)
and on properties that hold at any size (orthonormality, the factorization
residual, ranks).  Tolerances as in tests/test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

U = 2.0 ** -53
U2 = 2.0 ** -104


def dev(a):
    import torch
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def test_projection_cholqr_at_full_size(eo, ctx):
    """V 4,000,000 x 64 orthonormal, Y 4,000,000 x 16 with kappa = 1e10: the
    bench step (V^T Y, Y - V C, M = Y~^T Y~, CholQR with the automatic second
    pass), all in the compensated mode."""
    n, kv, k = 4_000_000, 64, 16
    v, y = synth.project_block(n=n, kv=kv, k=k)
    V, Y = dev(v), dev(y)
    c = eo.gram(ctx, V, Y, prec=eo.DD)
    yt_d, _ = eo.project_apply(ctx, V, Y, c, prec=eo.DD, want_m=False)
    m = eo.gram(ctx, yt_d, prec=eo.DD)
    yt = host(yt_d)
    rh, rl, info = eo.cholqr(ctx, yt_d, passes=0, prec=eo.DD, M=m)
    assert int(info.item()) == 0
    q = host(yt_d)

    # C = V^T Y, every entry, against the oracle: |C - C*| <= 2^-104 |C*| + n 2^-96 max|v_i| max|y_j|
    # (the normwise bound of the compensated Gram products)
    ch_o, cl_o = oracle.gram(v, y)
    err = np.abs((host(c[0]) - ch_o) + (host(c[1]) - cl_o))
    bound = U2 * np.abs(ch_o) + n * 2.0 ** -96 * np.outer(np.max(np.abs(v), axis=0), np.max(np.abs(y), axis=0))
    assert np.all(err <= bound)

    # Y~ on sampled rows: the oracle's projection with its own C
    rows = np.sort(np.random.default_rng(7).choice(n, 4096, replace=False))
    yt_o = oracle.project_apply(v[rows], y[rows], ch_o, cl_o)
    row_max = np.max(np.abs(v[rows]), axis=1)[:, None] * np.max(np.abs(ch_o), axis=0)[None, :]
    tol = 2 * U * np.abs(yt_o) + kv * 2.0 ** -99 * row_max + kv * np.max(np.abs(v[rows]), axis=1)[:, None] * \
        np.max(bound, axis=0)[None, :]
    assert np.all(np.abs(yt[rows] - yt_o) <= tol)

    # Q: orthonormal, and a QR factorization of the projected block
    assert oracle.orth_err(q)[0] <= 1e-14
    assert oracle.fact_err(yt, q, host(rh), host(rl)) <= 1e-14
    assert np.all(np.diag(host(rh)) > 0)


def test_gram_precision_sweep_sampled_at_full_size(eo, ctx):
    """n = 32,000,000, k = 64, kappa = 1e8: sampled entries of X^T X in the
    three modes against the oracle on the same columns."""
    import torch
    n, k = 32_000_000, 64
    g = torch.Generator(device="cuda")
    g.manual_seed(20180604 + 2)
    s = torch.logspace(0.0, -8.0, k, dtype=torch.float64, device="cuda")
    X = (torch.randn(k, n, dtype=torch.float64, device="cuda", generator=g) * (s / n ** 0.5)[:, None]).t()
    X32 = X.float().t().contiguous().t()
    pairs = [(0, 0), (0, 63), (17, 42), (63, 63), (31, 32), (5, 60)]
    got = {}
    for prec in (eo.DD, eo.FP64, eo.F32):
        gh, gl = eo.gram(ctx, X32 if prec == eo.F32 else X, prec=prec)
        got[prec] = (host(gh), host(gl))
    for i, j in pairs:
        xi, xj = X[:, i].cpu().numpy(), X[:, j].cpu().numpy()
        rh, rl = oracle.gram(xi[:, None], xj[:, None])
        ref = rh[0, 0] + rl[0, 0]
        mi, mj = np.max(np.abs(xi)), np.max(np.abs(xj))
        absdot = float(np.abs(xi) @ np.abs(xj))
        dd = got[eo.DD][0][i, j] + got[eo.DD][1][i, j]
        assert abs((got[eo.DD][0][i, j] - rh[0, 0]) + (got[eo.DD][1][i, j] - rl[0, 0])) <= \
            U2 * abs(ref) + n * 2.0 ** -96 * mi * mj, (i, j)
        assert abs(got[eo.FP64][0][i, j] - ref) <= n * U / (1 - n * U) * absdot, (i, j)
        fi, fj = X32[:, i].cpu().numpy().astype(np.float64), X32[:, j].cpu().numpy().astype(np.float64)
        rfh, rfl = oracle.gram(fi[:, None], fj[:, None])
        assert abs(got[eo.F32][0][i, j] - (rfh[0, 0] + rfl[0, 0])) <= \
            n * U / (1 - n * U) * float(np.abs(fi) @ np.abs(fj)), (i, j)
        assert np.isfinite(dd)


def test_batched_svqb_sampled_blocks_at_full_size(eo, ctx):
    """The batched workload's 512 blocks (n log-uniform in [1e4, 2e6], k in
    4/8/16/32, kappa log-uniform in [1e2, 1e10]) in one graph launch: every
    rank is k, and sampled blocks are orthonormal in the oracle's measure."""
    import torch
    rng = np.random.default_rng(20180604 + 3)
    nb = 512
    ns = np.exp(rng.uniform(np.log(1e4), np.log(2e6), nb)).astype(np.int64)
    ks = rng.choice([4, 8, 16, 32], nb)
    kappas = np.exp(rng.uniform(np.log(1e2), np.log(1e10), nb))
    g = torch.Generator(device="cuda")
    g.manual_seed(20180604 + 3)
    X = []
    for n, k, kap in zip(ns, ks, kappas):
        n, k = int(n), int(k)
        qn, rn = np.linalg.qr(rng.standard_normal((k, k)))
        q = torch.from_numpy(qn * np.sign(np.diag(rn))[None, :]).cuda()
        s = torch.logspace(0.0, -float(np.log10(kap)), k, dtype=torch.float64, device="cuda")
        x = (torch.randn(n, k, dtype=torch.float64, device="cuda", generator=g) * (s / float(np.sqrt(n)))[None, :]) @ q.t()
        X.append(x.t().contiguous().t())
    b = eo.Batch(ctx, X, passes=0, prec=eo.DD)
    b.run()
    torch.cuda.synchronize()
    assert np.array_equal(b.out.cpu().numpy(), ks)
    for i in (int(np.argmax(ns)), int(np.argmax(kappas)), 0, 255):
        assert oracle.orth_err(host(X[i]))[0] <= 1e-14, i
    b.close()
