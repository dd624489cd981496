"""Batched orthogonalization (eo_batch_*): many blocks of uneven n and k in one
CUDA graph launch, with autotuned launch shapes.

Each block of a batch runs the kernels of a single eo_svqb / eo_cholqr call.
With the default launch shapes (and always in EO_FP64) every block must equal
the single call bitwise, whatever the branch count.  Tuned shapes cut a
block's rows into other chunks, and each chunk aligns its exact sums to its
own exponents, so results may move within the EO_DD bound; they must then be
within that bound of the single call and bitwise equal to the same block
batched alone (its shape depends on its own (k, n) only).  The batch is also
checked against the binary128 oracle directly (the SVQB tolerance of the
single-call tests: both factor a Gram matrix accurate to (n + 64) 2^-104
relative, and a perturbation eps of M moves Q by at most ~kappa^2 eps).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
U2 = 2.0 ** -104

# (n, k, kappa): uneven rows (odd n, n = 0, n below and above the tuning
# threshold of 4096 rows) and every k of the batched workload plus k = 1
SHAPES = [(5000, 4, 1e3), (20_000, 8, 1e6), (70_016, 16, 1e9), (9_000, 32, 1e4), (0, 3, 1.0),
          (4097, 1, 1.0), (33_333, 16, 1e2), (131_072, 32, 1e8), (1_000, 8, 1e10)]


def dev(a):
    import torch
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def blocks(shapes, seed=0, dtype=np.float64):
    out = []
    for i, (n, k, kappa) in enumerate(shapes):
        x = synth.conditioned(n, k, kappa, 4000 + 17 * i + seed) if n >= k else np.zeros((n, k), order="F")
        out.append(np.asfortranarray(x.astype(dtype)))
    return out


def same(a, b):
    return np.array_equal(a, b, equal_nan=True)


def dd_tol(n, k, kappa):
    """Bound on |Q - Q*| of one compensated SVQB/CholQR (see the module docstring)."""
    return 4 * U + 8 * kappa ** 2 * ((n + 64) * U2 + k * U2)


@pytest.mark.parametrize("branches,chains", [(0, False), (3, True), (1, False), (0, True)])
def test_batch_svqb_default_shapes_equal_single_calls(eo, ctx, branches, chains):
    import torch
    xs = blocks(SHAPES)
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, method=eo.BATCH_SVQB, passes=0, prec=eo.DD, tune=False, branches=branches, want_z=True,
                 chains=chains)
    b.run()
    torch.cuda.synchronize()
    ranks = b.out.cpu().numpy()
    # automatic second pass when lambda_max / lambda_min > 1e14, i.e. kappa > 1e7
    assert b.passes() == [2 if kappa > 1e7 else 1 for (_, _, kappa) in SHAPES]
    for i, x in enumerate(xs):
        d = dev(x)
        zh, zl, rank = eo.svqb(ctx, d, passes=0, prec=eo.DD)
        assert same(host(ds[i]), host(d)), i
        assert same(host(b.z[i][0]), host(zh)) and same(host(b.z[i][1]), host(zl)), i
        assert ranks[i] == int(rank.item()), i
    b.close()


def test_batch_svqb_tuned_shapes_same_alone_and_in_the_mix(eo, ctx):
    import torch
    xs = blocks(SHAPES)
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, method=eo.BATCH_SVQB, passes=0, prec=eo.DD, tune=True, want_z=True)
    b.run()
    torch.cuda.synchronize()
    ranks = b.out.cpu().numpy()
    for i, (n, k, kappa) in enumerate(SHAPES):
        # alone: a one-block batch of the same block, same context (same tuned shape)
        d1 = dev(xs[i])
        b1 = eo.Batch(ctx, [d1], method=eo.BATCH_SVQB, passes=0, prec=eo.DD, tune=True, want_z=True)
        assert b1.tile(0) == b.tile(i)
        b1.run()
        torch.cuda.synchronize()
        assert same(host(ds[i]), host(d1)), i
        assert same(host(b.z[i][0]), host(b1.z[0][0])) and same(host(b.z[i][1]), host(b1.z[0][1])), i
        assert int(b1.out[0].item()) == ranks[i]
        b1.close()
        # the single call (default shapes): within the compensated bound, twice (either may carry it)
        d = dev(xs[i])
        zh, zl, rank = eo.svqb(ctx, d, passes=0, prec=eo.DD)
        assert int(rank.item()) == ranks[i]
        if n > 0:
            assert np.max(np.abs(host(ds[i]) - host(d))) <= 2 * dd_tol(n, k, kappa), i
    b.close()


def test_batch_tiles_and_kernel_count(eo, ctx):
    shapes = [s for s in SHAPES if s[0] > 0]
    xs = blocks(shapes)
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, passes=0, prec=eo.DD)
    bc = eo.Batch(ctx, ds, passes=0, prec=eo.DD, chains=True)
    # chains: one graph node per kernel of the single calls; phases: one
    # status launch and one factorization launch per pass for all blocks
    before = ctx.launches()
    for x in xs:
        eo.svqb(ctx, dev(x), passes=0, prec=eo.DD)
    assert bc.kernels() == ctx.launches() - before
    nb = len(shapes)
    assert b.kernels() == bc.kernels() - nb * (1 + 2) + 1 + 2
    bc.close()
    for i, (n, k, _) in enumerate(shapes):
        g, r = b.tile(i)
        if n < 4096:
            assert (g, r) == (0, 0)
        else:
            assert 1 <= g <= 152 and 1 <= r <= 152
    assert b.branches() == min(len(shapes), 16)
    b.close()


def test_batch_matches_oracle(eo, ctx):
    import torch
    shapes = [(3000, 4, 1e4), (20_000, 16, 1e6), (8_192, 32, 1e3), (777, 3, 1.0)]
    xs = blocks(shapes, seed=5)
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, passes=1, prec=eo.DD, want_z=True)
    b.run()
    torch.cuda.synchronize()
    for i, (n, k, kappa) in enumerate(shapes):
        q_o, (zh_o, zl_o), rank_o = oracle.svqb(xs[i])
        tol = dd_tol(n, k, kappa)
        assert np.max(np.abs(host(ds[i]) - q_o)) <= tol, i
        z = host(b.z[i][0]) + host(b.z[i][1])
        assert np.max(np.abs(z - (zh_o + zl_o))) <= tol * np.max(np.abs(zh_o)), i
        assert int(b.out[i].item()) == rank_o == k
        assert oracle.orth_err(host(ds[i]))[0] <= 1e-14


def test_batch_cholqr_equals_single_calls_and_reports_breakdown(eo, ctx):
    import torch
    shapes = [(6000, 4, 1e2), (12_345, 16, 1e7), (50_000, 8, 1e4), (2048, 32, 1e3)]
    xs = blocks(shapes, seed=9)
    xs[2][:, 2] = 0.0  # third pivot of block 2 is zero
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, method=eo.BATCH_CHOLQR, passes=2, prec=eo.DD, want_z=True, tune=False)
    bc = eo.Batch(ctx, [dev(x) for x in xs], method=eo.BATCH_CHOLQR, passes=2, prec=eo.DD, tune=False, chains=True)
    bc.run()
    b.run()
    torch.cuda.synchronize()
    info = b.out.cpu().numpy()
    assert info[2] == 3 and info[0] == info[1] == info[3] == 0
    assert np.array_equal(bc.out.cpu().numpy(), info)
    bc.close()
    for i, x in enumerate(xs):
        d = dev(x)
        rh, rl, inf = eo.cholqr(ctx, d, passes=2, prec=eo.DD)
        assert same(host(ds[i]), host(d)), i
        assert same(host(b.z[i][0]), host(rh)) and same(host(b.z[i][1]), host(rl)), i
        assert info[i] == int(inf.item())


def test_batch_rerun_equals_repeated_calls(eo, ctx):
    import torch
    shapes = [(9000, 8, 1e8), (40_000, 16, 1e5), (4500, 32, 1e2)]
    xs = blocks(shapes, seed=3)
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, passes=1, prec=eo.DD, tune=False)
    b.run()
    b.run()
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        d = dev(x)
        eo.svqb(ctx, d, passes=1, prec=eo.DD)
        eo.svqb(ctx, d, passes=1, prec=eo.DD)
        assert same(host(ds[i]), host(d)), i


def test_batch_fp64_equals_single_calls(eo, ctx):
    import torch
    shapes = [(10_000, 4, 1e3), (30_000, 16, 1e4), (7_001, 32, 1e2)]
    xs = blocks(shapes, seed=11)
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, passes=2, prec=eo.FP64, branches=2)
    b.run()
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        d = dev(x)
        eo.svqb(ctx, d, passes=2, prec=eo.FP64)
        assert same(host(ds[i]), host(d)), i


def test_tune_cache_roundtrip(eo, tmp_path):
    path = str(tmp_path / "tiles.txt")
    shapes = [(20_000, 8, 1e2), (300_000, 16, 1e2), (70_000, 32, 1e2)]
    ds = [dev(x) for x in blocks(shapes, seed=13)]
    c1 = eo.Context(0)
    c1.tune_cache(path)
    b1 = eo.Batch(c1, ds, passes=1, prec=eo.DD)
    tiles1 = [b1.tile(i) for i in range(len(shapes))]
    lines = open(path).read().split("\n")
    assert len([l for l in lines if l.strip()]) == len(shapes)
    before = open(path).read()
    c2 = eo.Context(0)
    c2.tune_cache(path)
    b2 = eo.Batch(c2, ds, passes=1, prec=eo.DD)
    assert [b2.tile(i) for i in range(len(shapes))] == tiles1
    assert open(path).read() == before  # nothing left to tune
    b1.close()
    b2.close()
    c1.close()
    c2.close()


def test_batch_rejects_bad_blocks(eo, ctx):
    import torch
    x = dev(synth.gaussian(100, 3, 1))
    with pytest.raises(ValueError):
        eo.Batch(ctx, [])
    wide = torch.zeros((65, 100), dtype=torch.float64, device="cuda").t()  # 100 x 65: k > 64
    with pytest.raises(eo.EoError) as e:
        eo.Batch(ctx, [x, wide])
    assert e.value.status == eo.EINVAL
    with pytest.raises(eo.EoError):
        eo.Batch(ctx, [x], branches=65)


def test_batch_wide_odd_and_tiny_blocks_equal_single_calls(eo, ctx):
    """k = 64 and odd k above 16 (tensor-core updates in groups of 16
    columns through the branch scratch), one-row blocks, default shapes."""
    import torch
    shapes = [(3000, 64, 1e3), (5001, 33, 1e6), (1, 5, 1.0), (2048, 17, 1e9), (40_000, 48, 1e4)]
    xs = []
    for i, (n, k, kappa) in enumerate(shapes):
        xs.append(synth.conditioned(n, k, kappa, 4300 + i) if n >= k else synth.gaussian(n, k, 4300 + i))
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, passes=0, prec=eo.DD, tune=False, branches=2, want_z=True)
    b.run()
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        d = dev(x)
        zh, zl, rank = eo.svqb(ctx, d, passes=0, prec=eo.DD)
        assert same(host(ds[i]), host(d)), i
        assert same(host(b.z[i][0]), host(zh)) and same(host(b.z[i][1]), host(zl)), i
        assert int(b.out[i].item()) == int(rank.item())
    b.close()


def test_batch_f32_inputs_equal_single_calls(eo, ctx):
    import torch
    shapes = [(10_000, 8, 1e2), (20_001, 16, 1e3), (3_000, 32, 1e2)]
    xs = [np.asfortranarray(synth.conditioned(n, k, kappa, 4400 + i).astype(np.float32))
          for i, (n, k, kappa) in enumerate(shapes)]
    ds = [dev(x) for x in xs]
    b = eo.Batch(ctx, ds, method=eo.BATCH_CHOLQR, passes=2, prec=eo.F32)
    b.run()
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        d = dev(x)
        eo.cholqr(ctx, d, passes=2, prec=eo.F32)
        assert same(host(ds[i]), host(d)), i
    b.close()


def test_batch_two_pass_blocks_match_oracle(eo, ctx):
    """Blocks that take the automatic second pass (kappa > 1e7) against the
    oracle's two-pass SVQB, with the two-pass bound (4 x one pass: the first
    pass's difference survives the second only in its skew part)."""
    import torch
    shapes = [(20_000, 8, 1e9), (70_016, 16, 1e10), (9_000, 32, 1e8), (4_097, 4, 1e12), (12_000, 16, 1e5)]
    xs = blocks(shapes, seed=9)
    ds = [dev(x) for x in xs]
    for tune in (False, True):
        for d, x in zip(ds, xs):
            d.copy_(dev(x))
        b = eo.Batch(ctx, ds, passes=0, prec=eo.DD, tune=tune, want_z=True)
        b.run()
        torch.cuda.synchronize()
        passes = b.passes()
        for i, (n, k, kappa) in enumerate(shapes):
            assert passes[i] == (2 if kappa > 1e7 else 1), i
            q_o, (zh_o, zl_o), rank_o = oracle.svqb(xs[i], passes=passes[i])
            tol = (4 if passes[i] == 2 else 1) * dd_tol(n, k, kappa) + 8 * U
            assert np.max(np.abs(host(ds[i]) - q_o)) <= tol, (i, tune)
            z = host(b.z[i][0]) + host(b.z[i][1])
            assert np.max(np.abs(z - (zh_o + zl_o))) <= tol * np.max(np.abs(zh_o)), (i, tune)
            assert int(b.out[i].item()) == rank_o == k
            assert oracle.orth_err(host(ds[i]))[0] <= 1e-14
        b.close()
