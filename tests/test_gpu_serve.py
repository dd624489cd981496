"""Request server (eo_server_*): resident bases, blocks orthogonalized against
them (Y - V (V^T Y), then compensated CholQR with the automatic second pass)
on concurrent slots under a device-memory budget.

Every slot runs the library's default launch shapes and the compensated sums
are exact, so a request's result must be bitwise that of the single calls
(eo_project with the fused Gram + eo_cholqr), whether it ran alone or mixed
with others.  One request is also checked against the binary128 oracle.
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


def empty_like(t):
    import torch
    return torch.empty((t.shape[1], t.shape[0]), dtype=t.dtype, device=t.device).t()


# (n, kv, k, kappa of the new block)
CLIENTS = [(50_000, 8, 2, 1e4), (120_001, 16, 4, 1e8), (80_000, 32, 8, 1e12), (60_000, 64, 16, 1e6),
           (33_333, 16, 4, 1e10), (200_000, 64, 16, 1e3)]


def make_clients(seed=0):
    out = []
    for i, (n, kv, k, kappa) in enumerate(CLIENTS):
        v = synth.orthonormal_basis(n, kv, 7000 + i + seed)
        y = synth.conditioned(n, k, kappa, 7100 + i + seed)
        out.append((dev(v), dev(y)))
    return out


def single_calls(eo, ctx, V, Y):
    import torch
    out = empty_like(Y)
    _, _, m = eo.project(ctx, V, Y, Yout=out, prec=eo.DD, want_m=True)
    rh, rl, info = eo.cholqr(ctx, out, passes=0, prec=eo.DD, M=m)
    torch.cuda.synchronize()
    return host(out), host(rh), host(rl), int(info.item())


def test_server_results_same_alone_and_in_the_mix(eo, ctx):
    import torch
    clients = make_clients()
    ref = [single_calls(eo, ctx, V, Y) for V, Y in clients]
    srv = eo.Server(ctx, budget=64 << 30, slots=4)
    ids = [srv.add_basis(V) for V, _ in clients]
    # alone: one request at a time
    for (V, Y), b, r in zip(clients, ids, ref):
        out = empty_like(Y)
        R = (torch.zeros((Y.shape[1], Y.shape[1]), dtype=torch.float64, device="cuda").t(),
             torch.zeros((Y.shape[1], Y.shape[1]), dtype=torch.float64, device="cuda").t())
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        rid = srv.submit(b, Y, Yout=out, R=R, info=info)
        st, lat = srv.wait(rid)
        assert st == eo.OK and lat > 0
        assert np.array_equal(host(out), r[0])
        assert np.array_equal(host(R[0]), r[1]) and np.array_equal(host(R[1]), r[2])
        assert int(info.item()) == r[3] == 0
    # in the mix: every client three times, submitted at once (same-basis
    # requests run in order; all write their own outputs)
    outs = []
    for rep in range(3):
        for (V, Y), b in zip(clients, ids):
            out = empty_like(Y)
            outs.append((out, srv.submit(b, Y, Yout=out), len(outs) % len(clients)))
    for out, rid, i in outs:
        st, _ = srv.wait(rid)
        assert st == eo.OK
        assert np.array_equal(host(out), ref[i][0]), i
    stats = srv.stats()
    assert stats["peak_running"] > 1 and stats["queued"] == 0 and stats["running"] == 0
    done = srv.poll()
    assert len(done) == len(clients) + len(outs) and all(s == eo.OK for _, _, _, s in done)
    srv.close()


def test_server_request_matches_oracle(eo, ctx):
    import torch
    n, kv, k, kappa = 20_000, 16, 4, 1e6
    v = synth.orthonormal_basis(n, kv, 7300)
    y = synth.conditioned(n, k, kappa, 7301)
    srv = eo.Server(ctx, budget=8 << 30, slots=2)
    b = srv.add_basis(dev(v))
    out = empty_like(dev(y))
    rid = srv.submit(b, dev(y), Yout=out)
    assert srv.wait(rid)[0] == eo.OK
    yt, _, m = oracle.project(v, y)
    q_o, _, info = oracle.cholqr(yt, passes=1, m=m)
    assert info == 0
    # the projection leaves Y~ with kappa(Y~) ~ kappa(Y); CholQR's bound from the single-call tests
    tol = 4 * U + 8 * kappa ** 2 * ((n + 64) * U2 + k * U2)
    assert np.max(np.abs(host(out) - q_o)) <= tol
    assert oracle.orth_err(host(out))[0] <= 1e-14
    # one projection pass: storing Y~ in FP64 leaves ~u ||Y|| inside span(V),
    # which R^{-1} (~kappa / ||Y||) scales up, so ||V^T Q|| ~ u kappa (the
    # reason the paper iterates the two phases)
    assert oracle.cross_err(v, host(out)) <= 4 * U * kappa * np.sqrt(k)
    srv.close()


def test_server_budget_is_enforced(eo, ctx):
    import torch
    V = dev(synth.orthonormal_basis(10_000, 8, 7400))  # 640 KB
    Y = dev(synth.gaussian(10_000, 8, 7401))
    slots_bytes = 2 * 2 * 8 * 64 * 64  # two slots' Gram buffers are charged at creation
    srv = eo.Server(ctx, budget=slots_bytes + 740_000, slots=2)  # 100 KB beside the basis
    b = srv.add_basis(V)
    assert srv.stats()["resident"] == slots_bytes + 640_000
    with pytest.raises(eo.EoError) as e:
        srv.add_basis(V)  # a second copy does not fit
    assert e.value.status == eo.ENOMEM
    with pytest.raises(eo.EoError) as e:
        srv.submit(b, Y)  # the block (640 KB) can never fit next to the basis
    assert e.value.status == eo.ENOMEM
    small = Y[:, :1]
    rid = srv.submit(b, small)  # 80 KB (in place) fits
    assert srv.wait(rid)[0] == eo.OK
    srv.close()


def test_server_same_basis_runs_in_order(eo, ctx):
    import torch
    n, kv, k = 30_000, 8, 2
    V = dev(synth.orthonormal_basis(n, kv, 7500))
    Y = dev(synth.conditioned(n, k, 1e3, 7501))
    # reference: orthogonalize, then orthogonalize the result again
    a = empty_like(Y)
    _, _, m = eo.project(ctx, V, Y, Yout=a, prec=eo.DD)
    eo.cholqr(ctx, a, passes=0, prec=eo.DD, M=m)
    bref = empty_like(Y)
    _, _, m = eo.project(ctx, V, a, Yout=bref, prec=eo.DD)
    eo.cholqr(ctx, bref, passes=0, prec=eo.DD, M=m)
    torch.cuda.synchronize()
    srv = eo.Server(ctx, budget=8 << 30, slots=4)
    bid = srv.add_basis(V)
    o1, o2 = empty_like(Y), empty_like(Y)
    r1 = srv.submit(bid, Y, Yout=o1)
    r2 = srv.submit(bid, o1, Yout=o2)  # reads the first request's output
    assert srv.wait(r2)[0] == eo.OK and srv.wait(r1)[0] == eo.OK
    assert np.array_equal(host(o1), host(a)) and np.array_equal(host(o2), host(bref))
    srv.close()


def test_server_wide_request_equals_single_calls(eo, ctx):
    """A block of 24 columns (its CholQR update runs in groups of 16 columns
    and may grow the slot's scratch on first use)."""
    n, kv, k = 30_000, 32, 24
    V = dev(synth.orthonormal_basis(n, kv, 7600))
    Y = dev(synth.conditioned(n, k, 1e6, 7601))
    ref = single_calls(eo, ctx, V, Y)
    srv = eo.Server(ctx, budget=8 << 30, slots=2)
    b = srv.add_basis(V)
    out = empty_like(Y)
    rid = srv.submit(b, Y, Yout=out)
    assert srv.wait(rid)[0] == eo.OK
    assert np.array_equal(host(out), ref[0])
    srv.close()
