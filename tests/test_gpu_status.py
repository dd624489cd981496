"""The device-side failure record: a bounded wait that runs out is reported
by eo_device_status as EO_ETIMEOUT (the failure is made on purpose by a
one-thread kernel whose wait on an mbarrier that nothing completes is
bounded by 50 ms; no GPU fault is involved), the record is cleared by the
call, and the context stays usable afterwards."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_cleared(eo):
    import torch
    ctx = eo.Context(0)
    try:
        assert ctx.device_status() == eo.OK  # nothing recorded (and any old record cleared)
        ctx.selftest_wait_timeout(0.05)
        assert ctx.device_status() == eo.ETIMEOUT
        assert "ran out" in eo.lib().eo_last_error(ctx.h).decode()
        assert ctx.device_status() == eo.OK  # cleared by the previous call
        # the context and the tensor-core kernels still work
        x = synth.gaussian(30_000, 16, 950)
        d = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
        gh, gl = eo.gram(ctx, d, prec=eo.DD)
        torch.cuda.synchronize()
        rh, rl = oracle.gram(x)
        err = np.abs((gh.cpu().numpy() - rh) + (gl.cpu().numpy() - rl))
        assert np.all(err <= 2.0 ** -104 * np.abs(rh) + 30_000 * 2.0 ** -96 * np.max(np.abs(x)) ** 2)
        assert ctx.device_status() == eo.OK
    finally:
        ctx.close()


def test_selftest_rejects_bad_limits(eo):
    ctx = eo.Context(0)
    try:
        for s in (0.0, -1.0, 2.5):
            assert eo.lib().eo_selftest_wait_timeout(ctx.h, s) == eo.EINVAL
    finally:
        ctx.close()
