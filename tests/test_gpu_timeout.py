"""A bounded device wait that runs out: the persistent Cholesky's grid barriers
give up after a limit, report IHS_ETIMEOUT and leave the context usable.

The wait is made to run out on the host's say-so, with no fault: a test-only
knob read at context creation (IHS_TEST_BARRIER_UNREACHABLE=1) makes the first
barrier of the context's first persistent factorisation ask for one arrival
more than its grid can give, so every CTA's wait reaches the limit
(IHS_BARRIER_LIMIT_MS, lowered here to 50 ms) and the CTAs leave; that kernel
has no bulk copies in flight.  The next factorisation on the same context runs
normally and meets the oracle."""
import time

import numpy as np
import pytest

from oracle import linalg
from paper_2006_05874_gb300 import problems

pytestmark = pytest.mark.gpu


def test_factor_wait_runs_out_and_context_recovers(torch_cuda, monkeypatch):
    from paper_2006_05874_gb300 import ihs

    torch = torch_cuda
    monkeypatch.setenv("IHS_TEST_BARRIER_UNREACHABLE", "1")
    monkeypatch.setenv("IHS_BARRIER_LIMIT_MS", "50")
    ctx = ihs.Context()
    monkeypatch.delenv("IHS_TEST_BARRIER_UNREACHABLE")
    monkeypatch.delenv("IHS_BARRIER_LIMIT_MS")
    try:
        m, d, nu = 200, 300, 0.1          # k = 200: the persistent Cholesky (k > 32)
        SA = problems.random_matrix(m, d, seed=9, scale=1.0 / np.sqrt(d))
        SAg = torch.from_numpy(SA).cuda()
        t0 = time.perf_counter()
        with pytest.raises(ihs.IHSError) as e:
            ctx.factor(SAg, nu)
        assert e.value.status == ihs.IHS_ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        # the same context, the knob spent: a correct factor and apply
        F = ctx.factor(SAg, nu)
        g = problems.random_vector(d, seed=10)
        gt = torch.empty(d, device="cuda")
        r = F.apply_hinv(torch.from_numpy(g).cuda(), gt)
        F.destroy()
        ref = linalg.WoodburyFactor(SA, nu).apply(g)
        assert np.linalg.norm(gt.cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
        assert abs(r - linalg.newton_decrement(g, ref)) <= 1e-9 * abs(linalg.newton_decrement(g, ref))
    finally:
        ctx.destroy()


def test_knob_is_off_by_default(ctx, torch_cuda):
    torch = torch_cuda
    SA = torch.from_numpy(problems.random_matrix(100, 160, seed=11, scale=0.1)).cuda()
    F = ctx.factor(SA, 0.2)
    F.destroy()
