"""The bounded-wait path on the GPU, exercised without a fault: a warp waits
on an mbarrier that nothing arrives on, gives up after its poll limit and the
host reads ETIMEOUT.  The context stays usable, and the library's own counter
of abandoned waits (which only the kernels' real waits advance) is untouched."""
import numpy as np
import pytest

from paper_2111_10140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_10140_gb300 import binding as B
    return B, torch


def test_wait_that_never_completes_reports_timeout(env):
    B, torch = env
    w = W.random_problem(3000, 3, [(0, 1, 2)], 0.2, 32, 6, seed=81)
    plan = B.anova_fastsum_plan(torch.from_numpy(w.X).cuda(), w.windows, w.ell, n=w.n, m=w.m, eps_B=0.25,
                                precision=B.FP32)
    alpha = torch.from_numpy(w.alpha).float().cuda()
    before = torch.empty_like(alpha)
    B.anova_matvec(plan, alpha, before)
    torch.cuda.synchronize()
    counted = B.anova_wait_timeouts()
    for polls in (1, 1000):
        assert B.anova_debug_wait_probe(polls) == B.ETIMEOUT
    assert B.anova_wait_timeouts() == counted
    after = torch.empty_like(alpha)
    B.anova_matvec(plan, alpha, after)
    torch.cuda.synchronize()
    assert np.array_equal(np.isfinite(after.cpu().numpy()), np.ones(w.N, bool))
    rel = np.linalg.norm((after - before).cpu().numpy()) / np.linalg.norm(before.cpu().numpy())
    assert rel <= 1e-6   # same operator, atomic order may differ
