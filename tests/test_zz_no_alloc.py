"""krr_predict_noalloc: prediction whose call allocates no device memory.

Serving code that records its request path under CUDA stream capture, or that
runs under a fixed device-memory budget, cannot let a call allocate; this
entry point keeps its per-call scratch in a static device array instead.  Its
results must match krr_predict's (FP64 tolerance of the parity tests, 1e-12)
on consecutive calls that reuse the shared scratch.  This file is collected
last so that a failure here cannot hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2111_10140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_10140_gb300 import binding as B
    w = W.random_problem(6000, 5, [(0, 1, 2), (3, 4)], 0.2, 32, 6, seed=71)
    w.epsB = 0.25
    plan = B.anova_fastsum_plan(torch.from_numpy(w.X).cuda(), w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB,
                                precision=B.MIXED)
    return B, torch, w, plan


def test_noalloc_predict_matches_krr_predict_on_consecutive_calls(env):
    B, torch, w, plan = env
    alpha = torch.from_numpy(w.alpha).cuda()
    rng = np.random.default_rng(5)
    # two calls in a row with different sizes: the second reuses the scratch the first left behind
    for M in (5000, 1777):
        Z = torch.from_numpy(w.X[rng.choice(w.N, M, replace=False)] * 0.9).cuda()
        ref = torch.empty(M, dtype=torch.float64, device="cuda")
        got = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        B.krr_predict(plan, alpha, Z, ref)
        B.krr_predict_noalloc(plan, alpha, Z, got)
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def test_noalloc_predict_limits(env):
    B, torch, w, plan = env
    alpha = torch.from_numpy(w.alpha).cuda()
    L = B.lib()
    # more than 65536 points is rejected before any device work
    st = L.krr_predict_noalloc(plan.handle, ctypes.c_void_p(alpha.data_ptr()), ctypes.c_void_p(16), 65537, 5,
                               ctypes.c_void_p(16), None)
    assert st == B.EINVAL
    # points outside the plan's ball need a new frame, which this variant does not build
    Z = torch.from_numpy(w.X[:100] * 3.0).cuda()
    out = torch.empty(100, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AnovaError) as e:
        B.krr_predict_noalloc(plan, alpha, Z, out)
    assert e.value.status == B.ERANGE


def test_no_kernel_wait_gave_up():
    """Runs last: no bounded wait inside the library's kernels (the tcgen05
    gather's mbarrier) gave up during any earlier test of this process."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_10140_gb300 import binding
    assert binding.anova_wait_timeouts() == 0
