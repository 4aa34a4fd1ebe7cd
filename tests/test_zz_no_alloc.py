"""krr_predict_noalloc: prediction whose call allocates no device memory.

A server that holds a fixed device-memory budget, or a process whose device
allocator belongs to another framework, cannot let a call allocate while it
serves a request; this entry point keeps its per-call scratch in a static
device array instead.  Its results must match krr_predict's on consecutive
calls that reuse the shared scratch (the FP64 path to 1e-12, the FP32 path to
1e-6, and both against the oracle's fast summation), including a call at the
capacity limit of 65536 test points, and device free memory must not move
across a call.  This file is collected last so that a failure here cannot
hide the other GPU tests.
"""
import ctypes
import gc

import numpy as np
import pytest

import oracle
from paper_2111_10140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CAPACITY = 65536


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
    X = torch.from_numpy(w.X).cuda()
    plans = {p: B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=getattr(B, p))
             for p in ("MIXED", "FP32")}
    return B, torch, w, plans


# the FP64 path (a plan with FP64 data) and the FP32-only path, at their parity tolerances
TOL = {"MIXED": 1e-12, "FP32": 1e-6}
ORACLE_TOL = {"MIXED": 1e-12, "FP32": 1e-5}


@pytest.mark.parametrize("prec", ["MIXED", "FP32"])
def test_noalloc_predict_matches_krr_predict_on_consecutive_calls(env, prec):
    B, torch, w, plans = env
    plan = plans[prec]
    alpha = torch.from_numpy(w.alpha).cuda()
    rng = np.random.default_rng(5)
    # two calls in a row with different sizes: the second reuses the scratch the first left behind
    for M in (5000, 1777):
        Zh = w.X[rng.choice(w.N, M, replace=False)] * 0.9
        Z = torch.from_numpy(Zh).cuda()
        ref = torch.empty(M, dtype=torch.float64, device="cuda")
        got = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        B.krr_predict(plan, alpha, Z, ref)
        B.krr_predict_noalloc(plan, alpha, Z, got)
        g = got.cpu().numpy()
        assert rel(g, ref.cpu().numpy()) <= TOL[prec]
        orc = oracle.fastsum(Zh, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha, sigma=w.sigma, epsB=w.epsB, p=w.p)
        assert rel(g, orc) <= ORACLE_TOL[prec]


@pytest.mark.parametrize("prec", ["MIXED", "FP32"])
def test_noalloc_predict_at_capacity(env, prec):
    """M = 65536 exactly: the largest call the static array serves."""
    B, torch, w, plans = env
    plan = plans[prec]
    alpha = torch.from_numpy(w.alpha).cuda()
    Zh = w.X[np.random.default_rng(6).choice(w.N, CAPACITY, replace=True)] * 0.85
    Z = torch.from_numpy(Zh).cuda()
    ref = torch.empty(CAPACITY, dtype=torch.float64, device="cuda")
    got = torch.full((CAPACITY,), float("nan"), dtype=torch.float64, device="cuda")
    B.krr_predict(plan, alpha, Z, ref)
    B.krr_predict_noalloc(plan, alpha, Z, got)
    g = got.cpu().numpy()
    assert np.all(np.isfinite(g))
    assert rel(g, ref.cpu().numpy()) <= TOL[prec]
    orc = oracle.fastsum(Zh, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha, sigma=w.sigma, epsB=w.epsB, p=w.p)
    assert rel(g, orc) <= ORACLE_TOL[prec]


def test_noalloc_predict_leaves_device_memory_unchanged(env):
    B, torch, w, plans = env
    plan = plans["MIXED"]
    alpha = torch.from_numpy(w.alpha).cuda()
    Z = torch.from_numpy(w.X[:3000] * 0.9).cuda()
    out = torch.empty(3000, dtype=torch.float64, device="cuda")
    B.krr_predict_noalloc(plan, alpha, Z, out)           # warm-up: module load, scratch address lookup
    gc.collect()                                          # tensors left by earlier tests are freed now, not below
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    used0 = torch.cuda.memory_allocated()
    for _ in range(3):
        B.krr_predict_noalloc(plan, alpha, Z, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == used0


def test_noalloc_predict_limits(env):
    B, torch, w, plans = env
    plan = plans["MIXED"]
    alpha = torch.from_numpy(w.alpha).cuda()
    L = B.lib()
    # more than 65536 points is rejected before any device work
    st = L.krr_predict_noalloc(plan.handle, ctypes.c_void_p(alpha.data_ptr()), ctypes.c_void_p(16), CAPACITY + 1, 5,
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
    kernels' mbarriers) gave up during any earlier test of this process."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_10140_gb300 import binding
    assert binding.anova_wait_timeouts() == 0
