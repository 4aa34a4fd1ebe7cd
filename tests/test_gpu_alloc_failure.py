"""Out-of-memory error paths without a device fault: the library's host-side
hook makes its k-th device allocation fail, for k = 1, 2, ... until a call
completes.  Every failing call must return ENOMEM or ECUDA, and afterwards the
device memory in use must be what it was before the call: nothing the call
had allocated stays allocated (cudaMalloc'd memory back in the device's free
bytes, stream-ordered memory back in the pool)."""
import numpy as np
import pytest

from paper_2111_10140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_10140_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def snapshot(B, torch):
    torch.cuda.synchronize()
    return B.anova_debug_memory()


def same_memory(a, b):
    """Nothing left allocated: the pool's used bytes match, and the device's free
    bytes differ only by what the pool reserved or released meanwhile."""
    return a["pool_used"] == b["pool_used"] and a["free"] - b["free"] == b["pool_reserved"] - a["pool_reserved"]


def sweep(B, torch, call, max_k=64):
    """Fail allocation k = 1, 2, ... of `call`; returns the number of allocations
    the call makes (the first k at which it completes, minus one)."""
    call()                                   # warm-up: lazily created buffers exist from now on
    for k in range(1, max_k + 1):
        before = snapshot(B, torch)
        B.anova_debug_fail_alloc(k)
        try:
            call()
            done = True
        except B.AnovaError as e:
            assert e.status in (B.ENOMEM, B.ECUDA), (k, e.status)
            done = False
        finally:
            B.anova_debug_fail_alloc(0)
        after = snapshot(B, torch)
        if done:
            return k - 1
        assert same_memory(before, after), (k, before, after)
    raise AssertionError("the call made more allocations than the sweep covers")


@pytest.fixture(scope="module")
def problem(B, torch):
    w = W.random_problem(3000, 6, [(0, 1, 2), (3, 4), (5,)], 0.2, [16, 32, 32], 6, seed=91)
    w.epsB = 0.25
    X = torch.from_numpy(w.X).cuda()
    return w, X


def test_plan_creation_frees_on_failure(B, torch, problem):
    w, X = problem
    plans = []

    def call():
        plans.append(B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED))
        plans.pop().close()

    assert sweep(B, torch, call) > 10


def test_predict_and_model_free_on_failure(B, torch, problem):
    w, X = problem
    plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
    alpha = torch.from_numpy(w.alpha).cuda()
    # test points inside and partly outside the ball (the re-framed windows allocate too)
    Z = torch.from_numpy(np.concatenate([w.X[:400] * 0.9, w.X[400:500] * 1.6])).cuda()
    out = torch.empty(Z.shape[0], dtype=torch.float64, device="cuda")
    assert sweep(B, torch, lambda: B.krr_predict(plan, alpha, Z, out)) > 0

    def model_call():
        m = B.Model(plan, alpha)
        m.predict(Z, out)
        m.close()

    # a model builds grids in two frames per window and bins its test points per window: many allocations
    assert sweep(B, torch, model_call, max_k=400) > 0
    plan.close()


def test_solve_and_window_construction_free_on_failure(B, torch, problem):
    w, X = problem
    plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
    y = torch.from_numpy(w.y).cuda()
    a = torch.zeros_like(y)
    assert sweep(B, torch, lambda: B.krr_cg_solve(plan, 1e-1, y, a, 1e-8, 500)) > 0
    plan.close()
    labels = torch.from_numpy((w.X[:, 0] > 0).astype(np.int32)).cuda()
    assert sweep(B, torch, lambda: B.anova_mis(X, labels, 2)) > 0
    assert sweep(B, torch, lambda: B.anova_zscore_fit(X)) > 0
