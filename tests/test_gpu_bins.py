"""Bin sides other than the default rule (anova_fastsum_plan_bins) give the
oracle's fast summation, and the autotuner returns sides a plan takes."""
import numpy as np
import pytest

import oracle
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


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


WINS = [(0, 1, 2), (3, 4), (5,)]


@pytest.mark.parametrize("sides", [(2, 2, 4), (4, 4, 2), (2, 4, 4), (4, 2, 2)])
def test_bin_sides_match_oracle(B, torch, sides):
    w = W.random_problem(4000, 6, WINS, 0.25, [32, 32, 32], 6, seed=700 + sum(sides))
    w.epsB = 0.25
    X = torch.from_numpy(w.X).cuda()
    plan = B.anova_fastsum_plan_bins(X, w.windows, w.ell, sides, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
    for l, win in enumerate(WINS):
        info = B.anova_plan_window_bins(plan, l)
        assert info["dense"] and info["bin_side"] == sides[len(win) - 1]
        assert info["region"] == sides[len(win) - 1] + 2 * w.m
    ref = oracle.fastsum(None, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha, sigma=w.sigma, epsB=w.epsB, p=w.p)
    a64 = torch.from_numpy(w.alpha).cuda()
    o64 = torch.empty_like(a64)
    B.anova_matvec(plan, a64, o64)
    assert rel(o64.cpu().numpy(), ref) <= 1e-12
    a32 = a64.float()
    o32 = torch.empty_like(a32)
    B.anova_matvec(plan, a32, o32)
    assert rel(o32.cpu().numpy(), ref) <= 1e-5


def test_inadmissible_side_falls_back(B, torch):
    w = W.random_problem(2000, 3, [(0, 1, 2)], 0.25, 32, 6, seed=710)
    X = torch.from_numpy(w.X).cuda()
    plan = B.anova_fastsum_plan_bins(X, w.windows, w.ell, (0, 0, 6), n=w.n, m=w.m, precision=B.FP32)
    info = B.anova_plan_window_bins(plan, 0)
    assert info["bin_side"] == 2 and info["region"] == 14    # 6 + 2 m > 16: the default rule


def test_autotune_returns_sides_a_plan_takes(B, torch):
    w = W.random_problem(20000, 6, WINS, 0.25, [32, 32, 32], 6, seed=720)
    w.epsB = 0.25
    X = torch.from_numpy(w.X).cuda()
    sides, ms = B.anova_autotune_bins(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.FP32, reps=5)
    assert ms > 0
    plan = B.anova_fastsum_plan_bins(X, w.windows, w.ell, sides, n=w.n, m=w.m, eps_B=w.epsB, precision=B.FP32)
    for l, win in enumerate(WINS):
        s = sides[len(win) - 1]
        if s:
            assert B.anova_plan_window_bins(plan, l)["bin_side"] == s


def test_binning_of_long_histograms_matches_oracle(B, torch):
    """N = 20000 nodes in a 3-D window of 32768 bins: the bins x chunks
    histogram (98304 counts) goes through the multi-block scan; the FP64 product
    must still be the oracle's."""
    w = W.random_problem(20000, 4, [(0, 1, 2), (3,)], 0.25, [32, 32], 6, seed=720)
    w.epsB = 0.25
    X = torch.from_numpy(w.X).cuda()
    plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
    info = B.anova_plan_window_bins(plan, 0)
    nbins = (2 * w.n[0] // info["bin_side"]) ** 3
    assert nbins * ((w.N + 8191) // 8192) > 4 * 8192
    ref = oracle.fastsum(None, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha, sigma=w.sigma, epsB=w.epsB, p=w.p)
    a64 = torch.from_numpy(w.alpha).cuda()
    o64 = torch.empty_like(a64)
    B.anova_matvec(plan, a64, o64)
    assert rel(o64.cpu().numpy(), ref) <= 1e-12
    o32 = torch.empty_like(a64.float())
    B.anova_matvec(plan, a64.float(), o32)
    assert rel(o32.cpu().numpy(), ref) <= 1e-5


def test_autotune_kernels_sets_forms_that_keep_the_oracle_product(B, torch):
    """anova_autotune_kernels leaves the plan on the forms it reports, and the
    FP32 product on those forms is still the oracle's to the FP32 bar; every
    form it can pick is checked the same way."""
    w = W.random_problem(20000, 6, WINS, 0.25, [32, 32, 32], 6, seed=730)
    w.epsB = 0.25
    X = torch.from_numpy(w.X).cuda()
    plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
    ref = oracle.fastsum(None, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha, sigma=w.sigma, epsB=w.epsB, p=w.p)
    a32 = torch.from_numpy(w.alpha).cuda().float()
    o32 = torch.empty_like(a32)
    choice, ms = B.anova_autotune_kernels(plan, reps=3)
    assert ms > 0
    assert choice["spread3"] in B.SPREAD3_FORMS and choice["gather3"] in B.GATHER3_FORMS
    assert choice["schedule"] in (0, 1, 2, 3)
    names = B.anova_dense3_kernels(plan)
    spread_name = {"fma": "k_spread3_f32<R>", "mma.sync": "k_spread3_tc<R>",
                   "mma.sync pipelined": "k_spread3_tcp<R>",
                   "mma.sync fp16 split": "k_spread3_tch<R>"}[choice["spread3"]]
    assert names["spread"] == spread_name
    if choice["gather3"] == "fma":
        assert names["gather"] == "k_gather3_f32<R>"
    B.anova_matvec(plan, a32, o32)
    assert rel(o32.cpu().numpy(), ref) <= 1e-5
    assert B.anova_plan_get_kernels(plan) == choice
    # each form the tuner chooses between gives the oracle's product
    for sp in B.SPREAD3_FORMS:
        for ga in B.GATHER3_FORMS:
            for mode in (0, 1, 2, 3):
                B.anova_plan_set_kernels(plan, sp, ga, mode)
                assert B.anova_plan_get_kernels(plan) == {"spread3": sp, "gather3": ga, "schedule": mode}
                o32.zero_()
                B.anova_matvec(plan, a32, o32)
                assert rel(o32.cpu().numpy(), ref) <= 1e-5, (sp, ga, mode)
    with pytest.raises(B.AnovaError):
        B.anova_autotune_kernels(plan, reps=0)
