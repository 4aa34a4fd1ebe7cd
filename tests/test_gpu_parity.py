"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative 2-norm): FP64 path vs the same-parameter oracle fast
summation 1e-12, FP32 path 1e-5; fast summation vs the direct sum 1e-5 where
the parameters reach it.  The GPU window is the Kaiser-Bessel window scaled to
psi(0) = 1, so its spread grid equals the oracle's divided by phi(0)^dims and
its multiplier D_k the oracle's times phi(0)^(2 dims).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2111_10140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

B_KB = oracle.kb_b(2.0)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


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


def phi0(m):
    return math.sinh(B_KB * m) / (math.pi * m)


def make_plan(B, torch, w, precision):
    X = torch.from_numpy(w.X).cuda()
    return B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                precision=precision)


def oracle_fast(w, Z=None, alpha=None):
    return oracle.fastsum(Z, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha if alpha is None else alpha,
                          sigma=w.sigma, epsB=w.epsB, p=w.p)


CASES = {
    "tiny_2d": lambda: W.plain_tiny(N=2000),
    "small_3d": lambda: W.random_problem(3000, 6, [(0, 1, 2), (3, 4, 5)], 0.2, 16, 4, seed=21),
    "mixed_dims_ragged": lambda: W.random_problem(2777, 7, [(0, 1, 2), (3, 4), (5,), (6,)], 0.25,
                                                  [16, 32, 64, 32], 5, seed=22),
    "overlapping": lambda: W.random_problem(1500, 4, [(0, 1, 2), (1, 2), (2, 3)], 0.3, 16, 3, seed=23),
}


@pytest.mark.parametrize("case", list(CASES))
def test_frame_and_multiplier_match_oracle(B, torch, case):
    w = CASES[case]()
    plan = make_plan(B, torch, w, B.FP64)
    for l, win in enumerate(w.windows):
        info = B.anova_plan_window(plan, l)
        c, s = oracle.window_frame(w.X, win, 0.25 - w.epsB / 2)
        np.testing.assert_allclose(info["centre"], c, rtol=0, atol=1e-15)
        assert info["scale"] == pytest.approx(s, rel=1e-14)
        dA, n, nos = len(win), w.n[l], 2 * w.n[l]
        re, _ = oracle.kernel_coeffs(dA, n, s * w.ell, w.epsB, w.p)
        D = oracle.diag(dA, n, nos, w.m, B_KB, re)
        Dg = B.anova_debug_diag(plan, l) / phi0(w.m) ** (2 * dA)
        assert rel(Dg, D) <= 1e-12


@pytest.mark.parametrize("case", list(CASES))
def test_spread_grid_matches_oracle(B, torch, case):
    w = CASES[case]()
    plan = make_plan(B, torch, w, B.MIXED)
    a64 = torch.from_numpy(w.alpha).cuda()
    for l, win in enumerate(w.windows):
        c, s = oracle.window_frame(w.X, win, 0.25 - w.epsB / 2)
        xt = s * (w.X[:, list(win)] - c)
        dA, nos = len(win), 2 * w.n[l]
        g_or = oracle.spread(xt, nos, w.m, B_KB, w.alpha) / phi0(w.m) ** dA
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            grid = torch.zeros((nos,) * dA, dtype=dt, device="cuda")
            B.anova_debug_spread(plan, l, a64.to(dt), grid)
            assert rel(grid.double().cpu().numpy(), g_or) <= tol, (l, dt)


@pytest.mark.parametrize("case", list(CASES))
def test_matvec_matches_oracle_fastsum(B, torch, case):
    w = CASES[case]()
    plan = make_plan(B, torch, w, B.MIXED)
    ref = oracle_fast(w)
    a64 = torch.from_numpy(w.alpha).cuda()
    out64 = torch.empty_like(a64)
    B.anova_matvec(plan, a64, out64)
    assert rel(out64.cpu().numpy(), ref) <= 1e-12
    a32 = a64.float()
    out32 = torch.empty_like(a32)
    B.anova_matvec(plan, a32, out32)
    assert rel(out32.cpu().numpy(), ref) <= 1e-5


def test_matvec_matches_direct_sum(B, torch):
    w = W.plain_tiny(N=2000)
    plan = make_plan(B, torch, w, B.FP32)
    direct = oracle.direct(w.X, w.X, w.windows, w.eta, w.ell, w.alpha)
    a = torch.from_numpy(w.alpha).float().cuda()
    out = torch.empty_like(a)
    B.anova_matvec(plan, a, out)
    assert rel(out.cpu().numpy(), direct) <= 1e-5


def test_multiple_rhs_and_weights(B, torch):
    w = W.random_problem(1200, 5, [(0, 1, 2), (3, 4)], 0.2, 16, 4, seed=31)
    eta = np.array([0.3, 1.7])
    X = torch.from_numpy(w.X).cuda()
    plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, weights=eta, precision=B.FP64)
    A = np.random.default_rng(2).standard_normal((3, w.N))
    out = torch.empty((3, w.N), dtype=torch.float64, device="cuda")
    B.anova_matvec(plan, torch.from_numpy(A).cuda(), out)
    for r in range(3):
        ref = oracle.fastsum(None, w.X, w.windows, eta, w.ell, w.n, w.m, A[r], epsB=w.epsB, p=w.p)
        assert rel(out[r].cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("N", [1, 2, 31, 1025])
def test_small_and_ragged_sizes(B, torch, N):
    w = W.random_problem(N, 3, [(0, 1, 2)], 0.2, 8, 2, seed=N)
    plan = make_plan(B, torch, w, B.FP64)
    ref = oracle_fast(w)
    a = torch.from_numpy(w.alpha).cuda()
    out = torch.empty_like(a)
    B.anova_matvec(plan, a, out)
    assert rel(out.cpu().numpy(), ref) <= 1e-12


def test_identical_points_degenerate_frame(B, torch):
    """All nodes equal: the frame has radius 0 (scale 1) and K is the all-ones matrix."""
    X = np.tile(np.array([[0.1, -0.2, 0.3]]), (50, 1))
    alpha = np.random.default_rng(0).standard_normal(50)
    plan = B.anova_fastsum_plan(torch.from_numpy(X).cuda(), [(0, 1, 2)], 0.2, n=16, m=4, precision=B.FP64)
    out = torch.empty(50, dtype=torch.float64, device="cuda")
    B.anova_matvec(plan, torch.from_numpy(alpha).cuda(), out)
    ref = oracle.fastsum(None, X, [(0, 1, 2)], [1.0], 0.2, [16], 4, alpha)
    assert rel(out.cpu().numpy(), ref) <= 1e-12
    assert rel(out.cpu().numpy(), np.full(50, alpha.sum())) <= 1e-6


def test_empty_problem(B, torch):
    X = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    plan = B.anova_fastsum_plan(X, [(0, 1, 2)], 0.2, n=16, m=4, precision=B.MIXED)
    a = torch.zeros(0, dtype=torch.float64, device="cuda")
    out = torch.zeros(0, dtype=torch.float64, device="cuda")
    B.anova_matvec(plan, a, out)
    st, its, relres = B.krr_cg_solve(plan, 1e-2, a, out, 1e-8, 10)
    assert st == B.OK and its[0] == 0


def test_cg_matches_oracle_and_dense_solve(B, torch):
    w = W.random_problem(400, 4, [(0, 1), (2, 3)], 0.15, 32, 4, seed=41)
    lam = 1e-2
    plan = make_plan(B, torch, w, B.FP64)
    y = torch.from_numpy(w.y).cuda()
    alpha = torch.zeros_like(y)
    st, its, relres = B.krr_cg_solve(plan, lam, y, alpha, 1e-10, 1000)
    assert st == B.OK and relres[0] <= 1e-10
    a_or, it_or, rel_or = oracle.cg(w.X, w.windows, w.eta, w.ell, w.n, w.m, lam, w.y, 1e-10, 1000,
                                    epsB=w.epsB, p=w.p)
    # CG in floating point: iteration counts agree up to rounding effects, and
    # both iterates solve the same system to 1e-10, so they differ by at most
    # about cond(K + lambda I) * 2e-10
    assert abs(int(its[0]) - it_or) <= max(3, it_or // 10)
    K = np.stack([oracle.direct(w.X, w.X, w.windows, w.eta, w.ell, e) for e in np.eye(w.N)], axis=1)
    cond = np.linalg.cond(K + lam * np.eye(w.N))
    assert rel(alpha.cpu().numpy(), a_or) <= 4 * cond * 1e-10


@pytest.mark.parametrize("precision", ["FP32", "MIXED"])
def test_cg_reduced_precision_reaches_tolerance(B, torch, precision):
    w = W.plain_tiny(N=2000)
    plan = make_plan(B, torch, w, getattr(B, precision))
    y = torch.from_numpy(w.y).cuda()
    alpha = torch.zeros_like(y)
    tol = 1e-8 if precision == "MIXED" else 1e-4
    st, its, relres = B.krr_cg_solve(plan, w.lam, y, alpha, tol, 3000)
    # mixed refinement meets tol on the FP64 residual; plain FP32 CG stops on its
    # recursive residual, and the FP32 operator error moves the true one a little
    assert st == B.OK and relres[0] <= (tol if precision == "MIXED" else 2 * tol)
    # the FP64 oracle operator agrees that alpha solves the system
    q = oracle_fast(w, alpha=alpha.cpu().numpy()) + w.lam * alpha.cpu().numpy()
    assert rel(q, w.y) <= (2e-8 if precision == "MIXED" else 3 * tol)


@pytest.mark.parametrize("form", ["fma", "mma.sync", "mma.sync pipelined", "mma.sync fp16 split"])
@pytest.mark.parametrize("precision", ["FP32", "MIXED"])
def test_cg_every_spread_form_reaches_tolerance(B, torch, form, precision):
    """CG feeds the FP32 operator FP64 vectors: every 3-D spread form (the FP16
    split one scales them by their largest entry first) must still solve the
    system.  Mixed refinement must meet tol on the FP64 residual, as the FP64
    oracle operator sees it.  Plain FP32 CG solves the FP32 operator's system:
    its recursive residual drifts from the true one (hence 10 tol on relres),
    and the FP64 operator sees the FP32 operator's error (about 1e-6 relative;
    the truncated TF32 heads of the TF32 forms round one way) amplified by the
    system's conditioning, so the oracle residual is held to 1e-2 there."""
    w = W.random_problem(3000, 6, [(0, 1, 2), (3, 4, 5)], 0.25, 32, 6, seed=61)
    w.epsB = 0.25
    plan = make_plan(B, torch, w, getattr(B, precision))
    B.anova_plan_set_kernels(plan, form, "tcgen05 persistent", 2)
    assert B.anova_plan_get_kernels(plan)["spread3"] == form
    y = torch.from_numpy(w.y).cuda()
    alpha = torch.zeros_like(y)
    tol = 1e-8 if precision == "MIXED" else 1e-4
    st, its, relres = B.krr_cg_solve(plan, w.lam, y, alpha, tol, 3000)
    assert st == B.OK and relres[0] <= (tol if precision == "MIXED" else 10 * tol)
    q = oracle_fast(w, alpha=alpha.cpu().numpy()) + w.lam * alpha.cpu().numpy()
    assert rel(q, w.y) <= (2e-8 if precision == "MIXED" else 1e-2)


@pytest.mark.parametrize("scale_z", [0.5, 1.7])
def test_predict_matches_oracle(B, torch, scale_z):
    w = W.random_problem(1500, 5, [(0, 1, 2), (3, 4)], 0.2, 32, 6, seed=51)
    w.epsB = 0.25
    Z = W.random_problem(333, 5, [(0, 1, 2), (3, 4)], 0.2, 32, 6, seed=52).X * scale_z
    plan = make_plan(B, torch, w, B.FP64)
    out = torch.empty(Z.shape[0], dtype=torch.float64, device="cuda")
    B.krr_predict(plan, torch.from_numpy(w.alpha).cuda(), torch.from_numpy(Z).cuda(), out)
    ref = oracle_fast(w, Z=Z)
    assert rel(out.cpu().numpy(), ref) <= 1e-12
    direct = oracle.direct(Z, w.X, w.windows, w.eta, w.ell, w.alpha)
    assert rel(out.cpu().numpy(), direct) <= 1e-5


def wide_rho(fr):
    """rho of a model's wide frame: largest value <= 2 with the Gaussian's
    Fourier transform at the band edge, exp(-(pi ell_l n / (2 rho))^2), below 1e-12."""
    return min(2.0, math.pi * fr["ell_l"] * fr["n"] / (2 * math.sqrt(math.log(1e12))))


def wide_frame_rows(w, frames):
    """Rows that make the oracle's joint frame (bounding-box midpoint, scale
    R_B / max radius of nodes and test points, Sec. 4.2) equal to the
    widened frame of each window: centre unchanged, scale / rho.  Every
    feature sits at its window's centre except one, moved by the wide radius
    along one axis of one window."""
    RB = 0.25 - 0.5 * w.epsB
    base = np.zeros(w.d)
    for win, fr in zip(w.windows, frames):
        base[list(win)] = fr["centre"]
    rows = []
    for win, fr in zip(w.windows, frames):
        r = wide_rho(fr) * RB / fr["scale"]
        for t, f in enumerate(win):
            for sgn in (-1.0, 1.0):
                row = base.copy()
                row[f] = fr["centre"][t] + sgn * r
                rows.append(row)
    return np.array(rows)


def radial_scaled(Z, w, frames, targets):
    """Z with each (disjoint) window's features scaled about the window centre
    so that the window's largest test-point radius equals targets[l]."""
    Z = Z.copy()
    for win, fr, tr in zip(w.windows, frames, targets):
        dz = Z[:, list(win)] - fr["centre"]
        Z[:, list(win)] = fr["centre"] + dz * (tr / np.linalg.norm(dz, axis=1).max())
    return Z


@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_model_predict_matches_oracle(B, torch, precision):
    """krr_model: the convolved grids computed once give the oracle's fast
    summation (FP64 1e-12, FP32 1e-5) for test points inside the nodes' ball
    (plan frame), for points beyond it but inside rho times its radius (wide
    frame: the oracle's joint frame is pinned to it by extra rows) and for
    points further out (per-window summation in the joint frame, as
    krr_predict); all three within 1e-5 of the direct sum.  Several host
    threads on their own streams predicting on one model give the serial
    results."""
    import threading
    wins = [(0, 1, 2), (3, 4), (5,)]
    w = W.random_problem(2500, 6, wins, 0.3, 32, 6, seed=53)
    w.epsB = 0.25
    Zraw = W.random_problem(777, 6, wins, 0.3, 32, 6, seed=54).X
    plan = make_plan(B, torch, w, getattr(B, precision))
    frames = [B.anova_plan_window(plan, l) for l in range(len(wins))]
    RB = 0.25 - 0.5 * w.epsB
    rX = [RB / fr["scale"] for fr in frames]              # nodes' largest radius per window
    rho = [wide_rho(fr) for fr in frames]
    assert min(rho) > 1.2
    alpha = torch.from_numpy(w.alpha).cuda()
    model = B.Model(plan, alpha)
    del alpha                                 # the model holds its own copy
    tol = 1e-12 if precision == "FP64" else 1e-5
    cases = [
        (radial_scaled(Zraw, w, frames, [0.9 * r for r in rX]), None),
        (radial_scaled(Zraw, w, frames, [0.5 * (1 + q) * r for q, r in zip(rho, rX)]),
         wide_frame_rows(w, frames)),
        (radial_scaled(Zraw, w, frames, [1.3 * q * r for q, r in zip(rho, rX)]), None),
    ]
    for Z, extra in cases:
        Zt = torch.from_numpy(np.ascontiguousarray(Z)).cuda()
        out = torch.empty(Z.shape[0], dtype=torch.float64, device="cuda")
        model.predict(Zt, out)
        got = out.cpu().numpy()
        Zo = Z if extra is None else np.vstack([Z, extra])
        ref = oracle_fast(w, Z=Zo)[:Z.shape[0]]
        assert rel(got, ref) <= tol
        assert rel(got, oracle.direct(Z, w.X, w.windows, w.eta, w.ell, w.alpha)) <= 1e-5
    Zin = cases[0][0]
    Zt = torch.from_numpy(Zin).cuda()
    out = torch.empty(Zin.shape[0], dtype=torch.float64, device="cuda")
    model.predict(Zt, out)
    serial = out.cpu().numpy()
    outs = [torch.full_like(out, float("nan")) for _ in range(4)]
    torch.cuda.synchronize()
    errs = []

    def work(k):
        try:
            s = torch.cuda.Stream()
            for _ in range(5):
                model.predict(Zt, outs[k], stream=s)
        except Exception as e:   # reported below
            errs.append(e)

    ts = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    for o in outs:
        assert rel(o.cpu().numpy(), serial) <= (1e-13 if precision == "FP64" else 1e-6)
    model.close()


def test_repeat_runs_agree(B, torch):
    w = W.random_problem(5000, 3, [(0, 1, 2)], 0.2, 32, 6, seed=61)
    plan = make_plan(B, torch, w, B.MIXED)
    for dt, tol in ((torch.float64, 1e-14), (torch.float32, 1e-6)):
        a = torch.from_numpy(w.alpha).to(dt).cuda()
        o1, o2 = torch.empty_like(a), torch.empty_like(a)
        B.anova_matvec(plan, a, o1)
        B.anova_matvec(plan, a, o2)
        assert rel(o1.cpu().numpy(), o2.cpu().numpy()) <= tol


@pytest.mark.slow
def test_full_mid_workload_parity(B, torch):
    """N = 1e5, three 3-D windows (n = 32, m = 6): every output against the oracle."""
    w = W.plain_mid()
    plan = make_plan(B, torch, w, B.MIXED)
    ref = oracle_fast(w)
    a64 = torch.from_numpy(w.alpha).cuda()
    out = torch.empty_like(a64)
    B.anova_matvec(plan, a64, out)
    assert rel(out.cpu().numpy(), ref) <= 1e-12
    a32 = a64.float()
    out32 = torch.empty_like(a32)
    B.anova_matvec(plan, a32, out32)
    assert rel(out32.cpu().numpy(), ref) <= 1e-5
    idx = np.random.default_rng(7).choice(w.N, 500, replace=False)
    direct = oracle.direct(w.X[idx], w.X, w.windows, w.eta, w.ell, w.alpha)
    assert rel(out32.cpu().numpy()[idx], direct) <= 1e-5
    # the launch configuration the benchmark times: 3-D bins of 4 cells (region 16)
    X = torch.from_numpy(w.X).cuda()
    plan16 = B.anova_fastsum_plan_bins(X, w.windows, w.ell, [0, 0, 4], n=w.n, m=w.m, sigma=w.sigma,
                                       eps_B=w.epsB, p=w.p, precision=B.MIXED)
    assert B.anova_plan_window_bins(plan16, 0)["region"] == 16
    B.anova_matvec(plan16, a64, out)
    assert rel(out.cpu().numpy(), ref) <= 1e-12
    B.anova_matvec(plan16, a32, out32)
    assert rel(out32.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("n,m", [(64, 6), (16, 7), (16, 5), (16, 3), (8, 1)])
def test_dense_region_sizes(B, torch, n, m):
    """3-D windows on the dense kernels with other region sizes R = Tb + 2m:
    n = 64 (bin side 4, R = 16), m = 7 (R = 16), m = 5 (R = 12), m = 3 (R = 8), m = 1 (R = 4)."""
    w = W.random_problem(4000, 3, [(0, 1, 2)], 0.25, n, m, seed=80 + m + n)
    w.epsB = 0.25
    plan = make_plan(B, torch, w, B.MIXED)
    ref = oracle_fast(w)
    a64 = torch.from_numpy(w.alpha).cuda()
    out64 = torch.empty_like(a64)
    B.anova_matvec(plan, a64, out64)
    assert rel(out64.cpu().numpy(), ref) <= 1e-12
    a32 = a64.float()
    out32 = torch.empty_like(a32)
    B.anova_matvec(plan, a32, out32)
    assert rel(out32.cpu().numpy(), ref) <= 1e-5


def test_graph_replay_matches_direct_calls(B, torch):
    """anova_matvec replays a captured launch sequence from the second call on;
    new inputs in the same buffers must give new results."""
    w = W.random_problem(3000, 6, [(0, 1, 2), (3, 4, 5)], 0.2, 16, 4, seed=91)
    plan = make_plan(B, torch, w, B.MIXED)
    a = torch.from_numpy(w.alpha).float().cuda()
    out = torch.empty_like(a)
    rng = np.random.default_rng(3)
    for call in range(4):
        vals = rng.standard_normal(w.N)
        a.copy_(torch.from_numpy(vals).float())
        B.anova_matvec(plan, a, out)
        ref = oracle_fast(w, alpha=vals)
        assert rel(out.cpu().numpy(), ref) <= 1e-5, call


@pytest.mark.parametrize("n,m,epsB", [(4, 1, 0.25), (8, 3, 0.25), (16, 7, 0.25), (32, 6, 0.25), (64, 7, 0.25),
                                      (64, 6, 1 / 16), (128, 6, 0.25)])
def test_dense_small_windows(B, torch, n, m, epsB):
    """1-D and 2-D windows on the dense FP32 kernels (and the generic FP64 ones);
    their FFT on the batched box kernel where it fits one block's shared
    memory (a box that covers the whole grid at n = 16, m = 7; n = 128 falls
    back to the per-axis kernels in 2-D)."""
    w = W.random_problem(5000, 3, [(0,), (1, 2)], 0.25, n, m, seed=100 + n + m)
    w.epsB = epsB
    plan = make_plan(B, torch, w, B.MIXED)
    ref = oracle_fast(w)
    a64 = torch.from_numpy(w.alpha).cuda()
    out64 = torch.empty_like(a64)
    B.anova_matvec(plan, a64, out64)
    assert rel(out64.cpu().numpy(), ref) <= 1e-12
    a32 = a64.float()
    out32 = torch.empty_like(a32)
    B.anova_matvec(plan, a32, out32)
    assert rel(out32.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("dtype,tol", [("FP64", 1e-12), ("FP32", 1e-5)])
def test_direct_matvec_matches_oracle_direct(B, torch, dtype, tol):
    w = W.random_problem(1500, 7, [(0, 1, 2), (3, 4), (5,), (6,)], 0.2, 16, 4, seed=111)
    Z = W.random_problem(700, 7, [(0, 1, 2), (3, 4), (5,), (6,)], 0.2, 16, 4, seed=112).X
    eta = np.array([0.1, 0.2, 0.3, 0.4])
    out = torch.empty(Z.shape[0], dtype=torch.float64, device="cuda")
    B.anova_direct_matvec(torch.from_numpy(Z).cuda(), torch.from_numpy(w.X).cuda(), w.windows, w.ell,
                          torch.from_numpy(w.alpha).cuda(), out, weights=eta, dtype=getattr(B, dtype))
    ref = oracle.direct(Z, w.X, w.windows, eta, w.ell, w.alpha)
    assert rel(out.cpu().numpy(), ref) <= tol


@pytest.mark.slow
def test_precision_form_full_size_sampled(B, torch):
    """The precision form at its full size (N = 1e6, d = 28, nine windows of 1-3
    features): on 256 sampled rows the FP64 product is within the fast
    summation's error of the oracle's direct sum (1e-6 at these parameters) and
    the FP32 product within 1e-5; over all rows FP32 agrees with FP64 to 1e-5."""
    w = W.precision_form()
    X = torch.from_numpy(w.X).cuda()
    plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                precision=B.MIXED)
    a64 = torch.from_numpy(w.alpha).cuda()
    o64 = torch.empty_like(a64)
    B.anova_matvec(plan, a64, o64)
    a32 = a64.float()
    o32 = torch.empty_like(a32)
    B.anova_matvec(plan, a32, o32)
    g64, g32 = o64.cpu().numpy(), o32.double().cpu().numpy()
    assert rel(g32, g64) <= 1e-5
    idx = np.sort(np.random.default_rng(11).choice(w.N, 256, replace=False))
    direct = oracle.direct(w.X[idx], w.X, w.windows, w.eta, w.ell, w.alpha)
    assert rel(g64[idx], direct) <= 1e-6
    assert rel(g32[idx], direct) <= 1e-5
    plan.close()
