"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the fast summation: it only draws points,
coefficients and right-hand sides with numpy's ``default_rng`` and applies the
caller-side preprocessing (per-feature min-max mapping into the ball, Sec. 6.1
"z-score normalised" data).  Both the CUDA library's tests and the oracle
consume the arrays it returns.

The paper's five data sets (Sec. 6, Telescope, HIGGS, SUSY, YearPredictionMSD,
cod-rna) are not available; these generators stand in for them with the same
shapes (N up to 1e6, d from 6 to 28, windows of 1-3 features, Sec. 5).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

EPS_B = 1.0 / 16
R_B = 0.25 - EPS_B / 2          # radius of the ball the nodes are mapped into


@dataclass
class Workload:
    name: str
    X: np.ndarray                 # N x d, float64, row-major
    windows: list                 # list of tuples of 0-based feature indices
    eta: np.ndarray               # P weights
    ell: float                    # Gaussian width, kernel exp(-||x-y||^2/ell^2)
    n: list                       # bandwidth per window
    m: int                        # window cutoff
    sigma: float                  # oversampling
    alpha: np.ndarray             # N coefficients for single matvecs
    y: np.ndarray                 # KRR right-hand side
    lam: float                    # ridge parameter lambda
    tol: float                    # CG relative residual target
    epsB: float = EPS_B           # regularisation width of the fast summation
    p: int = 8                    # two-point Taylor degree parameter (degree 2p-1)
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.X.shape[0]

    @property
    def d(self):
        return self.X.shape[1]


def _minmax_into_ball(X, windows, radius=R_B):
    """Per feature, map [min, max] affinely onto [-a, a] with a = radius/sqrt(|W|),
    so every window's points lie in the ball of the given radius."""
    Xs = X.copy()
    for w in windows:
        a = radius / np.sqrt(len(w))
        for f in w:
            lo, hi = X[:, f].min(), X[:, f].max()
            span = hi - lo if hi > lo else 1.0
            Xs[:, f] = -a + 2.0 * a * (X[:, f] - lo) / span
    return Xs


def _unit(X):
    lo, hi = X.min(axis=0), X.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    return (X - lo) / span


def plain_tiny(N=2000, seed=0):
    """N=2000, d=6 uniform features, 2-D windows {1,2},{3,4},{5,6}, ell=0.1,
    n=32, m=4, sigma=2; lambda=1e-2, tol 1e-8."""
    rng = np.random.default_rng(seed)
    raw = rng.uniform(0.0, 1.0, size=(N, 6))
    windows = [(0, 1), (2, 3), (4, 5)]
    X = _minmax_into_ball(raw, windows)
    alpha = rng.standard_normal(N)
    y = np.sin(2 * np.pi * raw[:, 0]) + raw[:, 2] * raw[:, 3] + 0.1 * rng.standard_normal(N)
    P = len(windows)
    return Workload("plain_tiny_N2000_d6_3x2D", X, windows, np.full(P, 1.0 / P), 0.1,
                    [32] * P, 4, 2.0, alpha, y, 1e-2, 1e-8)


def plain_mid(N=100_000, seed=1):
    """N=1e5, d=9 standard normal features min-max scaled per window,
    3-D windows {1,2,3},{4,5,6},{7,8,9}, ell=0.2, n=32, m=6, sigma=2;
    lambda=1e-3, tol 1e-6."""
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((N, 9))
    windows = [(0, 1, 2), (3, 4, 5), (6, 7, 8)]
    X = _minmax_into_ball(raw, windows)
    u = _unit(raw)
    alpha = rng.standard_normal(N)
    y = sum(np.sin(2 * np.pi * u[:, list(w)].mean(axis=1)) for w in windows)
    y = y + 0.05 * rng.standard_normal(N)
    P = len(windows)
    return Workload("plain_mid_N100000_d9_3x3D", X, windows, np.full(P, 1.0 / P), 0.2,
                    [32] * P, 6, 2.0, alpha, y, 1e-3, 1e-6, epsB=0.25)


def precision_form(N=1_000_000, seed=2):
    """N=1e6, d=28 standardised features, columns {0,4,8,10,13,17} Student-t(3);
    windows 3x3-D, 4x2-D, 2x1-D; ell=0.25; n=64 (1-D/2-D), 32 (3-D); m=6;
    lambda=1e-2, tol 1e-8."""
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((N, 28))
    heavy = [0, 4, 8, 10, 13, 17]
    for c in heavy:
        t = rng.standard_t(3.0, size=N)
        raw[:, c] = (t - t.mean()) / t.std()
    windows = [(0, 1, 2), (3, 4, 5), (6, 7, 8), (9, 10), (11, 12), (13, 14), (15, 16), (17,), (18,)]
    X = _minmax_into_ball(raw, windows)
    u = _unit(raw)
    alpha = rng.standard_normal(N)
    y = sum(np.sin(2 * np.pi * u[:, list(w)].mean(axis=1)) for w in windows)
    y = y + 0.05 * rng.standard_normal(N)
    P = len(windows)
    n = [32 if len(w) == 3 else 64 for w in windows]
    return Workload(f"precision_N{N}_d28_mixed", X, windows, np.full(P, 1.0 / P), 0.25,
                    n, 6, 2.0, alpha, y, 1e-2, 1e-8, epsB=0.25,
                    meta={"heavy_tailed": heavy})


def random_problem(N, d, windows, ell, n, m, seed, dist="normal"):
    """Generic generator for tests: points min-max mapped into the ball."""
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((N, d)) if dist == "normal" else rng.uniform(0, 1, (N, d))
    X = _minmax_into_ball(raw, windows)
    alpha = rng.standard_normal(N)
    P = len(windows)
    nv = list(n) if hasattr(n, "__len__") else [n] * P
    y = rng.standard_normal(N)
    return Workload(f"random_N{N}_d{d}", X, windows, np.full(P, 1.0 / P), ell, nv, m, 2.0,
                    alpha, y, 1e-2, 1e-8)


CONFIGS = {"plain_tiny": plain_tiny, "plain_mid": plain_mid, "precision_form": precision_form}


def serving_problem(N, seed, M_test=0):
    """One problem of the serving stream: d uniform in 9..28 standard normal
    features, 3..9 windows of 1-3 distinct features (n = 32 for 3-D windows,
    64 otherwise, m = 6, eps_B = 0.25), ell = 0.25, lambda = 1e-2, y a sum of
    per-window smooth functions plus noise.  With M_test > 0 another M_test
    rows are drawn with the training rows and min-max mapped together with
    them (a held-out split); they are returned in meta["Z"]."""
    rng = np.random.default_rng(seed)
    d = int(rng.integers(9, 29))
    P = int(rng.integers(3, 10))
    feats = list(rng.permutation(d))
    windows = []
    while len(windows) < P and feats:
        k = min(int(rng.integers(1, 4)), len(feats))
        windows.append(tuple(sorted(int(f) for f in feats[:k])))
        feats = feats[k:]
    raw = rng.standard_normal((N + M_test, d))
    Xall = _minmax_into_ball(raw, windows)
    u = _unit(raw[:N])
    y = sum(np.sin(2 * np.pi * u[:, list(w)].mean(axis=1)) for w in windows) + 0.05 * rng.standard_normal(N)
    P = len(windows)
    n = [32 if len(w) == 3 else 64 for w in windows]
    return Workload(f"serving_N{N}_d{d}_P{P}", np.ascontiguousarray(Xall[:N]), windows, np.full(P, 1.0 / P), 0.25,
                    n, 6, 2.0, rng.standard_normal(N), y, 1e-2, 1e-6, epsB=0.25,
                    meta={"Z": np.ascontiguousarray(Xall[N:])})


def batch_problem(N, seed, nrhs=16, lam_range=(1e-4, 1e-1)):
    """One problem of the batching form: d uniform in 6..15 standard normal
    features, windows of 1-3 distinct features covering at most all of them,
    ell log-uniform in [0.05, 0.5], lambda log-uniform in [1e-4, 1e-1], nrhs
    right-hand sides N(0, 1) (meta["Y"], nrhs x N); m = 6, eps_B = 0.25, n = 16
    (3-D, ell >= 0.15) or 32 (3-D) and 32 / 64 for 1-D and 2-D (64 when
    ell < 0.1)."""
    rng = np.random.default_rng(seed)
    d = int(rng.integers(6, 16))
    feats = list(rng.permutation(d))
    windows = []
    while feats and len(windows) < 5:
        k = min(int(rng.integers(1, 4)), len(feats))
        windows.append(tuple(sorted(int(f) for f in feats[:k])))
        feats = feats[k:]
    ell = float(10 ** rng.uniform(np.log10(0.05), np.log10(0.5)))
    lam = float(10 ** rng.uniform(np.log10(lam_range[0]), np.log10(lam_range[1])))
    raw = rng.standard_normal((N, d))
    X = _minmax_into_ball(raw, windows)
    n = [(16 if ell >= 0.15 else 32) if len(w) == 3 else (64 if ell < 0.1 else 32) for w in windows]
    P = len(windows)
    Y = rng.standard_normal((nrhs, N))
    return Workload(f"batch_N{N}_d{d}_P{P}", X, windows, np.full(P, 1.0 / P), ell, n, 6, 2.0,
                    rng.standard_normal(N), Y[0].copy(), lam, 1e-6, epsB=0.25, meta={"Y": Y})


def batch_form(count=64, seed=3, nrhs=16, lam_range=(1e-4, 1e-1)):
    """The batching form: `count` problems with N log-uniform in [2^10, 2^17]."""
    rng = np.random.default_rng(seed)
    Ns = np.round(2.0 ** rng.uniform(10, 17, size=count)).astype(int)
    return [batch_problem(int(N), seed=10_000 * seed + k, nrhs=nrhs, lam_range=lam_range)
            for k, N in enumerate(Ns)]
