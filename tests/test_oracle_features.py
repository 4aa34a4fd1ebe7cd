"""Pins of the window-construction reference (oracle/features.py) to facts
fixed by the definitions (Sec. 5, Sec. 6.1) and by information theory."""
import math

import numpy as np

from oracle import features as F


def test_zscore_hand_example():
    X = np.array([[1.0, 5.0], [3.0, 5.0], [5.0, 5.0]])
    mean, std = F.zscore_fit(X)
    assert np.allclose(mean, [3.0, 5.0])
    assert np.allclose(std, [math.sqrt(8.0 / 3.0), 1.0])      # constant column: std 1
    Z = F.zscore_apply(X, mean, std)
    assert np.allclose(Z[:, 0], np.array([-2.0, 0.0, 2.0]) / math.sqrt(8.0 / 3.0))
    assert np.allclose(Z[:, 1], 0.0)


def test_zscore_moments_and_test_split():
    rng = np.random.default_rng(1)
    X = rng.standard_t(3.0, size=(5000, 4)) * [1, 10, 0.1, 3] + [0, 5, -2, 1]
    mean, std = F.zscore_fit(X)
    Z = F.zscore_apply(X, mean, std)
    assert np.allclose(Z.mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(Z.std(axis=0), 1.0, atol=1e-12)
    T = rng.standard_normal((10, 4))
    assert np.allclose(F.zscore_apply(T, mean, std), (T - mean) / std)   # training statistics only


def test_fine_index_edges():
    assert F.fine_index(0.0, 0.0, 1.0, 8) == 0
    assert F.fine_index(1.0, 0.0, 1.0, 8) == 7          # the last bin is closed
    assert F.fine_index(0.5, 0.0, 1.0, 8) == 4
    assert F.fine_index(0.4999, 0.0, 1.0, 8) == 3
    assert F.fine_index(3.0, 3.0, 3.0, 8) == 0          # constant column


def test_quantile_bins_equal_counts():
    # distinct values, N a multiple of B: every quantile bin holds N / B values
    rng = np.random.default_rng(2)
    col = rng.permutation(np.arange(1600, dtype=float)) ** 1.5
    q = F.quantile_bins(col, 16, F=1 << 20)
    assert np.array_equal(np.bincount(q, minlength=16), np.full(16, 100))
    # monotone: a larger value never lands in a lower bin
    o = np.argsort(col)
    assert np.all(np.diff(q[o]) >= 0)


def test_mis_independent_label_is_zero():
    # joint counts that factorise exactly: every bin holds both classes equally
    col = np.repeat(np.arange(16, dtype=float), 10)
    labels = np.tile(np.array([0, 1] * 5), 16)
    assert abs(F.mis(col[:, None], labels, 2)[0]) < 1e-15


def test_mis_deterministic_label_is_entropy():
    # label a function of the bin: I(X; Y) = H(Y); two balanced classes -> ln 2
    col = np.arange(320, dtype=float)
    labels = (F.quantile_bins(col, 16) >= 8).astype(int)
    assert abs(F.mis(col[:, None], labels, 2)[0] - math.log(2.0)) < 1e-14
    # four balanced classes -> ln 4
    labels4 = F.quantile_bins(col, 16) // 4
    assert abs(F.mis(col[:, None], labels4, 4)[0] - math.log(4.0)) < 1e-14


def test_mis_matches_histogram_formula_by_brute_force():
    # the plug-in MI equals H(Y) - H(Y | Q) computed from the same bins
    rng = np.random.default_rng(3)
    X = rng.standard_normal((600, 3))
    y = (X[:, 0] + 0.5 * rng.standard_normal(600) > 0).astype(int)
    m = F.mis(X, y, 2, B=8)
    for f in range(3):
        q = F.quantile_bins(X[:, f], 8)
        py = np.bincount(y, minlength=2) / 600
        hy = -sum(p * math.log(p) for p in py if p > 0)
        hyq = 0.0
        for a in range(8):
            sel = q == a
            if sel.sum() == 0:
                continue
            pa = sel.mean()
            pya = np.bincount(y[sel], minlength=2) / sel.sum()
            hyq += pa * -sum(p * math.log(p) for p in pya if p > 0)
        assert abs(m[f] - (hy - hyq)) < 1e-12
    assert m[0] > 5 * max(m[1], m[2])     # the informative feature ranks first


def test_windows_from_mis_grouping():
    s = [0.1, 0.9, 0.0, 0.5, 0.5, 0.3, 0.7, 0.05]
    assert F.windows_from_mis(s, 0.0) == [(1, 6, 3), (4, 5, 0), (7, 2)]
    assert F.windows_from_mis(s, 0.06) == [(1, 6, 3), (4, 5, 0)]
    assert F.windows_from_mis(s, 0.2) == [(1, 6, 3), (4, 5)]
    assert F.windows_from_mis(s, 1.0) == []
