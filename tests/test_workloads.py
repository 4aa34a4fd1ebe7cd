"""The seeded input generators produce what the input recipes state: shapes,
windows, parameters, the caller-side mapping into the ball, determinism per
seed (every GPU test and the benchmark rely on the same arrays for a seed)."""
import numpy as np
import pytest

from paper_2111_10140_gb300 import workloads as W


def _in_ball(w, radius=W.R_B):
    for win in w.windows:
        r = np.linalg.norm(w.X[:, list(win)], axis=1)
        assert r.max() <= radius * (1 + 1e-12)
        a = radius / np.sqrt(len(win))
        for f in win:   # every feature of a window spans exactly [-a, a]
            assert w.X[:, f].min() == pytest.approx(-a, abs=1e-15)
            assert w.X[:, f].max() == pytest.approx(a, abs=1e-15)


def test_plain_tiny_recipe():
    w = W.plain_tiny()
    assert (w.N, w.d) == (2000, 6)
    assert w.windows == [(0, 1), (2, 3), (4, 5)]
    assert (w.ell, w.n, w.m, w.sigma, w.lam, w.tol, w.epsB, w.p) == (0.1, [32] * 3, 4, 2.0, 1e-2, 1e-8, 1 / 16, 8)
    np.testing.assert_allclose(w.eta, 1 / 3)
    _in_ball(w)


def test_plain_mid_recipe():
    w = W.plain_mid()
    assert (w.N, w.d) == (100_000, 9)
    assert w.windows == [(0, 1, 2), (3, 4, 5), (6, 7, 8)]
    assert (w.ell, w.n, w.m, w.lam, w.tol, w.epsB) == (0.2, [32] * 3, 6, 1e-3, 1e-6, 0.25)
    _in_ball(w)


def test_precision_form_recipe_small_n():
    w = W.precision_form(N=20_000)
    assert w.d == 28
    assert [len(x) for x in w.windows] == [3, 3, 3, 2, 2, 2, 2, 1, 1]
    assert sorted(f for x in w.windows for f in x) == list(range(19))   # features 19..27 unused
    assert w.n == [32, 32, 32, 64, 64, 64, 64, 64, 64]
    assert (w.ell, w.m, w.lam, w.tol, w.epsB) == (0.25, 6, 1e-2, 1e-8, 0.25)
    assert w.meta["heavy_tailed"] == [0, 4, 8, 10, 13, 17]
    _in_ball(w)


@pytest.mark.parametrize("make", [lambda s: W.plain_tiny(seed=s), lambda s: W.plain_mid(N=5000, seed=s),
                                  lambda s: W.precision_form(N=3000, seed=s),
                                  lambda s: W.serving_problem(3000, s, M_test=100),
                                  lambda s: W.batch_problem(2000, s)])
def test_same_seed_same_arrays(make):
    a, b, c = make(5), make(5), make(6)
    for f in ("X", "alpha", "y"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
        assert not np.array_equal(getattr(a, f), getattr(c, f))


def test_serving_problem_ranges():
    for seed in range(20):
        w = W.serving_problem(2000, seed, M_test=50)
        assert 9 <= w.d <= 28 and 1 <= len(w.windows) <= 9
        feats = [f for x in w.windows for f in x]
        assert len(feats) == len(set(feats)) and all(0 <= f < w.d for f in feats)
        assert all(1 <= len(x) <= 3 for x in w.windows)
        assert w.n == [32 if len(x) == 3 else 64 for x in w.windows]
        assert w.meta["Z"].shape == (50, w.d)
        # training and held-out rows were mapped together: all of them inside the ball
        for win in w.windows:
            allr = np.linalg.norm(np.vstack([w.X, w.meta["Z"]])[:, list(win)], axis=1)
            assert allr.max() <= W.R_B * (1 + 1e-12)


def test_batch_form_shapes():
    probs = W.batch_form(count=12, seed=3, nrhs=4)
    assert len(probs) == 12
    for w in probs:
        assert 2 ** 10 - 1 <= w.N <= 2 ** 17 + 1
        assert 6 <= w.d <= 15 and 1 <= len(w.windows) <= 5
        assert 0.05 <= w.ell <= 0.5 and 1e-4 <= w.lam <= 1e-1
        assert w.meta["Y"].shape == (4, w.N)
        assert np.array_equal(w.y, w.meta["Y"][0])
        _in_ball(w)
