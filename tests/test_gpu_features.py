"""Window construction on the GPU (z-score, mutual information score, grouping)
against the plain reference in oracle/features.py (Sec. 5, Sec. 6.1)."""
import numpy as np
import pytest

from oracle import features as F

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


def data(N=20000, d=12, seed=7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, d)) * rng.uniform(0.1, 10, d) + rng.uniform(-5, 5, d)
    X[:, 3] = rng.standard_t(3.0, N)                  # heavy tails
    X[:, 5] = np.round(X[:, 5])                       # repeated values (ties)
    X[:, 7] = 2.5                                     # constant column
    z = 1.5 * X[:, 0] / X[:, 0].std() - X[:, 2] / X[:, 2].std() + 0.5 * np.sin(X[:, 4])
    y = (z + 0.7 * rng.standard_normal(N) > 0).astype(np.int32)
    return X, y


def test_zscore_matches_oracle(B, torch):
    X, _ = data()
    N = X.shape[0]
    # the column sums run in another order: N u (u = 2^-53) bounds the difference
    tol = 2 * N * 2.0 ** -53
    Xd = torch.from_numpy(X).cuda()
    mean, sd = B.anova_zscore_fit(Xd)
    m_ref, s_ref = F.zscore_fit(X)
    scale = np.abs(X).max(axis=0)
    assert np.all(np.abs(mean.cpu().numpy() - m_ref) <= tol * scale)
    assert np.allclose(sd.cpu().numpy(), s_ref, rtol=tol, atol=0)
    T = np.random.default_rng(8).standard_normal((500, X.shape[1]))
    Td = torch.from_numpy(T).cuda()
    B.anova_zscore_apply(Td, mean, sd)
    assert np.allclose(Td.cpu().numpy(), F.zscore_apply(T, m_ref, s_ref), rtol=10 * tol, atol=10 * tol)


# nclass <= 4 takes the two-pass form (privatised (fine bin, class) counts), 6 the three-pass one
@pytest.mark.parametrize("bins,nclass", [(16, 2), (8, 3), (16, 6)])
def test_mis_and_windows_match_oracle(B, torch, bins, nclass):
    X, y = data()
    if nclass == 3:
        y = (y + (X[:, 1] > 0)).astype(np.int32)
    if nclass == 6:
        y = (y + 2 * (X[:, 1] > 0) + 2 * (X[:, 4] > X[:, 4].mean())).astype(np.int32)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    got = B.anova_mis(Xd, yd, nclass, bins)
    ref = F.mis(X, y, nclass, B=bins)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)
    assert got[7] == 0.0                               # constant column: one bin, no information
    for thr in (0.0, 1e-3, 0.01):
        assert B.anova_windows_from_mis(got, thr) == F.windows_from_mis(ref, thr)


def test_mis_rejects_bad_labels(B, torch):
    X, y = data(N=1000)
    y = y.copy()
    y[17] = 5
    with pytest.raises(B.AnovaError):
        B.anova_mis(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 2, 16)


def boundary_data(N=20000, seed=9):
    """Columns whose values sit on the fine-bin boundaries lo + k (hi - lo) / 4096
    of the definition and on the doubles just beside them, plus ordinary
    columns: every fine bin must be the definition's, evaluated in FP64."""
    rng = np.random.default_rng(seed)
    cols = []
    for lo, hi in [(-3.7, 4.1), (1e6, 1e6 + 3.0), (-1e-3, 2e-3), (-250.0, -249.5)]:
        k = rng.integers(0, 4097, N)
        v = lo + k * ((hi - lo) / 4096.0)
        step = rng.integers(-2, 3, N)
        v = np.where(step > 0, np.nextafter(v, np.inf), np.where(step < 0, np.nextafter(v, -np.inf), v))
        v = np.clip(v, lo, hi)
        v[:2] = (lo, hi)
        cols.append(v)
    cols.append(rng.standard_normal(N))
    cols.append(rng.standard_t(3.0, N))
    cols.append(np.round(rng.standard_normal(N) * 4))
    cols.append(np.full(N, 2.5))
    X = np.stack(cols, axis=1)
    y = rng.integers(0, 2, N).astype(np.int32)
    return X, y


def test_mis_fine_bins_match_definition(B, torch):
    X, _ = boundary_data()
    got = B.anova_mis_fine_bins(torch.from_numpy(X).cuda()).cpu().numpy()
    for c in range(X.shape[1]):
        lo, hi = float(X[:, c].min()), float(X[:, c].max())
        ref = np.array([F.fine_index(float(v), lo, hi) for v in X[:, c]])
        bad = np.flatnonzero(got[:, c] != ref)
        assert bad.size == 0, (c, bad[:5], got[bad[:5], c], ref[bad[:5]])


def test_mis_on_boundary_values_matches_oracle(B, torch):
    X, y = boundary_data(N=6000, seed=10)
    got = B.anova_mis(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 2, 64)
    ref = F.mis(X, y, 2, B=64)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)
