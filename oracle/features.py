"""Plain FP64 reference for the window construction upstream of the fast
summation (arXiv 2111.10140, Sec. 5 and Sec. 6.1).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` may
import it.  Plain numpy and Python loops; no blocking or reordering beyond the
definitions below.

  zscore_fit / zscore_apply   Sec. 6.1 (data preprocessing): every column
                              standardised to mean 0 and standard deviation 1
                              with statistics of the training data only.
  mis                         Sec. 5: mutual information score between one
                              feature and the label.  The paper names the
                              score but not its estimator; this is the plug-in
                              estimate on quantile bins defined in ``mis``.
  windows_from_mis            Sec. 5: features ranked by score, those below the
                              threshold dropped, the rest grouped three at a
                              time in rank order, the last group taking the
                              one to three left.
"""
from __future__ import annotations

import math

import numpy as np

FINE_BINS = 4096


def zscore_fit(X):
    """Column means and standard deviations (population form, divisor N) of
    the training data; a constant column gets standard deviation 1 so that it
    is only centred."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    mean = X.sum(axis=0) / N
    std = np.sqrt(((X - mean) ** 2).sum(axis=0) / N)
    std = np.where(std > 0.0, std, 1.0)
    return mean, std


def zscore_apply(X, mean, std):
    return (np.asarray(X, dtype=np.float64) - mean) / std


def fine_index(v, lo, hi, F=FINE_BINS):
    """Equal-width fine bin of value v on [lo, hi]: floor((v - lo) F / (hi - lo)),
    the last bin closed; everything in bin 0 when hi == lo."""
    if not hi > lo:
        return 0
    j = int(math.floor((v - lo) * F / (hi - lo)))
    return min(max(j, 0), F - 1)


def quantile_bins(col, B, F=FINE_BINS):
    """Quantile bin (0..B-1) of every value of one column: the fine bin's
    mid-rank fraction (C_j + c_j / 2) / N, with C_j the count below fine bin j
    and c_j its own count, times B, rounded down -- in integers,
    floor(B (2 C_j + c_j) / (2 N))."""
    col = np.asarray(col, dtype=np.float64)
    N = col.shape[0]
    lo, hi = float(col.min()), float(col.max())
    j = np.array([fine_index(float(v), lo, hi, F) for v in col], dtype=np.int64)
    c = np.bincount(j, minlength=F).astype(np.int64)
    C = np.concatenate([[0], np.cumsum(c)[:-1]])
    q = np.minimum((B * (2 * C + c)) // (2 * N), B - 1)
    return q[j]


def mis(X, labels, nclass, B=16, F=FINE_BINS):
    """Mutual information (nats) between each column's quantile bin and the
    label: sum over (bin q, class y) with n_qy > 0 of
    (n_qy / N) ln(N n_qy / (n_q n_y))."""
    X = np.asarray(X, dtype=np.float64)
    labels = np.asarray(labels, dtype=np.int64)
    N, d = X.shape
    out = np.zeros(d)
    for f in range(d):
        q = quantile_bins(X[:, f], B, F)
        n = np.zeros((B, nclass), dtype=np.int64)
        for a, y in zip(q, labels):
            n[a, y] += 1
        nq = n.sum(axis=1)
        ny = n.sum(axis=0)
        s = 0.0
        for a in range(B):
            for y in range(nclass):
                if n[a, y] > 0:
                    s += (n[a, y] / N) * math.log(N * n[a, y] / (nq[a] * ny[y]))
        out[f] = s
    return out


def windows_from_mis(scores, threshold=0.0):
    """Feature windows: indices sorted by score (descending; equal scores by
    index), those with score < threshold dropped, then consecutive groups of
    three; the last group holds the remaining one to three features."""
    order = sorted(range(len(scores)), key=lambda f: (-scores[f], f))
    keep = [f for f in order if scores[f] >= threshold]
    return [tuple(keep[i:i + 3]) for i in range(0, len(keep), 3)]
