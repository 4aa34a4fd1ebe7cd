"""The operand splits the tensor-core spreads use, emulated on the CPU, against
the bounds their kernels' comments and the design notes state.  Both compute
a product a*b of FP32 operands as head*head + head*tail + tail*head in FP32
accumulation, with exact products.

* FP16 split (spread form 3): h = FP16(x) rounded to nearest, l = FP16(x - h),
  operands in [-1, 1].  Bound per product: 3 * 2^-22 |ab| from the dropped
  l*l and the tails' roundings while the tails are normal FP16 (both operands
  at least 2^-2), plus 2^-24 (|a| + |b|) from FP16's subnormal spacing below
  that (absolute, not relative, accuracy for tiny operands).
* TF32 split by truncation (spread form 2): head = x with its low 13 mantissa
  bits cleared, tail = x - head exact in FP32, of which the tensor core reads
  the TF32 bits (truncated): each operand is kept to 2^-20 of itself, each
  product to 3 * 2^-20 (measured worst 2^-19.3), and for positive operands the
  error has one sign (the design notes' bias, mean about -2^-22)."""
import numpy as np


def f16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def fp16_split_product(a, b):
    a32 = np.asarray(a, dtype=np.float32)
    b32 = np.asarray(b, dtype=np.float32)
    ha, hb = f16(a32), f16(b32)
    la = f16(a32.astype(np.float64) - ha)
    lb = f16(b32.astype(np.float64) - hb)
    return ha * hb + ha * lb + la * hb


def tf32_trunc(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32).astype(np.float64)


def tf32_split_product(a, b):
    a32 = np.asarray(a, dtype=np.float32)
    b32 = np.asarray(b, dtype=np.float32)
    ha, hb = tf32_trunc(a32), tf32_trunc(b32)
    ta = (a32.astype(np.float64) - ha).astype(np.float32)    # exact in FP32
    tb = (b32.astype(np.float64) - hb).astype(np.float32)
    return ha * hb + ha * tf32_trunc(tb) + tf32_trunc(ta) * hb


def operands(rng, n):
    """Signs random, magnitudes log-uniform from 1 down to 2^-30 (into FP16's subnormals)."""
    mag = 2.0 ** rng.uniform(-30, 0, n)
    return (rng.choice([-1.0, 1.0], n) * mag).astype(np.float32)


def test_fp16_split_error_bound():
    rng = np.random.default_rng(5)
    a, b = operands(rng, 200_000), operands(rng, 200_000)
    exact = a.astype(np.float64) * b.astype(np.float64)
    err = np.abs(fp16_split_product(a, b) - exact)
    bound = 3 * 2.0 ** -22 * np.abs(exact) + 2.0 ** -24 * (np.abs(a) + np.abs(b))
    assert np.all(err <= bound)
    # where both operands are at least 2^-2 the error is relative
    big = (np.abs(a) >= 0.25) & (np.abs(b) >= 0.25)
    assert big.sum() > 500
    assert np.all(err[big] <= 3 * 2.0 ** -22 * np.abs(exact[big]))


def test_fp16_split_bound_is_not_loose():
    """The bound is met with little room: the measured worst case is within a
    factor 8 of it, so a split that lost a term would fail the test above."""
    rng = np.random.default_rng(6)
    a = rng.uniform(0.25, 1.0, 200_000).astype(np.float32)
    b = rng.uniform(0.25, 1.0, 200_000).astype(np.float32)
    exact = a.astype(np.float64) * b.astype(np.float64)
    rel = np.abs(fp16_split_product(a, b) - exact) / exact
    assert rel.max() > 3 * 2.0 ** -22 / 8
    # dropping the head*tail term breaks the bound by orders of magnitude
    ha, hb = f16(a), f16(b)
    la = f16(a.astype(np.float64) - ha)
    two_terms = ha * hb + la * hb
    assert (np.abs(two_terms - exact) / exact).max() > 100 * 3 * 2.0 ** -22


def test_tf32_truncated_split_bound_and_sign():
    rng = np.random.default_rng(7)
    a = rng.uniform(2.0 ** -20, 1.0, 200_000).astype(np.float32)
    b = rng.uniform(2.0 ** -20, 1.0, 200_000).astype(np.float32)
    exact = a.astype(np.float64) * b.astype(np.float64)
    d = tf32_split_product(a, b) - exact
    assert np.all(np.abs(d) <= 3 * 2.0 ** -20 * exact)
    assert np.abs(d / exact).max() > 2.0 ** -20       # the single-operand figure is not enough
    # truncation only removes magnitude: for positive operands the product never rises
    assert np.all(d <= 0.0)
    assert np.mean(d / exact) < -2.0 ** -25
