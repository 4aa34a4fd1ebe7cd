"""The FP32 fast path of the MIS fine bins, emulated on the CPU bit for bit
(numpy float32 arithmetic with the kernel's operation order and directed
roundings), against the definition the oracle uses: the fine bin of v on
[lo, hi] is floor((v - lo) F / (hi - lo)) in FP64, clamped to [0, F - 1].

Per column the kernel stores lo and F / (hi - lo) rounded to FP32 and a bound
delta on |t - t_def| (t the FP32 estimate of the position); an element whose t
lies at least delta from every integer takes floor(t), every other element
goes to the exact threshold search.  The claim checked here: whenever the fast
path answers, its answer is the definition's bin -- on values spread over the
column, on the bin boundaries lo + k (hi - lo) / F and on the doubles beside
them, for columns of ordinary, large, tiny and offset magnitudes."""
import math

import numpy as np

F = 4096


def approx_float(v):
    """FP32 value from the FP64 high word (mantissa truncated to 20 bits); 0
    outside FP32's normal exponent range."""
    bits = np.asarray(v, dtype=np.float64).view(np.uint64)
    h = (bits >> np.uint64(32)).astype(np.int64)
    e = (h >> 20) & 0x7FF
    sign = h & 0x80000000
    mag = ((h & 0x7FFFFFFF) - (896 << 20)) << 3
    out = (sign | (mag & 0x7FFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where((e <= 896) | (e >= 1151), np.float32(0.0), out)


def round_down32(x):
    f = np.float32(x)
    return np.nextafter(f, np.float32(-np.inf)) if float(f) > x else f


def round_up32(x):
    f = np.float32(x)
    return np.nextafter(f, np.float32(np.inf)) if float(f) < x else f


def screen(lo, hi):
    M, sfd = max(abs(lo), abs(hi)), F / (hi - lo)
    delta = 1.25 * (sfd * M * (2.0 ** -20 + 2.0 ** -24) + sfd * 2.0 ** -126) + 1e-3
    if not (M < 1e37) or not (sfd < 1e37) or not (delta < 0.25):
        delta = 1.0
    return np.float32(lo), np.float32(sfd), round_up32(delta)


def fast_bin(v, scr):
    lof, sf, dl = scr
    with np.errstate(over="ignore", invalid="ignore"):
        t = (approx_float(v) - lof) * sf            # two FP32 operations, each rounded to nearest
    out = np.full(t.shape, -1, dtype=np.int64)
    if not dl < np.float32(0.5):
        return out
    low = t < round_down32(1.0 - float(dl))
    high = t >= round_up32(float(F - 1) + float(dl))
    fl = np.floor(t)
    mid = ~low & ~high & (t == t)
    ok = mid & ~((t - fl < dl) | (fl + np.float32(1.0) - t < dl))
    out[low] = 0
    out[high] = F - 1
    out[ok] = fl[ok].astype(np.int64)
    return out


def definition(v, lo, hi):
    j = np.floor((v - lo) * F / (hi - lo))
    return np.clip(j, 0, F - 1).astype(np.int64)


def column_values(rng, lo, hi, n):
    h = hi - lo
    k = rng.integers(0, F + 1, n // 2)
    edges = lo + k * (h / F)                       # on the boundaries (as FP64 rounds them)
    nudged = np.nextafter(edges, np.where(rng.random(n // 2) < 0.5, -np.inf, np.inf))
    inside = lo + rng.random(n) * h
    v = np.concatenate([edges, nudged, inside, [lo, hi]])
    return np.clip(v, lo, hi)


COLUMNS = [(-3.0, 4.5), (0.0, 1.0), (-1e-3, 2e-3), (1e6, 1e6 + 3.0), (-2.5e9, 7.1e9), (1e-30, 5e-30),
           (1234.5, 1234.5 + 1e-6), (-1e38, 1e38)]


def test_fast_path_answers_only_with_the_definitions_bin():
    rng = np.random.default_rng(11)
    answered = 0
    for lo, hi in COLUMNS:
        v = column_values(rng, lo, hi, 200_000)
        j = fast_bin(v, screen(lo, hi))
        ref = definition(v, lo, hi)
        hit = j >= 0
        assert np.array_equal(j[hit], ref[hit]), (lo, hi)
        answered += int(hit.sum())
    assert answered > 0


def test_fast_path_takes_most_elements_of_ordinary_columns():
    """Away from the boundaries the estimate decides: on values drawn inside an
    ordinary column, under 2 % go to the threshold search; columns whose range
    is tiny against their magnitude (or beyond FP32) all go there."""
    rng = np.random.default_rng(12)
    for lo, hi in [(-3.0, 4.5), (0.0, 1.0), (-2.5e9, 7.1e9)]:
        v = lo + rng.random(100_000) * (hi - lo)
        assert (fast_bin(v, screen(lo, hi)) < 0).mean() < 0.02
    for lo, hi in [(1234.5, 1234.5 + 1e-6), (-1e38, 1e38)]:
        assert screen(lo, hi)[2] == np.float32(1.0)
        assert (fast_bin(np.array([lo, hi]), screen(lo, hi)) < 0).all()


def test_emulated_definition_matches_the_scalar_form():
    """definition() above is the oracle's fine_index, vectorised."""
    rng = np.random.default_rng(13)
    lo, hi = -3.0, 4.5
    v = column_values(rng, lo, hi, 2000)
    scalar = [min(max(int(math.floor((x - lo) * F / (hi - lo))), 0), F - 1) for x in v]
    assert np.array_equal(definition(v, lo, hi), np.array(scalar))


def test_a_bound_without_its_magnitude_term_is_caught(monkeypatch):
    """The check above has teeth: with delta = 1e-3 alone (the rounding of v and
    lo to FP32 left out) the fast path answers wrongly on some column."""
    import sys
    mod = sys.modules[__name__]
    full = mod.screen

    def weak(lo, hi):
        lof, sf, dl = full(lo, hi)
        return lof, sf, (np.float32(1e-3) if dl < np.float32(0.25) else dl)

    monkeypatch.setattr(mod, "screen", weak)
    rng = np.random.default_rng(11)
    wrong = 0
    for lo, hi in COLUMNS:
        v = column_values(rng, lo, hi, 200_000)
        j = fast_bin(v, mod.screen(lo, hi))
        hit = j >= 0
        wrong += int((j[hit] != definition(v, lo, hi)[hit]).sum())
    assert wrong > 0
