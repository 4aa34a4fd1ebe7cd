"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check goes through an
independent route (a hand-worked example, a library routine such as numpy's FFT,
scipy's quadrature or Hermite interpolation, a brute-force NDFT written from
Eq. (adjnfft)/(nfft), a dense LAPACK solve, or an invariant such as symmetry).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2111_10140_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
B = oracle.kb_b(2.0)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# ----------------------------------------------------------------- O1 direct sum
def test_direct_hand_worked_example():
    pts, alpha, outs = [], None, {}
    with open(os.path.join(GOLDEN, "direct_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, rest = line.split(None, 1)
            if key == "point":
                pts.append([float(v) for v in rest.split()])
            elif key == "alpha":
                alpha = np.array([float(v) for v in rest.split()])
            else:
                outs[int(key[3:])] = eval(rest, {"exp": math.exp})
    X = np.array(pts)
    got = oracle.direct(X, X, [(0, 1), (2,)], [0.5, 0.5], 0.1, alpha)
    want = np.array([outs[i] for i in range(3)])
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


def _dense_direct(X, windows, eta, ell):
    N = X.shape[0]
    return np.stack([oracle.direct(X, X, windows, eta, ell, e) for e in np.eye(N)], axis=1)


def test_direct_symmetric_psd_unit_diagonal():
    w = W.random_problem(120, 7, [(0, 1, 2), (3, 4), (5,), (6,)], 0.15, 16, 4, seed=11)
    K = _dense_direct(w.X, w.windows, w.eta, w.ell)
    assert np.max(np.abs(K - K.T)) <= 1e-14
    assert np.linalg.eigvalsh(K).min() >= -1e-12
    np.testing.assert_allclose(np.diag(K), np.sum(w.eta), rtol=0, atol=1e-15)


def test_direct_linear_over_windows_and_test_points():
    w = W.random_problem(200, 6, [(0, 1, 2), (3, 4), (5,)], 0.2, 16, 4, seed=3)
    Z = np.random.default_rng(4).uniform(-0.2, 0.2, size=(50, 6))
    eta = np.array([0.2, 0.5, 0.3])
    full = oracle.direct(Z, w.X, w.windows, eta, w.ell, w.alpha)
    parts = sum(eta[l] * oracle.direct(Z, w.X, [w.windows[l]], [1.0], w.ell, w.alpha)
                for l in range(3))
    np.testing.assert_allclose(full, parts, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ Kaiser-Bessel pair
def test_bessel_i0_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    for x in [0.0, 1e-3, 0.5, 3.0, 10.0, 18.85, 28.27, 40.0]:
        assert abs(oracle.bessel_i0(x) - sp.i0(x)) <= 1e-14 * sp.i0(x)


@pytest.mark.parametrize("m,nos", [(4, 64), (6, 64), (6, 128)])
def test_kb_window_fourier_pair_by_quadrature(m, nos):
    """phi(t) on [-m, m] integrated against exp(-2 pi i k t / nos) must give
    I0(m sqrt(b^2 - (2 pi k/nos)^2)) up to the window's truncation: the cut
    tail of the band-limited window is O(1) in absolute terms, against
    I0(m b) ~ 1e7 (m=4) to 1e11 (m=6)."""
    integrate = pytest.importorskip("scipy.integrate")
    for k in [0, 1, 5, nos // 4 - 1, nos // 4]:
        val, _ = integrate.quad(lambda t: oracle.kb_phi(t, m, B) * math.cos(2 * math.pi * k * t / nos),
                                -m, m, limit=400, epsabs=0, epsrel=1e-13)
        want = oracle.kb_phihat(k, nos, m, B)
        assert abs(val - want) <= 0.1 + 1e-12 * want


def test_kb_window_edges():
    m = 6
    assert oracle.kb_phi(m, m, B) == pytest.approx(B / math.pi, rel=1e-15)
    assert oracle.kb_phi(m + 1e-9, m, B) == 0.0
    assert oracle.kb_phi(0.3, m, B) == oracle.kb_phi(-0.3, m, B)
    # continuity at |t| = m
    assert oracle.kb_phi(m - 1e-9, m, B) == pytest.approx(B / math.pi, rel=1e-6)


# ------------------------------------------------------- regularised kernel K_R
def test_gauss_derivatives_match_sympy():
    sympy = pytest.importorskip("sympy")
    r = sympy.symbols("r")
    ell = 0.2
    f = sympy.exp(-r ** 2 / sympy.Rational(1, 25))
    for j in range(0, 9):
        dj = sympy.lambdify(r, sympy.diff(f, r, j), "math")
        for x in [0.0, 0.1, 0.4375, 0.5]:
            want = dj(x)
            got = oracle.gauss_deriv(j, x, ell)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("p,eps,ell", [(4, 1 / 16, 0.2), (8, 1 / 16, 0.2), (8, 0.25, 0.114), (6, 1 / 8, 0.1)])
def test_two_point_taylor_is_the_hermite_interpolant(p, eps, ell):
    """The transition polynomial must be THE degree-(2p-1) Hermite interpolant
    of (K^(j)(a), j<p) and (c, 0, ..., 0) at 1/2; scipy's Krogh interpolator
    builds it independently from the same data."""
    interp = pytest.importorskip("scipy.interpolate")
    a, e = 0.5 - eps, 0.5
    c = math.exp(-0.25 / ell ** 2)
    xi = [a] * p + [e] * p
    yi = [oracle.gauss_deriv(j, a, ell) for j in range(p)] + [c] + [0.0] * (p - 1)
    K = interp.KroghInterpolator(xi, yi)
    scale = max(yi[0], c)
    for r in np.linspace(a, e, 17):
        want = float(K(r))
        got = oracle.two_point_taylor(r, a, e, p, ell, c)
        assert abs(got - want) <= 1e-9 * scale


def test_kreg_pieces():
    ell, eps, p = 0.2, 1 / 16, 8
    a = 0.5 - eps
    c = math.exp(-0.25 / ell ** 2)
    for r in [0.0, 0.1, 0.3, a]:
        assert oracle.kreg(r, ell, eps, p) == pytest.approx(math.exp(-r * r / ell ** 2), rel=1e-15)
    assert oracle.kreg(a + 1e-12, ell, eps, p) == pytest.approx(math.exp(-a * a / ell ** 2), rel=1e-9)
    assert oracle.kreg(0.5, ell, eps, p) == pytest.approx(c, rel=1e-12)
    assert oracle.kreg(0.7, ell, eps, p) == c


# ------------------------------------------------------------------ b_k and D_k
def _kreg_samples(dA, n, ell, eps, p):
    j = (np.arange(n) - n // 2) / n
    grids = np.meshgrid(*([j] * dA), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    return np.vectorize(lambda v: oracle.kreg(v, ell, eps, p))(r)


@pytest.mark.parametrize("dA,n,ell,eps", [(1, 32, 0.2, 1 / 16), (2, 16, 0.15, 1 / 8), (3, 8, 0.3, 1 / 4)])
def test_kernel_coeffs_equal_numpy_fft_of_samples(dA, n, ell, eps):
    """b_k = n^{-d} sum_j K_R(j/n) exp(-2 pi i k.j/n): numpy's FFT of the same
    samples, with the centred index convention of I_n, must agree."""
    f = _kreg_samples(dA, n, ell, eps, 8)
    want = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(f))) / n ** dA
    re, im = oracle.kernel_coeffs(dA, n, ell, eps, 8)
    assert np.max(np.abs(re - want.real)) <= 1e-14 * np.max(np.abs(want))
    assert np.max(np.abs(im)) <= 1e-15 * np.max(np.abs(re))  # real and even (reading S7)


@pytest.mark.parametrize("dA,n,ell", [(1, 64, 0.06), (2, 64, 0.06), (3, 48, 0.09)])
def test_kernel_coeffs_closed_form_gaussian(dA, n, ell):
    """For a narrow Gaussian the periodisation is negligible and b_k equals the
    continuous transform (sqrt(pi) ell)^d exp(-pi^2 ell^2 |k|^2) (aliasing
    exp(-pi^2 ell^2 n^2/4) and the tail beyond 1/2 - epsB both below 1e-11)."""
    re, _ = oracle.kernel_coeffs(dA, n, ell, 1 / 16, 8)
    k = np.arange(n) - n // 2
    grids = np.meshgrid(*([k] * dA), indexing="ij")
    k2 = sum(g * g for g in grids)
    want = (math.sqrt(math.pi) * ell) ** dA * np.exp(-math.pi ** 2 * ell ** 2 * k2)
    assert np.max(np.abs(re - want)) <= 1e-11 * want.max()


def test_kernel_coeffs_interpolate_samples():
    """sum_k b_k exp(2 pi i k.j/n) reproduces K_R(j/n) at every grid node."""
    n, ell = 16, 0.2
    re, _ = oracle.kernel_coeffs(2, n, ell, 1 / 8, 6)
    back = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(re))) * n ** 2
    want = _kreg_samples(2, n, ell, 1 / 8, 6)
    assert np.max(np.abs(back.real - want)) <= 1e-14


def test_diag_divides_by_window_transform():
    n, nos, m = 8, 16, 3
    bk = np.random.default_rng(0).standard_normal((n, n))
    D = oracle.diag(2, n, nos, m, B, bk)
    for k0 in range(n):
        for k1 in range(n):
            den = (oracle.kb_phihat(k0 - n // 2, nos, m, B) * oracle.kb_phihat(k1 - n // 2, nos, m, B)) ** 2
            assert D[k0, k1] == pytest.approx(bk[k0, k1] / den, rel=1e-14)


# ---------------------------------------------------------------- NFFT pieces
def test_grid_dft_matches_numpy_fft():
    rng = np.random.default_rng(1)
    for dA, nos, n in [(1, 32, 16), (2, 16, 8), (3, 8, 4)]:
        g = rng.standard_normal((nos,) * dA)
        full = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(g)))
        sl = tuple(slice(nos // 2 - n // 2, nos // 2 + n // 2) for _ in range(dA))
        got = oracle.grid_dft(g, n)
        assert np.max(np.abs(got - full[sl])) <= 1e-12 * np.max(np.abs(full))
        H = rng.standard_normal((n,) * dA) + 1j * rng.standard_normal((n,) * dA)
        Hp = np.zeros((nos,) * dA, complex)
        Hp[sl] = H
        want = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(Hp))) * nos ** dA
        got = oracle.grid_idft(H, nos)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def _ball_nodes(N, dA, seed, radius=W.R_B):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((N, dA))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radius * rng.uniform(0, 1, N) ** (1.0 / dA)
    return v * r[:, None]


def _numpy_adjoint_ndft(xt, n, c):
    k = np.arange(n) - n // 2
    dA = xt.shape[1]
    grids = np.meshgrid(*([k] * dA), indexing="ij")
    K = np.stack([g.ravel() for g in grids], axis=1)
    return (np.exp(-2j * np.pi * K @ xt.T) @ c).reshape((n,) * dA)


@pytest.mark.parametrize("dA,n,m,tol", [(1, 32, 4, 1e-7), (2, 16, 4, 1e-7), (2, 16, 6, 1e-10), (3, 8, 6, 1e-10)])
def test_adjoint_nfft_matches_brute_force(dA, n, m, tol):
    """Window method for Eq. (adjnfft) vs the plain sum; the error must be at
    the Kaiser-Bessel level exp(-2 pi m sqrt(1-1/sigma))."""
    xt = _ball_nodes(150, dA, seed=dA + m)
    c = np.random.default_rng(9).standard_normal(150)
    want = _numpy_adjoint_ndft(xt, n, c)
    assert rel(oracle.adjoint_ndft(xt, n, c), want) <= 1e-13
    got = oracle.adjoint_nfft(xt, n, 2 * n, m, B, c)
    assert rel(got, want) <= tol


@pytest.mark.parametrize("dA,n,m,tol", [(1, 32, 4, 1e-7), (2, 16, 6, 1e-10), (3, 8, 6, 1e-10)])
def test_nfft_matches_brute_force(dA, n, m, tol):
    """Window method for Eq. (nfft) on real-even coefficients vs the plain sum."""
    xt = _ball_nodes(120, dA, seed=20 + dA)
    rng = np.random.default_rng(5)
    fh = rng.standard_normal((n,) * dA)
    # make it even so that f is real: f_k = f_{-k} (index -n/2 has no partner, zero it)
    for ax in range(dA):
        fh = 0.5 * (fh + np.flip(np.roll(fh, -1, axis=ax), axis=ax))
    sl = [slice(None)] * dA
    for ax in range(dA):
        s = list(sl)
        s[ax] = 0
        fh[tuple(s)] = 0.0
    k = np.arange(n) - n // 2
    grids = np.meshgrid(*([k] * dA), indexing="ij")
    K = np.stack([g.ravel() for g in grids], axis=1)
    want = (np.exp(2j * np.pi * xt @ K.T) @ fh.ravel())
    assert np.max(np.abs(want.imag)) <= 1e-12 * np.max(np.abs(want.real))
    got = oracle.nfft_real(xt, n, 2 * n, m, B, fh.astype(complex))
    assert rel(got, want.real) <= tol


# ----------------------------------------------------------- O2 fast summation
def _frame_coords(X, w, epsB):
    c, s = oracle.window_frame(X, w, 0.25 - epsB / 2)
    return s * (X[:, list(w)] - c), s


def test_frame_maps_into_ball_and_touches_it():
    w = W.random_problem(500, 4, [(0, 1, 2), (3,)], 0.2, 16, 4, seed=2)
    for win in w.windows:
        xt, s = _frame_coords(w.X + 3.7, win, 1 / 16)
        r = np.linalg.norm(xt, axis=1)
        assert r.max() == pytest.approx(0.25 - 1 / 32, rel=1e-14)
        lo, hi = xt.min(axis=0), xt.max(axis=0)
        np.testing.assert_allclose(lo, -hi, atol=1e-15)  # bounding-box midpoint is the centre


def test_fastsum_window_symmetric_operator():
    """Phi D Phi^* with one node set is symmetric up to rounding: gather is the
    transpose of spread and D is real."""
    w = W.random_problem(300, 3, [(0, 1, 2)], 0.2, 16, 4, seed=7)
    xt, s = _frame_coords(w.X, (0, 1, 2), 1 / 8)
    n, nos, m = 16, 32, 4
    re, _ = oracle.kernel_coeffs(3, n, s * w.ell, 1 / 8, 8)
    D = oracle.diag(3, n, nos, m, B, re)
    rng = np.random.default_rng(1)
    v, u = rng.standard_normal(300), rng.standard_normal(300)
    Kv, _, imag = oracle.fastsum_window(xt, xt, n, nos, m, B, D, v)
    Ku, _, _ = oracle.fastsum_window(xt, xt, n, nos, m, B, D, u)
    assert abs(u @ Kv - v @ Ku) <= 1e-13 * abs(u @ Kv)
    # The imaginary part of h comes only from the unpaired frequencies k_t = -n/2
    # of I_n (the output takes the real part): with D zeroed there, h is real.
    assert imag > 0.0
    D0 = D.copy()
    for ax in range(3):
        idx = [slice(None)] * 3
        idx[ax] = 0
        D0[tuple(idx)] = 0.0
    _, _, imag0 = oracle.fastsum_window(xt, xt, n, nos, m, B, D0, v)
    assert imag0 <= 1e-13


def test_fastsum_converges_to_direct_as_n_and_m_grow():
    w = W.random_problem(400, 2, [(0, 1)], 0.1, 16, 4, seed=5)
    direct = oracle.direct(w.X, w.X, w.windows, w.eta, w.ell, w.alpha)
    errs = []
    for n, m in [(8, 2), (16, 3), (32, 4), (64, 6)]:
        f = oracle.fastsum(None, w.X, w.windows, w.eta, w.ell, [n], m, w.alpha, epsB=1 / 16)
        errs.append(rel(f, direct))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-8


def test_fastsum_tiny_config_matches_direct():
    w = W.plain_tiny()
    direct = oracle.direct(w.X, w.X, w.windows, w.eta, w.ell, w.alpha)
    f = oracle.fastsum(None, w.X, w.windows, w.eta, w.ell, w.n, w.m, w.alpha, epsB=w.epsB, p=w.p)
    assert rel(f, direct) <= 1e-6


def test_fastsum_linear_over_windows_and_translation_invariant():
    w = W.random_problem(300, 5, [(0, 1, 2), (3, 4)], 0.2, 16, 4, seed=8)
    eta = np.array([0.7, 0.3])
    full = oracle.fastsum(None, w.X, w.windows, eta, w.ell, [16, 16], 4, w.alpha, epsB=1 / 8)
    parts = sum(eta[l] * oracle.fastsum(None, w.X, [w.windows[l]], [1.0], w.ell, [16], 4, w.alpha, epsB=1 / 8)
                for l in range(2))
    assert rel(full, parts) <= 1e-14
    moved = oracle.fastsum(None, w.X + 5.25, w.windows, eta, w.ell, [16, 16], 4, w.alpha, epsB=1 / 8)
    assert rel(moved, full) <= 1e-12


def test_fastsum_predict_frame_rule():
    """Test points outside the ball of the training frame switch to the joint
    frame; the result is still the kernel sum of Eq. (kernelsum)."""
    RB = 0.25 - 1 / 32
    # Zout reaches radius 0.45 of the training frame: pairs further apart than
    # 1/2 - epsB there would meet the periodisation (about 7e-4 error with
    # ell = 0.15), so only the joint frame meets the tolerance.
    for scale, ell in ((0.5, 0.1), (2.5, 0.15)):
        w = W.random_problem(300, 2, [(0, 1)], ell, 32, 4, seed=12)
        Z = w.X[:40] * scale
        c, s = oracle.window_frame(w.X, (0, 1), RB)
        assert (s * np.linalg.norm(Z - c, axis=1).max() > RB) == (scale > 1)
        d = oracle.direct(Z, w.X, w.windows, w.eta, w.ell, w.alpha)
        f = oracle.fastsum(Z, w.X, w.windows, w.eta, w.ell, [32], 4, w.alpha, epsB=1 / 16)
        assert rel(f, d) <= 1e-6


# ------------------------------------------------------------------- O3 CG
def test_cg_matches_dense_solve():
    w = W.random_problem(250, 4, [(0, 1), (2, 3)], 0.15, 32, 4, seed=13)
    lam = 1e-2
    K = _dense_direct(w.X, w.windows, w.eta, w.ell)
    want = np.linalg.solve(K + lam * np.eye(w.N), w.y)
    a, it, relres = oracle.cg(w.X, w.windows, w.eta, w.ell, 32, 4, lam, w.y, 1e-12, 2000, use_direct=True)
    assert relres <= 1e-11
    cond = np.linalg.cond(K + lam * np.eye(w.N))
    assert rel(a, want) <= 10 * cond * 1e-12
    af, itf, relf = oracle.cg(w.X, w.windows, w.eta, w.ell, 32, 4, lam, w.y, 1e-10, 2000, epsB=1 / 16)
    assert relf <= 1e-9
    # with the fast operator the solution moves by at most cond x operator error
    Kf = np.stack([oracle.fastsum(None, w.X, w.windows, w.eta, w.ell, 32, 4, e, epsB=1 / 16)
                   for e in np.eye(w.N)], axis=1)
    op_err = np.linalg.norm(Kf - K, 2) / np.linalg.norm(K + lam * np.eye(w.N), 2)
    assert op_err <= 1e-6
    assert rel(af, want) <= 2 * cond * op_err + 1e-9
