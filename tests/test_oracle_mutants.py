"""The oracle's pins must catch plausible mistakes in the oracle.

Each case below plants one mistake (a dropped term, a wrong sign, factor,
index, bound or operand) in a copy of ``oracle/anova_oracle.c``, compiles the
copy on the CPU, points the oracle's wrapper at it and runs the pins of
``test_oracle.py`` that guard that part.  At least one of them must fail.  The
unmodified source, compiled the same way, must pass the same pins (the
control), so a failure is due to the planted mistake and not to the harness.
The window-construction reference ``oracle/features.py`` gets the same
treatment against the pins of ``test_oracle_features.py``.
"""
import ctypes
import os
import types

import numpy as np
import pytest

import oracle
import test_oracle as T
import test_oracle_features as TF
from oracle import features as FEAT

SRC = os.path.join(os.path.dirname(oracle.__file__), "anova_oracle.c")


# pin groups: each entry calls pins of test_oracle.py with fixed parameters
def pins_direct():
    T.test_direct_hand_worked_example()
    T.test_direct_symmetric_psd_unit_diagonal()
    T.test_direct_linear_over_windows_and_test_points()


def pins_frame():
    T.test_frame_maps_into_ball_and_touches_it()


def pins_bessel_kb():
    T.test_bessel_i0_matches_scipy()
    T.test_kb_window_edges()
    T.test_kb_window_fourier_pair_by_quadrature(6, 64)


def pins_gauss():
    T.test_gauss_derivatives_match_sympy()


def pins_taylor():
    T.test_two_point_taylor_is_the_hermite_interpolant(8, 1 / 16, 0.2)
    T.test_two_point_taylor_is_the_hermite_interpolant(4, 1 / 16, 0.2)
    T.test_kreg_pieces()


def pins_coeffs():
    T.test_kernel_coeffs_equal_numpy_fft_of_samples(2, 16, 0.15, 1 / 8)
    T.test_kernel_coeffs_closed_form_gaussian(2, 64, 0.06)
    T.test_kernel_coeffs_interpolate_samples()


def pins_diag():
    T.test_diag_divides_by_window_transform()


def pins_dft():
    T.test_grid_dft_matches_numpy_fft()


def pins_nfft():
    T.test_adjoint_nfft_matches_brute_force(2, 16, 6, 1e-10)
    T.test_adjoint_nfft_matches_brute_force(3, 8, 6, 1e-10)
    T.test_nfft_matches_brute_force(2, 16, 6, 1e-10)
    T.test_nfft_matches_brute_force(3, 8, 6, 1e-10)


def pins_fastsum():
    T.test_fastsum_window_symmetric_operator()
    T.test_fastsum_tiny_config_matches_direct()
    T.test_fastsum_linear_over_windows_and_translation_invariant()
    T.test_fastsum_predict_frame_rule()


def pins_cg():
    T.test_cg_matches_dense_solve()


PIN_GROUPS = {
    "direct": pins_direct, "frame": pins_frame, "bessel_kb": pins_bessel_kb, "gauss": pins_gauss,
    "taylor": pins_taylor, "coeffs": pins_coeffs, "diag": pins_diag, "dft": pins_dft,
    "nfft": pins_nfft, "fastsum": pins_fastsum, "cg": pins_cg,
}

# (id, text in anova_oracle.c, planted replacement, which occurrence (0-based), pin group)
MUTANTS = [
    # O1 direct sum
    ("direct_half_width", "sl += alpha[j] * exp(-r2 * inv_ell2);",
     "sl += alpha[j] * exp(-0.5 * r2 * inv_ell2);", 0, "direct"),
    ("direct_eta_dropped", "acc += eta[l] * sl;", "acc += sl;", 0, "direct"),
    ("direct_feature_index", "double df = Z[i * ldz + w[t]] - X[j * ldx + w[t]];",
     "double df = Z[i * ldz + w[t]] - X[j * ldx + t];", 0, "direct"),
    ("direct_sign", "sl += alpha[j] * exp(-r2 * inv_ell2);",
     "sl -= alpha[j] * exp(-r2 * inv_ell2);", 0, "direct"),
    # frame
    ("frame_centre_is_min", "centre[t] = 0.5 * (lo + hi);", "centre[t] = lo;", 0, "frame"),
    ("frame_no_sqrt", "rmax = sqrt(rmax);", "rmax = rmax * 1.0;", 0, "frame"),
    # Kaiser-Bessel pair
    ("i0_series_factorial", "term *= q / ((double)k * (double)k);", "term *= q / (double)k;", 0,
     "bessel_kb"),
    ("kb_sin_for_sinh", "return sinh(b * s) / (M_PI * s);", "return sin(b * s) / (M_PI * s);", 0,
     "bessel_kb"),
    ("kb_edge_value", "if (s == 0.0) return b / M_PI;", "if (s == 0.0) return 0.0;", 0, "bessel_kb"),
    ("kb_hat_frequency", "double w = 2.0 * M_PI * (double)k / (double)nos;",
     "double w = M_PI * (double)k / (double)nos;", 0, "bessel_kb"),
    # regularised kernel
    ("hermite_recursion", "double hn = 2.0 * x * h - 2.0 * (double)i * hm;",
     "double hn = 2.0 * x * h - (double)i * hm;", 0, "gauss"),
    ("deriv_sign", "double sgn = (j % 2) ? -1.0 : 1.0;", "double sgn = 1.0;", 0, "gauss"),
    ("deriv_power", "return sgn * pow(ell, -(double)j) * Hj * exp(-x * x);",
     "return sgn * pow(ell, -(double)(j + 1)) * Hj * exp(-x * x);", 0, "gauss"),
    ("taylor_inner_bound", "for (int q = 0; q <= p - 1 - j; q++) {",
     "for (int q = 0; q < p - 1 - j; q++) {", 0, "taylor"),
    ("taylor_endpoint_swap", "sum += fa * pow(r - a, (double)j) / fact * pow(ue, (double)p) * inner_a;",
     "sum += fa * pow(r - a, (double)j) / fact * pow(ua, (double)p) * inner_a;", 0, "taylor"),
    ("taylor_factorial", "if (j > 0) fact *= (double)j;", "if (j > 1) fact *= (double)(j - 1);", 0,
     "taylor"),
    ("kreg_constant", "double c = exp(-0.25 / (ell * ell));", "double c = exp(-0.5 / (ell * ell));", 0,
     "taylor"),
    # b_k and D_k
    ("coeffs_normalisation", "double sc = 1.0 / (double)tot;", "double sc = 1.0 / (double)n;", 0,
     "coeffs"),
    ("coeffs_uncentred", "long j = rem % n - n / 2;", "long j = rem % n;", 0, "coeffs"),
    ("coeffs_radius_squared", "f[idx] = orc_kreg(sqrt(r2), ell, epsB, p);",
     "f[idx] = orc_kreg(r2, ell, epsB, p);", 0, "coeffs"),
    ("diag_not_squared", "den *= ph * ph;", "den *= ph;", 0, "diag"),
    # DFT
    ("dft_uncentred_input", "long u = i - Lin / 2;", "long u = i;", 0, "dft"),
    ("dft_sign", "double ang = sgn * 2.0 * M_PI * (double)r / (double)Ndft;",
     "double ang = -sgn * 2.0 * M_PI * (double)r / (double)Ndft;", 0, "dft"),
    ("dft_imag_cross_term", "ar += xr * cr - xi * ci;", "ar += xr * cr + xi * ci;", 0, "dft"),
    # spread / gather and the brute-force NDFT
    ("spread_mirrored_taps", "pos = pos * nos + centred_pos(u0[t] + tap[t], nos);",
     "pos = pos * nos + centred_pos(u0[t] - tap[t], nos);", 0, "nfft"),
    ("spread_axes_transposed", "wprod *= wts[t][tap[t]];", "wprod *= wts[dA - 1 - t][tap[t]];", 0,
     "nfft"),
    ("gather_reversed_taps", "wprod *= wts[t][tap[t]];", "wprod *= wts[t][ntap - 1 - tap[t]];", 1,
     "nfft"),
    ("gather_grid_scale", "double y = (double)nos * xt[j * dA + t];",
     "double y = (double)(nos / 2) * xt[j * dA + t];", 1, "nfft"),
    ("adjoint_nfft_no_deconvolution", "g_re[idx] /= den;", "g_re[idx] /= 1.0;", 0, "nfft"),
    ("brute_force_ndft_sign", "ai += c[j] * sin(-2.0 * M_PI * ph);", "ai += c[j] * sin(2.0 * M_PI * ph);",
     0, "nfft"),
    # fast summation
    ("fastsum_ell_unscaled", "double ell_l = s * ell;", "double ell_l = ell;", 0, "fastsum"),
    ("fastsum_eta_dropped", "out[i] += eta[l] * sl[i];", "out[i] += sl[i];", 0, "fastsum"),
    ("fastsum_imag_not_multiplied", "Gr[idx] *= D[idx]; Gi[idx] *= D[idx];", "Gr[idx] *= D[idx];", 0,
     "fastsum"),
    ("fastsum_gathers_imag", "orc_gather(zt, Nz, dA, nos, m, b, hr, out);",
     "orc_gather(zt, Nz, dA, nos, m, b, hi, out);", 0, "fastsum"),
    ("fastsum_no_joint_frame", "if (s * sqrt(rmax) > RB) orc_window_frame",
     "if (0 && s * sqrt(rmax) > RB) orc_window_frame", 0, "fastsum"),
    ("fastsum_ball_radius", "const double RB = 0.25 - 0.5 * epsB;", "const double RB = 0.25 + 0.5 * epsB;",
     0, "fastsum"),
    # CG
    ("cg_beta_inverted", "double beta = rr_new / rr;", "double beta = rr / rr_new;", 0, "cg"),
    ("cg_residual_step", "r[i] -= a * q[i];", "r[i] -= q[i];", 0, "cg"),
    ("cg_lambda_dropped", "for (long i = 0; i < N; i++) out[i] += lambda * v[i];",
     "for (long i = 0; i < N; i++) out[i] += 0.0 * v[i];", 0, "cg"),
]


def _replace_nth(text, old, new, nth):
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"mutation site not found: {old!r} (occurrence {nth})"
    return text[:pos] + new + text[pos + len(old):]


def _compile(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return oracle.bind(ctypes.CDLL(oracle.compile_library(str(src), str(tmp_path / f"lib{name}.so"))))


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


def test_control_unmodified_source_passes_every_pin_group(tmp_path, monkeypatch, source):
    monkeypatch.setattr(oracle, "_lib", _compile(tmp_path, "control", source))
    for group in PIN_GROUPS.values():
        group()


@pytest.mark.parametrize("mid,old,new,nth,group", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, source, mid, old, new, nth, group):
    mutated = _replace_nth(source, old, new, nth)
    assert mutated != source
    monkeypatch.setattr(oracle, "_lib", _compile(tmp_path, mid, mutated))
    with np.errstate(all="ignore"):
        with pytest.raises((AssertionError, ValueError, np.linalg.LinAlgError, FloatingPointError)):
            PIN_GROUPS[group]()


# ------------------------------------------------- window construction (numpy)
FEAT_SRC = FEAT.__file__


def pins_features():
    for name in dir(TF):
        if name.startswith("test_"):
            getattr(TF, name)()


FEAT_MUTANTS = [
    ("zscore_sample_divisor", "std = np.sqrt(((X - mean) ** 2).sum(axis=0) / N)",
     "std = np.sqrt(((X - mean) ** 2).sum(axis=0) / (N - 1))"),
    ("zscore_constant_column", "std = np.where(std > 0.0, std, 1.0)", "std = std + 0.0"),
    ("zscore_apply_variance", "return (np.asarray(X, dtype=np.float64) - mean) / std",
     "return (np.asarray(X, dtype=np.float64) - mean) / std ** 2"),
    ("fine_last_bin_open", "return min(max(j, 0), F - 1)", "return max(j, 0)"),
    ("fine_rounds", "j = int(math.floor((v - lo) * F / (hi - lo)))", "j = int(round((v - lo) * F / (hi - lo)))"),
    ("quantile_counts_shifted", "C = np.concatenate([[0], np.cumsum(c)[:-1]])", "C = np.cumsum(c)"),
    ("mis_missing_N", "math.log(N * n[a, y] / (nq[a] * ny[y]))", "math.log(n[a, y] / (nq[a] * ny[y]))"),
    ("mis_conditional_weight", "s += (n[a, y] / N) * math.log", "s += (n[a, y] / nq[a]) * math.log"),
    ("mis_class_marginal", "ny = n.sum(axis=0)", "ny = n.sum(axis=0) * 0 + n.sum(axis=0).max()"),
    ("windows_ascending", "key=lambda f: (-scores[f], f)", "key=lambda f: (scores[f], f)"),
    ("windows_tie_order", "key=lambda f: (-scores[f], f)", "key=lambda f: (-scores[f], -f)"),
    ("windows_strict_threshold", "if scores[f] >= threshold", "if scores[f] > threshold"),
    ("windows_pairs", "tuple(keep[i:i + 3])", "tuple(keep[i:i + 2])"),
]


def _load_feature_mutant(text):
    mod = types.ModuleType("oracle.features_mutant")
    exec(compile(text, FEAT_SRC, "exec"), mod.__dict__)
    return mod


def _patch_features(monkeypatch, mod):
    for name in ("zscore_fit", "zscore_apply", "fine_index", "quantile_bins", "mis", "windows_from_mis"):
        monkeypatch.setattr(FEAT, name, getattr(mod, name))


def test_features_control_passes(monkeypatch):
    with open(FEAT_SRC) as f:
        _patch_features(monkeypatch, _load_feature_mutant(f.read()))
    pins_features()


@pytest.mark.parametrize("mid,old,new", FEAT_MUTANTS, ids=[m[0] for m in FEAT_MUTANTS])
def test_feature_pins_catch_planted_mistake(monkeypatch, mid, old, new):
    with open(FEAT_SRC) as f:
        text = f.read()
    mutated = _replace_nth(text, old, new, 0)
    assert mutated != text
    _patch_features(monkeypatch, _load_feature_mutant(mutated))
    with np.errstate(all="ignore"):
        with pytest.raises((AssertionError, ValueError, IndexError, ZeroDivisionError)):
            pins_features()
