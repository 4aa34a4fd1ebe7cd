"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point that include/anova_gb300.h declares; argument validation that
needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "anova_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_10140_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["anova_fastsum_plan", "anova_matvec", "krr_cg_solve", "krr_predict",
                     "anova_plan_destroy", "anova_status_string", "anova_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in the header but not exported"


def test_status_strings(lib):
    from paper_2111_10140_gb300 import binding as B
    L = B.lib()
    for s in range(7):
        assert L.anova_status_string(s).decode().startswith("ANOVA_")
    assert L.anova_status_string(99).decode() == "unknown anova_status"


def test_plan_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Validation runs before any CUDA call, so it is testable on the CPU."""
    from paper_2111_10140_gb300 import binding as B
    import numpy as np
    L = B.lib()
    h = ctypes.c_void_p()
    W = np.array([[0, 1, -1]], dtype=np.int32)
    n = np.array([32], dtype=np.int32)
    pi32 = ctypes.POINTER(ctypes.c_int32)

    def plan(**kw):
        args = dict(points=ctypes.c_void_p(16), N=10, d=2, ld=2, W=W, P=1, ell=0.1, n=n, m=4,
                    sigma=2.0, eps=1 / 16, p=8, prec=B.FP64)
        args.update(kw)
        return L.anova_fastsum_plan(args["points"], args["N"], args["d"], args["ld"],
                                    args["W"].ctypes.data_as(pi32), args["P"], None, args["ell"],
                                    args["n"].ctypes.data_as(pi32), args["m"], args["sigma"], args["eps"],
                                    args["p"], args["prec"], None, ctypes.byref(h))

    assert plan(ell=-1.0) == B.EINVAL
    assert plan(m=0) == B.EINVAL
    assert plan(m=13) == B.EINVAL
    assert plan(n=np.array([31], dtype=np.int32)) == B.EINVAL
    assert plan(n=np.array([4], dtype=np.int32), m=4) == B.EINVAL          # 2m+2 > sigma n
    assert plan(W=np.array([[0, 5, -1]], dtype=np.int32)) == B.EINVAL      # feature out of range
    assert plan(W=np.array([[0, 0, -1]], dtype=np.int32)) == B.EINVAL      # repeated feature
    assert plan(W=np.array([[-1, -1, -1]], dtype=np.int32)) == B.EINVAL    # empty window
    assert plan(W=np.array([[0, -1, 1]], dtype=np.int32)) == B.EINVAL      # bad padding
    assert plan(eps=0.5) == B.EINVAL
    assert plan(p=0) == B.EINVAL
    assert plan(prec=7) == B.EINVAL
    assert plan(ld=1) == B.EINVAL
    assert plan(sigma=1.7) == B.EINVAL                                   # sigma n not an integer
    assert h.value is None
    assert "ell" in L.anova_last_error().decode() or L.anova_last_error().decode() != ""


def test_wait_probe_rejects_bad_poll_counts_without_touching_the_gpu(lib):
    from paper_2111_10140_gb300 import binding as B
    L = B.lib()
    assert L.anova_debug_wait_probe(0, None) == B.EINVAL
    assert L.anova_debug_wait_probe((1 << 22) + 1, None) == B.EINVAL
    assert "polls" in L.anova_last_error().decode()


def test_plan_settings_reject_bad_arguments_without_touching_the_gpu(lib):
    """The kernel-form, schedule and tuning entry points check their arguments
    before any CUDA call (NULL plan, forms or schedule out of range)."""
    import ctypes
    from paper_2111_10140_gb300 import binding as B
    L = B.lib()
    forms = (ctypes.c_int32 * 3)(2, 3, 2)
    assert L.anova_plan_set_kernels(None, forms) == B.EINVAL
    assert L.anova_plan_get_kernels(None, forms) == B.EINVAL
    assert L.anova_plan_set_overlap(None, 1) == B.EINVAL
    assert L.anova_plan_set_tensor_cores(None, 1) == B.EINVAL
    choice = (ctypes.c_int32 * 3)()
    ms = ctypes.c_double()
    assert L.anova_autotune_kernels(None, 5, choice, ctypes.byref(ms), None) == B.EINVAL


def test_bin_rule_is_host_logic(lib):
    """The plan's binning rule for one window, computed without a GPU."""
    from paper_2111_10140_gb300 import binding as B
    rule = B.anova_plan_bin_rule
    assert rule(3, 32, 6) == {"bin_side": 2, "region": 14, "dense": True, "nbins": 32 ** 3}
    assert rule(3, 32, 6, bin_side=[0, 0, 4]) == {"bin_side": 4, "region": 16, "dense": True, "nbins": 16 ** 3}
    assert rule(3, 32, 6, bin_side=[0, 0, 6])["bin_side"] == 2      # region 18 > 16: the request is ignored
    assert rule(3, 32, 6, bin_side=[0, 0, 3])["bin_side"] == 2      # odd side: ignored
    assert rule(3, 32, 6, bin_side=[4, 4, 0])["bin_side"] == 2      # requests for other dimensions
    assert rule(3, 64, 6) == {"bin_side": 4, "region": 16, "dense": True, "nbins": 32 ** 3}   # 2 gives 64^3 bins
    assert rule(3, 32, 7) == {"bin_side": 2, "region": 16, "dense": True, "nbins": 32 ** 3}
    r = rule(3, 32, 8)                                               # region 2 + 16 > 16: generic kernels
    assert not r["dense"] and r["nbins"] <= 32768
    r = rule(3, 128, 6)                                              # too many bins for the dense kernels
    assert not r["dense"] and r["nbins"] <= 32768
    assert rule(2, 64, 6) == {"bin_side": 2, "region": 14, "dense": True, "nbins": 64 ** 2}
    assert rule(1, 64, 6) == {"bin_side": 4, "region": 16, "dense": True, "nbins": 32}
    assert rule(1, 64, 6, bin_side=[6, 0, 0])["bin_side"] == 4      # region 18 > 16: default
    assert rule(1, 64, 4, bin_side=[8, 0, 0]) == {"bin_side": 8, "region": 16, "dense": True, "nbins": 16}
    for bad in [dict(dims=4, n=32, m=6), dict(dims=3, n=31, m=6), dict(dims=3, n=4, m=6),
                dict(dims=3, n=32, m=0), dict(dims=3, n=32, m=6, sigma=1.7)]:
        with pytest.raises(B.AnovaError) as e:
            rule(**bad)
        assert e.value.status == B.EINVAL


def test_windows_from_mis_is_host_logic_matching_the_reference(lib):
    """anova_windows_from_mis runs on the host: the same windows as the
    reference grouping of Sec. 5 for random scores with ties and thresholds."""
    import numpy as np
    from oracle import features as F
    from paper_2111_10140_gb300 import binding as B
    rng = np.random.default_rng(3)
    for trial in range(200):
        d = int(rng.integers(1, 40))
        s = np.round(rng.uniform(0, 1, d), int(rng.integers(1, 3)))    # rounding makes ties
        thr = float(rng.choice([0.0, 0.2, 0.5, 1.1]))
        assert B.anova_windows_from_mis(s, thr) == F.windows_from_mis(list(s), thr)
    for bad in (np.array([0.1, np.nan, 0.3]), np.array([np.inf, 0.2])):
        with pytest.raises(B.AnovaError) as e:
            B.anova_windows_from_mis(bad)
        assert e.value.status == B.EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2111_10140_gb300 import binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        B.lib()
