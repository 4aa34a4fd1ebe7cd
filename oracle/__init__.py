"""Plain FP64 CPU oracle for the ANOVA-Gaussian fast summation (arXiv 2111.10140).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it shares no code with it.

The arithmetic lives in ``anova_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Parts and the passages they follow (all pinned by ``tests/test_oracle.py``):
  direct         O1, Sec. 2 Eq. (mult_with_K), Sec. 3 Eq. (extended_Gaussian_ANOVA_kernel)
  window_frame   node scaling h^{-1} x into the torus, Sec. 4.2
  kb_phi/phihat  Kaiser-Bessel window pair (NFFT parameters left to the NFFT3 paper, Sec. 4.1)
  kreg           regularised (periodised) kernel with polynomial transition, Sec. 4.2
  kernel_coeffs  b_k from a DFT of equispaced samples of the periodised kernel, Sec. 4.2
  spread/gather  window steps of the adjoint NFFT / NFFT, Eq. (adjnfft), Eq. (nfft)
  fastsum        s = Phi_z D Phi^* alpha summed over the windows, Sec. 4.3 and Sec. 5
  cg             CG on (K + lambda I) alpha = y, Sec. 2
  adjoint_ndft   brute-force Eq. (adjnfft)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "anova_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def compile_library(src: str, out: str) -> str:
    """Compile one C source of the oracle into a shared library with gcc (FP64, OpenMP)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile anova_oracle.c into the package's shared library."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_library(_SRC, _LIB_PATH)


def bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    d, i, L, p_d, p_i = (ctypes.c_double, ctypes.c_int, ctypes.c_long, _dp, _ip)
    sig = {
        "orc_direct": (None, [p_d, L, L, p_d, L, L, p_i, i, p_d, d, p_d, p_d]),
        "orc_window_frame": (None, [p_d, L, L, p_d, L, L, p_i, d, p_d, p_d]),
        "orc_bessel_i0": (d, [d]),
        "orc_kb_phi": (d, [d, i, d]),
        "orc_kb_phihat": (d, [L, L, i, d]),
        "orc_gauss_deriv": (d, [i, d, d]),
        "orc_two_point_taylor": (d, [d, d, d, i, d, d]),
        "orc_kreg": (d, [d, d, d, i]),
        "orc_kernel_coeffs": (None, [i, i, d, d, i, p_d, p_d]),
        "orc_diag": (None, [i, i, i, i, d, p_d, p_d]),
        "orc_spread": (None, [p_d, L, i, i, i, d, p_d, p_d]),
        "orc_gather": (None, [p_d, L, i, i, i, d, p_d, p_d]),
        "orc_grid_dft": (None, [p_d, i, i, i, p_d, p_d]),
        "orc_grid_idft": (None, [p_d, p_d, i, i, i, p_d, p_d]),
        "orc_adjoint_ndft": (None, [p_d, L, i, i, p_d, p_d, p_d]),
        "orc_adjoint_nfft": (None, [p_d, L, i, i, i, i, d, p_d, p_d, p_d]),
        "orc_nfft_real": (None, [p_d, L, i, i, i, i, d, p_d, p_d, p_d]),
        "orc_fastsum_window": (None, [p_d, L, p_d, L, i, i, i, i, d, p_d, p_d, p_d, p_d, p_d]),
        "orc_fastsum": (i, [p_d, L, L, p_d, L, L, p_i, i, p_d, d, p_i, i, d, d, i, p_d, p_d]),
        "orc_cg": (i, [p_d, L, L, p_i, i, p_d, d, p_i, i, d, d, i, i, d, p_d, d, i, p_d, p_d]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _pi(a):
    return a.ctypes.data_as(_ip)


def kb_b(sigma: float = 2.0) -> float:
    """Kaiser-Bessel shape parameter b = pi (2 - 1/sigma)."""
    return float(np.pi * (2.0 - 1.0 / sigma))


def windows_array(windows) -> np.ndarray:
    """P x 3 int32, -1 padded, from a list of feature-index tuples (0-based)."""
    out = -np.ones((len(windows), 3), dtype=np.int32)
    for l, w in enumerate(windows):
        out[l, :len(w)] = w
    return out


# --------------------------------------------------------------------------- O1
def direct(Z, X, windows, eta, ell, alpha):
    lib = _load()
    Z, X, alpha = _f64(Z), _f64(X), _f64(alpha)
    W = windows_array(windows) if not isinstance(windows, np.ndarray) else _i32(windows)
    eta = _f64(eta)
    out = np.zeros(Z.shape[0])
    lib.orc_direct(_pd(Z), Z.shape[0], Z.shape[1], _pd(X), X.shape[0], X.shape[1],
                   _pi(W), W.shape[0], _pd(eta), float(ell), _pd(alpha), _pd(out))
    return out


# ------------------------------------------------------------------- frame & KB
def window_frame(X, w, RB, Z=None):
    lib = _load()
    X = _f64(X)
    wa = np.full(3, -1, dtype=np.int32)
    wa[:len(w)] = w
    c = np.zeros(3)
    s = np.zeros(1)
    if Z is None:
        lib.orc_window_frame(_pd(X), X.shape[0], X.shape[1], None, 0, 0, _pi(wa), RB, _pd(c), _pd(s))
    else:
        Z = _f64(Z)
        lib.orc_window_frame(_pd(X), X.shape[0], X.shape[1], _pd(Z), Z.shape[0], Z.shape[1],
                             _pi(wa), RB, _pd(c), _pd(s))
    return c[:len(w)].copy(), float(s[0])


def bessel_i0(x):
    return _load().orc_bessel_i0(float(x))


def kb_phi(t, m, b):
    return _load().orc_kb_phi(float(t), int(m), float(b))


def kb_phihat(k, nos, m, b):
    return _load().orc_kb_phihat(int(k), int(nos), int(m), float(b))


def gauss_deriv(j, r, ell):
    return _load().orc_gauss_deriv(int(j), float(r), float(ell))


def two_point_taylor(r, a, e, p, ell, c):
    return _load().orc_two_point_taylor(float(r), float(a), float(e), int(p), float(ell), float(c))


def kreg(r, ell, epsB, p):
    return _load().orc_kreg(float(r), float(ell), float(epsB), int(p))


def kernel_coeffs(dA, n, ell, epsB=1.0 / 16, p=8):
    """b_k on I_n^dA (centred index), returned as (real, imag), shape (n,)*dA."""
    lib = _load()
    re = np.zeros(n ** dA)
    im = np.zeros(n ** dA)
    lib.orc_kernel_coeffs(dA, n, float(ell), float(epsB), int(p), _pd(re), _pd(im))
    return re.reshape((n,) * dA), im.reshape((n,) * dA)


def diag(dA, n, nos, m, b, bk):
    lib = _load()
    bk = _f64(bk).ravel()
    D = np.zeros(n ** dA)
    lib.orc_diag(dA, n, nos, m, float(b), _pd(bk), _pd(D))
    return D.reshape((n,) * dA)


# ------------------------------------------------------------- NFFT building blocks
def spread(xt, nos, m, b, alpha):
    lib = _load()
    xt = _f64(xt)
    N, dA = xt.shape
    g = np.zeros(nos ** dA)
    lib.orc_spread(_pd(xt), N, dA, nos, m, float(b), _pd(_f64(alpha)), _pd(g))
    return g.reshape((nos,) * dA)


def gather(xt, nos, m, b, h):
    lib = _load()
    xt = _f64(xt)
    N, dA = xt.shape
    out = np.zeros(N)
    lib.orc_gather(_pd(xt), N, dA, nos, m, float(b), _pd(_f64(h).ravel()), _pd(out))
    return out


def grid_dft(g, n):
    lib = _load()
    g = _f64(g)
    dA, nos = g.ndim, g.shape[0]
    re = np.zeros(n ** dA)
    im = np.zeros(n ** dA)
    lib.orc_grid_dft(_pd(g.ravel()), dA, nos, n, _pd(re), _pd(im))
    return (re + 1j * im).reshape((n,) * dA)


def grid_idft(H, nos):
    lib = _load()
    H = np.asarray(H)
    dA, n = H.ndim, H.shape[0]
    hr, hi = _f64(H.real).ravel(), _f64(H.imag).ravel()
    re = np.zeros(nos ** dA)
    im = np.zeros(nos ** dA)
    lib.orc_grid_idft(_pd(hr), _pd(hi), dA, nos, n, _pd(re), _pd(im))
    return (re + 1j * im).reshape((nos,) * dA)


def adjoint_ndft(xt, n, c):
    lib = _load()
    xt = _f64(xt)
    N, dA = xt.shape
    re = np.zeros(n ** dA)
    im = np.zeros(n ** dA)
    lib.orc_adjoint_ndft(_pd(xt), N, dA, n, _pd(_f64(c)), _pd(re), _pd(im))
    return (re + 1j * im).reshape((n,) * dA)


def adjoint_nfft(xt, n, nos, m, b, c):
    lib = _load()
    xt = _f64(xt)
    N, dA = xt.shape
    re = np.zeros(n ** dA)
    im = np.zeros(n ** dA)
    lib.orc_adjoint_nfft(_pd(xt), N, dA, n, nos, m, float(b), _pd(_f64(c)), _pd(re), _pd(im))
    return (re + 1j * im).reshape((n,) * dA)


def nfft_real(xt, n, nos, m, b, fhat):
    lib = _load()
    xt = _f64(xt)
    N, dA = xt.shape
    fhat = np.asarray(fhat)
    fr, fi = _f64(fhat.real).ravel(), _f64(fhat.imag).ravel()
    out = np.zeros(N)
    lib.orc_nfft_real(_pd(xt), N, dA, n, nos, m, float(b), _pd(fr), _pd(fi), _pd(out))
    return out


def fastsum_window(zt, xt, n, nos, m, b, D, alpha):
    """One window of Eq. (fastsum) on torus coordinates.
    Returns (s, spread grid g, max |Im h| / max |Re h|)."""
    lib = _load()
    zt, xt = _f64(zt), _f64(xt)
    dA = xt.shape[1]
    out = np.zeros(zt.shape[0])
    grid = np.zeros(nos ** dA)
    im = np.zeros(1)
    lib.orc_fastsum_window(_pd(zt), zt.shape[0], _pd(xt), xt.shape[0], dA, n, nos, m, float(b),
                           _pd(_f64(D).ravel()), _pd(_f64(alpha)), _pd(out), _pd(grid), _pd(im))
    return out, grid.reshape((nos,) * dA), float(im[0])


def fastsum(Z, X, windows, eta, ell, nvec, m, alpha, sigma=2.0, epsB=1.0 / 16, p=8):
    """Fast ANOVA summation (Sec. 4.3, Sec. 5).  Pass Z=None for K alpha."""
    lib = _load()
    X = _f64(X)
    same = Z is None
    Zc = X if same else _f64(Z)
    W = windows_array(windows) if not isinstance(windows, np.ndarray) else _i32(windows)
    P = W.shape[0]
    nv = _i32(np.broadcast_to(np.asarray(nvec, dtype=np.int32), (P,)))
    out = np.zeros(Zc.shape[0])
    rc = lib.orc_fastsum(_pd(Zc), Zc.shape[0], Zc.shape[1], _pd(X), X.shape[0], X.shape[1],
                         _pi(W), P, _pd(_f64(eta)), float(ell), _pi(nv), int(m), float(sigma),
                         float(epsB), int(p), _pd(_f64(alpha)), _pd(out))
    if rc != 0:
        raise ValueError("orc_fastsum: invalid window")
    return out


def cg(X, windows, eta, ell, nvec, m, lam, y, tol, maxit, use_direct=False,
       sigma=2.0, epsB=1.0 / 16, p=8):
    """CG on (K + lambda I) alpha = y; returns (alpha, iterations, true relative residual)."""
    lib = _load()
    X = _f64(X)
    W = windows_array(windows) if not isinstance(windows, np.ndarray) else _i32(windows)
    P = W.shape[0]
    nv = _i32(np.broadcast_to(np.asarray(nvec, dtype=np.int32), (P,)))
    alpha = np.zeros(X.shape[0])
    rel = np.zeros(1)
    it = lib.orc_cg(_pd(X), X.shape[0], X.shape[1], _pi(W), P, _pd(_f64(eta)), float(ell),
                    _pi(nv), int(m), float(sigma), float(epsB), int(p), int(bool(use_direct)),
                    float(lam), _pd(_f64(y)), float(tol), int(maxit), _pd(alpha), _pd(rel))
    return alpha, int(it), float(rel[0])
