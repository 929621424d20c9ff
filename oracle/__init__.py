"""The oracle: a plain FP64 CPU reference for Eq. 1 (GWAS sequence of GLS problems).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only permitted users.  The GPU product path
(``paper_1210_7325_gb300``) never imports this package, and this package never
imports the product path: the two share no code.

``oracle.c`` holds the arithmetic (see its header for the steps and the
passages they follow); this module compiles it with gcc and wraps it with
ctypes.  ``exact.py`` holds an exact-rational brute force used to pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Pivot thresholds for the p x p solve (pivot d_j <= TAU * S_jj marks S_i as
# not SPD).  d_j / S_jj is the fraction of column j's weight left after the
# earlier columns are projected out: about 1/3 or more for a real SNP against
# an intercept, and at rounding level (1e-14 in FP64, 1e-8 in the mixed paths)
# for an exactly collinear one.  The thresholds sit between, with margin on
# both sides.
TAU_FP64 = 2.0 ** -30
TAU_MIXED = 2.0 ** -16


def build(src: str = _SRC, out: str = _LIB, extra_flags=()) -> str:
    """Compile ``src`` into the shared library ``out`` (atomic rename)."""
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(out))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", *extra_flags, src, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        raise RuntimeError(f"oracle build failed:\n{e.stderr}") from e
    os.replace(tmp, out)
    return out


def _needs_build() -> bool:
    return (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    vp = ctypes.c_void_p
    lib.gls_oracle_potrf.argtypes = [i64, vp, i64, vp, i64, i32]
    lib.gls_oracle_potrf.restype = i64
    lib.gls_oracle_trsv.argtypes = [i64, vp, i64, vp]
    lib.gls_oracle_trsv.restype = None
    lib.gls_oracle_gls.argtypes = [i64, i32, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp,
                                   dbl, i32]
    lib.gls_oracle_gls.restype = i64
    lib.gls_oracle_gls_sampled.argtypes = [i64, i32, vp, i64, vp, i64, vp, i64, vp, vp, i64,
                                           vp, i64, vp, dbl, i32]
    lib.gls_oracle_gls_sampled.restype = i64
    lib.gls_oracle_gls_factored.argtypes = [i64, i32, vp, vp, i64, vp, i64, vp, i64, vp, i64,
                                            vp, dbl, i32]
    lib.gls_oracle_gls_factored.restype = i64
    return lib


def load_library(path: str) -> ctypes.CDLL:
    """Load an oracle build at ``path`` (used for the mutation tests too)."""
    return _declare(ctypes.CDLL(path))


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if _needs_build():
                build()
            _lib = load_library(_LIB)
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def potrf(M: np.ndarray, nthreads: int = 1):
    """Cholesky of the lower triangle of M. Returns (L, info)."""
    M = np.asfortranarray(M, dtype=np.float64)
    n = M.shape[0]
    L = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib().gls_oracle_potrf(n, _ptr(M), max(n, 1), _ptr(L), max(n, 1), nthreads)
    return L, int(info)


def trsv(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L x = b (lower, non-unit) by forward substitution."""
    L = np.asfortranarray(L, dtype=np.float64)
    x = np.array(b, dtype=np.float64, copy=True)
    lib().gls_oracle_trsv(L.shape[0], _ptr(L), max(L.shape[0], 1), _ptr(x))
    return x


def _prep(M, XL, y, XR, p):
    M = np.asfortranarray(M, dtype=np.float64)
    n = np.asarray(XR).shape[0] if M.size == 0 else M.shape[0]
    if p > 1:
        XL = np.asfortranarray(XL, dtype=np.float64).reshape(n, p - 1, order="F")
    else:
        XL = np.zeros((n, 1), dtype=np.float64, order="F")
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(n)
    XR = np.asfortranarray(XR, dtype=np.int8)
    assert XR.shape[0] == n
    return M, n, XL, y, XR


def gls(M, XL, y, XR, tau: float = TAU_FP64, nthreads: int = 1, library=None):
    """b_i for every column of XR (n x k int8).

    Returns (B, status, info): B is p x k float64, status k int32.
    """
    p = (0 if XL is None else np.asarray(XL).reshape(np.asarray(M).shape[0], -1).shape[1]) + 1
    M, n, XL, y, XR = _prep(M, XL, y, XR, p)
    k = XR.shape[1]
    B = np.full((p, k), np.nan, dtype=np.float64, order="F")
    status = np.zeros(k, dtype=np.int32)
    L = library if library is not None else lib()
    info = L.gls_oracle_gls(n, p, _ptr(M), n, _ptr(XL), n, _ptr(y), k, _ptr(XR), n, _ptr(B),
                            p, _ptr(status), float(tau), int(nthreads))
    if info < 0:
        raise ValueError("oracle rejected its arguments")
    return B, status, int(info)


def gls_sampled(M, XL, y, XR, idx, tau: float = TAU_FP64, nthreads: int = 1):
    """b_i for the SNP columns idx of XR only. Returns (B[:, len(idx)], status, info)."""
    p = (0 if XL is None else np.asarray(XL).reshape(np.asarray(M).shape[0], -1).shape[1]) + 1
    M, n, XL, y, _ = _prep(M, XL, y, np.zeros((np.asarray(M).shape[0], 0), np.int8), p)
    XRc = np.asfortranarray(XR, dtype=np.int8)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    B = np.full((p, idx.size), np.nan, dtype=np.float64, order="F")
    status = np.zeros(idx.size, dtype=np.int32)
    info = lib().gls_oracle_gls_sampled(n, p, _ptr(M), n, _ptr(XL), n, _ptr(y), idx.size,
                                        _ptr(idx), _ptr(XRc), XRc.shape[0], _ptr(B), p,
                                        _ptr(status), float(tau), int(nthreads))
    if info < 0:
        raise ValueError("oracle rejected its arguments")
    return B, status, int(info)


def gls_factored(L, XL, y, XR, tau: float = TAU_FP64, nthreads: int = 1):
    """b_i for every column of XR given the Cholesky factor L of M (n x n,
    lower, as returned by ``potrf``).  Returns (B, status)."""
    L = np.asfortranarray(L, dtype=np.float64)
    n = L.shape[0]
    p = (0 if XL is None else np.asarray(XL).reshape(n, -1).shape[1]) + 1
    _, _, XL, y, XR = _prep(np.zeros((n, 0)), XL, y, XR, p)
    k = XR.shape[1]
    B = np.full((p, k), np.nan, dtype=np.float64, order="F")
    status = np.zeros(k, dtype=np.int32)
    r = lib().gls_oracle_gls_factored(n, p, _ptr(L), _ptr(XL), n, _ptr(y), k, _ptr(XR), n,
                                      _ptr(B), p, _ptr(status), float(tau), int(nthreads))
    if r < 0:
        raise ValueError("oracle rejected its arguments")
    return B, status
