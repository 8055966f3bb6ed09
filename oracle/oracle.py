"""ctypes front end of the FP64 C oracle (test infrastructure).

The arithmetic lives in ``dct_oracle.c``; this module only compiles it with
gcc, marshals numpy arrays and returns float64 results.  Definitions followed:
Eq. 1 (orthonormal DCT-II matrix), Eq. 2 (forward ``Q_h X Q_w^T`` and inverse
``Q_h^T Y Q_w``), Section 7.1 (rectangles), Section 2.1 (round trip equals X;
FFTW REDFT10/REDFT01 unnormalized pair, factor 2n per axis), Prop. 1 / Eq. 4
(transform, diagonal spectral operator, inverse).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

NORM_ORTHO = 0
NORM_NONE = 1
_DIR_FORWARD = 1
_DIR_INVERSE = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dct_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            f32p = ctypes.POINTER(ctypes.c_float)
            f64p = ctypes.POINTER(ctypes.c_double)
            for name in ("oracle_forward", "oracle_inverse", "oracle_roundtrip"):
                fn = getattr(lib, name)
                fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, f32p, f64p,
                               ctypes.c_int64, ctypes.c_int]
                fn.restype = ctypes.c_int
            lib.oracle_spectral.argtypes = [ctypes.c_int, ctypes.c_int, f64p, f32p, f64p,
                                            ctypes.c_int64, ctypes.c_int]
            lib.oracle_spectral.restype = ctypes.c_int
            lib.oracle_bruteforce.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, f32p, f64p]
            lib.oracle_bruteforce.restype = ctypes.c_int
            lib.oracle_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, f64p]
            lib.oracle_matrix.restype = None
            lib.oracle_cospi_frac.argtypes = [ctypes.c_int64, ctypes.c_int64]
            lib.oracle_cospi_frac.restype = ctypes.c_double
            lib.oracle_set_fault.argtypes = [ctypes.c_int]
            lib.oracle_default_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _as_batch(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim < 2:
        raise ValueError("need (..., h, w)")
    h, w = x.shape[-2:]
    batch = int(np.prod(x.shape[:-2], dtype=np.int64)) if x.ndim > 2 else 1
    return x, h, w, batch


def _run(name: str, x: np.ndarray, norm: int, threads: int) -> np.ndarray:
    lib = _load()
    x, h, w, batch = _as_batch(x)
    out = np.empty(x.shape, dtype=np.float64)
    if batch:
        rc = getattr(lib, name)(h, w, norm,
                                x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                batch, threads)
        if rc != 0:
            raise ValueError(f"{name} rejected h={h} w={w}")
    return out


def forward(x: np.ndarray, norm: int = NORM_ORTHO, threads: int = 0) -> np.ndarray:
    """Eq. 2 forward ``M_h X M_w^T`` of every trailing h x w array, in FP64."""
    return _run("oracle_forward", x, norm, threads)


def inverse(y: np.ndarray, norm: int = NORM_ORTHO, threads: int = 0) -> np.ndarray:
    """Eq. 2 inverse ``Q_h^T Y Q_w`` (DCT-III) of every trailing array, in FP64."""
    return _run("oracle_inverse", y, norm, threads)


def roundtrip(x: np.ndarray, norm: int = NORM_ORTHO, threads: int = 0) -> np.ndarray:
    """FP64 composition ``C^{-1}(C(X))`` (normalized); exact result is X."""
    return _run("oracle_roundtrip", x, norm, threads)


def spectral(x: np.ndarray, lam: np.ndarray, threads: int = 0) -> np.ndarray:
    """Prop. 1 / Eq. 4: ``U^T Lambda U X = Q_h^T (Lambda o (Q_h X Q_w^T)) Q_w``
    of every trailing h x w array, in FP64, with the orthonormal Q of Eq. 1;
    ``lam`` is the h x w diagonal (``lam[k, l]`` multiplies coefficient k, l)."""
    lib = _load()
    x, h, w, batch = _as_batch(x)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    if lam.shape != (h, w):
        raise ValueError(f"lambda must be ({h}, {w}), got {lam.shape}")
    out = np.empty(x.shape, dtype=np.float64)
    if batch:
        rc = lib.oracle_spectral(h, w, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), batch, threads)
        if rc != 0:
            raise ValueError(f"oracle_spectral rejected h={h} w={w}")
    return out


def bruteforce(x: np.ndarray, direction: str = "forward", norm: int = NORM_ORTHO) -> np.ndarray:
    """O(h^2 w^2) direct double sum with libm cosines, one array at a time."""
    lib = _load()
    x, h, w, batch = _as_batch(x)
    d = _DIR_FORWARD if direction == "forward" else _DIR_INVERSE
    xs = x.reshape(batch, h, w)
    out = np.empty((batch, h, w), dtype=np.float64)
    for b in range(batch):
        xb = np.ascontiguousarray(xs[b])
        ob = out[b]
        lib.oracle_bruteforce(h, w, d, norm,
                              xb.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              ob.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out.reshape(x.shape)


def matrix(n: int, direction: str = "forward", norm: int = NORM_ORTHO) -> np.ndarray:
    """The 1D operator M with 2D result ``M_h X M_w^T`` (ORTHO forward: Q_n)."""
    lib = _load()
    m = np.empty((n, n), dtype=np.float64)
    d = _DIR_FORWARD if direction == "forward" else _DIR_INVERSE
    lib.oracle_matrix(n, d, norm, m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return m


def cospi_frac(m: int, d: int) -> float:
    """cos(pi m / d) with exact integer argument reduction."""
    return _load().oracle_cospi_frac(m, d)


def set_fault(code: int) -> None:
    """Plant a known mistake in the oracle (tests of the pins only; 0 = off)."""
    _load().oracle_set_fault(int(code))


def default_threads() -> int:
    """Host threads the oracle uses by default (the process's CPU affinity)."""
    return int(_load().oracle_default_threads())
