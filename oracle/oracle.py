"""ctypes binding of the C oracle, plus the thresholds from ``oracle.theta``.

TEST INFRASTRUCTURE (see the package docstring). Arrays are numpy float64,
C-contiguous, square, row-major. Nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import build as _build
from . import theta as _theta

SCHEMES = {"new": 0, "ps": 1, "pade26": 2, "pade": 3}


class _Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("s", ctypes.c_int), ("products", ctypes.c_int),
                ("status", ctypes.c_int), ("norm1", ctypes.c_double)]


@dataclasses.dataclass
class Info:
    m: int
    s: int
    products: int
    status: int
    norm1: float


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        L.orc_gemm.argtypes = [i64, dp, dp, dp]
        L.orc_norm1.argtypes = [i64, dp]
        L.orc_norm1.restype = ctypes.c_double
        L.orc_taylor_new.argtypes = [i64, dp, ctypes.c_int, dp]
        L.orc_taylor_ps.argtypes = [i64, dp, ctypes.c_int, dp]
        L.orc_pade.argtypes = [i64, dp, ctypes.c_int, dp]
        L.orc_solve.argtypes = [i64, dp, dp, dp]
        L.orc_select.argtypes = [ctypes.c_double, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)]
        L.orc_expm.argtypes = [i64, dp, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(_Info)]
        L.orc_expm_upper.argtypes = [i64, dp, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(_Info)]
        L.orc_is_upper.argtypes = [i64, dp]
        L.orc_coeffs.argtypes = [ctypes.c_int, dp]
        L.orc_set_mutation.argtypes = [ctypes.c_int]
        L.orc_product_count.restype = ctypes.c_longlong
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_power_norms.argtypes = [i64, dp, dp]
        L.orc_select_certified.argtypes = [dp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _sq(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a


def gemm(A, B) -> np.ndarray:
    A, B = _sq(A), _sq(B)
    C = np.empty_like(A)
    lib().orc_gemm(A.shape[0], _p(A), _p(B), _p(C))
    return C


def norm1(A) -> float:
    A = _sq(A)
    return lib().orc_norm1(A.shape[0], _p(A))


def taylor_new(X, m: int) -> np.ndarray:
    X = _sq(X)
    T = np.empty_like(X)
    if lib().orc_taylor_new(X.shape[0], _p(X), m, _p(T)) < 0:
        raise ValueError(f"unsupported degree {m}")
    return T


def taylor_ps(X, m: int) -> np.ndarray:
    X = _sq(X)
    T = np.empty_like(X)
    if lib().orc_taylor_ps(X.shape[0], _p(X), m, _p(T)) < 0:
        raise ValueError(f"unsupported degree {m}")
    return T


def pade(X, two_m: int) -> np.ndarray:
    X = _sq(X)
    R = np.empty_like(X)
    rc = lib().orc_pade(X.shape[0], _p(X), two_m, _p(R))
    if rc < 0:
        raise ValueError(f"pade r_{two_m} failed ({rc})")
    return R


def solve(P, Q) -> np.ndarray:
    """P^-1 Q by the comparator's Gaussian elimination with partial pivoting on
    all right-hand sides at once, then back substitution (the solve of eq. pade26)."""
    P = _sq(P).copy()
    Q = _sq(Q).copy()
    if P.shape != Q.shape:
        raise ValueError("P and Q must have the same shape")
    R = np.empty_like(P)
    if lib().orc_solve(P.shape[0], _p(P), _p(Q), _p(R)):
        raise ValueError("singular matrix")
    return R


def theta_array(scheme: str, u: float = 2.0 ** -53) -> np.ndarray:
    return np.array(_theta.theta_array(scheme, u), dtype=np.float64)


def select(norm: float, scheme: str = "new", u: float = 2.0 ** -53) -> tuple[int, int]:
    th = theta_array(scheme, u)
    m, s = ctypes.c_int(), ctypes.c_int()
    rc = lib().orc_select(norm, SCHEMES[scheme], _p(th), ctypes.byref(m), ctypes.byref(s))
    if rc:
        raise ValueError("non-finite norm")
    return m.value, s.value


def expm(A, scheme: str = "new", u: float = 2.0 ** -53, m: int | None = None,
         s: int | None = None) -> tuple[np.ndarray, Info]:
    """exp(A) by scaling and squaring; (m, s) selected by the theta rule unless
    both are given."""
    A = _sq(A)
    out = np.empty_like(A)
    th = theta_array(scheme, u)
    info = _Info()
    mf = m if (m is not None and s is not None) else 0
    sf = s if (m is not None and s is not None) else -1
    lib().orc_expm(A.shape[0], _p(A), _p(out), SCHEMES[scheme], _p(th), mf, sf, ctypes.byref(info))
    return out, Info(info.m, info.s, info.products, info.status, info.norm1)


def expm_upper(A, scheme: str = "new", u: float = 2.0 ** -53, m: int | None = None,
               s: int | None = None) -> tuple[np.ndarray, Info]:
    """exp(A) for an upper triangular A, with the exact diagonal and first
    superdiagonal of exp(2^-q A) put in after the polynomial and every squaring
    (Section 5, concluding remarks). Raises ValueError when A is not upper
    triangular."""
    A = _sq(A)
    if not lib().orc_is_upper(A.shape[0], _p(A)):
        raise ValueError("matrix is not upper triangular")
    out = np.empty_like(A)
    th = theta_array(scheme, u)
    info = _Info()
    mf = m if (m is not None and s is not None) else 0
    sf = s if (m is not None and s is not None) else -1
    lib().orc_expm_upper(A.shape[0], _p(A), _p(out), SCHEMES[scheme], _p(th), mf, sf, ctypes.byref(info))
    return out, Info(info.m, info.s, info.products, info.status, info.norm1)


def coeffs(which: int) -> np.ndarray:
    buf = np.zeros(64)
    n = lib().orc_coeffs(which, _p(buf))
    return buf[:n].copy()


def set_mutation(code: int) -> None:
    lib().orc_set_mutation(code)


def product_count() -> int:
    return lib().orc_product_count()


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Cap the threads of the oracle's products (timing only; results do not change)."""
    lib().orc_set_num_threads(int(n))


def power_norms(A) -> np.ndarray:
    """[||A||_1, ||A^2||_1, ||A^3||_1, ||A^4||_1] from oracle products."""
    A = _sq(A)
    out = np.zeros(4)
    lib().orc_power_norms(A.shape[0], _p(A), _p(out))
    return out


def select_certified(norms, scheme: str = "new", u: float = 2.0 ** -53) -> tuple[int, int]:
    """Cheapest (m, s) certified by ||A||_1 or by alpha_2 = max(||A^2||^(1/2), ||A^3||^(1/3))."""
    nv = np.ascontiguousarray(np.asarray(norms, dtype=np.float64)[:3])
    th = theta_array(scheme, u)
    m, s = ctypes.c_int(), ctypes.c_int()
    if lib().orc_select_certified(_p(nv), SCHEMES[scheme], _p(th), ctypes.byref(m), ctypes.byref(s)):
        raise ValueError("non-finite norms")
    return m.value, s.value
