"""CPU FP64 oracle for A X = B X Lambda (Eq. 1) — test infrastructure only.

Thin ctypes wrapper over ``oracle/oracle.c``: Cholesky (Eq. 2), C = U^-T A U^-1
by two triangular solves (Eq. 3), Householder tridiagonalisation and implicit
QL (variant TD, Section 2.2), inverse iteration on T, and X = U^-1 Y (Eq. 4),
plus a cyclic Jacobi brute force.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the GPU library.

Matrices are numpy float64 arrays in column-major (Fortran) order; every
function copies its inputs, so callers' arrays are never modified.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (plain C, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        lib.oracle_potrf.argtypes = [i64, dp, i64]
        lib.oracle_potrf.restype = ip
        lib.oracle_sygst.argtypes = [i64, dp, i64, dp, i64]
        lib.oracle_sygst.restype = None
        lib.oracle_backsolve.argtypes = [i64, i64, dp, i64, dp, i64]
        lib.oracle_backsolve.restype = None
        lib.oracle_tridiag.argtypes = [i64, dp, i64, dp, dp, dp]
        lib.oracle_tridiag.restype = None
        lib.oracle_apply_q.argtypes = [i64, dp, i64, dp, i64, dp, i64]
        lib.oracle_apply_q.restype = None
        lib.oracle_sturm_count.argtypes = [i64, dp, dp, ctypes.c_double]
        lib.oracle_sturm_count.restype = i64
        lib.oracle_tql.argtypes = [i64, dp, dp, dp, i64]
        lib.oracle_tql.restype = ip
        lib.oracle_tri_invit.argtypes = [i64, dp, dp, i64, dp, dp, i64]
        lib.oracle_tri_invit.restype = None
        lib.oracle_jacobi.argtypes = [i64, dp, i64, dp, dp, i64]
        lib.oracle_jacobi.restype = ip
        lib.oracle_gsyeig.argtypes = [i64, dp, i64, dp, i64, i64, ip, ip, dp, dp, i64]
        lib.oracle_gsyeig.restype = ip
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ip
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


class NotSPD(Exception):
    """Cholesky met a non-positive pivot; ``index`` is 1-based (Eq. 2)."""

    def __init__(self, index: int):
        super().__init__(f"B is not positive definite (pivot {index})")
        self.index = index


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def potrf(B) -> np.ndarray:
    """Upper U with B = U^T U (Eq. 2); strictly lower part returned as zeros."""
    Bc = _f64(B)
    n = Bc.shape[0]
    info = _load().oracle_potrf(n, _p(Bc), n)
    if info:
        raise NotSPD(info)
    return np.triu(Bc)


def sygst(A, U) -> np.ndarray:
    """C = U^-T A U^-1 (Eq. 3) from the lower triangle of A; full symmetric C."""
    Ac = _f64(A)
    Uc = _f64(U)
    n = Ac.shape[0]
    _load().oracle_sygst(n, _p(Ac), n, _p(Uc), n)
    return Ac


def backsolve(U, Y) -> np.ndarray:
    """X = U^-1 Y (Eq. 4)."""
    Uc = _f64(U)
    Yc = _f64(Y)
    if Yc.ndim == 1:
        Yc = Yc.reshape(-1, 1, order="F")
    n, s = Yc.shape
    _load().oracle_backsolve(n, s, _p(Uc), n, _p(Yc), n)
    return Yc


def tridiag(C):
    """Householder reduction Q^T C Q = T (Section 2.2): returns (d, e, reflectors, tau)."""
    Cc = _f64(C)
    n = Cc.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n, 1))
    tau = np.zeros(max(n, 1))
    _load().oracle_tridiag(n, _p(Cc), n, _p(d), _p(e), _p(tau))
    return d, e[: max(n - 1, 0)].copy(), Cc, tau


def apply_q(refl, tau, Z) -> np.ndarray:
    """Y = Q Z with Q the product of the reflectors left by :func:`tridiag`."""
    Zc = _f64(Z)
    if Zc.ndim == 1:
        Zc = Zc.reshape(-1, 1, order="F")
    n, s = Zc.shape
    R = _f64(refl)
    t = _f64(np.concatenate([tau, np.zeros(1)]))
    _load().oracle_apply_q(n, _p(R), n, _p(t), s, _p(Zc), n)
    return Zc


def sturm_count(d, e, x: float) -> int:
    """Number of eigenvalues of the tridiagonal (d, e) strictly below x."""
    dc = _f64(d)
    ec = _f64(np.concatenate([np.asarray(e, dtype=np.float64), np.zeros(1)]))
    return int(_load().oracle_sturm_count(len(dc), _p(dc), _p(ec), float(x)))


def tql(d, e, vectors: bool = False):
    """All eigenvalues (ascending) of the tridiagonal (d, e) by implicit QL,
    and the eigenvector matrix when ``vectors``."""
    dc = _f64(d)
    n = len(dc)
    ec = _f64(np.concatenate([np.asarray(e, dtype=np.float64), np.zeros(1)]))
    Z = None
    if vectors:
        Z = np.asfortranarray(np.eye(n))
        st = _load().oracle_tql(n, _p(dc), _p(ec), _p(Z), n)
    else:
        st = _load().oracle_tql(n, _p(dc), _p(ec), None, 0)
    if st:
        raise RuntimeError("implicit QL did not converge")
    return (dc, Z) if vectors else dc


def tri_invit(d, e, lam) -> np.ndarray:
    """Eigenvectors of the tridiagonal (d, e) for the ascending eigenvalues lam."""
    dc = _f64(d)
    n = len(dc)
    ec = _f64(np.concatenate([np.asarray(e, dtype=np.float64), np.zeros(1)]))
    lc = _f64(lam)
    s = len(lc)
    Z = np.zeros((n, s), order="F")
    _load().oracle_tri_invit(n, _p(dc), _p(ec), s, _p(lc), _p(Z), n)
    return Z


def jacobi(C):
    """Brute-force cyclic Jacobi on a small full symmetric C: (w ascending, V)."""
    Cc = _f64(C)
    n = Cc.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    st = _load().oracle_jacobi(n, _p(Cc), n, _p(w), _p(V), n)
    if st:
        raise RuntimeError("Jacobi did not converge")
    return w, V


def gsyeig(A, B, s: int, which: str = "smallest", vectors: str = "auto"):
    """The s smallest (or largest) eigenpairs of the pencil (A, B) (Eq. 1):
    returns (w ascending, X with X^T B X = I).  ``vectors``: "ql" accumulates
    all QL rotations (small n), "invit" uses inverse iteration on T."""
    Ac = _f64(A)
    Bc = _f64(B)
    n = Ac.shape[0]
    if not (1 <= s <= n):
        raise ValueError("need 1 <= s <= n")
    mode = {"ql": 0, "invit": 1}.get(vectors, 0 if n <= 1024 else 1)
    w = np.zeros(s)
    X = np.zeros((n, s), order="F")
    info = _load().oracle_gsyeig(n, _p(Ac), n, _p(Bc), n, s, 1 if which == "largest" else 0, mode, _p(w), _p(X), n)
    if info > 0:
        raise NotSPD(info)
    if info < 0:
        raise RuntimeError("implicit QL did not converge")
    return w, X
