"""Plain CPU FP64 oracle for the recursive factorizations of Peise & Bientinesi,
"Recursive Algorithms for Dense Linear Algebra: The ReLAPACK Collection"
(arXiv 1602.06763).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library's
product path never does; it shares no code with the CUDA implementation.

The arithmetic lives in ``oracle.c`` (compiled to ``liboracle.so`` by
``oracle/build.py``); this module only marshals numpy arrays.  The oracle of
the emulated FP64 GEMM (not in the paper) is ``oracle/ozaki.py``, exact
integer arithmetic in Python and numpy.  Matrices are
numpy float64 arrays in Fortran (column-major) order, as LAPACK stores them;
each call works on a copy unless ``inplace=True``.

Passages followed (Section / Figure of the paper):
  potrf   Section 5 (xpotrf), Section 3 halving scheme, potf2 base case
  getrf   Section 5 (xgetrf, P L U with row pivoting), Section 3 halving
  trtri   Section 3, Fig. 4 updates (1)-(4), trti2 base case
  lauum   Section 5 (xlauum, A := L^T L)
  potri   Section 5 (xtrtri as the building block of potri) = trtri + lauum
  split   Section 3 footnote: halves that are multiples of 8 when the size allows
"""
from __future__ import annotations

import ctypes
import os
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "liboracle.so")
        if not os.path.exists(path):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(path)
        sig = {
            "or_split": (_i64, [_i64]),
            "or_potf2": (_i64, [_i64, _ptr, _i64]),
            "or_potrf": (_i64, [_i64, _ptr, _i64, _i64]),
            "or_getf2": (_i64, [_i64, _i64, _ptr, _i64, _ptr]),
            "or_getrf": (_i64, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_laswp": (None, [_i64, _ptr, _i64, _i64, _i64, _ptr]),
            "or_trti2": (None, [ctypes.c_int, _i64, _ptr, _i64]),
            "or_trtri": (_i64, [ctypes.c_int, _i64, _ptr, _i64, _i64]),
            "or_lauu2": (None, [_i64, _ptr, _i64]),
            "or_lauum": (None, [_i64, _ptr, _i64, _i64]),
            "or_potri": (_i64, [_i64, _ptr, _i64, _i64]),
            "or_getrs": (None, [_i64, _i64, _ptr, _i64, _ptr, _ptr, _i64]),
            "or_potrs": (None, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_getri": (None, [_i64, _ptr, _i64, _ptr, _ptr, _i64]),
            "or_zpotrf": (_i64, [_i64, _ptr, _i64, _i64]),
            "or_zgetrf": (_i64, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_zlaswp": (None, [_i64, _ptr, _i64, _i64, _i64, _ptr]),
            "or_res_zchol": (_dbl, [_i64, _ptr, _i64, _ptr, _i64]),
            "or_res_zlu": (_dbl, [_i64, _i64, _ptr, _i64, _ptr, _i64, _ptr]),
            "or_ztrtri": (_i64, [ctypes.c_int, _i64, _ptr, _i64]),
            "or_zlauum": (None, [_i64, _ptr, _i64]),
            "or_zpotri": (_i64, [_i64, _ptr, _i64]),
            "or_zgetri": (None, [_i64, _ptr, _i64, _ptr, _ptr, _i64]),
            "or_sygst": (_i64, [ctypes.c_int, _i64, _ptr, _i64, _ptr, _i64]),
            "or_gemm": (None, [ctypes.c_int, ctypes.c_int, _i64, _i64, _i64, _dbl,
                               _ptr, _i64, _ptr, _i64, _ptr, _i64]),
            "or_syrk_lower": (None, [ctypes.c_int, _i64, _i64, _dbl, _ptr, _i64, _ptr, _i64]),
            "or_trsm_llnx": (None, [ctypes.c_int, _i64, _i64, _dbl, _ptr, _i64, _ptr, _i64]),
            "or_trsm_rltn": (None, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_trsm_lunn": (None, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_trsm_lltn": (None, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_trmm_rlnn": (None, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_trmm_lltn": (None, [_i64, _i64, _ptr, _i64, _ptr, _i64]),
            "or_res_chol": (_dbl, [_i64, _ptr, _i64, _ptr, _i64]),
            "or_res_lu": (_dbl, [_i64, _i64, _ptr, _i64, _ptr, _i64, _ptr]),
            "or_res_trtri": (_dbl, [_i64, _ptr, _i64, _ptr, _i64]),
            "or_res_potri": (_dbl, [_i64, _ptr, _i64, _ptr, _i64]),
            "or_probe_chol": (_dbl, [_i64, _ptr, _i64, _ptr, _i64, _ptr]),
            "or_probe_lu": (_dbl, [_i64, _ptr, _i64, _ptr, _i64, _ptr, _ptr]),
            "or_probe_trtri": (_dbl, [_i64, _ptr, _i64, _ptr, _i64, _ptr]),
            "or_probe_potri": (_dbl, [_i64, _ptr, _i64, _ptr, _i64, _ptr]),
            "or_backward_error": (_dbl, [_i64, _i64, _ptr, _i64, _ptr, _i64, _ptr, _i64]),
            "or_trtri_level_flops": (_dbl, [_i64, _i64, _ptr, _i64, _i64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _f64(a, copy=True):
    a = np.asarray(a, dtype=np.float64)
    if copy:
        return np.array(a, dtype=np.float64, order="F", copy=True)
    if not a.flags.f_contiguous:
        raise ValueError("in-place oracle calls need a Fortran-ordered float64 array")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ld(a):
    return max(1, a.shape[0])


def split(n: int) -> int:
    """Section 3 footnote: first half size, a multiple of 8 when the size allows."""
    return int(_lib().or_split(n))


def potf2(A, inplace=False):
    A = _f64(A, not inplace)
    info = _lib().or_potf2(A.shape[0], _p(A), _ld(A))
    return A, int(info)


def potrf(A, c=24, inplace=False):
    """Recursive lower Cholesky; returns (A with L in its lower triangle, info)."""
    A = _f64(A, not inplace)
    info = _lib().or_potrf(A.shape[0], _p(A), _ld(A), c)
    return A, int(info)


def getf2(A, inplace=False):
    A = _f64(A, not inplace)
    m, n = A.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    info = _lib().or_getf2(m, n, _p(A), _ld(A), _p(ipiv))
    return A, ipiv[: min(m, n)], int(info)


def getrf(A, c=24, inplace=False):
    """Recursive LU with row pivoting; returns (LU, ipiv 1-based int32, info)."""
    A = _f64(A, not inplace)
    m, n = A.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    info = _lib().or_getrf(m, n, _p(A), _ld(A), _p(ipiv), c)
    return A, ipiv[: min(m, n)], int(info)


def laswp(A, k1, k2, ipiv, inplace=False):
    A = _f64(A, not inplace)
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _lib().or_laswp(A.shape[1], _p(A), _ld(A), k1, k2, _p(ipiv))
    return A


def trti2(A, unit=False, inplace=False):
    A = _f64(A, not inplace)
    _lib().or_trti2(int(unit), A.shape[0], _p(A), _ld(A))
    return A


def trtri(A, unit=False, c=24, inplace=False):
    """Recursive lower triangular inverse (Fig. 4); returns (A, info)."""
    A = _f64(A, not inplace)
    info = _lib().or_trtri(int(unit), A.shape[0], _p(A), _ld(A), c)
    return A, int(info)


def lauu2(A, inplace=False):
    A = _f64(A, not inplace)
    _lib().or_lauu2(A.shape[0], _p(A), _ld(A))
    return A


def lauum(A, c=24, inplace=False):
    """Recursive A := L^T L (lower triangle written)."""
    A = _f64(A, not inplace)
    _lib().or_lauum(A.shape[0], _p(A), _ld(A), c)
    return A


def potri(A, c=24, inplace=False):
    """trtri then lauum on the Cholesky factor stored in A; returns (A, info)."""
    A = _f64(A, not inplace)
    info = _lib().or_potri(A.shape[0], _p(A), _ld(A), c)
    return A, int(info)


def gemm(A, B, C, alpha=1.0, ta=False, tb=False):
    """C + alpha op(A) op(B) by the plain definition (returns a new array)."""
    A = _f64(A)
    B = _f64(B)
    C = _f64(C)
    m, n = C.shape
    k = A.shape[0] if ta else A.shape[1]
    _lib().or_gemm(int(ta), int(tb), m, n, k, alpha, _p(A), _ld(A), _p(B), _ld(B),
                   _p(C), _ld(C))
    return C


def syrk_lower(A, C, alpha=1.0, trans=False):
    """Lower triangle of C + alpha op(A) op(A)^T (op(A) = A^T if trans)."""
    A = _f64(A)
    C = _f64(C)
    n = C.shape[0]
    k = A.shape[0] if trans else A.shape[1]
    _lib().or_syrk_lower(int(trans), n, k, alpha, _p(A), _ld(A), _p(C), _ld(C))
    return C


def trsm_lln(L, B, alpha=1.0, unit=False):
    """alpha L^{-1} B, L lower (forward substitution by columns)."""
    L = _f64(L)
    B = _f64(B)
    _lib().or_trsm_llnx(int(unit), B.shape[0], B.shape[1], alpha, _p(L), _ld(L), _p(B), _ld(B))
    return B


def trsm_rlt(L, B):
    """B L^{-T}, L lower non-unit."""
    L = _f64(L)
    B = _f64(B)
    _lib().or_trsm_rltn(B.shape[0], B.shape[1], _p(L), _ld(L), _p(B), _ld(B))
    return B


def trsm_lun(U, B):
    """U^{-1} B, U upper non-unit (back substitution)."""
    U = _f64(U)
    B = _f64(B)
    _lib().or_trsm_lunn(B.shape[0], B.shape[1], _p(U), _ld(U), _p(B), _ld(B))
    return B


def trsm_llt(L, B):
    """L^{-T} B, L lower non-unit."""
    L = _f64(L)
    B = _f64(B)
    _lib().or_trsm_lltn(B.shape[0], B.shape[1], _p(L), _ld(L), _p(B), _ld(B))
    return B


def trmm_rln(L, B):
    """B L, L lower non-unit."""
    L = _f64(L)
    B = _f64(B)
    _lib().or_trmm_rlnn(B.shape[0], B.shape[1], _p(L), _ld(L), _p(B), _ld(B))
    return B


def trmm_llt(L, B):
    """L^T B, L lower non-unit."""
    L = _f64(L)
    B = _f64(B)
    _lib().or_trmm_lltn(B.shape[0], B.shape[1], _p(L), _ld(L), _p(B), _ld(B))
    return B


def getrs(LU, ipiv, B):
    LU = _f64(LU, copy=False) if np.asarray(LU).flags.f_contiguous else _f64(LU)
    B = _f64(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _lib().or_getrs(LU.shape[0], B.shape[1], _p(LU), _ld(LU), _p(ipiv), _p(B), _ld(B))
    return B


def potrs(L, B):
    L = _f64(L, copy=False) if np.asarray(L).flags.f_contiguous else _f64(L)
    B = _f64(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    _lib().or_potrs(L.shape[0], B.shape[1], _p(L), _ld(L), _p(B), _ld(B))
    return B


def getri(LU, ipiv):
    """A^{-1} from P A = L U (LU and 1-based ipiv as or_getrf returns them)."""
    LU = _f64(LU, copy=False) if np.asarray(LU).flags.f_contiguous else _f64(LU)
    n = LU.shape[0]
    X = np.zeros((n, n), order="F")
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _lib().or_getri(n, _p(LU), _ld(LU), _p(ipiv), _p(X), _ld(X))
    return X


def _c128(a, copy=True):
    a = np.asarray(a, dtype=np.complex128)
    return np.array(a, dtype=np.complex128, order="F", copy=True) if copy else np.asfortranarray(a)


def zpotrf(A, c=24):
    """Recursive complex Cholesky A = L L^H (lower); returns (A with L, info)."""
    A = _c128(A)
    info = _lib().or_zpotrf(A.shape[0], _p(A), _ld(A), c)
    return A, int(info)


def zgetrf(A, c=24):
    """Recursive complex LU with partial pivoting on |Re| + |Im|; returns
    (LU, 1-based ipiv, info)."""
    A = _c128(A)
    m, n = A.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    info = _lib().or_zgetrf(m, n, _p(A), _ld(A), _p(ipiv), c)
    return A, ipiv[:min(m, n)], int(info)


def ztrtri(L, unit=False):
    """L^{-1} (lower, complex), by substitution; returns (A, info)."""
    L = _c128(L)
    info = _lib().or_ztrtri(int(unit), L.shape[0], _p(L), _ld(L))
    return L, int(info)


def zlauum(L):
    """L^H L (lower triangle written)."""
    L = _c128(L)
    _lib().or_zlauum(L.shape[0], _p(L), _ld(L))
    return L


def zpotri(L):
    """(L L^H)^{-1} from the factor L; returns (A, info)."""
    L = _c128(L)
    info = _lib().or_zpotri(L.shape[0], _p(L), _ld(L))
    return L, int(info)


def zgetri(LU, ipiv):
    """A^{-1} from P A = L U (complex)."""
    LU = _c128(LU)
    n = LU.shape[0]
    X = np.zeros((n, n), dtype=np.complex128, order="F")
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _lib().or_zgetri(n, _p(LU), _ld(LU), _p(piv), _p(X), _ld(X))
    return X


def res_zchol(A0, L):
    """||A - L L^H||_1 / (n eps ||A||_1), eps = 2^-53 (lower parts used)."""
    A0, L = _c128(A0), _c128(L)
    return float(_lib().or_res_zchol(A0.shape[0], _p(A0), _ld(A0), _p(L), _ld(L)))


def res_zlu(A0, LU, ipiv):
    """||P A - L U||_1 / (n eps ||A||_1)."""
    A0, LU = _c128(A0), _c128(LU)
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    return float(_lib().or_res_zlu(A0.shape[0], A0.shape[1], _p(A0), _ld(A0), _p(LU), _ld(LU), _p(ipiv)))


def sygst(itype, A, L):
    """itype 1: L^{-1} A L^{-T}; itype 2/3: L^T A L (A symmetric, lower triangle
    read and written; the strictly upper part of the result is A's)."""
    A = _f64(A)
    L = _f64(L, copy=False) if np.asarray(L).flags.f_contiguous else _f64(L)
    rc = _lib().or_sygst(int(itype), A.shape[0], _p(A), _ld(A), _p(L), _ld(L))
    if rc != 0:
        raise ValueError("or_sygst failed: %d" % rc)
    return A


def _ro(a):
    a = np.asarray(a, dtype=np.float64)
    return a if a.flags.f_contiguous else np.asfortranarray(a)


def res_chol(A0, L):
    """||A - L L^T||_1 / (n eps ||A||_1), eps = 2^-53 (lower parts used)."""
    A0, L = _ro(A0), _ro(L)
    return float(_lib().or_res_chol(A0.shape[0], _p(A0), _ld(A0), _p(L), _ld(L)))


def res_lu(A0, LU, ipiv):
    """||P A - L U||_1 / (max(m,n) eps ||A||_1)."""
    A0, LU = _ro(A0), _ro(LU)
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    m, n = A0.shape
    return float(_lib().or_res_lu(m, n, _p(A0), _ld(A0), _p(LU), _ld(LU), _p(ipiv)))


def res_trtri(L, X):
    """||L X - I||_1 / (n eps ||L||_1 ||X||_1) (lower parts used)."""
    L, X = _ro(L), _ro(X)
    return float(_lib().or_res_trtri(L.shape[0], _p(L), _ld(L), _p(X), _ld(X)))


def res_potri(A0, X):
    """||A X - I||_1 / (n eps ||A||_1 ||X||_1), A and X symmetric (lower)."""
    A0, X = _ro(A0), _ro(X)
    return float(_lib().or_res_potri(A0.shape[0], _p(A0), _ld(A0), _p(X), _ld(X)))


def probe_chol(A0, L, x):
    """||A x - L L^T x||_inf / (n eps ||A||_inf ||x||_inf), O(n^2)."""
    A0, L = _ro(A0), _ro(L)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_lib().or_probe_chol(A0.shape[0], _p(A0), _ld(A0), _p(L), _ld(L), _p(x)))


def probe_lu(A0, LU, ipiv, x):
    """||P A x - L U x||_inf / (n eps ||A||_inf ||x||_inf), O(n^2)."""
    A0, LU = _ro(A0), _ro(LU)
    ipiv = np.ascontiguousarray(ipiv, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_lib().or_probe_lu(A0.shape[0], _p(A0), _ld(A0), _p(LU), _ld(LU),
                                    _p(ipiv), _p(x)))


def probe_trtri(L, X, x):
    """||L X x - x||_inf / (n eps ||L||_inf ||X||_inf ||x||_inf), O(n^2)."""
    L, X = _ro(L), _ro(X)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_lib().or_probe_trtri(L.shape[0], _p(L), _ld(L), _p(X), _ld(X), _p(x)))


def probe_potri(A0, X, x):
    """||A X x - x||_inf / (n eps ||A||_inf ||X||_inf ||x||_inf), O(n^2)."""
    A0, X = _ro(A0), _ro(X)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_lib().or_probe_potri(A0.shape[0], _p(A0), _ld(A0), _p(X), _ld(X), _p(x)))


def backward_error(A, X, B):
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A, X, B = _ro(A), _ro(X), _ro(B)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
        B = B.reshape(-1, 1, order="F")
    return float(_lib().or_backward_error(A.shape[0], X.shape[1], _p(A), _ld(A),
                                          _p(X), _ld(X), _p(B), _ld(B)))


def trtri_level_flops(n, c=24, levels=8):
    """Flops of the TRMM+TRSM calls per recursion level of trtri, and the total."""
    shares = np.zeros(levels, dtype=np.float64)
    total = _lib().or_trtri_level_flops(n, c, _p(shares), levels, 0)
    return shares, float(total)


def tril(A):
    return np.tril(np.asarray(A))
