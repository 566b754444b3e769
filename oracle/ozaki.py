"""Oracle of the FP64 GEMM emulated with 8-bit digit slices (the Ozaki
scheme: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free transformations
of matrix multiplication by using fast routines of matrix multiplication and
its applications", Numer. Algorithms 59, 2012, with integer digits).  Not in
the paper: it stands behind the library's emulated FP64 updates.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle/``): only ``tests/`` may
import it; the library never does, and this file shares no code with it.

The method, step by step, in exact integer arithmetic (Python integers, so
nothing here rounds except the final conversion to binary64):

1. Row scaling.  For row i of op(A), x_i = the exponent of its largest
   magnitude (max in [2^(x_i - 1), 2^x_i)); e_i = x_i + 1, so every scaled
   entry q = a 2^-e_i has |q| < 1/2.  Columns of op(B) likewise (f_j).  A row
   of zeros has e = 0.
2. Fixed point.  Q = round(q 2^(8S)) with ties away from zero (|q| < 1/2
   keeps |Q| < 2^(8S-1)).
3. Digits.  Q = sum_{s=1..S} d_s 256^(S-s): the S - 1 low digits are the
   balanced residues ((Q + 128) mod 256) - 128 in [-128, 127], taken from the
   bottom; the top digit d_1 is what remains (|d_1| <= 128).
4. Products.  (op(A) op(B))_ij ~ 2^(e_i + f_j) sum over digit pairs (s, t)
   with s + t <= S + 1 of 2^(-8(s + t)) sum_k dA_s(i, k) dB_t(k, j); pairs
   with s + t > S + 1 are left out.
5. Conversion.  With T_L the exact sum of the pairs of level L = s + t,
   V = sum_L T_L 2^(8(S + 1 - L)) is an integer; the result is V 2^(e_i + f_j
   - 8(S + 1)), rounded once to binary64 (round to nearest, ties to even).

The result is a deterministic function of A and B, so an implementation that
keeps every intermediate sum exact and rounds once at the end returns the
same binary64 values.
"""
from __future__ import annotations

import math

import numpy as np


def exponent_of_max(v: float) -> int:
    """e with max < 2^(e - 1) for a row maximum v >= 0 (0 for v = 0)."""
    if v == 0.0:
        return 0
    _, x = math.frexp(v)          # v = m 2^x, m in [1/2, 1)
    return x + 1


def fixed_point(a: float, e: int, S: int) -> int:
    """round(a 2^(8S - e)), ties away from zero, exactly (a binary64)."""
    if a == 0.0:
        return 0
    num, den = abs(a).as_integer_ratio()        # |a| = num / den, den a power of two
    shift = 8 * S - e
    if shift >= 0:
        num <<= shift
    else:
        den <<= -shift
    q = (2 * num + den) // (2 * den)            # floor(num / den + 1/2)
    return -q if a < 0 else q


def digits(Q: int, S: int):
    """[d_1, ..., d_S], most significant first, with Q = sum d_s 256^(S - s)."""
    low = []
    for _ in range(S - 1):
        d = ((Q + 128) % 256) - 128
        low.append(d)
        Q = (Q - d) // 256
    return [Q] + low[::-1]


def slice_rows(X: np.ndarray, S: int):
    """Exponents (one per row) and digit planes D[s][i][k] of the rows of X."""
    X = np.asarray(X, dtype=np.float64)
    rows, k = X.shape
    e = [exponent_of_max(float(np.max(np.abs(X[i])))) if k else 0 for i in range(rows)]
    D = np.zeros((S, rows, k), dtype=np.int64)      # |d| <= 128
    for i in range(rows):
        for kk in range(k):
            ds = digits(fixed_point(float(X[i, kk]), e[i], S), S)
            for s in range(S):
                D[s, i, kk] = ds[s]
    return e, D


def level_sums(DA, DB, S: int):
    """T[L] = sum over pairs (s, t), s + t = L <= S + 1, of DA_s DB_t^T
    (exact: int64 products of digits <= 2^14, sums far below 2^63 for the
    sizes this oracle is used at)."""
    T = {}
    for s in range(1, S + 1):
        for t in range(1, S + 2 - s):
            P = DA[s - 1].dot(DB[t - 1].T)
            T[s + t] = P if (s + t) not in T else T[s + t] + P
    return T


def gemm(A, B, S: int = 7, ta: bool = False, tb: bool = False) -> np.ndarray:
    """op(A) op(B) by the emulation with S digit planes (6, 7 or 8), as
    binary64.  Small sizes only (k <= 2^20 keeps the int64 sums exact)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert S in (6, 7, 8)
    opA = A.T if ta else A
    opB = B.T if tb else B
    eA, DA = slice_rows(opA, S)
    eB, DB = slice_rows(opB.T, S)           # rows of op(B)^T = columns of op(B)
    T = level_sums(DA, DB, S)
    m, n = opA.shape[0], opB.shape[1]
    C = np.zeros((m, n))
    lmax = S + 1
    for i in range(m):
        for j in range(n):
            V = sum(int(T[L][i, j]) << (8 * (lmax - L)) for L in T)
            scale = eA[i] + eB[j] - 8 * lmax
            C[i, j] = math.ldexp(float(V), scale) if V else 0.0
    return np.asfortranarray(C)
