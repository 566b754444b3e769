"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: the paper's printed
per-level flop shares (Section 3, Fig. 5), closed forms of 2x2 cases, factors
that are exact in binary64 (integer / dyadic constructions), exact rational
brute force on tiny inputs, LAPACK through scipy, and the backward-error bound
of the required accuracy (residual / (n eps ||A||) <= 10).  The planted-mistake
tests show that each check fails when a plausible error (a dropped update, a
wrong sign, a transposed block, a swapped pivot) is put into the oracle's
output.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from paper_1602_06763_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -53
BOUND = 10.0


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------
# split rule and the paper's flop shares
# ----------------------------------------------------------------------------

def test_split_rule(oracle):
    for n in range(2, 600):
        n1 = oracle.split(n)
        assert 0 < n1 < n
        if n >= 16:
            assert n1 % 8 == 0 and abs(n1 - n / 2) <= 4


def _round_half_up(x, d):
    q = 10 ** d
    return math.floor(x * q + 0.5) / q


def test_trtri_level_flop_shares_match_paper(oracle):
    g = load("trtri_flop_shares.json")
    # exact halving (a power-of-two multiple of 8) reproduces the paper's
    # 2 (n/2)^3 / (n^3/3) derivation level by level
    n = 2048
    shares, total = oracle.trtri_level_flops(n, c=g["c_paper"], levels=4)
    assert total == pytest.approx(n ** 3 / 3.0, rel=1e-12)
    pct = 100.0 * shares / (n ** 3 / 3.0)
    for got, want, d in zip(pct, g["shares_percent_printed"], g["printed_decimals"]):
        assert _round_half_up(got, d) == pytest.approx(want)
    # the paper's own size n = 2000 with the paper's split rule
    shares, total = oracle.trtri_level_flops(g["n_paper"], c=g["c_paper"], levels=4)
    pct = 100.0 * shares / (g["n_paper"] ** 3 / 3.0)
    assert np.all(np.abs(pct - np.array(g["shares_percent_printed"])) < 0.06)
    # TRMM + TRSM carry more than 99.6 % of the flops for c < 100
    for c in (24, 99):
        shares, total = oracle.trtri_level_flops(g["n_paper"], c=c, levels=64)
        assert 100.0 * shares.sum() / total >= g["blas3_share_percent_at_least"]


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------

def test_closed_forms_2x2(oracle):
    g = load("closed_forms_2x2.json")
    A = np.array(g["potrf"]["A"], order="F")
    L, info = oracle.potrf(A, c=1)
    assert info == 0
    assert np.array_equal(np.tril(L), np.array(g["potrf"]["L"]))

    A = np.array(g["getrf"]["A"], order="F")
    LU, ipiv, info = oracle.getrf(A, c=1)
    assert info == 0 and list(ipiv) == g["getrf"]["ipiv"]
    assert LU[0, 0] == 3.0 and LU[0, 1] == 4.0
    assert LU[1, 0] == 1.0 / 3.0                     # one correctly rounded division
    assert abs(LU[1, 1] - 2.0 / 3.0) <= 2 * EPS      # u22 = 2 - (1/3)*4

    L = np.array(g["trtri"]["L"], order="F")
    X, info = oracle.trtri(L, c=1)
    assert info == 0 and np.array_equal(np.tril(X), np.array(g["trtri"]["X"]))

    L = np.array(g["lauum"]["L"], order="F")
    A = oracle.lauum(L, c=1)
    assert np.array_equal(np.tril(A), np.array(g["lauum"]["A"]))


def test_closed_forms_3x3_symbolic(oracle):
    sympy = pytest.importorskip("sympy")
    a, b, c, d, e, f = (sympy.Rational(v) for v in (9, 3, 6, 5, 2, 14))
    M = sympy.Matrix([[a, b, c], [b, d, e], [c, e, f]])
    Lsym = M.cholesky(hermitian=False)
    A = np.array(M.tolist(), dtype=np.float64, order="F")
    L, info = oracle.potrf(A, c=1)
    assert info == 0
    Lexp = np.array(Lsym.evalf(30).tolist(), dtype=np.float64)
    assert np.max(np.abs(np.tril(L) - Lexp)) <= 8 * EPS * np.max(np.abs(Lexp))
    # TRTRI of the symbolic factor, LAUUM of it
    X, info = oracle.trtri(np.asfortranarray(Lexp), c=1)
    Xexp = np.array(Lsym.inv().evalf(30).tolist(), dtype=np.float64)
    assert np.max(np.abs(np.tril(X) - Xexp)) <= 16 * EPS * np.max(np.abs(Xexp))
    P = oracle.lauum(np.asfortranarray(Lexp), c=1)
    Pexp = np.array((Lsym.T * Lsym).evalf(30).tolist(), dtype=np.float64)
    assert np.max(np.abs(np.tril(P) - np.tril(Pexp))) <= 16 * EPS * np.max(np.abs(Pexp))


# ----------------------------------------------------------------------------
# exact constructions (bit-exact expected results)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("c", [1, 2, 24, 6])
def test_integer_cholesky_6x6_exact(oracle, c):
    L = inputs.integer_chol_6()
    A = inputs.product_lower(L)
    F, info = oracle.potrf(A, c=c)
    assert info == 0
    assert np.array_equal(np.tril(F), L)
    assert np.array_equal(np.triu(F, 1), np.triu(A, 1))   # upper part untouched


@pytest.mark.parametrize("n,c", [(37, 1), (100, 24), (130, 130), (200, 8)])
def test_integer_cholesky_exact(oracle, n, c):
    L = inputs.integer_chol(n, seed=inputs.seed_for(0, n))
    A = inputs.product_lower(L)
    F, info = oracle.potrf(A, c=c)
    assert info == 0 and np.array_equal(np.tril(F), L)
    assert oracle.res_chol(A, F) == 0.0


@pytest.mark.parametrize("n,c", [(7, 1), (50, 2), (130, 24), (97, 97), (160, 16)])
def test_dyadic_lu_exact(oracle, n, c):
    A, L, U, perm = inputs.dyadic_lu(n, seed=inputs.seed_for(1, n))
    F, ipiv, info = oracle.getrf(A, c=c)
    assert info == 0
    assert np.array_equal(ipiv, inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1) + np.eye(n), L)
    assert np.array_equal(np.triu(F), U)


def test_lu_rectangular_shapes(oracle):
    for m, n in [(90, 40), (40, 90), (65, 64), (1, 30), (30, 1)]:
        A = inputs.uniform(m, n, seed=inputs.seed_for(1, 1000 + m + n))
        F, ipiv, info = oracle.getrf(A, c=8)
        assert info == 0 and oracle.res_lu(A, F, ipiv) <= BOUND
        Fs, piv, infos = lapack.dgetrf(A)
        assert np.array_equal(ipiv, piv + 1)


@pytest.mark.parametrize("n,c", [(5, 1), (64, 24), (150, 16), (201, 201)])
def test_integer_trtri_exact(oracle, n, c):
    L = inputs.integer_trtri(n, seed=inputs.seed_for(1, 300 + n))
    X, info = oracle.trtri(L, c=c)
    assert info == 0
    # L X = I exactly (integer matmul on exactly representable dyadics)
    prod = np.tril(L) @ np.tril(X)
    assert np.array_equal(prod, np.eye(n))
    # trtri(trtri(L)) = L
    Y, info = oracle.trtri(X, c=c)
    assert np.array_equal(np.tril(Y), np.tril(L))
    assert np.array_equal(np.triu(X, 1), np.triu(L, 1))   # upper part untouched


@pytest.mark.parametrize("n,c", [(3, 1), (70, 24), (129, 16)])
def test_integer_lauum_exact(oracle, n, c):
    L = inputs.integer_chol(n, seed=inputs.seed_for(1, 500 + n))
    P = oracle.lauum(L, c=c)
    Li = np.tril(L).astype(np.int64)
    want = (Li.T @ Li).astype(np.float64)
    assert np.array_equal(np.tril(P), np.tril(want))
    assert np.array_equal(np.triu(P, 1), np.triu(L, 1))


# ----------------------------------------------------------------------------
# exact rational brute force on tiny inputs
# ----------------------------------------------------------------------------

def _gepp_fractions(A):
    """Gaussian elimination with partial pivoting in exact rationals
    (independent of the oracle): returns LU (Fractions), ipiv (1-based), the
    relative gap between the top two candidates of each column."""
    n = len(A)
    M = [[Fraction(x) for x in row] for row in A]
    ipiv, gaps = [], []
    for j in range(n):
        cand = sorted(((abs(M[i][j]), i) for i in range(j, n)), key=lambda t: (-t[0], t[1]))
        p = cand[0][1]
        if len(cand) > 1 and cand[0][0] > 0:
            gaps.append(float((cand[0][0] - cand[1][0]) / cand[0][0]))
        else:
            gaps.append(1.0)
        ipiv.append(p + 1)
        M[j], M[p] = M[p], M[j]
        if M[j][j] != 0:
            for i in range(j + 1, n):
                M[i][j] = M[i][j] / M[j][j]
                for k in range(j + 1, n):
                    M[i][k] -= M[i][j] * M[j][k]
    return M, ipiv, gaps


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_lu_brute_force_rational(oracle, n):
    for k in range(5):
        A = inputs.uniform(n, n, seed=inputs.seed_for(1, 700 + 10 * n + k))
        M, ipiv, gaps = _gepp_fractions(A.tolist())
        F, piv, info = oracle.getrf(A, c=1 + k % 3)
        assert info == 0
        assert all(g > 1e-12 for g in gaps)
        assert list(piv) == ipiv
        exact = np.array([[float(x) for x in row] for row in M])
        assert np.max(np.abs(F - exact)) <= 64 * n * EPS * max(1.0, np.max(np.abs(exact)))


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_cholesky_brute_force_rational(oracle, n):
    import decimal
    decimal.getcontext().prec = 50
    for k in range(4):
        A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 800 + 10 * n + k))
        # exact LDL^T in rationals, then L sqrt(D) to 50 digits
        M = [[Fraction(x) for x in row] for row in A.tolist()]
        Lr = [[Fraction(0)] * n for _ in range(n)]
        D = [Fraction(0)] * n
        for j in range(n):
            D[j] = M[j][j] - sum(Lr[j][t] ** 2 * D[t] for t in range(j))
            Lr[j][j] = Fraction(1)
            for i in range(j + 1, n):
                Lr[i][j] = (M[i][j] - sum(Lr[i][t] * Lr[j][t] * D[t] for t in range(j))) / D[j]
        sq = [decimal.Decimal(d.numerator) / decimal.Decimal(d.denominator) for d in D]
        sq = [s.sqrt() for s in sq]
        exact = np.zeros((n, n))
        for j in range(n):
            for i in range(j, n):
                v = decimal.Decimal(Lr[i][j].numerator) / decimal.Decimal(Lr[i][j].denominator)
                exact[i, j] = float(v * sq[j])
        F, info = oracle.potrf(A, c=1 + k % 3)
        assert info == 0
        assert np.max(np.abs(np.tril(F) - exact)) <= 16 * n * EPS * np.max(np.abs(exact))


def test_trtri_lauum_brute_force_rational(oracle):
    for n in (1, 3, 6):
        L = np.tril(inputs.uniform(n, n, seed=inputs.seed_for(1, 900 + n)))
        L[np.diag_indices(n)] += 2.0
        Lf = [[Fraction(x) for x in row] for row in L.tolist()]
        # exact inverse by forward substitution on L x = e_j
        X = [[Fraction(0)] * n for _ in range(n)]
        for j in range(n):
            for i in range(j, n):
                rhs = Fraction(1 if i == j else 0) - sum(Lf[i][k] * X[k][j] for k in range(j, i))
                X[i][j] = rhs / Lf[i][i]
        Xe = np.array([[float(x) for x in r] for r in X])
        Xo, info = oracle.trtri(np.asfortranarray(L), c=2)
        assert np.max(np.abs(np.tril(Xo) - Xe)) <= 32 * n * EPS * np.max(np.abs(Xe))
        P = [[sum(Lf[k][i] * Lf[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
        Pe = np.array([[float(x) for x in r] for r in P])
        Po = oracle.lauum(np.asfortranarray(L), c=2)
        assert np.max(np.abs(np.tril(Po) - np.tril(Pe))) <= 8 * n * EPS * np.max(np.abs(Pe))


# ----------------------------------------------------------------------------
# LAPACK (scipy) cross-checks: special cases that reduce to a library routine
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 17, 100, 257])
def test_potrf_vs_lapack(oracle, n):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, n))
    for c in (1, 2, 24, n):
        F, info = oracle.potrf(A, c=c)
        assert info == 0 and oracle.res_chol(A, F) <= BOUND
        Ls, infos = lapack.dpotrf(A, lower=1)
        kappa = np.linalg.cond(A)
        assert np.max(np.abs(np.tril(F) - np.tril(Ls))) <= 2 * BOUND * n * EPS * kappa * np.max(np.abs(Ls))


@pytest.mark.parametrize("n", [1, 2, 17, 100, 257])
def test_getrf_vs_lapack(oracle, n):
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, n))
    Fs, piv, infos = lapack.dgetrf(A)
    for c in (1, 2, 24, n):
        F, ipiv, info = oracle.getrf(A, c=c)
        assert info == 0 and oracle.res_lu(A, F, ipiv) <= BOUND
        assert np.array_equal(ipiv, piv + 1)
        kappa = np.linalg.cond(A)
        assert np.max(np.abs(F - Fs)) <= 2 * BOUND * n * EPS * kappa * max(1.0, np.max(np.abs(Fs)))


@pytest.mark.parametrize("n", [1, 2, 33, 128, 200])
def test_trtri_lauum_potri_vs_lapack(oracle, n):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 100 + n))
    L, info = oracle.potrf(A, c=24)
    L = np.asfortranarray(np.tril(L))
    for c in (1, 2, 24, n):
        X, info = oracle.trtri(L, c=c)
        assert info == 0 and oracle.res_trtri(L, X) <= BOUND
        Xs, infos = lapack.dtrtri(L, lower=1)
        kl = np.linalg.cond(L)
        assert np.max(np.abs(np.tril(X) - np.tril(Xs))) <= 2 * BOUND * n * EPS * kl * np.max(np.abs(Xs))
        P = oracle.lauum(L, c=c)
        Ps, infos = lapack.dlauum(L, lower=1)
        assert np.max(np.abs(np.tril(P) - np.tril(Ps))) <= 4 * n * EPS * np.max(np.abs(Ps))
        Ai, info = oracle.potri(L, c=c)
        assert info == 0 and oracle.res_potri(A, Ai) <= BOUND


# ----------------------------------------------------------------------------
# info semantics (LAPACK's meanings)
# ----------------------------------------------------------------------------

def test_potrf_info_not_spd(oracle):
    n = 60
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 42))
    for k in (0, 7, 31, 59):
        B = A.copy(order="F")
        B[k, k] = -1.0
        for c in (1, 8, 24, n):
            F, info = oracle.potrf(B, c=c)
            _, infos = lapack.dpotrf(B, lower=1)
            assert info == infos > 0
            assert np.allclose(np.tril(F[: info - 1, : info - 1]),
                               np.linalg.cholesky(B[: info - 1, : info - 1]), rtol=1e-12, atol=1e-12)


def test_getrf_info_singular(oracle):
    n = 50
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 43))
    for k in (0, 13, 49):
        B = A.copy(order="F")
        B[:, k] = 0.0
        for c in (1, 8, n):
            F, ipiv, info = oracle.getrf(B, c=c)
            Fs, piv, infos = lapack.dgetrf(B)
            assert info == infos == k + 1
            assert np.array_equal(ipiv, piv + 1)
            assert oracle.res_lu(B, F, ipiv) <= BOUND


def test_trtri_info_zero_diagonal(oracle):
    n = 40
    L = np.tril(inputs.uniform(n, n, seed=inputs.seed_for(1, 44))) + 3 * np.eye(n)
    L = np.asfortranarray(L)
    L[17, 17] = 0.0
    L[30, 30] = 0.0
    X, info = oracle.trtri(L, c=8)
    assert info == 18 and np.array_equal(X, L)


# ----------------------------------------------------------------------------
# random residual bounds and crossover invariance (bound <= 10)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [3, 64, 129, 300, 512])
def test_residual_bounds_all_crossovers(oracle, n):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 1000 + n))
    G = inputs.uniform(n, n, seed=inputs.seed_for(1, 1000 + n))
    for c in (1, 2, 24, n):
        L, info = oracle.potrf(A, c=c)
        assert info == 0 and oracle.res_chol(A, L) <= BOUND
        F, ipiv, info = oracle.getrf(G, c=c)
        assert info == 0 and oracle.res_lu(G, F, ipiv) <= BOUND
    x = inputs.normal(n, 1, seed=7).ravel()
    assert oracle.probe_chol(A, L, x) <= BOUND
    assert oracle.probe_lu(G, F, ipiv, x) <= BOUND


def test_blas3_definitions_vs_library(oracle):
    import scipy.linalg as sl
    A = inputs.uniform(37, 23, seed=1)
    B = inputs.uniform(23, 41, seed=2)
    C = inputs.uniform(37, 41, seed=3)
    got = oracle.gemm(A, B, C, alpha=-2.0)
    assert np.max(np.abs(got - (C - 2.0 * A @ B))) <= 64 * EPS * 23
    got = oracle.gemm(A.T.copy(), B.T.copy(), C, alpha=1.0, ta=True, tb=True)
    assert np.max(np.abs(got - (C + A @ B))) <= 64 * EPS * 23
    S = inputs.uniform(30, 30, seed=4)
    got = oracle.syrk_lower(A[:30], S, alpha=-1.0)
    assert np.max(np.abs(np.tril(got - (S - A[:30] @ A[:30].T)))) <= 64 * EPS * 23
    assert np.array_equal(np.triu(got, 1), np.triu(S, 1))
    L = np.tril(inputs.uniform(23, 23, seed=5)) + 3 * np.eye(23)
    U = np.triu(inputs.uniform(23, 23, seed=6)) + 3 * np.eye(23)
    X = inputs.uniform(23, 9, seed=7)
    Y = inputs.uniform(9, 23, seed=8)
    tol = 1e-13
    assert np.allclose(oracle.trsm_lln(L, X, alpha=0.5), sl.solve_triangular(L, 0.5 * X, lower=True), atol=tol)
    Lu = np.tril(L, -1) + np.eye(23)
    assert np.allclose(oracle.trsm_lln(L, X, unit=True), sl.solve_triangular(Lu, X, lower=True), atol=tol)
    assert np.allclose(oracle.trsm_llt(L, X), sl.solve_triangular(L.T, X, lower=False), atol=tol)
    assert np.allclose(oracle.trsm_lun(U, X), sl.solve_triangular(U, X, lower=False), atol=tol)
    assert np.allclose(oracle.trsm_rlt(L, Y), sl.solve_triangular(L, Y.T, lower=True).T, atol=tol)
    assert np.allclose(oracle.trmm_rln(L, Y), Y @ L, atol=tol)
    assert np.allclose(oracle.trmm_llt(L, X), L.T @ X, atol=tol)


def test_laswp_definition(oracle):
    A = inputs.uniform(9, 4, seed=1)
    ipiv = np.array([3, 2, 9, 4], dtype=np.int32)
    B = oracle.laswp(A, 0, 4, ipiv)
    want = A.copy()
    for i, p in enumerate(ipiv):
        want[[i, p - 1]] = want[[p - 1, i]]
    assert np.array_equal(B, want)


def test_solves_backward_error(oracle):
    n = 120
    A = inputs.uniform(n, n, seed=inputs.seed_for(2, 1))
    B = inputs.normal(n, 3, seed=inputs.seed_for(2, 2))
    F, ipiv, info = oracle.getrf(A, c=24)
    X = oracle.getrs(F, ipiv, B)
    assert oracle.backward_error(A, X, B) <= 10 * n * EPS
    S = inputs.spd_bbt(n, seed=inputs.seed_for(2, 3))
    L, info = oracle.potrf(S, c=24)
    X = oracle.potrs(L, B)
    assert oracle.backward_error(S, X, B) <= 10 * n * EPS


# ----------------------------------------------------------------------------
# planted mistakes: each pin fails on a plausible error in the oracle's output
# ----------------------------------------------------------------------------

def test_planted_mistakes_are_caught(oracle):
    n = 96
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 5))
    L, info = oracle.potrf(A, c=24)
    L = np.asfortranarray(np.tril(L))
    # dropped SYRK update: factor A22 without subtracting A21 A21^T
    n1 = oracle.split(n)
    bad = L.copy(order="F")
    bad[n1:, n1:] = np.linalg.cholesky(A[n1:, n1:])
    assert oracle.res_chol(A, bad) > 1e6
    # wrong sign in one entry
    bad = L.copy(order="F")
    bad[50, 3] = -bad[50, 3]
    assert oracle.res_chol(A, bad) > 1e3
    # transposed off-diagonal block (A21 <-> A12^T shape mix-up)
    bad = L.copy(order="F")
    bad[n1:n1 + 8, :8] = bad[n1:n1 + 8, :8].T
    assert oracle.res_chol(A, bad) > 1e3
    # swapped pivot in LU
    G = inputs.uniform(n, n, seed=inputs.seed_for(1, 5))
    F, ipiv, info = oracle.getrf(G, c=24)
    p2 = ipiv.copy()
    p2[10] = p2[10] + 1 if p2[10] < n else p2[10] - 1
    assert oracle.res_lu(G, F, p2) > 1e3
    # TRTRI with the TRSM sign dropped
    X, info = oracle.trtri(L, c=24)
    bad = np.asfortranarray(np.tril(X))
    bad[n1:, :n1] = -bad[n1:, :n1]
    assert oracle.res_trtri(L, bad) > 1e3
    # probe residuals flag the same mistake
    x = inputs.normal(n, 1, seed=3).ravel()
    badL = L.copy(order="F")
    badL[50, 3] = -badL[50, 3]
    assert oracle.probe_chol(A, badL, x) > 1e3


# ----------------------------------------------------------------------------
# sygst (Section 5, xsygst): A := L^{-1} A L^{-T} (itype 1), L^T A L (2, 3)
# ----------------------------------------------------------------------------

def test_sygst_closed_form_2x2(oracle):
    a, b, d, p, q, r = 8.0, 5.0, 16.0, 2.0, 1.0, 4.0
    A = np.array([[a, 99.0], [b, d]], order="F")          # the upper entry is not referenced
    L = np.array([[p, 0.0], [q, r]], order="F")
    X = oracle.sygst(1, A, L)
    assert X[0, 0] == a / p ** 2 == 2.0
    assert X[1, 0] == (p * b - q * a) / (p * p * r) == 0.125
    assert X[1, 1] == (d - 2 * q * b / p + q * q * a / p ** 2) / r ** 2 == 0.8125
    assert X[0, 1] == 99.0
    for itype in (2, 3):
        X = oracle.sygst(itype, A, L)
        assert X[0, 0] == p * p * a + 2 * p * q * b + q * q * d == 68.0
        assert X[1, 0] == r * (p * b + q * d) == 104.0
        assert X[1, 1] == r * r * d == 256.0
        assert X[0, 1] == 99.0


def _int_sym(n, seed, lim=3):
    r = np.random.default_rng(seed)
    M = r.integers(-lim, lim + 1, size=(n, n)).astype(np.float64)
    return np.asfortranarray(np.tril(M) + np.tril(M, -1).T)


@pytest.mark.parametrize("n", [1, 3, 40, 130])
def test_sygst_integer_exact(oracle, n):
    L = inputs.integer_chol(n, seed=inputs.seed_for(0, 700 + n), offdiag=1, diag=(1, 1))
    M = _int_sym(n, seed=inputs.seed_for(0, 710 + n))
    Li, Mi = L.astype(np.int64), M.astype(np.int64)
    A = np.asfortranarray((Li @ Mi @ Li.T).astype(np.float64))
    # L^{-1} (L M L^T) L^{-T} = M exactly: every intermediate is an integer < 2^53
    X = oracle.sygst(1, A, L)
    assert np.array_equal(np.tril(X), np.tril(M))
    X = oracle.sygst(2, M, L)
    assert np.array_equal(np.tril(X), np.tril((Li.T @ Mi @ Li).astype(np.float64)))


@pytest.mark.parametrize("itype", [1, 2, 3])
@pytest.mark.parametrize("n", [1, 17, 100])
def test_sygst_vs_lapack(oracle, itype, n):
    Bm = inputs.spd_bbt(n, seed=inputs.seed_for(0, 720 + n))
    L = np.asfortranarray(np.linalg.cholesky(Bm))
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 730 + n))
    ref, info = lapack.dsygst(A, L, itype=itype, lower=1)
    assert info == 0
    X = oracle.sygst(itype, A, L)
    scale = np.max(np.abs(np.tril(ref)))
    assert np.max(np.abs(np.tril(X) - np.tril(ref))) <= 64 * n * 2.0 ** -53 * scale


@pytest.mark.parametrize("n", [1, 2, 4, 5])
def test_sygst_brute_force_rational(oracle, n):
    Bm = inputs.spd_bbt(n, seed=inputs.seed_for(0, 740 + n))
    L = np.asfortranarray(np.linalg.cholesky(Bm))
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 750 + n))
    Lf = [[Fraction(x) for x in row] for row in L.tolist()]
    Af = [[Fraction(x) for x in row] for row in A.tolist()]
    # exact L^{-1} by forward substitution on the identity
    Inv = [[Fraction(0)] * n for _ in range(n)]
    for j in range(n):
        for i in range(n):
            s = Fraction(1 if i == j else 0) - sum(Lf[i][k] * Inv[k][j] for k in range(i))
            Inv[i][j] = s / Lf[i][i]
    for itype in (1, 2):
        if itype == 1:
            P = [[sum(Inv[i][k] * Af[k][l] for k in range(n)) for l in range(n)] for i in range(n)]
            E = [[sum(P[i][l] * Inv[j][l] for l in range(n)) for j in range(n)] for i in range(n)]
        else:
            P = [[sum(Lf[k][i] * Af[k][l] for k in range(n)) for l in range(n)] for i in range(n)]
            E = [[sum(P[i][l] * Lf[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
        X = oracle.sygst(itype, A, L)
        ex = np.array([[float(E[i][j]) for j in range(n)] for i in range(n)])
        scale = max(1.0, np.max(np.abs(ex)))
        assert np.max(np.abs(np.tril(X) - np.tril(ex))) <= 32 * n * 2.0 ** -53 * scale


def test_sygst_planted_mistakes_are_caught(oracle):
    n = 60
    Bm = inputs.spd_bbt(n, seed=inputs.seed_for(0, 760))
    L = np.asfortranarray(np.linalg.cholesky(Bm))
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 770))
    ref, _ = lapack.dsygst(A, L, itype=1, lower=1)
    tol = 64 * n * 2.0 ** -53 * np.max(np.abs(ref))
    Li = np.linalg.inv(L)
    wrong_side = Li.T @ A @ Li                        # inverse applied on the wrong sides
    assert np.max(np.abs(np.tril(wrong_side) - np.tril(ref))) > 1e6 * tol
    X = oracle.sygst(1, A, L)
    bad = X.copy(order="F")
    bad[40, 7] *= -1                                  # one sign flipped
    assert np.max(np.abs(np.tril(bad) - np.tril(ref))) > 1e3 * tol
    assert np.max(np.abs(np.tril(X) - np.tril(ref))) <= tol


# ----------------------------------------------------------------------------
# getri (xtrtri as building block of xgetri, Section 5): A^{-1} from P L U
# ----------------------------------------------------------------------------

def test_getri_closed_form_2x2(oracle):
    A = np.array([[1.0, 2.0], [3.0, 4.0]], order="F")
    F, ipiv, info = oracle.getrf(A, c=1)
    X = oracle.getri(F, ipiv)
    det = 1.0 * 4.0 - 2.0 * 3.0
    ex = np.array([[4.0, -2.0], [-3.0, 1.0]]) / det
    assert np.max(np.abs(X - ex)) <= 4 * 2.0 ** -53 * 2.0


def _unimodular_factors(n, seed):
    """Integer unit-lower L, integer upper U with diagonal +-1 and a pivot
    sequence: A = P^T L U has det +-1 and an integer inverse."""
    r = np.random.default_rng(seed)
    L = np.tril(r.integers(-1, 2, size=(n, n)).astype(np.float64), -1) + np.eye(n)
    U = np.triu(r.integers(-1, 2, size=(n, n)).astype(np.float64), 1)
    U[np.diag_indices(n)] = r.choice([-1.0, 1.0], size=n)
    ipiv = np.array([r.integers(j + 1, n + 1) for j in range(n)], dtype=np.int32)
    F = np.asfortranarray(np.tril(L, -1) + U)
    P = np.eye(n)
    for j in range(n):
        p = ipiv[j] - 1
        P[[j, p]] = P[[p, j]]
    A = P.T @ L @ U
    return F, ipiv, A


@pytest.mark.parametrize("n", [1, 4, 30])
def test_getri_integer_exact(oracle, n):
    F, ipiv, A = _unimodular_factors(n, inputs.seed_for(0, 900 + n))
    X = oracle.getri(F, ipiv)
    assert np.array_equal(X, np.round(X))                       # integer inverse, exactly
    assert np.array_equal(A @ X, np.eye(n))


@pytest.mark.parametrize("n", [1, 2, 17, 100])
def test_getri_vs_lapack(oracle, n):
    A = inputs.uniform(n, n, seed=inputs.seed_for(0, 910 + n))
    F, ipiv, info = oracle.getrf(A, c=24)
    lu, piv, _ = lapack.dgetrf(A)
    assert np.array_equal(piv + 1, ipiv)
    ref, info = lapack.dgetri(lu, piv)
    assert info == 0
    X = oracle.getri(F, ipiv)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(X - ref)) <= 64 * n * 2.0 ** -53 * kappa * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [1, 3, 5])
def test_getri_brute_force_rational(oracle, n):
    A = inputs.uniform(n, n, seed=inputs.seed_for(0, 920 + n))
    M = [[Fraction(x) for x in row] for row in A.tolist()]
    # exact inverse by Gauss-Jordan on [A | I] in rationals
    aug = [M[i] + [Fraction(1 if i == j else 0) for j in range(n)] for i in range(n)]
    for j in range(n):
        p = next(i for i in range(j, n) if aug[i][j] != 0)
        aug[j], aug[p] = aug[p], aug[j]
        piv = aug[j][j]
        aug[j] = [v / piv for v in aug[j]]
        for i in range(n):
            if i != j and aug[i][j] != 0:
                f = aug[i][j]
                aug[i] = [a - f * b for a, b in zip(aug[i], aug[j])]
    ex = np.array([[float(aug[i][n + j]) for j in range(n)] for i in range(n)])
    F, ipiv, info = oracle.getrf(A, c=1)
    X = oracle.getri(F, ipiv)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(X - ex)) <= 16 * n * 2.0 ** -53 * kappa * np.max(np.abs(ex))


# ----------------------------------------------------------------------------
# complex double (zpotrf / zgetrf): A = L L^H, P A = L U with |Re| + |Im| pivots
# ----------------------------------------------------------------------------

def test_complex_closed_forms_2x2(oracle):
    A = np.array([[4.0, 2 - 2j], [2 + 2j, 6.0]], dtype=complex, order="F")
    L, info = oracle.zpotrf(A, c=1)
    assert info == 0
    assert L[0, 0] == 2.0 and L[1, 0] == (2 + 2j) / 2.0 and L[1, 1] == np.sqrt(6.0 - 8.0 / 4.0)
    G = np.array([[1.0, 2j], [3.0, 4.0]], dtype=complex, order="F")
    F, ipiv, info = oracle.zgetrf(G, c=1)
    assert info == 0 and list(ipiv) == [2, 2]
    assert F[0, 0] == 3.0 and F[0, 1] == 4.0 and F[1, 0] == 1.0 / 3.0
    assert abs(F[1, 1] - (2j - 4.0 / 3.0)) <= 4 * 2.0 ** -53 * 2.0


@pytest.mark.parametrize("n,c", [(5, 1), (60, 8), (130, 24)])
def test_zpotrf_gaussian_integers_exact(oracle, n, c):
    L = inputs.gaussian_int_chol(n, inputs.seed_for(0, 1100 + n))
    A = np.asfortranarray(L @ L.conj().T)
    X, info = oracle.zpotrf(A, c=c)
    assert info == 0
    assert np.array_equal(np.tril(X), L)


@pytest.mark.parametrize("n,c", [(6, 1), (70, 8), (150, 24)])
def test_zgetrf_dyadic_exact(oracle, n, c):
    A, L, U, perm = inputs.complex_dyadic_lu(n, inputs.seed_for(0, 1200 + n))
    F, ipiv, info = oracle.zgetrf(A, c=c)
    assert info == 0
    assert np.array_equal(ipiv, inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1) + np.eye(n), L) and np.array_equal(np.triu(F), U)


@pytest.mark.parametrize("n", [1, 2, 17, 100, 257])
def test_zpotrf_zgetrf_vs_lapack(oracle, n):
    A = inputs.herm_spd(n, inputs.seed_for(0, 1300 + n))
    L, info = oracle.zpotrf(A, c=24)
    ref, info_l = lapack.zpotrf(A, lower=1)
    assert info == info_l == 0
    assert np.max(np.abs(np.tril(L) - np.tril(ref))) <= 64 * n * 2.0 ** -53 * np.max(np.abs(ref))
    assert oracle.res_zchol(A, np.tril(L)) <= 10.0
    G = inputs.complex_uniform(n, n, inputs.seed_for(0, 1400 + n))
    F, ipiv, info = oracle.zgetrf(G, c=24)
    lu, piv, info_l = lapack.zgetrf(G)
    assert info == info_l == 0
    assert np.array_equal(ipiv, piv + 1)
    kappa = np.linalg.cond(G)
    assert np.max(np.abs(F - lu)) <= 64 * n * 2.0 ** -53 * kappa * np.max(np.abs(lu))
    assert oracle.res_zlu(G, F, ipiv) <= 10.0


@pytest.mark.parametrize("n", [1, 2, 4])
def test_zgetrf_brute_force_gaussian_rationals(oracle, n):
    """Partial pivoting on |Re| + |Im| in exact Gaussian-rational arithmetic."""
    r = np.random.default_rng(inputs.seed_for(0, 1500 + n))
    G = (r.integers(-8, 9, size=(n, n)) + 1j * r.integers(-8, 9, size=(n, n))) / 8.0
    M = [[(Fraction(z.real), Fraction(z.imag)) for z in row] for row in G.tolist()]

    def mul(a, b):
        return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])

    def div(a, b):
        d = b[0] * b[0] + b[1] * b[1]
        return ((a[0] * b[0] + a[1] * b[1]) / d, (a[1] * b[0] - a[0] * b[1]) / d)

    piv = []
    for j in range(n):
        p = max(range(j, n), key=lambda i: (abs(M[i][j][0]) + abs(M[i][j][1]), -i))
        piv.append(p + 1)
        M[j], M[p] = M[p], M[j]
        if M[j][j] != (0, 0):
            for i in range(j + 1, n):
                M[i][j] = div(M[i][j], M[j][j])
                for k in range(j + 1, n):
                    t = mul(M[i][j], M[j][k])
                    M[i][k] = (M[i][k][0] - t[0], M[i][k][1] - t[1])
    ex = np.array([[float(a) + 1j * float(b) for (a, b) in row] for row in M])
    F, ipiv, info = oracle.zgetrf(np.asfortranarray(G), c=1)
    assert list(ipiv) == piv
    assert np.max(np.abs(F - ex)) <= 16 * n * 2.0 ** -53 * max(1.0, np.max(np.abs(ex))) * np.linalg.cond(G)


def test_complex_planted_mistakes_are_caught(oracle):
    n = 80
    A = inputs.herm_spd(n, inputs.seed_for(0, 1600))
    L, _ = oracle.zpotrf(A, c=24)
    L = np.tril(L)
    assert oracle.res_zchol(A, L) <= 10.0
    assert oracle.res_zchol(A, np.asfortranarray(L.conj())) > 1e6          # conjugate dropped
    bad = L.copy(order="F")
    bad[40, 5] = -bad[40, 5]
    assert oracle.res_zchol(A, bad) > 1e3
    G = inputs.complex_uniform(n, n, inputs.seed_for(0, 1601))
    F, ipiv, _ = oracle.zgetrf(G, c=24)
    assert oracle.res_zlu(G, F, ipiv) <= 10.0
    p2 = ipiv.copy()
    p2[10] = p2[10] + 1 if p2[10] < n else p2[10] - 1
    assert oracle.res_zlu(G, F, p2) > 1e3


# ----------------------------------------------------------------------------
# uplo = 'U': each upper form is the lower form of the transposed storage
# (A = U^T U with U = L^T).  The GPU path computes the upper forms that way;
# here the identity itself is pinned against LAPACK's own upper routines.
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 5, 100, 257])
def test_upper_forms_are_the_transposed_lower_forms(oracle, n):
    tol = 64 * n * 2.0 ** -53
    A = inputs.spd_bbt(n, seed=inputs.seed_for(0, 1700 + n))
    L, info = oracle.potrf(np.asfortranarray(A.T))
    U = np.triu(np.tril(L).T)
    ref, info_l = lapack.dpotrf(A, lower=0)
    assert info == info_l == 0
    assert np.max(np.abs(U - np.triu(ref))) <= tol * np.max(np.abs(ref))
    for unit in (False, True):
        X, _ = oracle.trtri(np.asfortranarray(np.tril(U.T)), unit=unit)
        ref, _ = lapack.dtrtri(U, lower=0, unitdiag=int(unit))
        k = 1 if unit else 0                       # a unit diagonal is not referenced
        ref = np.triu(ref, k)
        assert np.max(np.abs(np.triu(np.tril(X).T, k) - ref), initial=0.0) <= tol * 8 * max(1.0, np.max(np.abs(ref), initial=0.0))
    P = oracle.lauum(np.asfortranarray(np.tril(U.T)))
    ref, _ = lapack.dlauum(U, lower=0)
    assert np.max(np.abs(np.triu(np.tril(P).T) - np.triu(ref))) <= tol * np.max(np.abs(ref))
    Q, _ = oracle.potri(np.asfortranarray(np.tril(U.T)))
    ref, _ = lapack.dpotri(U, lower=0)
    assert np.max(np.abs(np.triu(np.tril(Q).T) - np.triu(ref))) <= tol * 8 * np.max(np.abs(ref))
    M = inputs.spd_bbt(n, seed=inputs.seed_for(0, 1710 + n))
    for itype in (1, 2):
        S = oracle.sygst(itype, np.asfortranarray(M.T), np.asfortranarray(np.tril(U.T)))
        ref, _ = lapack.dsygst(M, U, itype=itype, lower=0)
        assert np.max(np.abs(np.triu(np.tril(S).T) - np.triu(ref))) <= tol * 8 * np.max(np.abs(ref))
    H = inputs.herm_spd(n, inputs.seed_for(0, 1720 + n))
    Lz, info = oracle.zpotrf(np.asfortranarray(H.conj().T))
    ref, info_l = lapack.zpotrf(H, lower=0)
    assert info == info_l == 0
    assert np.max(np.abs(np.triu(np.tril(Lz).conj().T) - np.triu(ref))) <= tol * np.max(np.abs(ref))


# ----------------------------------------------------------------------------
# the emulated FP64 GEMM (oracle/ozaki.py): not in the paper; pinned by the
# exact product of integers, the scheme's error bound against exact rational
# products, the digit identity, and planted mistakes that the bound catches
# ----------------------------------------------------------------------------

from fractions import Fraction  # noqa: E402

from oracle import ozaki  # noqa: E402


def test_ozaki_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(11)
    for S in (6, 7, 8):
        for _ in range(2000):
            q = rng.uniform(-0.5, 0.5) * 2.0 ** int(rng.integers(-40, 1))
            Q = ozaki.fixed_point(q, 0, S)
            d = ozaki.digits(Q, S)
            assert sum(ds * 256 ** (S - 1 - i) for i, ds in enumerate(d)) == Q
            assert all(-128 <= x <= 127 for x in d[1:]) and -128 <= d[0] <= 128
        # near 1/2 the top digit reaches 128 (no carry out)
        Q = ozaki.fixed_point(0.5 - 2.0 ** -54, 0, S)
        assert ozaki.digits(Q, S)[0] == 128
    # ties round away from zero
    assert ozaki.fixed_point(2.0 ** -57 * 3, 0, 7) == 2 and ozaki.fixed_point(-(2.0 ** -57) * 3, 0, 7) == -2
    assert ozaki.exponent_of_max(1.0) == 2 and ozaki.exponent_of_max(0.75) == 1
    assert ozaki.exponent_of_max(5e-324) == -1072 and ozaki.exponent_of_max(0.0) == 0


@pytest.mark.parametrize("S", [6, 7, 8])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True), (False, True)])
def test_ozaki_integer_products_exact(S, ta, tb):
    rng = np.random.default_rng(12 + S)
    A = rng.integers(-1000, 1001, size=(40, 23)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(40, 17)).astype(np.float64)
    A = A if ta else np.asfortranarray(A.T)                   # op(A): 23 x 40
    B = np.asfortranarray(B.T) if tb else B                   # op(B): 40 x 17
    exact = (A.T if ta else A).astype(np.int64) @ (B.T if tb else B).astype(np.int64)
    assert np.array_equal(ozaki.gemm(A, B, S, ta, tb), exact.astype(np.float64))


def _exact_product(A, B):
    m, k = A.shape
    n = B.shape[1]
    Af = [[Fraction(float(v)) for v in row] for row in A]
    Bf = [[Fraction(float(B[kk, j])) for kk in range(k)] for j in range(n)]
    return [[sum(a * b for a, b in zip(Af[i], Bf[j])) for j in range(n)] for i in range(m)]


def _bound_ok(C, A, B, S, exact, levels_dropped=0):
    m, k = A.shape
    ok = True
    for i in range(m):
        ea = ozaki.exponent_of_max(float(np.max(np.abs(A[i]))))
        for j in range(B.shape[1]):
            eb = ozaki.exponent_of_max(float(np.max(np.abs(B[:, j]))))
            bound = Fraction(k * (S + 1)) * Fraction(2) ** (-8 * S - 2 + ea + eb)
            bound += abs(exact[i][j]) * Fraction(2) ** -53
            ok &= abs(Fraction(float(C[i, j])) - exact[i][j]) <= bound
    return ok


@pytest.mark.parametrize("S", [6, 7, 8])
def test_ozaki_error_bound_against_exact_rationals(S):
    rng = np.random.default_rng(13 + S)
    A = rng.standard_normal((6, 40)) * np.exp2(rng.integers(-20, 20, size=(6, 1)))
    B = rng.standard_normal((40, 5)) * np.exp2(rng.integers(-20, 20, size=(1, 5)))
    A[2, :] = 0.0
    exact = _exact_product(A, B)
    C = ozaki.gemm(A, B, S)
    assert _bound_ok(C, A, B, S, exact)
    assert np.all(C[2, :] == 0.0)


def test_ozaki_planted_mistakes_break_the_bound():
    """A dropped top level, or digit planes taken in reverse order, leave the
    derived bound by orders of magnitude."""
    S = 7
    rng = np.random.default_rng(14)
    A = rng.standard_normal((5, 30))
    B = rng.standard_normal((30, 4))
    exact = _exact_product(A, B)
    eA, DA = ozaki.slice_rows(A, S)
    eB, DB = ozaki.slice_rows(B.T, S)

    def combine(T):
        C = np.zeros((5, 4))
        for i in range(5):
            for j in range(4):
                V = sum(int(T[L][i, j]) << (8 * (S + 1 - L)) for L in T)
                C[i, j] = np.ldexp(float(V), eA[i] + eB[j] - 8 * (S + 1))
        return C

    T = ozaki.level_sums(DA, DB, S)
    assert _bound_ok(combine(T), A, B, S, exact)
    T_drop = dict(T)
    del T_drop[S + 1]
    assert not _bound_ok(combine(T_drop), A, B, S, exact)
    T_rev = ozaki.level_sums(DA[::-1], DB, S)
    assert not _bound_ok(combine(T_rev), A, B, S, exact)


# ----------------------------------------------------------------------------
# complex inversions (oracle ztrtri / zlauum / zpotri / zgetri)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 6, 40, 100])
def test_complex_inversions_exact_on_gaussian_integers(oracle, n):
    L, Linv = inputs.gaussian_unit_trtri(n, inputs.seed_for(0, 1800 + n))
    X, info = oracle.ztrtri(L)
    assert info == 0 and np.array_equal(np.tril(X), Linv)
    Lu = np.asfortranarray(np.tril(np.diag(1.0 / np.diag(L)) @ L))
    X, _ = oracle.ztrtri(Lu, unit=True)
    assert np.array_equal(np.tril(X, -1), np.tril(Linv @ np.diag(np.diag(L)), -1))
    P = oracle.zlauum(L)
    assert np.array_equal(np.tril(P), np.tril(L.conj().T @ L))
    Q, info = oracle.zpotri(L)
    assert info == 0 and np.array_equal(np.tril(Q), np.tril(Linv.conj().T @ Linv))


@pytest.mark.parametrize("n", [1, 17, 120])
def test_complex_inversions_vs_lapack(oracle, n):
    tol = 64 * n * 2.0 ** -53
    H = inputs.herm_spd(n, inputs.seed_for(0, 1900 + n))
    L = np.asfortranarray(np.tril(oracle.zpotrf(H)[0]))
    X, info = oracle.ztrtri(L)
    ref, info_l = lapack.ztrtri(L, lower=1)
    assert info == info_l == 0
    assert np.max(np.abs(np.tril(X) - np.tril(ref))) <= tol * 8 * np.max(np.abs(ref))
    P = oracle.zlauum(L)
    ref, _ = lapack.zlauum(L, lower=1)
    assert np.max(np.abs(np.tril(P) - np.tril(ref))) <= tol * np.max(np.abs(ref))
    Q, info = oracle.zpotri(L)
    ref, _ = lapack.zpotri(L, lower=1)
    assert np.max(np.abs(np.tril(Q) - np.tril(ref))) <= tol * 8 * np.max(np.abs(ref))
    G = inputs.complex_uniform(n, n, inputs.seed_for(0, 1950 + n))
    F, ipiv, info = oracle.zgetrf(G)
    Xg = oracle.zgetri(F, ipiv)
    ref, info_l = lapack.zgetri(*lapack.zgetrf(G)[:2])
    kappa = np.linalg.cond(G)
    assert np.max(np.abs(Xg - ref)) <= tol * 8 * kappa * np.max(np.abs(ref))
    assert np.max(np.abs(G @ Xg - np.eye(n))) <= tol * 8 * kappa


def test_complex_inversion_planted_mistakes(oracle):
    """Dropping the conjugate in L^H L, or the interchanges in getri, is seen."""
    n = 30
    L, Linv = inputs.gaussian_unit_trtri(n, inputs.seed_for(0, 1990))
    P = oracle.zlauum(L)
    assert not np.array_equal(np.tril(P), np.tril(L.T @ L))
    G = inputs.complex_uniform(n, n, inputs.seed_for(0, 1991))
    F, ipiv, _ = oracle.zgetrf(G)
    assert np.max(np.abs(G @ oracle.zgetri(F, ipiv) - np.eye(n))) < 1e-10
    assert np.max(np.abs(G @ oracle.zgetri(F, np.arange(1, n + 1)) - np.eye(n))) > 1e-3
