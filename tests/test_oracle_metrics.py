"""Pins for the oracle's accuracy metrics (no GPU).

The GPU parity tests at large orders and every precision-form verdict rest on
five metric functions of the oracle: the normwise backward error of a solve,
the random-probe residuals of LU, of the triangular inverse and of the SPD
inverse, and the full POTRI residual.  Each is tied here to values fixed by
the mathematics, not by the oracle:

* closed forms: small dyadic cases whose factors or inverses are exact in
  binary64, with one entry moved by delta = 2^-30; the residual vector is then
  delta times a known column, so the metric's value follows by hand (the
  derivation is written beside each case).  The norms in each denominator
  are chosen so that the plausible slips (a 1-norm for an inf-norm, a
  dropped ||x|| or ||b||, the first column instead of the worst, a
  permutation left out, an upper triangle read) change the value;
* exact rational evaluation of the definitions on tiny random inputs (Python
  ``fractions``, n <= 6), where nothing rounds but the one intermediate the
  probes store: y = U x (or X x), rounded once to binary64 before the second
  product.  That rounding adds at most ||L|| ||U|| / (2 n ||A||) to the probe
  in its own units, far below the pass bound;
* planted mistakes: a wrong answer (a sign flipped in x, a probe without the
  row interchanges, an inverse with one block transposed, a residual taken
  against L instead of A) must move the metric far past the pass bound of 10.

Metrics follow the normwise definitions used for LAPACK's test ratios: for a
solve eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), for a
factorization or an inverse the residual over n eps times the norms of the
operands, eps = 2^-53.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_1602_06763_gb300 import inputs

EPS = 2.0 ** -53
DELTA = 2.0 ** -30
BOUND = 10.0


def _F(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _perm_from_ipiv(ipiv):
    """Rows of P A: perm[i] = original row at position i after the swaps
    ipiv (1-based, applied in order)."""
    n = len(ipiv)
    perm = list(range(n))
    for i, p in enumerate(ipiv):
        p -= 1
        perm[i], perm[p] = perm[p], perm[i]
    return perm


# ----------------------------------------------------------------------------
# backward error of a solve
# ----------------------------------------------------------------------------

def test_backward_error_closed_form(oracle):
    # A = [[1,2],[3,4]]: ||A||_inf = 7 (||A||_1 = 6).
    # column 0: x = (1, 1), A x = (3, 7), b = (3, 7.25): r = (0, 1/4),
    #   eta_0 = (1/4) / (7*1 + 7.25) = 1/57.
    # column 1: x = (1, -3) (||x||_inf = 3, ||x||_1 = 4), A x = (-5, -9),
    #   b = (-4, -8.5): r = (1, 1/2) (||r||_inf = 1, ||r||_1 = 3/2),
    #   eta_1 = 1 / (7*3 + 8.5) = 2/59  -> the maximum.
    A = _F([[1, 2], [3, 4]])
    X = _F([[1, 1], [1, -3]])
    B = _F([[3, -4], [7.25, -8.5]])
    got = oracle.backward_error(A, X, B)
    assert got == pytest.approx(2.0 / 59.0, rel=1e-15)
    # the slips this value rules out
    for wrong in (1 / 57, 1 / 9,           # first column only; ||x|| dropped (col 1: 1/9)
                  1 / 37, 1 / 27, 1 / 21,  # ||x||_1; ||A||_1; ||b|| dropped
                  1.5 / 29.5):             # ||r||_1
        assert abs(got - wrong) > 1e-3
    # one right-hand side given as a vector
    assert oracle.backward_error(A, X[:, 0], B[:, 0]) == pytest.approx(1.0 / 57.0, rel=1e-15)
    # an exact solution has eta = 0, also a zero right-hand side with x = 0
    # (no perturbation is needed; the quotient would be 0/0)
    assert oracle.backward_error(A, X, A @ X) == 0.0
    Z = X.copy(order="F")
    Z[:, 0] = 0.0
    assert oracle.backward_error(A, Z, A @ Z) == 0.0
    Bz = B.copy(order="F")
    Bz[:, 0] = 0.0
    assert oracle.backward_error(A, Z, Bz) == pytest.approx(2.0 / 59.0, rel=1e-15)


def test_backward_error_exact_rational(oracle):
    r = np.random.default_rng(11)
    for n, nrhs in ((1, 1), (3, 2), (5, 3), (6, 1)):
        A = _F(r.uniform(-1, 1, (n, n)))
        X = _F(r.normal(size=(n, nrhs)))
        B = _F(A @ X + r.normal(size=(n, nrhs)) * 1e-6)
        worst = Fr(0)
        an = max(sum(abs(Fr(A[i, k])) for k in range(n)) for i in range(n))
        for j in range(nrhs):
            rn = max(abs(Fr(B[i, j]) - sum(Fr(A[i, k]) * Fr(X[k, j]) for k in range(n)))
                     for i in range(n))
            xn = max(abs(Fr(X[i, j])) for i in range(n))
            bn = max(abs(Fr(B[i, j])) for i in range(n))
            worst = max(worst, rn / (an * xn + bn))
        assert oracle.backward_error(A, X, B) == pytest.approx(float(worst), rel=1e-12)


def test_backward_error_planted_mistakes(oracle):
    n = 120
    A = inputs.uniform(n, n, seed=inputs.seed_for(2, 11))
    B = inputs.normal(n, 4, seed=inputs.seed_for(2, 12))
    F, ipiv, info = oracle.getrf(A, c=24)
    X = oracle.getrs(F, ipiv, B)
    good = oracle.backward_error(A, X, B)
    assert good <= 10 * n * EPS
    # one entry of one solution column with its sign flipped
    bad = X.copy(order="F")
    bad[37, 2] = -bad[37, 2]
    assert oracle.backward_error(A, bad, B) > 1e-4
    # the columns of X permuted (solutions paired with the wrong b)
    assert oracle.backward_error(A, _F(X[:, ::-1]), B) > 1e-2
    # a solution of A^T x = b instead
    assert oracle.backward_error(A, _F(np.linalg.solve(A.T, B)), B) > 1e-2


# ----------------------------------------------------------------------------
# LU probe residual ||P A x - L (U x)||_inf / (n eps ||A||_inf ||x||_inf)
# ----------------------------------------------------------------------------

def _dyadic_lu3():
    L = np.array([[1, 0, 0], [0.5, 1, 0], [-0.25, 0.5, 1]])
    U = np.array([[4, 2, -2], [0, 2, 1], [0, 0, 1]], dtype=float)
    ipiv = np.array([3, 3, 3], dtype=np.int32)       # swap rows 1<->3, then 2<->3
    perm = _perm_from_ipiv(ipiv)                      # (P A)[i] = A[perm[i]]
    LUp = L @ U                                       # rows (4,2,-2), (2,3,0), (-1,1/2,2)
    A = np.empty_like(LUp)
    A[perm, :] = LUp
    F = np.tril(L, -1) + U
    return _F(A), _F(F), ipiv


def test_probe_lu_closed_form(oracle):
    A, F, ipiv = _dyadic_lu3()
    x = np.array([1.0, -1.0, 2.0])                    # ||x||_inf = 2 (||x||_1 = 4)
    # exact factors: every product and sum is exact, the residual is 0
    assert oracle.probe_lu(A, F, ipiv, x) == 0.0
    # U(1,3) moved by delta: L U' x - L U x = delta x_3 L e_1 = 2 delta (1, 1/2, -1/4),
    # ||.||_inf = 2 delta; ||A||_inf = 8 (row sums 8, 5, 7/2; ||A||_1 = 7), so
    # probe = 2 delta / (3 eps 8 2) = delta / (24 eps)
    Fp = F.copy(order="F")
    Fp[0, 2] += DELTA
    assert oracle.probe_lu(A, Fp, ipiv, x) == pytest.approx(DELTA / (24 * EPS), rel=1e-15)
    # L(3,1) moved by delta: the residual is delta (U x)_1 e_3 = delta (4 - 2 - 4) e_3,
    # ||.||_inf = 2 delta again (the unit diagonal of L is implicit)
    Fl = F.copy(order="F")
    Fl[2, 0] += DELTA
    assert oracle.probe_lu(A, Fl, ipiv, x) == pytest.approx(DELTA / (24 * EPS), rel=1e-15)


def test_probe_lu_exact_rational(oracle):
    r = np.random.default_rng(12)
    for n in (2, 4, 6):
        G = inputs.uniform(n, n, seed=int(r.integers(1 << 30)))
        F, ipiv, info = oracle.getrf(G, c=2)
        x = r.normal(size=n)
        perm = _perm_from_ipiv(ipiv)
        Fq = [[Fr(F[i, k]) for k in range(n)] for i in range(n)]
        # y = U x, rounded once to binary64 as the probe stores it
        y = [Fr(float(sum(Fq[i][k] * Fr(x[k]) for k in range(i, n)))) for i in range(n)]
        res = max(abs(sum(Fr(G[perm[i], k]) * Fr(x[k]) for k in range(n))
                      - sum(Fq[i][k] * y[k] for k in range(i)) - y[i]) for i in range(n))
        an = max(sum(abs(Fr(G[i, k])) for k in range(n)) for i in range(n))
        xn = max(abs(Fr(v)) for v in x)
        want = res / (n * Fr(EPS) * an * xn)
        assert oracle.probe_lu(G, F, ipiv, x) == pytest.approx(float(want), rel=1e-10, abs=1e-12)


def test_probe_lu_planted_mistakes(oracle):
    A, F, ipiv = _dyadic_lu3()
    x = np.array([1.0, -1.0, 2.0])
    # the probe without P (identity interchanges) on a pivoted factorization
    assert oracle.probe_lu(A, F, np.arange(1, 4, dtype=np.int32), x) > 1e12
    n = 200
    G = inputs.uniform(n, n, seed=inputs.seed_for(1, 21))
    F, ipiv, info = oracle.getrf(G, c=24)
    x = inputs.normal(n, 1, seed=5).ravel()
    assert oracle.probe_lu(G, F, ipiv, x) <= BOUND
    assert oracle.probe_lu(G, F, np.arange(1, n + 1, dtype=np.int32), x) > 1e6
    p2 = ipiv.copy()
    j = int(np.argmax(p2 != np.arange(1, n + 1)))
    p2[j] = j + 1                                      # one interchange dropped
    assert oracle.probe_lu(G, F, p2, x) > 1e6
    bad = F.copy(order="F")
    bad[150, 20] = -bad[150, 20]                       # a sign flip in L
    assert oracle.probe_lu(G, bad, ipiv, x) > 1e3
    bad = F.copy(order="F")
    bad[:8, 100:108] = bad[:8, 100:108].T              # a transposed block of U
    assert oracle.probe_lu(G, bad, ipiv, x) > 1e3


# ----------------------------------------------------------------------------
# TRTRI probe residual ||L (X x) - x||_inf / (n eps ||L||_inf ||X||_inf ||x||_inf)
# ----------------------------------------------------------------------------

def test_probe_trtri_closed_form(oracle):
    # L = [[2,0],[1,4]], X = L^-1 = [[1/2,0],[-1/8,1/4]] exactly.
    L = _F([[2, 0], [1, 4]])
    X = _F([[0.5, 0], [-0.125, 0.25]])
    x = np.array([1.0, 1.0])
    assert oracle.probe_trtri(L, X, x) == 0.0
    # X(2,1) moved by delta: L X' x - x = delta x_1 L e_2 = delta (0, 4), ||.|| = 4 delta;
    # ||L||_inf = 5 (||L||_1 = 4), ||X'||_inf = 1/2, so probe = 4 delta / (2 eps 5 1/2)
    Xp = X.copy(order="F")
    Xp[1, 0] += DELTA
    want = 4 * DELTA / (5 * EPS)
    assert oracle.probe_trtri(L, Xp, x) == pytest.approx(want, rel=1e-15)
    # the strictly upper triangles are not referenced
    Lg, Xg = L.copy(order="F"), Xp.copy(order="F")
    Lg[0, 1] = 1e30
    Xg[0, 1] = -1e30
    assert oracle.probe_trtri(Lg, Xg, x) == pytest.approx(want, rel=1e-15)


def test_probe_trtri_exact_rational(oracle):
    r = np.random.default_rng(13)
    for n in (1, 3, 6):
        L = np.tril(r.uniform(-1, 1, (n, n))) + 2 * np.eye(n)
        X = np.tril(np.linalg.inv(L))
        x = r.normal(size=n)
        Lq = [[Fr(L[i, k]) for k in range(n)] for i in range(n)]
        Xq = [[Fr(X[i, k]) for k in range(n)] for i in range(n)]
        y = [Fr(float(sum(Xq[i][k] * Fr(x[k]) for k in range(i + 1)))) for i in range(n)]
        res = max(abs(sum(Lq[i][k] * y[k] for k in range(i + 1)) - Fr(x[i])) for i in range(n))
        ln = max(sum(abs(Lq[i][k]) for k in range(i + 1)) for i in range(n))
        xnm = max(sum(abs(Xq[i][k]) for k in range(i + 1)) for i in range(n))
        want = res / (n * Fr(EPS) * ln * xnm * max(abs(Fr(v)) for v in x))
        assert oracle.probe_trtri(_F(L), _F(X), x) == pytest.approx(float(want), rel=1e-10, abs=1e-12)


def test_probe_trtri_planted_mistakes(oracle):
    n = 96
    L = inputs.integer_trtri(n, seed=inputs.seed_for(1, 31))
    X, info = oracle.trtri(L, c=24)
    x = inputs.normal(n, 1, seed=9).ravel()
    assert info == 0 and oracle.probe_trtri(L, X, x) <= BOUND
    n1 = oracle.split(n)
    bad = np.asfortranarray(np.tril(X))
    bad[n1:, :n1] = -bad[n1:, :n1]                     # the TRSM's sign dropped
    assert oracle.probe_trtri(L, bad, x) > 1e3
    bad = np.asfortranarray(np.tril(X))
    bad[n1:n1 + 8, :8] = bad[n1:n1 + 8, :8].T          # a transposed block
    assert oracle.probe_trtri(L, bad, x) > 1e3
    # the inverse taken with a unit diagonal (the diag flag mixed up)
    Lu = np.tril(L, -1) + np.eye(n)
    assert oracle.probe_trtri(L, _F(np.tril(np.linalg.inv(Lu))), x) > 1e3


# ----------------------------------------------------------------------------
# POTRI: full residual ||A X - I||_1 / (n eps ||A||_1 ||X||_1) and its probe
# ||A (X x) - x||_inf / (n eps ||A||_inf ||X||_inf ||x||_inf), A and X symmetric
# with their lower triangles stored
# ----------------------------------------------------------------------------

def _potri3():
    # L = [[1,0,0],[1,1,0],[0,1,1]]: A = L L^T = [[1,1,0],[1,2,1],[0,1,2]]
    # (||A||_1 = ||A||_inf = 4), A^-1 = L^-T L^-1 = [[3,-2,1],[-2,2,-1],[1,-1,1]].
    A = _F([[1, 1, 0], [1, 2, 1], [0, 1, 2]])
    X = _F([[3, -2, 1], [-2, 2, -1], [1, -1, 1]])
    return A, X


def test_potri_metrics_closed_form(oracle):
    A, X = _potri3()
    x = np.array([1.0, 1.0, 1.0])
    assert oracle.res_potri(A, np.tril(X)) == 0.0
    assert oracle.probe_potri(A, np.tril(X), x) == 0.0
    # X(3,1) = X(1,3) moved by delta (only the lower entry is stored):
    # A X' - I = delta A (e3 e1^T + e1 e3^T): column 1 = delta (0,1,2), column 3 =
    # delta (1,1,0); ||.||_1 = 3 delta (||.||_inf would be 2 delta);
    # ||X'||_1 = 6 + delta, so res = 3 delta / (3 eps 4 (6 + delta)).
    Xp = np.tril(X).copy(order="F")
    Xp[2, 0] += DELTA
    want_res = DELTA / (4 * EPS * (6 + DELTA))
    assert oracle.res_potri(A, Xp) == pytest.approx(want_res, rel=1e-15)
    # probe with x = (1,1,1): A X' x - x = delta A (1, 0, 1) = delta (1, 2, 2), ||.|| = 2 delta,
    # so probe = 2 delta / (3 eps 4 (6 + delta) 1)
    want_probe = DELTA / (6 * EPS * (6 + DELTA))
    assert oracle.probe_potri(A, Xp, x) == pytest.approx(want_probe, rel=1e-15)
    # the strictly upper triangles are not referenced (symmetry by mirroring)
    Ag, Xg = A.copy(order="F"), Xp.copy(order="F")
    Ag[0, 2] = Ag[0, 1] = 1e30
    Xg[0, 1] = Xg[1, 2] = -1e30
    assert oracle.res_potri(Ag, Xg) == pytest.approx(want_res, rel=1e-15)
    assert oracle.probe_potri(Ag, Xg, x) == pytest.approx(want_probe, rel=1e-15)


def test_potri_metrics_exact_rational(oracle):
    r = np.random.default_rng(14)
    for n in (1, 2, 5):
        A = inputs.spd_bbt(n, seed=int(r.integers(1 << 30)))
        X = np.linalg.inv(A)
        X = np.tril(X)
        x = r.normal(size=n)

        def sym(M, i, k):
            return Fr(M[i, k]) if i >= k else Fr(M[k, i])

        Aq = [[sym(A, i, k) for k in range(n)] for i in range(n)]
        Xq = [[sym(X, i, k) for k in range(n)] for i in range(n)]
        R = [[sum(Aq[i][k] * Xq[k][j] for k in range(n)) - (1 if i == j else 0)
              for j in range(n)] for i in range(n)]
        n1 = lambda M: max(sum(abs(M[i][j]) for i in range(n)) for j in range(n))  # noqa: E731
        want = n1(R) / (n * Fr(EPS) * n1(Aq) * n1(Xq))
        assert oracle.res_potri(A, X) == pytest.approx(float(want), rel=1e-10, abs=1e-12)
        y = [Fr(float(sum(Xq[i][k] * Fr(x[k]) for k in range(n)))) for i in range(n)]
        res = max(abs(sum(Aq[i][k] * y[k] for k in range(n)) - Fr(x[i])) for i in range(n))
        ninf = lambda M: max(sum(abs(v) for v in row) for row in M)  # noqa: E731
        want = res / (n * Fr(EPS) * ninf(Aq) * ninf(Xq) * max(abs(Fr(v)) for v in x))
        assert oracle.probe_potri(A, X, x) == pytest.approx(float(want), rel=1e-10, abs=1e-12)


def test_potri_metrics_planted_mistakes(oracle):
    n = 96
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 41))
    L, info = oracle.potrf(A, c=24)
    L = np.asfortranarray(np.tril(L))
    X, info = oracle.potri(L, c=24)
    X = np.asfortranarray(np.tril(X))
    x = inputs.normal(n, 1, seed=4).ravel()
    assert oracle.res_potri(A, X) <= BOUND and oracle.probe_potri(A, X, x) <= BOUND
    n1 = oracle.split(n)
    # one off-diagonal block of the stored triangle transposed
    bad = X.copy(order="F")
    bad[n1:n1 + 8, :8] = bad[n1:n1 + 8, :8].T
    assert oracle.res_potri(A, bad) > 1e3 and oracle.probe_potri(A, bad, x) > 1e3
    # the residual taken against L instead of A
    assert oracle.res_potri(L, X) > 1e3 and oracle.probe_potri(L, X, x) > 1e3
    # the inverse of L (TRTRI alone, LAUUM left out)
    Li, info = oracle.trtri(L, c=24)
    assert oracle.res_potri(A, Li) > 1e3 and oracle.probe_potri(A, Li, x) > 1e3
    # a sign flip in one entry
    bad = X.copy(order="F")
    bad[70, 11] = -bad[70, 11]
    assert oracle.res_potri(A, bad) > 1e3 and oracle.probe_potri(A, bad, x) > 10
