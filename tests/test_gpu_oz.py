"""FP64 updates emulated on the BF16 tensor cores (rl_dgemm_oz, rl_dpotrf_oz,
rl_dgetrf_oz): integer products exact bit for bit, random products within the
scheme's error bound (S + 1) k 2^(-8S-2) 2^(eA_i + eB_j) against an
extended-precision reference, every transpose combination and ragged tile edges, Inf/NaN
confined to their row or column, and the factorizations held to the same
residual bound, exact cases and pivots as the native FP64 path."""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def oz_gemm(S, ta, tb, A, B, C0, alpha=1.0, beta=0.0):
    r = G.lib()
    t = G.torch()
    m, n = C0.shape
    k = A.shape[0] if ta else A.shape[1]
    dA, dB, dC = G.DevMat(A), G.DevMat(B), G.DevMat(C0)
    lw = r.rl_oz_work_size(m, n, k, S)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_dgemm_oz(S, "T" if ta else "N", "T" if tb else "N", m, n, k, alpha, dA.ptr(), dA.lda, dB.ptr(),
                       dB.lda, beta, dC.ptr(), dC.lda, w, lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert dC.canaries_intact()
    return dC.get()


def op(X, tr):
    return X.T if tr else X


@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("m,n,k", [(130, 70, 300), (256, 192, 1000), (1, 1, 1), (300, 65, 129)])
def test_integer_products_exact(ta, tb, m, n, k):
    rng = np.random.default_rng(7000 + m + n + k)
    A = rng.integers(-1000, 1001, size=(k, m) if ta else (m, k)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(n, k) if tb else (k, n)).astype(np.float64)
    C0 = rng.integers(-5, 6, size=(m, n)).astype(np.float64)
    exact = op(A, ta).astype(np.int64) @ op(B, tb).astype(np.int64)
    C = oz_gemm(7, ta, tb, A, B, C0, alpha=-1.0, beta=1.0)
    assert np.array_equal(C, C0 - exact.astype(np.float64))
    C = oz_gemm(7, ta, tb, A, B, C0)
    assert np.array_equal(C, exact.astype(np.float64))


def exp_of(v):
    v = np.asarray(v, dtype=np.float64)
    e = np.frexp(v)[1] + 1
    return np.where(v == 0, 0, e)


@pytest.mark.parametrize("S", [6, 7, 8])
@pytest.mark.parametrize("ta,tb", [(False, True), (True, False)])
def test_random_products_within_the_bound(S, ta, tb):
    rng = np.random.default_rng(7100 + S)
    m, n, k = 200, 100, 300
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-30, 30, size=(m, 1)))
    B = rng.standard_normal((k, n)) * np.exp2(rng.integers(-30, 30, size=(1, n)))
    A[5, :] = 0.0
    A[7, 3] = 1e-300
    exact = A.astype(np.longdouble) @ B.astype(np.longdouble)
    C = oz_gemm(S, ta, tb, np.asfortranarray(A.T) if ta else A, np.asfortranarray(B.T) if tb else B,
                np.zeros((m, n)))
    eA = exp_of(np.max(np.abs(A), axis=1))[:, None]
    eB = exp_of(np.max(np.abs(B), axis=0))[None, :]
    # truncated digits (2^(-8S-1) each side) and the pairs left out: (S + 1) 2^(-8S-2) per term
    bound = k * (S + 1) * np.exp2(-8.0 * S - 2 + eA + eB) + 2.0 ** -52 * np.abs(exact.astype(np.float64))
    err = np.abs((C.astype(np.longdouble) - exact).astype(np.float64))
    assert np.all(err <= bound)
    assert np.all(C[5, :] == 0.0)
    # as accurate as an FP64 GEMM: the largest error within a small multiple of FP64's
    if S >= 7:
        err64 = np.abs(((A @ B).astype(np.longdouble) - exact).astype(np.float64))
        scale = np.exp2(eA + eB)
        assert np.max(err / scale) <= 4 * max(np.max(err64 / scale), 2.0 ** -60)


def test_nonfinite_confined_to_its_row_and_column():
    rng = np.random.default_rng(7200)
    m, n, k = 150, 90, 260
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    A[11, 40] = np.inf
    B[100, 33] = np.nan
    C = oz_gemm(7, False, False, A, B, np.zeros((m, n)))
    assert np.all(np.isnan(C[11, :])) and np.all(np.isnan(C[:, 33]))
    mask = np.ones((m, n), dtype=bool)
    mask[11, :] = False
    mask[:, 33] = False
    ref = A.copy()
    ref[11, 40] = 0.0
    Bf = B.copy()
    Bf[100, 33] = 0.0
    assert np.max(np.abs(C[mask] - (ref @ Bf)[mask])) <= 1e-12 * np.max(np.abs(ref @ Bf))


def test_arguments_and_workspace():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(64, dtype=t.float64, device="cuda")
    assert r.rl_dgemm_oz(5, "N", "N", 4, 4, 4, 1.0, buf, 4, buf, 4, 0.0, buf, 4, None, 0) == -1
    assert r.rl_dgemm_oz(7, "X", "N", 4, 4, 4, 1.0, buf, 4, buf, 4, 0.0, buf, 4, None, 0) == -2
    assert r.rl_dgemm_oz(7, "N", "N", 4, 4, 4, 1.0, buf, 3, buf, 4, 0.0, buf, 4, None, 0) == -9
    assert r.rl_dgemm_oz(7, "N", "N", 4, 4, 4, 1.0, buf, 4, buf, 4, 0.0, buf, 4, None, 0) == r.RL_ERR_WORKSPACE
    assert r.rl_oz_work_size(4, 4, 4, 9) == 0
    assert r.rl_dpotrf_oz(7, "L", 300, buf, 300, buf, None, 0) == r.RL_ERR_WORKSPACE


@pytest.fixture
def oz_min_64():
    r = G.lib()
    old = r.rl_get_param(r.RL_PARAM_OZ_MIN)
    assert r.rl_set_param(r.RL_PARAM_OZ_MIN, 64) == 0
    yield
    assert r.rl_set_param(r.RL_PARAM_OZ_MIN, old) == 0


def potrf_oz(A, S=7):
    r = G.lib()
    t = G.torch()
    n = A.shape[0]
    d = G.DevMat(A)
    info = G.int_buf(1, -77)
    lw = r.rl_dpotrf_oz_work_size(n, S)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_dpotrf_oz(S, "L", n, d.ptr(), n, info.data_ptr(), w, lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), int(info[0])


def getrf_oz(A, S=7):
    r = G.lib()
    t = G.torch()
    m, n = A.shape
    d = G.DevMat(A)
    info = G.int_buf(1, -77)
    ipiv = G.int_buf(min(m, n), -5)
    lw = r.rl_dgetrf_oz_work_size(m, n, S)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    st = r.rl_dgetrf_oz(S, m, n, d.ptr(), m, ipiv.data_ptr(), info.data_ptr(), w, lw)
    G.sync()
    assert st == 0, r.rl_status_string(st)
    assert d.canaries_intact()
    return d.get(), ipiv.cpu().numpy()[:min(m, n)].copy(), int(info[0])


@pytest.mark.parametrize("n", [300, 1100])
def test_potrf_oz(n, oz_min_64):
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 7300 + n))
    L, info = potrf_oz(A)
    assert info == 0
    assert oracle.res_chol(A, np.tril(L)) <= 10.0
    ref, _ = oracle.potrf(A)
    assert np.max(np.abs(np.tril(L) - np.tril(ref))) <= 64 * n * 2.0 ** -53 * np.max(np.abs(ref))


def test_potrf_oz_integer_exact(oz_min_64):
    n = 600
    Lx = inputs.integer_chol(n, seed=inputs.seed_for(1, 7400))
    L, info = potrf_oz(inputs.product_lower(Lx))
    assert info == 0
    assert np.array_equal(np.tril(L), Lx)


@pytest.mark.parametrize("m,n", [(1100, 1100), (900, 400)])
def test_getrf_oz(m, n, oz_min_64):
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 7500 + m + n))
    F, ipiv, info = getrf_oz(A)
    assert info == 0
    assert oracle.res_lu(A, F, ipiv) <= 10.0
    ref, opiv, _ = oracle.getrf(A)
    t = min(G.first_near_tie(F), G.first_near_tie(ref))
    assert np.array_equal(ipiv[:t], opiv[:t])


def test_getrf_oz_dyadic_exact(oz_min_64):
    n = 600
    A, L, U, perm = inputs.dyadic_lu(n, seed=inputs.seed_for(1, 7600))
    F, ipiv, info = getrf_oz(A)
    assert info == 0
    assert np.array_equal(ipiv, inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1) + np.eye(n), L) and np.array_equal(np.triu(F), U)


@pytest.mark.parametrize("S,bound", [(6, 200.0), (8, 10.0)])
def test_potrf_oz_other_slices(S, bound, oz_min_64):
    """6 planes carry 48 bits (a bound 56 times looser than 7 planes'); 8
    planes carry 64."""
    n = 700
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 7700 + S))
    L, info = potrf_oz(A, S=S)
    assert info == 0
    assert oracle.res_chol(A, np.tril(L)) <= bound


def test_potrf_oz_upper(oz_min_64):
    r = G.lib()
    t = G.torch()
    n = 600
    Lx = inputs.integer_chol(n, seed=inputs.seed_for(1, 7800))
    A = inputs.product_lower(Lx)
    A0 = np.asfortranarray(np.triu(A) + np.tril(np.full((n, n), 7.5), -1))
    d = G.DevMat(A0)
    info = G.int_buf(1, -77)
    lw = r.rl_dpotrf_oz_work_size(n, 7)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dpotrf_oz(7, "U", n, d.ptr(), n, info.data_ptr(), w, lw) == 0
    G.sync()
    assert int(info[0]) == 0
    X = d.get()
    assert np.array_equal(np.triu(X), np.triu(Lx.T))
    assert np.array_equal(np.tril(X, -1), np.tril(A0, -1))


def test_getrf_oz_wide(oz_min_64):
    m, n = 400, 1000
    A = inputs.uniform(m, n, seed=inputs.seed_for(1, 7900))
    F, ipiv, info = getrf_oz(A)
    assert info == 0
    assert oracle.res_lu(A, F, ipiv) <= 10.0


@pytest.mark.parametrize("S", [6, 7, 8])
@pytest.mark.parametrize("ta,tb,m,n,k", [(False, False, 150, 70, 300), (True, False, 129, 64, 200),
                                         (False, True, 40, 130, 513), (True, True, 200, 33, 64)])
def test_bit_identical_to_the_oracle(S, ta, tb, m, n, k):
    """Every intermediate sum of the scheme is exact and the result is rounded
    once, so the GPU returns the oracle's binary64 values bit for bit (k <=
    600 keeps the integer accumulators below 2^53 before that rounding)."""
    from oracle import ozaki
    rng = np.random.default_rng(7400 + S + m + k)
    opA = rng.standard_normal((m, k)) * np.exp2(rng.integers(-25, 25, size=(m, 1)))
    opB = rng.standard_normal((k, n)) * np.exp2(rng.integers(-25, 25, size=(1, n)))
    opA[m // 3, :] = 0.0
    A = np.asfortranarray(opA.T) if ta else opA
    B = np.asfortranarray(opB.T) if tb else opB
    ref = ozaki.gemm(A, B, S, ta, tb)
    C = oz_gemm(S, ta, tb, A, B, np.zeros((m, n)))
    assert np.array_equal(C, ref)
