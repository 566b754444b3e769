"""rl_dsygst (Section 5, xsygst) against the oracle's definition: itype 1
(A := L^{-1} A L^{-T}) and 2/3 (A := L^T A L), with and without the n/2
buffer, on orders that cross the 64-order base case and the recursion's
splits; integer inputs bit for bit; the strictly upper triangle untouched.

Tolerance: max |X - X_oracle| <= 64 n eps max |X_oracle| (eps = 2^-53), for
well-conditioned L (the Cholesky factor of B B^T + n I).
"""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53
SENTINEL = -12345.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _with_upper_sentinel(A):
    A = np.array(A, dtype=np.float64, order="F")
    A[np.triu_indices(A.shape[0], 1)] = SENTINEL
    return A


def run_sygst(itype, A, L, use_work):
    r = G.lib()
    t = G.torch()
    n = A.shape[0]
    dA, dL = G.DevMat(_with_upper_sentinel(A), lda=n + 3), G.DevMat(L, lda=n + 1)
    lw = r.rl_dsygst_work_size(n) if use_work else 0
    w = t.empty(max(lw, 1), dtype=t.uint8, device="cuda") if use_work else None
    assert r.rl_dsygst(itype, "L", n, dA.ptr(), dA.lda, dL.ptr(), dL.lda, w, lw) == 0
    G.sync()
    assert dA.canaries_intact() and dL.canaries_intact()
    X = dA.get()
    assert np.all(X[np.triu_indices(n, 1)] == SENTINEL)
    return X


@pytest.mark.parametrize("use_work", [True, False])
@pytest.mark.parametrize("itype", [1, 2, 3])
@pytest.mark.parametrize("n", [1, 17, 64, 65, 130, 300, 701])
def test_sygst_vs_oracle(n, itype, use_work):
    Bm = inputs.spd_bbt(n, seed=inputs.seed_for(1, 800 + n))
    L = np.asfortranarray(np.tril(oracle.potrf(Bm, c=24)[0]))
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 810 + n))
    X = run_sygst(itype, A, L, use_work)
    ref = oracle.sygst(itype, A, L)
    scale = max(1e-300, np.max(np.abs(np.tril(ref))))
    assert np.max(np.abs(np.tril(X) - np.tril(ref))) <= 64 * n * EPS * scale


@pytest.mark.parametrize("n", [5, 64, 200])
def test_sygst_integer_exact(n):
    L = inputs.integer_chol(n, seed=inputs.seed_for(1, 820 + n), offdiag=1, diag=(1, 1))
    rng = np.random.default_rng(inputs.seed_for(1, 830 + n))
    M = rng.integers(-3, 4, size=(n, n)).astype(np.float64)
    M = np.asfortranarray(np.tril(M) + np.tril(M, -1).T)
    Li, Mi = L.astype(np.int64), M.astype(np.int64)
    A = np.asfortranarray((Li @ Mi @ Li.T).astype(np.float64))
    X = run_sygst(1, A, L, True)
    assert np.array_equal(np.tril(X), np.tril(M))
    X = run_sygst(2, M, L, True)
    assert np.array_equal(np.tril(X), np.tril((Li.T @ Mi @ Li).astype(np.float64)))


def test_sygst_arguments():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(300 * 300, dtype=t.float64, device="cuda")
    assert r.rl_dsygst(4, "L", 3, buf, 3, buf, 3, None, 0) == -1
    assert r.rl_dsygst(1, "X", 3, buf, 3, buf, 3, None, 0) == -2
    assert r.rl_dsygst(1, "L", 3, buf, 2, buf, 3, None, 0) == -5
    assert r.rl_dsygst(1, "L", 3, buf, 3, buf, 2, None, 0) == -7
    assert r.rl_dsygst(1, "U", 3, buf, 3, buf, 2, None, 0) == -7
    lw = r.rl_dsygst_work_size(300)
    assert lw > 0 and r.rl_dsygst_work_size(64) == 0
    w = t.zeros(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dsygst(1, "L", 300, buf, 300, buf, 300, w, lw - 8) == r.RL_ERR_WORKSPACE
