"""rl_dgetri against the oracle's definition (A X = I on the same LU
factors): orders crossing the 64-order blocks, a unimodular integer case bit
for bit, a zero pivot (info, A unchanged), and the argument checks.

Tolerance: max |X - X_oracle| <= 64 n eps kappa(A) max |X_oracle|, the
forward-error bound of two backward-stable inverses from the same factors.
"""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def run_getri(F, ipiv, lda_pad=2):
    r = G.lib()
    t = G.torch()
    n = F.shape[0]
    dA = G.DevMat(F, lda=n + lda_pad)
    dp = t.from_numpy(np.ascontiguousarray(ipiv, dtype=np.int32)).cuda()
    info = G.int_buf(1, -9)
    lw = r.rl_dgetri_work_size(n)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_dgetri(n, dA.ptr(), dA.lda, dp, info, w, lw) == 0
    G.sync()
    assert dA.canaries_intact()
    return dA.get(), int(info[0])


@pytest.mark.parametrize("n", [1, 2, 17, 64, 65, 130, 300, 701])
def test_getri_vs_oracle(n):
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 900 + n))
    F, ipiv, info = oracle.getrf(A, c=24)
    assert info == 0
    X, info = run_getri(F, ipiv)
    assert info == 0
    ref = oracle.getri(F, ipiv)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(X - ref)) <= 64 * n * EPS * kappa * np.max(np.abs(ref))
    # and it is an inverse: ||A X - I||_1 / (||A||_1 ||X||_1) small
    R = A @ X - np.eye(n)
    assert np.linalg.norm(R, 1) <= 8 * n * EPS * np.linalg.norm(A, 1) * np.linalg.norm(X, 1)


def _unimodular_factors(n, seed):
    r = np.random.default_rng(seed)
    L = np.tril(r.integers(-1, 2, size=(n, n)).astype(np.float64), -1) + np.eye(n)
    U = np.triu(r.integers(-1, 2, size=(n, n)).astype(np.float64), 1)
    U[np.diag_indices(n)] = r.choice([-1.0, 1.0], size=n)
    ipiv = np.array([r.integers(j + 1, n + 1) for j in range(n)], dtype=np.int32)
    return np.asfortranarray(np.tril(L, -1) + U), ipiv


@pytest.mark.parametrize("n", [5, 40, 70])
def test_getri_integer_exact(n):
    F, ipiv = _unimodular_factors(n, inputs.seed_for(1, 950 + n))
    ref = oracle.getri(F, ipiv)
    # the integer inverse grows quickly with n; the case is exact only while
    # every intermediate stays below 2^53
    assert np.max(np.abs(ref)) < 2.0 ** 40
    X, info = run_getri(F, ipiv)
    assert info == 0
    assert np.array_equal(X, ref)


def test_getri_zero_pivot_leaves_a():
    n = 100
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 990))
    F, ipiv, _ = oracle.getrf(A, c=24)
    F[37, 37] = 0.0
    X, info = run_getri(F, ipiv)
    assert info == 38
    assert np.array_equal(X, F)


def test_getri_arguments():
    r = G.lib()
    t = G.torch()
    buf = t.zeros(64, dtype=t.float64, device="cuda")
    piv = t.ones(8, dtype=t.int32, device="cuda")
    info = G.int_buf(1)
    assert r.rl_dgetri(-1, buf, 1, piv, info, None, 0) == -1
    assert r.rl_dgetri(4, buf, 3, piv, info, None, 0) == -3
    assert r.rl_dgetri(4, buf, 4, piv, None, None, 0) == r.RL_ERR_NULL_POINTER
    assert r.rl_dgetri(4, buf, 4, piv, info, None, 0) == r.RL_ERR_WORKSPACE
    assert r.rl_dgetri(50000, buf, 50000, piv, info, None, 0) == r.RL_ERR_UNSUPPORTED
