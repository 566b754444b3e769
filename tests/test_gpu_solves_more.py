"""The remaining solve forms: rl_dgetrs / rl_sgetrs with trans = 'T'
(U^T Y = B, L^T Z = Y, X = P^T Z with the interchanges last first) against
the oracle's backward error, the reverse interchanges alone on an identity
factor at an order beyond the shared-memory staging, and the complex solves
rl_zgetrs / rl_zpotrs ('L' and 'U') against an extended-precision residual."""
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


@pytest.mark.parametrize("n,nrhs", [(1, 1), (70, 3), (700, 5), (2100, 17)])
def test_dgetrs_transposed(n, nrhs):
    r = G.lib()
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 8000 + n))
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(1, 8100 + n))
    F, ipiv, info = G.getrf(A)
    assert info == 0
    dF, dB = G.DevMat(F), G.DevMat(B, lda=n + 2)
    dp = G.torch().from_numpy(ipiv.astype(np.int32)).cuda()
    for trans in ("T", "C"):
        dB = G.DevMat(B, lda=n + 2)
        assert r.rl_dgetrs(trans, n, nrhs, dF.ptr(), dF.lda, dp.data_ptr(), dB.ptr(), dB.lda) == 0
        G.sync()
        assert dB.canaries_intact()
        assert np.array_equal(dF.get(), F)                  # the factors are not touched
        assert oracle.backward_error(np.asfortranarray(A.T), dB.get(), B) <= 10 * n * EPS


def test_sgetrs_transposed():
    r = G.lib()
    t = G.torch()
    n, nrhs = 900, 4
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 8200)).astype(np.float32).astype(np.float64)
    B = inputs.normal(n, nrhs, seed=inputs.seed_for(1, 8201)).astype(np.float32).astype(np.float64)
    dA = t.from_numpy(np.asfortranarray(A, dtype=np.float32).ravel(order="F").copy()).cuda()
    ipiv, info = G.int_buf(n, -5), G.int_buf(1, -77)
    lw = r.rl_dgetrf_work_size(n, n)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_sgetrf(n, n, dA.data_ptr(), n, ipiv.data_ptr(), info.data_ptr(), w.data_ptr(), lw) == 0
    dB = t.from_numpy(np.asfortranarray(B, dtype=np.float32).ravel(order="F").copy()).cuda()
    assert r.rl_sgetrs("T", n, nrhs, dA.data_ptr(), n, ipiv.data_ptr(), dB.data_ptr(), n) == 0
    G.sync()
    X = dB.cpu().numpy().reshape(nrhs, n).T.astype(np.float64)
    assert oracle.backward_error(np.asfortranarray(A.T), np.asfortranarray(X), B) <= 10 * n * 2.0 ** -24


def test_reverse_interchanges_beyond_staging():
    """A^T X = B with the identity as L and U: X = P^T B exactly, at an order
    whose columns do not fit in shared memory (the global-memory walk)."""
    r = G.lib()
    t = G.torch()
    n = 30000
    rng = np.random.default_rng(8300)
    ipiv = (np.arange(n) + rng.integers(0, 50, size=n)).clip(max=n - 1).astype(np.int32) + 1
    b = rng.standard_normal((n, 2))
    dI = t.eye(n, dtype=t.float64, device="cuda")
    dp = t.from_numpy(ipiv).cuda()
    dB = t.from_numpy(np.asfortranarray(b).ravel(order="F").copy()).cuda()
    assert r.rl_dgetrs("T", n, 2, dI.data_ptr(), n, dp.data_ptr(), dB.data_ptr(), n) == 0
    G.sync()
    x = b.copy()
    for i in range(n - 1, -1, -1):
        p = ipiv[i] - 1
        x[[i, p]] = x[[p, i]]
    assert np.array_equal(dB.cpu().numpy().reshape(2, n).T, x)


def zdev(A):
    return G.torch().from_numpy(np.asfortranarray(A, dtype=np.complex128).ravel(order="F").copy()).cuda()


def zhost(d, m, n):
    return np.asfortranarray(d.cpu().numpy().reshape(n, m).T)


def zres(A, X, B):
    """||A X - B||_1 / (||A||_1 ||X||_1 n eps), in extended precision."""
    Al, Xl, Bl = (np.asarray(v, dtype=np.clongdouble) for v in (A, X, B))
    R = (Al @ Xl - Bl).astype(np.complex128)
    n = A.shape[0]
    return np.abs(R).sum(0).max() / (np.abs(A).sum(0).max() * np.abs(X).sum(0).max() * n * EPS)


@pytest.mark.parametrize("n", [1, 65, 500])
def test_zgetrs_zpotrs(n):
    r = G.lib()
    t = G.torch()
    nrhs = 3
    A = inputs.complex_uniform(n, n, inputs.seed_for(1, 8400 + n))
    B = inputs.complex_uniform(n, nrhs, inputs.seed_for(1, 8401 + n))
    dA = zdev(A)
    ipiv, info = G.int_buf(n, -5), G.int_buf(1, -77)
    lw = r.rl_dgetrf_work_size(n, n)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_zgetrf(n, n, dA.data_ptr(), n, ipiv.data_ptr(), info.data_ptr(), w.data_ptr(), lw) == 0
    dB = zdev(B)
    assert r.rl_zgetrs("N", n, nrhs, dA.data_ptr(), n, ipiv.data_ptr(), dB.data_ptr(), n) == 0
    G.sync()
    assert int(info[0]) == 0
    assert zres(A, zhost(dB, n, nrhs), B) <= 10.0
    assert r.rl_zgetrs("T", n, nrhs, dA.data_ptr(), n, ipiv.data_ptr(), dB.data_ptr(), n) == r.RL_ERR_UNSUPPORTED
    H = inputs.herm_spd(n, inputs.seed_for(1, 8402 + n))
    for uplo in ("L", "U"):
        dH = zdev(H)
        assert r.rl_zpotrf(uplo, n, dH.data_ptr(), n, info.data_ptr()) == 0
        dB = zdev(B)
        assert r.rl_zpotrs(uplo, n, nrhs, dH.data_ptr(), n, dB.data_ptr(), n) == 0
        G.sync()
        assert int(info[0]) == 0
        assert zres(H, zhost(dB, n, nrhs), B) <= 10.0
