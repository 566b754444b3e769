"""Single-precision peers (rl_spotrf / rl_sgetrf / rl_sgetrs / rl_spotrs)
against the oracle: residuals measured in units of the FP32 rounding unit
2^-24 (<= 10), ipiv equal to the oracle's on the FP32-rounded input up to
the first near-tie, exact inputs bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1602_06763_gb300 import inputs

from . import gpu_util as G

pytestmark = pytest.mark.gpu
SCALE = 2.0 ** -53 / 2.0 ** -24     # oracle metrics use 2^-53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def to_dev32(A):
    t = G.torch()
    return t.from_numpy(np.asfortranarray(A, dtype=np.float32).ravel(order="F").copy()).cuda()


def from_dev32(d, m, n):
    return np.asfortranarray(d.cpu().numpy().reshape(n, m).T.astype(np.float64))


@pytest.mark.parametrize("n", [1, 33, 200, 700])
def test_spotrf_sgetrf_vs_oracle(n):
    r = G.lib()
    t = G.torch()
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 3000 + n)).astype(np.float32).astype(np.float64)
    dA = to_dev32(A)
    info = G.int_buf(1, -7)
    assert r.rl_spotrf("L", n, dA.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    assert int(info[0]) == 0
    L = from_dev32(dA, n, n)
    assert oracle.res_chol(A, L) * SCALE <= 10.0
    Gm = inputs.uniform(n, n, seed=inputs.seed_for(1, 3100 + n)).astype(np.float32).astype(np.float64)
    dG = to_dev32(Gm)
    ipiv = G.int_buf(n, -5)
    lw = r.rl_dgetrf_work_size(n, n)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_sgetrf(n, n, dG.data_ptr(), n, ipiv.data_ptr(), info.data_ptr(), work.data_ptr(), lw) == 0
    G.sync()
    F = from_dev32(dG, n, n)
    piv = ipiv.cpu().numpy()[:n]
    assert int(info[0]) == 0
    assert oracle.res_lu(Gm, F, piv) * SCALE <= 10.0
    # solves: recursive TRSM (no workspace) and the one-launch flow solve
    B = inputs.normal(n, 3, seed=inputs.seed_for(1, 3200 + n)).astype(np.float32).astype(np.float64)
    for use_work in (False, True):
        lw = r.rl_trs_work_size(n, 3) if use_work else 0
        w = t.zeros(lw, dtype=t.uint8, device="cuda") if use_work else None
        dB = to_dev32(B)
        assert r.rl_sgetrs("N", n, 3, dG.data_ptr(), n, ipiv.data_ptr(), dB.data_ptr(), n, w, lw) == 0
        G.sync()
        X = from_dev32(dB, n, 3)
        assert oracle.backward_error(Gm, X, B) <= 10 * n * 2.0 ** -24
        dB = to_dev32(B)
        assert r.rl_spotrs("L", n, 3, dA.data_ptr(), n, dB.data_ptr(), n, w, lw) == 0
        G.sync()
        assert oracle.backward_error(A, from_dev32(dB, n, 3), B) <= 10 * n * 2.0 ** -24


def test_single_exact_inputs():
    r = G.lib()
    t = G.torch()
    n = 150
    L = inputs.integer_chol(n, seed=inputs.seed_for(1, 3300), offdiag=1, diag=(1, 2))
    A = inputs.product_lower(L)
    dA = to_dev32(A)
    info = G.int_buf(1, -7)
    assert r.rl_spotrf("L", n, dA.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    assert np.array_equal(np.tril(from_dev32(dA, n, n)), L)
    A, Lx, U, perm = inputs.dyadic_lu(n, seed=inputs.seed_for(1, 3400))
    dA = to_dev32(A)
    ipiv = G.int_buf(n, -5)
    lw = r.rl_dgetrf_work_size(n, n)
    work = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_sgetrf(n, n, dA.data_ptr(), n, ipiv.data_ptr(), info.data_ptr(), work.data_ptr(), lw) == 0
    G.sync()
    F = from_dev32(dA, n, n)
    assert np.array_equal(ipiv.cpu().numpy()[:n], inputs.expected_ipiv(perm))
    assert np.array_equal(np.tril(F, -1) + np.eye(n), Lx) and np.array_equal(np.triu(F), U)


@pytest.mark.parametrize("n", [1, 40, 130, 300])
def test_strtri_slauum_spotri_vs_oracle(n):
    r = G.lib()
    A = inputs.spd_bbt(n, seed=inputs.seed_for(1, 3500 + n)).astype(np.float32).astype(np.float64)
    L64, info = oracle.potrf(A, c=24)
    L = np.asfortranarray(np.tril(L64).astype(np.float32).astype(np.float64))
    info = G.int_buf(1, -7)
    # trtri: ||L X - I|| / (n u ||L|| ||X||) in FP32 units
    dX = to_dev32(L)
    assert r.rl_strtri("L", "N", n, dX.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    assert int(info[0]) == 0
    X = np.tril(from_dev32(dX, n, n))
    assert oracle.res_trtri(L, X) * SCALE <= 10.0
    # lauum against the oracle's product
    dX = to_dev32(L)
    assert r.rl_slauum("L", n, dX.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    got = np.tril(from_dev32(dX, n, n))
    ref = np.tril(L.T @ L)
    assert np.max(np.abs(got - ref)) <= 4 * n * 2.0 ** -24 * np.max(np.abs(ref))
    # potri: the inverse of A = L L^T
    dX = to_dev32(L)
    assert r.rl_spotri("L", n, dX.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    Xp = np.tril(from_dev32(dX, n, n))
    LLt = L @ L.T
    assert oracle.res_potri(LLt, Xp) * SCALE <= 10.0


def test_strtri_exact_and_zero_diagonal():
    r = G.lib()
    n = 120
    L = inputs.integer_trtri(n, seed=inputs.seed_for(1, 3600))
    dX = to_dev32(L)
    info = G.int_buf(1, -7)
    assert r.rl_strtri("L", "N", n, dX.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    X = np.tril(from_dev32(dX, n, n))
    ref, _ = oracle.trtri(L, c=24)
    assert np.array_equal(X, np.tril(ref))
    Z = L.copy(order="F")
    Z[77, 77] = 0.0
    dZ = to_dev32(Z)
    assert r.rl_strtri("L", "N", n, dZ.data_ptr(), n, info.data_ptr()) == 0
    G.sync()
    assert int(info[0]) == 78
    assert np.array_equal(from_dev32(dZ, n, n), Z)


@pytest.mark.parametrize("n", [1, 130, 700])
def test_sgetri_ssygst_vs_oracle(n):
    r = G.lib()
    t = G.torch()
    A = inputs.uniform(n, n, seed=inputs.seed_for(1, 3700 + n)).astype(np.float32).astype(np.float64)
    F, ipiv, info = oracle.getrf(A, c=24)
    F32 = F.astype(np.float32).astype(np.float64)
    dF = to_dev32(F32)
    dp = t.from_numpy(np.ascontiguousarray(ipiv, dtype=np.int32)).cuda()
    info = G.int_buf(1, -7)
    lw = r.rl_sgetri_work_size(n)
    w = t.empty(lw, dtype=t.uint8, device="cuda")
    assert r.rl_sgetri(n, dF, n, dp, info, w, lw) == 0
    G.sync()
    assert int(info[0]) == 0
    X = from_dev32(dF, n, n)
    ref = oracle.getri(F32, ipiv)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(X - ref)) <= 64 * n * 2.0 ** -24 * kappa * np.max(np.abs(ref))
    # sygst itype 1 and 2, with the buffer
    S = inputs.spd_bbt(n, seed=inputs.seed_for(1, 3800 + n)).astype(np.float32).astype(np.float64)
    Bm = inputs.spd_bbt(n, seed=inputs.seed_for(1, 3900 + n))
    L = np.tril(oracle.potrf(Bm, c=24)[0]).astype(np.float32).astype(np.float64)
    for itype in (1, 2):
        dS, dL = to_dev32(S), to_dev32(L)
        lw = max(r.rl_ssygst_work_size(n), 4)
        w = t.empty(lw, dtype=t.uint8, device="cuda")
        assert r.rl_ssygst(itype, "L", n, dS, n, dL, n, w, lw) == 0
        G.sync()
        got = np.tril(from_dev32(dS, n, n))
        ref = np.tril(oracle.sygst(itype, S, L))
        assert np.max(np.abs(got - ref)) <= 64 * n * 2.0 ** -24 * np.max(np.abs(ref))
